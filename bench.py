#!/usr/bin/env python
"""Benchmark: voxel-increments/s of the staggered RVE load increment
(crystal plasticity + FFT Newton-Krylov equilibrium + FFT phase field) on
the 64^3 / 50-grain periodic Voronoi polycrystal (R = -1 uniaxial-strain
cycle at 0.6 %, 40 increments per cycle), mixed FP32/FP64 path vs the plain
FP64 path.

A step is one load increment (GND, constitutive updates, residuals, GMRES,
F update, phase field, clamp, commit).  N GPUs run N independent replicas
(weak scaling, no data-path collective).  Prints one JSON line on rank 0.

--impl reference times the FP64 CPU oracle on the host cores instead (each
step one increment of the same workload).
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2304_01125_gb300 import inputs as I  # noqa: E402

METRIC = "voxel-increments/s (CP+FFT equilibrium+phase-field), mixed vs FP64 on GPU at <=1e-4"
CONFIG_NAME = "poly64"
L2_NOTE = ("working set > L2 (the handle's device memory, {gb:.1f} GB mixed per RVE) and a "
           "256 MB L2 flush before every step")
# kernel families bound by HBM traffic (the constitutive update is ALU-bound;
# cuFFT is a library; "other" carries no byte count)
HBM_FAMILIES = ("tangent_apply", "precond_grad", "contract", "gmres_dot", "gs_update",
                "gmres_xupdate", "kbar", "residual", "f_update", "phase_field", "gnd",
                "reductions")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_traffic.json")


def args_():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=80)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", default=CONFIG_NAME)
    p.add_argument("--tol", default="paper", choices=["paper", "parity32", "parity64"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-damage-window", action="store_true")
    p.add_argument("--no-batch-window", action="store_true",
                   help="default config: skip the short batched-workload figure")
    p.add_argument("--batch-threads", type=int, default=None,
                   help="--config batch32: host threads driving the handles")
    p.add_argument("--batch-split", action="store_true",
                   help="--config batch32 on N GPUs: split the one batch's RVEs over the "
                        "ranks by estimated cost (strong scaling) instead of giving every "
                        "rank its own batch of distinct RVEs (weak scaling)")
    p.add_argument("--no-classes", action="store_true",
                   help="--config batch32: no lockstep classes (every handle on its own)")
    p.add_argument("--classes-all", action="store_true",
                   help="--config batch32: lockstep classes at every grid size (default: up "
                        "to 2^16 voxels)")
    p.add_argument("--no-autotune", action="store_true",
                   help="--config batch32: default kernel variants (no per-size autotuning)")
    p.add_argument("--verbose", action="store_true")
    p.add_argument("--ref-budget-s", type=float, default=150.0,
                   help="--impl reference: stop timing the oracle after this many seconds")
    return p.parse_args()


# the translation units that hold device code, and every header: ncu
# counters taken on other kernel code are not reported (the host-only
# drivers rve.cu and batch.cu launch the same kernels)
KERNEL_SOURCES = ("kernels_cp.cu", "kernels_spec.cu", "kernels_fft.cu", "noalloc.cu")
HOST_HEADERS = ("rve_impl.cuh",)  # the drivers' shared host code


def source_sha1():
    """Hash of the kernel sources (device-code translation units and all
    headers)."""
    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_2304_01125_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f in KERNEL_SOURCES or (f.endswith((".cuh", ".h")) and f not in HOST_HEADERS):
            h.update(f.encode())
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()


def ncu_traffic(family, workload):
    """DRAM bytes per launch of the family's kernel from the committed ncu
    summary, or None when absent, taken on other kernel sources or on
    another workload (traffic per launch depends on the grid, and on what
    stays in L2)."""
    try:
        d = json.load(open(TRAFFIC_FILE))
    except (OSError, ValueError):
        return None
    e = d.get(workload, {}).get(family)
    if not e or e.get("source_sha1") != source_sha1():
        return None
    return e.get("dram_bytes_per_launch")


class Driver:
    """Runs a workload's increments on one handle (GPU or oracle).  Under a
    stress mask (uniaxial stress) the stress-controlled components of each
    increment start from the previous increment's solved macroscopic F."""

    def __init__(self, cfg):
        self.cfg, self.F = cfg, None

    def __call__(self, r, k):
        args, kw = I.increment_args(self.cfg, k, self.F)
        s, st = r.run_increment(*args, **kw)
        if kw and s == 0:
            self.F = np.array(st["Fbar"])
        return s, st


def workload_options(a, cfg):
    """Solver options of a workload: the --tol preset with the config's own
    overrides; mixed-control workloads (large plastic strains at the R = 0
    peaks) with cut-back on."""
    over = dict(cfg.get("options", {}))
    if cfg["stress_mask"] is not None:
        over.setdefault("max_cutbacks", 4)
    return I.solver_options(a.tol, **over)


def workload_desc(name, cfg):
    c = I.CONFIGS[name]
    n = "x".join(str(x) for x in cfg["n"])
    grains = c.get("grains", len(cfg["euler"]))
    ctl = "uniaxial strain" if cfg["stress_mask"] is None else "uniaxial stress (mixed control)"
    ratio = "R=0" if c.get("ratio", -1) == 0 else "R=-1"
    return (f"{name}: {n} voxels, {grains} grains, {ratio} {ctl} {100 * c['amplitude']:g}%, "
            f"{c['inc_per_cycle']} increments/cycle")


def probe_dominant(FF, cfg, mat, opts, stream, prec):
    """Per-family kernel times over plastic increments of the workload
    (untimed, on a separate handle): the HBM-bound family with the largest
    total time is the one the timed region measures."""
    import torch
    n = cfg["n"]
    # the probe is untimed: its graph replays are all timed (shares comparable
    # with an ncu launch list of the same window)
    old = os.environ.get("FATIGUEFFT_PROF_SAMPLE")
    os.environ["FATIGUEFFT_PROF_SAMPLE"] = "1"
    r = FF.RVE(n, I.VOXEL_MM, cfg["grain_ids"], cfg["euler"], mat, opts, prec=prec,
               stream=stream)
    if old is None:
        del os.environ["FATIGUEFFT_PROF_SAMPLE"]
    else:
        os.environ["FATIGUEFFT_PROF_SAMPLE"] = old
    drv = Driver(cfg)
    p0, p1 = cfg.get("probe", (8, 14))
    for k in range(p0):
        drv(r, k)
    r.profile(FF.KERNEL_FAMILIES)
    torch.cuda.nvtx.range_push(f"probe_{prec}")  # the window of the committed ncu launch list
    for k in range(p0, p1):
        drv(r, k)
    bd = r.profile_read(reset=True)
    torch.cuda.nvtx.range_pop()
    r.close()
    hbm = {k: v for k, v in bd.items() if k in HBM_FAMILIES and v[1] > 0 and v[2] > 0}
    return max(hbm, key=lambda k: hbm[k][0]), bd


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(self.rows)}


def rank_barrier(ws, dev=None):
    """Device synchronise (when dev is a CUDA device), then a process-group
    barrier when more than one rank runs."""
    import torch
    if dev is not None and dev.type == "cuda":
        torch.cuda.synchronize(dev)
    if ws > 1:
        import torch.distributed as tdist
        tdist.barrier()


def rank_max(x, ws, dev=None):
    """x maximised over the ranks (the slowest rank's time); the reduction
    tensor lives on dev (the rank's GPU under NCCL, the host under gloo)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as tdist
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def rank_sum(x, ws, dev=None):
    """x summed over the ranks (units, iterations and launches of the whole
    job); the reduction tensor lives on dev as in rank_max."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as tdist
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    tdist.all_reduce(t, op=tdist.ReduceOp.SUM)
    return float(t.item())


def rve_cost(n):
    """Estimated cost of one RVE's increment: every Krylov step runs two
    9-field transforms (N log N) and passes over the N voxels."""
    N = int(np.prod(n))
    return N * max(1.0, float(np.log2(N)))


def partition_units(costs, ranks):
    """Independent RVEs split over ranks by longest processing time first:
    the costliest unit goes to the least-loaded rank (ties to the lower rank
    and the lower unit index).  Returns each rank's unit indices, ascending.
    The largest load is within 4/3 of the best split."""
    if ranks < 1 or ranks > len(costs):
        raise ValueError(f"{len(costs)} units cannot fill {ranks} ranks")
    load = [0.0] * ranks
    parts = [[] for _ in range(ranks)]
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(range(ranks), key=lambda r: (load[r], r))
        parts[r].append(i)
        load[r] += costs[i]
    return [sorted(p) for p in parts]


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# A damage-active window of the timed workload's grid (poly64_damage:
# softer slip, full storage of the plastic work, small G_crit): increments
# DAMAGE_WINDOW[0] .. DAMAGE_WINDOW[1] - 1 (0-based) of the first tensile
# half take the first plastic steps, set W_crit and nucleate damage.
DAMAGE_CONFIG = "poly64_damage"
DAMAGE_WINDOW = (4, 8)


def damage_window(FF, a, stream, flush):
    """The mixed path on a damage-active window: voxel-increments/s, the
    phase-field PCG iterations and the phase-field kernels' achieved bytes/s
    (CUDA events per launch, algorithmic bytes) against the copy peak."""
    import torch
    cfg = I.build_config(DAMAGE_CONFIG)
    n, N = cfg["n"], int(np.prod(cfg["n"]))
    mat = I.material("baseline", **cfg["material"])
    opts = workload_options(a, cfg)
    r = FF.RVE(n, I.VOXEL_MM, cfg["grain_ids"], cfg["euler"], mat, opts, prec="mixed",
               stream=stream)
    drv = Driver(cfg)
    w0, w1 = DAMAGE_WINDOW
    for k in range(w0):
        drv(r, k)
    r.profile(["phase_field"])
    ms, stats = [], []
    with torch.cuda.stream(stream):
        for k in range(w0, w1):
            flush.fill_(float(k))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s, st = drv(r, k)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            stats.append(st)
    pf = r.profile_read(reset=True).get("phase_field", (0.0, 0, 0.0))
    r.profile([])
    cracked = stats[-1]["cracked"]
    phimax = float(np.max(r.field("phi")))
    r.close()
    hbm, kind = peaks()
    gbs = pf[2] / pf[0] / 1e6 if pf[0] > 0 else None
    return {"workload": f"{workload_desc(DAMAGE_CONFIG, cfg)}, tau_c0 250 MPa, xi_store 1, "
                        f"G_crit 7e-4 N/mm, increments {w0 + 1}-{w1}",
            "value": round(N * len(ms) / (sum(ms) / 1e3), 1), "unit": "voxel-increments/s",
            "ms_per_step": round(sum(ms) / len(ms), 3), "prec": "mixed",
            "iterations": {"staggered": sum(st["stag_it"] for st in stats),
                           "newton": sum(st["newton_it"] for st in stats),
                           "gmres": sum(st["lin_it_total"] for st in stats),
                           "phase_field": sum(st["pf_it_total"] for st in stats)},
            "phi_max": round(phimax, 4), "cracked": int(cracked),
            "phase_field_kernels": {"launches": int(pf[1]), "ms": round(pf[0], 3),
                                    "algorithmic_bytes": int(pf[2]),
                                    "achieved_gbs": round(gbs, 1) if gbs else None,
                                    "frac": round(gbs / hbm, 4) if gbs else None,
                                    "peak_kind": kind}}


def run_ours(a):
    import torch

    from paper_2304_01125_gb300 import fatiguefft as FF

    ws, rank, local = dist()
    if ws > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2304_01125_gb300 import build as B
    B.build()
    cfg = I.build_config(a.config)
    n, N = cfg["n"], int(np.prod(cfg["n"]))
    prog = cfg["program"]
    assert a.warmup + a.steps <= len(prog)
    mat = I.material("baseline", **cfg.get("material", {}))
    opts = workload_options(a, cfg)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def barrier():
        rank_barrier(ws, dev)

    def max_over_ranks(x):
        return rank_max(x, ws, dev)

    results = {}
    fields = {}
    for prec in ("fp64", "mixed"):
        dom, breakdown = probe_dominant(FF, cfg, mat, opts, stream, prec)
        r = FF.RVE(n, I.VOXEL_MM, cfg["grain_ids"], cfg["euler"], mat, opts, prec=prec,
                   stream=stream)
        drv = Driver(cfg)
        for k in range(a.warmup):
            drv(r, k)
        # only the dominant family is timed (CUDA events in the same stream)
        r.profile([dom])
        barrier()
        clk = Clocks(local)
        clk.start()
        l0 = r.kernel_launches
        times, stats = [], []
        t_wall = time.perf_counter()
        torch.cuda.nvtx.range_push(f"timed_{prec}")
        with torch.cuda.stream(stream):
            for k in range(a.warmup, a.warmup + a.steps):
                flush.fill_(float(k))
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s, st = drv(r, k)
                e1.record(stream)
                stats.append(st)
                times.append((e0, e1))
        barrier()
        torch.cuda.nvtx.range_pop()
        t_wall = time.perf_counter() - t_wall
        clocks = clk.stop()
        launches = r.kernel_launches - l0
        ms = [e0.elapsed_time(e1) for e0, e1 in times]
        dom_prof = r.profile_read(reset=True).get(dom, (0.0, 0, 0.0))
        r.profile([])
        tot = max_over_ranks(sum(ms))
        results[prec] = dict(ms=ms, total_ms=tot, wall_s=t_wall, launches=launches,
                             stats=stats, breakdown=breakdown, dominant=dom,
                             dom_ms=dom_prof[0], dom_count=dom_prof[1], dom_bytes=dom_prof[2],
                             clocks=clocks,
                             device_bytes=r.device_bytes)
        fields[prec] = {f: r.field(f) for f in ("P", "phi", "F")}
        r.close()

    # mixed vs FP64 after the same increments (stress, damage, strain fluctuation)
    def relerr(f, sub=None):
        x, y = fields["mixed"][f], fields["fp64"][f]
        if sub is not None:
            x, y = x - sub, y - sub
        ny = float(np.linalg.norm(y))
        return float(np.linalg.norm(x - y) / ny) if ny > 0 else float(np.abs(x).max())

    eye = np.eye(3).reshape(9, 1)
    errs = {"stress_P": relerr("P"), "damage_phi": relerr("phi"),
            "strain_F_minus_I": relerr("F", eye)}

    # end to end through the public API with host buffers: per step the
    # increment's inputs (Fbar, dt) from pinned host memory and the damage
    # field read back to pinned host memory
    r = FF.RVE(n, I.VOXEL_MM, cfg["grain_ids"], cfg["euler"], mat, opts, prec="mixed",
               stream=stream)
    drv0 = Driver(cfg)
    for k in range(a.warmup):
        drv0(r, k)
    ckpt = r.state_save()  # the window is run three times from here (median)
    mixed_ctl = cfg["stress_mask"] is not None
    host_in = torch.empty((a.steps, 10), dtype=torch.float64).pin_memory()
    for i, k in enumerate(range(a.warmup, a.warmup + a.steps)):
        host_in[i, :9] = torch.from_numpy(prog[k][0])
        host_in[i, 9] = prog[k][1]
    host_out = torch.empty(N, dtype=torch.float64).pin_memory()
    e2e_runs = []
    for _ in range(3):
        r.state_load(ckpt)
        drv = Driver(cfg)
        drv.F = drv0.F
        barrier()
        t0 = time.perf_counter()
        for i in range(a.steps):
            row = host_in[i].numpy()
            if mixed_ctl:  # the guess of the stress-controlled components is the last solved F
                drv(r, a.warmup + i)
            else:
                r.run_increment(row[:9], float(row[9]))
            FF.load().fields_out(r._h, FF.FIELDS["phi"][0], host_out.data_ptr(),
                                 host_out.nbytes, 0)
        barrier()
        e2e_runs.append(max_over_ranks(time.perf_counter() - t0))
    e2e_s = statistics.median(e2e_runs)
    r.close()

    if rank != 0:
        return None
    mx = results["mixed"]
    f64 = results["fp64"]
    value = ws * N * a.steps / (mx["total_ms"] / 1e3)
    value64 = ws * N * a.steps / (f64["total_ms"] / 1e3)
    hbm, peak_kind = peaks()
    dom = mx["dominant"]
    roof = None
    if mx["dom_count"] and mx["dom_ms"] > 0:
        avg_s = mx["dom_ms"] / mx["dom_count"] / 1e3
        bytes_per_launch = mx["dom_bytes"] / mx["dom_count"]
        achieved = bytes_per_launch / avg_s / 1e9
        traffic = ncu_traffic(dom, a.config)
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4),
                "traffic": int(traffic) if traffic is not None else None,
                "kernel": dom, "peak_kind": f"{peak_kind} (copy bandwidth, burst)",
                "algorithmic_bytes_per_launch": int(bytes_per_launch),
                "avg_launch_us": round(avg_s * 1e6, 2), "launches": mx["dom_count"],
                "timing": "CUDA events around the kernel inside the timed region; launches "
                          "replayed from GMRES step graphs are timed on every 8th replay"}
    line = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": "voxel-increments/s",
        "n_gpus": ws,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": round(mx["total_ms"] / a.steps, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic (seeded periodic Voronoi, uniform SO(3) orientations)",
        "config": {"workload": f"{workload_desc(a.config, cfg)}, increments {a.warmup + 1}-"
                               f"{a.warmup + a.steps}",
                   "tolerances": a.tol, "l2": L2_NOTE.format(gb=mx["device_bytes"] / 1e9),
                   "parallelism": f"replicas x{ws}"},
        "fp64": {"value": round(value64, 1), "ms_per_step": round(f64["total_ms"] / a.steps, 3),
                 "dominant_kernel": f64["dominant"]},
        "mixed_speedup_vs_fp64": round(value / value64, 3),
        # the same at equal Krylov work: time per GMRES iteration (the mixed
        # path stops GMRES at an FP32 round-off floor and runs fewer)
        "mixed_speedup_vs_fp64_per_gmres_iteration": round(
            (f64["total_ms"] / max(1, sum(s["lin_it_total"] for s in f64["stats"]))) /
            (mx["total_ms"] / max(1, sum(s["lin_it_total"] for s in mx["stats"]))), 3),
        "mixed_vs_fp64_rel_l2": errs,
        "e2e": {"value": round(ws * N * a.steps / e2e_s, 1), "unit": "voxel-increments/s",
                "h2d_bytes_per_step": 80 + (72 + 36 if mixed_ctl else 0),
                "d2h_bytes_per_step": 8 * N,
                "timing": "wall clock of the window through the public API, median of three "
                          "runs from a checkpoint taken after the warm-up",
                "runs_s": [round(x, 4) for x in e2e_runs]},
        "gpu_launches": int(mx["launches"]),
        "roofline": roof,
        "clocks": mx["clocks"],
        "iterations": {p: {"newton": sum(s["newton_it"] for s in results[p]["stats"]),
                           "gmres": sum(s["lin_it_total"] for s in results[p]["stats"]),
                           "staggered": sum(s["stag_it"] for s in results[p]["stats"]),
                           "phase_field": sum(s["pf_it_total"] for s in results[p]["stats"]),
                           "voxel_gmres_per_s": round(
                               N * sum(s["lin_it_total"] for s in results[p]["stats"]) /
                               (results[p]["total_ms"] / 1e3), 1)}
                       for p in results},
        "kernel_ms_probe": {
            p: {k: round(v[0], 3) for k, v in results[p]["breakdown"].items() if v[1]}
            for p in results},
        "kernel_launches_probe": {
            p: {k: int(v[1]) for k, v in results[p]["breakdown"].items() if v[1]}
            for p in results},
        "kernel_gbs_probe": {
            p: {k: round(v[2] / v[0] / 1e6, 1)
                for k, v in results[p]["breakdown"].items() if v[2] > 0 and v[0] > 0}
            for p in results},
    }
    p0, p1 = cfg.get("probe", (8, 14))
    line["probe_increments"] = [p0 + 1, p1]
    if a.config == CONFIG_NAME and not a.no_damage_window:
        line["damage_window"] = damage_window(FF, a, stream, flush)
    if a.config == CONFIG_NAME and ws == 1 and not a.no_batch_window:
        # the batched workload (32 RVEs of 32^3-96^3, the smallest grids in a
        # lockstep size class): increments 4-13, as `--config batch32`
        import copy
        b = copy.copy(a)
        b.steps, b.warmup = 10, 3
        bl = run_batch(b, short=True)
        line["batch_window"] = {k: bl[k] for k in ("value", "unit", "ms_per_step", "steps",
                                                   "warmup", "roofline", "iterations",
                                                   "kernel_variants")}
        line["batch_window"]["workload"] = bl["config"]["workload"]
        line["batch_window"]["parallelism"] = bl["config"]["parallelism"]
        # 32 cells of 32^3 (one lockstep class) against the same cells on
        # 32 streams: where the lockstep classes pay
        small = {}
        for cls in (True, False):
            b2 = copy.copy(b)
            b2.config, b2.no_classes, b2.classes_all = "batch32x32", not cls, False
            sl = run_batch(b2, short=True)
            small["classes" if cls else "streams"] = {
                "value": sl["value"], "ms_per_step": sl["ms_per_step"],
                "voxel_gmres_per_s": sl["iterations"]["voxel_gmres_per_s"]}
        small["workload"] = sl["config"]["workload"]
        small["unit"] = "voxel-increments/s"
        line["batch_window_32x32"] = small
    if ws == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg, mat, opts, a)
    return line


def run_batch(a, short=False):
    """The batched workload: 32 polycrystals with grids from {32,48,64,96}^3
    (`batch32`; `batch32x32`: 32 of 32^3) and 20-150 grains, advanced
    together (batch_run_increment: lockstep size classes, other handles on
    their own streams), mixed precision.  A step is one load increment of
    every RVE.

    On N ranks (one GPU each) the RVEs are independent units and no data
    crosses ranks: by default rank r advances its own batch of distinct RVEs
    (the units r*count .. (r+1)*count - 1 of the seeded sequence; weak
    scaling); with --batch-split the one batch's RVEs are split over the
    ranks by estimated cost (strong scaling).  The timed steps sit between
    barriers, the time is the slowest rank's and the units are summed over
    the ranks."""
    import torch

    from paper_2304_01125_gb300 import build as B
    from paper_2304_01125_gb300 import fatiguefft as FF

    ws, rank, local = dist()
    if ws > 1 and not short:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    c = I.CONFIGS[a.config if a.config.startswith("batch") else "batch32"]
    split = ws > 1 and a.batch_split
    if split:
        every = I.batch_configs(seed=c["seed"], count=c["count"], sizes=c["sizes"],
                                grains=c["grains"])
        part = partition_units([rve_cost(x["n"]) for x in every], ws)
        cfgs = [every[i] for i in part[rank]]
    else:
        cfgs = I.batch_configs(seed=c["seed"] + rank * c["count"], count=c["count"],
                               sizes=c["sizes"], grains=c["grains"])
    prog = I.uniaxial_cycle_program(c["amplitude"], c["inc_per_cycle"], c["cycles"])
    assert a.warmup + a.steps <= len(prog)
    mat = I.material("baseline")
    # a few of these RVEs stall at the load peaks with the full-step tangent:
    # increments are cut back (halved) on non-convergence, detected early
    opts = I.solver_options(a.tol, max_lin=300, max_cutbacks=4)
    # the Arnoldi step's kernel variant per grid size, timed on this GPU
    # (autotune.py; the unfused variants, which a lockstep class runs)
    variants = {}
    if not a.no_autotune:
        from paper_2304_01125_gb300 import autotune as AT
        for n in sorted({tuple(x["n"]) for x in cfgs}):
            variants[n] = AT.best_variant(n, "mixed", fused=a.no_classes)
    nvox = [int(np.prod(x["n"])) for x in cfgs]
    Ntot = sum(nvox)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def make():
        rv = [FF.RVE(x["n"], I.VOXEL_MM, x["grain_ids"], x["euler"], mat,
                     dict(opts, kernel_variant=variants.get(tuple(x["n"]), 0)), prec="mixed",
                     stream=torch.cuda.Stream(device=dev)) for x in cfgs]
        return rv, FF.Batch(rv, threads=a.batch_threads,
                            classes=False if a.no_classes else ("all" if a.classes_all else True))

    def step(b, k):
        return b.run_increment([prog[k][0]] * len(cfgs), [prog[k][1]] * len(cfgs))

    rves, b = make()
    for k in range(a.warmup):
        step(b, k)
    for r in rves:
        r.profile(["tangent_apply"])
    b.classes(timing=True)
    rank_barrier(ws, dev)
    clk = Clocks(local)
    clk.start()
    l0 = sum(r.kernel_launches for r in rves)
    ms, its, vits, cuts = [], 0, 0, 0
    for k in range(a.warmup, a.warmup + a.steps):
        flush.fill_(float(k))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        _, _, st = step(b, k)  # returns once every RVE's stream is idle
        e1.record()
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        its += sum(x["lin_it_total"] for x in st)
        vits += sum(nv * x["lin_it_total"] for nv, x in zip(nvox, st))
        cuts += sum(x["cutbacks"] for x in st)
    rank_barrier(ws, dev)
    clocks = clk.stop()
    launches = sum(r.kernel_launches for r in rves) - l0
    prof = [r.profile_read(reset=True).get("tangent_apply", (0.0, 0, 0.0)) for r in rves]
    dms, dcnt, dbytes = (sum(p[i] for p in prof) for i in range(3))
    cls = b.classes(timing=False)
    b.close()
    for r in rves:
        r.close()
    total_s = rank_max(sum(ms) / 1e3, ws, dev)
    Njob = int(rank_sum(Ntot, ws, dev))  # voxels of every rank's RVEs
    its, vits, cuts = (int(rank_sum(x, ws, dev)) for x in (its, vits, cuts))
    launches = int(rank_sum(launches, ws, dev))
    Rjob = int(rank_sum(len(cfgs), ws, dev))
    value = Njob * a.steps / total_s
    hbm, peak_kind = peaks()
    roof = None
    g_ms = sum(c[2] for c in cls)
    g_by = sum(c[3] for c in cls)
    g_n = sum(c[1] for c in cls)
    if g_ms > 0:
        # the lockstep classes' Krylov column graphs: every member's two
        # 9-field transforms, tangent apply, contraction + dots and update
        avg_s = g_ms / 1e3 / max(g_n, 1)
        roof = {"bound": "hbm", "achieved": round(g_by / (g_ms / 1e3) / 1e9, 1), "peak": hbm,
                "unit": "GB/s", "frac": round(g_by / (g_ms / 1e3) / 1e9 / hbm, 4),
                "traffic": None,
                "kernel": "class Krylov column graph (batched 9-field transforms, tangent "
                          "applies, contraction+dots, updates of all members)",
                "peak_kind": f"{peak_kind} (copy bandwidth, burst)",
                "algorithmic_bytes_per_launch": int(g_by / max(g_n, 1)),
                "avg_launch_us": round(avg_s * 1e6, 2), "launches": int(g_n),
                "timing": "CUDA events on each class's stream around its graph launches; the "
                          "classes run concurrently, so a launch's interval includes time "
                          "shared with the other classes (a lower bound on its bandwidth)"}
    elif dcnt and dms > 0:
        avg_s = dms / dcnt / 1e3
        bpl = dbytes / dcnt
        roof = {"bound": "hbm", "achieved": round(bpl / avg_s / 1e9, 1), "peak": hbm,
                "unit": "GB/s", "frac": round(bpl / avg_s / 1e9 / hbm, 4), "traffic": None,
                "kernel": "tangent_apply (mean over the batch's grid sizes)",
                "peak_kind": f"{peak_kind} (copy bandwidth, burst)",
                "algorithmic_bytes_per_launch": int(bpl), "avg_launch_us": round(avg_s * 1e6, 2),
                "launches": int(dcnt),
                "timing": "CUDA events on each RVE's stream while the other RVEs' kernels run "
                          "concurrently: a launch's interval includes time shared with them, so "
                          "this is a lower bound on the kernel's own bandwidth"}
    if short:
        e2e_s = serial_s = None
    else:
        e2e_s, serial_s = batch_e2e_and_serial(a, make, step, nvox, prog, ws, dev)
    sizes = {}
    for x in (every if split else cfgs):
        sizes[x["n"][0]] = sizes.get(x["n"][0], 0) + 1
    line = batch_line(a, ws, rank, Rjob, sizes, Njob, total_s, value, e2e_s, serial_s, launches,
                      roof, clocks, its, cuts, cls, variants, vits, split)
    if ws > 1 and not short:
        import torch.distributed as tdist
        tdist.destroy_process_group()
    return line


def batch_e2e_and_serial(a, make, step, nvox, prog, ws=1, dev=None):
    """End to end (fresh handles, inputs from pinned host memory, every RVE's
    damage field read back each step) and the handles run one after
    another: wall seconds of the same increments (the slowest rank's)."""
    import torch

    from paper_2304_01125_gb300 import fatiguefft as FF
    rves, b = make()
    for k in range(a.warmup):
        step(b, k)
    host_out = [torch.empty(nv, dtype=torch.float64).pin_memory() for nv in nvox]
    rank_barrier(ws, dev)
    t0 = time.perf_counter()
    for k in range(a.warmup, a.warmup + a.steps):
        step(b, k)
        for r, h in zip(rves, host_out):
            FF.load().fields_out(r._h, FF.FIELDS["phi"][0], h.data_ptr(), h.nbytes, 0)
    rank_barrier(ws, dev)
    e2e_s = rank_max(time.perf_counter() - t0, ws, dev)
    b.close()
    for r in rves:
        r.close()
    # the same increments with the handles advanced one after another (no
    # concurrency): what the batch gains over running the RVEs in turn
    rves, b = make()
    for k in range(a.warmup):
        step(b, k)
    rank_barrier(ws, dev)
    t0 = time.perf_counter()
    for k in range(a.warmup, a.warmup + a.steps):
        for r in rves:
            r.run_increment(prog[k][0], prog[k][1])
    rank_barrier(ws, dev)
    serial_s = rank_max(time.perf_counter() - t0, ws, dev)
    b.close()
    for r in rves:
        r.close()
    return e2e_s, serial_s


def batch_line(a, ws, rank, Rjob, sizes, Ntot, total_s, value, e2e_s, serial_s, launches, roof,
               clocks, its, cuts, cls, variants, vits, split=False):
    """The batch's JSON line.  Rjob (RVEs), Ntot (voxels), launches, its,
    cuts and vits are the whole job's (summed over the ranks), total_s the slowest rank's seconds
    over the timed steps; sizes counts the grids of the job's RVEs (of the
    one batch when it is split, of rank 0's batch otherwise)."""
    names = a.config if a.config.startswith("batch") else "batch32"
    if ws == 1:
        who = f"{names}: {sum(sizes.values())} RVEs"
    elif split:
        who = f"{names} split over {ws} ranks by estimated cost: {sum(sizes.values())} RVEs"
    else:
        who = (f"{names} on each of {ws} ranks (distinct seeded RVEs per rank): "
               f"{sum(sizes.values())} RVEs per rank, rank 0's")
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "voxel-increments/s",
        "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": round(total_s * 1e3 / a.steps, 3), "higher_is_better": True,
        "scaling": "strong" if split else "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic (seeded periodic Voronoi, uniform SO(3) orientations)",
        "config": {"workload": f"{who}, grids "
                               + ", ".join(f"{k}^3 x{v}" for k, v in sorted(sizes.items()))
                               + f" ({Ntot} voxels in the job), 20-150 grains, R=-1 uniaxial "
                                 f"strain 0.6%, "
                               f"30 increments/cycle, increments {a.warmup + 1}-"
                               f"{a.warmup + a.steps}",
                   "tolerances": a.tol, "cutbacks": "on (max_cutbacks 4, max_lin 300)",
                   "l2": ("working set > L2 (32 handles) and a 256 MB L2 flush before every "
                          "step"),
                   "parallelism": ("one stream per RVE" if a.no_classes or not cls else
                                   "lockstep size classes "
                                   + ", ".join(f"{c[0]} members" for c in cls)
                                   + " (one graph launch per Krylov column per class, batched "
                                     "9-field transforms); one stream per RVE otherwise")
                                  + ("" if ws == 1 else
                                     f"; {ws} ranks, one GPU each, no data exchanged between "
                                     "ranks")},
        "e2e": None if e2e_s is None else {
            "value": round(Ntot * a.steps / e2e_s, 1), "unit": "voxel-increments/s",
            "h2d_bytes_per_step": 80 * Rjob, "d2h_bytes_per_step": 8 * Ntot},
        "gpu_launches": int(launches), "roofline": roof, "clocks": clocks,
        "iterations": {"gmres": its, "cutbacks": cuts,
                       "voxel_gmres_per_s": round(vits / total_s, 1),
                       "note": "voxel_gmres_per_s: sum over RVEs of voxels x GMRES iterations "
                               "per second of the timed steps (Krylov throughput independent "
                               "of how many iterations the increments need)"},
        "serial": None if serial_s is None else {
            "value": round(Ntot * a.steps / serial_s, 1), "unit": "voxel-increments/s",
            "note": "the same increments, one handle after another (wall clock)"},
        "host_threads": a.batch_threads or "hardware concurrency",
        "kernel_variants": ({f"{n[0]}^3": v for n, v in sorted(variants.items())}
                            or "default (bulk-copy update pass, unfused)"),
    }
    return line if rank == 0 else None


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the
    machine type), recorded beside the oracle's timings."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine() or "unknown"


def cpu_baseline(cfg, mat, opts, a, budget_s=30.0):
    """The FP64 oracle as it stands, on the host cores: the timed window's
    increments from its first, as many as fit in about budget_s seconds
    (at least one), after the same warm-up increments run on the oracle,
    untimed -- the start of the window the reference arm times."""
    import oracle as O
    import oracle.build as OB

    OB.build()
    threads = os.cpu_count() or 1
    r = O.RVE(cfg["n"], I.VOXEL_MM, cfg["grain_ids"], cfg["euler"], mat, opts, threads=threads)
    drv = Driver(cfg)
    for k in range(a.warmup):
        drv(r, k)
    N = int(np.prod(cfg["n"]))
    t0 = time.perf_counter()
    increments = 0
    for k in range(a.warmup, a.warmup + a.steps):
        drv(r, k)
        increments += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": round(N * increments / dt, 1), "unit": "voxel-increments/s",
            "cores": threads, "cpu": cpu_model(), "kind": "oracle",
            "sample": f"{increments} increment(s) of the timed window "
                      f"(increments {a.warmup + 1}-{a.warmup + increments}), {dt:.1f} s"}


def run_reference(a):
    ws, rank, local = dist()
    if rank != 0:
        return None
    import oracle as O
    import oracle.build as OB

    OB.build()
    cfg = I.build_config(a.config)
    N = int(np.prod(cfg["n"]))
    mat = I.material("baseline", **cfg.get("material", {}))
    opts = workload_options(a, cfg)
    threads = os.cpu_count() or 1
    r = O.RVE(cfg["n"], I.VOXEL_MM, cfg["grain_ids"], cfg["euler"], mat, opts, threads=threads)
    drv = Driver(cfg)
    for k in range(a.warmup):
        drv(r, k)
    t0 = time.perf_counter()
    done = 0
    for k in range(a.warmup, a.warmup + a.steps):
        drv(r, k)
        done += 1
        if time.perf_counter() - t0 > a.ref_budget_s:
            break
    dt = time.perf_counter() - t0
    value = N * done / dt
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 1),
        "unit": "voxel-increments/s", "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": round(dt / done * 1e3, 1), "higher_is_better": True,
        "steps_timed": done,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded periodic Voronoi, uniform SO(3) orientations)",
        "config": {"workload": f"{workload_desc(a.config, cfg)}, increments {a.warmup + 1}-"
                               f"{a.warmup + a.steps}", "tolerances": a.tol},
        "cpu_baseline": {"value": round(value, 1), "unit": "voxel-increments/s",
                         "cores": threads, "cpu": cpu_model(), "kind": "oracle",
                         "sample": f"{done} full increments of the workload (increments "
                                   f"{a.warmup + 1}-{a.warmup + done}; the run stops timing "
                                   f"after {a.ref_budget_s:.0f} s), {dt:.1f} s"},
        "e2e": {"value": round(value, 1), "unit": "voxel-increments/s",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    a = args_()
    if a.impl == "reference":
        line = run_reference(a)
    elif a.config in ("batch32", "batch32x32"):
        line = run_batch(a)
    else:
        line = run_ours(a)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
