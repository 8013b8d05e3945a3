"""Command-line driver: run a configuration's loading program on the GPU and
write one JSON line of statistics per increment.

    python -m paper_2304_01125_gb300.run --config plate256_sx100 --increments 20 \\
        --prec mixed --out stats.jsonl

Each line holds the increment index, its status, dt, the macroscopic F and
the mean degraded first Piola stress, the iteration counts of the staggered
loop, Newton, GMRES and the phase field, local failures, cut-backs, mixed
control rounds and the cracked-voxel count; with --phi-max also the largest
phase-field value, stored energy density G_s and the number of voxels whose
W_crit is set (field reads per increment).  --mat and --opt override
material constants and solver options (KEY=VALUE, repeatable).  Under a stress mask
(uniaxial stress, plane stress of the plates) the stress-controlled
components of each increment start from the previous solved F.  The run
stops at the first increment that fails.  --checkpoint writes the state
(state_save) after the last converged increment; --fields-out writes the
final phase field and W_crit (NumPy .npz, FP32).
"""
import argparse
import json
import sys
import time

import numpy as np

from . import inputs as I

STAT_KEYS = ("stag_it", "newton_it", "lin_it_total", "pf_it_total", "local_fail", "cutbacks",
             "mixed_it", "cracked", "converged")


def drive(rve, cfg, increments, emit, phi_max=False, after=None):
    """Run increments [0, increments) of cfg's program on rve (anything with
    the RVE's run_increment and field methods), calling emit(record) after
    each and after(k) after each converged one; returns the number of
    converged increments."""
    F = None
    done = 0
    for k in range(min(increments, len(cfg["program"]))):
        args, kw = I.increment_args(cfg, k, F)
        t0 = time.perf_counter()
        s, st = rve.run_increment(*args, check=False, **kw)
        rec = {"increment": k, "status": int(s), "dt": float(args[1]),
               "ms": round((time.perf_counter() - t0) * 1e3, 3)}
        rec.update({key: st[key] for key in STAT_KEYS if key in st})
        rec["Fbar"] = [float(x) for x in st["Fbar"]]
        rec["Pbar"] = [float(x) for x in st["Pbar"]]
        if phi_max and s == 0:
            rec["phi_max"] = float(np.max(rve.field("phi")))
            rec["gs_max"] = float(np.max(rve.field("Gs")))
            rec["wcrit_set"] = int(np.count_nonzero(rve.field("Wcrit")))
        emit(rec)
        if s != 0:
            break
        done += 1
        if after is not None:
            after(k)
        if kw:
            F = np.array(st["Fbar"])
    return done


def option_overrides(tol, pairs):
    """Solver options from KEY=VALUE strings: the numeric options of the
    preset (typed as the preset's), `kernel_variant` (int) and `derivative`
    (spectral | willot); ValueError for anything else."""
    base = I.solver_options(tol)
    out = {}
    for kv in pairs:
        k, v = kv.split("=", 1)
        if k == "derivative":
            if v not in ("spectral", "willot"):
                raise ValueError(f"derivative must be spectral or willot, not {v}")
            out[k] = v
        elif k == "kernel_variant":
            out[k] = int(v)
        elif k in base:
            out[k] = type(base[k])(float(v))
        else:
            raise ValueError(f"unknown solver option {k}")
    return out


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    p.add_argument("--config", default="poly64",
                   choices=sorted(k for k in I.CONFIGS if "sizes" not in I.CONFIGS[k]))
    p.add_argument("--increments", type=int, default=10)
    p.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    p.add_argument("--tol", default="paper", choices=["paper", "parity32", "parity64"])
    p.add_argument("--n", default=None, help="grid override, e.g. 32,32,32")
    p.add_argument("--max-cutbacks", type=int, default=None)
    p.add_argument("--phi-max", action="store_true")
    p.add_argument("--out", default="-", help="JSON lines file (- for stdout)")
    p.add_argument("--checkpoint", default=None, help="write state_save here at the end")
    p.add_argument("--cycles", type=int, default=None, help="loading cycles (default: the config's)")
    p.add_argument("--fields-out", default=None, help="write phi and Wcrit (.npz) at the end")
    p.add_argument("--fields-every", type=int, default=0,
                   help="with --fields-out: also write <stem>_<increment>.npz after every K "
                        "converged increments")
    p.add_argument("--mat", action="append", default=[], help="material override KEY=VALUE")
    p.add_argument("--opt", action="append", default=[], help="solver option override KEY=VALUE")
    a = p.parse_args(argv)
    if a.config == "batch32":
        p.error("batch32 is a set of RVEs: use bench.py --config batch32")
    import torch
    from . import fatiguefft as FF

    n = tuple(int(x) for x in a.n.split(",")) if a.n else None
    cfg = I.build_config(a.config, n_override=n, cycles=a.cycles)
    over = dict(cfg.get("options", {}))
    if a.max_cutbacks is not None:
        over["max_cutbacks"] = a.max_cutbacks
    try:
        over.update(option_overrides(a.tol, a.opt))
    except ValueError as e:
        p.error(str(e))
    opts = I.solver_options(a.tol, **over)
    mat = I.material("baseline", **cfg.get("material", {}))
    for kv in a.mat:
        k, v = kv.split("=", 1)
        if k not in mat:
            p.error(f"unknown material constant {k}")
        mat[k] = float(v)
    rve = FF.RVE(cfg["n"], cfg["h"], cfg["grain_ids"], cfg["euler"], mat,
                 opts, prec=a.prec, stream=torch.cuda.Stream(), phi0=cfg["phi0"],
                 elastic_only=cfg["elastic_only"])
    out = sys.stdout if a.out == "-" else open(a.out, "w")

    def save_fields(k, path):
        np.savez_compressed(path, phi=rve.field("phi").astype(np.float32),
                            Wcrit=rve.field("Wcrit").astype(np.float32), increment=k)

    def after(k):
        if a.fields_out and a.fields_every > 0 and (k + 1) % a.fields_every == 0:
            stem = a.fields_out[:-4] if a.fields_out.endswith(".npz") else a.fields_out
            save_fields(k, f"{stem}_{k + 1:05d}.npz")

    try:
        done = drive(rve, cfg, a.increments,
                     lambda rec: (out.write(json.dumps(rec) + "\n"), out.flush()),
                     phi_max=a.phi_max, after=after)
        if a.checkpoint:
            with open(a.checkpoint, "wb") as f:
                f.write(rve.state_save())
        if a.fields_out:
            save_fields(done - 1, a.fields_out)
    finally:
        if out is not sys.stdout:
            out.close()
        rve.close()
    return 0 if done == min(a.increments, len(cfg["program"])) else 1


if __name__ == "__main__":
    sys.exit(main())
