"""Per-grid choice of the Arnoldi step's kernel variant, measured on the GPU
at first use and cached in a JSON file.

The library has two variant bits (``kernel_variant`` in the solver options,
see include/fatiguefft.h): the fused x pass (inverse real transform along x,
tangent apply and forward real transform in one kernel between batched 2-D
transforms) and the register-streaming Arnoldi update pass (in place of the
pipelined bulk-copy one).  All variants give the same results to the Krylov
tolerance; which is fastest depends on the grid (how much of a step is
launch latency and how much is memory traffic) and on the precision.  The
tuner times a few elastic increments of a small synthetic polycrystal on the
grid for every candidate, per GMRES iteration, and keeps the fastest.

Cache: ``$FATIGUEFFT_AUTOTUNE_CACHE`` or ``~/.cache/fatiguefft/autotune.json``,
keyed by the GPU name, the grid and the precision.
"""
import json
import math
import os
import tempfile

from . import inputs as I

CACHE_ENV = "FATIGUEFFT_AUTOTUNE_CACHE"


def cache_path():
    return os.environ.get(CACHE_ENV) or os.path.join(os.path.expanduser("~"), ".cache",
                                                     "fatiguefft", "autotune.json")


def candidates(n, fused=True):
    """Variant values worth timing on grid n: the fused x pass only where the
    library can use it (n0 a power of two in [8, 512], not a line) and when
    allowed (a lockstep batch class runs the unfused step)."""
    n0 = int(n[0])
    fused_ok = fused and 8 <= n0 <= 512 and (n0 & (n0 - 1)) == 0 and (n[1] > 1 or n[2] > 1)
    return [0, 2] + ([1, 3] if fused_ok else [])


def measure(n, prec, variant, stream=None, increments=2):
    """Device milliseconds per GMRES iteration of `increments` elastic
    increments of a three-grain polycrystal on grid n (after one untimed
    increment that captures the step graphs); the best of the increments."""
    import torch

    from . import fatiguefft as FF
    gid, eul = I.voronoi(n, 3, 7)
    opts = I.solver_options("paper", kernel_variant=int(variant))
    stream = stream or torch.cuda.Stream()
    r = FF.RVE(n, I.VOXEL_MM, gid, eul, I.material("baseline"), opts, prec=prec,
               stream=stream)
    prog = I.uniaxial_cycle_program(0.002, 8, 1)
    try:
        r.run_increment(*prog[0])
        best = math.inf
        for Fb, dt in prog[1:1 + increments]:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, st = r.run_increment(Fb, dt)
            e1.record(stream)
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / max(1, st["lin_it_total"]))
    finally:
        r.close()
    return best


def _load(path):
    """The cache's entries; an unreadable or malformed file counts as empty."""
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {}
    return data if isinstance(data, dict) else {}


def _cached(data, key, allowed):
    """The stored variant for key if it is one of the allowed values, else
    None (a damaged or outdated entry is measured again)."""
    e = data.get(key)
    v = e.get("kernel_variant") if isinstance(e, dict) else None
    return v if type(v) is int and v in allowed else None


def _store(path, data):
    """Write the cache atomically; a cache that cannot be written (a
    read-only home, a full disk) only costs the measurement next time."""
    tmp = None
    try:
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=os.path.dirname(path) or ".", suffix=".tmp")
        with os.fdopen(fd, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        if tmp and os.path.exists(tmp):
            os.unlink(tmp)


def best_variant(n, prec, device_name=None, stream=None, path=None, refresh=False,
                 measure_fn=None, fused=True):
    """The fastest kernel variant for grid n and precision prec on this GPU
    (fused=False: among the unfused ones): from the cache, else measured
    (measure_fn(n, prec, variant) -> ms per GMRES iteration; the GPU
    measurement by default) and stored."""
    n = tuple(int(x) for x in n)
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name()
    path = path or cache_path()
    key = f"{device_name}|{n[0]}x{n[1]}x{n[2]}|{prec}" + ("" if fused else "|unfused")
    allowed = candidates(n, fused)
    hit = _cached(_load(path), key, allowed)
    if hit is not None and not refresh:
        return hit
    fn = measure_fn or (lambda nn, pp, v: measure(nn, pp, v, stream=stream))
    times = {v: float(fn(n, prec, v)) for v in allowed}
    best = min(times, key=lambda v: (times[v], v))
    data = _load(path)  # another process may have written meanwhile
    data[key] = {"kernel_variant": best,
                 "ms_per_gmres_iteration": {str(v): round(t, 6) for v, t in times.items()}}
    _store(path, data)
    return best
