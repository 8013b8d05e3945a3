"""The batched bench's host logic on the CPU: run_batch driven through
stand-ins for the library's handles and batch and for the CUDA calls, so
that the step loop, the timing, the sums and the JSON line are exercised
without a GPU.  The stand-ins report fixed iteration counts and fixed
event times, so every number of the line is known in advance."""
import argparse
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

EVENT_MS = 5.0  # every timed step


class _Event:
    def __init__(self, enable_timing=False):
        pass

    def record(self, stream=None):
        pass

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return EVENT_MS


class _Stream:
    def __init__(self, device=None):
        pass


class _RVE:
    def __init__(self, n, h, gid, eul, mat, opts, prec, stream):
        self.n = n
        self.opts = opts
        self.kernel_launches = 0
        self._h = None

    def profile(self, names):
        pass

    def profile_read(self, reset=False):
        return {"tangent_apply": (1.0, 4, 4e8)}

    def run_increment(self, Fbar, dt):
        self.kernel_launches += 10
        return 0, {}

    def close(self):
        pass


class _Batch:
    made = []

    def __init__(self, rves, threads=None, classes=True):
        self.rves = rves
        self.cls = classes
        _Batch.made.append(self)

    def run_increment(self, Fbars, dts):
        assert len(Fbars) == len(dts) == len(self.rves)
        for r in self.rves:
            r.kernel_launches += 10
        return 0, [0] * len(self.rves), [{"lin_it_total": 3, "cutbacks": 0}
                                          for _ in self.rves]

    def classes(self, timing=None):
        return [(2, 8, 4.0, 2e8)] if self.cls else []

    def close(self):
        pass


class _Lib:
    def fields_out(self, h, fid, ptr, nbytes, on_device):
        return 0


@pytest.fixture
def fake(monkeypatch):
    import torch

    import bench
    from paper_2304_01125_gb300 import build as B
    from paper_2304_01125_gb300 import fatiguefft as FF

    seeds = []

    def batch_configs(seed, count, sizes, grains):
        seeds.append(seed)
        rng = np.random.default_rng(seed)
        out = []
        for r in range(count):
            s = int(sizes[rng.integers(len(sizes))]) // 8  # tiny stand-in grids
            out.append(dict(n=(s, s, s), grain_ids=np.zeros(s ** 3, np.int32),
                            euler=np.zeros((1, 3))))
        return out

    orig_empty = torch.empty

    def empty(*shape, **kw):
        kw.pop("device", None)
        return orig_empty(16, **kw) if kw.get("dtype") == torch.float32 else \
            orig_empty(*shape, **kw)

    monkeypatch.setattr(B, "build", lambda *a, **k: None)
    monkeypatch.setattr(FF, "RVE", _RVE)
    monkeypatch.setattr(FF, "Batch", _Batch)
    monkeypatch.setattr(FF, "load", lambda: _Lib())
    monkeypatch.setattr(bench.I, "batch_configs", batch_configs)
    monkeypatch.setattr(bench, "Clocks", lambda i: argparse.Namespace(
        start=lambda: None, stop=lambda: {"sm_mhz": None, "reasons": []}))
    monkeypatch.setattr(torch, "empty", empty)
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self: self)
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda d=None: None)
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "Stream", _Stream)
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    _Batch.made.clear()
    return seeds


def _args(**kw):
    d = dict(config="batch32", steps=2, warmup=3, tol="paper", no_autotune=True,
             no_classes=False, classes_all=False, batch_threads=None, batch_split=False)
    d.update(kw)
    return argparse.Namespace(**d)


def test_batch_window_line(fake):
    """The default bench line's batch window (one rank, short): every
    figure follows from the stand-ins' counts and times."""
    import bench
    line = bench.run_batch(_args(), short=True)
    assert fake == [bench.I.CONFIGS["batch32"]["seed"]]  # rank 0's units: the batch itself
    rves = _Batch.made[0].rves
    N = sum(int(np.prod(r.n)) for r in rves)
    assert line["value"] == pytest.approx(N * 2 / (2 * EVENT_MS / 1e3), rel=1e-6)
    assert line["ms_per_step"] == EVENT_MS and line["scaling"] == "weak"
    assert line["iterations"]["gmres"] == 3 * len(rves) * 2
    assert line["gpu_launches"] == 10 * len(rves) * 2
    assert line["e2e"] is None and line["serial"] is None
    # the class graphs' bytes over their event time
    assert line["roofline"]["achieved"] == pytest.approx(2e8 / 4e-3 / 1e9, abs=0.1)
    assert f"({N} voxels in the job)" in line["config"]["workload"]
    assert "lockstep size classes 2 members" in line["config"]["parallelism"]


def test_batch_full_line_has_e2e_and_serial(fake):
    import bench
    line = bench.run_batch(_args(no_classes=True))
    rves = _Batch.made[0].rves
    N = sum(int(np.prod(r.n)) for r in rves)
    assert line["e2e"]["value"] > 0 and line["serial"]["value"] > 0
    assert line["e2e"]["d2h_bytes_per_step"] == 8 * N
    assert line["e2e"]["h2d_bytes_per_step"] == 80 * len(rves)
    assert line["config"]["parallelism"] == "one stream per RVE"
    # without classes the roofline falls back to the tangent apply's events
    assert line["roofline"]["kernel"].startswith("tangent_apply")
    assert line["roofline"]["achieved"] == pytest.approx(4e8 / 4 / (1.0 / 4 / 1e3) / 1e9, abs=0.1)
