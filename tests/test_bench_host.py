"""Host logic of bench.py that needs no GPU: the increment driver (solved
macroscopic F carried between increments under a stress mask), the
per-workload solver options and the workload description."""
import numpy as np

import bench
from paper_2304_01125_gb300 import inputs as I


class FakeRVE:
    """Records run_increment calls; 'solves' the stress-controlled
    components by adding a fixed offset to the guess."""

    def __init__(self):
        self.calls = []

    def run_increment(self, Fbar, dt, Pbar=None, stress_mask=None):
        self.calls.append((np.array(Fbar), dt, stress_mask))
        F = np.array(Fbar, dtype=float)
        if stress_mask is not None:
            F = F + 0.01 * (np.asarray(stress_mask) == 1)
        return 0, {"Fbar": F.tolist()}


def test_driver_carries_the_solved_lateral_strain():
    cfg = I.build_config("poly64_r0", n_override=(4, 4, 4))
    m = cfg["stress_mask"]
    r, drv = FakeRVE(), bench.Driver(cfg)
    for k in range(3):
        drv(r, k)
    F0, F1, F2 = (c[0] for c in r.calls)
    assert np.array_equal(F0, cfg["program"][0][0])
    assert np.allclose(F1[m == 1], F0[m == 1] + 0.01)  # previous solved value
    assert np.allclose(F2[m == 1], F0[m == 1] + 0.02)
    assert np.array_equal(F2[m == 0], cfg["program"][2][0][m == 0])
    assert all(np.array_equal(c[2], m) for c in r.calls)


def test_driver_under_strain_control_passes_the_targets():
    cfg = I.build_config("poly64", n_override=(4, 4, 4))
    r, drv = FakeRVE(), bench.Driver(cfg)
    for k in range(2):
        drv(r, k)
    for (F, dt, m), (Fb, dtb) in zip(r.calls, cfg["program"]):
        assert np.array_equal(F, Fb) and dt == dtb and m is None
    assert drv.F is None


def test_workload_options_and_description():
    class A:
        tol = "paper"

    strain = I.build_config("poly64", n_override=(4, 4, 4))
    mixed = I.build_config("poly64_r0", n_override=(4, 4, 4))
    assert bench.workload_options(A, strain) == I.solver_options("paper")
    assert bench.workload_options(A, mixed)["max_cutbacks"] == 4
    assert bench.workload_desc("poly64", strain).startswith(
        "poly64: 4x4x4 voxels, 50 grains, R=-1 uniaxial strain 0.6%")
    assert "R=0 uniaxial stress (mixed control) 2%" in bench.workload_desc("poly64_r0", mixed)


def test_committed_traffic_applies_only_to_its_workload_and_sources(tmp_path, monkeypatch):
    """roofline.traffic comes from the committed ncu summary only for the
    workload it was captured on and while the kernel sources hash to the
    recorded value."""
    import json
    sha = bench.source_sha1()
    f = tmp_path / "t.json"
    f.write_text(json.dumps({"poly64": {"gmres_dot": {"dram_bytes_per_launch": 123,
                                                      "source_sha1": sha}},
                             "poly128": {"gmres_dot": {"dram_bytes_per_launch": 7,
                                                       "source_sha1": "old"}}}))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.ncu_traffic("gmres_dot", "poly64") == 123
    assert bench.ncu_traffic("gmres_dot", "poly256") is None  # other workload
    assert bench.ncu_traffic("gmres_dot", "poly128") is None  # other kernel sources
    assert bench.ncu_traffic("tangent_apply", "poly64") is None


def test_cpu_model_is_a_name():
    import bench
    m = bench.cpu_model()
    assert isinstance(m, str) and m and "\n" not in m
