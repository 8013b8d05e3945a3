"""The command-line driver's loop without a GPU: one JSON-serialisable
record per increment with the statistics, the solved macroscopic F carried
into the stress-controlled components of the next increment, a stop at the
first failed increment."""
import json

import numpy as np

from paper_2304_01125_gb300 import inputs as I
from paper_2304_01125_gb300 import run


class FakeRVE:
    def __init__(self, fail_at=None):
        self.calls, self.fail_at = [], fail_at

    def run_increment(self, Fbar, dt, check=True, Pbar=None, stress_mask=None):
        k = len(self.calls)
        self.calls.append(np.array(Fbar))
        F = np.array(Fbar, dtype=float)
        if stress_mask is not None:
            F = F - 1e-3 * (np.asarray(stress_mask) == 1)
        st = {key: 1 for key in run.STAT_KEYS}
        st.update(Fbar=F.tolist(), Pbar=[0.0] * 9)
        return (-5 if k == self.fail_at else 0), st

    def field(self, name):
        return np.array([0.25, 0.5])


def test_records_and_carried_lateral_strain():
    cfg = I.build_config("plate256_bx45", n_override=(8, 8, 1))
    recs = []
    r = FakeRVE()
    done = run.drive(r, cfg, 3, recs.append, phi_max=True)
    assert done == 3 and [x["increment"] for x in recs] == [0, 1, 2]
    for x in recs:
        json.dumps(x)
        assert x["status"] == 0 and x["phi_max"] == 0.5 and len(x["Fbar"]) == 9
        assert all(k in x for k in run.STAT_KEYS)
    m = cfg["stress_mask"]
    assert np.allclose(r.calls[1][m == 1], r.calls[0][m == 1] - 1e-3)
    assert np.array_equal(r.calls[1][m == 0], cfg["program"][1][0][m == 0])


def test_stops_at_the_first_failure():
    cfg = I.build_config("poly64", n_override=(4, 4, 4))
    recs = []
    done = run.drive(FakeRVE(fail_at=1), cfg, 5, recs.append)
    assert done == 1 and len(recs) == 2 and recs[-1]["status"] == -5
    assert "phi_max" not in recs[0]


def test_option_overrides():
    o = run.option_overrides("paper", ["max_lin=5000", "tol_lin=1e-6", "derivative=willot",
                                       "kernel_variant=2"])
    assert o == {"max_lin": 5000, "tol_lin": 1e-6, "derivative": "willot", "kernel_variant": 2}
    assert isinstance(o["max_lin"], int)
    import pytest
    for bad in (["derivative=central"], ["no_such=1"]):
        with pytest.raises(ValueError):
            run.option_overrides("paper", bad)
