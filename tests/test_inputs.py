"""Seeded input generators (host logic shared by the tests, smoke and the
benchmark): the R = -1 triangle-wave loading programs."""
import numpy as np

from paper_2304_01125_gb300 import inputs as I


def _eps(prog):
    return np.array([F[4] - 1.0 for F, _ in prog])


def test_cycle_program_multiple_of_four_hits_the_peaks():
    a, rate = 0.006, 1e-3
    prog = I.uniaxial_cycle_program(a, 40, 3, eps_rate=rate)
    e = _eps(prog)
    assert len(prog) == 120
    assert np.isclose(e.max(), a) and np.isclose(e.min(), -a)
    assert np.allclose(e[9::40], a) and np.allclose(e[29::40], -a)
    assert np.allclose(e[39::40], 0.0, atol=1e-15)
    dts = np.array([dt for _, dt in prog])
    assert np.allclose(dts, (a / 10) / rate)


def test_cycle_program_equal_time_sampling():
    a, rate = 0.006, 1e-3
    prog = I.uniaxial_cycle_program(a, 30, 2, eps_rate=rate)
    e = _eps(prog)
    assert len(prog) == 60
    assert np.all(np.abs(e) <= a + 1e-15)
    assert np.allclose(e[29::30], 0.0, atol=1e-15)  # each cycle ends at zero strain
    dts = np.array([dt for _, dt in prog])
    assert np.all(dts > 0) and np.allclose(dts, 4 * a / (rate * 30))
    # the strain rate never exceeds the nominal one
    de = np.abs(np.diff(np.concatenate([[0.0], e])))
    assert np.all(de <= rate * dts + 1e-15)
