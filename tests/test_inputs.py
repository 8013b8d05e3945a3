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


def test_cycle_program_4q_plus_2_hits_the_peaks_without_holds():
    a, rate = 0.006, 1e-3
    prog = I.uniaxial_cycle_program(a, 30, 2, eps_rate=rate)
    e = _eps(prog)
    assert len(prog) == 60
    assert np.isclose(e.max(), a) and np.isclose(e.min(), -a)
    assert np.allclose(e[7::30], a) and np.allclose(e[22::30], -a)
    de = np.abs(np.diff(np.concatenate([[0.0], e])))
    step = 4 * a / 30
    assert np.isclose(de[0], step / 2) and np.allclose(de[1:], step)  # no zero increments
    dts = np.array([dt for _, dt in prog])
    assert np.allclose(dts, de / rate)


def test_cycle_program_rejects_odd_counts():
    import pytest
    with pytest.raises(ValueError):
        I.uniaxial_cycle_program(0.006, 31, 1)
