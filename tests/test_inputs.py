"""Seeded input generators (host logic shared by the tests, smoke and the
benchmark): the loading programs, the stress masks and the plate
microstructures."""
import numpy as np
import pytest

import oracle as O
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


def test_pulsating_program():
    """R = 0 loading of Sec. 4: 0 -> eps_max -> 0 per cycle, equal steps,
    peak and zero sampled, no increment that holds the strain."""
    prog = I.pulsating_cycle_program(0.02, 8, 2)
    eps = np.array([F[4] - 1.0 for F, _ in prog])
    assert np.allclose(eps, [0.005, 0.01, 0.015, 0.02, 0.015, 0.01, 0.005, 0.0] * 2)
    assert min(eps) >= 0.0 and abs(eps.max() - 0.02) < 1e-15
    assert np.allclose([dt for _, dt in prog], 0.005 / 1e-3)
    F = prog[0][0].reshape(3, 3)
    assert np.array_equal(F - np.diag(np.diag(F)), np.zeros((3, 3))) and F[0, 0] == F[2, 2] == 1
    with pytest.raises(ValueError):
        I.pulsating_cycle_program(0.02, 7, 1)


def test_stress_mask_and_increment_args():
    m = I.uniaxial_stress_mask(1)
    assert m.tolist() == [1, 0, 0, 0, 0, 0, 0, 0, 1]
    assert I.uniaxial_stress_mask(0).tolist() == [0, 0, 0, 0, 1, 0, 0, 0, 1]
    cfg = I.build_config("poly64_r0", n_override=(4, 4, 4))
    assert np.array_equal(cfg["stress_mask"], m)
    (F0, dt0), kw = I.increment_args(cfg, 0)
    assert np.array_equal(F0, cfg["program"][0][0]) and np.array_equal(kw["stress_mask"], m)
    prev = np.eye(3).reshape(9) + 0.1
    (F1, _), _ = I.increment_args(cfg, 1, prev)
    assert np.array_equal(F1[m == 1], prev[m == 1])
    assert np.array_equal(F1[m == 0], cfg["program"][1][0][m == 0])
    strain = I.build_config("poly64", n_override=(4, 4, 4))
    assert strain["stress_mask"] is None
    (Fs, _), kws = I.increment_args(strain, 0, prev)
    assert kws == {} and np.array_equal(Fs, strain["program"][0][0])


def test_bicrystal_geometry():
    n = (16, 16, 1)
    for b in ("perpendicular", "45"):
        gid, eul = I.bicrystal(n, b, (0, 0, 0), (1, 1, 1))
        g = gid.reshape(16, 16)  # (y, x)
        assert g.sum() == 128 and eul.shape == (2, 3)
    gid, _ = I.bicrystal(n, "perpendicular", (0, 0, 0), (1, 1, 1))
    g = gid.reshape(16, 16)
    assert np.all(g == g[:, :1]) and g[:, 0].tolist() == [0] * 4 + [1] * 8 + [0] * 4
    gid, _ = I.bicrystal(n, "45", (0, 0, 0), (1, 1, 1))
    g = gid.reshape(16, 16)
    assert np.array_equal(g, np.roll(np.roll(g, 1, axis=1), -1, axis=0))  # boundaries along x + y
    with pytest.raises(ValueError):
        I.bicrystal((16, 8, 1), "45", (0, 0, 0), (1, 1, 1))


def test_y111_orientation():
    """EULER_Y111 puts a <111> lattice direction on the sample y axis."""
    Q = O.euler_to_Q(I.EULER_Y111)
    d = Q.T @ np.array([0.0, 1.0, 0.0])
    assert np.allclose(np.abs(d), 1 / np.sqrt(3), atol=1e-15)
    assert np.allclose(O.euler_to_Q(I.EULER_Y100), np.eye(3))


def test_plate_configs():
    for name in ("plate256_sx100", "plate256_sx111", "plate256_bx90", "plate256_bx45",
                 "plate256x128_notch"):
        c = I.build_config(name)
        assert c["n"][2] == 1 and c["stress_mask"] is not None
        assert c["grain_ids"].size == int(np.prod(c["n"]))
    c = I.build_config("plate256_sx100")
    phi = c["phi0"].reshape(256, 256)
    ys, xs = np.nonzero(phi)
    assert (xs.min(), xs.max(), ys.min(), ys.max()) == (96, 159, 127, 128)
    assert np.array_equal(c["elastic_only"], (c["phi0"] > 0).astype(np.uint8))
    c = I.build_config("plate256x128_notch")
    phi = c["phi0"].reshape(128, 256)
    assert np.all(phi[:8] == 1) and np.all(phi[120:] == 1) and np.all(phi[8:120, :100] == 0)
    assert np.all(phi[8:24, 127:129] == 1) and np.all(phi[24:120, 127:129] == 0)
    assert c["stress_mask"].tolist() == [0, 0, 0, 0, 1, 0, 0, 0, 1]
    assert c["program"][0][0][0] > 1.0 and c["program"][0][0][4] == 1.0


@pytest.mark.parametrize("n,grains,sigma", [((96, 96, 1), 40, 0.3), ((32, 32, 32), 40, 0.5)])
def test_lognormal_polycrystal(n, grains, sigma):
    """Log-normal grain sizes (Sec. 4.3, 4.4): every grain present, each
    cell's size within 2 % (or half a voxel) of its log-normal target, the
    measured equivalent diameters carrying the targets' order and log spread,
    and the targets filling the box."""
    from scipy.stats import spearmanr
    gid, eul, d = I.lognormal_polycrystal(n, grains, sigma, 3)
    D = 2 if n[2] == 1 else 3
    unit = np.pi / 4 if D == 2 else np.pi / 6
    h = I.VOXEL_MM
    cnt = np.bincount(gid, minlength=grains)
    target = unit * d ** D / h ** D
    assert gid.size == int(np.prod(n)) and eul.shape == (grains, 3)
    assert np.all(cnt > 0) and np.all(np.abs(cnt - target) <= 0.02 * target + 0.5)
    assert abs(target.sum() - gid.size) < 1e-6 * gid.size
    de = (cnt * h ** D / unit) ** (1.0 / D)
    assert spearmanr(d, de).correlation > 0.99
    assert abs(np.log(de).std() - np.log(d).std()) < 0.02
    g2, e2, d2 = I.lognormal_polycrystal(n, grains, sigma, 3)
    assert np.array_equal(gid, g2) and np.array_equal(eul, e2)


def test_lognormal_configs():
    c = I.build_config("plate256_poly62", n_override=(64, 64, 1))
    assert len(np.unique(c["grain_ids"])) == 62 and c["stress_mask"] is not None
    c = I.build_config("poly128_ln64", n_override=(24, 24, 24))
    assert len(np.unique(c["grain_ids"])) == 64
    assert np.array_equal(c["stress_mask"], I.uniaxial_stress_mask(1))
    eps = np.array([F[4] - 1.0 for F, _ in c["program"]])
    assert abs(eps.max() - 0.02) < 1e-15 and eps.min() >= 0.0


def test_cycle_override_extends_the_loading():
    """build_config(cycles=...) repeats the configuration's cycle: the same
    increments, more of them (plates too)."""
    import numpy as np
    from paper_2304_01125_gb300 import inputs as I
    for name, n in (("poly128_damage", (8, 8, 8)), ("plate256_sx100", (8, 8, 1))):
        base = I.build_config(name, n)
        c = I.CONFIGS[name]
        more = I.build_config(name, n, cycles=c["cycles"] + 2)
        per = c["inc_per_cycle"]
        assert len(more["program"]) == len(base["program"]) + 2 * per
        for (Fa, da), (Fb, db) in zip(base["program"], more["program"]):
            assert np.array_equal(Fa, Fb) and da == db


def test_batch_units_are_one_seeded_sequence():
    """Rank r of a weak-scaled batched run takes units r*count .. (r+1)*count
    - 1 of one seeded sequence (seed + count*r): the same RVEs as the tail
    of a batch twice as long, and none shared between ranks."""
    a = I.batch_configs(seed=2000, count=6, sizes=(8, 12), grains=(2, 5))
    b = I.batch_configs(seed=2006, count=6, sizes=(8, 12), grains=(2, 5))
    both = I.batch_configs(seed=2000, count=12, sizes=(8, 12), grains=(2, 5))
    for x, y in zip(a + b, both):
        assert x["n"] == y["n"]
        assert np.array_equal(x["grain_ids"], y["grain_ids"])
        assert np.array_equal(x["euler"], y["euler"])
    assert not any(np.array_equal(x["euler"], y["euler"]) for x in a for y in b
                   if x["euler"].shape == y["euler"].shape)
