"""Batched RVEs (batch_create / batch_run_increment): uneven grids advanced
concurrently on their own streams give the same bits as each RVE advanced
alone; a failing handle reports its own status without stopping the
others; invalid batches are rejected."""
import numpy as np
import pytest

from paper_2304_01125_gb300 import build as B
from paper_2304_01125_gb300 import fatiguefft as FF
from paper_2304_01125_gb300 import inputs as I

pytestmark = pytest.mark.gpu
H = I.VOXEL_MM
MAT = dict(I.material("baseline"), tau_c0=250.0)
GRIDS = [(8, 8, 8), (10, 8, 6), (12, 10, 8), (6, 6, 6), (9, 7, 5)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    FF.load()


def _make(n, seed, prec, opts=None):
    import torch
    gid, eul = I.voronoi(n, 3, seed)
    return FF.RVE(n, H, gid, eul, MAT, opts or I.solver_options(
        "parity64" if prec == "fp64" else "parity32"), prec=prec, stream=torch.cuda.Stream())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_matches_single_runs(prec):
    prog = I.uniaxial_cycle_program(0.006, 24, 1)[:4]
    batch_rves = [_make(n, 30 + i, prec) for i, n in enumerate(GRIDS)]
    b = FF.Batch(batch_rves, threads=3)
    its = 0
    for Fb, dt in prog:
        s, per, stats = b.run_increment([Fb] * len(GRIDS), [dt] * len(GRIDS))
        assert s == FF.FFT_OK and per == [0] * len(GRIDS)
        its += sum(x["lin_it_total"] for x in stats)
    assert its > 0
    b.close()
    for i, n in enumerate(GRIDS):
        r = _make(n, 30 + i, prec)
        for Fb, dt in prog:
            r.run_increment(Fb, dt)
        for f in ("F", "P", "Fp", "gamma"):
            assert np.array_equal(r.field(f), batch_rves[i].field(f)), (n, f)
        r.close()
    for r in batch_rves:
        r.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_mixed_control_matches_single_runs(prec):
    """batch_run_increment_mixed: three uneven grids under uniaxial stress
    (lateral mean stresses zero), each handle's stress-controlled components
    started from its own previous solved F, give the same bits as each
    handle run alone with run_increment_mixed."""
    grids = GRIDS[:3]
    m = I.uniaxial_stress_mask(1)
    prog = I.uniaxial_cycle_program(0.006, 24, 1)[:4]

    def guesses(prev, Fb):
        return [Fb.copy() if p is None else np.where(m == 1, p, Fb) for p in prev]

    batch_rves = [_make(n, 60 + i, prec) for i, n in enumerate(grids)]
    b = FF.Batch(batch_rves, threads=2)
    prev = [None] * len(grids)
    for Fb, dt in prog:
        s, per, stats = b.run_increment(guesses(prev, Fb), [dt] * len(grids),
                                        stress_masks=[m] * len(grids))
        assert s == FF.FFT_OK and all(x["mixed_it"] >= 1 for x in stats)
        prev = [np.array(x["Fbar"]) for x in stats]
    b.close()
    for i, n in enumerate(grids):
        r = _make(n, 60 + i, prec)
        p = None
        for Fb, dt in prog:
            _, st = r.run_increment(guesses([p], Fb)[0], dt, Pbar=np.zeros(9), stress_mask=m)
            p = np.array(st["Fbar"])
        assert np.array_equal(p, prev[i])
        for f in ("F", "P", "Fp", "gamma"):
            assert np.array_equal(r.field(f), batch_rves[i].field(f)), (n, f)
        r.close()
    for r in batch_rves:
        r.close()


def test_failing_handle_does_not_stop_the_others():
    prog = I.uniaxial_cycle_program(0.004, 8, 1)
    capped = I.solver_options("parity32", max_lin=1, tol_lin=1e-14)
    rves = [_make((8, 8, 8), 41, "mixed"), _make((6, 6, 6), 42, "mixed", opts=capped),
            _make((10, 8, 6), 43, "mixed")]
    b = FF.Batch(rves)
    Fb, dt = prog[0]
    s, per, stats = b.run_increment([Fb] * 3, [dt] * 3, check=False)
    assert s == FF.FFT_ERR_NOT_CONVERGED
    assert per == [FF.FFT_OK, FF.FFT_ERR_NOT_CONVERGED, FF.FFT_OK]
    assert stats[0]["lin_it_total"] > 0 and stats[2]["lin_it_total"] > 0
    assert np.abs(rves[0].field("F").mean(axis=1) - Fb).max() < 1e-7
    b.close()
    for r in rves:
        r.close()


def test_batch_rejects_shared_or_default_streams():
    import torch
    n = (4, 4, 4)
    gid, eul = I.single_crystal(n)
    opts = I.solver_options("paper")
    st = torch.cuda.Stream()
    a = FF.RVE(n, H, gid, eul, MAT, opts, prec="mixed", stream=st)
    c = FF.RVE(n, H, gid, eul, MAT, opts, prec="mixed", stream=st)
    d = FF.RVE(n, H, gid, eul, MAT, opts, prec="mixed")  # legacy default stream
    for group in ([a, c], [a, a], [a, d]):
        with pytest.raises(FF.FFTError):
            FF.Batch(group)
    for r in (a, c, d):
        r.close()


def test_cutback_recovers_a_batch_rve_at_peak_load():
    """One of the batched-workload RVEs (96^3, 43 grains) at the first 0.6 %
    peak: restarted GMRES on the full-step tangent stalls (the plastic
    voxels' rate-dependent tangent is orders softer than the averaged one);
    with max_cutbacks the increment is redone as halves and converges, and
    the macroscopic state is the requested one."""
    import torch
    c = I.CONFIGS["batch32"]
    cfgs = I.batch_configs(seed=c["seed"], count=c["count"], sizes=c["sizes"],
                           grains=c["grains"])
    prog = I.uniaxial_cycle_program(c["amplitude"], c["inc_per_cycle"], c["cycles"])
    x = cfgs[26]
    mat = I.material("baseline")
    res = {}
    for cut in (0, 4):
        r = FF.RVE(x["n"], H, x["grain_ids"], x["euler"], mat,
                   I.solver_options("paper", max_lin=300, max_cutbacks=cut), prec="mixed",
                   stream=torch.cuda.Stream())
        for k in range(7):
            s, st = r.run_increment(*prog[k])
            assert st["cutbacks"] == 0
        Ft_before = r.field("Ft")
        Fb, dt = prog[7]
        s, st = r.run_increment(Fb, dt, check=False)
        res[cut] = (s, st["cutbacks"])
        if cut == 0:
            assert s == FF.FFT_ERR_NOT_CONVERGED
            assert np.array_equal(r.field("Ft"), Ft_before)  # nothing committed
        else:
            assert s == FF.FFT_OK and st["cutbacks"] >= 1
            F = r.field("F")
            assert np.abs(F.mean(axis=1) - Fb).max() < 1e-7
            assert np.array_equal(r.field("Ft"), F)
        r.close()


def test_cutback_under_mixed_control_matches_oracle():
    """Cut-back under mixed control (uniaxial stress): a single 0.6 % step
    from rest that Newton cannot take whole (max_newton 6, at most 100
    Krylov iterations per solve) is redone as halves; the FP64 path takes the
    same halvings as the oracle and reaches its solved macroscopic F and
    fields, the mixed path converges through halvings with the lateral
    stresses held."""
    import torch
    import oracle as O
    n = (6, 6, 6)
    gid, eul = I.voronoi(n, 3, 11)
    mat = dict(I.material("baseline"), tau_c0=250.0)
    m = I.uniaxial_stress_mask(1)
    Fb, dt = I.uniaxial_cycle_program(0.006, 4, 1)[0]
    opts = I.solver_options("paper", max_newton=6, max_lin=100, max_cutbacks=3)
    o = O.RVE(n, H, gid, eul, mat, opts)
    so, sto = o.run_increment(Fb, dt, Pbar=np.zeros(9), stress_mask=m)
    assert so == 0 and sto["cutbacks"] >= 1
    for prec in ("fp64", "mixed"):
        r = FF.RVE(n, H, gid, eul, mat, opts, prec=prec, stream=torch.cuda.Stream())
        s, st = r.run_increment(Fb, dt, Pbar=np.zeros(9), stress_mask=m)
        assert s == FF.FFT_OK and st["cutbacks"] >= 1
        P = np.array(st["Pbar"])
        assert np.abs(P[m == 1]).max() <= 1.01 * opts["tol_newton"] * np.abs(P).max()
        if prec == "fp64":
            assert st["cutbacks"] == sto["cutbacks"]
            assert np.abs(np.array(st["Fbar"]) - np.array(sto["Fbar"])).max() < 1e-9
            for f in ("F", "P", "Fp"):
                a, b = r.field(f), o.field(f)
                assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(b), f
        r.close()


def test_cutback_with_a_changing_stress_target_matches_oracle():
    """Cut-back under mixed control when the stress target moves between
    increments (lateral stresses 0 -> -40 MPa with a step from 0.3 to
    0.7 %): each half takes half of the stress change; the FP64 path takes
    the oracle's halvings and reaches its solved macroscopic F and fields."""
    import torch
    import oracle as O
    n = (6, 6, 6)
    gid, eul = I.voronoi(n, 3, 11)
    mat = dict(I.material("baseline"), tau_c0=250.0)
    m = I.uniaxial_stress_mask(1)
    prog = I.uniaxial_cycle_program(0.006, 8, 1)
    P1 = np.zeros(9)
    P1[0] = P1[8] = -40.0
    Fb = prog[1][0].copy()
    Fb[4] += 0.001
    opts = I.solver_options("paper", max_newton=10, max_lin=100, max_cutbacks=3)
    o = O.RVE(n, H, gid, eul, mat, opts)
    r = FF.RVE(n, H, gid, eul, mat, opts, prec="fp64", stream=torch.cuda.Stream())
    res = []
    for h in (o, r):
        s, st = h.run_increment(prog[0][0], prog[0][1], Pbar=np.zeros(9), stress_mask=m)
        assert s == 0
        guess = np.where(m == 1, np.array(st["Fbar"]), Fb)
        s, st = h.run_increment(guess, 4.0, Pbar=P1, stress_mask=m)
        assert s == 0 and st["cutbacks"] >= 1
        res.append(st)
    assert res[0]["cutbacks"] == res[1]["cutbacks"]
    assert np.abs(np.array(res[0]["Fbar"]) - np.array(res[1]["Fbar"])).max() < 1e-9
    for f in ("F", "P", "Fp"):
        a, b = r.field(f), o.field(f)
        assert np.linalg.norm(a - b) <= 1e-8 * np.linalg.norm(b), f
    r.close()


def test_bounded_wait_gives_up_on_a_barrier_nothing_completes():
    """The pipelined update pass's mbarrier waits are bounded: on a barrier
    that no copy completes, the wait returns after its round limit (and the
    context stays usable: a solve runs afterwards)."""
    import time
    L = FF.load()
    t0 = time.time()
    assert L.fft_selftest_bounded_wait(256) == 1
    assert time.time() - t0 < 30
    assert L.fft_selftest_bounded_wait(0) == -2
    r = _make((6, 6, 6), 5, "mixed")
    s, _ = r.run_increment(*I.uniaxial_cycle_program(0.004, 8, 1)[0])
    assert s == FF.FFT_OK
    r.close()


# ------------------------------------------------------------ lockstep classes
def _same_as_alone(batch_rves, make, prog, fields=("F", "P", "Fp", "gamma")):
    """Each batch handle against a fresh handle run alone through prog:
    the same status, iteration counts and field bits."""
    out = []
    for i, br in enumerate(batch_rves):
        r = make(i)
        sts = []
        for Fb, dt in prog:
            s, st = r.run_increment(Fb, dt, check=False)
            sts.append((s, st["newton_it"], st["lin_it_total"], st["stag_it"],
                        st["pf_it_total"], st["cutbacks"]))
        out.append(sts)
        for f in fields:
            assert np.array_equal(r.field(f), br.field(f)), (i, f)
        r.close()
    return out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_lockstep_class_matches_single_runs(prec):
    """Four handles of one grid form a lockstep class (one graph launch per
    Krylov column for all four, one batched transform per direction), a
    fifth of another grid runs on its own: every handle's iteration counts
    and fields are those of the handle run alone, bit for bit."""
    prog = I.uniaxial_cycle_program(0.006, 24, 1)[:4]
    grids = [(12, 10, 8)] * 4 + [(8, 8, 8)]
    make = lambda i: _make(grids[i], 70 + i, prec)  # noqa: E731
    rves = [make(i) for i in range(len(grids))]
    b = FF.Batch(rves, threads=2)
    got = [[] for _ in rves]
    for Fb, dt in prog:
        s, per, stats = b.run_increment([Fb] * len(rves), [dt] * len(rves))
        assert s == FF.FFT_OK
        for i, st in enumerate(stats):
            got[i].append((per[i], st["newton_it"], st["lin_it_total"], st["stag_it"],
                           st["pf_it_total"], st["cutbacks"]))
    cls = b.classes()
    assert len(cls) == 1 and cls[0][0] == 4 and cls[0][1] > 0, cls
    b.close()
    assert sum(x[2] for x in got[0]) > 0
    assert _same_as_alone(rves, make, prog) == got
    for r in rves:
        r.close()


def test_lockstep_class_without_classes_flag():
    """classes=False forms no class: the same handles run one by one."""
    grids = [(8, 8, 8)] * 3
    rves = [_make(n, 80 + i, "mixed") for i, n in enumerate(grids)]
    b = FF.Batch(rves, classes=False)
    assert b.classes() == []
    Fb, dt = I.uniaxial_cycle_program(0.004, 8, 1)[0]
    s, per, _ = b.run_increment([Fb] * 3, [dt] * 3)
    assert s == FF.FFT_OK
    b.close()
    for r in rves:
        r.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_lockstep_class_through_crack_growth(prec):
    """Three 12^3 polycrystals (the damaged-regime workload of the damage
    parity test, three seeds) as one lockstep class through damage
    nucleation and unstable growth (30 increments, up to tens of staggered
    iterations per increment, members leaving the staggered loop at
    different iterations): statuses, iteration counts (Newton, GMRES,
    staggered, phase-field) and the damage and stress fields equal those of
    each handle run alone."""
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "make_damage12", os.path.join(os.path.dirname(__file__), "golden", "make_damage12.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    import torch
    _, _, mat, prog, opts = mod.setup()

    def make(i):
        gid, eul = I.voronoi(mod.N_GRID, 4, 31 + i)
        return FF.RVE(mod.N_GRID, H, gid, eul, mat, opts, prec=prec, stream=torch.cuda.Stream())

    rves = [make(i) for i in range(3)]
    b = FF.Batch(rves, threads=1)
    got = [[] for _ in rves]
    for Fb, dt in prog:
        s, per, stats = b.run_increment([Fb] * 3, [dt] * 3, check=False)
        for i, st in enumerate(stats):
            got[i].append((per[i], st["newton_it"], st["lin_it_total"], st["stag_it"],
                           st["pf_it_total"], st["cutbacks"]))
    assert b.classes()[0][0] == 3
    b.close()
    assert max(x[4] for x in got[0]) > 0  # the phase field was solved
    assert _same_as_alone(rves, make, prog, fields=("phi", "P", "F")) == got
    for r in rves:
        r.close()


def test_lockstep_class_cuts_back_a_member():
    """Two 96^3 batched-workload RVEs as a class through the first 0.6 %
    peak, where one needs a cut-back (max_lin 300): that member is cut back
    on its own after the lockstep attempt, and both end as when run alone."""
    import torch
    c = I.CONFIGS["batch32"]
    cfgs = I.batch_configs(seed=c["seed"], count=c["count"], sizes=c["sizes"],
                           grains=c["grains"])
    prog = I.uniaxial_cycle_program(c["amplitude"], c["inc_per_cycle"], c["cycles"])[:8]
    pick = [26] + [i for i, x in enumerate(cfgs) if x["n"] == cfgs[26]["n"] and i != 26][:1]
    opts = I.solver_options("paper", max_lin=300, max_cutbacks=4)
    mat = I.material("baseline")

    def make(i):
        x = cfgs[pick[i]]
        return FF.RVE(x["n"], H, x["grain_ids"], x["euler"], mat, opts, prec="mixed",
                      stream=torch.cuda.Stream())

    rves = [make(i) for i in range(2)]
    b = FF.Batch(rves, classes="all")
    got = [[] for _ in rves]
    for Fb, dt in prog:
        s, per, stats = b.run_increment([Fb] * 2, [dt] * 2)
        for i, st in enumerate(stats):
            got[i].append((per[i], st["newton_it"], st["lin_it_total"], st["stag_it"],
                           st["pf_it_total"], st["cutbacks"]))
    assert b.classes()[0][0] == 2
    b.close()
    assert sum(x[5] for x in got[0]) >= 1  # the cut-back happened
    assert _same_as_alone(rves, make, prog) == got
    for r in rves:
        r.close()


def test_a_handle_joins_one_batch_at_a_time():
    """A lockstep class takes over its members' Arnoldi scratch while its
    batch exists: a handle in a live batch is refused by another batch
    (FFT_ERR_ARG, nothing changed) and not released by rve_destroy, and is
    accepted again once the first batch is closed."""
    a, c = _make((8, 8, 8), 70, "mixed"), _make((8, 8, 8), 71, "mixed")
    b1 = FF.Batch([a, c])
    for group in ([a], [c, a]):
        with pytest.raises(FF.FFTError):
            FF.Batch(group)
    # destroying a handle that is still in a batch leaves it alive
    FF.load().rve_destroy(a._h)
    assert b"still in a batch" in FF.load().fft_last_error(a._h)
    Fb, dt = I.uniaxial_cycle_program(0.004, 8, 1)[0]
    s, _, _ = b1.run_increment([Fb] * 2, [dt] * 2)
    assert s == FF.FFT_OK
    b1.close()
    b2 = FF.Batch([c, a])
    Fb, dt = I.uniaxial_cycle_program(0.004, 8, 1)[1]
    s, _, _ = b2.run_increment([Fb] * 2, [dt] * 2)
    assert s == FF.FFT_OK
    b2.close()
    a.close()
    c.close()


def test_closing_a_class_member_closes_its_batch_first():
    """A lockstep class keeps part of its members' buffers in its arenas:
    closing a member handle closes the batch first (the binding keeps that
    order), after which the other members run on their own."""
    grids = [(8, 8, 8)] * 3
    rves = [_make(n, 90 + i, "mixed") for i, n in enumerate(grids)]
    b = FF.Batch(rves)
    assert b.classes()[0][0] == 3
    Fb, dt = I.uniaxial_cycle_program(0.004, 8, 1)[0]
    s, _, _ = b.run_increment([Fb] * 3, [dt] * 3)
    assert s == FF.FFT_OK
    rves[0].close()
    assert b._h is None
    for r in rves[1:]:
        s, st = r.run_increment(*I.uniaxial_cycle_program(0.004, 8, 1)[1])
        assert s == FF.FFT_OK and st["lin_it_total"] >= 0
        r.close()


@pytest.mark.parametrize("prec,grid", [("fp64", (10, 8, 6)), ("mixed", (10, 8, 6)),
                                       ("mixed", (16, 16, 1))])
def test_lockstep_class_under_mixed_control(prec, grid):
    """batch_run_increment_mixed with the handles in one lockstep class (three
    polycrystals of one grid under uniaxial stress, the lateral mean stresses
    zero; a 16 x 16 x 1 grid is a set of plates under plane stress): the
    outer mixed-control rounds run in lockstep too, and every handle's solved
    F, statistics and fields equal those of the handle run alone with
    run_increment_mixed."""
    m = I.uniaxial_stress_mask(1)
    prog = I.uniaxial_cycle_program(0.006, 24, 1)[:4]

    def guesses(prev, Fb):
        return [Fb.copy() if p is None else np.where(m == 1, p, Fb) for p in prev]

    rves = [_make(grid, 100 + i, prec) for i in range(3)]
    b = FF.Batch(rves, threads=2)
    assert b.classes()[0][0] == 3
    prev = [None] * 3
    got = [[] for _ in rves]
    for Fb, dt in prog:
        s, per, stats = b.run_increment(guesses(prev, Fb), [dt] * 3, stress_masks=[m] * 3)
        assert s == FF.FFT_OK and all(x["mixed_it"] >= 1 for x in stats)
        prev = [np.array(x["Fbar"]) for x in stats]
        for i, x in enumerate(stats):
            got[i].append((x["newton_it"], x["lin_it_total"], x["mixed_it"], x["stag_it"]))
    b.close()
    for i in range(3):
        r = _make(grid, 100 + i, prec)
        p = None
        mine = []
        for Fb, dt in prog:
            _, st = r.run_increment(guesses([p], Fb)[0], dt, Pbar=np.zeros(9), stress_mask=m)
            p = np.array(st["Fbar"])
            mine.append((st["newton_it"], st["lin_it_total"], st["mixed_it"], st["stag_it"]))
        assert mine == got[i] and np.array_equal(p, prev[i])
        for f in ("F", "P", "Fp", "gamma"):
            assert np.array_equal(r.field(f), rves[i].field(f)), (i, f)
        r.close()
    for r in rves:
        r.close()
