"""Pins of the FP64 CPU oracle against facts fixed by the paper and by the
mathematics (closed forms, brute force, library routines, invariants).

Each test names the passage it pins.  None of them compares the oracle with
itself or retypes one of its formulas: they use an independent route to the
same number, chosen so that a dropped term, a wrong sign, a transposed operand
or a mis-scaled frequency fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2304_01125_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")
MAT = I.material("baseline")
H = I.VOXEL_MM


def cubic_voigt(m):
    C = np.zeros((6, 6))
    C[:3, :3] = m["C12"]
    for i in range(3):
        C[i, i] = m["C11"]
        C[3 + i, 3 + i] = m["C44"]
    return C


def cubic_apply_np(m, E):
    """S = C : E for the cubic lattice tensor, through the 6x6 Voigt matrix
    with engineering shear strains (independent of the oracle's routine)."""
    e = np.array([E[0, 0], E[1, 1], E[2, 2], 2 * E[1, 2], 2 * E[0, 2], 2 * E[0, 1]])
    s = cubic_voigt(m) @ e
    return np.array([[s[0], s[5], s[4]], [s[5], s[1], s[3]], [s[4], s[3], s[2]]])


# --------------------------------------------------------------------- P6
@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 3, 3), (6, 6, 6), (1, 1, 48), (1, 96, 1),
                                   (5, 3, 2)])
def test_fft_matches_numpy_and_naive_dft(shape):
    """Sec. 3.1: the DFT of a voxel field computed by an FFT.  The oracle's
    own FFT equals numpy's FFT and its own naive DFT; inverse is 1/N."""
    rng = np.random.default_rng(sum(shape))
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    f = O.fft3d(a, -1)
    ref = np.fft.fftn(a)
    tol = 1e-12 * np.abs(ref).max()
    assert np.abs(f - ref).max() < tol
    if np.prod(shape) <= 512:
        assert np.abs(O.fft3d(a, -1, naive=True) - ref).max() < tol
    assert np.abs(O.fft3d(f, +1) - a).max() < 1e-13 * np.abs(a).max() * 10


def test_fft_parseval():
    rng = np.random.default_rng(0)
    a = rng.standard_normal((6, 4, 8))
    f = O.fft3d(a.astype(complex), -1)
    assert abs((np.abs(f) ** 2).sum() / a.size - (a ** 2).sum()) < 1e-10 * (a ** 2).sum()


# --------------------------------------------------------------- tables
def test_material_preset_is_table1():
    """Table 1 and Sec. 4 values, from the committed fixture."""
    t = json.load(open(os.path.join(GOLD, "table1_cmsx4.json")))
    m = I.material("paper")
    assert m["C11"] == t["C11_GPa"] * 1e3 and m["C12"] == t["C12_GPa"] * 1e3
    assert m["C44"] == t["C44_GPa"] * 1e3 and m["tau_c0"] == t["tau_c0_MPa"]
    assert m["b"] == t["b_mm"] and m["nu_D"] == t["nu_D_per_s"]
    assert m["k_B"] == t["k_J_per_K"] and m["dF"] == t["dF_J"]
    assert m["rho_m"] == t["rho_m_per_mm2"] and m["lambda_h"] == t["lambda_per_mm2"]
    assert m["T"] == t["T_K"] and m["k_res"] == t["k_residual"]
    assert abs(m["G_crit"] - t["G_crit_J_per_m2"] * 1e-3) < 1e-15  # J/m^2 -> N/mm
    assert abs(m["ell"] - t["ell_um"] * 1e-3) < 1e-15
    assert abs(m["ell_Fp"] - t["ell_Fp_um"] * 1e-3) < 1e-15
    assert abs(I.VOXEL_MM - t["voxel_um"] * 1e-3) < 1e-15


def test_fcc_slip_systems():
    """Sec. 2.1: N_s = 12 FCC {111}<110> systems (textbook set, unordered).
    A system is identified by its Schmid dyad s (x) n up to sign."""
    def canon(sv, nv):
        P = np.outer(sv / np.linalg.norm(sv), nv / np.linalg.norm(nv)).reshape(9)
        k = np.nonzero(np.abs(P) > 1e-9)[0][0]
        return tuple(np.round(P * np.sign(P[k]), 9))

    s, n = O.fcc_systems()
    ref = np.loadtxt(os.path.join(GOLD, "fcc_111_110.txt"))
    want = {canon(row[3:], row[:3]) for row in ref}
    got = set()
    for a in range(12):
        assert abs(np.linalg.norm(s[a]) - 1) < 1e-15 and abs(np.linalg.norm(n[a]) - 1) < 1e-15
        assert abs(s[a] @ n[a]) < 1e-15
        got.add(canon(s[a], n[a]))
    assert got == want and len(got) == 12


def test_euler_rotation_is_bunge():
    """Bunge z-x-z: (phi1, 0, 0) is a rotation about z; Q is proper orthogonal;
    Q(phi1, Phi, phi2) composes three elementary rotations."""
    def rz(a):
        c, s = np.cos(a), np.sin(a)
        return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])

    def rx(a):
        c, s = np.cos(a), np.sin(a)
        return np.array([[1.0, 0, 0], [0, c, -s], [0, s, c]])

    e = np.array([0.4, 1.1, -0.7])
    Q = O.euler_to_Q(e)
    # active rotation lattice -> sample: Rz(phi1) Rx(Phi) Rz(phi2)
    assert np.abs(Q - rz(e[0]) @ rx(e[1]) @ rz(e[2])).max() < 1e-15
    assert abs(np.linalg.det(Q) - 1) < 1e-14


# ------------------------------------------------------------------ P2
def test_elastic_uniaxial_closed_form():
    """Sec. 2.1 with the elastic reading S = C:E: a [100] crystal under
    F = I + eps e2 (x) e2 below yield gives E22 = ((1+eps)^2-1)/2,
    S22 = C11 E22, S11 = S33 = C12 E22, P22 = (1+eps) S22, and the tensile
    energy of Eq. decMiehe is 1/2 C11 ln(1+eps)^2 (0 in compression)."""
    for eps in (0.004, -0.004):
        F = np.eye(3)
        F[1, 1] += eps
        r = O.cp_point(MAT, np.eye(3), F, np.eye(3), MAT["rho_ssd0"], 0.0, 1.0)
        E = ((1 + eps) ** 2 - 1) / 2
        assert r["fail"] == 0 and np.all(r["dgamma"] == 0)
        assert abs(r["P"][1, 1] - (1 + eps) * MAT["C11"] * E) < 1e-9
        assert abs(r["P"][0, 0] - MAT["C12"] * E) < 1e-9
        assert abs(r["P"][2, 2] - MAT["C12"] * E) < 1e-9
        assert np.abs(r["P"] - np.diag(np.diag(r["P"]))).max() < 1e-12
        we = 0.5 * MAT["C11"] * np.log(1 + eps) ** 2 if eps > 0 else 0.0
        assert abs(r["We_plus"] - we) < 1e-12


def test_elastic_simple_shear_closed_form():
    """Sec. 2.1 with S = C:E and tensor (not engineering) shear strains: a
    [100] crystal under F = I + g e1 (x) e2 below yield has E12 = E21 = g/2,
    E22 = g^2/2, so S12 = 2 C44 E12 = C44 g, S22 = C11 g^2/2, S11 = S33 =
    C12 g^2/2, and P = F S."""
    g = 2e-3
    F = np.eye(3)
    F[0, 1] = g
    r = O.cp_point(MAT, np.eye(3), F, np.eye(3), MAT["rho_ssd0"], 0.0, 1.0)
    assert r["fail"] == 0 and np.all(r["dgamma"] == 0)
    E22 = g * g / 2
    S = np.array([[MAT["C12"] * E22, MAT["C44"] * g, 0.0],
                  [MAT["C44"] * g, MAT["C11"] * E22, 0.0],
                  [0.0, 0.0, MAT["C12"] * E22]])
    assert np.abs(r["P"] - F @ S).max() < 1e-9


def test_elastic_rotated_crystal_frame_covariance():
    """Sec. 2.1: rotating the crystal and the loading together leaves the
    response unchanged (P rotates with Q)."""
    rng = np.random.default_rng(5)
    Q = O.euler_to_Q(rng.random(3) * 3)
    F0 = np.eye(3) + 1e-3 * rng.standard_normal((3, 3))
    r0 = O.cp_point(MAT, np.eye(3), F0, np.eye(3), MAT["rho_ssd0"], 0.0, 1.0)
    r1 = O.cp_point(MAT, Q, Q @ F0 @ Q.T, np.eye(3), MAT["rho_ssd0"], 0.0, 1.0)
    assert np.abs(Q @ r0["P"] @ Q.T - r1["P"]).max() < 1e-9


# ------------------------------------------------------------------ P3
def _single_slip_case(dt):
    """A lattice-frame simple shear along system 0 with tau_c between the
    largest and the second largest trial resolved shear, so only system 0
    slips."""
    s, n = O.fcc_systems()
    Fgrad = 4e-3 * np.outer(s[0], n[0])
    F = np.eye(3) + Fgrad
    E = 0.5 * (F.T @ F - np.eye(3))
    S = cubic_apply_np(MAT, E)
    tau = np.array([s[a] @ S @ n[a] for a in range(12)])
    order = np.argsort(-np.abs(tau))
    assert order[0] == 0
    tc = 0.5 * (abs(tau[0]) + abs(tau[order[1]]))
    m = dict(MAT, tau_c0=tc, mu=0.0)  # tau_c = tc exactly
    return m, F, s, n, tc


@pytest.mark.parametrize("dt", [0.05, 1.0, 30.0])
def test_single_slip_by_bisection(dt):
    """Eq. flowrule with one active system reduces to one scalar equation
    dg = dt g0 sinh((tau(dg) - tau_c)/sT), tau(dg) = s.S(dg).n, S = C:E_e,
    E_e = (Fe^T Fe - I)/2, Fe = F (I - dg s(x)n).  Solved here by bisection."""
    m, F, s, n, tc = _single_slip_case(dt)
    kT = m["k_B"] * m["T"]
    g0 = m["rho_m"] * m["b"] ** 2 * m["nu_D"] * np.exp(-m["dF"] / kT)
    sT = kT / (m["dV"] * 1e-3)
    P0 = np.outer(s[0], n[0])

    def tau_of(dg):
        Fe = F @ (np.eye(3) - dg * P0)
        S = cubic_apply_np(m, 0.5 * (Fe.T @ Fe - np.eye(3)))
        return s[0] @ S @ n[0]

    def f(dg):
        return dg - dt * g0 * np.sinh((tau_of(dg) - tc) / sT)

    lo, hi = 0.0, 0.01
    assert f(lo) < 0 < f(hi)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) < 0:
            lo = mid
        else:
            hi = mid
    dg_ref = 0.5 * (lo + hi)
    r = O.cp_point(m, np.eye(3), F, np.eye(3), 0.0, 0.0, dt, tol_local=1e-10)
    assert r["fail"] == 0
    assert abs(r["dgamma"][0] - dg_ref) < 1e-12 + 1e-9 * dg_ref
    assert np.all(r["dgamma"][1:] == 0)
    assert np.all(np.abs(r["tau"][1:]) <= tc)
    # plastic work increment and SSD increment of Sec. 2.1/2.3
    assert abs(r["dWp"] - tau_of(dg_ref) * dg_ref) < 1e-9 * abs(r["dWp"]) + 1e-14
    Lp = dg_ref * P0
    assert abs(r["drho_ssd"] - m["lambda_h"] * np.sqrt(2 / 3 * np.sum(Lp * Lp))) < \
        1e-8 * r["drho_ssd"]


def test_slip_rate_limits():
    """Rate dependence of Eq. flowrule: slip grows with the step and vanishes
    with it (monotone in dt); a long
    step relaxes the resolved shear to tau_c + sT*asinh(dg/(dt g0))."""
    m, F, s, n, tc = _single_slip_case(1.0)
    dgs = [O.cp_point(m, np.eye(3), F, np.eye(3), 0.0, 0.0, dt)["dgamma"][0]
           for dt in (1e-30, 1e-12, 1e-3, 1.0)]
    assert dgs[0] < 1e-15 and all(a < b for a, b in zip(dgs, dgs[1:]))
    r = O.cp_point(m, np.eye(3), F, np.eye(3), 0.0, 0.0, 1e4)
    kT = m["k_B"] * m["T"]
    g0 = m["rho_m"] * m["b"] ** 2 * m["nu_D"] * np.exp(-m["dF"] / kT)
    sT = kT / (m["dV"] * 1e-3)
    over = r["tau"][0] - tc
    assert 0 < over < 1e-3 and abs(over - sT * np.arcsinh(r["dgamma"][0] / (1e4 * g0))) < 1e-9


def test_elastic_only_voxel_does_not_slip():
    """Pre-crack voxels (Sec. 4.1 soft elastic region) never slip."""
    m, F, s, n, tc = _single_slip_case(1.0)
    r = O.cp_point(m, np.eye(3), F, np.eye(3), 0.0, 0.0, 1.0, elastic_only=True)
    assert np.all(r["dgamma"] == 0)


# ----------------------------------------------------------------- P11
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_tangent_matches_finite_differences(seed):
    """Eq. newton needs K = dP/dF (consistent tangent): compare with central
    differences of P in plastic states (several active systems)."""
    rng = np.random.default_rng(seed)
    Q = O.euler_to_Q(rng.random(3) * 3)
    F = np.eye(3) + 0.004 * rng.standard_normal((3, 3))
    FpL = np.eye(3) + 0.001 * rng.standard_normal((3, 3))
    args = (MAT, Q)
    r = O.cp_point(*args, F, FpL, MAT["rho_ssd0"], 1e5, 1.0, tol_local=1e-10)
    assert r["fail"] == 0
    d = 1e-7
    Kfd = np.zeros((9, 9))
    for c in range(9):
        Fp = F.reshape(9).copy()
        Fm = F.reshape(9).copy()
        Fp[c] += d
        Fm[c] -= d
        Pp = O.cp_point(*args, Fp, FpL, MAT["rho_ssd0"], 1e5, 1.0, tol_local=1e-10,
                        tangent=False)
        Pm = O.cp_point(*args, Fm, FpL, MAT["rho_ssd0"], 1e5, 1.0, tol_local=1e-10,
                        tangent=False)
        Kfd[:, c] = (Pp["P"] - Pm["P"]).reshape(9) / (2 * d)
    assert np.abs(r["K"] - Kfd).max() < 1e-6 * np.abs(Kfd).max()


def test_local_solve_robust_on_extreme_states():
    """The local update converges from large trial overstress (many systems
    active), and its solution satisfies the slip law on every system."""
    rng = np.random.default_rng(3)
    kT = MAT["k_B"] * MAT["T"]
    g0 = MAT["rho_m"] * MAT["b"] ** 2 * MAT["nu_D"] * np.exp(-MAT["dF"] / kT)
    sT = kT / (MAT["dV"] * 1e-3)
    for _ in range(60):
        Q = O.euler_to_Q(I.random_orientations(rng, 1)[0])
        F = np.eye(3) + 0.01 * rng.standard_normal((3, 3))
        FpL = np.eye(3) + 0.003 * rng.standard_normal((3, 3))
        dt = float(rng.choice([0.1, 1.0, 20.0]))
        r = O.cp_point(MAT, Q, F, FpL, MAT["rho_ssd0"], 1e5, dt, tol_local=1e-9,
                       tangent=False)
        assert r["fail"] == 0
        for a in range(12):
            over = abs(r["tau"][a]) - r["tau_c"]
            if r["dgamma"][a] == 0:
                assert over <= 1e-7
            else:
                # slip law (Eq. flowrule) holds to the local tolerance in stress
                assert np.sign(r["dgamma"][a]) == np.sign(r["tau"][a])
                inv = sT * np.arcsinh(abs(r["dgamma"][a]) / (dt * g0))
                assert abs(over - inv) < 1e-8


def test_local_solve_matches_an_independent_solver():
    local_solve_check()


def local_solve_check():
    """Sec. 2.1, Eqs. flowrule and the multiplicative split: the local slip
    problem restated here from the paper (F_p^-1 = F_pn^-1 (I - sum dg s(x)n),
    F_e = F F_p^-1 in the lattice frame, S = C : (F_e^T F_e - I)/2 through the
    Voigt matrix, tau = S : s(x)n, |tau| - tau_c = sT asinh(|dg| / (dt g0))
    on slipping systems, |tau| <= tau_c on the others) and solved by another
    method -- continuation in the time step from a nearly elastic 1e-4 dt up
    to dt, each stage by the library's Powell hybrid root finder on all 12
    systems at once (no active set, no line search) -- gives the oracle's
    slips on generic multi-slip states (2 to 8 systems slipping) to 1e-10;
    the oracle's stress and plastic deformation follow from its slips by
    the same restated equations."""
    so = pytest.importorskip("scipy.optimize")
    mat = dict(MAT, tau_c0=150.0)
    s, n = O.fcc_systems()
    kT = mat["k_B"] * mat["T"]
    g0 = mat["rho_m"] * mat["b"] ** 2 * mat["nu_D"] * np.exp(-mat["dF"] / kT)
    sT = kT / (mat["dV"] * 1e-3)
    rng = np.random.default_rng(5)
    nact = set()
    for _ in range(16):
        Q = O.euler_to_Q(I.random_orientations(rng, 1)[0])
        e = 0.004 * (1 + rng.random())
        F = np.diag([1 - 0.3 * e, 1 + e, 1 - 0.3 * e]) + 0.0005 * rng.standard_normal((3, 3))
        FpL = np.eye(3) + 0.002 * rng.standard_normal((3, 3))
        dt = float(rng.choice([0.1, 1.0, 10.0]))
        r = O.cp_point(mat, Q, F, FpL, mat["rho_ssd0"], 1e5, dt, tol_local=1e-9, tangent=False)
        assert r["fail"] == 0
        tc = mat["tau_c0"] + mat["mu"] * mat["b"] * np.sqrt(mat["rho_ssd0"] + 1e5)
        assert abs(r["tau_c"] - tc) < 1e-12 * tc
        FL = Q.T @ F @ Q
        A = np.linalg.inv(FpL)

        def state(dg):
            Fpi = A @ (np.eye(3) - sum(dg[a] * np.outer(s[a], n[a]) for a in range(12)))
            Fe = FL @ Fpi
            S = cubic_apply_np(mat, 0.5 * (Fe.T @ Fe - np.eye(3)))
            return np.array([s[a] @ S @ n[a] for a in range(12)]), Fe, S, Fpi

        def res(dg, d):
            tau = state(dg)[0]
            return sT * np.arcsinh(dg / (d * g0)) - np.sign(tau) * np.maximum(np.abs(tau) - tc, 0)

        x = np.zeros(12)
        for d in np.geomspace(dt * 1e-4, dt, 41):
            x = so.root(lambda z: res(z, d), x, method="hybr", options=dict(xtol=1e-15)).x
        assert np.abs(res(x, dt)).max() < 1e-9  # MPa: a root of the restated problem
        ref = np.abs(x).max()
        assert ref > 0 and np.abs(r["dgamma"] - x).max() < 1e-10 * ref
        nact.add(int(np.sum(r["dgamma"] != 0)))
        tau, Fe, S, Fpi = state(r["dgamma"])
        assert np.abs(tau - r["tau"]).max() < 1e-9 * np.abs(tau).max()
        P = Q @ (Fe @ S @ Fpi.T) @ Q.T
        assert np.abs(P - r["P"]).max() < 1e-10 * np.abs(P).max()
        assert np.abs(np.linalg.inv(Fpi) - r["Fp_L"]).max() < 1e-12
    assert min(nact) <= 3 and max(nact) >= 6


# ----------------------------------------------------------------- P13
def test_eigen_split_degenerate_and_rotated():
    """Eq. decMiehe: eps+ from the eigen-decomposition of 1/2 ln(Fe Fe^T),
    including repeated eigenvalues; the Jacobi routine reproduces a known
    spectrum in a rotated basis."""
    a, b = 3e-3, -2e-3
    Fe = np.diag([1 + a, 1 + a, 1 + b])
    ep = np.diag([np.log(1 + a), np.log(1 + a), 0.0])
    we = 0.5 * np.sum(ep * cubic_apply_np(MAT, ep))
    assert abs(O.we_plus(MAT, Fe) - we) < 1e-12 * we
    rng = np.random.default_rng(2)
    R = O.euler_to_Q(rng.random(3) * 3)
    D = np.array([0.3, 0.3, -1.2])
    w, V = O.sym_eig3(R @ np.diag(D) @ R.T)
    assert np.abs(np.sort(w) - np.sort(D)).max() < 1e-14
    assert np.abs(V @ np.diag(w) @ V.T - R @ np.diag(D) @ R.T).max() < 1e-14
    assert O.we_plus(MAT, np.diag([1 - a, 1 + b, 1 - a])) == 0.0


def test_we_plus_generic_state_numpy():
    """Eq. decMiehe at generic elastic states F_e = R U (a finite lattice
    rotation R, a stretch U with eigenvalues either side of 1): eps =
    1/2 ln(F_e F_e^T) from NumPy's eigh, eps+ its positive spectral part and
    W_e+ = 1/2 eps+ : C : eps+ with the cubic Voigt matrix.  With a finite R
    the left (F_e F_e^T) and right (F_e^T F_e) stretches give different
    energies in the anisotropic crystal, so the pin fixes the left one."""
    rng = np.random.default_rng(11)
    for _ in range(8):
        R = O.euler_to_Q(rng.random(3) * 3)
        W = O.euler_to_Q(rng.random(3) * 3)
        d = np.array([0.004, -0.002, 0.004 * (2 * rng.random() - 1)])
        Fe = R @ W @ np.diag(1 + d) @ W.T
        lam, V = np.linalg.eigh(Fe @ Fe.T)
        e = 0.5 * np.log(lam)
        assert e.min() < 0 < e.max()
        ep = V @ np.diag(np.maximum(e, 0)) @ V.T
        we = 0.5 * np.sum(ep * cubic_apply_np(MAT, ep))
        assert abs(O.we_plus(MAT, Fe) - we) < 1e-10 * we
        # the right stretch's energy differs: the pin tells them apart
        lam_r, V_r = np.linalg.eigh(Fe.T @ Fe)
        ep_r = V_r @ np.diag(np.maximum(0.5 * np.log(lam_r), 0)) @ V_r.T
        assert abs(0.5 * np.sum(ep_r * cubic_apply_np(MAT, ep_r)) - we) > 1e-4 * we


# ------------------------------------------------------------------ P5
def test_green_operator_identities():
    """Eq. precf with Eq. avstiff: M(xi)(xi.K.xi) = I, and the projection
    Gamma_ijkl = xi_j M_ik xi_l is idempotent under K: Gamma:K:Gamma = Gamma;
    M = 0 at xi = 0."""
    rng = np.random.default_rng(4)
    A = rng.standard_normal((9, 9))
    K = A @ A.T + 9 * np.eye(9)
    K4 = K.reshape(3, 3, 3, 3)
    for _ in range(5):
        xi = rng.standard_normal(3)
        M = O.green_precond(K, xi)
        A3 = np.einsum("j,ijkl,l->ik", xi, K4, xi)
        assert np.abs(M @ A3 - np.eye(3)).max() < 1e-12
        G = np.einsum("j,ik,l->ijkl", xi, M, xi)
        GKG = np.einsum("ijab,abcd,cdkl->ijkl", G, K4, G)
        assert np.abs(GKG - G).max() < 1e-12 * np.abs(G).max()
    assert np.all(O.green_precond(K, np.zeros(3)) == 0)


# ------------------------------------------------------------------ P4
def _green_1mlap(n, h, ell):
    """Discrete Green's function of (1 - ell^2 lap) with the spectral
    Laplacian (-|xi|^2), via numpy's FFT."""
    k = [2 * np.pi * np.fft.fftfreq(nn, d=h) for nn in n]
    KX = k[0][None, None, :]
    KY = k[1][None, :, None]
    KZ = k[2][:, None, None]
    ghat = 1.0 / (1.0 + ell ** 2 * (KX ** 2 + KY ** 2 + KZ ** 2))
    return np.real(np.fft.ifftn(ghat))


def test_phase_field_uniform_source():
    """Eq. phase with uniform S: the Laplacian vanishes, (1+2S) phi = 2S,
    phi = 2S/(1+2S)."""
    n = (4, 4, 4)
    S = np.full(64, 0.37)
    phi, it, st = O.phase_field(n, H, 2 * H, S, np.zeros(64), np.zeros(64), tol=1e-14)
    assert st == 0
    assert np.abs(phi - 2 * 0.37 / (1 + 2 * 0.37)).max() < 1e-13


def test_phase_field_point_source_exact():
    """Eq. phase with S = s0 at one voxel: phi = 2 s0 (1 - phi0) G(x - x0),
    phi0 = 2 s0 G(0) / (1 + 2 s0 G(0)), G the discrete Green's function of
    (1 - ell^2 lap) (Eq. precph operator), computed with numpy."""
    n = (8, 6, 5)
    N = int(np.prod(n))
    ell = 2 * H
    S = np.zeros(N)
    v0 = 3 + 8 * (2 + 6 * 1)
    S[v0] = 0.8
    phi, it, st = O.phase_field(n, H, ell, S, np.zeros(N), np.zeros(N), tol=1e-14)
    G = _green_1mlap(n, H, ell).reshape(-1)
    G0 = G[0]
    phi0 = 2 * 0.8 * G0 / (1 + 2 * 0.8 * G0)
    Gs = np.roll(G.reshape(n[::-1]), (1, 2, 3), axis=(0, 1, 2)).reshape(-1)
    want = 2 * 0.8 * (1 - phi0) * Gs
    assert st == 0 and np.abs(phi - want).max() < 1e-12


def test_phase_field_1d_profile_exp():
    """Eq. strpf 1-D: the Green's function of (1 - ell^2 d2/dx2) on a period L
    is cosh((L/2 - |x|)/ell) / (2 ell sinh(L/(2 ell))); the spectral solution
    approaches it as ell/h grows (the exp(-|x|/ell) profile)."""
    N = 128
    errs = []
    for ratio in (2, 4, 8):
        ell = ratio * H
        S = np.zeros(N)
        S[0] = 1e-6  # linear regime: phi = 2 s0 G
        phi, it, st = O.phase_field((N, 1, 1), H, ell, S, np.zeros(N), np.zeros(N),
                                    tol=1e-15)
        x = np.minimum(np.arange(N), N - np.arange(N)) * H
        L = N * H
        cont = np.cosh((L / 2 - x) / ell) / (2 * ell * np.sinh(L / (2 * ell)))
        prof = phi / (2e-6 * (1 - phi[0])) / H  # per unit length
        errs.append(np.abs(prof - cont).max() / cont.max())
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.05


def test_phase_field_irreversibility_clamp():
    """Algorithm 1 clamp: phi_i = max(phi_i, phi_t) pointwise."""
    n = (4, 4, 4)
    rng = np.random.default_rng(1)
    S = rng.random(64) * 0.1
    phit = np.where(rng.random(64) > 0.7, 0.9, 0.0)
    phi, it, st = O.phase_field(n, H, 2 * H, S, phit, phit, tol=1e-13)
    assert np.all(phi >= phit) and np.all(phi < 1)
    free, _, _ = O.phase_field(n, H, 2 * H, S, phit, np.zeros(64), tol=1e-13)
    assert np.abs(np.maximum(free, phit) - phi).max() < 1e-12


def test_phase_field_zero_drive_keeps_phi_t():
    n = (4, 4, 4)
    phit = np.linspace(0, 1, 64)
    phi, it, st = O.phase_field(n, H, 2 * H, np.zeros(64), phit, phit)
    assert it == 0 and np.all(phi == phit)


# ------------------------------------------------------------ P7 / P8
def _qfield(N, Q=np.eye(3)):
    return np.tile(Q.reshape(9), N)


def _spectral_grad(n, h, v):
    """grad of a periodic scalar field with the derivative multiplier i xi,
    zero on the Nyquist frequency (numpy FFT)."""
    out = []
    shape = n[::-1]
    vh = np.fft.fftn(v.reshape(shape))
    for d in range(3):
        k = 2 * np.pi * np.fft.fftfreq(n[d], d=h)
        if n[d] % 2 == 0:
            k[n[d] // 2] = 0.0
        ax = 2 - d
        shp = [1, 1, 1]
        shp[ax] = n[d]
        out.append(np.real(np.fft.ifftn(vh * 1j * k.reshape(shp))).reshape(-1))
    return out


def test_nye_of_compatible_field_vanishes():
    """Eq. nye1 / nyeindexfourier: the curl of a gradient is zero, so a
    compatible plastic distortion F_p = I + grad(v) carries no GNDs."""
    n = (8, 6, 4)
    N = int(np.prod(n))
    rng = np.random.default_rng(7)
    Fp = np.zeros((9, N))
    for i in range(3):
        v = rng.standard_normal(N) * 1e-6
        g = _spectral_grad(n, H, v)
        for j in range(3):
            Fp[3 * i + j] = g[j] + (1.0 if i == j else 0.0)
    Lam, rho = O.gnd_field(n, H, MAT, _qfield(N), Fp)
    assert np.abs(Lam).max() < 1e-12 and rho.max() < 1e-12 / MAT["b"]


def test_nye_single_slip_sinusoid():
    """Eq. nye1 with the regularisation of Sec. 3.1: F_p = I + g(x) s(x)n,
    g = g0 sin(k.x) gives Lambda_ij = s_i (grad g x n)_j / (1 + ell_Fp^2 k^2),
    and the min-norm densities reproduce it with ||rho|| <= |grad g|/b."""
    n = (16, 8, 8)
    N = int(np.prod(n))
    s, nn = O.fcc_systems()
    kvec = 2 * np.pi * np.array([2 / (n[0] * H), 1 / (n[1] * H), 0.0])
    x = (np.arange(n[0])) * H
    y = (np.arange(n[1])) * H
    z = (np.arange(n[2])) * H
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    phase = (kvec[0] * X + kvec[1] * Y).reshape(-1)
    g0 = 1e-4
    g = g0 * np.sin(phase)
    Fp = np.zeros((9, N))
    P0 = np.outer(s[0], nn[0]).reshape(9)
    for c in range(9):
        Fp[c] = P0[c] * g + (1.0 if c in (0, 4, 8) else 0.0)
    Lam, rho = O.gnd_field(n, H, MAT, _qfield(N), Fp)
    reg = 1.0 / (1.0 + MAT["ell_Fp"] ** 2 * (kvec @ kvec))
    dg = g0 * np.cos(phase)[None, :] * kvec[:, None]  # grad g, 3 x N
    cr = np.cross(dg.T, nn[0]).T  # (grad g x n)
    want = np.einsum("i,jv->ijv", s[0], cr).reshape(9, N) * reg
    assert np.abs(Lam - want).max() < 1e-9 * np.abs(want).max()
    A, Ap = O.gnd_basis()
    assert np.abs(A @ Ap @ A - A).max() < 1e-13
    assert np.linalg.matrix_rank(A) == 9
    rvec = Ap @ Lam / MAT["b"]
    assert np.abs(A @ rvec - Lam / MAT["b"]).max() < 1e-9 * np.abs(Lam / MAT["b"]).max()
    gradn = np.linalg.norm(dg, axis=0) * reg / MAT["b"]
    assert np.all(rho <= gradn * (1 + 1e-9) + 1e-6)
    # the minimum-norm densities: Ap is the Moore-Penrose inverse of the
    # basis (NumPy's), and rho_GND is their norm per voxel
    assert np.abs(Ap - np.linalg.pinv(A)).max() < 1e-10 * np.abs(Ap).max()
    want_rho = np.linalg.norm(np.linalg.pinv(A) @ Lam, axis=0) / MAT["b"]
    assert np.abs(rho - want_rho).max() < 1e-9 * want_rho.max()


def test_nye_constant_fp_and_regulariser():
    """A constant F_p passes the regulariser unchanged and has no curl."""
    n = (4, 4, 4)
    N = 64
    Fp = np.tile((np.eye(3) + 1e-3 * np.arange(9).reshape(3, 3)).reshape(9, 1), (1, N))
    Lam, rho = O.gnd_field(n, H, MAT, _qfield(N), Fp)
    assert np.abs(Lam).max() < 1e-14


# ------------------------------------------------------ P1 / P9 / P12
def _run(n, gid, eul, opts, prog, phi0=None, mask=None, naive=False, mat=MAT):
    r = O.RVE(n, H, gid, eul, mat, opts, phi0=phi0, elastic_only=mask, naive=naive)
    stats = []
    for Fb, dt in prog:
        s, st = r.run_increment(Fb, dt)
        assert s == 0, st
        stats.append(st)
    return r, stats


def test_homogeneous_medium_uniform_strain():
    """Eqs. momentum and fdef: a single crystal with no defect stays uniform,
    F = Fbar exactly, with zero Krylov iterations (the residual vanishes)."""
    n = (4, 4, 4)
    gid, eul = I.single_crystal(n, (0.3, 0.9, 1.7))
    prog = I.uniaxial_cycle_program(0.004, 8, 1)[:3]
    r, stats = _run(n, gid, eul, I.solver_options("parity64"), prog)
    F = r.field("F")
    assert np.abs(F - prog[-1][0][:, None]).max() < 1e-15
    assert all(s["lin_it_total"] == 0 for s in stats)


def test_mean_strain_and_damage_bounds_polycrystal():
    """Eq. fdef: the fluctuation has zero mean, <F> = Fbar; Algorithm 1:
    phi_t <= phi <= 1 through the history, with damage switched on early by a
    small G_crit."""
    n = (6, 6, 6)
    gid, eul = I.voronoi(n, 3, 11)
    mat = dict(MAT, tau_c0=250.0, G_crit=1e-9, xi_store=1.0)
    prog = I.uniaxial_cycle_program(0.006, 24, 1)[:5]
    r = O.RVE(n, H, gid, eul, mat, I.solver_options("paper"))
    prev = np.zeros(int(np.prod(n)))
    for Fb, dt in prog:
        s, st = r.run_increment(Fb, dt)
        assert s == 0
        F = r.field("F")
        assert np.abs(F.mean(axis=1) - Fb).max() < 1e-14
        phi = r.field("phi_t")
        assert np.all(phi >= prev) and np.all(phi <= 1.0)
        prev = phi
    assert prev.max() > 0  # damage actually evolved


def test_naive_dft_vs_fft_full_solve():
    """A 4^3 polycrystal solved with the naive DFT and with the FFT agrees to
    round-off through plastic increments (transform independence)."""
    n = (4, 4, 4)
    gid, eul = I.voronoi(n, 3, 5)
    prog = I.uniaxial_cycle_program(0.008, 16, 1)[:5]
    opts = I.solver_options("parity64")
    a, _ = _run(n, gid, eul, opts, prog, naive=False)
    b, _ = _run(n, gid, eul, opts, prog, naive=True)
    for f in ("F", "Fp", "rho_ssd", "Wp"):
        x, y = a.field(f), b.field(f)
        assert np.abs(x - y).max() <= 1e-12 * max(np.abs(x).max(), 1e-30), f
    assert a.field("gamma").max() > 0  # plasticity happened


@pytest.mark.slow
def test_precrack_mirror_symmetry():
    """Sec. 4.1 geometry: a [100] single crystal with a centred pre-crack is
    mirror-symmetric about the plane x = 7.5 h (16^3 grid with the crack on
    x = 6..9): F_xx, F_yy, F_zz, F_yz are even and F_xy, F_xz odd."""
    cfg = I.build_config("sx16", n_override=(16, 8, 4))
    prog = cfg["program"][:3]
    r, _ = _run(cfg["n"], cfg["grain_ids"], cfg["euler"], I.solver_options("parity64"), prog,
                phi0=cfg["phi0"], mask=cfg["elastic_only"])
    n = cfg["n"]
    F = r.field("F").reshape(3, 3, n[2], n[1], n[0])
    Fm = F[..., ::-1]
    sign = np.array([[1, -1, -1], [-1, 1, 1], [-1, 1, 1]])
    for i in range(3):
        for j in range(3):
            assert np.abs(F[i, j] - sign[i, j] * Fm[i, j]).max() < 1e-12
    assert np.abs(F[0, 1]).max() > 1e-6  # the crack does perturb the field


def test_mixed_control_uniaxial_stress_closed_form():
    """Mixed stress/strain control (the paper's mixed-control extension):
    a [100] single crystal, F22 = 1 + eps prescribed and the other eight
    components of the mean first Piola stress held at zero, tiny eps so the
    response is linear elastic.  Cubic elasticity gives the lateral strains
    -C12 / (C11 + C12) eps, no shear, and the axial stress
    E100 eps = (C11 - C12)(C11 + 2 C12) / (C11 + C12) eps."""
    mat = I.material("baseline")
    n = (4, 4, 4)
    gid, eul = I.single_crystal(n)
    r = O.RVE(n, I.VOXEL_MM, gid, eul, mat, I.solver_options("parity64"))
    eps = 1e-5
    F = np.eye(3).reshape(9).copy()
    F[4] += eps
    mask = np.ones(9, dtype=int)
    mask[4] = 0
    s, st = r.run_increment(F, eps / 1e-3, Pbar=np.zeros(9), stress_mask=mask)
    assert s == 0 and st["mixed_it"] >= 1
    C11, C12 = mat["C11"], mat["C12"]
    Fb = np.array(st["Fbar"]).reshape(3, 3)
    lat = -C12 / (C11 + C12) * eps
    assert abs(Fb[0, 0] - 1 - lat) < 2e-3 * abs(lat)
    assert abs(Fb[2, 2] - 1 - lat) < 2e-3 * abs(lat)
    off = Fb - np.diag(np.diag(Fb))
    assert np.abs(off).max() < 1e-12
    P = np.array(st["Pbar"]).reshape(3, 3)
    E100 = (C11 - C12) * (C11 + 2 * C12) / (C11 + C12)
    assert abs(P[1, 1] - E100 * eps) < 2e-3 * E100 * eps
    Pl = P.copy()
    Pl[1, 1] = 0
    assert np.abs(Pl).max() < 1e-7 * abs(P[1, 1])
    # the mean F of the field is the solved macroscopic F
    assert np.abs(r.field("F").mean(axis=1) - Fb.reshape(9)).max() < 1e-13


def test_plate_matches_extruded_cell():
    """A one-voxel-thick periodic plate (n2 = 1, every frequency has xi_z = 0)
    under plane stress (mixed control, P11 = P33 = 0, in-plane uniaxial F22)
    equals, to round-off, a three-voxel-thick cell with the same in-plane
    microstructure extruded along z, whose fields are z-uniform by symmetry:
    F, P, F_p, rho_SSD and the GND density from the plastic F_p of the
    previous increments."""
    mat = dict(I.material("baseline"), tau_c0=150.0)
    n2, n3 = (8, 6, 1), (8, 6, 3)
    gid, eul = I.voronoi(n2, 3, 7)
    gid3 = np.tile(gid.reshape(1, 6, 8), (3, 1, 1)).reshape(-1)
    opts = I.solver_options("paper")
    a = O.RVE(n2, I.VOXEL_MM, gid, eul, mat, opts)
    b = O.RVE(n3, I.VOXEL_MM, gid3, eul, mat, opts)
    m = I.uniaxial_stress_mask(1)
    Fa = Fb_ = None
    for k, (Fb, dt) in enumerate(I.uniaxial_cycle_program(0.006, 24, 1)[:4]):
        ga = Fb.copy() if Fa is None else np.where(m == 1, Fa, Fb)
        gb = Fb.copy() if Fb_ is None else np.where(m == 1, Fb_, Fb)
        sa, sta = a.run_increment(ga, dt, Pbar=np.zeros(9), stress_mask=m)
        sb, stb = b.run_increment(gb, dt, Pbar=np.zeros(9), stress_mask=m)
        assert sa == 0 and sb == 0 and sta["mixed_it"] == stb["mixed_it"]
        Fa, Fb_ = np.array(sta["Fbar"]), np.array(stb["Fbar"])
        assert np.abs(Fa - Fb_).max() < 1e-14
    floor = {"F": 1e-4, "P": 1.0, "Fp": 1e-7, "rho_gnd": 1e2, "rho_ssd": 1e2}
    for f, fl in floor.items():
        A = a.field(f).reshape(-1, 1, 6, 8)
        B = b.field(f).reshape(-1, 3, 6, 8)
        if f in ("F", "Fp"):
            eye = np.eye(3).reshape(9, 1, 1, 1)
            A, B = A - eye, B - eye
        assert np.abs(B - A).max() <= 1e-10 * max(np.abs(A).max(), fl), f
    assert np.abs(a.field("rho_gnd")).max() > 1e3  # the plastic F_p is curl-carrying
    assert abs(np.array(sta["Pbar"])[8]) <= opts["tol_newton"] * abs(sta["Pbar"][4])


def test_cutback_equals_explicit_halves():
    """Cut-back (max_cutbacks, an extension of Algorithm 1): a single 0.6 %
    step from rest that Newton cannot take whole (max_newton 6, at most 100
    Krylov iterations per solve) is redone as
    halves of the step, recursively; the result equals, bit for bit, the
    same halves requested one by one from a handle with cut-back off, by the
    definition: the first half to the midpoint of the committed and the
    requested macroscopic F, the second to the request."""
    n = (6, 6, 6)
    gid, eul = I.voronoi(n, 3, 11)
    mat = dict(I.material("baseline"), tau_c0=250.0)
    Fb, dt = I.uniaxial_cycle_program(0.006, 4, 1)[0]
    a = O.RVE(n, I.VOXEL_MM, gid, eul, mat,
              I.solver_options("paper", max_newton=6, max_lin=100, max_cutbacks=3))
    s, st = a.run_increment(Fb, dt)
    assert s == 0 and st["cutbacks"] >= 1
    b = O.RVE(n, I.VOXEL_MM, gid, eul, mat,
              I.solver_options("paper", max_newton=6, max_lin=100, max_cutbacks=0))
    committed = [np.eye(3).reshape(9)]
    halvings = [0]

    def attempt(F, t):
        s, _ = b.run_increment(F, t)
        if s == 0:
            committed[0] = F.copy()
        return s

    def halves(F, t, depth):
        halvings[0] += 1
        mid = 0.5 * (committed[0] + F)
        s = attempt(mid, 0.5 * t)
        if s == -5 and depth < 3:
            s = halves(mid, 0.5 * t, depth + 1)
        if s:
            return s
        s = attempt(F, 0.5 * t)
        if s == -5 and depth < 3:
            s = halves(F, 0.5 * t, depth + 1)
        return s

    assert attempt(Fb, dt) == -5
    assert halves(Fb, dt, 1) == 0
    assert halvings[0] == st["cutbacks"]
    for f in ("F", "P", "Fp", "rho_ssd", "gamma", "Wp"):
        assert np.array_equal(a.field(f), b.field(f)), f


@pytest.mark.parametrize("scheme", ["willot", "spectral"])
def test_laminate_exact_with_willot_derivatives(scheme):
    """An elastic laminate of two cubic crystals, layers of 5 and 11 voxels
    normal to x and aligned with the grid, under a general macroscopic F: its
    exact solution is uniform in each layer, with F's y and z columns equal
    to Fbar (compatibility), the tractions P_ix continuous across the
    interfaces and <F> = Fbar.  Willot's rotated finite differences
    represent that field exactly, so the discrete solve reaches it to solver
    precision.  The layer pattern has a Nyquist component, which the
    spectral derivatives of Sec. 3.1 drop: their solution oscillates
    voxel to voxel, which shows the checks discriminate."""
    n = (16, 4, 4)
    N = 16 * 4 * 4
    x = np.tile(np.arange(16), 16)
    gid = (x >= 5).astype(np.int32)
    eul = np.array([[0.0, 0.0, 0.0], [0.4, 0.9, 0.3]])
    mat = I.material("baseline")
    opts = I.solver_options("parity64", derivative=scheme)
    r = O.RVE(n, I.VOXEL_MM, gid, eul, mat, opts, elastic_only=np.ones(N, dtype=np.uint8))
    rng = np.random.default_rng(4)
    Fbar = np.eye(3).reshape(9) + 1e-3 * rng.standard_normal(9)
    s, st = r.run_increment(Fbar, 1.0)
    assert s == 0
    F, P = r.field("F"), r.field("P")
    eps = np.abs(Fbar - np.eye(3).reshape(9)).max()
    spread = max(np.abs(F[:, gid == g] - F[:, gid == g].mean(axis=1, keepdims=True)).max()
                 for g in (0, 1))
    assert np.abs(F.mean(axis=1) - Fbar).max() < 1e-14
    if scheme == "spectral":
        assert spread > 1e-3 * eps
        return
    assert spread < 1e-10 * eps
    yz = [c for c in range(9) if c % 3 != 0]  # F_iy, F_iz
    assert np.abs(F[yz] - Fbar[yz, None]).max() < 1e-10 * eps
    PA, PB = P[:, gid == 0].mean(axis=1), P[:, gid == 1].mean(axis=1)
    assert np.abs(PA[[0, 3, 6]] - PB[[0, 3, 6]]).max() < 1e-8 * np.abs(P).max()
    assert np.abs(PA - PB).max() > 1e-3 * np.abs(P).max()  # the layers do differ


@pytest.mark.parametrize("scheme", ["willot", "spectral"])
def test_willot_matches_real_space_finite_differences(scheme):
    """Willot's rotated scheme against an independent real-space solve of
    the same discrete problem: a 6 x 6 x 4 cell with a 3 x 3 x 2 inclusion
    of another orientation, elastic, under a macroscopic strain of 1e-6
    (the finite-strain law is then linear to about 1e-6 relative, with the
    tangent at F = I).  In real space the rotated gradient of voxel p is the
    forward difference along j averaged over the four edges parallel to j
    of the cell whose lowest corner is node p; equilibrium is its transpose
    applied to the stress.  The periodic system G^T K G u = -G^T K E is
    solved directly and the strain E + G u compared with the oracle's
    F - I.  The spectral scheme is a different discretisation and misses it,
    which shows the comparison discriminates."""
    n0, n1, n2 = n = (6, 6, 4)
    N = n0 * n1 * n2
    z, y, x = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(n0), indexing="ij")
    gid = ((x >= 1) & (x <= 3) & (y >= 2) & (y <= 4) & (z >= 1) & (z <= 2)).astype(np.int32)
    gid = gid.reshape(-1)
    eul = np.array([[0.0, 0.0, 0.0], [0.7, 1.1, 0.2]])
    mat = I.material("baseline")
    h = I.VOXEL_MM
    rng = np.random.default_rng(8)
    E = 1e-6 * rng.standard_normal(9)
    r = O.RVE(n, h, gid, eul, mat, I.solver_options("parity64", derivative=scheme),
              elastic_only=np.ones(N, dtype=np.uint8))
    s, _ = r.run_increment(np.eye(3).reshape(9) + E, 1.0)
    assert s == 0
    eps_orc = r.field("F") - np.eye(3).reshape(9, 1)

    def node(ix, iy, iz):
        return (ix % n0) + n0 * ((iy % n1) + n1 * (iz % n2))

    G = np.zeros((9 * N, 3 * N))
    for v in range(N):
        p = (v % n0, (v // n0) % n1, v // (n0 * n1))
        for j in range(3):
            k, l = [a for a in range(3) if a != j]
            for a in (0, 1):
                for b in (0, 1):
                    st = list(p)
                    st[k] += a
                    st[l] += b
                    en = list(st)
                    en[j] += 1
                    for i in range(3):
                        G[9 * v + 3 * i + j, 3 * node(*en) + i] += 0.25 / h
                        G[9 * v + 3 * i + j, 3 * node(*st) + i] -= 0.25 / h
    Ks = [O.cp_point(mat, O.euler_to_Q(e), np.eye(3), np.eye(3), mat["rho_ssd0"], 0.0, 1.0,
                     elastic_only=True)["K"] for e in eul]
    Kb = np.zeros((9 * N, 9 * N))
    for v in range(N):
        Kb[9 * v:9 * v + 9, 9 * v:9 * v + 9] = Ks[gid[v]]
    Ev = np.tile(E, N)
    u = np.linalg.lstsq(G.T @ Kb @ G, -G.T @ Kb @ Ev, rcond=1e-12)[0]
    eps_fd = (Ev + G @ u).reshape(N, 9).T
    err = np.abs(eps_orc - eps_fd).max() / np.abs(eps_fd).max()
    if scheme == "willot":
        assert err < 1e-5
    else:
        assert err > 1e-3


def test_damped_newton_passes_the_yield_plateau():
    """The paper's loading (2 %, R = 0) under uniaxial stress on an 8^3,
    50-grain cell: near 1.1 % strain the full-step Newton falls into a
    two-cycle (the ratio of its test stuck near 0.2, |b| alternating between
    two values); with the damping of the update on stagnation every
    increment up to there converges without cut-back and holds the lateral
    stresses at zero."""
    cfg = I.build_config("poly64_r0", n_override=(8, 8, 8))
    mat = I.material("baseline")
    opts = I.solver_options("paper")
    r = O.RVE(cfg["n"], I.VOXEL_MM, cfg["grain_ids"], cfg["euler"], mat, opts)
    F = None
    for k in range(12):
        a, kw = I.increment_args(cfg, k, F)
        s, st = r.run_increment(*a, **kw)
        assert s == 0 and st["cutbacks"] == 0, (k, st)
        F = np.array(st["Fbar"])
        P = np.array(st["Pbar"])
        assert max(abs(P[0]), abs(P[8])) <= opts["tol_newton"] * np.abs(P).max()
    assert F[4] - 1.0 > 0.0119 and P[4] > 1000.0  # past the yield plateau


def test_mixed_cutback_equals_explicit_halves():
    """Cut-back under mixed control (uniaxial stress), by the same
    definition as under strain control plus its one addition: the second
    half's stress-controlled components start from the solved midpoint.  A
    single 0.6 % step from rest that fails whole equals, bit for bit, the
    same halves requested one by one with cut-back off, each half's guess of
    the lateral components built that way."""
    n = (6, 6, 6)
    gid, eul = I.voronoi(n, 3, 11)
    mat = dict(I.material("baseline"), tau_c0=250.0)
    m = I.uniaxial_stress_mask(1)
    Fb, dt = I.uniaxial_cycle_program(0.006, 4, 1)[0]
    kw = dict(max_newton=6, max_lin=100)
    a = O.RVE(n, I.VOXEL_MM, gid, eul, mat, I.solver_options("paper", max_cutbacks=3, **kw))
    s, st = a.run_increment(Fb, dt, Pbar=np.zeros(9), stress_mask=m)
    assert s == 0 and st["cutbacks"] >= 1
    b = O.RVE(n, I.VOXEL_MM, gid, eul, mat, I.solver_options("paper", max_cutbacks=0, **kw))
    committed = [np.eye(3).reshape(9)]
    halvings = [0]

    def attempt(F, t):
        s, st = b.run_increment(F, t, Pbar=np.zeros(9), stress_mask=m)
        if s == 0:
            committed[0] = np.array(st["Fbar"])
        return s

    def halves(F, t, depth):
        halvings[0] += 1
        mid = 0.5 * (committed[0] + F)
        s = attempt(mid, 0.5 * t)
        if s == -5 and depth < 3:
            s = halves(mid, 0.5 * t, depth + 1)
        if s:
            return s
        last = np.where(m == 1, committed[0], F)
        s = attempt(last, 0.5 * t)
        if s == -5 and depth < 3:
            s = halves(last, 0.5 * t, depth + 1)
        return s

    assert attempt(Fb, dt) == -5
    assert halves(Fb, dt, 1) == 0
    assert halvings[0] == st["cutbacks"]
    assert np.array_equal(committed[0], np.array(st["Fbar"]))
    for f in ("F", "P", "Fp", "rho_ssd", "gamma"):
        assert np.array_equal(a.field(f), b.field(f)), f


# ------------------------------------------------ history and driving force
# (shear, dilatation) history of a crystal in the lattice frame, shear along
# FCC system 0: yield, a further push with a 0.05 % dilatation on top (which
# resolves no shear on any system but raises W_e+, so that H_max stays above
# the later W_e+), elastic unloading, reversed yield, a reversed push,
# elastic unloading and re-yield (only system 0 ever slips; checked below).
_HIST_SHEAR = ((2e-3, 0.0), (4e-3, 0.0), (6e-3, 5e-4), (4e-3, 0.0), (0.0, 0.0), (-4e-3, 0.0),
               (-6e-3, 0.0), (-2e-3, 0.0), (2e-3, 0.0), (6e-3, 0.0), (3e-3, 0.0))


def _bisect(f, lo, hi):
    assert f(lo) < 0 < f(hi)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) < 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _history_by_hand(m, g_crit, dt=1.0):
    """The history of Sec. 2.1 and 2.3 for a homogeneous crystal (F = Fbar
    everywhere, so grad F_p = 0 and rho_GND = 0) under _HIST_SHEAR, built
    from quantities pinned elsewhere and written out here step by step:
      dgamma (one active system) by bisection of the scalar slip law,
      dW_p = tau dgamma, drho_SSD = lambda sqrt(2/3 dL:dL) with dL = dgamma P0,
      G_s += xi dW_p / sqrt(rho_SSD,n+1 + rho_GND)            (Eq. Gs, R10),
      W_e+ = 1/2 eps+ : C : eps+, eps = 1/2 ln(Fe Fe^T)      (Eq. decMiehe),
      H_max = max over the committed states of W_e+          (Eq. crit),
      W_crit = H_max + W_p at the first state with G_s >= G_crit (R9),
      S = <(W_e+ + W_p) / W_crit - 1> with the current W_e+  (Eq. zeta),
      phi = 2 S / (1 + 2 S) for a uniform drive, clamped by phi_t
                                                   (Eqs. strpf, phase; Alg. 1).
    Returns one dict per increment."""
    s, n = O.fcc_systems()
    P0 = np.outer(s[0], n[0])
    kT = m["k_B"] * m["T"]
    g0 = m["rho_m"] * m["b"] ** 2 * m["nu_D"] * np.exp(-m["dF"] / kT)
    sT = kT / (m["dV"] * 1e-3)
    tc = m["tau_c0"]
    Fpi, rho, Wp, Gs, Hmax, Wc, phi = np.eye(3), m["rho_ssd0"], 0.0, 0.0, 0.0, 0.0, 0.0
    out = []
    for e, dil in _HIST_SHEAR:
        F = (1.0 + dil) * (np.eye(3) + e * P0)

        def tau(dg, a=0):
            Fe = F @ Fpi @ (np.eye(3) - dg * P0)
            S = cubic_apply_np(m, 0.5 * (Fe.T @ Fe - np.eye(3)))
            return s[a] @ S @ n[a]

        dg = 0.0
        if abs(tau(0.0)) > tc:
            sg = np.sign(tau(0.0))
            dg = sg * _bisect(lambda x: x - dt * g0 * np.sinh((sg * tau(sg * x) - tc) / sT),
                              0.0, 0.01)
        t0 = tau(dg)
        assert all(abs(tau(dg, a)) < tc for a in range(1, 12))  # one active system
        Fpi = Fpi @ (np.eye(3) - dg * P0)
        Fe = F @ Fpi
        dW = t0 * dg
        rho = rho + m["lambda_h"] * np.sqrt(2.0 / 3.0) * abs(dg) * np.linalg.norm(P0)
        Wp += dW
        Gs += m["xi_store"] * dW / np.sqrt(rho)
        lam, V = np.linalg.eigh(Fe @ Fe.T)
        ep = V @ np.diag(np.maximum(0.5 * np.log(lam), 0.0)) @ V.T
        We = 0.5 * np.sum(ep * cubic_apply_np(m, ep))
        Hmax = max(Hmax, We)
        if Wc == 0.0 and Gs >= g_crit:
            Wc = Hmax + Wp
        S = max(0.0, (We + Wp) / Wc - 1.0) if Wc > 0 else 0.0
        phi = max(phi, 2 * S / (1 + 2 * S))
        out.append(dict(Fbar=F.reshape(9), dgamma=dg, rho_ssd=rho, Wp=Wp, Gs=Gs, We=We,
                        Hmax=Hmax, Wcrit=Wc, drive=S, phi_t=phi))
    return out


def history_chain_check():
    """Runs the oracle's Algorithm 1 on a 2 x 2 x 2 homogeneous crystal
    through _HIST_SHEAR and compares every committed history field with
    _history_by_hand.  G_crit is placed between G_s of the fifth and sixth
    increments, so W_crit is set at reversed yield, after the tensile peak
    (H_max > W_e+ there), and S is then positive at the reversed push and
    zero again on unloading (W_e+ < H_max).  Raises AssertionError on any
    mismatch (the mutation tests plant mistakes in the oracle and expect
    one)."""
    s, n = O.fcc_systems()
    m, _, _, _, tc = _single_slip_case(1.0)
    m = dict(m, G_crit=np.inf)
    free = _history_by_hand(m, np.inf)
    gs = [h["Gs"] for h in free]
    assert gs[4] < gs[5]
    m["G_crit"] = 0.5 * (gs[4] + gs[5])
    ref = _history_by_hand(m, m["G_crit"])
    # the sequence exercises what the pin is about
    assert ref[5]["Wcrit"] > 0 and ref[4]["Wcrit"] == 0
    assert ref[5]["Hmax"] > 1.05 * ref[5]["We"]
    assert ref[6]["drive"] > 0 and ref[7]["drive"] == 0
    assert ref[7]["Hmax"] + ref[7]["Wp"] > ref[7]["Wcrit"]
    r = O.RVE((2, 2, 2), H, np.zeros(8, dtype=np.int32), np.zeros(3), m,
              I.solver_options("parity64"))
    try:
        for k, h in enumerate(ref):
            st, stats = r.run_increment(h["Fbar"], 1.0)
            assert st == 0, (k, stats)
            got = {f: r.field(f) for f in ("rho_ssd", "Wp", "Gs", "We", "Hmax", "Wcrit",
                                            "drive", "phi_t")}
            gam = r.field("gamma")
            assert np.all(gam[1:] == 0)
            for f, v in got.items():
                assert np.ptp(v) == 0, (k, f)  # homogeneous
                want = h[f]
                assert abs(v[0] - want) <= 1e-9 * abs(want) + 1e-13, (k, f, v[0], want)
    finally:
        r.close()


def test_history_and_driving_force_chain():
    """Sec. 2.3 (Eqs. Gs, crit, zeta) with readings R9, R10 and A14: the
    stored energy density, the maximum tensile energy across a load reversal,
    the W_crit event and its value, and the driving force from the current
    W_e+, against a hand-built chain on a homogeneous crystal."""
    history_chain_check()


def _spectral_freqs(n, h):
    """Angular frequencies per axis, shaped for (n2, n1, n0) arrays."""
    ks = [2 * np.pi * np.fft.fftfreq(n[d], d=1.0 / n[d]) / (n[d] * h) for d in range(3)]
    return ks[0][None, None, :], ks[1][None, :, None], ks[2][:, None, None]


def staggered_fixed_point_check():
    """Algorithm 1 converged, at an increment where the crack grows over 13
    staggered iterations (6^3 three-grain polycrystal, damage parameters of
    the damage tests, tight tolerances): the degraded stress g(phi) P is in
    equilibrium (Eq. momentum: i xi_j F{g P}_ij = 0, the derivative zero on
    the Nyquist frequency of an even axis) and phi solves Eq. phase for the
    final drive, (1 + 2S) phi - ell^2 lap(phi) = 2S, wherever it lies above
    phi_t -- both residuals computed here with NumPy's FFT."""
    n = (6, 6, 6)
    gid, eul = I.voronoi(n, 3, 31)
    mat = I.material("baseline", tau_c0=250.0, G_crit=7e-4, xi_store=1.0)
    prog = I.uniaxial_cycle_program(0.006, 24, 2)
    r = O.RVE(n, H, gid, eul, mat, I.solver_options("parity64"))
    for Fb, dt in prog[:26]:
        assert r.run_increment(Fb, dt)[0] == 0
    phit = r.field("phi").reshape(n[::-1]).copy()
    s, st = r.run_increment(*prog[26])
    assert s == 0 and st["stag_it"] >= 5 and st["pf_it_total"] > 0
    x, y, z = _spectral_freqs(n, H)
    # equilibrium of the degraded stress
    P = r.field("P").reshape((9,) + n[::-1])
    Ph = np.fft.fftn(P, axes=(1, 2, 3))
    xd = [np.where(np.isclose(np.abs(k), np.pi / H), 0.0, k) for k in (x, y, z)]
    div = [sum(1j * xd[j] * Ph[3 * i + j] for j in range(3)) for i in range(3)]
    scale = np.pi / H * np.abs(Ph).max()
    assert max(np.abs(d).max() for d in div) < 1e-9 * scale
    # the phase-field equation where phi is not held at phi_t
    phi = r.field("phi").reshape(n[::-1])
    S = r.field("drive").reshape(n[::-1])
    lap = np.real(np.fft.ifftn(-(x ** 2 + y ** 2 + z ** 2) * np.fft.fftn(phi)))
    res = (1 + 2 * S) * phi - mat["ell"] ** 2 * lap - 2 * S
    free = phi > phit + 1e-12
    assert free.sum() > 0 and phi.max() > 0.05
    assert np.abs(res[free]).max() < 1e-9 * (2 * S).max()


def test_staggered_fixed_point_satisfies_both_equations():
    staggered_fixed_point_check()


def test_mixed_cutback_halves_a_changing_stress_target():
    """Cut-back under mixed control when the stress target changes between
    increments: each half takes half of the load change, so the first half
    aims the stress-controlled components at the midpoint of the committed
    target (the previous increment's) and the new one.  An increment that
    fails whole (a step from 0.3 to 0.7 % with the lateral stresses moving
    from 0 to -40 MPa) equals, bit for bit, the same halves requested one by one with
    cut-back off, each half's targets built that way."""
    n = (6, 6, 6)
    gid, eul = I.voronoi(n, 3, 11)
    mat = dict(I.material("baseline"), tau_c0=250.0)
    m = I.uniaxial_stress_mask(1)
    prog = I.uniaxial_cycle_program(0.006, 8, 1)
    P0, P1 = np.zeros(9), np.zeros(9)
    P1[0] = P1[8] = -40.0
    kw = dict(max_newton=10, max_lin=100)
    a = O.RVE(n, I.VOXEL_MM, gid, eul, mat, I.solver_options("paper", max_cutbacks=3, **kw))
    b = O.RVE(n, I.VOXEL_MM, gid, eul, mat, I.solver_options("paper", max_cutbacks=0, **kw))
    # a first, small increment at zero lateral stress, taken whole by both
    F1 = prog[0][0]
    s, st1 = a.run_increment(F1, prog[0][1], Pbar=P0, stress_mask=m)
    assert s == 0 and st1["cutbacks"] == 0
    s, stb = b.run_increment(F1, prog[0][1], Pbar=P0, stress_mask=m)
    assert s == 0
    committed = [np.array(stb["Fbar"]), P0.copy()]
    # then a large step that also moves the lateral stress target
    Fb = prog[1][0].copy()
    Fb[4] += 0.001
    dt = 4.0
    guess = np.where(m == 1, committed[0], Fb)
    s, st = a.run_increment(guess, dt, Pbar=P1, stress_mask=m)
    assert s == 0 and st["cutbacks"] >= 1
    halvings = [0]

    def attempt(F, P, t):
        s, stx = b.run_increment(F, t, Pbar=P, stress_mask=m)
        if s == 0:
            committed[0] = np.array(stx["Fbar"])
            committed[1] = P.copy()
        return s

    def halves(F, P, t, depth):
        halvings[0] += 1
        mid = 0.5 * (committed[0] + F)
        Pm = np.where(m == 1, 0.5 * (committed[1] + P), P)
        s = attempt(mid, Pm, 0.5 * t)
        if s == -5 and depth < 3:
            s = halves(mid, Pm, 0.5 * t, depth + 1)
        if s:
            return s
        last = np.where(m == 1, committed[0], F)
        s = attempt(last, P, 0.5 * t)
        if s == -5 and depth < 3:
            s = halves(last, P, 0.5 * t, depth + 1)
        return s

    assert attempt(guess, P1, dt) == -5
    assert halves(guess, P1, dt, 1) == 0
    assert halvings[0] == st["cutbacks"]
    assert np.array_equal(committed[0], np.array(st["Fbar"]))
    for f in ("F", "P", "Fp", "rho_ssd", "gamma"):
        assert np.array_equal(a.field(f), b.field(f)), f
    # the lateral stresses reached the new target within the mixed-control
    # stop rule, tol_newton max|<gP>|
    Pm = a.field("P").mean(axis=1)
    band = 5e-3 * np.abs(Pm).max()
    assert abs(Pm[0] + 40.0) <= band and abs(Pm[8] + 40.0) <= band
