"""Mutation checks of the oracle's pins: a plausible mistake planted in a
copy of the oracle's sources (built on the CPU into a temporary folder) must
make a pin fail.  The committed oracle is never modified.

Each mutant names the passage whose restatement it breaks."""
import os
import shutil
import subprocess

import pytest

import oracle as O
from oracle import build as OB
import test_oracle_pins as pins
from test_oracle_pins import history_chain_check, local_solve_check, staggered_fixed_point_check

MUTANTS = {
    # Eq. Gs / R10: the stored energy increment divides by the density after
    # the increment's SSD growth, not before it
    "gs_uses_old_rho": ("rve.cpp", "std::sqrt(rho_new + r->rho_gnd[v])",
                        "std::sqrt(r->rho_t[v] + r->rho_gnd[v])"),
    # Eq. crit / R9: W_crit is H_max + W_p at the event, not W_p alone
    "wcrit_without_hmax": ("rve.cpp", "wc = r->Hmax_tr[v] + r->Wp_tr[v];",
                           "wc = r->Wp_tr[v];"),
    # Eq. zeta / A14: the drive uses the current W_e+, the maximum only
    # enters W_crit
    "drive_uses_hmax": ("rve.cpp", "(res.We_plus + r->Wp_tr[v]) / wc",
                        "(r->Hmax_tr[v] + r->Wp_tr[v]) / wc"),
}


# mistakes in the local crystal-plasticity update (Sec. 2.1), against the
# pin that restates it and solves it by another method
MUTANTS_CP = {
    # the implicit update F_p^-1 = F_pn^-1 (I - sum dgamma s (x) n) with the
    # sign of the plastic increment flipped
    "fp_update_sign": ("cp.cpp", "ev.M = sub(eye3(), dL);", "ev.M = add(eye3(), dL);"),
    # Taylor hardening without the GND density
    "hardening_without_gnd": ("cp.cpp", "std::sqrt(rho_ssd_n + rho_gnd)",
                              "std::sqrt(rho_ssd_n)"),
    # the elastic strain as the small-strain sym(F_e) - I instead of
    # (F_e^T F_e - I) / 2
    "small_strain_measure": ("cp.cpp",
                             "const M3 Ee = scale(sub(mul(tr(ev.Fe), ev.Fe), eye3()), 0.5);\n"
                             "    ev.S = cubic_apply(m, Ee);",
                             "const M3 Ee = sub(scale(add(ev.Fe, tr(ev.Fe)), 0.5), eye3());\n"
                             "    ev.S = cubic_apply(m, Ee);"),
    # the thermal stress kT / dV with dV left in mm^3 (tau dV in N mm)
    "thermal_stress_units": ("cp.cpp", "kT / (m.dV * 1e-3)", "kT / m.dV"),
}


# mistakes in the phase-field solve (Eqs. strpf, phase), against its
# closed-form pins (uniform source, exact discrete point source, 1-D profile)
MUTANTS_PF = {
    # the reaction term (1 + 2S) phi written as (1 + S) phi
    "pf_reaction_factor": ("rve.cpp", "y[v] += (1.0 + 2.0 * S[v]) * x[v];",
                           "y[v] += (1.0 + S[v]) * x[v];"),
    # the right-hand side 2S written as S
    "pf_source_factor": ("rve.cpp", "r[v] = 2.0 * S[v] - q[v];", "r[v] = S[v] - q[v];"),
    # the length scale entering the operator unsquared
    "pf_ell_unsquared": ("rve.cpp", "const double l2 = ell * ell;\n    std::vector<double> lap_w",
                         "const double l2 = ell;\n    std::vector<double> lap_w"),
}


# mistakes in the GND stage (Eqs. nye1, nyeindexfourier, the F_p
# regularisation) and in the cubic elasticity (Sec. 2.1), against their pins
MUTANTS_NYE = {
    # the curl taken over the first index of F_p instead of the second
    "nye_transposed_fp": ("rve.cpp", "* Fh[3 * i + l][v];", "* Fh[3 * l + i][v];"),
    # the regularisation length entering unsquared
    "nye_reg_unsquared": ("rve.cpp", "const double l2 = m.ell_Fp * m.ell_Fp;",
                          "const double l2 = m.ell_Fp;"),
    # the dislocation densities multiplied by b instead of divided
    "gnd_times_burgers": ("rve.cpp", "x /= m.b;", "x *= m.b;"),
}
MUTANTS_EL = {
    # tensor shear strains taken as engineering ones: sigma_12 = C44 e_12
    "cubic_shear_half": ("cp.cpp", "S[1] = S[3] = 2.0 * m.C44 * 0.5 * (E[1] + E[3]);",
                         "S[1] = S[3] = m.C44 * 0.5 * (E[1] + E[3]);"),
    # C11 and C12 exchanged on the diagonal
    "cubic_c11_c12": ("cp.cpp", "S[0] = (m.C11 - m.C12) * E[0] + m.C12 * tr_;",
                      "S[0] = (m.C12 - m.C11) * E[0] + m.C11 * tr_;"),
}


# Algorithm 1: the staggered loop stopped after its first pass, and two
# mistakes in the Newton-Krylov solve inside it
MUTANTS_ALG1 = {
    "stag_single_pass": ("rve.cpp", "r->converged = cF && cP;", "r->converged = true;"),
    # the Krylov solve of Sec. 3.1 with one Givens rotation applied with the
    # wrong sign (its residual estimate no longer that of the iterate)
    "givens_sign": ("rve.cpp", "H[i + 1][k] = -sn[i] * H[i][k] + cs[i] * H[i + 1][k];",
                    "H[i + 1][k] = sn[i] * H[i][k] + cs[i] * H[i + 1][k];"),
    # the Newton update of Eq. fdef subtracted instead of added
    "newton_update_sign": ("rve.cpp", "r->F[(3 * i + j) * N + v] += alpha * g[v];",
                           "r->F[(3 * i + j) * N + v] -= alpha * g[v];"),
}
# the Green preconditioner contracted over the wrong indices (Eq. precf),
# and the mixed-control correction with its sign flipped
MUTANTS_OPS = {
    "green_wrong_indices": ("rve.cpp", "s += xi[j] * Kbar[9 * (3 * i + j) + 3 * k + l] * xi[l];",
                            "s += xi[j] * Kbar[9 * (3 * j + i) + 3 * l + k] * xi[l];"),
    "mixed_correction_sign": ("rve.cpp", "d[a] = -(Pbar[S[a]] - r->Pstar[S[a]]);",
                              "d[a] = (Pbar[S[a]] - r->Pstar[S[a]]);"),
}


def ops_checks(name):
    if name.startswith("green"):
        pins.test_green_operator_identities()
    else:
        pins.test_mixed_control_uniaxial_stress_closed_form()


def nye_checks():
    pins.test_nye_of_compatible_field_vanishes()
    pins.test_nye_single_slip_sinusoid()
    pins.test_nye_constant_fp_and_regulariser()


def elastic_checks():
    pins.test_elastic_uniaxial_closed_form()
    pins.test_elastic_simple_shear_closed_form()
    pins.test_elastic_rotated_crystal_frame_covariance()


def phase_field_checks():
    pins.test_phase_field_uniform_source()
    pins.test_phase_field_point_source_exact()
    pins.test_phase_field_1d_profile_exp()


# the extensions: Willot's rotated derivative without its edge averaging
# (R33), the cut-back's first half taking the whole step (R28), the Newton
# damping switched off (R31)
MUTANTS_EXT = {
    "willot_unaveraged": ("rve.cpp", "if (l != j) s *= 0.5 * (1.0 + e[l]);",
                          "if (l != j) s *= 1.0;"),
    "cutback_full_dt": ("rve.cpp", "int s = attempt(r, mid, Pmid, mask, 0.5 * dt, st);",
                        "int s = attempt(r, mid, Pmid, mask, dt, st);"),
    "no_newton_damping": ("rve.cpp", "alpha = std::max(0.5 * alpha, 1.0 / 16);",
                          "alpha = alpha;"),
}


def ext_checks(name):
    if name.startswith("willot"):
        pins.test_willot_matches_real_space_finite_differences("willot")
    elif name.startswith("cutback"):
        pins.test_cutback_equals_explicit_halves()
    else:
        pins.test_damped_newton_passes_the_yield_plateau()


# further mistakes in the crystal-plasticity point update (Sec. 2.1), each
# against the pin that restates the step it breaks
MUTANTS_KIN = {
    # the Schmid tensor n (x) s in place of s (x) n
    "schmid_transposed": ("cp.cpp", "sl.P[a] = outer(sl.s[a], sl.n[a]);",
                          "sl.P[a] = outer(sl.n[a], sl.s[a]);"),
    # the first Piola-Kirchhoff stress without the pull-back by F_p^-T
    "pk1_without_fp": ("cp.cpp", "const M3 PL = mul(ev.Fe, mul(S, FpinvT));",
                       "const M3 PL = mul(ev.Fe, S);"),
    # F rotated into the lattice frame with Q and Q^T exchanged
    "lattice_frame_transposed": ("cp.cpp", "const M3 FL = mul(tr(Q), mul(F, Q));",
                                 "const M3 FL = mul(Q, mul(F, tr(Q)));"),
    # the SSD increment without the 2/3 of the equivalent plastic strain
    "ssd_rate_factor": ("cp.cpp", "m.lambda_h * std::sqrt(2.0 / 3.0 * ddot(dL, dL))",
                        "m.lambda_h * std::sqrt(ddot(dL, dL))"),
    # the reference slip dt g0 of Eq. flowrule without the time step
    "rate_without_dt": ("cp.cpp", "tau_c, dt * g0, sT", "tau_c, g0, sT"),
    # the consistent tangent without the change of F_p^-1 with the slips
    "tangent_without_slip_term": ("cp.cpp", "mul(mul(Fes, dM), SFpinvT)",
                                  "scale(mul(mul(Fes, dM), SFpinvT), 0.0)"),
}


def kin_checks(name):
    if name.startswith("ssd"):
        pins.test_single_slip_by_bisection(1.0)
    elif name.startswith("rate"):
        pins.test_slip_rate_limits()
    elif name.startswith("tangent"):
        pins.test_tangent_matches_finite_differences(1)
    else:
        local_solve_check()


# the tensile elastic energy of Eq. decMiehe
MUTANTS_WE = {
    # the right stretch F_e^T F_e in place of the left one
    "we_right_stretch": ("cp.cpp", "const M3 Bdev = sub(mul(Fe, tr(Fe)), eye3());",
                         "const M3 Bdev = sub(mul(tr(Fe), Fe), eye3());"),
    # the Green-Lagrange strain in place of the logarithmic one
    "we_green_strain": ("cp.cpp", "const double e = 0.5 * std::log1p(mu[k]);",
                        "const double e = 0.5 * mu[k];"),
    # no split: compressive principal strains kept
    "we_no_split": ("cp.cpp", "if (e <= 0.0) continue;", "if (e != e) continue;"),
}


def we_checks():
    pins.test_eigen_split_degenerate_and_rotated()
    pins.test_we_plus_generic_state_numpy()


# the building blocks: the orientation matrix (Sec. 2.1, Bunge angles), the
# transform (Sec. 3.1) and the irreversibility clamp (Algorithm 1)
MUTANTS_BASE = {
    # g (sample to lattice) returned in place of Q = g^T
    "euler_not_transposed": ("cp.cpp", "Q[3 * i + j] = g[3 * j + i];",
                             "Q[3 * i + j] = g[3 * i + j];"),
    # the twiddle factors off the quarter turns with the opposite sign
    "fft_twiddle_sign": ("fft.cpp", "const double a = sign * two_pi * (double)t / (double)n;",
                         "const double a = -sign * two_pi * (double)t / (double)n;"),
    # the damage no longer held at or above phi_t
    "pf_clamp_dropped": ("rve.cpp", "phi[v] = std::max(x[v], phi_t[v]);", "phi[v] = x[v];"),
}


def base_checks(name):
    if name.startswith("euler"):
        pins.test_euler_rotation_is_bunge()
    elif name.startswith("fft"):
        pins.test_fft_matches_numpy_and_naive_dft((6, 6, 6))
    else:
        pins.test_phase_field_irreversibility_clamp()


ALL_MUTANTS = {**MUTANTS, **MUTANTS_CP, **MUTANTS_PF, **MUTANTS_NYE, **MUTANTS_EL,
               **MUTANTS_ALG1, **MUTANTS_OPS, **MUTANTS_EXT, **MUTANTS_KIN, **MUTANTS_WE,
               **MUTANTS_BASE}


def _build_mutant(tmp, name):
    fname, old, new = ALL_MUTANTS[name]
    src = os.path.join(tmp, "src_" + name)
    os.makedirs(src, exist_ok=True)
    for f in OB.SOURCES + ["oracle.h", "oracle_internal.hpp"]:
        shutil.copy(os.path.join(OB.HERE, f), src)
    p = os.path.join(src, fname)
    text = open(p).read()
    assert text.count(old) == 1, (name, "the planted site must match exactly once")
    open(p, "w").write(text.replace(old, new))
    out = os.path.join(tmp, f"lib_{name}.so")
    subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-pthread",
                    *[os.path.join(src, s) for s in OB.SOURCES], "-o", out], check=True)
    return out


@pytest.fixture(scope="module")
def mutant_libs(tmp_path_factory):
    """Every mutant built once, concurrently (the compiles dominate)."""
    from concurrent.futures import ThreadPoolExecutor
    tmp = str(tmp_path_factory.mktemp("mutants"))
    names = sorted(ALL_MUTANTS)
    with ThreadPoolExecutor(max_workers=min(len(names), os.cpu_count() or 1)) as ex:
        paths = list(ex.map(lambda n: _build_mutant(tmp, n), names))
    return dict(zip(names, paths))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_history_pin_catches_mutant(name, mutant_libs):
    path = mutant_libs[name]
    with O.library(path):
        with pytest.raises(AssertionError):
            history_chain_check()
    history_chain_check()  # the committed oracle still passes


@pytest.mark.parametrize("name", sorted(MUTANTS_CP))
def test_local_solve_pin_catches_mutant(name, mutant_libs):
    path = mutant_libs[name]
    with O.library(path):
        with pytest.raises(AssertionError):
            local_solve_check()


@pytest.mark.parametrize("name", sorted(MUTANTS_PF))
def test_phase_field_pins_catch_mutant(name, mutant_libs):
    path = mutant_libs[name]
    with O.library(path):
        with pytest.raises(AssertionError):
            phase_field_checks()


@pytest.mark.parametrize("name", sorted(MUTANTS_NYE))
def test_gnd_pins_catch_mutant(name, mutant_libs):
    path = mutant_libs[name]
    with O.library(path):
        with pytest.raises(AssertionError):
            nye_checks()


@pytest.mark.parametrize("name", sorted(MUTANTS_EL))
def test_elastic_pins_catch_mutant(name, mutant_libs):
    path = mutant_libs[name]
    with O.library(path):
        with pytest.raises(AssertionError):
            elastic_checks()


@pytest.mark.parametrize("name", sorted(MUTANTS_ALG1))
def test_fixed_point_pin_catches_mutant(name, mutant_libs):
    path = mutant_libs[name]
    with O.library(path):
        with pytest.raises(AssertionError):
            staggered_fixed_point_check()


@pytest.mark.parametrize("name", sorted(MUTANTS_OPS))
def test_operator_pins_catch_mutant(name, mutant_libs):
    path = mutant_libs[name]
    with O.library(path):
        with pytest.raises(AssertionError):
            ops_checks(name)


@pytest.mark.parametrize("name", sorted(MUTANTS_EXT))
def test_extension_pins_catch_mutant(name, mutant_libs):
    path = mutant_libs[name]
    with O.library(path):
        with pytest.raises(AssertionError):
            ext_checks(name)


@pytest.mark.parametrize("name", sorted(MUTANTS_KIN))
def test_point_update_pins_catch_mutant(name, mutant_libs):
    path = mutant_libs[name]
    with O.library(path):
        with pytest.raises(AssertionError):
            kin_checks(name)


@pytest.mark.parametrize("name", sorted(MUTANTS_WE))
def test_energy_split_pins_catch_mutant(name, mutant_libs):
    path = mutant_libs[name]
    with O.library(path):
        with pytest.raises(AssertionError):
            we_checks()


@pytest.mark.parametrize("name", sorted(MUTANTS_BASE))
def test_building_block_pins_catch_mutant(name, mutant_libs):
    path = mutant_libs[name]
    with O.library(path):
        with pytest.raises(AssertionError):
            base_checks(name)
