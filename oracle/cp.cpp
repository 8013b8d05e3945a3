// Oracle constitutive update (test infrastructure only).
//
// Per-voxel crystal plasticity of Sec. 2.1 (multiplicative split, Eq. 1;
// plastic velocity gradient from 12 FCC slip systems; thermally activated
// slip law, Eq. flowrule; Taylor hardening; SSD evolution), the tensile
// elastic energy of Eq. decMiehe and the history of Sec. 2.3.  Everything is
// evaluated in the lattice frame; tensors are rotated in and out with Q.
//
// Readings of the paper used here (the paper leaves these open):
//  - slip law with sign and threshold: dgamma = dt*g0*sgn(tau)*
//    sinh(<|tau| - tau_c>/sT), sT = k_B T / dV (dV in mm^3, tau*dV in N mm
//    = 1e-3 J), g0 = rho_m b^2 nu_D exp(-dF/(k_B T));
//  - L_p = sum dgamma s (x) n (slip along s on planes normal to n);
//  - implicit (end-of-step stress) first-order update of the inverse plastic
//    deformation: Fp^-1 = Fp_n^-1 (I - sum dgamma s(x)n);
//  - elastic law S = C : E_e, E_e = (Fe^T Fe - I)/2, P = Fe S Fp^-T, with
//    the cubic C in the lattice frame; tau = S : (s (x) n);
//  - hardening explicit over the step: tau_c = tau_c0 + mu b sqrt(rho_ssd_n +
//    rho_gnd), the same on every system;
//  - W_e+ = 1/2 eps+ : C : eps+ with eps = 1/2 ln(Fe Fe^T), both in the
//    lattice frame.
#include <cstring>

#include "oracle_internal.hpp"

namespace orc {

// ---------- threading ----------
static int g_threads = 0;
int n_threads() {
    if (g_threads > 0) return g_threads;
    const char* e = std::getenv("ORACLE_THREADS");
    if (e && std::atoi(e) > 0) return std::atoi(e);
    const unsigned hc = std::thread::hardware_concurrency();
    return hc ? (int)hc : 1;
}
void set_threads(int n) { g_threads = n; }

// ---------- dense solve ----------
bool solve_dense(int n, double* A, double* b) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0) return false;
        if (piv != c) {
            for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
            std::swap(b[c], b[piv]);
        }
        for (int r = c + 1; r < n; ++r) {
            const double f = A[r * n + c] / A[c * n + c];
            if (f == 0.0) continue;
            for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * b[k];
        b[r] = s / A[r * n + r];
    }
    return true;
}

// ---------- cubic elasticity (lattice frame) ----------
M3 cubic_apply(const orc_material& m, const M3& E) {
    M3 S{};
    const double tr_ = E[0] + E[4] + E[8];
    S[0] = (m.C11 - m.C12) * E[0] + m.C12 * tr_;
    S[4] = (m.C11 - m.C12) * E[4] + m.C12 * tr_;
    S[8] = (m.C11 - m.C12) * E[8] + m.C12 * tr_;
    S[1] = S[3] = 2.0 * m.C44 * 0.5 * (E[1] + E[3]);
    S[2] = S[6] = 2.0 * m.C44 * 0.5 * (E[2] + E[6]);
    S[5] = S[7] = 2.0 * m.C44 * 0.5 * (E[5] + E[7]);
    return S;
}

// ---------- FCC {111}<110> (textbook geometry) ----------
static const double kPlanes[4][3] = {{1, 1, 1}, {-1, 1, 1}, {1, -1, 1}, {1, 1, -1}};
static const double kDirs[12][3] = {
    {0, 1, -1}, {1, 0, -1}, {1, -1, 0},   // on (1 1 1)
    {0, 1, -1}, {1, 0, 1},  {1, 1, 0},    // on (-1 1 1)
    {0, 1, 1},  {1, 0, -1}, {1, 1, 0},    // on (1 -1 1)
    {0, 1, 1},  {1, 0, 1},  {1, -1, 0}};  // on (1 1 -1)

struct Slip {
    double s[12][3], n[12][3];
    M3 P[12];  // s (x) n
};
static Slip make_slip() {
    Slip sl{};
    for (int a = 0; a < 12; ++a) {
        const double* pl = kPlanes[a / 3];
        for (int i = 0; i < 3; ++i) {
            sl.s[a][i] = kDirs[a][i] / std::sqrt(2.0);
            sl.n[a][i] = pl[i] / std::sqrt(3.0);
        }
        sl.P[a] = outer(sl.s[a], sl.n[a]);
    }
    return sl;
}
static const Slip& slip() {
    static const Slip s = make_slip();
    return s;
}

// ---------- symmetric eigen-decomposition (cyclic Jacobi) ----------
static void jacobi3(const M3& A0, double w[3], M3& V) {
    M3 A = A0;
    V = eye3();
    for (int sweep = 0; sweep < 60; ++sweep) {
        const double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
        const double dia = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
        if (off <= 1e-30 * dia || off == 0.0) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                const double apq = A[3 * p + q];
                if (apq == 0.0) continue;
                const double app = A[3 * p + p], aqq = A[3 * q + q];
                const double theta = (aqq - app) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) /
                                 (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                // A <- J^T A J with the rotation in the (p, q) plane
                for (int k = 0; k < 3; ++k) {
                    const double akp = A[3 * k + p], akq = A[3 * k + q];
                    A[3 * k + p] = c * akp - s * akq;
                    A[3 * k + q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    const double apk = A[3 * p + k], aqk = A[3 * q + k];
                    A[3 * p + k] = c * apk - s * aqk;
                    A[3 * q + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {
                    const double vkp = V[3 * k + p], vkq = V[3 * k + q];
                    V[3 * k + p] = c * vkp - s * vkq;
                    V[3 * k + q] = s * vkp + c * vkq;
                }
            }
    }
    w[0] = A[0];
    w[1] = A[4];
    w[2] = A[8];
}

// W_e+ (Eq. decMiehe, read with the factor 1/2 of an energy): eps = 1/2
// ln(Fe Fe^T) through the eigenvalues 1 + mu_i of Fe Fe^T.
static double we_plus(const orc_material& m, const M3& Fe) {
    const M3 Bdev = sub(mul(Fe, tr(Fe)), eye3());
    double mu[3];
    M3 V;
    jacobi3(Bdev, mu, V);
    M3 ep{};
    for (int k = 0; k < 3; ++k) {
        const double e = 0.5 * std::log1p(mu[k]);
        if (e <= 0.0) continue;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) ep[3 * i + j] += e * V[3 * i + k] * V[3 * j + k];
    }
    return 0.5 * ddot(ep, cubic_apply(m, ep));
}

// ---------- the constitutive point update ----------
static const int kVoigt[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
static const double kVw[6] = {1, 1, 1, 2, 2, 2};
static M3 from_voigt(const double* x) {
    M3 a{};
    for (int m = 0; m < 6; ++m) {
        a[3 * kVoigt[m][0] + kVoigt[m][1]] = x[m];
        a[3 * kVoigt[m][1] + kVoigt[m][0]] = x[m];
    }
    return a;
}
static void to_voigt(const M3& a, double* x) {
    for (int m = 0; m < 6; ++m) x[m] = a[3 * kVoigt[m][0] + kVoigt[m][1]];
}

struct SlipEval {
    double dg[12], a[12], tau[12];
    M3 M, Fe, S;
};

// State at given slip increments: M = I - sum dg P, Fe = Fe* M,
// E_e = (Fe^T Fe - I)/2, S = C : E_e, tau = S : P.
static void eval_slip(const orc_material& m, const M3& Fes, const double* dg, SlipEval& ev) {
    const Slip& sl = slip();
    M3 dL{};
    for (int a = 0; a < 12; ++a) {
        ev.dg[a] = dg[a];
        dL = add(dL, scale(sl.P[a], dg[a]));
    }
    ev.M = sub(eye3(), dL);
    ev.Fe = mul(Fes, ev.M);
    const M3 Ee = scale(sub(mul(tr(ev.Fe), ev.Fe), eye3()), 0.5);
    ev.S = cubic_apply(m, Ee);
    for (int a = 0; a < 12; ++a) ev.tau[a] = ddot(ev.S, sl.P[a]);
}

// B^a = C : sym(Fe^T Fe* P^a): the change of S per unit slip on system a is
// -B^a (from E_e = (M^T C* M - I)/2).
static M3 bmat(const orc_material& m, const M3& Fes, const M3& Fe, int a) {
    return cubic_apply(m, sym(mul(mul(tr(Fe), Fes), slip().P[a])));
}

// Potential whose stationary point is the local update (exactly in small
// strain): elastic energy 1/2 E_e : C : E_e plus, per active system, the
// dissipation tau_c y + sT (y asinh(y/c) - sqrt(y^2 + c^2) + c).  Used only as
// the line-search merit of the Newton iteration below.
static double potential(const orc_material& m, const SlipEval& ev, const double* y,
                        const bool* act, double tau_c, double c, double sT) {
    const M3 Ee = scale(sub(mul(tr(ev.Fe), ev.Fe), eye3()), 0.5);
    double psi = 0.5 * ddot(Ee, ev.S);
    for (int a = 0; a < 12; ++a)
        if (act[a])
            psi += tau_c * y[a] +
                   sT * (y[a] * std::asinh(y[a] / c) -
                         y[a] * y[a] / (std::sqrt(y[a] * y[a] + c * c) + c));
    return psi;
}

// Local update: the slip law is imposed in its inverse form on the active
// systems, sigma*tau - tau_c - sT*asinh(y/c) = 0 with dgamma = sigma*y,
// y >= 0, c = dt*g0; inactive systems have dgamma = 0 and |tau| <= tau_c.
// Active-set Newton: systems whose y reaches 0 with a negative residual
// leave the set; once the set is solved, the most overstressed inactive
// system (|tau| > tau_c) joins it, one at a time.  While the
// residual is large the Newton step is backtracked on the potential above.
static int local_solve(const orc_material& m, const M3& Fes, double tau_c, double c, double sT,
                       bool elastic_only, double tol, int max_it, SlipEval& ev, int* iters) {
    const Slip& sl = slip();
    double dg[12] = {0}, y[12] = {0}, sg[12] = {0};
    bool act[12] = {false};
    eval_slip(m, Fes, dg, ev);
    for (int a = 0; a < 12; ++a) ev.a[a] = 0.0;
    *iters = 0;
    if (elastic_only || c <= 0.0) return 0;
    auto slips = [&](const double* yy, double* d) {
        for (int a = 0; a < 12; ++a) d[a] = act[a] ? sg[a] * yy[a] : 0.0;
    };
    const double far = tau_c;
    int total = 0;
    for (int outer = 0; outer < 60; ++outer) {
        bool inner_ok = false;
        for (int it = 0; it < max_it; ++it, ++total) {
            slips(y, dg);
            eval_slip(m, Fes, dg, ev);
            double r[12] = {0}, rmax = 0;
            bool dropped = false;
            for (int a = 0; a < 12; ++a) {
                if (!act[a]) continue;
                r[a] = sg[a] * ev.tau[a] - tau_c - sT * std::asinh(y[a] / c);
                if (y[a] == 0.0 && r[a] < 0.0) {
                    act[a] = false;
                    dropped = true;
                }
            }
            if (dropped) continue;
            for (int a = 0; a < 12; ++a)
                if (act[a]) rmax = std::max(rmax, std::fabs(r[a]));
            if (rmax <= tol) {
                inner_ok = true;
                break;
            }
            int idx[12], na = 0;
            for (int a = 0; a < 12; ++a)
                if (act[a]) idx[na++] = a;
            double J[144], dy[12];
            for (int i = 0; i < na; ++i) {
                const int a = idx[i];
                for (int j = 0; j < na; ++j) {
                    const int b = idx[j];
                    J[na * i + j] = -sg[a] * sg[b] * ddot(sl.P[a], bmat(m, Fes, ev.Fe, b));
                }
                J[na * i + i] -= sT / std::sqrt(c * c + y[a] * y[a]);
                dy[i] = -r[a];
            }
            if (!solve_dense(na, J, dy)) return 1;
            double dmax = 0, ymax = c;
            for (int i = 0; i < na; ++i) {
                dmax = std::max(dmax, std::fabs(dy[i]));
                ymax = std::max(ymax, y[idx[i]]);
            }
            if (dmax <= 1e-15 * ymax) {  // stagnation at round-off
                inner_ok = true;
                break;
            }
            double ytry[12];
            for (int a = 0; a < 12; ++a) ytry[a] = y[a];
            for (int i = 0; i < na; ++i) ytry[idx[i]] = std::max(0.0, y[idx[i]] + dy[i]);
            if (rmax > far) {
                const double psi0 = potential(m, ev, y, act, tau_c, c, sT);
                double lam = 1.0;
                SlipEval et;
                double dtry[12];
                for (int ls = 0; ls < 8; ++ls) {
                    slips(ytry, dtry);
                    eval_slip(m, Fes, dtry, et);
                    if (potential(m, et, ytry, act, tau_c, c, sT) <= psi0) break;
                    lam *= 0.5;
                    for (int i = 0; i < na; ++i)
                        ytry[idx[i]] = std::max(0.0, y[idx[i]] + lam * dy[i]);
                }
            }
            for (int a = 0; a < 12; ++a) y[a] = ytry[a];
        }
        if (!inner_ok) {
            *iters = total;
            return 1;
        }
        // the most overstressed inactive system joins the set
        int best = -1;
        double over = 0.0;
        for (int a = 0; a < 12; ++a)
            if (!act[a] && std::fabs(ev.tau[a]) - tau_c > over) {
                over = std::fabs(ev.tau[a]) - tau_c;
                best = a;
            }
        if (best >= 0) {
            act[best] = true;
            sg[best] = ev.tau[best] > 0 ? 1.0 : -1.0;
            y[best] = 0.0;
        }
        if (best < 0) {
            *iters = total + 1;
            for (int a = 0; a < 12; ++a)
                ev.a[a] = act[a] ? std::sqrt(c * c + y[a] * y[a]) / sT : 0.0;
            return 0;
        }
    }
    *iters = total;
    return 1;
}

// 6x6 dR/dS of R(S) = S - C : E_e(S) (Voigt vectors, weights 2 on the shear
// entries of the contraction with sym(P)); a[a] = d dgamma / d tau.
static void jacobian(const orc_material& m, const M3& Fes, const SlipEval& ev, double* J) {
    const Slip& sl = slip();
    for (int i = 0; i < 36; ++i) J[i] = (i % 7 == 0) ? 1.0 : 0.0;
    for (int a = 0; a < 12; ++a) {
        if (ev.a[a] == 0.0) continue;
        double bv[6], pv[6];
        to_voigt(bmat(m, Fes, ev.Fe, a), bv);
        to_voigt(sym(sl.P[a]), pv);
        for (int r = 0; r < 6; ++r)
            for (int c = 0; c < 6; ++c) J[6 * r + c] += ev.a[a] * bv[r] * kVw[c] * pv[c];
    }
}

int cp_point(const orc_material& m, const M3& Q, const M3& F, const M3& FpL, double rho_ssd_n,
             double rho_gnd, double dt, bool elastic_only, double tol_local, int max_local,
             bool want_tangent, orc_cp_result& out) {
    const Slip& sl = slip();
    const double kT = m.k_B * m.T;
    const double g0 = m.rho_m * m.b * m.b * m.nu_D * std::exp(-m.dF / kT);
    const double sT = kT / (m.dV * 1e-3);
    const double tau_c = m.tau_c0 + m.mu * m.b * std::sqrt(rho_ssd_n + rho_gnd);

    const M3 FL = mul(tr(Q), mul(F, Q));
    const M3 A = inv(FpL);  // Fp_n^-1
    const M3 Fes = mul(FL, A);
    SlipEval ev;
    int it = 0;
    const int fail = local_solve(m, Fes, tau_c, dt * g0, sT, elastic_only, tol_local, max_local,
                                 ev, &it);
    if (elastic_only || dt <= 0.0)
        for (int a = 0; a < 12; ++a) ev.a[a] = 0.0;
    const M3 S = ev.S;
    const M3 Fpinv = mul(A, ev.M);
    const M3 FpinvT = tr(Fpinv);
    const M3 PL = mul(ev.Fe, mul(S, FpinvT));

    // outputs in the sample frame
    const M3 Ps = mul(Q, mul(PL, tr(Q)));
    for (int i = 0; i < 9; ++i) out.P[i] = Ps[i];
    to_voigt(S, out.S_L);
    const M3 FpNew = inv(Fpinv);
    for (int i = 0; i < 9; ++i) out.Fp_L[i] = FpNew[i];
    M3 dL{};
    double dWp = 0;
    for (int a = 0; a < 12; ++a) {
        out.dgamma[a] = ev.dg[a];
        out.tau[a] = ev.tau[a];
        dWp += ev.tau[a] * ev.dg[a];
        dL = add(dL, scale(sl.P[a], ev.dg[a]));
    }
    out.tau_c = tau_c;
    out.dWp = dWp;
    out.drho_ssd = m.lambda_h * std::sqrt(2.0 / 3.0 * ddot(dL, dL));
    out.We_plus = we_plus(m, ev.Fe);
    out.iters = it;
    out.fail = fail;

    if (want_tangent) {
        double J[36];
        jacobian(m, Fes, ev, J);
        double KL[81];
        const M3 X1 = mul(Fpinv, mul(S, FpinvT));  // Fp^-1 S Fp^-T
        const M3 SFpinvT = mul(S, FpinvT);
        const M3 FeS = mul(ev.Fe, S);
        const M3 AT = tr(A);
        for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) {
                M3 dF{};
                dF[3 * k + l] = 1.0;
                double rhs[6], Jc[36];
                to_voigt(cubic_apply(m, sym(mul(tr(ev.Fe), mul(dF, Fpinv)))), rhs);
                std::memcpy(Jc, J, sizeof(J));
                solve_dense(6, Jc, rhs);
                const M3 dS = from_voigt(rhs);
                M3 dM{};
                for (int a = 0; a < 12; ++a) {
                    if (ev.a[a] == 0.0) continue;
                    const double ddg = ev.a[a] * ddot(dS, sl.P[a]);
                    dM = sub(dM, scale(sl.P[a], ddg));
                }
                const M3 dP = add(add(mul(dF, X1), mul(mul(Fes, dM), SFpinvT)),
                                  add(mul(mul(ev.Fe, dS), FpinvT), mul(mul(FeS, tr(dM)), AT)));
                for (int ij = 0; ij < 9; ++ij) KL[9 * ij + 3 * k + l] = dP[ij];
            }
        // K_s,ijkl = Q_ia Q_jb Q_kc Q_ld K_L,abcd
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) {
                        double s = 0;
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b)
                                for (int c = 0; c < 3; ++c)
                                    for (int d = 0; d < 3; ++d)
                                        s += Q[3 * i + a] * Q[3 * j + b] * Q[3 * k + c] *
                                             Q[3 * l + d] * KL[9 * (3 * a + b) + 3 * c + d];
                        out.K[9 * (3 * i + j) + 3 * k + l] = s;
                    }
    }
    return fail;
}

double we_plus_public(const orc_material& m, const M3& Fe) { return we_plus(m, Fe); }
void sym_eig3_public(const M3& A, double w[3], M3& V) { jacobi3(A, w, V); }

}  // namespace orc

using namespace orc;

extern "C" {

void orc_material_paper(orc_material* m) {
    // Table 1 (CMSX-4) and Sec. 4; dV, mu, xi_store and rho_ssd0 are readings.
    m->C11 = 250e3;
    m->C12 = 161e3;
    m->C44 = 129e3;
    m->tau_c0 = 350.0;
    m->b = 3.5e-7;
    m->nu_D = 1e11;
    m->k_B = 1.4e-23;
    m->T = 295.0;
    m->dF = 4.9e-20;
    m->rho_m = 5.0e6;
    m->lambda_h = 150e6;
    m->dV = 20.0 * m->b * m->b * m->b;
    m->mu = m->C44;
    m->xi_store = 0.05;
    m->rho_ssd0 = m->rho_m;
    m->G_crit = 4e-3;
    m->ell = 2.34e-3;
    m->ell_Fp = 1.56e-3;
    m->k_res = 1e-5;
}

void orc_euler_to_Q(const double e[3], double Q[9]) {
    const double c1 = std::cos(e[0]), s1 = std::sin(e[0]);
    const double c = std::cos(e[1]), s = std::sin(e[1]);
    const double c2 = std::cos(e[2]), s2 = std::sin(e[2]);
    // g maps sample to lattice coordinates (Bunge z-x-z, passive); Q = g^T
    const double g[9] = {c1 * c2 - s1 * s2 * c,  s1 * c2 + c1 * s2 * c,  s2 * s,
                         -c1 * s2 - s1 * c2 * c, -s1 * s2 + c1 * c2 * c, c2 * s,
                         s1 * s,                 -c1 * s,                c};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Q[3 * i + j] = g[3 * j + i];
}

void orc_fcc_systems(double s[36], double n[36]) {
    const Slip& sl = slip();
    for (int a = 0; a < 12; ++a)
        for (int i = 0; i < 3; ++i) {
            s[3 * a + i] = sl.s[a][i];
            n[3 * a + i] = sl.n[a][i];
        }
}

int orc_cp_point(const orc_material* m, const double Q[9], const double F[9], const double Fp_L[9],
                 double rho_ssd_n, double rho_gnd, double dt, int elastic_only, double tol_local,
                 int max_local, int want_tangent, orc_cp_result* out) {
    return cp_point(*m, from_ptr(Q), from_ptr(F), from_ptr(Fp_L), rho_ssd_n, rho_gnd, dt,
                    elastic_only != 0, tol_local, max_local, want_tangent != 0, *out);
}

double orc_we_plus(const orc_material* m, const double Fe_L[9]) {
    return we_plus_public(*m, from_ptr(Fe_L));
}

void orc_sym_eig3(const double A[9], double w[3], double V[9]) {
    M3 v;
    sym_eig3_public(from_ptr(A), w, v);
    for (int i = 0; i < 9; ++i) V[i] = v[i];
}

}  // extern "C"
