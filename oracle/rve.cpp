// Oracle RVE solver (test infrastructure only).
//
// Spectral field operators of Sec. 3.1 and the alternating minimisation of
// Algorithm 1, written on the FULL complex spectrum with the paper's
// frequency vectors xi_i = 2 pi (n_i - floor(N_i/2)) / L_i (stored in natural
// FFT order).  Unknowns live on every frequency, inner products are plain
// sums over all frequencies, and no real-transform symmetry is used.
//
// Readings (the paper leaves these open):
//  - first-derivative multipliers i xi_j are zero on the Nyquist frequency of
//    an even axis; the Laplacian keeps -|xi|^2 there;
//  - Eq. fdef read as F = F^-1{u (x) i xi} + Fbar;
//  - the Krylov solver of Eq. newton is restarted GMRES with right
//    preconditioning by the Green operator of Eq. precf, built from the
//    volume average (Eq. avstiff) of the degraded consistent tangent;
//  - Eq. precph read as M_phi = [1 + ell^2 |xi|^2]^-1;
//  - F_p regularisation read with ell_Fp^2;
//  - Nye tensor Lambda_ij = eps_jkl d_k Fp_il over the whole domain,
//    GND densities by the minimum-norm solution over 12 edge + 6 screw unit
//    dyads, divided by b;
//  - Algorithm 1 ratios guarded: converged when ||F_i - F_{i-1}|| <=
//    tol * max(||F_i - F_t||, 1e-12) (same for phi);
//  - the Krylov solve stops at max(tol_lin ||b||, 1e-12 s_b) with s_b the
//    norm of the terms F{g P}_ij xi_j summed into b: below that the residual
//    is round-off (a residual already that small gets no correction);
//  - an equilibrium solve whose phase field has not changed since the last
//    solve is skipped (same problem, same answer), and the increment is then
//    converged;
//  - when the driving force S is zero everywhere the unconstrained
//    phase-field solution is 0, so the clamped solution is phi_t exactly.
#include <cstdio>
#include <cstring>

#include "oracle_internal.hpp"

namespace orc {
int cp_point(const orc_material& m, const M3& Q, const M3& F, const M3& FpL, double rho_ssd_n,
             double rho_gnd, double dt, bool elastic_only, double tol_local, int max_local,
             bool want_tangent, orc_cp_result& out);

// ---------- frequencies ----------
struct Freq {
    int n[3];
    size_t N;
    double h;
    std::vector<double> xi[3];   // full frequency per axis index
    std::vector<double> xid[3];  // derivative frequency (Nyquist -> 0)
    std::vector<cplx> shift[3];  // exp(i xi h): a shift by one voxel along the axis
};
static Freq make_freq(const int n[3], double h) {
    Freq f;
    for (int d = 0; d < 3; ++d) {
        f.n[d] = n[d];
        const double L = n[d] * h;
        f.xi[d].resize(n[d]);
        f.xid[d].resize(n[d]);
        const int half_up = (n[d] + 1) / 2;
        for (int mm = 0; mm < n[d]; ++mm) {
            const int kk = mm < half_up ? mm : mm - n[d];
            f.xi[d][mm] = 2.0 * M_PI * kk / L;
            const bool nyq = (n[d] % 2 == 0) && (kk == -n[d] / 2);
            f.xid[d][mm] = nyq ? 0.0 : f.xi[d][mm];
            // exactly -1 at the Nyquist index, so that the rotated scheme's
            // factor (1 + e) vanishes there (its null modes) without round-off
            f.shift[d].push_back(nyq ? cplx(-1.0, 0.0) : std::polar(1.0, 2.0 * M_PI * kk / n[d]));
        }
    }
    f.N = (size_t)n[0] * n[1] * n[2];
    f.h = h;
    return f;
}

// Willot's rotated finite-difference derivative (Willot 2015, Comptes Rendus
// Mecanique 343): the forward difference along j averaged over the four cell
// edges parallel to j, i.e. in Fourier D_j = (e_j - 1)/h prod_{l != j} (1 +
// e_l)/2 with e_l = exp(i xi_l h).  It replaces i xi_j in the gradient; its
// adjoint -conj(D_j) replaces i xi_j in the divergence.
static inline void willot_symbol(const Freq& f, size_t v, cplx D[3]) {
    const int idx[3] = {(int)(v % f.n[0]), (int)((v / f.n[0]) % f.n[1]),
                        (int)(v / ((size_t)f.n[0] * f.n[1]))};
    cplx e[3];
    for (int d = 0; d < 3; ++d) e[d] = f.shift[d][idx[d]];
    for (int j = 0; j < 3; ++j) {
        cplx s = (e[j] - 1.0) / f.h;
        for (int l = 0; l < 3; ++l)
            if (l != j) s *= 0.5 * (1.0 + e[l]);
        D[j] = s;
    }
}

// Green preconditioner of the rotated scheme at one frequency:
// [conj(D) . Kbar . D]^-1, a Hermitian 3 x 3 inverted by cofactors; zero
// where D = 0 (the zero frequency and the scheme's null modes).
static void green_willot(const double* Kbar, const cplx D[3], cplx Minv[9]) {
    if (std::abs(D[0]) == 0 && std::abs(D[1]) == 0 && std::abs(D[2]) == 0) {
        for (int i = 0; i < 9; ++i) Minv[i] = 0.0;
        return;
    }
    cplx A[9];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) {
            cplx s = 0.0;
            for (int j = 0; j < 3; ++j)
                for (int l = 0; l < 3; ++l)
                    s += std::conj(D[j]) * Kbar[9 * (3 * i + j) + 3 * k + l] * D[l];
            A[3 * i + k] = s;
        }
    const cplx c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8],
               c02 = A[3] * A[7] - A[4] * A[6];
    const cplx det = A[0] * c00 + A[1] * c01 + A[2] * c02;
    Minv[0] = c00 / det;
    Minv[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    Minv[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    Minv[3] = c01 / det;
    Minv[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    Minv[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    Minv[6] = c02 / det;
    Minv[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    Minv[8] = (A[0] * A[4] - A[1] * A[3]) / det;
}
static inline void kvec(const Freq& f, size_t v, double xi[3], double xid[3]) {
    const int a = v % f.n[0], b = (v / f.n[0]) % f.n[1], c = v / ((size_t)f.n[0] * f.n[1]);
    xi[0] = f.xi[0][a];
    xi[1] = f.xi[1][b];
    xi[2] = f.xi[2][c];
    xid[0] = f.xid[0][a];
    xid[1] = f.xid[1][b];
    xid[2] = f.xid[2][c];
}

static void fwd(const Freq& f, const double* real, std::vector<cplx>& out, bool naive) {
    out.resize(f.N);
    for (size_t v = 0; v < f.N; ++v) out[v] = cplx(real[v], 0.0);
    fft3d(f.n, out.data(), -1, naive);
}
static void inv_real(const Freq& f, std::vector<cplx>& spec, double* real, bool naive) {
    fft3d(f.n, spec.data(), +1, naive);
    for (size_t v = 0; v < f.N; ++v) real[v] = spec[v].real();
}

// ---------- GND basis ----------
static const double kScrew[6][3] = {{0, 1, -1}, {1, 0, -1}, {1, -1, 0},
                                    {1, 0, 1},  {1, 1, 0},  {0, 1, 1}};
static void gnd_basis(double A[162], double Ap[162]) {
    double s[36], n[36];
    orc_fcc_systems(s, n);
    for (int c = 0; c < 18; ++c) {
        double bb[3], tt[3];
        if (c < 12) {
            const double* b = s + 3 * c;
            const double* nn = n + 3 * c;
            // t = n x b
            tt[0] = nn[1] * b[2] - nn[2] * b[1];
            tt[1] = nn[2] * b[0] - nn[0] * b[2];
            tt[2] = nn[0] * b[1] - nn[1] * b[0];
            for (int i = 0; i < 3; ++i) bb[i] = b[i];
        } else {
            for (int i = 0; i < 3; ++i) bb[i] = tt[i] = kScrew[c - 12][i] / std::sqrt(2.0);
        }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) A[18 * (3 * i + j) + c] = bb[i] * tt[j];
    }
    // Ap = A^T (A A^T)^-1
    double AAt[81];
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 9; ++c) {
            double x = 0;
            for (int k = 0; k < 18; ++k) x += A[18 * r + k] * A[18 * c + k];
            AAt[9 * r + c] = x;
        }
    double G[81];
    for (int c = 0; c < 9; ++c) {
        double M[81], e[9] = {0};
        std::memcpy(M, AAt, sizeof(M));
        e[c] = 1.0;
        solve_dense(9, M, e);
        for (int r = 0; r < 9; ++r) G[9 * r + c] = e[r];
    }
    for (int k = 0; k < 18; ++k)
        for (int c = 0; c < 9; ++c) {
            double x = 0;
            for (int r = 0; r < 9; ++r) x += A[18 * r + k] * G[9 * r + c];
            Ap[9 * k + c] = x;
        }
}

static void gnd_field(const int n[3], double h, const orc_material& m, const double* Qv,
                      const double* Fp, bool naive, double* Lambda, double* rho) {
    const Freq f = make_freq(n, h);
    const size_t N = f.N;
    std::vector<std::vector<cplx>> Fh(9);
    for (int c = 0; c < 9; ++c) fwd(f, Fp + c * N, Fh[c], naive);
    static const int eps[3][3][3] = {{{0, 0, 0}, {0, 0, 1}, {0, -1, 0}},
                                     {{0, 0, -1}, {0, 0, 0}, {1, 0, 0}},
                                     {{0, 1, 0}, {-1, 0, 0}, {0, 0, 0}}};
    std::vector<std::vector<cplx>> Lh(9, std::vector<cplx>(N));
    const double l2 = m.ell_Fp * m.ell_Fp;
    for (size_t v = 0; v < N; ++v) {
        double xi[3], xid[3];
        kvec(f, v, xi, xid);
        const double reg = 1.0 / (1.0 + l2 * (xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]));
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                cplx s(0, 0);
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l)
                        if (eps[j][k][l])
                            s += (double)eps[j][k][l] * cplx(0.0, xid[k]) * Fh[3 * i + l][v];
                Lh[3 * i + j][v] = s * reg;
            }
    }
    for (int c = 0; c < 9; ++c) inv_real(f, Lh[c], Lambda + c * N, naive);
    double A[162], Ap[162];
    gnd_basis(A, Ap);
    for (size_t v = 0; v < N; ++v) {
        M3 Lam{}, Q{};
        for (int c = 0; c < 9; ++c) {
            Lam[c] = Lambda[c * N + v];
            Q[c] = Qv[9 * v + c];
        }
        const M3 LL = mul(tr(Q), mul(Lam, Q));
        double r2 = 0;
        for (int k = 0; k < 18; ++k) {
            double x = 0;
            for (int c = 0; c < 9; ++c) x += Ap[9 * k + c] * LL[c];
            x /= m.b;
            r2 += x * x;
        }
        rho[v] = std::sqrt(r2);
    }
}

// Green preconditioner at one frequency: [xi . Kbar . xi]^-1 (Eq. precf).
static void green(const double* Kbar, const double xi[3], double Minv[9]) {
    double A[9];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) {
            double s = 0;
            for (int j = 0; j < 3; ++j)
                for (int l = 0; l < 3; ++l) s += xi[j] * Kbar[9 * (3 * i + j) + 3 * k + l] * xi[l];
            A[3 * i + k] = s;
        }
    if (xi[0] == 0 && xi[1] == 0 && xi[2] == 0) {
        for (int i = 0; i < 9; ++i) Minv[i] = 0;
        return;
    }
    M3 a;
    for (int i = 0; i < 9; ++i) a[i] = A[i];
    const M3 ai = inv(a);
    for (int i = 0; i < 9; ++i) Minv[i] = ai[i];
}

// Phase-field PCG on (1 + 2S) phi - ell^2 lap(phi) = 2S with M_phi.
static int phase_field(const int n[3], double h, double ell, const double* S,
                       const double* phi_prev, const double* phi_t, double tol, int max_it,
                       bool naive, double* phi, int* iters) {
    const Freq f = make_freq(n, h);
    const size_t N = f.N;
    double smax = 0;
    for (size_t v = 0; v < N; ++v) smax = std::max(smax, S[v]);
    *iters = 0;
    if (smax == 0.0) {
        for (size_t v = 0; v < N; ++v) phi[v] = std::max(0.0, phi_t[v]);
        return 0;
    }
    const double l2 = ell * ell;
    std::vector<double> lap_w(N), pre_w(N);
    for (size_t v = 0; v < N; ++v) {
        double xi[3], xid[3];
        kvec(f, v, xi, xid);
        const double k2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
        lap_w[v] = l2 * k2;
        pre_w[v] = 1.0 / (1.0 + l2 * k2);
    }
    auto spectral = [&](const std::vector<double>& in, const std::vector<double>& w,
                        std::vector<double>& out) {
        std::vector<cplx> sp;
        fwd(f, in.data(), sp, naive);
        for (size_t v = 0; v < N; ++v) sp[v] *= w[v];
        out.resize(N);
        inv_real(f, sp, out.data(), naive);
    };
    auto apply_A = [&](const std::vector<double>& x, std::vector<double>& y) {
        spectral(x, lap_w, y);  // ell^2 (-lap) x
        for (size_t v = 0; v < N; ++v) y[v] += (1.0 + 2.0 * S[v]) * x[v];
    };
    std::vector<double> x(phi_prev, phi_prev + N), r(N), z, p, q;
    apply_A(x, q);
    double bn = 0;
    for (size_t v = 0; v < N; ++v) {
        r[v] = 2.0 * S[v] - q[v];
        bn += 4.0 * S[v] * S[v];
    }
    bn = std::sqrt(bn);
    auto nrm = [&](const std::vector<double>& a) {
        double s = 0;
        for (size_t v = 0; v < N; ++v) s += a[v] * a[v];
        return std::sqrt(s);
    };
    int it = 0, status = 0;
    if (nrm(r) > tol * bn) {
        spectral(r, pre_w, z);
        p = z;
        double rz = 0;
        for (size_t v = 0; v < N; ++v) rz += r[v] * z[v];
        status = 1;
        for (it = 1; it <= max_it; ++it) {
            apply_A(p, q);
            double pq = 0;
            for (size_t v = 0; v < N; ++v) pq += p[v] * q[v];
            const double alpha = rz / pq;
            for (size_t v = 0; v < N; ++v) {
                x[v] += alpha * p[v];
                r[v] -= alpha * q[v];
            }
            if (nrm(r) <= tol * bn) {
                status = 0;
                break;
            }
            spectral(r, pre_w, z);
            double rz2 = 0;
            for (size_t v = 0; v < N; ++v) rz2 += r[v] * z[v];
            const double beta = rz2 / rz;
            rz = rz2;
            for (size_t v = 0; v < N; ++v) p[v] = z[v] + beta * p[v];
        }
        if (it > max_it) it = max_it;
    }
    *iters = it;
    for (size_t v = 0; v < N; ++v) phi[v] = std::max(x[v], phi_t[v]);  // irreversibility
    return status;
}

}  // namespace orc

using namespace orc;

// ---------- the RVE object ----------
enum { ST_NEW = 0, ST_APPLIED = 1, ST_EQUIL = 2, ST_DAMAGE = 3, ST_COMMITTED = 4 };

struct orc_rve {
    int n[3];
    size_t N;
    double h;
    orc_material m;
    orc_options o;
    Freq f;
    std::vector<double> Qv;  // 9N per voxel rotation
    std::vector<uint8_t> elastic;
    // state
    std::vector<double> F, Ft, Fprev, FpLt, rho_t, Wp_t, Gs_t, Hmax_t, Wcrit_t, gam_t;
    std::vector<double> phi, phi_t, rho_gnd;
    // trial history at the current iterate (from the last damage update)
    std::vector<double> FpL_tr, rho_tr, Wp_tr, Gs_tr, Hmax_tr, Wcrit_tr, gam_tr, drive, We, Pund;
    double Fbar_t[9], Fbar[9], dt;
    bool mixed = false;  // mixed stress/strain control (orc_apply_increment_mixed)
    int mask[9] = {0};
    double Pstar[9] = {0};
    // mean degraded stress <g P> at the last damage update, and the committed
    // macroscopic stress: the target on stress-controlled components, the
    // mean on the others (the start of a halved stress path under cut-back)
    double Pbar_cur[9] = {0}, Pbar_t[9] = {0};
    int state, stag_it;
    bool phi_changed, skipped, converged;
};

static void rotate_fp_to_sample(const orc_rve* r, const std::vector<double>& FpL, std::vector<double>& Fps) {
    const size_t N = r->N;
    Fps.assign(9 * N, 0.0);
    for (size_t v = 0; v < N; ++v) {
        M3 Q, A;
        for (int c = 0; c < 9; ++c) {
            Q[c] = r->Qv[9 * v + c];
            A[c] = FpL[c * N + v];
        }
        const M3 B = mul(Q, mul(A, tr(Q)));
        for (int c = 0; c < 9; ++c) Fps[c * N + v] = B[c];
    }
}

static M3 voxel9(const std::vector<double>& a, size_t N, size_t v) {
    M3 x;
    for (int c = 0; c < 9; ++c) x[c] = a[c * N + v];
    return x;
}

static double gdeg(const orc_rve* r, double phi) {
    return (1.0 - phi) * (1.0 - phi) + r->m.k_res;
}

// Constitutive update at every voxel of the current F; fills P (undegraded),
// optionally the tangent, and the trial history.
static int cp_all(orc_rve* r, std::vector<double>* K, bool history) {
    const size_t N = r->N;
    r->Pund.assign(9 * N, 0.0);
    if (K) K->assign(81 * N, 0.0);
    std::vector<int> fails(N, 0);
    parallel_for((int)N, [&](int vi) {
        const size_t v = (size_t)vi;
        M3 Q;
        for (int c = 0; c < 9; ++c) Q[c] = r->Qv[9 * v + c];
        orc_cp_result res;
        fails[v] = cp_point(r->m, Q, voxel9(r->F, N, v), voxel9(r->FpLt, N, v), r->rho_t[v],
                            r->rho_gnd[v], r->dt, r->elastic[v] != 0, r->o.tol_local,
                            r->o.max_local, K != nullptr, res);
        for (int c = 0; c < 9; ++c) r->Pund[c * N + v] = res.P[c];
        if (K)
            for (int c = 0; c < 81; ++c) (*K)[81 * v + c] = res.K[c];
        if (history) {
            for (int c = 0; c < 9; ++c) r->FpL_tr[c * N + v] = res.Fp_L[c];
            const double rho_new = r->rho_t[v] + res.drho_ssd;
            r->rho_tr[v] = rho_new;
            r->Wp_tr[v] = r->Wp_t[v] + res.dWp;
            r->Gs_tr[v] = r->Gs_t[v] + r->m.xi_store * res.dWp / std::sqrt(rho_new + r->rho_gnd[v]);
            r->Hmax_tr[v] = std::max(r->Hmax_t[v], res.We_plus);
            for (int a = 0; a < 12; ++a)
                r->gam_tr[a * N + v] = r->gam_t[a * N + v] + std::fabs(res.dgamma[a]);
            double wc = r->Wcrit_t[v];
            if (wc == 0.0 && r->Gs_tr[v] >= r->m.G_crit) wc = r->Hmax_tr[v] + r->Wp_tr[v];
            r->Wcrit_tr[v] = wc;
            r->We[v] = res.We_plus;
            r->drive[v] = wc > 0.0 ? std::max(0.0, (res.We_plus + r->Wp_tr[v]) / wc - 1.0) : 0.0;
        }
    });
    int nf = 0;
    for (size_t v = 0; v < N; ++v) nf += fails[v];
    return nf;
}

static double maxabs_diff(const std::vector<double>& a, const std::vector<double>& b) {
    double s = 0;
    for (size_t i = 0; i < a.size(); ++i) s = std::max(s, std::fabs(a[i] - b[i]));
    return s;
}

static void compute_gnd(orc_rve* r) {
    std::vector<double> Fps, Lam(9 * r->N);
    rotate_fp_to_sample(r, r->FpLt, Fps);
    gnd_field(r->n, r->h, r->m, r->Qv.data(), Fps.data(), r->o.use_naive_dft != 0, Lam.data(),
              r->rho_gnd.data());
}

extern "C" {

void orc_gnd_basis(double A[162], double Apinv[162]) { gnd_basis(A, Apinv); }

void orc_green_precond(const double Kbar[81], const double xi[3], double Minv[9]) {
    green(Kbar, xi, Minv);
}

void orc_gnd_field(const int n[3], double h, const orc_material* m, const double* Q_per_voxel,
                   const double* Fp, int naive, double* Lambda, double* rho_gnd) {
    gnd_field(n, h, *m, Q_per_voxel, Fp, naive != 0, Lambda, rho_gnd);
}

int orc_phase_field(const int n[3], double h, double ell, const double* S,
                    const double* phi_prev, const double* phi_t, double tol, int max_it,
                    int naive, double* phi_out, int* iters) {
    return phase_field(n, h, ell, S, phi_prev, phi_t, tol, max_it, naive != 0, phi_out, iters);
}

orc_rve* orc_rve_create(const int n[3], double h, const int32_t* grain_ids, int n_grains,
                        const double* euler, const orc_material* m, const orc_options* o,
                        const double* phi0, const uint8_t* elastic_only) {
    orc_rve* r = new orc_rve();
    for (int d = 0; d < 3; ++d) r->n[d] = n[d];
    r->N = (size_t)n[0] * n[1] * n[2];
    r->h = h;
    r->m = *m;
    r->o = *o;
    if (o->n_threads > 0) set_threads(o->n_threads);
    r->f = make_freq(n, h);
    const size_t N = r->N;
    std::vector<double> Qg(9 * (size_t)n_grains);
    for (int g = 0; g < n_grains; ++g) orc_euler_to_Q(euler + 3 * g, Qg.data() + 9 * g);
    r->Qv.resize(9 * N);
    for (size_t v = 0; v < N; ++v)
        for (int c = 0; c < 9; ++c) r->Qv[9 * v + c] = Qg[9 * grain_ids[v] + c];
    r->elastic.assign(N, 0);
    if (elastic_only)
        for (size_t v = 0; v < N; ++v) r->elastic[v] = elastic_only[v];
    auto eye_field = [&](std::vector<double>& a) {
        a.assign(9 * N, 0.0);
        for (size_t v = 0; v < N; ++v) a[0 * N + v] = a[4 * N + v] = a[8 * N + v] = 1.0;
    };
    eye_field(r->F);
    eye_field(r->Ft);
    eye_field(r->Fprev);
    eye_field(r->FpLt);
    eye_field(r->FpL_tr);
    r->rho_t.assign(N, m->rho_ssd0);
    r->rho_tr = r->rho_t;
    for (auto* a : {&r->Wp_t, &r->Gs_t, &r->Hmax_t, &r->Wcrit_t, &r->Wp_tr, &r->Gs_tr,
                    &r->Hmax_tr, &r->Wcrit_tr, &r->drive, &r->We, &r->rho_gnd})
        a->assign(N, 0.0);
    r->gam_t.assign(12 * N, 0.0);
    r->gam_tr = r->gam_t;
    r->phi_t.assign(N, 0.0);
    if (phi0)
        for (size_t v = 0; v < N; ++v) r->phi_t[v] = phi0[v];
    r->phi = r->phi_t;
    r->Pund.assign(9 * N, 0.0);
    const double I9[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    std::memcpy(r->Fbar_t, I9, sizeof(I9));
    std::memcpy(r->Fbar, I9, sizeof(I9));
    r->dt = 0;
    r->state = ST_NEW;
    r->stag_it = 0;
    r->phi_changed = true;
    r->skipped = false;
    r->converged = false;
    return r;
}

void orc_rve_destroy(orc_rve* r) { delete r; }

int orc_commit(orc_rve* r) {
    if (r->state != ST_DAMAGE || !r->converged) return -7;
    r->FpLt = r->FpL_tr;
    r->rho_t = r->rho_tr;
    r->Wp_t = r->Wp_tr;
    r->Gs_t = r->Gs_tr;
    r->Hmax_t = r->Hmax_tr;
    r->Wcrit_t = r->Wcrit_tr;
    r->gam_t = r->gam_tr;
    r->Ft = r->F;
    r->phi_t = r->phi;
    std::memcpy(r->Fbar_t, r->Fbar, sizeof(r->Fbar));
    for (int c = 0; c < 9; ++c) r->Pbar_t[c] = (r->mixed && r->mask[c]) ? r->Pstar[c] : r->Pbar_cur[c];
    r->state = ST_COMMITTED;
    return 0;
}

int orc_apply_increment(orc_rve* r, const double Fbar[9], double dt) {
    if (r->state == ST_DAMAGE && r->converged) orc_commit(r);
    r->mixed = false;
    const size_t N = r->N;
    for (int c = 0; c < 9; ++c) {
        const double d = Fbar[c] - r->Fbar_t[c];
        for (size_t v = 0; v < N; ++v) r->F[c * N + v] = r->Ft[c * N + v] + d;
        r->Fbar[c] = Fbar[c];
    }
    r->phi = r->phi_t;
    r->dt = dt;
    compute_gnd(r);
    r->stag_it = 0;
    r->phi_changed = true;
    r->converged = false;
    r->state = ST_APPLIED;
    return 0;
}

// Newton iteration on the fluctuation at the current macroscopic F (Eq.
// newton with the Krylov solver of Sec. 3.1).
static const int kDampFrom = 4;

static int newton_solve(orc_rve* r, orc_stats* st) {
    const size_t N = r->N;
    const bool naive = r->o.use_naive_dft != 0;
    const Freq& f = r->f;
    std::vector<double> K;
    std::vector<double> Ks(81 * N), Pg(9 * N);
    // derivative symbols: i xi_j (spectral, Nyquist dropped) or Willot's D_j
    // for the gradient; i xi_j or -conj(D_j) for the divergence
    const bool willot = r->o.derivative == 1;
    auto dsym = [&](size_t v, int j) -> cplx {
        if (willot) {
            cplx D[3];
            willot_symbol(f, v, D);
            return D[j];
        }
        double xi[3], xid[3];
        kvec(f, v, xi, xid);
        return cplx(0.0, xid[j]);
    };
    auto dsym_div = [&](size_t v, int j) -> cplx {
        return willot ? -std::conj(dsym(v, j)) : dsym(v, j);
    };
    int status = -5;
    double alpha = 1.0, prev_ratio = 0.0;
    for (int it = 0; it < r->o.max_newton; ++it) {
        const int nf = cp_all(r, &K, false);
        if (st) {
            st->newton_it += 1;
            st->local_fail += nf;
        }
        double Kbar[81] = {0};
        for (size_t v = 0; v < N; ++v) {
            const double g = gdeg(r, r->phi[v]);
            for (int c = 0; c < 9; ++c) Pg[c * N + v] = g * r->Pund[c * N + v];
            for (int c = 0; c < 81; ++c) {
                Ks[81 * v + c] = g * K[81 * v + c];
                Kbar[c] += Ks[81 * v + c];
            }
        }
        for (int c = 0; c < 81; ++c) Kbar[c] /= (double)N;
        // right-hand side of Eq. newton, sign flipped: b = F{g P} . i xi
        std::vector<std::vector<cplx>> Ph(9);
        for (int c = 0; c < 9; ++c) fwd(f, Pg.data() + c * N, Ph[c], naive);
        std::vector<cplx> bvec[3], x[3];
        for (int i = 0; i < 3; ++i) {
            bvec[i].assign(N, 0.0);
            x[i].assign(N, 0.0);
        }
        std::vector<double> Minv(willot ? 0 : 9 * N);
        std::vector<cplx> MinvW(willot ? 9 * N : 0);
        for (size_t v = 0; v < N; ++v) {
            if (willot) {
                cplx D[3];
                willot_symbol(f, v, D);
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) bvec[i][v] -= Ph[3 * i + j][v] * std::conj(D[j]);
                green_willot(Kbar, D, &MinvW[9 * v]);
                continue;
            }
            double xi[3], xid[3];
            kvec(f, v, xi, xid);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) bvec[i][v] += Ph[3 * i + j][v] * cplx(0.0, xid[j]);
            green(Kbar, xid, &Minv[9 * v]);
        }
        typedef std::array<std::vector<cplx>, 3> Vec3;
        auto precond = [&](const Vec3& in, Vec3& out) {
            for (int i = 0; i < 3; ++i) out[i].assign(N, 0.0);
            for (size_t v = 0; v < N; ++v)
                for (int i = 0; i < 3; ++i)
                    for (int k = 0; k < 3; ++k)
                        out[i][v] += (willot ? MinvW[9 * v + 3 * i + k] : Minv[9 * v + 3 * i + k]) *
                                     in[k][v];
        };
        // A' u = -F{g K : F^-1{u (x) i xi}} . i xi
        auto apply_op = [&](const Vec3& u, Vec3& out) {
            std::vector<double> G(9 * N), T(9 * N);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    std::vector<cplx> s(N);
                    for (size_t v = 0; v < N; ++v) s[v] = u[i][v] * dsym(v, j);
                    inv_real(f, s, G.data() + (3 * i + j) * N, naive);
                }
            for (size_t v = 0; v < N; ++v)
                for (int a = 0; a < 9; ++a) {
                    double s = 0;
                    for (int b = 0; b < 9; ++b) s += Ks[81 * v + 9 * a + b] * G[b * N + v];
                    T[a * N + v] = s;
                }
            std::vector<std::vector<cplx>> Th(9);
            for (int c = 0; c < 9; ++c) fwd(f, T.data() + c * N, Th[c], naive);
            for (int i = 0; i < 3; ++i) out[i].assign(N, 0.0);
            for (size_t v = 0; v < N; ++v)
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) out[i][v] -= Th[3 * i + j][v] * dsym_div(v, j);
        };
        auto dot = [&](const Vec3& a, const Vec3& b) {
            double s = 0;
            for (int i = 0; i < 3; ++i)
                for (size_t v = 0; v < N; ++v)
                    s += a[i][v].real() * b[i][v].real() + a[i][v].imag() * b[i][v].imag();
            return s;
        };
        // Restarted GMRES with right preconditioning (Krylov solver of
        // Sec. 3.1): minimises ||b - A' M y|| over the Krylov space of A' M,
        // x = M y.  Modified Gram-Schmidt, Givens rotations.
        Vec3 bv, xs;
        for (int i = 0; i < 3; ++i) {
            bv[i] = bvec[i];
            xs[i].assign(N, 0.0);
        }
        const double bn = std::sqrt(dot(bv, bv));
        // round-off scale of b: ||F{gP}_ij xi_j|| before the sum over j
        double pn = 0;
        for (size_t v = 0; v < N; ++v)
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) pn += std::norm(Ph[3 * i + j][v]) * std::norm(dsym(v, j));
        pn = std::sqrt(pn);
        const double target = std::max(r->o.tol_lin * bn, 1e-12 * pn);
        int lin_it = 0;
        bool ok = bn <= target;
        const int mres = std::max(1, r->o.restart);
        while (!ok && lin_it < r->o.max_lin) {
            Vec3 rv, tmp;
            apply_op(xs, tmp);
            for (int i = 0; i < 3; ++i) {
                rv[i].resize(N);
                for (size_t v = 0; v < N; ++v) rv[i][v] = bv[i][v] - tmp[i][v];
            }
            const double beta = std::sqrt(dot(rv, rv));
            if (beta <= target) {
                ok = true;
                break;
            }
            std::vector<Vec3> V(1);
            for (int i = 0; i < 3; ++i) {
                V[0][i].resize(N);
                for (size_t v = 0; v < N; ++v) V[0][i][v] = rv[i][v] / beta;
            }
            std::vector<std::vector<double>> H(mres + 1, std::vector<double>(mres, 0.0));
            std::vector<double> cs(mres), sn(mres), g(mres + 1, 0.0);
            g[0] = beta;
            int k = 0;
            for (; k < mres && lin_it < r->o.max_lin; ++k) {
                ++lin_it;
                Vec3 z, w;
                precond(V[k], z);
                apply_op(z, w);
                for (int i = 0; i <= k; ++i) {
                    H[i][k] = dot(w, V[i]);
                    for (int c = 0; c < 3; ++c)
                        for (size_t v = 0; v < N; ++v) w[c][v] -= H[i][k] * V[i][c][v];
                }
                H[k + 1][k] = std::sqrt(dot(w, w));
                V.emplace_back();
                for (int c = 0; c < 3; ++c) {
                    V[k + 1][c].resize(N);
                    for (size_t v = 0; v < N; ++v)
                        V[k + 1][c][v] = H[k + 1][k] > 0 ? w[c][v] / H[k + 1][k] : 0.0;
                }
                for (int i = 0; i < k; ++i) {
                    const double t = cs[i] * H[i][k] + sn[i] * H[i + 1][k];
                    H[i + 1][k] = -sn[i] * H[i][k] + cs[i] * H[i + 1][k];
                    H[i][k] = t;
                }
                const double den = std::hypot(H[k][k], H[k + 1][k]);
                cs[k] = den > 0 ? H[k][k] / den : 1.0;
                sn[k] = den > 0 ? H[k + 1][k] / den : 0.0;
                H[k][k] = den;
                H[k + 1][k] = 0.0;
                g[k + 1] = -sn[k] * g[k];
                g[k] = cs[k] * g[k];
                if (std::getenv("ORACLE_VERBOSE") && (lin_it % 25 == 0 || lin_it < 5))
                    std::fprintf(stderr, "  gmres it %d  |r|/|b| %.3e  (|b| %.3e)\n", lin_it,
                                 std::fabs(g[k + 1]) / bn, bn);
                if (std::fabs(g[k + 1]) <= target) {
                    ++k;
                    ok = true;
                    break;
                }
            }
            // y = H^-1 g (upper triangular), x += M sum y_i V_i
            std::vector<double> y(k, 0.0);
            for (int i = k - 1; i >= 0; --i) {
                double s = g[i];
                for (int j = i + 1; j < k; ++j) s -= H[i][j] * y[j];
                y[i] = s / H[i][i];
            }
            Vec3 comb, dx;
            for (int c = 0; c < 3; ++c) {
                comb[c].assign(N, 0.0);
                for (int i = 0; i < k; ++i)
                    for (size_t v = 0; v < N; ++v) comb[c][v] += y[i] * V[i][c][v];
            }
            precond(comb, dx);
            for (int c = 0; c < 3; ++c)
                for (size_t v = 0; v < N; ++v) xs[c][v] += dx[c][v];
        }
        if (st) st->lin_it_total += lin_it;
        if (!ok) return -5;
        for (int i = 0; i < 3; ++i) x[i] = xs[i];
        // Newton update F += grad(du) (Eq. fdef), test of Sec. 3.1
        double gmax = 0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                std::vector<cplx> s(N);
                for (size_t v = 0; v < N; ++v) s[v] = x[i][v] * dsym(v, j);
                std::vector<double> g(N);
                inv_real(f, s, g.data(), naive);
                for (size_t v = 0; v < N; ++v) {
                    r->F[(3 * i + j) * N + v] += alpha * g[v];
                    gmax = std::max(gmax, std::fabs(g[v]));
                }
            }
        const double dF = std::max(maxabs_diff(r->F, r->Ft), 1e-30);
        const double ratio = gmax / dF;
        if (std::getenv("ORACLE_VERBOSE"))
            std::fprintf(stderr, "newton %d |b| %.3e lin %d gmax %.3e ratio %.3e alpha %.4f\n",
                         it, bn, lin_it, gmax, ratio, alpha);
        if (ratio < r->o.tol_newton) {
            status = 0;
            break;
        }
        // Damping (an extension; the paper's Newton takes full steps): from
        // the kDampFrom-th iteration on, an update after which the ratio did
        // not fall halves the length of the next (down to 1/16); one that
        // halved the ratio doubles it back (up to a full step).  This breaks
        // the two-cycles a kink in the slip law's tangent can trap Newton
        // in; a Newton iteration whose ratio keeps falling is untouched.
        if (it + 1 >= kDampFrom && ratio >= prev_ratio)
            alpha = std::max(0.5 * alpha, 1.0 / 16);
        else if (ratio < 0.5 * prev_ratio)
            alpha = std::min(2.0 * alpha, 1.0);
        prev_ratio = ratio;
    }
    return status;
}

// Solve the n x n system A x = b (row-major) by Gaussian elimination with
// partial pivoting; false if singular.
static bool dense_solve(int n, std::vector<double> A, std::vector<double>& b) {
    for (int c = 0; c < n; ++c) {
        int p = c;
        for (int r2 = c + 1; r2 < n; ++r2)
            if (std::fabs(A[r2 * n + c]) > std::fabs(A[p * n + c])) p = r2;
        if (A[p * n + c] == 0.0) return false;
        if (p != c) {
            for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[p * n + k]);
            std::swap(b[c], b[p]);
        }
        for (int r2 = c + 1; r2 < n; ++r2) {
            const double m = A[r2 * n + c] / A[c * n + c];
            for (int k = c; k < n; ++k) A[r2 * n + k] -= m * A[c * n + k];
            b[r2] -= m * b[c];
        }
    }
    for (int c = n - 1; c >= 0; --c) {
        double v = b[c];
        for (int k = c + 1; k < n; ++k) v -= A[c * n + k] * b[k];
        b[c] = v / A[c * n + c];
    }
    return true;
}

int orc_solve_equilibrium(orc_rve* r, orc_stats* st) {
    if (r->state != ST_APPLIED && r->state != ST_DAMAGE) return -7;
    const size_t N = r->N;
    r->Fprev = r->F;
    r->skipped = false;
    r->state = ST_EQUIL;
    if (r->stag_it >= 1 && !r->phi_changed) {
        r->skipped = true;
        if (st) st->skipped_equilibrium = 1;
        return 0;
    }
    for (int outer = 0;; ++outer) {
        const int s = newton_solve(r, st);
        if (s) return s;
        if (!r->mixed) return 0;
        // mixed control: <gP> and Kbar = <gK> at the converged F, then a
        // Newton step on the stress-controlled macroscopic components
        std::vector<double> K;
        const int nf = cp_all(r, &K, false);
        if (st) st->local_fail += nf;
        double Pbar[9] = {0}, Kbar[81] = {0};
        for (size_t v = 0; v < N; ++v) {
            const double g = gdeg(r, r->phi[v]);
            for (int c = 0; c < 9; ++c) Pbar[c] += g * r->Pund[c * N + v];
            for (int c = 0; c < 81; ++c) Kbar[c] += g * K[81 * v + c];
        }
        double pmax = 0, res = 0;
        int S[9], ns = 0;
        for (int c = 0; c < 9; ++c) {
            Pbar[c] /= (double)N;
            pmax = std::max(pmax, std::fabs(Pbar[c]));
            if (r->mask[c]) {
                S[ns++] = c;
                res = std::max(res, std::fabs(Pbar[c] - r->Pstar[c]));
            }
        }
        for (int c = 0; c < 81; ++c) Kbar[c] /= (double)N;
        if (st) st->mixed_it = outer + 1;
        if (std::getenv("ORACLE_VERBOSE"))
            std::fprintf(stderr, "mixed %d |Pbar - P*|_S %.3e (max|Pbar| %.3e)\n", outer, res,
                         pmax);
        if (res <= r->o.tol_newton * std::max(pmax, 1.0)) return 0;
        if (outer + 1 >= r->o.max_newton) return -5;
        std::vector<double> A(ns * ns), d(ns);
        for (int a = 0; a < ns; ++a) {
            d[a] = -(Pbar[S[a]] - r->Pstar[S[a]]);
            for (int b = 0; b < ns; ++b) A[a * ns + b] = Kbar[9 * S[a] + S[b]];
        }
        if (!dense_solve(ns, A, d)) return -6;
        for (int a = 0; a < ns; ++a) {
            const int c = S[a];
            r->Fbar[c] += d[a];
            for (size_t v = 0; v < N; ++v) r->F[c * N + v] += d[a];
        }
    }
}

int orc_update_damage(orc_rve* r, orc_stats* st) {
    if (r->state != ST_EQUIL) return -7;
    const size_t N = r->N;
    r->stag_it += 1;
    if (st) st->stag_it = r->stag_it;
    r->state = ST_DAMAGE;
    if (r->skipped) {
        r->converged = true;
        if (st) {
            st->res_F = 0;
            st->res_phi = 0;
            st->converged = 1;
        }
        return 0;
    }
    const int nf = cp_all(r, nullptr, true);
    if (st) st->local_fail += nf;
    std::vector<double> phi_new(N);
    int pf_it = 0;
    const int s = phase_field(r->n, r->h, r->m.ell, r->drive.data(), r->phi.data(),
                              r->phi_t.data(), r->o.tol_pf, r->o.max_pf,
                              r->o.use_naive_dft != 0, phi_new.data(), &pf_it);
    if (st) st->pf_it_total += pf_it;
    if (s != 0) return -5;
    const double dphi = maxabs_diff(phi_new, r->phi);
    const double dphit = maxabs_diff(phi_new, r->phi_t);
    const double dF = maxabs_diff(r->F, r->Fprev);
    const double dFt = maxabs_diff(r->F, r->Ft);
    r->phi_changed = false;
    for (size_t v = 0; v < N; ++v)
        if (phi_new[v] != r->phi[v]) {
            r->phi_changed = true;
            break;
        }
    r->phi = phi_new;
    const bool cF = dF <= r->o.tol_stag * std::max(dFt, 1e-12);
    const bool cP = dphi <= r->o.tol_stag * std::max(dphit, 1e-12);
    r->converged = cF && cP;
    for (int c = 0; c < 9; ++c) {
        double s2 = 0;
        for (size_t v = 0; v < N; ++v) s2 += gdeg(r, r->phi[v]) * r->Pund[c * N + v];
        r->Pbar_cur[c] = s2 / (double)N;
    }
    if (st) {
        st->res_F = dF / std::max(dFt, 1e-12);
        st->res_phi = dphi / std::max(dphit, 1e-12);
        st->converged = r->converged;
        for (int c = 0; c < 9; ++c) st->Pbar[c] = r->Pbar_cur[c];
        long cr = 0;
        for (size_t v = 0; v < N; ++v) cr += r->phi[v] >= 0.9;
        st->cracked = cr;
        std::memcpy(st->Fbar, r->Fbar, sizeof(r->Fbar));
    }
    return 0;
}

int orc_apply_increment_mixed(orc_rve* r, const double Fbar[9], const double Pstar[9],
                              const int mask[9], double dt) {
    const int s = orc_apply_increment(r, Fbar, dt);
    if (s) return s;
    int ns = 0;
    for (int c = 0; c < 9; ++c) {
        r->mask[c] = mask[c] ? 1 : 0;
        r->Pstar[c] = Pstar ? Pstar[c] : 0.0;
        ns += r->mask[c];
    }
    r->mixed = ns > 0;
    return 0;
}

static int run_loop(orc_rve* r, orc_stats* st) {
    for (int i = 0; i < r->o.max_stag; ++i) {
        int s = orc_solve_equilibrium(r, st);
        if (s) return s;
        s = orc_update_damage(r, st);
        if (s) return s;
        if (r->converged) return orc_commit(r);
    }
    return -5;
}

// One attempt at an increment, committed when converged; mask = nullptr is
// strain control.
static int attempt(orc_rve* r, const double Fbar[9], const double* Pstar, const int* mask,
                   double dt, orc_stats* st) {
    const int s = mask ? orc_apply_increment_mixed(r, Fbar, Pstar, mask, dt)
                       : orc_apply_increment(r, Fbar, dt);
    if (s) return s;
    return run_loop(r, st);
}

// Cut-back (an extension of Algorithm 1, off unless max_cutbacks > 0): an
// increment that does not converge is redone from the committed state as two
// halves of the load step, each half taking half of the change: the first
// to the midpoint of the committed and the requested macroscopic F and, on
// stress-controlled components, to the midpoint of the committed and the
// requested stress; the second to the request, with its stress-controlled
// components of F started from the solved midpoint.  Each half is halved
// again on failure, down to depth max_cutbacks.
static int halves(orc_rve* r, const double Fbar[9], const double* Pstar, const int* mask,
                  double dt, orc_stats* st, int depth) {
    if (st) st->cutbacks += 1;
    double mid[9], last[9], Pmid[9];
    for (int c = 0; c < 9; ++c) {
        mid[c] = 0.5 * (r->Fbar_t[c] + Fbar[c]);
        const double Pc = Pstar ? Pstar[c] : 0.0;
        Pmid[c] = (mask && mask[c]) ? 0.5 * (r->Pbar_t[c] + Pc) : Pc;
    }
    int s = attempt(r, mid, Pmid, mask, 0.5 * dt, st);
    if (s == -5 && depth < r->o.max_cutbacks) s = halves(r, mid, Pmid, mask, 0.5 * dt, st, depth + 1);
    if (s) return s;
    for (int c = 0; c < 9; ++c) last[c] = (mask && mask[c]) ? r->Fbar_t[c] : Fbar[c];
    s = attempt(r, last, Pstar, mask, 0.5 * dt, st);
    if (s == -5 && depth < r->o.max_cutbacks) s = halves(r, last, Pstar, mask, 0.5 * dt, st, depth + 1);
    return s;
}

static int run_with_cutbacks(orc_rve* r, const double Fbar[9], const double* Pstar,
                             const int* mask, double dt, orc_stats* st) {
    if (st) std::memset(st, 0, sizeof(*st));
    const int s = attempt(r, Fbar, Pstar, mask, dt, st);
    if (s != -5 || r->o.max_cutbacks <= 0) return s;
    return halves(r, Fbar, Pstar, mask, dt, st, 1);
}

int orc_run_increment_mixed(orc_rve* r, const double Fbar[9], const double Pstar[9],
                            const int mask[9], double dt, orc_stats* st) {
    return run_with_cutbacks(r, Fbar, Pstar, mask, dt, st);
}

int orc_run_increment(orc_rve* r, const double Fbar[9], double dt, orc_stats* st) {
    return run_with_cutbacks(r, Fbar, nullptr, nullptr, dt, st);
}

int orc_fields_out(const orc_rve* r, int field, double* dst) {
    const size_t N = r->N;
    auto cp = [&](const std::vector<double>& a) { std::memcpy(dst, a.data(), a.size() * 8); };
    switch (field) {
        case ORC_FIELD_F: cp(r->F); break;
        case ORC_FIELD_FT: cp(r->Ft); break;
        case ORC_FIELD_P:
            for (int c = 0; c < 9; ++c)
                for (size_t v = 0; v < N; ++v)
                    dst[c * N + v] = gdeg(r, r->phi[v]) * r->Pund[c * N + v];
            break;
        case ORC_FIELD_PHI: cp(r->phi); break;
        case ORC_FIELD_PHI_T: cp(r->phi_t); break;
        case ORC_FIELD_FP: {
            std::vector<double> Fps;
            rotate_fp_to_sample(r, r->FpLt, Fps);
            cp(Fps);
            break;
        }
        case ORC_FIELD_RHO_SSD: cp(r->rho_t); break;
        case ORC_FIELD_RHO_GND: cp(r->rho_gnd); break;
        case ORC_FIELD_WP: cp(r->Wp_t); break;
        case ORC_FIELD_GS: cp(r->Gs_t); break;
        case ORC_FIELD_HMAX: cp(r->Hmax_t); break;
        case ORC_FIELD_WCRIT: cp(r->Wcrit_t); break;
        case ORC_FIELD_DRIVE: cp(r->drive); break;
        case ORC_FIELD_GAMMA: cp(r->gam_t); break;
        case ORC_FIELD_WE: cp(r->We); break;
        default: return -1;
    }
    return 0;
}

int orc_fields_in(orc_rve* r, int field, const double* src) {
    const size_t N = r->N;
    auto cp = [&](std::vector<double>& a) { std::memcpy(a.data(), src, a.size() * 8); };
    switch (field) {
        case ORC_FIELD_F: cp(r->F); break;
        case ORC_FIELD_FT: cp(r->Ft); break;
        case ORC_FIELD_PHI: cp(r->phi); break;
        case ORC_FIELD_PHI_T: cp(r->phi_t); break;
        case ORC_FIELD_FP:
            for (size_t v = 0; v < N; ++v) {
                M3 Q, A;
                for (int c = 0; c < 9; ++c) {
                    Q[c] = r->Qv[9 * v + c];
                    A[c] = src[c * N + v];
                }
                const M3 B = mul(tr(Q), mul(A, Q));
                for (int c = 0; c < 9; ++c) r->FpLt[c * N + v] = B[c];
            }
            break;
        case ORC_FIELD_RHO_SSD: cp(r->rho_t); break;
        case ORC_FIELD_WP: cp(r->Wp_t); break;
        case ORC_FIELD_GS: cp(r->Gs_t); break;
        case ORC_FIELD_HMAX: cp(r->Hmax_t); break;
        case ORC_FIELD_WCRIT: cp(r->Wcrit_t); break;
        case ORC_FIELD_GAMMA: cp(r->gam_t); break;
        default: return -1;
    }
    return 0;
}

}  // extern "C"
