// Constitutive kernel (K-CP): crystal-plasticity update, consistent tangent
// and, optionally, tensile elastic energy, driving force and trial history,
// one voxel per thread.  Sec. 2.1 (Eqs. 1, flowrule, Taylor hardening, SSD
// evolution), Sec. 2.3 (stored energy density, Eqs. crit, decMiehe, zeta),
// Eq. newton (consistent tangent K = dP/dF).
#include "cp.cuh"
#include "launch.h"

namespace fatfft {

// 6x6 LU with partial pivoting (row stride 6); perm records the row swaps.
template <typename R>
__device__ void lu6(R* A, int* perm) {
    for (int c = 0; c < 6; ++c) {
        int piv = c;
        R best = fabs(A[6 * c + c]);
        for (int r = c + 1; r < 6; ++r)
            if (fabs(A[6 * r + c]) > best) {
                best = fabs(A[6 * r + c]);
                piv = r;
            }
        perm[c] = piv;
        if (piv != c)
            for (int k = 0; k < 6; ++k) {
                const R t = A[6 * c + k];
                A[6 * c + k] = A[6 * piv + k];
                A[6 * piv + k] = t;
            }
        const R inv = R(1) / A[6 * c + c];
        for (int r = c + 1; r < 6; ++r) {
            const R f = A[6 * r + c] * inv;
            A[6 * r + c] = f;
            for (int k = c + 1; k < 6; ++k) A[6 * r + k] -= f * A[6 * c + k];
        }
    }
}
template <typename R>
__device__ void lu6_solve(const R* A, const int* perm, R* b) {
    for (int c = 0; c < 6; ++c)
        if (perm[c] != c) {
            const R t = b[c];
            b[c] = b[perm[c]];
            b[perm[c]] = t;
        }
    for (int r = 1; r < 6; ++r)
        for (int k = 0; k < r; ++k) b[r] -= A[6 * r + k] * b[k];
    for (int r = 5; r >= 0; --r) {
        R s = b[r];
        for (int k = r + 1; k < 6; ++k) s -= A[6 * r + k] * b[k];
        b[r] = s / A[6 * r + r];
    }
}

// Resident CTAs per SM the register allocation is sized for.  The kernel is
// latency-bound at low occupancy: in FP32, three CTAs (168 registers, no
// spills) run it 12 % faster than the unconstrained 221 registers; the FP64
// instantiation spills heavily under that cap and keeps one.
template <typename R> struct CPMinBlocks { static constexpr int v = sizeof(R) == 4 ? 3 : 1; };

template <typename R, bool HIST>
__global__ void __launch_bounds__(128, CPMinBlocks<R>::v) k_constitutive(CPFields f, CPParams p) {
    const R C11 = (R)p.C11, C12 = (R)p.C12, C44 = (R)p.C44;
    const R sT = (R)p.sT, c = (R)(p.dt * p.g0), tol = (R)p.tol_local;
    const size_t N = f.N;
    const R* H = (const R*)f.H;
    const R* Hpi = (const R*)f.Hpi;
    const R* rg = (const R*)f.rho_gnd;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < N;
         v += (size_t)gridDim.x * blockDim.x) {
        const int g = f.grain[v];
        R Q[9], Hs[9], A[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            Q[k] = (R)f.Qg[9 * g + k];
            Hs[k] = H[k * N + v];
            A[k] = Hpi[k * N + v];
        }
        const bool elastic = f.elastic ? f.elastic[v] != 0 : false;
        const double rho_n = f.hist_c[0 * N + v] + f.hist_c[1 * N + v];
        const R rgnd = rg[v];
        const R tau_c = (R)(p.tau_c0 + p.mu_b * sqrt(rho_n + (double)rgnd));
        // lattice frame: F_L - I = Q^T H Q;  Fe* - I = HL + Hpi + HL Hpi
        R T1[9], HL[9], Hes[9];
        mtm3(Q, Hs, T1);
        mm3(T1, Q, HL);
        mm3(HL, A, T1);
#pragma unroll
        for (int k = 0; k < 9; ++k) Hes[k] = HL[k] + A[k] + T1[k];

        LocalState<R> st;
        R dg[12], da[12];
        int iters = 0;
        const bool ok = local_solve(Hes, tau_c, c, sT, C11, C12, C44, tol, p.max_local, elastic,
                                    st, dg, da, &iters);
        if (!ok && f.fail_count) atomicAdd(f.fail_count, 1);

        // Fp^-1 = (I + Hpi)(I - dL);  Fe = I + He;  Fe* = I + Hes
        R Fpi[9], Fe[9], Fes[9], Am[9], AdL[9];
        mm3(A, st.dL, AdL);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const R id = (k % 4 == 0) ? R(1) : R(0);
            Fpi[k] = id + A[k] - st.dL[k] - AdL[k];
            Fe[k] = id + st.He[k];
            Fes[k] = id + Hes[k];
            Am[k] = id + A[k];
        }
        // P_L = Fe S Fp^-T ; P = Q P_L Q^T
        R SFpT[9], PL[9], Ps[9];
        mmt3(st.S, Fpi, SFpT);
        mm3(Fe, SFpT, PL);
        mm3(Q, PL, T1);
        mmt3(T1, Q, Ps);
        R* P = (R*)f.P;
#pragma unroll
        for (int k = 0; k < 9; ++k) P[k * N + v] = Ps[k];

        if (f.K) {
            // J6 = I + sum_a da_a voigt(B^a) (w o voigt(sym P^a))^T at the solution
            R X[9];
            mtm3(Fe, Fes, X);
            R J[36];
            int perm[6];
#pragma unroll
            for (int k = 0; k < 36; ++k) J[k] = (k % 7 == 0) ? R(1) : R(0);
            for (int a = 0; a < 12; ++a) {
                if (da[a] == R(0)) continue;
                R B[9];
                bmat(X, a, C11, C12, C44, B);
                R pv[6];
#pragma unroll
                for (int m = 0; m < 6; ++m) {
                    const int i = voigt_i(m), j = voigt_j(m);
                    const R psym = R(0.5) * (slip_s<R>(a, i) * slip_n<R>(a, j) +
                                             slip_s<R>(a, j) * slip_n<R>(a, i));
                    pv[m] = (m < 3 ? R(1) : R(2)) * psym;
                }
#pragma unroll
                for (int r = 0; r < 6; ++r) {
                    const R br = da[a] * B[3 * voigt_i(r) + voigt_j(r)];
#pragma unroll
                    for (int cc = 0; cc < 6; ++cc) J[6 * r + cc] += br * pv[cc];
                }
            }
            lu6(J, perm);
            R X1[9], FeS[9];
            mm3(Fpi, SFpT, X1);  // Fp^-1 S Fp^-T
            mm3(Fe, st.S, FeS);
            R* K = (R*)f.K;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) {
                    // sample direction e_k (x) e_l -> lattice q_k (x) q_l, q_k = Q^T e_k
                    R dF[9];
#pragma unroll
                    for (int a = 0; a < 3; ++a)
#pragma unroll
                        for (int b = 0; b < 3; ++b) dF[3 * a + b] = Q[3 * k + a] * Q[3 * l + b];
                    R T[9], U[9], E[9], Sv[9];
                    mm3(dF, Fpi, T);
                    mtm3(Fe, T, U);
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int j = 0; j < 3; ++j)
                            E[3 * i + j] = R(0.5) * (U[3 * i + j] + U[3 * j + i]);
                    cubic_apply(C11, C12, C44, E, Sv);
                    R rhs[6];
#pragma unroll
                    for (int m = 0; m < 6; ++m) rhs[m] = Sv[3 * voigt_i(m) + voigt_j(m)];
                    lu6_solve(J, perm, rhs);
                    R dS[9];
#pragma unroll
                    for (int m = 0; m < 6; ++m) {
                        dS[3 * voigt_i(m) + voigt_j(m)] = rhs[m];
                        dS[3 * voigt_j(m) + voigt_i(m)] = rhs[m];
                    }
                    R dM[9];
#pragma unroll
                    for (int q = 0; q < 9; ++q) dM[q] = 0;
                    for (int a = 0; a < 12; ++a) {
                        if (da[a] == R(0)) continue;
                        const R co = -da[a] * resolve(dS, a);
#pragma unroll
                        for (int i = 0; i < 3; ++i)
#pragma unroll
                            for (int j = 0; j < 3; ++j)
                                dM[3 * i + j] += co * slip_s<R>(a, i) * slip_n<R>(a, j);
                    }
                    // dP_L = dF X1 + Fe* dM S Fp^-T + Fe dS Fp^-T + Fe S dM^T A^T
                    R dP[9], W1[9], W2[9];
                    mm3(dF, X1, dP);
                    mm3(Fes, dM, W1);
                    mm3(W1, SFpT, W2);
#pragma unroll
                    for (int q = 0; q < 9; ++q) dP[q] += W2[q];
                    mm3(Fe, dS, W1);
                    mmt3(W1, Fpi, W2);
#pragma unroll
                    for (int q = 0; q < 9; ++q) dP[q] += W2[q];
                    mmt3(FeS, dM, W1);
                    mmt3(W1, Am, W2);
#pragma unroll
                    for (int q = 0; q < 9; ++q) dP[q] += W2[q];
                    // back to the sample frame
                    mm3(Q, dP, W1);
                    mmt3(W1, Q, W2);
                    const int kl = 3 * k + l;
#pragma unroll
                    for (int ij = 0; ij < 9; ++ij) K[(size_t)(9 * ij + kl) * N + v] = W2[ij];
                }
        }

        if (HIST) {
            // plastic work, SSD increment, stored energy, W_e+, W_crit, S
            R dWp = 0, dLL = 0;
#pragma unroll
            for (int a = 0; a < 12; ++a) dWp += st.tau[a] * dg[a];
#pragma unroll
            for (int k = 0; k < 9; ++k) dLL += st.dL[k] * st.dL[k];
            const double drho = p.lambda_h * sqrt(2.0 / 3.0 * (double)dLL);
            const double* hc = f.hist_c;
            double* ht = f.hist_tr;
            double rs = hc[0 * N + v], rc = hc[1 * N + v];
            double ws = hc[2 * N + v], wc = hc[3 * N + v];
            double gs = hc[4 * N + v], gc = hc[5 * N + v];
            neumaier(rs, rc, drho);
            neumaier(ws, wc, (double)dWp);
            neumaier(gs, gc, p.xi_store * (double)dWp / sqrt(rs + rc + (double)rgnd));
            const R We = we_plus(st.He, C11, C12, C44);
            const double hmax = fmax(hc[6 * N + v], (double)We);
            double wcrit = hc[7 * N + v];
            if (wcrit == 0.0 && gs + gc >= p.G_crit) wcrit = hmax + (ws + wc);
            ht[0 * N + v] = rs;
            ht[1 * N + v] = rc;
            ht[2 * N + v] = ws;
            ht[3 * N + v] = wc;
            ht[4 * N + v] = gs;
            ht[5 * N + v] = gc;
            ht[6 * N + v] = hmax;
            ht[7 * N + v] = wcrit;
#pragma unroll
            for (int a = 0; a < 12; ++a) {
                double s_ = hc[(8 + 2 * a) * N + v], c_ = hc[(9 + 2 * a) * N + v];
                neumaier(s_, c_, fabs((double)dg[a]));
                ht[(8 + 2 * a) * N + v] = s_;
                ht[(9 + 2 * a) * N + v] = c_;
            }
            const double drive =
                wcrit > 0.0 ? fmax(0.0, ((double)We + ws + wc) / wcrit - 1.0) : 0.0;
            ((R*)f.drive)[v] = (R)drive;
            ((R*)f.We)[v] = We;
            R* Hpt = (R*)f.Hpi_tr;
#pragma unroll
            for (int k = 0; k < 9; ++k) Hpt[k * N + v] = A[k] - st.dL[k] - AdL[k];
        }
    }
}

void upload_slip_table(cudaStream_t s) {
    static const int planes[4][3] = {{1, 1, 1}, {-1, 1, 1}, {1, -1, 1}, {1, 1, -1}};
    static const int dirs[12][3] = {{0, 1, -1}, {1, 0, -1}, {1, -1, 0}, {0, 1, -1},
                                    {1, 0, 1},  {1, 1, 0},  {0, 1, 1},  {1, 0, -1},
                                    {1, 1, 0},  {0, 1, 1},  {1, 0, 1},  {1, -1, 0}};
    SlipTable t;
    for (int a = 0; a < 12; ++a)
        for (int i = 0; i < 3; ++i) {
            t.sd[a][i] = dirs[a][i] / sqrt(2.0);
            t.nd[a][i] = planes[a / 3][i] / sqrt(3.0);
            t.s[a][i] = (float)t.sd[a][i];
            t.n[a][i] = (float)t.nd[a][i];
        }
    cudaMemcpyToSymbolAsync(c_slip, &t, sizeof(t), 0, cudaMemcpyHostToDevice, s);
}

template <typename R>
void launch_constitutive(const CPFields& f, const CPParams& p, bool hist, cudaStream_t s) {
    const int threads = 128;
    size_t blocks = (f.N + threads - 1) / threads;
    if (hist)
        k_constitutive<R, true><<<(unsigned)blocks, threads, 0, s>>>(f, p);
    else
        k_constitutive<R, false><<<(unsigned)blocks, threads, 0, s>>>(f, p);
}

template void launch_constitutive<float>(const CPFields&, const CPParams&, bool, cudaStream_t);
template void launch_constitutive<double>(const CPFields&, const CPParams&, bool, cudaStream_t);

}  // namespace fatfft
