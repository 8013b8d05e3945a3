// Per-voxel crystal-plasticity update on the GPU (Sec. 2.1 constitutive
// equations, Sec. 2.3 stored energy density and driving force).
//
// One thread owns one voxel.  Everything is written in deviation form
// (H = F - I) so that the FP32 instantiation does not lose the O(1e-3)
// strains to cancellation against the identity.
//
// Model readings (the paper leaves these open; the same readings are used by
// the CPU oracle):
//  * slip law of Eq. flowrule with sign and threshold:
//      dgamma = dt g0 sgn(tau) sinh(<|tau| - tau_c> / sT),
//      g0 = rho_m b^2 nu_D exp(-dF / kT),  sT = kT / dV;
//  * L_p = sum dgamma s (x) n, implicit in the end-of-step stress, first-order
//    update of the inverse plastic deformation Fp^-1 = Fp_n^-1 (I - dL);
//  * S = C : E_e with E_e = (Fe^T Fe - I)/2, P = Fe S Fp^-T, tau = S : s(x)n,
//    cubic C in the lattice frame;
//  * Taylor hardening explicit over the step, one CRSS for all systems.
//
// The local problem is solved for the slip magnitudes y >= 0 of the active
// systems with the slip law in its inverse form sigma tau - tau_c -
// sT asinh(y / (dt g0)) = 0 (well conditioned where the sinh form is stiff),
// adding the most overstressed inactive system one at a time and dropping
// systems whose y reaches zero with a negative residual.  The consistent
// tangent follows from implicit differentiation of R(S) = S - C : E_e(S).
#pragma once
#include "common.cuh"
#include "launch.h"

namespace fatfft {

// FCC {111}<110> in the lattice frame: unit slip directions and normals.
struct SlipTable {
    float s[12][3], n[12][3];
    double sd[12][3], nd[12][3];
};
__constant__ SlipTable c_slip;  // this header is included by one translation unit only

template <typename R> __device__ __forceinline__ R slip_s(int a, int i);
template <> __device__ __forceinline__ float slip_s<float>(int a, int i) { return c_slip.s[a][i]; }
template <> __device__ __forceinline__ double slip_s<double>(int a, int i) { return c_slip.sd[a][i]; }
template <typename R> __device__ __forceinline__ R slip_n(int a, int i);
template <> __device__ __forceinline__ float slip_n<float>(int a, int i) { return c_slip.n[a][i]; }
template <> __device__ __forceinline__ double slip_n<double>(int a, int i) { return c_slip.nd[a][i]; }

template <typename R>
__device__ __forceinline__ void cubic_apply(R C11, R C12, R C44, const R* E, R* S) {
    const R tr = E[0] + E[4] + E[8];
    S[0] = (C11 - C12) * E[0] + C12 * tr;
    S[4] = (C11 - C12) * E[4] + C12 * tr;
    S[8] = (C11 - C12) * E[8] + C12 * tr;
    S[1] = S[3] = C44 * (E[1] + E[3]);
    S[2] = S[6] = C44 * (E[2] + E[6]);
    S[5] = S[7] = C44 * (E[5] + E[7]);
}

// s_a . X . n_a
template <typename R>
__device__ __forceinline__ R resolve(const R* X, int a) {
    R t = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const R si = slip_s<R>(a, i);
        t += si * (X[3 * i] * slip_n<R>(a, 0) + X[3 * i + 1] * slip_n<R>(a, 1) +
                   X[3 * i + 2] * slip_n<R>(a, 2));
    }
    return t;
}

// Green-Lagrange-type strain from a deviation H: (H + H^T + H^T H)/2.
template <typename R>
__device__ __forceinline__ void strain_from_dev(const R* He, R* E) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            E[3 * i + j] = R(0.5) * (He[3 * i + j] + He[3 * j + i] + He[i] * He[j] +
                                     He[3 + i] * He[3 + j] + He[6 + i] * He[6 + j]);
}

template <typename R>
struct LocalState {
    R dL[9], He[9], S[9], tau[12];
};

// State at slips dg: dL = sum dg P, Fe - I = Hes - dL - Hes dL, S = C : E_e.
template <typename R>
__device__ void eval_slip(const R* Hes, const R* dg, R C11, R C12, R C44, LocalState<R>& st) {
#pragma unroll
    for (int k = 0; k < 9; ++k) st.dL[k] = 0;
    for (int a = 0; a < 12; ++a) {
        const R d = dg[a];
        if (d == R(0)) continue;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) st.dL[3 * i + j] += d * slip_s<R>(a, i) * slip_n<R>(a, j);
    }
    R HdL[9];
    mm3(Hes, st.dL, HdL);
#pragma unroll
    for (int k = 0; k < 9; ++k) st.He[k] = Hes[k] - st.dL[k] - HdL[k];
    R E[9];
    strain_from_dev(st.He, E);
    cubic_apply(C11, C12, C44, E, st.S);
#pragma unroll
    for (int a = 0; a < 12; ++a) st.tau[a] = resolve(st.S, a);
}

// B^b = C : sym(X s_b (x) n_b) with X = Fe^T Fe*.
template <typename R>
__device__ __forceinline__ void bmat(const R* X, int b, R C11, R C12, R C44, R* B) {
    R u[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        u[i] = X[3 * i] * slip_s<R>(b, 0) + X[3 * i + 1] * slip_s<R>(b, 1) +
               X[3 * i + 2] * slip_s<R>(b, 2);
    R Y[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            Y[3 * i + j] = R(0.5) * (u[i] * slip_n<R>(b, j) + u[j] * slip_n<R>(b, i));
    cubic_apply(C11, C12, C44, Y, B);
}

// Dense solve with partial pivoting, row stride 12, in place (b <- x).
template <typename R>
__device__ bool gauss_solve(int n, R* A, R* b) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        R best = fabs(A[12 * c + c]);
        for (int r = c + 1; r < n; ++r) {
            const R v = fabs(A[12 * r + c]);
            if (v > best) {
                best = v;
                piv = r;
            }
        }
        if (best == R(0)) return false;
        if (piv != c) {
            for (int k = 0; k < n; ++k) {
                const R t = A[12 * c + k];
                A[12 * c + k] = A[12 * piv + k];
                A[12 * piv + k] = t;
            }
            const R t = b[c];
            b[c] = b[piv];
            b[piv] = t;
        }
        const R inv = R(1) / A[12 * c + c];
        for (int r = c + 1; r < n; ++r) {
            const R f = A[12 * r + c] * inv;
            for (int k = c; k < n; ++k) A[12 * r + k] -= f * A[12 * c + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        R s = b[r];
        for (int k = r + 1; k < n; ++k) s -= A[12 * r + k] * b[k];
        b[r] = s / A[12 * r + r];
    }
    return true;
}

template <typename R>
__device__ R local_potential(const LocalState<R>& st, const R* y, unsigned act, R tau_c, R c,
                             R sT) {
    R E[9];
    strain_from_dev(st.He, E);
    R psi = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) psi += E[k] * st.S[k];
    psi *= R(0.5);
    for (int a = 0; a < 12; ++a)
        if (act >> a & 1u) {
            const R ya = y[a];
            psi += tau_c * ya + sT * (ya * asinh(ya / c) - ya * ya / (sqrt(ya * ya + c * c) + c));
        }
    return psi;
}

// Active-set Newton on the inverse slip law.  On return st holds the state
// at the solution, dg the slip increments and da the derivatives
// d dgamma / d tau (0 on inactive systems).  Returns false if not converged.
template <typename R>
__device__ bool local_solve(const R* Hes, R tau_c, R c, R sT, R C11, R C12, R C44, R tol,
                            int max_it, bool elastic, LocalState<R>& st, R* dg, R* da,
                            int* iters) {
    R y[12], sg[12];
    unsigned act = 0;
#pragma unroll
    for (int a = 0; a < 12; ++a) {
        y[a] = 0;
        sg[a] = 0;
        dg[a] = 0;
        da[a] = 0;
    }
    eval_slip(Hes, dg, C11, C12, C44, st);
    *iters = 0;
    if (elastic || !(c > R(0))) return true;
    const R far = tau_c;
    const R step_floor = R(8) * R(Tr<R>::eps);
    int total = 0;
    for (int outer = 0; outer < 60; ++outer) {
        bool inner_ok = false;
        for (int it = 0; it < max_it; ++it, ++total) {
            for (int a = 0; a < 12; ++a) dg[a] = (act >> a & 1u) ? sg[a] * y[a] : R(0);
            eval_slip(Hes, dg, C11, C12, C44, st);
            R r[12], rmax = 0;
            bool dropped = false;
            for (int a = 0; a < 12; ++a) {
                r[a] = 0;
                if (!(act >> a & 1u)) continue;
                r[a] = sg[a] * st.tau[a] - tau_c - sT * asinh(y[a] / c);
                if (y[a] == R(0) && r[a] < R(0)) {
                    act &= ~(1u << a);
                    dropped = true;
                }
            }
            if (dropped) continue;
            for (int a = 0; a < 12; ++a)
                if (act >> a & 1u) rmax = fmax(rmax, fabs(r[a]));
            if (rmax <= tol) {
                inner_ok = true;
                break;
            }
            int idx[12], na = 0;
            for (int a = 0; a < 12; ++a)
                if (act >> a & 1u) idx[na++] = a;
            // X = Fe^T Fe* = I + He^T + Hes + He^T Hes
            R X[9], HtH[9];
            mtm3(st.He, Hes, HtH);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    X[3 * i + j] = (i == j ? R(1) : R(0)) + st.He[3 * j + i] + Hes[3 * i + j] +
                                   HtH[3 * i + j];
            R J[144], dy[12];
            for (int jj = 0; jj < na; ++jj) {
                const int b = idx[jj];
                R B[9];
                bmat(X, b, C11, C12, C44, B);
                for (int ii = 0; ii < na; ++ii) {
                    const int a = idx[ii];
                    J[12 * ii + jj] = -sg[a] * sg[b] * resolve(B, a);
                }
            }
            for (int ii = 0; ii < na; ++ii) {
                const int a = idx[ii];
                J[12 * ii + ii] -= sT / sqrt(c * c + y[a] * y[a]);
                dy[ii] = -r[a];
            }
            if (!gauss_solve(na, J, dy)) {
                *iters = total;
                return false;
            }
            R dmax = 0, ymax = c;
            for (int ii = 0; ii < na; ++ii) {
                dmax = fmax(dmax, fabs(dy[ii]));
                ymax = fmax(ymax, y[idx[ii]]);
            }
            if (dmax <= step_floor * ymax) {
                inner_ok = true;
                break;
            }
            R ytry[12];
            for (int a = 0; a < 12; ++a) ytry[a] = y[a];
            for (int ii = 0; ii < na; ++ii) ytry[idx[ii]] = fmax(R(0), y[idx[ii]] + dy[ii]);
            if (rmax > far) {
                const R psi0 = local_potential(st, y, act, tau_c, c, sT);
                R lam = 1;
                LocalState<R> tr;
                for (int ls = 0; ls < 8; ++ls) {
                    R dt_[12];
                    for (int a = 0; a < 12; ++a) dt_[a] = (act >> a & 1u) ? sg[a] * ytry[a] : R(0);
                    eval_slip(Hes, dt_, C11, C12, C44, tr);
                    if (local_potential(tr, ytry, act, tau_c, c, sT) <= psi0) break;
                    lam *= R(0.5);
                    for (int ii = 0; ii < na; ++ii)
                        ytry[idx[ii]] = fmax(R(0), y[idx[ii]] + lam * dy[ii]);
                }
            }
            for (int a = 0; a < 12; ++a) y[a] = ytry[a];
        }
        if (!inner_ok) {
            *iters = total;
            return false;
        }
        int best = -1;
        R over = 0;
        for (int a = 0; a < 12; ++a)
            if (!(act >> a & 1u) && fabs(st.tau[a]) - tau_c > over) {
                over = fabs(st.tau[a]) - tau_c;
                best = a;
            }
        if (best < 0) {
            *iters = total + 1;
            for (int a = 0; a < 12; ++a) {
                dg[a] = (act >> a & 1u) ? sg[a] * y[a] : R(0);
                da[a] = (act >> a & 1u) ? sqrt(c * c + y[a] * y[a]) / sT : R(0);
            }
            return true;
        }
        act |= 1u << best;
        sg[best] = st.tau[best] > R(0) ? R(1) : R(-1);
        y[best] = 0;
    }
    *iters = total;
    return false;
}

// Cyclic Jacobi eigen-decomposition of a symmetric 3x3 (eigenvectors in the
// columns of V).
template <typename R>
__device__ void jacobi3(R* A, R* w, R* V) {
#pragma unroll
    for (int k = 0; k < 9; ++k) V[k] = (k % 4 == 0) ? R(1) : R(0);
    for (int sweep = 0; sweep < 12; ++sweep) {
        const R off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
        const R dia = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
        if (off == R(0) || off <= R(Tr<R>::eps) * R(Tr<R>::eps) * R(1e-2) * dia) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                const R apq = A[3 * p + q];
                if (apq == R(0)) continue;
                const R theta = (A[3 * q + q] - A[3 * p + p]) / (R(2) * apq);
                const R t = (theta >= R(0) ? R(1) : R(-1)) /
                            (fabs(theta) + sqrt(theta * theta + R(1)));
                const R cc = R(1) / sqrt(t * t + R(1)), s = t * cc;
                for (int k = 0; k < 3; ++k) {
                    const R akp = A[3 * k + p], akq = A[3 * k + q];
                    A[3 * k + p] = cc * akp - s * akq;
                    A[3 * k + q] = s * akp + cc * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    const R apk = A[3 * p + k], aqk = A[3 * q + k];
                    A[3 * p + k] = cc * apk - s * aqk;
                    A[3 * q + k] = s * apk + cc * aqk;
                }
                for (int k = 0; k < 3; ++k) {
                    const R vkp = V[3 * k + p], vkq = V[3 * k + q];
                    V[3 * k + p] = cc * vkp - s * vkq;
                    V[3 * k + q] = s * vkp + cc * vkq;
                }
            }
    }
    w[0] = A[0];
    w[1] = A[4];
    w[2] = A[8];
}

// W_e+ of Eq. decMiehe (with the energy factor 1/2): eps = 1/2 ln(Fe Fe^T)
// from the eigenvalues 1 + mu of Fe Fe^T, positive part, 1/2 eps+ : C : eps+.
template <typename R>
__device__ R we_plus(const R* He, R C11, R C12, R C44) {
    R B[9];
    mmt3(He, He, B);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) B[3 * i + j] += He[3 * i + j] + He[3 * j + i];
    R mu[3], V[9];
    jacobi3(B, mu, V);
    R ep[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) ep[k] = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const R e = R(0.5) * log1p(mu[k]);
        if (e <= R(0)) continue;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) ep[3 * i + j] += e * V[3 * i + k] * V[3 * j + k];
    }
    R S[9];
    cubic_apply(C11, C12, C44, ep, S);
    R w = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) w += ep[k] * S[k];
    return R(0.5) * w;
}

// Voigt order (11,22,33,23,13,12)
__device__ __forceinline__ int voigt_i(int m) { return m < 3 ? m : (m == 3 ? 1 : 0); }
__device__ __forceinline__ int voigt_j(int m) { return m < 3 ? m : (m == 5 ? 1 : 2); }

}  // namespace fatfft
