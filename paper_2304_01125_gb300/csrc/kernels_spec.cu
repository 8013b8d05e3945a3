// Fourier-space and vector kernels of the fatiguefft library.
//
// Fields in real space are R[c][N] (component-major, x fastest).  Fourier
// fields use the real-to-complex half spectrum of cuFFT: Cx[c][Nh] with
// Nh = (n0/2 + 1) n1 n2 and the x frequency in [0, n0/2].  Inner products
// over the half spectrum carry the Hermitian weights 1 (kx = 0 and the
// Nyquist kx = n0/2 of an even n0) and 2 (all other kx), which makes them
// equal to the sums over the full spectrum (the real-transform symmetry
// reduction of Sec. 3.1).
//
// Frequencies: xi_i = 2 pi k_i / L_i with signed k_i (the paper's shifted
// frequency vectors, Sec. 3.1, in cuFFT's natural order).  First-derivative
// multipliers i xi_i are zero on the Nyquist frequency of an even axis; the
// Laplacian keeps -|xi|^2 there.
//
// Every reduction kernel runs a grid fixed by the problem size (kRedBlocks
// blocks; the dot pass of the Arnoldi step fewer on small grids); each
// block writes one FP64 partial per value and the last block to finish
// combines them in a fixed order (deterministic results, no separate
// finalisation launch).
#include <algorithm>

#include "bulk.cuh"
#include "common.cuh"
#include "spec.h"

namespace fatfft {

template <typename R> __device__ __forceinline__ R grid_tpl(const SGrid& g, int i);
template <> __device__ __forceinline__ float grid_tpl<float>(const SGrid& g, int i) {
    return i == 0 ? g.tpl0f : (i == 1 ? g.tpl1f : g.tpl2f);
}
template <> __device__ __forceinline__ double grid_tpl<double>(const SGrid& g, int i) {
    return i == 0 ? g.tpl0 : (i == 1 ? g.tpl1 : g.tpl2);
}

// Frequency, derivative frequency and Hermitian weight of half-spectrum
// entry e (32-bit index arithmetic: every grid here has Nh < 2^31).
template <typename R>
__device__ __forceinline__ void hs_freq(const SGrid& g, size_t e64, R* xi, R* xid, R& w) {
    const unsigned e = (unsigned)e64;
    const unsigned n0h = (unsigned)g.n0h, n1 = (unsigned)g.n1;
    const unsigned rest = fdiv(e, g.fd_n0h);
    const int kx = (int)(e - rest * n0h);
    const unsigned kz_ = fdiv(rest, g.fd_n1);
    const int ky = (int)(rest - kz_ * n1);
    const int kz = (int)kz_;
    const int sy = ky < (g.n1 + 1) / 2 ? ky : ky - g.n1;
    const int sz = kz < (g.n2 + 1) / 2 ? kz : kz - g.n2;
    // in the bulk type: FP32 kernels keep the frequency decode off the FP64 pipe
    xi[0] = grid_tpl<R>(g, 0) * (R)kx;
    xi[1] = grid_tpl<R>(g, 1) * (R)sy;
    xi[2] = grid_tpl<R>(g, 2) * (R)sz;
    const bool nyx = (g.n0 % 2 == 0) && kx == g.n0 / 2;
    const bool nyy = (g.n1 % 2 == 0) && ky == g.n1 / 2;
    const bool nyz = (g.n2 % 2 == 0) && kz == g.n2 / 2;
    xid[0] = nyx ? R(0) : xi[0];
    xid[1] = nyy ? R(0) : xi[1];
    xid[2] = nyz ? R(0) : xi[2];
    w = (kx == 0 || nyx) ? R(1) : R(2);
}

template <typename Cx>
__device__ __forceinline__ Cx cmul_i(Cx a, decltype(a.x) s) {  // a * (i s)
    Cx r;
    r.x = -a.y * s;
    r.y = a.x * s;
    return r;
}

template <typename Cx>
__device__ __forceinline__ Cx cmul(Cx a, Cx b) {
    Cx r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

// Willot's rotated-scheme gradient symbols at half-spectrum entry e:
// D_j = (e_j - 1)/h prod_{l != j} (1 + e_l)/2 with e_l = exp(2 pi i k_l / n_l)
// (the forward difference along j averaged over the four cell edges
// parallel to j).  sinpi/cospi are exact at the Nyquist index (e = -1), so
// the factors (1 + e) vanish there exactly: the scheme's null modes.
template <typename R> __device__ __forceinline__ void sincospi_r(R a, R* s, R* c);
template <> __device__ __forceinline__ void sincospi_r<float>(float a, float* s, float* c) {
    sincospif(a, s, c);
}
template <> __device__ __forceinline__ void sincospi_r<double>(double a, double* s, double* c) {
    sincospi(a, s, c);
}
template <typename R>
__device__ __forceinline__ void willot_D(const SGrid& g, size_t e64, typename Tr<R>::Cx* D) {
    typedef typename Tr<R>::Cx Cx;
    const unsigned e = (unsigned)e64;
    const unsigned n0h = (unsigned)g.n0h, n1 = (unsigned)g.n1;
    const unsigned rest = fdiv(e, g.fd_n0h);
    const unsigned kx = e - rest * n0h;
    const unsigned kz = fdiv(rest, g.fd_n1);
    const unsigned ky = rest - kz * n1;
    const unsigned k[3] = {kx, ky, kz};
    const int n[3] = {g.n0, g.n1, g.n2};
    Cx ev[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) sincospi_r<R>(R(2 * k[d]) / R(n[d]), &ev[d].y, &ev[d].x);
    const R ih = sizeof(R) == 8 ? (R)g.ih : (R)g.ihf;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        Cx s;
        s.x = (ev[j].x - R(1)) * ih;
        s.y = ev[j].y * ih;
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            if (l == j) continue;
            Cx h;
            h.x = R(0.5) * (R(1) + ev[l].x);
            h.y = R(0.5) * ev[l].y;
            s = cmul(s, h);
        }
        D[j] = s;
    }
}

#define GRID_STRIDE(i, n) \
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (n); i += (size_t)gridDim.x * blockDim.x)

// ------------------------------------------------------------- elementwise
template <typename R>
__global__ void k_add_uniform(R* H, const R* Ht, Mat9 d, size_t N) {
    GRID_STRIDE(v, N) {
#pragma unroll
        for (int c = 0; c < 9; ++c) H[c * N + v] = (R)((double)Ht[c * N + v] + d.a[c]);
    }
}
template <typename R>
void add_uniform(void* H, const void* Ht, const double* d, size_t N, cudaStream_t s) {
    Mat9 m;
    for (int c = 0; c < 9; ++c) m.a[c] = d[c];
    k_add_uniform<R><<<grid_for(N), kThreads, 0, s>>>((R*)H, (const R*)Ht, m, N);
}

// --------------------------------------------------------------------- GND
// F_p - I in the sample frame from the committed lattice-frame Fp^-1 - I:
// Fp - I = -(I + A)^-1 A, rotated with Q (no cancellation against I).
template <typename R>
__global__ void k_fp_sample(const R* Hpi, const int32_t* grain, const double* Qg, R* out,
                            size_t N) {
    GRID_STRIDE(v, N) {
        R A[9], Q[9], M[9];
        const int g = grain[v];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            A[k] = Hpi[k * N + v];
            Q[k] = (R)Qg[9 * g + k];
            M[k] = A[k] + ((k % 4 == 0) ? R(1) : R(0));
        }
        const R det = M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
                      M[2] * (M[3] * M[7] - M[4] * M[6]);
        const R id = R(1) / det;
        R Mi[9];
        Mi[0] = (M[4] * M[8] - M[5] * M[7]) * id;
        Mi[1] = (M[2] * M[7] - M[1] * M[8]) * id;
        Mi[2] = (M[1] * M[5] - M[2] * M[4]) * id;
        Mi[3] = (M[5] * M[6] - M[3] * M[8]) * id;
        Mi[4] = (M[0] * M[8] - M[2] * M[6]) * id;
        Mi[5] = (M[2] * M[3] - M[0] * M[5]) * id;
        Mi[6] = (M[3] * M[7] - M[4] * M[6]) * id;
        Mi[7] = (M[1] * M[6] - M[0] * M[7]) * id;
        Mi[8] = (M[0] * M[4] - M[1] * M[3]) * id;
        R Hp[9], T[9], Hs[9];
        mm3(Mi, A, Hp);
#pragma unroll
        for (int k = 0; k < 9; ++k) Hp[k] = -Hp[k];
        mm3(Q, Hp, T);
        mmt3(T, Q, Hs);
#pragma unroll
        for (int k = 0; k < 9; ++k) out[k * N + v] = Hs[k];
    }
}
template <typename R>
void fp_sample(const void* Hpi, const int32_t* grain, const double* Qg, void* out, size_t N,
               cudaStream_t s) {
    k_fp_sample<R><<<grid_for(N), kThreads, 0, s>>>((const R*)Hpi, grain, Qg, (R*)out, N);
}

// Nye tensor in Fourier space (Eq. nyeindexfourier) with the F_p
// regularisation 1/(1 + ell_Fp^2 |xi|^2): Lambda_ij = eps_jkl i xi_k Fp_il.
// In place on the 9-component half spectrum; folds in the 1/N of the inverse.
template <typename R>
__global__ void k_nye(typename Tr<R>::Cx* F, SGrid g, R l2, R invN) {
    typedef typename Tr<R>::Cx Cx;
    const size_t Nh = g.Nh;
    GRID_STRIDE(e, Nh) {
        R xi[3], xd[3], w;
        hs_freq<R>(g, e, xi, xd, w);
        const R reg = invN / (R(1) + l2 * (xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]));
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const Cx f0 = F[(3 * i + 0) * Nh + e], f1 = F[(3 * i + 1) * Nh + e],
                     f2 = F[(3 * i + 2) * Nh + e];
            Cx l0, l1, l2_;
            // Lambda_i0 = i(xi1 F_i2 - xi2 F_i1), Lambda_i1 = i(xi2 F_i0 - xi0 F_i2),
            // Lambda_i2 = i(xi0 F_i1 - xi1 F_i0)
            Cx a;
            a.x = xd[1] * f2.x - xd[2] * f1.x;
            a.y = xd[1] * f2.y - xd[2] * f1.y;
            l0 = cmul_i(a, reg);
            a.x = xd[2] * f0.x - xd[0] * f2.x;
            a.y = xd[2] * f0.y - xd[0] * f2.y;
            l1 = cmul_i(a, reg);
            a.x = xd[0] * f1.x - xd[1] * f0.x;
            a.y = xd[0] * f1.y - xd[1] * f0.y;
            l2_ = cmul_i(a, reg);
            F[(3 * i + 0) * Nh + e] = l0;
            F[(3 * i + 1) * Nh + e] = l1;
            F[(3 * i + 2) * Nh + e] = l2_;
        }
    }
}
template <typename R>
void nye(void* F, const SGrid& g, double l2, cudaStream_t s) {
    k_nye<R><<<grid_for(g.Nh), kThreads, 0, s>>>((typename Tr<R>::Cx*)F, g, (R)l2,
                                                 (R)(1.0 / (double)g.N));
}

// rho_GND = sqrt(lambda^T (A A^T)^-1 lambda) / b: the norm of the
// minimum-norm edge/screw densities (Eq. nye1), lambda = vec(Q^T Lambda Q).
template <typename R>
__global__ void k_gnd_rho(const R* Lam, const int32_t* grain, const double* Qg, const double* G81,
                          R inv_b, R* rho, size_t N) {
    __shared__ R Gs[81];
    for (int k = threadIdx.x; k < 81; k += blockDim.x) Gs[k] = (R)G81[k];
    __syncthreads();
    GRID_STRIDE(v, N) {
        R L[9], Q[9], T[9], LL[9];
        const int g = grain[v];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            L[k] = Lam[k * N + v];
            Q[k] = (R)Qg[9 * g + k];
        }
        mtm3(Q, L, T);
        mm3(T, Q, LL);
        R q = 0;
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            R t = 0;
#pragma unroll
            for (int b = 0; b < 9; ++b) t += Gs[9 * a + b] * LL[b];
            q += LL[a] * t;
        }
        rho[v] = sqrt(fmax(q, R(0))) * inv_b;
    }
}
template <typename R>
void gnd_rho(const void* Lam, const int32_t* grain, const double* Qg, const double* G81,
             double inv_b, void* rho, size_t N, cudaStream_t s) {
    k_gnd_rho<R><<<grid_for(N), kThreads, 0, s>>>((const R*)Lam, grain, Qg, G81, (R)inv_b,
                                                  (R*)rho, N);
}

// -------------------------------------------------------- averaged tangent
// Kbar = <g(phi) K> (Eq. avstiff).  One row of kRedBlocks blocks; each
// thread walks its voxels and issues the 81 component loads of a voxel
// together (independent, coalesced across the warp), accumulating in the
// bulk type; blocks combine in FP64 and the last block writes the means.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_kbar(const R* K, const R* phi, R kres, size_t N,
                                                   Red red) {
    R acc[81];
#pragma unroll
    for (int c = 0; c < 81; ++c) acc[c] = 0;
    GRID_STRIDE(v, N) {
        const R om = R(1) - phi[v];
        const R gv = om * om + kres;
#pragma unroll
        for (int c = 0; c < 81; ++c) acc[c] += gv * K[(size_t)c * N + v];
    }
    block_partials<81, kThreads>(acc, 81, 0u, red.part);
    grid_finish<kThreads, 81>(red, 81, 0u, 1.0 / (double)N);
}
template <typename R>
void kbar(const void* K, const void* phi, double kres, size_t N, const Red& red, cudaStream_t s) {
    k_kbar<R><<<kRedBlocks, kThreads, 0, s>>>((const R*)K, (const R*)phi, (R)kres, N, red);
}

// ------------------------------------------------------------------ residual
template <typename R>
__global__ void k_degrade(const R* P, const R* phi, R kres, R* out, size_t N) {
    GRID_STRIDE(v, N) {
        const R om = R(1) - phi[v];
        const R g = om * om + kres;
#pragma unroll
        for (int c = 0; c < 9; ++c) out[c * N + v] = g * P[c * N + v];
    }
}
template <typename R>
void degrade(const void* P, const void* phi, double kres, void* out, size_t N, cudaStream_t s) {
    k_degrade<R><<<grid_for(N), kThreads, 0, s>>>((const R*)P, (const R*)phi, (R)kres, (R*)out,
                                                  N);
}

// Offset of field c at half-spectrum entry e in the interleaved layout of
// the fused x pass: (9 r + c) n0h + kx for the row r = ky + n1 kz of e.
__device__ __forceinline__ size_t il_at(const SGrid& g, size_t e64, int c) {
    const unsigned e = (unsigned)e64;
    const unsigned n0h = (unsigned)g.n0h;
    const unsigned rest = fdiv(e, g.fd_n0h);
    return ((size_t)rest * 9 + c) * n0h + (e - rest * n0h);
}
// Offset of field c at entry e: component-major, or interleaved (IL).
template <bool IL>
__device__ __forceinline__ size_t fld_at(const SGrid& g, size_t e, int c) {
    return IL ? il_at(g, e, c) : (size_t)c * g.Nh + e;
}

// Partner of a half-spectrum entry on the kx = 0 plane (or kx = n0/2 for an
// even n0): the entry holding the conjugate frequency (-ky, -kz).  Returns
// false for entries off those planes.
__device__ __forceinline__ bool hs_partner(const SGrid& g, size_t e64, size_t& p) {
    const unsigned e = (unsigned)e64;
    const unsigned n0h = (unsigned)g.n0h, n1 = (unsigned)g.n1;
    const unsigned rest = fdiv(e, g.fd_n0h);
    const int kx = (int)(e - rest * n0h);
    if (!(kx == 0 || ((g.n0 % 2 == 0) && kx == g.n0 / 2))) return false;
    const unsigned kz_ = fdiv(rest, g.fd_n1);
    const int ky = (int)(rest - kz_ * n1), kz = (int)kz_;
    const int py = (g.n1 - ky) % g.n1, pz = (g.n2 - kz) % g.n2;
    p = (size_t)kx + (size_t)g.n0h * ((size_t)py + (size_t)g.n1 * pz);
    return true;
}

// sign * sum_j T_ij(e) i xi_j(e), i = 0..2, projected onto real fields: on the kx = 0 and Nyquist planes the
// value is the mean of the entry and the conjugate of its partner's value,
// so the pair is exactly conjugate (the inverse real transform ignores the
// anti-Hermitian part; left in, its forward-transform round-off is a
// residual no Krylov step can reduce).  The partner (kx, -ky, -kz) has the
// derivative frequencies (xd0, -xd1, -xd2) (exact: the Nyquist rows, where
// k and -k coincide, have zero multipliers).  Its entries are loaded with
// the entry's own (off the planes p = e, a cache hit), so no lane waits for
// a second round of loads.
template <typename R, bool IL = false, bool WIL = false>
__device__ __forceinline__ void div3_real(const typename Tr<R>::Cx* T, const SGrid& g, size_t e,
                                          const R* xd, R sign, typename Tr<R>::Cx* out) {
    typedef typename Tr<R>::Cx Cx;
    size_t p;
    const bool hp = hs_partner(g, e, p);
    if (!hp) p = e;
    Cx te[9], tp[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        te[q] = T[fld_at<IL>(g, e, q)];
        tp[q] = T[fld_at<IL>(g, p, q)];
    }
    if (WIL) {
        // divergence symbols S_j = -conj(D_j) (the adjoint of the rotated
        // gradient); the partner's are conj(S_j)
        Cx D[3];
        willot_D<R>(g, e, D);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            Cx s, r;
            s.x = s.y = r.x = r.y = 0;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                Cx S;
                S.x = -D[j].x;
                S.y = D[j].y;
                const Cx t = cmul(te[3 * i + j], S);
                s.x += t.x;
                s.y += t.y;
                S.y = -S.y;
                const Cx u = cmul(tp[3 * i + j], S);
                r.x += u.x;
                r.y += u.y;
            }
            out[i].x = sign * s.x;
            out[i].y = sign * s.y;
            if (hp) {
                out[i].x = R(0.5) * (out[i].x + sign * r.x);
                out[i].y = R(0.5) * (out[i].y - sign * r.y);
            }
        }
        return;
    }
    const R xp[3] = {xd[0], -xd[1], -xd[2]};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        Cx s, r;
        s.x = s.y = r.x = r.y = 0;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const Cx t = cmul_i(te[3 * i + j], xd[j]);
            s.x += t.x;
            s.y += t.y;
            const Cx u = cmul_i(tp[3 * i + j], xp[j]);
            r.x += u.x;
            r.y += u.y;
        }
        out[i].x = sign * s.x;
        out[i].y = sign * s.y;
        if (hp) {
            out[i].x = R(0.5) * (out[i].x + sign * r.x);
            out[i].y = R(0.5) * (out[i].y - sign * r.y);
        }
    }
}

// b_i = sum_j F{gP}_ij i xi_j (Eq. momentum / newton right-hand side, sign
// flipped), projected onto real fields.  out[0] = ||b||^2, out[1] = the
// round-off scale of b, sum_ij |F{gP}_ij xi_j|^2 (Hermitian-weighted).
template <typename R, bool WIL>
__global__ void k_residual(const typename Tr<R>::Cx* Ph, SGrid g, typename Tr<R>::Cx* b, Red red) {
    typedef typename Tr<R>::Cx Cx;
    const size_t Nh = g.Nh;
    R acc[2] = {R(0), R(0)};
    GRID_STRIDE(e, Nh) {
        R xi[3], xd[3], w;
        hs_freq<R>(g, e, xi, xd, w);
        Cx s[3];
        div3_real<R, false, WIL>(Ph, g, e, xd, R(1), s);
#pragma unroll
        R d2[3] = {xd[0] * xd[0], xd[1] * xd[1], xd[2] * xd[2]};
        if (WIL) {
            Cx D[3];
            willot_D<R>(g, e, D);
#pragma unroll
            for (int j = 0; j < 3; ++j) d2[j] = D[j].x * D[j].x + D[j].y * D[j].y;
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            b[i * Nh + e] = s[i];
            acc[0] += w * (s[i].x * s[i].x + s[i].y * s[i].y);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const Cx q = Ph[(3 * i + j) * Nh + e];
                acc[1] += w * (q.x * q.x + q.y * q.y) * d2[j];
            }
        }
    }
    block_partials<2, kThreads>(acc, 2, 0u, red.part);
    grid_finish<kThreads, 2>(red, 2, 0u, 1.0);
}
template <typename R>
void residual(const void* Ph, const SGrid& g, void* b, const Red& red, cudaStream_t s) {
    typedef typename Tr<R>::Cx Cx;
    if (g.willot)
        k_residual<R, true><<<kRedBlocks, kThreads, 0, s>>>((const Cx*)Ph, g, (Cx*)b, red);
    else
        k_residual<R, false><<<kRedBlocks, kThreads, 0, s>>>((const Cx*)Ph, g, (Cx*)b, red);
}

// -------------------------------------------------------------------- GMRES
// z = M(xi) v with the Green preconditioner M = [xi . Kbar . xi]^-1 of
// Eq. precf (Kbar in shared memory); z = 0 where every derivative frequency
// vanishes (the mean and the Nyquist corners, held at zero).
template <typename R>
__device__ __forceinline__ void green_apply(const R* Ks, const R* xd,
                                            const typename Tr<R>::Cx* v,
                                            typename Tr<R>::Cx* z) {
    if (xd[0] == R(0) && xd[1] == R(0) && xd[2] == R(0)) {
#pragma unroll
        for (int i = 0; i < 3; ++i) z[i].x = z[i].y = 0;
        return;
    }
    R A[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            R s = 0;
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
                for (int l = 0; l < 3; ++l) s += xd[j] * Ks[9 * (3 * i + j) + 3 * k + l] * xd[l];
            A[3 * i + k] = s;
        }
    // Invert A / s with s = |trace A| and scale back: A itself reaches
    // |xi|^2 C ~ 1e13 MPa/mm^2 near the Nyquist frequencies of a
    // micrometre voxel, so det A (~A^3) would overflow FP32 there and zero
    // M on those modes, which GMRES could then never reduce.
    const R tr = fabs(A[0]) + fabs(A[4]) + fabs(A[8]);
    const R is = tr > R(0) ? R(1) / tr : R(0);
#pragma unroll
    for (int q = 0; q < 9; ++q) A[q] *= is;
    const R det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                  A[2] * (A[3] * A[7] - A[4] * A[6]);
    const R id = is / det;  // (A / s)^-1 / s = A^-1
    R Mi[9];
    Mi[0] = (A[4] * A[8] - A[5] * A[7]) * id;
    Mi[1] = (A[2] * A[7] - A[1] * A[8]) * id;
    Mi[2] = (A[1] * A[5] - A[2] * A[4]) * id;
    Mi[3] = (A[5] * A[6] - A[3] * A[8]) * id;
    Mi[4] = (A[0] * A[8] - A[2] * A[6]) * id;
    Mi[5] = (A[2] * A[3] - A[0] * A[5]) * id;
    Mi[6] = (A[3] * A[7] - A[4] * A[6]) * id;
    Mi[7] = (A[1] * A[6] - A[0] * A[7]) * id;
    Mi[8] = (A[0] * A[4] - A[1] * A[3]) * id;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        z[i].x = Mi[3 * i] * v[0].x + Mi[3 * i + 1] * v[1].x + Mi[3 * i + 2] * v[2].x;
        z[i].y = Mi[3 * i] * v[0].y + Mi[3 * i + 1] * v[1].y + Mi[3 * i + 2] * v[2].y;
    }
}

// The Green preconditioner of Willot's scheme, [conj(D) . Kbar . D]^-1 (a
// complex 3 x 3, inverted by cofactors after scaling by its trace as above);
// zero where every symbol vanishes (the mean and the scheme's null modes).
template <typename R>
__device__ __forceinline__ void green_apply_w(const R* Ks, const typename Tr<R>::Cx* D,
                                              const typename Tr<R>::Cx* v,
                                              typename Tr<R>::Cx* z) {
    typedef typename Tr<R>::Cx Cx;
    const R dn = fabs(D[0].x) + fabs(D[0].y) + fabs(D[1].x) + fabs(D[1].y) + fabs(D[2].x) +
                 fabs(D[2].y);
    if (dn == R(0)) {
#pragma unroll
        for (int i = 0; i < 3; ++i) z[i].x = z[i].y = 0;
        return;
    }
    Cx A[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            Cx s;
            s.x = s.y = 0;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                Cx cj = D[j];
                cj.y = -cj.y;
#pragma unroll
                for (int l = 0; l < 3; ++l) {
                    const R kk = Ks[9 * (3 * i + j) + 3 * k + l];
                    const Cx t = cmul(cj, D[l]);
                    s.x += kk * t.x;
                    s.y += kk * t.y;
                }
            }
            A[3 * i + k] = s;
        }
    const R tr = fabs(A[0].x) + fabs(A[4].x) + fabs(A[8].x) + fabs(A[0].y) + fabs(A[4].y) +
                 fabs(A[8].y);
    const R is = R(1) / tr;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        A[q].x *= is;
        A[q].y *= is;
    }
    auto sub = [](Cx a, Cx b) {
        Cx r;
        r.x = a.x - b.x;
        r.y = a.y - b.y;
        return r;
    };
    Cx C[9];  // cofactors, transposed (the adjugate)
    C[0] = sub(cmul(A[4], A[8]), cmul(A[5], A[7]));
    C[1] = sub(cmul(A[2], A[7]), cmul(A[1], A[8]));
    C[2] = sub(cmul(A[1], A[5]), cmul(A[2], A[4]));
    C[3] = sub(cmul(A[5], A[6]), cmul(A[3], A[8]));
    C[4] = sub(cmul(A[0], A[8]), cmul(A[2], A[6]));
    C[5] = sub(cmul(A[2], A[3]), cmul(A[0], A[5]));
    C[6] = sub(cmul(A[3], A[7]), cmul(A[4], A[6]));
    C[7] = sub(cmul(A[1], A[6]), cmul(A[0], A[7]));
    C[8] = sub(cmul(A[0], A[4]), cmul(A[1], A[3]));
    Cx det = cmul(A[0], C[0]);
    const Cx d1 = cmul(A[1], C[3]), d2 = cmul(A[2], C[6]);
    det.x += d1.x + d2.x;
    det.y += d1.y + d2.y;
    // 1/det times the scale 1/tr: (A/tr)^-1 / tr = A^-1
    const R dd = det.x * det.x + det.y * det.y;
    Cx id;
    id.x = det.x / dd * is;
    id.y = -det.y / dd * is;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        Cx acc;
        acc.x = acc.y = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const Cx t = cmul(C[3 * i + k], v[k]);
            acc.x += t.x;
            acc.y += t.y;
        }
        z[i] = cmul(acc, id);
    }
}

// z = M v with the Green preconditioner of the grid's derivative scheme;
// D receives Willot's symbols when that scheme is selected.
template <typename R, bool WIL>
__device__ __forceinline__ void green_any(const SGrid& g, size_t e, const R* Ks, const R* xd,
                                          const typename Tr<R>::Cx* v, typename Tr<R>::Cx* z,
                                          typename Tr<R>::Cx* D) {
    if (WIL) {
        willot_D<R>(g, e, D);
        green_apply_w<R>(Ks, D, v, z);
    } else {
        green_apply<R>(Ks, xd, v, z);
    }
}
// gradient entry z_i d_j: d_j = i xi_j (spectral) or Willot's D_j
template <typename R, bool WIL>
__device__ __forceinline__ typename Tr<R>::Cx grad_sym(typename Tr<R>::Cx z, const R* xd,
                                                       const typename Tr<R>::Cx* D, int j) {
    return WIL ? cmul(z, D[j]) : cmul_i(z, xd[j]);
}

// v = scale * vin (optionally stored to vout); z = M(xi) v when use_pre,
// else z = v; G_ij = z_i i xi_j, the 9-component spectrum of grad z.
template <typename R, bool IL, bool WIL>
__global__ void __launch_bounds__(kThreads, 3) k_precond_grad(const typename Tr<R>::Cx* vin,
                                                              R scale, typename Tr<R>::Cx* vout,
                                                              const double* Kbar, SGrid g,
                                                              typename Tr<R>::Cx* G, int use_pre) {
    typedef typename Tr<R>::Cx Cx;
    __shared__ R Ks[81];
    for (int k = threadIdx.x; k < 81; k += blockDim.x) Ks[k] = (R)Kbar[k];
    __syncthreads();
    const size_t Nh = g.Nh;
    GRID_STRIDE(e, Nh) {
        R xi[3], xd[3], w;
        hs_freq<R>(g, e, xi, xd, w);
        Cx v[3], z[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            v[i] = vin[i * Nh + e];
            v[i].x *= scale;
            v[i].y *= scale;
            if (vout) vout[i * Nh + e] = v[i];
        }
        Cx D[3];
        if (use_pre) {
            green_any<R, WIL>(g, e, Ks, xd, v, z, D);
        } else {
            if (WIL) willot_D<R>(g, e, D);
#pragma unroll
            for (int i = 0; i < 3; ++i) z[i] = v[i];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                G[fld_at<IL>(g, e, 3 * i + j)] = grad_sym<R, WIL>(z[i], xd, D, j);
    }
}
template <typename R>
void precond_grad(const void* vin, double scale, void* vout, const double* Kbar, const SGrid& g,
                  void* G, int use_pre, cudaStream_t s, int il) {
    typedef typename Tr<R>::Cx Cx;
    if (il)
        k_precond_grad<R, true, false><<<grid_for(g.Nh), kThreads, 0, s>>>(
            (const Cx*)vin, (R)scale, (Cx*)vout, Kbar, g, (Cx*)G, use_pre);
    else if (g.willot)
        k_precond_grad<R, false, true><<<grid_for(g.Nh), kThreads, 0, s>>>(
            (const Cx*)vin, (R)scale, (Cx*)vout, Kbar, g, (Cx*)G, use_pre);
    else
        k_precond_grad<R, false, false><<<grid_for(g.Nh), kThreads, 0, s>>>(
            (const Cx*)vin, (R)scale, (Cx*)vout, Kbar, g, (Cx*)G, use_pre);
}

// tau = g(phi) K : grad z in place (grad z arrives scaled by N from the
// unnormalised inverse transform).  For even N each thread owns a pair of
// neighbouring voxels and moves them with one 2-wide load per component
// (every component offset c*N + v is then even, so the loads are aligned);
// odd N takes the one-voxel loop.
template <typename R> struct V2;
template <> struct V2<float> { typedef float2 T; };
template <> struct V2<double> { typedef double2 T; };
template <typename R>
__global__ void __launch_bounds__(kThreads) k_tangent_apply(R* G, const R* K, const R* phi, R kres,
                                                            R invN, size_t N, const int* act) {
    typedef typename V2<R>::T T2;
    if (act && *act == 0) return;  // a lockstep class member that has left the loop
    if (N & 1) {
        GRID_STRIDE(v, N) {
            R gz[9];
#pragma unroll
            for (int b = 0; b < 9; ++b) gz[b] = G[b * N + v];
            const R om = R(1) - phi[v];
            const R sc = (om * om + kres) * invN;
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                R t = 0;
#pragma unroll
                for (int b = 0; b < 9; ++b) t += K[(size_t)(9 * a + b) * N + v] * gz[b];
                G[a * N + v] = sc * t;
            }
        }
        return;
    }
    const size_t Np = N / 2;
    GRID_STRIDE(q, Np) {
        const size_t v = 2 * q;
        T2 gz[9];
#pragma unroll
        for (int b = 0; b < 9; ++b) gz[b] = *reinterpret_cast<const T2*>(G + b * N + v);
        const T2 ph = *reinterpret_cast<const T2*>(phi + v);
        const R o0 = R(1) - ph.x, o1 = R(1) - ph.y;
        const R s0 = (o0 * o0 + kres) * invN, s1 = (o1 * o1 + kres) * invN;
        T2 out[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            R t0 = 0, t1 = 0;
#pragma unroll
            for (int b = 0; b < 9; ++b) {
                const T2 k = *reinterpret_cast<const T2*>(K + (size_t)(9 * a + b) * N + v);
                t0 += k.x * gz[b].x;
                t1 += k.y * gz[b].y;
            }
            out[a].x = s0 * t0;
            out[a].y = s1 * t1;
        }
#pragma unroll
        for (int a = 0; a < 9; ++a) *reinterpret_cast<T2*>(G + a * N + v) = out[a];
    }
}
template <typename R>
void tangent_apply(void* G, const void* K, const void* phi, double kres, size_t N,
                   cudaStream_t s, const int* act) {
    k_tangent_apply<R><<<grid_for((N & 1) ? N : N / 2), kThreads, 0, s>>>(
        (R*)G, (const R*)K, (const R*)phi, (R)kres, (R)(1.0 / (double)N), N, act);
}

// ------------------------------------------------------ Arnoldi step kernels
// Arnoldi with classical Gram-Schmidt and delayed reorthogonalisation
// (DCGS2): the operator is applied to the candidate c_k, which has been
// projected once against the final basis Q_k = [q_0 .. q_{k-1}] but neither
// reorthogonalised nor normalised.  One pass over Q_k then gives both the
// reorthogonalisation coefficients a = Q_k^T c_k and the projections
// b = Q_k^T z of z = A M c_k; a second pass writes the final
// q_k = (c_k - Q_k a) / nu and the next candidate c_{k+1}.  Because
// A M Q_k = Q_{k+1} Hbar (the Arnoldi relation of the final columns),
//   A M q_k = (z - Q_{k+1} Hbar a) / nu,
// so the column k coefficients follow from a, b, alpha = c_k.c_k,
// beta = c_k.z and Hbar alone.  Per GMRES step: C2R, tangent apply, R2C,
// contraction fused with the dot pass (k_contract_dots), k_dcgs_update.
//
// The Krylov vectors are 3 Nh complex entries, component-major (stride Nh),
// weighted by the Hermitian weight of their frequency.  Hessenberg columns
// live on the device in FP64: Hd (final columns) and Hp (provisional
// columns), column i at offset i * kHcol.



// w = -div(T) = -sum_j i xi_j T_ij (the sign that makes the operator
// positive), projected onto real fields.
template <typename R, bool WIL>
__global__ void k_contract(const typename Tr<R>::Cx* T, SGrid g, typename Tr<R>::Cx* w) {
    typedef typename Tr<R>::Cx Cx;
    const size_t Nh = g.Nh;
    GRID_STRIDE(e, Nh) {
        R xi[3], xd[3], wt;
        hs_freq<R>(g, e, xi, xd, wt);
        Cx a[3];
        div3_real<R, false, WIL>(T, g, e, xd, R(-1), a);
#pragma unroll
        for (int c = 0; c < 3; ++c) w[c * Nh + e] = a[c];
    }
}
template <typename R>
void contract(const void* T, const SGrid& g, void* w, cudaStream_t s) {
    typedef typename Tr<R>::Cx Cx;
    if (g.willot)
        k_contract<R, true><<<grid_for(g.Nh), kThreads, 0, s>>>((const Cx*)T, g, (Cx*)w);
    else
        k_contract<R, false><<<grid_for(g.Nh), kThreads, 0, s>>>((const Cx*)T, g, (Cx*)w);
}

// Coefficients of DCGS2 step k from the dots d (layout above) and
// the Hessenberg columns (one warp, FP64):
//   nu = sqrt(alpha - |a|^2)          (|c_k - Q_k a|; 0 on breakdown)
//   column k-1, final:  Hp[k-1] + a (rows < k), nu (row k)
//   t = Hbar a over the final columns 0 .. k-1 (rows 0 .. k)
//   h_l = (b_l - t_l) / nu (l < k),  h_k = ((beta - a.b) / nu - t_k) / nu
//   dd_l = t_l / nu + h_l,  e_l = dd_l - a_l dd_k / nu
// Stores the final column k-1 to Hd, the provisional column k (h) to Hp,
// both to slot (rows at 0 and kSlotProv, nu at kSlotNu) for the host, and
// coef = [a (kMaxKrylov), e (kMaxKrylov), 1/nu, dd_k/nu] for k_dcgs_update.
// Hs: the final columns 0 .. k-2 and the provisional column k-1, staged in
// shared memory (column i at i * kHcol).
__device__ void dcgs_coefficients(int k, const double* d, const double* Hs, double* Hd, double* Hp,
                                  double* slot, double* coef) {
    const int l = threadIdx.x & 31;
    const double alpha = d[0], beta = d[1];
    const double al = l < k ? d[3 + 2 * l] : 0.0;
    const double bl = l < k ? d[4 + 2 * l] : 0.0;
    double aa = al * al, ab = al * bl;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        aa += __shfl_xor_sync(0xffffffffu, aa, o);
        ab += __shfl_xor_sync(0xffffffffu, ab, o);
    }
    const double nu2 = alpha - aa;
    const bool brk = !(nu2 > 1e-28 * alpha) || !(alpha > 0.0);
    const double nu = brk ? 0.0 : sqrt(nu2);
    const double inu = brk ? 0.0 : 1.0 / nu;
    // final column k-1 (row l in lane l); the other columns' row l prefetched
    double fin = 0.0;
    if (k >= 1 && l <= k) fin = l < k ? Hs[(k - 1) * kHcol + l] + al : nu;
    double t = 0.0;
    for (int i = 0; i < k; ++i) {  // uniform trip count: the shuffle needs all lanes
        const double ai = __shfl_sync(0xffffffffu, al, i);
        if (l <= i + 1 && l <= k) t += (i == k - 1 ? fin : Hs[i * kHcol + l]) * ai;
    }
    double h = 0.0;
    if (l < k) h = (bl - t) * inu;
    if (l == k) h = ((beta - ab) * inu - t) * inu;
    const double dd = t * inu + h;
    const double ddk = __shfl_sync(0xffffffffu, dd, k < 32 ? k : 31);
    if (l < k) {
        coef[l] = al;
        coef[kMaxKrylov + l] = dd - al * ddk * inu;
    }
    if (l == 0) {
        coef[2 * kMaxKrylov] = inu;
        coef[2 * kMaxKrylov + 1] = ddk * inu;
        slot[kSlotNu] = nu;
        slot[kSlotAlpha] = alpha;
        slot[kSlotA2] = aa;
        slot[kSlotErr] = 0.0;  // the pipelined kernels overwrite it with their error word
    }
    if (k >= 1 && l <= k) {
        Hd[(size_t)(k - 1) * kHcol + l] = fin;
        slot[l] = fin;
    }
    if (l <= k) {
        Hp[(size_t)k * kHcol + l] = h;
        slot[kSlotProv + l] = h;
    }
}

// Dots of step k: out[0] = alpha = c.c, out[1] = beta = c.z, out[2] = z.z,
// out[3 + 2i] = a_i = q_i.c, out[4 + 2i] = b_i = q_i.z (i < k <= NQ), held
// per thread in registers and combined across blocks in FP64.
// Tail of the dot pass: block partials, the last block's combine, the
// Hessenberg staging and the step coefficients (dcgs_coefficients).
template <typename A, int NQ>
__device__ __forceinline__ void dots_finish(const A (&acc)[3 + 2 * NQ], int k, const Red& red,
                                            double* Hd, double* Hp, double* slot, double* coef,
                                            const int* err) {
    // the update pass (launched as a programmatic dependent) may start
    // prefetching the basis while this grid reduces and forms coefficients
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    block_partials<3 + 2 * NQ, kThreads>(acc, 3 + 2 * k, 0u, red.part);
    if (grid_finish<kThreads, 3 + 2 * NQ>(red, 3 + 2 * k, 0u, 1.0)) {
        // the last block: stage the Hessenberg columns the step needs, then
        // warp 0 forms the coefficients (the dots were written by this block)
        __shared__ double s_H[NQ > 0 ? NQ * kHcol : 1];
        if (NQ > 0) {
            const int nH = (k - 1) * kHcol;
            for (int q = threadIdx.x; q < k * kHcol; q += blockDim.x)
                s_H[q] = q < nH ? __ldcg(Hd + q) : __ldcg(Hp + q);  // column k-1: provisional
        }
        __syncthreads();
        if (threadIdx.x < 32) dcgs_coefficients(k, red.out, s_H, Hd, Hp, slot, coef);
        // the pipelined update pass's error word, reported in the slot
        if (threadIdx.x == 0 && err) slot[kSlotErr] = (double)*(volatile const int*)err;
    }
}

// The GMRES operator's last step fused with the dot pass: per frequency,
// z = -div(T) projected onto real fields (as k_contract) is stored and, in
// the same pass, alpha = c.c, beta = c.z, |z|^2, a_i = q_i.c and
// b_i = q_i.z accumulate (the dot layout above); the tail forms the step's
// coefficients.  Saves the contraction's launch and tail and the re-read of
// z and c.
// A is the per-thread accumulator type: the bulk type R by default, or FP64
// (products and sums, FATIGUEFFT_DOT64=1) to measure what the FP32 partial
// sums of the mixed path cost in accuracy.
template <typename R, int NQ, bool IL, typename A, bool WIL>
__global__ void __launch_bounds__(kThreads, 2) k_contract_dots(
    const typename Tr<R>::Cx* T, SGrid g, typename Tr<R>::Cx* w, const typename Tr<R>::Cx* c,
    const typename Tr<R>::Cx* V, size_t vstride, int k, Red red, double* Hd, double* Hp,
    double* slot, double* coef, const int* err, const int* act) {
    typedef typename Tr<R>::Cx Cx;
    constexpr int G = NQ < 8 ? NQ : 8;
    if (act && *act == 0) return;
    A acc[3 + 2 * NQ];
#pragma unroll
    for (int v = 0; v < 3 + 2 * NQ; ++v) acc[v] = 0;
    const size_t Nh = g.Nh;
    GRID_STRIDE(e, Nh) {
        R xi[3], xd[3], wt;
        hs_freq<R>(g, e, xi, xd, wt);
        Cx zc[3], cv[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) cv[q] = c[q * Nh + e];
        div3_real<R, IL, WIL>(T, g, e, xd, R(-1), zc);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            w[q * Nh + e] = zc[q];
            acc[0] += (A)wt * ((A)cv[q].x * (A)cv[q].x + (A)cv[q].y * (A)cv[q].y);
            acc[1] += (A)wt * ((A)cv[q].x * (A)zc[q].x + (A)cv[q].y * (A)zc[q].y);
            acc[2] += (A)wt * ((A)zc[q].x * (A)zc[q].x + (A)zc[q].y * (A)zc[q].y);
        }
#pragma unroll
        for (int i0 = 0; i0 < NQ; i0 += 8) {
            Cx qv[G > 0 ? G : 1][3];
#pragma unroll
            for (int t = 0; t < G; ++t)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    if (i0 + t < k) {
                        qv[t][q] = V[(size_t)(i0 + t) * vstride + q * Nh + e];
                    } else {
                        qv[t][q].x = qv[t][q].y = 0;
                    }
                }
#pragma unroll
            for (int t = 0; t < G; ++t)
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    acc[3 + 2 * (i0 + t)] += (A)wt * ((A)qv[t][q].x * (A)cv[q].x +
                                                      (A)qv[t][q].y * (A)cv[q].y);
                    acc[4 + 2 * (i0 + t)] += (A)wt * ((A)qv[t][q].x * (A)zc[q].x +
                                                      (A)qv[t][q].y * (A)zc[q].y);
                }
        }
    }
    dots_finish<A, NQ>(acc, k, red, Hd, Hp, slot, coef, err);
}
template <typename R>
void contract_dots(const void* T, const SGrid& g, void* w, const void* c, const void* V,
                   size_t vstride, int k, const Red& red, double* Hd, double* Hp, double* slot,
                   double* coef, const BulkCfg* bc, cudaStream_t s, int il, int dot64,
                   const int* act) {
    typedef typename Tr<R>::Cx Cx;
    const Cx *TT = (const Cx*)T, *cc = (const Cx*)c, *VV = (const Cx*)V;
    Cx* ww = (Cx*)w;
    const int* err = bc ? bc->err : nullptr;
    // one frequency per thread up to the fixed reduction grid: small grids
    // (below about 44^3) launch fewer blocks, so that the dot passes of
    // several handles run side by side instead of each filling the GPU
    const int nb = (int)std::min<size_t>((size_t)kRedBlocks,
                                         std::max<size_t>(1, (g.Nh + kThreads - 1) / kThreads));
#define CDOTS(NQ)                                                                             \
    do {                                                                                      \
        if (il)                                                                               \
            k_contract_dots<R, NQ, true, R, false><<<nb, kThreads, 0, s>>>(                  \
                TT, g, ww, cc, VV, vstride, k, red, Hd, Hp, slot, coef, err, act);            \
        else if (g.willot)                                                                    \
            k_contract_dots<R, NQ, false, R, true><<<nb, kThreads, 0, s>>>(                  \
                TT, g, ww, cc, VV, vstride, k, red, Hd, Hp, slot, coef, err, act);            \
        else if (dot64)                                                                       \
            k_contract_dots<R, NQ, false, double, false><<<nb, kThreads, 0, s>>>(            \
                TT, g, ww, cc, VV, vstride, k, red, Hd, Hp, slot, coef, err, act);            \
        else                                                                                  \
            k_contract_dots<R, NQ, false, R, false><<<nb, kThreads, 0, s>>>(                 \
                TT, g, ww, cc, VV, vstride, k, red, Hd, Hp, slot, coef, err, act);            \
    } while (0)
    if (k <= 0)
        CDOTS(0);
    else if (k <= 4)
        CDOTS(4);
    else if (k <= 8)
        CDOTS(8);
    else if (k <= 16)
        CDOTS(16);
    else
        CDOTS(kMaxKrylov);
#undef CDOTS
}

// ------------------------------------------- pipelined Arnoldi update pass
// The same update as k_dcgs_update, with c_k, z and the basis streamed
// through a ring of kBulkS shared-memory stages filled by bulk asynchronous
// copies: one thread issues the copies kBulkS stages ahead and every thread
// consumes a stage once its mbarrier phase completes, so the bytes in flight
// per SM are set by the ring, not by registers.  Each CTA owns a contiguous
// run of tpc tiles of kUpdT frequencies (all three components); 256
// frequencies and 8 stages measured fastest of {64, 128, 256} x {8, 12, 16}
// at 64^3.  Used when
// every copy is 16-byte aligned (Nh even, or complex FP64).  A wait that
// runs out sets *err (reported to the host) and the CTA stops consuming,
// takes part in the reduction with what it has, and waits (again bounded)
// for its own copies still in flight before it exits.  (The dot pass keeps
// its register-streaming kernel: a pipelined version's per-stage
// synchronisation outweighed the deeper pipeline.)
#ifndef FATIGUEFFT_UPD_STAGES
#define FATIGUEFFT_UPD_STAGES 8
#endif
#ifndef FATIGUEFFT_UPD_TILE
#define FATIGUEFFT_UPD_TILE 256
#endif
constexpr int kBulkS = FATIGUEFFT_UPD_STAGES;  // ring stages
constexpr int kUpdT = FATIGUEFFT_UPD_TILE;     // frequencies per tile (= threads per CTA)

// bounded wait for the last copy issued into every stage (issued copies in all)
__device__ __forceinline__ void bulk_drain(uint64_t* full, int issued) {
    for (int s = 0; s < kBulkS && s < issued; ++s) {
        const int last = s + ((issued - 1 - s) / kBulkS) * kBulkS;
        mbar_wait(&full[s], (unsigned)(last / kBulkS) & 1u);
    }
}

template <typename R, bool IL, bool WIL>
__global__ void __launch_bounds__(kUpdT) k_dcgs_update_bulk(
    typename Tr<R>::Cx* V, size_t vstride, int k, const typename Tr<R>::Cx* z,
    const double* coef, const double* Kbar, SGrid g, typename Tr<R>::Cx* G, int tpc, Red red,
    int* err, const int* act) {
    typedef typename Tr<R>::Cx Cx;
    if (act && *act == 0) return;
    extern __shared__ __align__(128) unsigned char dyn[];
    Cx* buf = reinterpret_cast<Cx*>(dyn);  // [kBulkS][3][kUpdT]
    __shared__ __align__(8) uint64_t full[kBulkS];
    __shared__ R s_a[kMaxKrylov], s_e[kMaxKrylov];
    __shared__ R Ks[81];
    const unsigned Nh = (unsigned)g.Nh;
    const int ntiles = (int)((Nh + kUpdT - 1) / kUpdT);
    const int t0 = blockIdx.x * tpc, t1 = min(t0 + tpc, ntiles);
    const int nv = k + 2;  // per tile: c_k, q_0 .. q_{k-1}, then z (see below)
    const int total = t1 > t0 ? (t1 - t0) * nv : 0;
    const int tid = threadIdx.x;
    Cx* ck = V + (size_t)k * vstride;
    Cx* cn = V + (size_t)(k + 1) * vstride;
    int issued = 0;
    auto issue = [&](int L) {
        const int tile = t0 + L / nv, v = L % nv;
        const unsigned e0 = (unsigned)tile * kUpdT;
        const unsigned cnt = min((unsigned)kUpdT, Nh - e0);
        const Cx* src = v == 0 ? ck : v == nv - 1 ? z : V + (size_t)(v - 1) * vstride;
        uint64_t* b = &full[L % kBulkS];
        Cx* dst = buf + (size_t)(L % kBulkS) * 3 * kUpdT;
        mbar_arrive_tx(b, 3 * cnt * (unsigned)sizeof(Cx));
#pragma unroll
        for (int cc = 0; cc < 3; ++cc)
            bulk_load(dst + cc * kUpdT, src + (size_t)cc * Nh + e0, cnt * (unsigned)sizeof(Cx), b);
        issued = L + 1;
    };
    for (int q = tid; q < 81; q += blockDim.x) Ks[q] = (R)Kbar[q];
    if (tid == 0) {
        for (int s = 0; s < kBulkS; ++s) mbar_init(&full[s], 1);
        mbar_fence_init();
    }
    __syncthreads();
    // c_k and the basis were written before the dot pass (this grid's
    // programmatic predecessor) started, so their copies may start while it
    // still runs; z (its output), the coefficients, the outputs (slot k is
    // its input) and the shared reduction buffers wait for its completion.
    // z is the last load of each tile, so the first tile's z bounds the
    // early copies.
    if (tid == 0)
        for (int L = 0; L < min(min(kBulkS, total), nv - 1); ++L) issue(L);
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (tid == 0)
        for (int L = issued; L < min(kBulkS, total); ++L) issue(L);
    for (int q = tid; q < k; q += blockDim.x) {
        s_a[q] = (R)coef[q];
        s_e[q] = (R)coef[kMaxKrylov + q];
    }
    __syncthreads();
    const R inu = (R)coef[2 * kMaxKrylov], cc = (R)coef[2 * kMaxKrylov + 1];
    bool ok = true;
    int L = 0;
    R acc[1] = {R(0)};
    for (int tile = t0; tile < t1; ++tile) {
        const unsigned e = (unsigned)tile * kUpdT + tid;
        Cx sa[3], se[3], cv[3], zv[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) sa[q].x = sa[q].y = se[q].x = se[q].y = 0;
        for (int v = 0; v < nv; ++v) {
            const int st = L % kBulkS;
            if (ok && !mbar_wait(&full[st], (unsigned)(L / kBulkS) & 1u)) ok = false;
            const Cx* b = buf + (size_t)st * 3 * kUpdT;
            Cx x[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                if (ok && e < Nh) {
                    x[q] = b[q * kUpdT + tid];
                } else {
                    x[q].x = x[q].y = 0;
                }
            }
            if (v == 0) {
#pragma unroll
                for (int q = 0; q < 3; ++q) cv[q] = x[q];
            } else if (v == nv - 1) {
#pragma unroll
                for (int q = 0; q < 3; ++q) zv[q] = x[q];
            } else {
                const R ai = s_a[v - 1], ei = s_e[v - 1];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    sa[q].x += ai * x[q].x;
                    sa[q].y += ai * x[q].y;
                    se[q].x += ei * x[q].x;
                    se[q].y += ei * x[q].y;
                }
            }
            __syncthreads();
            if (tid == 0 && ok && L + kBulkS < total) issue(L + kBulkS);
            ++L;
        }
        if (ok && e < Nh) {
            R xi[3], xd[3], wt;
            hs_freq<R>(g, e, xi, xd, wt);
            Cx nx[3];
            R nn = 0;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                Cx qk;
                qk.x = (cv[q].x - sa[q].x) * inu;
                qk.y = (cv[q].y - sa[q].y) * inu;
                ck[(size_t)q * Nh + e] = qk;
                nx[q].x = zv[q].x * inu - se[q].x - cv[q].x * cc;
                nx[q].y = zv[q].y * inu - se[q].y - cv[q].y * cc;
                cn[(size_t)q * Nh + e] = nx[q];
                nn += nx[q].x * nx[q].x + nx[q].y * nx[q].y;
            }
            acc[0] += wt * nn;
            if (G) {
                Cx zz[3], D[3];
                green_any<R, WIL>(g, e, Ks, xd, nx, zz, D);
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        G[fld_at<IL>(g, e, 3 * i + j)] = grad_sym<R, WIL>(zz[i], xd, D, j);
            }
        }
    }
    if (!ok) atomicExch(err, 1);
    if (tid == 0 && !ok) bulk_drain(full, issued);
    block_partials<1, kUpdT>(acc, 1, 0u, red.part);
    grid_finish<kUpdT, 1>(red, 1, 0u, 1.0);
}

// Dynamic shared memory and the resident-CTA budget of the pipelined
// kernels (set once per handle, outside any stream capture).
template <typename R>
static size_t upd_bulk_smem() {
    return (size_t)kBulkS * 3 * kUpdT * sizeof(typename Tr<R>::Cx);
}
template <typename R>
int dcgs_bulk_setup(BulkCfg& bc) {
    int nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int su = (int)upd_bulk_smem<R>();
    int nu = 0;
    if (cudaFuncSetAttribute(k_dcgs_update_bulk<R, false, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, su) != cudaSuccess ||
        cudaFuncSetAttribute(k_dcgs_update_bulk<R, true, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, su) != cudaSuccess ||
        cudaFuncSetAttribute(k_dcgs_update_bulk<R, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, su) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nu, k_dcgs_update_bulk<R, false, false>,
                                                      kUpdT, su) != cudaSuccess)
        nu = 0;
    cudaGetLastError();
    // the reduction buffers hold kRedSlots x kRedBlocks partials
    bc.upd_blocks = min(nu * nsm, kRedSlots * kRedBlocks);
    return bc.upd_blocks > 0;
}

template <typename R>
static inline bool bulk_aligned(const SGrid& g) {
    return sizeof(typename Tr<R>::Cx) % 16 == 0 || g.Nh % 2 == 0;
}

static inline void tile_split(int ntiles, int maxb, int& tpc, int& nb) {
    tpc = (ntiles + maxb - 1) / maxb;
    if (tpc < 1) tpc = 1;
    nb = (ntiles + tpc - 1) / tpc;
}


// Update of step k with the coefficients from k_contract_dots (coef):
//   q_k = (c_k - Q_k a) / nu                     -> slot k (in place)
//   c_{k+1} = z / nu - Q_k e - c_k dd_k / nu     -> slot k + 1
//   G = (M c_{k+1}) (x) i xi                     -> the next step's gradient
// and out[0] = |c_{k+1}|^2.
template <typename R, bool IL, bool WIL>
__global__ void __launch_bounds__(kThreads, 2) k_dcgs_update(typename Tr<R>::Cx* V,
                                                             size_t vstride, int k,
                                                             const typename Tr<R>::Cx* z,
                                                             const double* coef,
                                                             const double* Kbar, SGrid g,
                                                             typename Tr<R>::Cx* G, Red red,
                                                             const int* act) {
    typedef typename Tr<R>::Cx Cx;
    if (act && *act == 0) return;
    __shared__ R s_a[kMaxKrylov], s_e[kMaxKrylov];
    __shared__ R Ks[81];
    for (int q = threadIdx.x; q < 81; q += blockDim.x) Ks[q] = (R)Kbar[q];
    for (int q = threadIdx.x; q < k; q += blockDim.x) {
        s_a[q] = (R)coef[q];
        s_e[q] = (R)coef[kMaxKrylov + q];
    }
    const R inu = (R)coef[2 * kMaxKrylov], cc = (R)coef[2 * kMaxKrylov + 1];
    __syncthreads();
    const size_t Nh = g.Nh;
    Cx* ck = V + (size_t)k * vstride;
    Cx* cn = V + (size_t)(k + 1) * vstride;
    R acc[1] = {};
    GRID_STRIDE(e, Nh) {
        R xi[3], xd[3], wt;
        hs_freq<R>(g, e, xi, xd, wt);
        Cx sa[3], se[3], cv[3], zv[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            sa[c].x = sa[c].y = se[c].x = se[c].y = 0;
            cv[c] = ck[c * Nh + e];
            zv[c] = z[c * Nh + e];
        }
#pragma unroll 4
        for (int i = 0; i < k; ++i) {
            const Cx* qi = V + (size_t)i * vstride;
            const R ai = s_a[i], ei = s_e[i];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const Cx q = qi[c * Nh + e];
                sa[c].x += ai * q.x;
                sa[c].y += ai * q.y;
                se[c].x += ei * q.x;
                se[c].y += ei * q.y;
            }
        }
        Cx nx[3];
        R nn = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Cx qk;
            qk.x = (cv[c].x - sa[c].x) * inu;
            qk.y = (cv[c].y - sa[c].y) * inu;
            ck[c * Nh + e] = qk;
            nx[c].x = zv[c].x * inu - se[c].x - cv[c].x * cc;
            nx[c].y = zv[c].y * inu - se[c].y - cv[c].y * cc;
            cn[c * Nh + e] = nx[c];
            nn += nx[c].x * nx[c].x + nx[c].y * nx[c].y;
        }
        acc[0] += wt * nn;
        if (G) {
            Cx zz[3], D[3];
            green_any<R, WIL>(g, e, Ks, xd, nx, zz, D);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j)
                    G[fld_at<IL>(g, e, 3 * i + j)] = grad_sym<R, WIL>(zz[i], xd, D, j);
        }
    }
    block_partials<1, kThreads>(acc, 1, 0u, red.part);
    grid_finish<kThreads, 1>(red, 1, 0u, 1.0);
}
template <typename R>
void dcgs_update(void* V, size_t vstride, int k, const void* z, const double* coef,
                 const double* Kbar, const SGrid& g, void* G, const Red& red, const BulkCfg* bc,
                 cudaStream_t s, int il, const int* act) {
    typedef typename Tr<R>::Cx Cx;
    if (bc && bulk_aligned<R>(g)) {
        int tpc, nb;
        tile_split((int)((g.Nh + kUpdT - 1) / kUpdT), bc->upd_blocks, tpc, nb);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)nb);
        cfg.blockDim = dim3(kUpdT);
        cfg.dynamicSmemBytes = upd_bulk_smem<R>();
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (il)
            cudaLaunchKernelEx(&cfg, k_dcgs_update_bulk<R, true, false>, (Cx*)V, vstride, k,
                               (const Cx*)z, coef, Kbar, g, (Cx*)G, tpc, red, bc->err, act);
        else if (g.willot)
            cudaLaunchKernelEx(&cfg, k_dcgs_update_bulk<R, false, true>, (Cx*)V, vstride, k,
                               (const Cx*)z, coef, Kbar, g, (Cx*)G, tpc, red, bc->err, act);
        else
            cudaLaunchKernelEx(&cfg, k_dcgs_update_bulk<R, false, false>, (Cx*)V, vstride, k,
                               (const Cx*)z, coef, Kbar, g, (Cx*)G, tpc, red, bc->err, act);
        return;
    }
    if (il)
        k_dcgs_update<R, true, false><<<grid_for(g.Nh), kThreads, 0, s>>>(
            (Cx*)V, vstride, k, (const Cx*)z, coef, Kbar, g, (Cx*)G, red, act);
    else if (g.willot)
        k_dcgs_update<R, false, true><<<grid_for(g.Nh), kThreads, 0, s>>>(
            (Cx*)V, vstride, k, (const Cx*)z, coef, Kbar, g, (Cx*)G, red, act);
    else
        k_dcgs_update<R, false, false><<<grid_for(g.Nh), kThreads, 0, s>>>(
            (Cx*)V, vstride, k, (const Cx*)z, coef, Kbar, g, (Cx*)G, red, act);
}

// x += M (sum_i y_i V_i)  (right-preconditioned GMRES update)
template <typename R, bool WIL>
__global__ void k_xupdate(typename Tr<R>::Cx* x, const typename Tr<R>::Cx* V, size_t vstride,
                          int k, const double* y, const double* Kbar, SGrid g) {
    typedef typename Tr<R>::Cx Cx;
    __shared__ R Ks[81];
    for (int q = threadIdx.x; q < 81; q += blockDim.x) Ks[q] = (R)Kbar[q];
    __syncthreads();
    const size_t Nh = g.Nh;
    GRID_STRIDE(e, Nh) {
        R xi[3], xd[3], wt;
        hs_freq<R>(g, e, xi, xd, wt);
        Cx c[3], z[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) c[i].x = c[i].y = 0;
        for (int q = 0; q < k; ++q) {
            const R yq = (R)y[q];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const Cx v = V[(size_t)q * vstride + i * Nh + e];
                c[i].x += yq * v.x;
                c[i].y += yq * v.y;
            }
        }
        Cx D[3];
        green_any<R, WIL>(g, e, Ks, xd, c, z, D);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            Cx xv = x[i * Nh + e];
            xv.x += z[i].x;
            xv.y += z[i].y;
            x[i * Nh + e] = xv;
        }
    }
}
template <typename R>
void xupdate(void* x, const void* V, size_t vstride, int k, const double* y, const double* Kbar,
             const SGrid& g, cudaStream_t s) {
    typedef typename Tr<R>::Cx Cx;
    if (g.willot)
        k_xupdate<R, true><<<grid_for(g.Nh), kThreads, 0, s>>>((Cx*)x, (const Cx*)V, vstride, k,
                                                               y, Kbar, g);
    else
        k_xupdate<R, false><<<grid_for(g.Nh), kThreads, 0, s>>>((Cx*)x, (const Cx*)V, vstride, k,
                                                                y, Kbar, g);
}

// out = alpha a + beta b (complex vectors of n3 entries; b may be null)
template <typename R>
__global__ void k_axpby(typename Tr<R>::Cx* out, const typename Tr<R>::Cx* a,
                        const typename Tr<R>::Cx* b, R alpha, R beta, size_t n) {
    typedef typename Tr<R>::Cx Cx;
    GRID_STRIDE(e, n) {
        Cx r = a[e];
        r.x *= alpha;
        r.y *= alpha;
        if (b) {
            const Cx q = b[e];
            r.x += beta * q.x;
            r.y += beta * q.y;
        }
        out[e] = r;
    }
}
template <typename R>
void axpby(void* out, const void* a, const void* b, double alpha, double beta, size_t n,
           cudaStream_t s) {
    typedef typename Tr<R>::Cx Cx;
    k_axpby<R><<<grid_for(n), kThreads, 0, s>>>((Cx*)out, (const Cx*)a, (const Cx*)b, (R)alpha,
                                                (R)beta, n);
}

// ||v||^2 (Hermitian-weighted) of a 3-component half-spectrum vector.
template <typename R>
__global__ void k_norm2(const typename Tr<R>::Cx* v, SGrid g, Red red) {
    typedef typename Tr<R>::Cx Cx;
    R acc[1] = {};
    GRID_STRIDE(e, g.Nh) {
        R xi[3], xd[3], wt;
        hs_freq<R>(g, e, xi, xd, wt);
        R nn = 0;  // ||v||^2 -> out[0]
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const Cx q = v[c * g.Nh + e];
            nn += q.x * q.x + q.y * q.y;
        }
        acc[0] += wt * nn;
    }
    block_partials<1, kThreads>(acc, 1, 0u, red.part);
    grid_finish<kThreads, 1>(red, 1, 0u, 1.0);
}
template <typename R>
void norm2(const void* v, const SGrid& g, const Red& red, cudaStream_t s) {
    k_norm2<R><<<kRedBlocks, kThreads, 0, s>>>((const typename Tr<R>::Cx*)v, g, red);
}

// ----------------------------------------------------------- Newton update
// H += grad(du) (arriving scaled by N); out[0] = max |grad du|,
// out[1] = max |H - Ht| (the Newton test of Sec. 3.1).
template <typename R>
__global__ void k_fupdate(R* H, const R* G, R invN, const R* Ht, size_t N, Red red) {
    R acc[2] = {};
    GRID_STRIDE(v, N) {
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            const R d = G[c * N + v] * invN;
            const R h = H[c * N + v] + d;
            H[c * N + v] = h;
            acc[0] = fmax(acc[0], fabs(d));
            acc[1] = fmax(acc[1], fabs(h - Ht[c * N + v]));
        }
    }
    block_partials<2, kThreads>(acc, 2, 3u, red.part);
    grid_finish<kThreads, 2>(red, 2, 3u, 1.0);
}
template <typename R>
void fupdate(void* H, const void* G, const void* Ht, size_t N, const Red& red, cudaStream_t s) {
    k_fupdate<R><<<kRedBlocks, kThreads, 0, s>>>((R*)H, (const R*)G, (R)(1.0 / (double)N),
                                                 (const R*)Ht, N, red);
}

// Algorithm 1 ratios and the mean degraded stress in one pass:
// out[0] = max |H - Hprev|, out[1] = max |H - Ht|, out[2 + c] = <g(phi) P_c>.
template <typename R>
__global__ void k_stag_stats(const R* H, const R* Hprev, const R* Ht, const R* P, const R* phi,
                             R kres, size_t N, Red red) {
    R acc[11] = {};
    GRID_STRIDE(v, N) {
        const R om = R(1) - phi[v];
        const R g = om * om + kres;
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            const R h = H[c * N + v];
            acc[0] = fmax(acc[0], fabs(h - Hprev[c * N + v]));
            acc[1] = fmax(acc[1], fabs(h - Ht[c * N + v]));
            acc[2 + c] += g * P[c * N + v];
        }
    }
    block_partials<11, kThreads>(acc, 11, 3u, red.part);
    grid_finish<kThreads, 11>(red, 11, 3u, 1.0 / (double)N);
}
template <typename R>
void stag_stats(const void* H, const void* Hprev, const void* Ht, const void* P, const void* phi,
                double kres, size_t N, const Red& red, cudaStream_t s) {
    k_stag_stats<R><<<kRedBlocks, kThreads, 0, s>>>((const R*)H, (const R*)Hprev, (const R*)Ht,
                                                    (const R*)P, (const R*)phi, (R)kres, N, red);
}

template <typename R>
__global__ void k_maxval(const R* a, size_t n, Red red) {
    R acc[1] = {};
    GRID_STRIDE(i, n) acc[0] = fmax(acc[0], a[i]);
    block_partials<1, kThreads>(acc, 1, 1u, red.part);
    grid_finish<kThreads, 1>(red, 1, 1u, 1.0);
}
template <typename R>
void maxval(const void* a, size_t n, const Red& red, cudaStream_t s) {
    k_maxval<R><<<kRedBlocks, kThreads, 0, s>>>((const R*)a, n, red);
}

// ------------------------------------------------------------- phase field
// mode 0: f *= ell^2 |xi|^2 / N  (the -ell^2 lap term);  mode 1: f *= 1 /
// (N (1 + ell^2 |xi|^2))  (M_phi, Eq. precph read with ell^2).
template <typename R>
__global__ void k_pf_spec(typename Tr<R>::Cx* f, SGrid g, R l2, R invN, int mode) {
    typedef typename Tr<R>::Cx Cx;
    GRID_STRIDE(e, g.Nh) {
        R xi[3], xd[3], w;
        hs_freq<R>(g, e, xi, xd, w);
        const R k2 = l2 * (xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
        const R m = mode == 0 ? k2 * invN : invN / (R(1) + k2);
        Cx a = f[e];
        a.x *= m;
        a.y *= m;
        f[e] = a;
    }
}
template <typename R>
void pf_spec(void* f, const SGrid& g, double l2, int mode, cudaStream_t s) {
    k_pf_spec<R><<<grid_for(g.Nh), kThreads, 0, s>>>((typename Tr<R>::Cx*)f, g, (R)l2,
                                                     (R)(1.0 / (double)g.N), mode);
}

// r = 2S - (1 + 2S) x - lapx; out[0] = ||r||^2, out[1] = ||2S||^2
template <typename R>
__global__ void k_pf_init(const R* x, const R* lapx, const R* S, R* r, size_t N, Red red) {
    R acc[2] = {};
    GRID_STRIDE(v, N) {
        const R s2 = R(2) * S[v];
        const R rv = s2 - (R(1) + s2) * x[v] - lapx[v];
        r[v] = rv;
        acc[0] += rv * rv;
        acc[1] += s2 * s2;
    }
    block_partials<2, kThreads>(acc, 2, 0u, red.part);
    grid_finish<kThreads, 2>(red, 2, 0u, 1.0);
}
template <typename R>
void pf_init(const void* x, const void* lapx, const void* S, void* r, size_t N, const Red& red,
             cudaStream_t s) {
    k_pf_init<R><<<kRedBlocks, kThreads, 0, s>>>((const R*)x, (const R*)lapx, (const R*)S, (R*)r,
                                                 N, red);
}

template <typename R>
__global__ void k_rdot(const R* a, const R* b, size_t N, Red red) {
    R acc[1] = {};
    GRID_STRIDE(v, N) acc[0] += a[v] * b[v];
    block_partials<1, kThreads>(acc, 1, 0u, red.part);
    grid_finish<kThreads, 1>(red, 1, 0u, 1.0);
}
template <typename R>
void rdot(const void* a, const void* b, size_t N, const Red& red, cudaStream_t s) {
    k_rdot<R><<<kRedBlocks, kThreads, 0, s>>>((const R*)a, (const R*)b, N, red);
}

// q = t + 2 S p  (A p through the recurrence t = M^-1 p);  out[0] = <p, q>
template <typename R>
__global__ void k_pf_q(const R* t, const R* p, const R* S, R* q, size_t N, Red red) {
    R acc[1] = {};
    GRID_STRIDE(v, N) {
        const R qv = t[v] + R(2) * S[v] * p[v];
        q[v] = qv;
        acc[0] += p[v] * qv;
    }
    block_partials<1, kThreads>(acc, 1, 0u, red.part);
    grid_finish<kThreads, 1>(red, 1, 0u, 1.0);
}
template <typename R>
void pf_q(const void* t, const void* p, const void* S, void* q, size_t N, const Red& red,
          cudaStream_t s) {
    k_pf_q<R><<<kRedBlocks, kThreads, 0, s>>>((const R*)t, (const R*)p, (const R*)S, (R*)q, N,
                                              red);
}

// x += alpha p; r -= alpha q; out[0] = ||r||^2
template <typename R>
__global__ void k_pf_xr(R* x, R* r, const R* p, const R* q, R alpha, size_t N, Red red) {
    R acc[1] = {};
    GRID_STRIDE(v, N) {
        x[v] += alpha * p[v];
        const R rv = r[v] - alpha * q[v];
        r[v] = rv;
        acc[0] += rv * rv;
    }
    block_partials<1, kThreads>(acc, 1, 0u, red.part);
    grid_finish<kThreads, 1>(red, 1, 0u, 1.0);
}
template <typename R>
void pf_xr(void* x, void* r, const void* p, const void* q, double alpha, size_t N, const Red& red,
           cudaStream_t s) {
    k_pf_xr<R><<<kRedBlocks, kThreads, 0, s>>>((R*)x, (R*)r, (const R*)p, (const R*)q, (R)alpha,
                                               N, red);
}

// p = z + beta p; t = r + beta t
template <typename R>
__global__ void k_pf_pt(R* p, R* t, const R* z, const R* r, R beta, size_t N) {
    GRID_STRIDE(v, N) {
        p[v] = z[v] + beta * p[v];
        t[v] = r[v] + beta * t[v];
    }
}
template <typename R>
void pf_pt(void* p, void* t, const void* z, const void* r, double beta, size_t N,
           cudaStream_t s) {
    k_pf_pt<R><<<grid_for(N), kThreads, 0, s>>>((R*)p, (R*)t, (const R*)z, (const R*)r, (R)beta,
                                                N);
}

// phi_new = max(x, phi_t) (irreversibility, Algorithm 1); out: max
// |phi_new - phi_old|, max |phi_new - phi_t|, count of changed and of
// cracked (phi >= 0.9) voxels.
template <typename R>
__global__ void k_pf_clamp(const R* x, const R* phi_t, R* phi, size_t N, Red red) {
    R acc[4] = {};
    GRID_STRIDE(v, N) {
        const R pt = phi_t[v];
        const R pn = fmax(x[v], pt);
        const R po = phi[v];
        phi[v] = pn;
        acc[0] = fmax(acc[0], fabs(pn - po));
        acc[1] = fmax(acc[1], fabs(pn - pt));
        acc[2] += pn != po ? R(1) : R(0);
        acc[3] += pn >= R(0.9) ? R(1) : R(0);
    }
    block_partials<4, kThreads>(acc, 4, 3u, red.part);
    grid_finish<kThreads, 4>(red, 4, 3u, 1.0);
}
template <typename R>
void pf_clamp(const void* x, const void* phi_t, void* phi, size_t N, const Red& red,
              cudaStream_t s) {
    k_pf_clamp<R><<<kRedBlocks, kThreads, 0, s>>>((const R*)x, (const R*)phi_t, (R*)phi, N, red);
}

// ----------------------------------------------------------- conversions
template <typename R>
__global__ void k_to_double(const R* src, double* dst, size_t n, size_t N, int add_eye) {
    GRID_STRIDE(i, n) {
        double v = (double)src[i];
        if (add_eye) {
            const size_t c = i / N;
            if (c == 0 || c == 4 || c == 8) v += 1.0;
        }
        dst[i] = v;
    }
}
template <typename R>
void to_double(const void* src, double* dst, size_t n, size_t N, int add_eye, cudaStream_t s) {
    k_to_double<R><<<grid_for(n), kThreads, 0, s>>>((const R*)src, dst, n, N, add_eye);
}
template <typename R>
__global__ void k_from_double(const double* src, R* dst, size_t n, size_t N, int sub_eye) {
    GRID_STRIDE(i, n) {
        double v = src[i];
        if (sub_eye) {
            const size_t c = i / N;
            if (c == 0 || c == 4 || c == 8) v -= 1.0;
        }
        dst[i] = (R)v;
    }
}
template <typename R>
void from_double(const double* src, void* dst, size_t n, size_t N, int sub_eye, cudaStream_t s) {
    k_from_double<R><<<grid_for(n), kThreads, 0, s>>>(src, (R*)dst, n, N, sub_eye);
}
__global__ void k_hist_sum(const double* hist, int slot, int comp, int count, double* dst,
                           size_t N) {
    GRID_STRIDE(i, (size_t)count * N) {
        const size_t c = i / N, v = i % N;
        const int s = slot + (int)c * (comp ? 2 : 1);
        double x = hist[(size_t)s * N + v];
        if (comp) x += hist[(size_t)(s + 1) * N + v];
        dst[i] = x;
    }
}
void hist_sum(const double* hist, int slot, int comp, int count, double* dst, size_t N,
              cudaStream_t s) {
    k_hist_sum<<<grid_for((size_t)count * N), kThreads, 0, s>>>(hist, slot, comp, count, dst, N);
}
__global__ void k_hist_set(double* hist, int slot, int comp, int count, const double* src,
                           size_t N) {
    GRID_STRIDE(i, (size_t)count * N) {
        const size_t c = i / N, v = i % N;
        const int s = slot + (int)c * (comp ? 2 : 1);
        hist[(size_t)s * N + v] = src[i];
        if (comp) hist[(size_t)(s + 1) * N + v] = 0.0;
    }
}
void hist_set(double* hist, int slot, int comp, int count, const double* src, size_t N,
              cudaStream_t s) {
    k_hist_set<<<grid_for((size_t)count * N), kThreads, 0, s>>>(hist, slot, comp, count, src, N);
}
// Fp^-1 - I (lattice) from a sample-frame F_p: inverse of Q^T F_p Q.
template <typename R>
__global__ void k_fp_in(const double* Fp, const int32_t* grain, const double* Qg, R* Hpi,
                        size_t N) {
    GRID_STRIDE(v, N) {
        double F[9], Q[9], T[9], L[9];
        const int g = grain[v];
        for (int k = 0; k < 9; ++k) {
            F[k] = Fp[k * N + v];
            Q[k] = Qg[9 * g + k];
        }
        mtm3(Q, F, T);
        mm3(T, Q, L);
        const double det = L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) +
                           L[2] * (L[3] * L[7] - L[4] * L[6]);
        double Li[9];
        Li[0] = (L[4] * L[8] - L[5] * L[7]) / det;
        Li[1] = (L[2] * L[7] - L[1] * L[8]) / det;
        Li[2] = (L[1] * L[5] - L[2] * L[4]) / det;
        Li[3] = (L[5] * L[6] - L[3] * L[8]) / det;
        Li[4] = (L[0] * L[8] - L[2] * L[6]) / det;
        Li[5] = (L[2] * L[3] - L[0] * L[5]) / det;
        Li[6] = (L[3] * L[7] - L[4] * L[6]) / det;
        Li[7] = (L[1] * L[6] - L[0] * L[7]) / det;
        Li[8] = (L[0] * L[4] - L[1] * L[3]) / det;
        for (int k = 0; k < 9; ++k) Hpi[k * N + v] = (R)(Li[k] - ((k % 4 == 0) ? 1.0 : 0.0));
    }
}
template <typename R>
void fp_in(const double* Fp, const int32_t* grain, const double* Qg, void* Hpi, size_t N,
           cudaStream_t s) {
    k_fp_in<R><<<grid_for(N), kThreads, 0, s>>>(Fp, grain, Qg, (R*)Hpi, N);
}

// ------------------------------------------------------ bounded-wait self-test
// One warp waits on an mbarrier that nothing arrives on: the bounded wait
// must give up after `limit` rounds (out = 1), not spin; out = 2 would mean
// it reported a phase that never completed.
__global__ void k_selftest_wait(int* out, unsigned limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    const bool done = mbar_wait(&bar, 0u, limit);
    if (threadIdx.x == 0) out[0] = done ? 2 : 1;
}
int selftest_bounded_wait(unsigned limit) {
    int* d = nullptr;
    int h = 0;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return -1;
    k_selftest_wait<<<1, 32>>>(d, limit);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? h : -1;
}

// ------------------------------------------------------- instantiations
#define INST(R)                                                                                \
    template void add_uniform<R>(void*, const void*, const double*, size_t, cudaStream_t);      \
    template void fp_sample<R>(const void*, const int32_t*, const double*, void*, size_t,       \
                               cudaStream_t);                                                   \
    template void nye<R>(void*, const SGrid&, double, cudaStream_t);                            \
    template void gnd_rho<R>(const void*, const int32_t*, const double*, const double*, double, \
                             void*, size_t, cudaStream_t);                                      \
    template void kbar<R>(const void*, const void*, double, size_t, const Red&, cudaStream_t);  \
    template void degrade<R>(const void*, const void*, double, void*, size_t, cudaStream_t);    \
    template void residual<R>(const void*, const SGrid&, void*, const Red&, cudaStream_t);      \
    template void precond_grad<R>(const void*, double, void*, const double*, const SGrid&,      \
                                  void*, int, cudaStream_t, int);                               \
    template void tangent_apply<R>(void*, const void*, const void*, double, size_t,             \
                                   cudaStream_t, const int*);                                   \
    template void contract<R>(const void*, const SGrid&, void*, cudaStream_t);                  \
    template void dcgs_update<R>(void*, size_t, int, const void*, const double*,                \
                                 const double*, const SGrid&, void*, const Red&,                \
                                 const BulkCfg*, cudaStream_t, int, const int*);                \
    template int dcgs_bulk_setup<R>(BulkCfg&);                                                  \
    template void contract_dots<R>(const void*, const SGrid&, void*, const void*, const void*,  \
                                   size_t, int, const Red&, double*, double*, double*, double*, \
                                   const BulkCfg*, cudaStream_t, int, int, const int*);         \
    template void norm2<R>(const void*, const SGrid&, const Red&, cudaStream_t);                \
    template void xupdate<R>(void*, const void*, size_t, int, const double*, const double*,     \
                             const SGrid&, cudaStream_t);                                       \
    template void axpby<R>(void*, const void*, const void*, double, double, size_t,             \
                           cudaStream_t);                                                       \
    template void fupdate<R>(void*, const void*, const void*, size_t, const Red&, cudaStream_t);\
    template void stag_stats<R>(const void*, const void*, const void*, const void*,             \
                                const void*, double, size_t, const Red&, cudaStream_t);         \
    template void maxval<R>(const void*, size_t, const Red&, cudaStream_t);                     \
    template void pf_spec<R>(void*, const SGrid&, double, int, cudaStream_t);                   \
    template void pf_init<R>(const void*, const void*, const void*, void*, size_t, const Red&,  \
                             cudaStream_t);                                                     \
    template void rdot<R>(const void*, const void*, size_t, const Red&, cudaStream_t);          \
    template void pf_q<R>(const void*, const void*, const void*, void*, size_t, const Red&,     \
                          cudaStream_t);                                                        \
    template void pf_xr<R>(void*, void*, const void*, const void*, double, size_t, const Red&,  \
                           cudaStream_t);                                                       \
    template void pf_pt<R>(void*, void*, const void*, const void*, double, size_t,              \
                           cudaStream_t);                                                       \
    template void pf_clamp<R>(const void*, const void*, void*, size_t, const Red&,              \
                              cudaStream_t);                                                    \
    template void to_double<R>(const void*, double*, size_t, size_t, int, cudaStream_t);        \
    template void from_double<R>(const double*, void*, size_t, size_t, int, cudaStream_t);      \
    template void fp_in<R>(const double*, const int32_t*, const double*, void*, size_t,         \
                           cudaStream_t);
INST(float)
INST(double)

}  // namespace fatfft
