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
// Every reduction kernel runs exactly kRedBlocks blocks and writes one partial
// per block and value; k_finalize_* combine them in a fixed order.
#include "common.cuh"
#include "spec.h"

namespace fatfft {

template <typename R>
__device__ __forceinline__ void hs_freq(const SGrid& g, size_t e, R* xi, R* xid, R& w) {
    const int kx = (int)(e % g.n0h);
    const size_t rest = e / g.n0h;
    const int ky = (int)(rest % g.n1);
    const int kz = (int)(rest / g.n1);
    const int sy = ky < (g.n1 + 1) / 2 ? ky : ky - g.n1;
    const int sz = kz < (g.n2 + 1) / 2 ? kz : kz - g.n2;
    xi[0] = (R)(g.tpl0 * kx);
    xi[1] = (R)(g.tpl1 * sy);
    xi[2] = (R)(g.tpl2 * sz);
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

#define GRID_STRIDE(i, n) \
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (n); i += (size_t)gridDim.x * blockDim.x)

// ---------------------------------------------------------------- finalize
__global__ void k_finalize_sum(const double* part, int nb, double scale, double* out) {
    __shared__ double sh[32];
    double a = 0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) a += part[(size_t)blockIdx.x * nb + i];
    const double s = block_sum<kThreads>(a, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = s * scale;
}
__global__ void k_finalize_max(const double* part, int nb, double* out) {
    __shared__ double sh[32];
    double a = 0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) a = fmax(a, part[(size_t)blockIdx.x * nb + i]);
    const double s = block_max<kThreads>(a, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}
void finalize_sum(const double* part, int nvals, double scale, double* out, cudaStream_t s) {
    k_finalize_sum<<<nvals, kThreads, 0, s>>>(part, kRedBlocks, scale, out);
}
void finalize_max(const double* part, int nvals, double* out, cudaStream_t s) {
    k_finalize_max<<<nvals, kThreads, 0, s>>>(part, kRedBlocks, out);
}

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
// Kbar = <g(phi) K> (Eq. avstiff), partial sums per component (grid.y = 81).
template <typename R>
__global__ void k_kbar(const R* K, const R* phi, R kres, size_t N, double* part) {
    __shared__ double sh[32];
    const int c = blockIdx.y;
    double a = 0;
    GRID_STRIDE(v, N) {
        const R om = R(1) - phi[v];
        a += (double)((om * om + kres) * K[(size_t)c * N + v]);
    }
    const double s = block_sum<kThreads>(a, sh);
    if (threadIdx.x == 0) part[(size_t)c * gridDim.x + blockIdx.x] = s;
}
template <typename R>
void kbar(const void* K, const void* phi, double kres, size_t N, double* part, cudaStream_t s) {
    k_kbar<R><<<dim3(kRedBlocks, 81), kThreads, 0, s>>>((const R*)K, (const R*)phi, (R)kres, N,
                                                        part);
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

// b_i = sum_j F{gP}_ij i xi_j (Eq. momentum / newton right-hand side, sign
// flipped); partials of ||b||^2 and of the round-off scale of b,
// sum_ij |F{gP}_ij xi_j|^2 (Hermitian-weighted).
template <typename R>
__global__ void k_residual(const typename Tr<R>::Cx* Ph, SGrid g, typename Tr<R>::Cx* b,
                           double* part) {
    typedef typename Tr<R>::Cx Cx;
    __shared__ double sh[32];
    const size_t Nh = g.Nh;
    double nb = 0, np = 0;
    GRID_STRIDE(e, Nh) {
        R xi[3], xd[3], w;
        hs_freq<R>(g, e, xi, xd, w);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            Cx s;
            s.x = 0;
            s.y = 0;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const Cx p = Ph[(3 * i + j) * Nh + e];
                np += (double)w * ((double)p.x * p.x + (double)p.y * p.y) * (double)xd[j] *
                      (double)xd[j];
                const Cx t = cmul_i(p, xd[j]);
                s.x += t.x;
                s.y += t.y;
            }
            b[i * Nh + e] = s;
            nb += (double)w * ((double)s.x * s.x + (double)s.y * s.y);
        }
    }
    double r = block_sum<kThreads>(nb, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = r;
    r = block_sum<kThreads>(np, sh);
    if (threadIdx.x == 0) part[kRedBlocks + blockIdx.x] = r;
}
template <typename R>
void residual(const void* Ph, const SGrid& g, void* b, double* part, cudaStream_t s) {
    k_residual<R><<<kRedBlocks, kThreads, 0, s>>>((const typename Tr<R>::Cx*)Ph, g,
                                                  (typename Tr<R>::Cx*)b, part);
}

// Projection onto real fields: on the kx = 0 plane (and kx = n0/2 for even
// n0) the entries at (ky, kz) and (-ky, -kz) are set to the mean of one and
// the conjugate of the other; self-conjugate entries lose their imaginary
// part.  The inverse real transform ignores the anti-Hermitian part, so
// without this the forward transform's round-off there is a residual the
// Krylov solver cannot reduce.
template <typename R>
__global__ void k_hermitize(typename Tr<R>::Cx* v, int ncomp, SGrid g) {
    typedef typename Tr<R>::Cx Cx;
    const int planes = (g.n0 % 2 == 0 && g.n0 > 1) ? 2 : 1;
    const size_t per = (size_t)g.n1 * g.n2;
    GRID_STRIDE(t, per * planes * ncomp) {
        const size_t q = t % per;
        const int pl = (int)((t / per) % planes);
        const int c = (int)(t / (per * planes));
        const int kx = pl == 0 ? 0 : g.n0 / 2;
        const int ky = (int)(q % g.n1), kz = (int)(q / g.n1);
        const int py = (g.n1 - ky) % g.n1, pz = (g.n2 - kz) % g.n2;
        const size_t qp = (size_t)py + (size_t)g.n1 * pz;
        if (qp < q) continue;  // the partner with the smaller index does the pair
        Cx* base = v + (size_t)c * g.Nh;
        const size_t e = (size_t)kx + (size_t)g.n0h * q;
        const size_t ep = (size_t)kx + (size_t)g.n0h * qp;
        const Cx a = base[e], b = base[ep];
        if (qp == q) {
            Cx r = a;
            r.y = 0;
            base[e] = r;
        } else {
            Cx m;
            m.x = R(0.5) * (a.x + b.x);
            m.y = R(0.5) * (a.y - b.y);
            base[e] = m;
            m.y = -m.y;
            base[ep] = m;
        }
    }
}
template <typename R>
void hermitize(void* v, int ncomp, const SGrid& g, cudaStream_t s) {
    const size_t n = (size_t)g.n1 * g.n2 * ((g.n0 % 2 == 0 && g.n0 > 1) ? 2 : 1) * ncomp;
    k_hermitize<R><<<grid_for(n), kThreads, 0, s>>>((typename Tr<R>::Cx*)v, ncomp, g);
}

// -------------------------------------------------------------------- GMRES
// v = scale * vin (optionally stored to vout); z = M(xi) v with the Green
// preconditioner M = [xi . Kbar . xi]^-1 (Eq. precf) when use_pre, else z =
// v; G_ij = z_i i xi_j, the 9-component spectrum of grad z.
template <typename R>
__global__ void k_precond_grad(const typename Tr<R>::Cx* vin, R scale,
                               typename Tr<R>::Cx* vout, const double* Kbar, SGrid g,
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
        if (use_pre) {
            const bool zero = xd[0] == R(0) && xd[1] == R(0) && xd[2] == R(0);
            if (zero) {
#pragma unroll
                for (int i = 0; i < 3; ++i) z[i].x = z[i].y = 0;
            } else {
                R A[9];
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        R s = 0;
#pragma unroll
                        for (int j = 0; j < 3; ++j)
#pragma unroll
                            for (int l = 0; l < 3; ++l)
                                s += xd[j] * Ks[9 * (3 * i + j) + 3 * k + l] * xd[l];
                        A[3 * i + k] = s;
                    }
                const R det = A[0] * (A[4] * A[8] - A[5] * A[7]) -
                              A[1] * (A[3] * A[8] - A[5] * A[6]) +
                              A[2] * (A[3] * A[7] - A[4] * A[6]);
                const R id = R(1) / det;
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
        } else {
#pragma unroll
            for (int i = 0; i < 3; ++i) z[i] = v[i];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) G[(3 * i + j) * Nh + e] = cmul_i(z[i], xd[j]);
    }
}
template <typename R>
void precond_grad(const void* vin, double scale, void* vout, const double* Kbar, const SGrid& g,
                  void* G, int use_pre, cudaStream_t s) {
    typedef typename Tr<R>::Cx Cx;
    k_precond_grad<R><<<grid_for(g.Nh), kThreads, 0, s>>>((const Cx*)vin, (R)scale, (Cx*)vout,
                                                          Kbar, g, (Cx*)G, use_pre);
}

// tau = g(phi) K : grad z in place (grad z arrives scaled by N from the
// unnormalised inverse transform).
template <typename R>
__global__ void k_tangent_apply(R* G, const R* K, const R* phi, R kres, R invN, size_t N) {
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
}
template <typename R>
void tangent_apply(void* G, const void* K, const void* phi, double kres, size_t N,
                   cudaStream_t s) {
    k_tangent_apply<R><<<grid_for(N), kThreads, 0, s>>>((R*)G, (const R*)K, (const R*)phi,
                                                        (R)kres, (R)(1.0 / (double)N), N);
}

// w_i = -sum_j i xi_j T_ij (divergence, sign giving the positive operator)
template <typename R>
__global__ void k_contract(const typename Tr<R>::Cx* T, SGrid g, typename Tr<R>::Cx* w) {
    typedef typename Tr<R>::Cx Cx;
    const size_t Nh = g.Nh;
    GRID_STRIDE(e, Nh) {
        R xi[3], xd[3], wt;
        hs_freq<R>(g, e, xi, xd, wt);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            Cx s;
            s.x = 0;
            s.y = 0;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const Cx t = cmul_i(T[(3 * i + j) * Nh + e], xd[j]);
                s.x -= t.x;
                s.y -= t.y;
            }
            w[i * Nh + e] = s;
        }
    }
}
template <typename R>
void contract(const void* T, const SGrid& g, void* w, cudaStream_t s) {
    typedef typename Tr<R>::Cx Cx;
    k_contract<R><<<grid_for(g.Nh), kThreads, 0, s>>>((const Cx*)T, g, (Cx*)w);
}

// Partial Hermitian-weighted dots <V_y, w> for y < nv, and <w, w> for y = nv.
template <typename R>
__global__ void k_mdot(const typename Tr<R>::Cx* w, const typename Tr<R>::Cx* V, size_t vstride,
                       int nv, SGrid g, double* part) {
    typedef typename Tr<R>::Cx Cx;
    __shared__ double sh[32];
    const size_t Nh = g.Nh;
    const int y = blockIdx.y;
    const Cx* a = y < nv ? V + (size_t)y * vstride : w;
    double acc = 0;
    GRID_STRIDE(e, Nh) {
        R xi[3], xd[3], wt;
        hs_freq<R>(g, e, xi, xd, wt);
        R s = 0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const Cx p = a[i * Nh + e], q = w[i * Nh + e];
            s += p.x * q.x + p.y * q.y;
        }
        acc += (double)wt * (double)s;
    }
    const double r = block_sum<kThreads>(acc, sh);
    if (threadIdx.x == 0) part[(size_t)y * gridDim.x + blockIdx.x] = r;
}
template <typename R>
void mdot(const void* w, const void* V, size_t vstride, int nv, int with_norm, const SGrid& g,
          double* part, cudaStream_t s) {
    typedef typename Tr<R>::Cx Cx;
    k_mdot<R><<<dim3(kRedBlocks, nv + (with_norm ? 1 : 0)), kThreads, 0, s>>>(
        (const Cx*)w, (const Cx*)V, vstride, nv, g, part);
}

// w -= sum_i h_i V_i
template <typename R>
__global__ void k_gs_update(typename Tr<R>::Cx* w, const typename Tr<R>::Cx* V, size_t vstride,
                            int nv, const double* h, size_t n3) {
    typedef typename Tr<R>::Cx Cx;
    GRID_STRIDE(e, n3) {
        Cx a = w[e];
        for (int i = 0; i < nv; ++i) {
            const R hi = (R)h[i];
            const Cx v = V[(size_t)i * vstride + e];
            a.x -= hi * v.x;
            a.y -= hi * v.y;
        }
        w[e] = a;
    }
}
template <typename R>
void gs_update(void* w, const void* V, size_t vstride, int nv, const double* h, size_t n3,
               cudaStream_t s) {
    typedef typename Tr<R>::Cx Cx;
    k_gs_update<R><<<grid_for(n3), kThreads, 0, s>>>((Cx*)w, (const Cx*)V, vstride, nv, h, n3);
}

// x += M (sum_i y_i V_i)  (right-preconditioned GMRES update)
template <typename R>
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
        if (xd[0] == R(0) && xd[1] == R(0) && xd[2] == R(0)) continue;
        Cx c[3];
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
        R A[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int kk = 0; kk < 3; ++kk) {
                R s = 0;
#pragma unroll
                for (int j = 0; j < 3; ++j)
#pragma unroll
                    for (int l = 0; l < 3; ++l) s += xd[j] * Ks[9 * (3 * i + j) + 3 * kk + l] * xd[l];
                A[3 * i + kk] = s;
            }
        const R det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                      A[2] * (A[3] * A[7] - A[4] * A[6]);
        const R id = R(1) / det;
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
            Cx xv = x[i * Nh + e];
            xv.x += Mi[3 * i] * c[0].x + Mi[3 * i + 1] * c[1].x + Mi[3 * i + 2] * c[2].x;
            xv.y += Mi[3 * i] * c[0].y + Mi[3 * i + 1] * c[1].y + Mi[3 * i + 2] * c[2].y;
            x[i * Nh + e] = xv;
        }
    }
}
template <typename R>
void xupdate(void* x, const void* V, size_t vstride, int k, const double* y, const double* Kbar,
             const SGrid& g, cudaStream_t s) {
    typedef typename Tr<R>::Cx Cx;
    k_xupdate<R><<<grid_for(g.Nh), kThreads, 0, s>>>((Cx*)x, (const Cx*)V, vstride, k, y, Kbar,
                                                     g);
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

// ----------------------------------------------------------- Newton update
// H += grad(du) (arriving scaled by N); partial maxima of |grad du| and
// |H - Ht| (the test of Sec. 3.1).
template <typename R>
__global__ void k_fupdate(R* H, const R* G, R invN, const R* Ht, size_t N, double* part) {
    __shared__ double sh[32];
    double m0 = 0, m1 = 0;
    GRID_STRIDE(v, N) {
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            const R d = G[c * N + v] * invN;
            const R h = H[c * N + v] + d;
            H[c * N + v] = h;
            m0 = fmax(m0, (double)fabs(d));
            m1 = fmax(m1, (double)fabs(h - Ht[c * N + v]));
        }
    }
    double r = block_max<kThreads>(m0, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = r;
    r = block_max<kThreads>(m1, sh);
    if (threadIdx.x == 0) part[kRedBlocks + blockIdx.x] = r;
}
template <typename R>
void fupdate(void* H, const void* G, const void* Ht, size_t N, double* part, cudaStream_t s) {
    k_fupdate<R><<<kRedBlocks, kThreads, 0, s>>>((R*)H, (const R*)G, (R)(1.0 / (double)N),
                                                 (const R*)Ht, N, part);
}

template <typename R>
__global__ void k_maxdiff(const R* a, const R* b, size_t n, double* part) {
    __shared__ double sh[32];
    double m = 0;
    GRID_STRIDE(i, n) m = fmax(m, (double)fabs(a[i] - b[i]));
    const double r = block_max<kThreads>(m, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = r;
}
template <typename R>
void maxdiff(const void* a, const void* b, size_t n, double* part, cudaStream_t s) {
    k_maxdiff<R><<<kRedBlocks, kThreads, 0, s>>>((const R*)a, (const R*)b, n, part);
}

template <typename R>
__global__ void k_maxval(const R* a, size_t n, double* part) {
    __shared__ double sh[32];
    double m = 0;
    GRID_STRIDE(i, n) m = fmax(m, (double)a[i]);
    const double r = block_max<kThreads>(m, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = r;
}
template <typename R>
void maxval(const void* a, size_t n, double* part, cudaStream_t s) {
    k_maxval<R><<<kRedBlocks, kThreads, 0, s>>>((const R*)a, n, part);
}

// <g(phi) P_c> partial sums (grid.y = 9)
template <typename R>
__global__ void k_pbar(const R* P, const R* phi, R kres, size_t N, double* part) {
    __shared__ double sh[32];
    const int c = blockIdx.y;
    double a = 0;
    GRID_STRIDE(v, N) {
        const R om = R(1) - phi[v];
        a += (double)((om * om + kres) * P[(size_t)c * N + v]);
    }
    const double s = block_sum<kThreads>(a, sh);
    if (threadIdx.x == 0) part[(size_t)c * gridDim.x + blockIdx.x] = s;
}
template <typename R>
void pbar(const void* P, const void* phi, double kres, size_t N, double* part, cudaStream_t s) {
    k_pbar<R><<<dim3(kRedBlocks, 9), kThreads, 0, s>>>((const R*)P, (const R*)phi, (R)kres, N,
                                                       part);
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

// r = 2S - (1 + 2S) x - lapx; partials ||r||^2 and ||2S||^2
template <typename R>
__global__ void k_pf_init(const R* x, const R* lapx, const R* S, R* r, size_t N, double* part) {
    __shared__ double sh[32];
    double a = 0, b = 0;
    GRID_STRIDE(v, N) {
        const R s2 = R(2) * S[v];
        const R rv = s2 - (R(1) + s2) * x[v] - lapx[v];
        r[v] = rv;
        a += (double)rv * rv;
        b += (double)s2 * s2;
    }
    double q = block_sum<kThreads>(a, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = q;
    q = block_sum<kThreads>(b, sh);
    if (threadIdx.x == 0) part[kRedBlocks + blockIdx.x] = q;
}
template <typename R>
void pf_init(const void* x, const void* lapx, const void* S, void* r, size_t N, double* part,
             cudaStream_t s) {
    k_pf_init<R><<<kRedBlocks, kThreads, 0, s>>>((const R*)x, (const R*)lapx, (const R*)S,
                                                 (R*)r, N, part);
}

template <typename R>
__global__ void k_rdot(const R* a, const R* b, size_t N, double* part) {
    __shared__ double sh[32];
    double acc = 0;
    GRID_STRIDE(v, N) acc += (double)a[v] * (double)b[v];
    const double q = block_sum<kThreads>(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = q;
}
template <typename R>
void rdot(const void* a, const void* b, size_t N, double* part, cudaStream_t s) {
    k_rdot<R><<<kRedBlocks, kThreads, 0, s>>>((const R*)a, (const R*)b, N, part);
}

// q = t + 2 S p  (A p through the recurrence t = M^-1 p);  partial <p, q>
template <typename R>
__global__ void k_pf_q(const R* t, const R* p, const R* S, R* q, size_t N, double* part) {
    __shared__ double sh[32];
    double acc = 0;
    GRID_STRIDE(v, N) {
        const R qv = t[v] + R(2) * S[v] * p[v];
        q[v] = qv;
        acc += (double)p[v] * qv;
    }
    const double r = block_sum<kThreads>(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = r;
}
template <typename R>
void pf_q(const void* t, const void* p, const void* S, void* q, size_t N, double* part,
          cudaStream_t s) {
    k_pf_q<R><<<kRedBlocks, kThreads, 0, s>>>((const R*)t, (const R*)p, (const R*)S, (R*)q, N,
                                              part);
}

// x += alpha p; r -= alpha q; partial ||r||^2
template <typename R>
__global__ void k_pf_xr(R* x, R* r, const R* p, const R* q, R alpha, size_t N, double* part) {
    __shared__ double sh[32];
    double acc = 0;
    GRID_STRIDE(v, N) {
        x[v] += alpha * p[v];
        const R rv = r[v] - alpha * q[v];
        r[v] = rv;
        acc += (double)rv * rv;
    }
    const double q2 = block_sum<kThreads>(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = q2;
}
template <typename R>
void pf_xr(void* x, void* r, const void* p, const void* q, double alpha, size_t N, double* part,
           cudaStream_t s) {
    k_pf_xr<R><<<kRedBlocks, kThreads, 0, s>>>((R*)x, (R*)r, (const R*)p, (const R*)q, (R)alpha,
                                               N, part);
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

// phi_new = max(x, phi_t) (irreversibility, Algorithm 1); partial maxima of
// |phi_new - phi_old|, |phi_new - phi_t|, and counts of changed and cracked
// (phi >= 0.9) voxels.
template <typename R>
__global__ void k_pf_clamp(const R* x, const R* phi_t, R* phi, size_t N, double* part) {
    __shared__ double sh[32];
    double m0 = 0, m1 = 0, c0 = 0, c1 = 0;
    GRID_STRIDE(v, N) {
        const R pt = phi_t[v];
        const R pn = fmax(x[v], pt);
        const R po = phi[v];
        phi[v] = pn;
        m0 = fmax(m0, (double)fabs(pn - po));
        m1 = fmax(m1, (double)fabs(pn - pt));
        c0 += pn != po ? 1.0 : 0.0;
        c1 += pn >= R(0.9) ? 1.0 : 0.0;
    }
    double r = block_max<kThreads>(m0, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = r;
    r = block_max<kThreads>(m1, sh);
    if (threadIdx.x == 0) part[kRedBlocks + blockIdx.x] = r;
    r = block_sum<kThreads>(c0, sh);
    if (threadIdx.x == 0) part[2 * kRedBlocks + blockIdx.x] = r;
    r = block_sum<kThreads>(c1, sh);
    if (threadIdx.x == 0) part[3 * kRedBlocks + blockIdx.x] = r;
}
template <typename R>
void pf_clamp(const void* x, const void* phi_t, void* phi, size_t N, double* part,
              cudaStream_t s) {
    k_pf_clamp<R><<<kRedBlocks, kThreads, 0, s>>>((const R*)x, (const R*)phi_t, (R*)phi, N, part);
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

// ------------------------------------------------------- instantiations
#define INST(R)                                                                                \
    template void add_uniform<R>(void*, const void*, const double*, size_t, cudaStream_t);      \
    template void fp_sample<R>(const void*, const int32_t*, const double*, void*, size_t,       \
                               cudaStream_t);                                                   \
    template void nye<R>(void*, const SGrid&, double, cudaStream_t);                            \
    template void gnd_rho<R>(const void*, const int32_t*, const double*, const double*, double, \
                             void*, size_t, cudaStream_t);                                      \
    template void kbar<R>(const void*, const void*, double, size_t, double*, cudaStream_t);     \
    template void degrade<R>(const void*, const void*, double, void*, size_t, cudaStream_t);    \
    template void residual<R>(const void*, const SGrid&, void*, double*, cudaStream_t);         \
    template void precond_grad<R>(const void*, double, void*, const double*, const SGrid&,      \
                                  void*, int, cudaStream_t);                                    \
    template void tangent_apply<R>(void*, const void*, const void*, double, size_t,             \
                                   cudaStream_t);                                               \
    template void contract<R>(const void*, const SGrid&, void*, cudaStream_t);                  \
    template void hermitize<R>(void*, int, const SGrid&, cudaStream_t);                         \
    template void mdot<R>(const void*, const void*, size_t, int, int, const SGrid&, double*,    \
                          cudaStream_t);                                                        \
    template void gs_update<R>(void*, const void*, size_t, int, const double*, size_t,          \
                               cudaStream_t);                                                   \
    template void xupdate<R>(void*, const void*, size_t, int, const double*, const double*,     \
                             const SGrid&, cudaStream_t);                                       \
    template void axpby<R>(void*, const void*, const void*, double, double, size_t,             \
                           cudaStream_t);                                                       \
    template void fupdate<R>(void*, const void*, const void*, size_t, double*, cudaStream_t);   \
    template void maxdiff<R>(const void*, const void*, size_t, double*, cudaStream_t);          \
    template void maxval<R>(const void*, size_t, double*, cudaStream_t);                        \
    template void pbar<R>(const void*, const void*, double, size_t, double*, cudaStream_t);     \
    template void pf_spec<R>(void*, const SGrid&, double, int, cudaStream_t);                   \
    template void pf_init<R>(const void*, const void*, const void*, void*, size_t, double*,     \
                             cudaStream_t);                                                     \
    template void rdot<R>(const void*, const void*, size_t, double*, cudaStream_t);             \
    template void pf_q<R>(const void*, const void*, const void*, void*, size_t, double*,        \
                          cudaStream_t);                                                        \
    template void pf_xr<R>(void*, void*, const void*, const void*, double, size_t, double*,     \
                           cudaStream_t);                                                       \
    template void pf_pt<R>(void*, void*, const void*, const void*, double, size_t,              \
                           cudaStream_t);                                                       \
    template void pf_clamp<R>(const void*, const void*, void*, size_t, double*, cudaStream_t);  \
    template void to_double<R>(const void*, double*, size_t, size_t, int, cudaStream_t);        \
    template void from_double<R>(const double*, void*, size_t, size_t, int, cudaStream_t);      \
    template void fp_in<R>(const double*, const int32_t*, const double*, void*, size_t,         \
                           cudaStream_t);
INST(float)
INST(double)

}  // namespace fatfft
