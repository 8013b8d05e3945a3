// Fused x pass of the GMRES operator
//   w = -div( g(phi) K : grad( M c ) )          (Eqs. newton, precf)
// The Arnoldi step keeps its 9-component gradient and stress spectra in an
// interleaved half-spectrum layout, row (y, z) by row: entry kx of field c in
// row r at (9 r + c) n0h + kx (n0h = n0/2 + 1), so that
//   * the transforms along y and z are one batched 2-D complex transform
//     over (z, y) (batch 9 n0h, element stride 9 n0h, done by cuFFT), and
//   * this kernel does, per block of rows, everything along x at once: the
//     inverse real transform of all 9 gradient components of each row, the
//     tangent apply tau = g(phi) K : grad z / N at every voxel of the rows,
//     and the forward real transform of tau -- the gradient and the stress
//     field never exist in real space in memory, and the tangent apply is
//     not a separate pass over the 9 real fields.
// The real transforms along x use the half-length complex transform
// (z[m] = x[2m] + i x[2m+1], length n0/2) with the usual split of the
// even and odd parts, a radix-4/2 Stockham iteration per warp in shared
// memory (warp-synchronous, no block barrier) and twiddles from a table
// computed on the host in double precision.  Conventions as in the rest of
// the library: forward unnormalised, inverse unnormalised (1/N folded into
// the tangent apply), and the inverse reads only the real parts of the
// kx = 0 and Nyquist entries.
#include <cmath>

#include "common.cuh"
#include "spec.h"

namespace fatfft {

// Radix-R DFT in registers (R = 2 or 4); SIGN = -1 forward, +1 inverse.
template <typename Cx, typename R, int SIGN>
__device__ __forceinline__ void dft_r(Cx* v, int rad) {
    if (rad == 2) {
        const Cx a = v[0], b = v[1];
        v[0].x = a.x + b.x;
        v[0].y = a.y + b.y;
        v[1].x = a.x - b.x;
        v[1].y = a.y - b.y;
        return;
    }
    // y1 = (a0 - a2) + w (a1 - a3), y3 = (a0 - a2) - w (a1 - a3), w = SIGN i
    Cx t0, t1, t2, t3;
    t0.x = v[0].x + v[2].x;
    t0.y = v[0].y + v[2].y;
    t1.x = v[0].x - v[2].x;
    t1.y = v[0].y - v[2].y;
    t2.x = v[1].x + v[3].x;
    t2.y = v[1].y + v[3].y;
    const R dx = v[1].x - v[3].x, dy = v[1].y - v[3].y;
    t3.x = -R(SIGN) * dy;  // SIGN i (dx + i dy)
    t3.y = R(SIGN) * dx;
    v[0].x = t0.x + t2.x;
    v[0].y = t0.y + t2.y;
    v[2].x = t0.x - t2.x;
    v[2].y = t0.y - t2.y;
    v[1].x = t1.x + t3.x;
    v[1].y = t1.y + t3.y;
    v[3].x = t1.x - t3.x;
    v[3].y = t1.y - t3.y;
}

// ncol lines of length m (a power of two) owned by one warp, line c at
// a[c * m]; b is scratch of the same size.  Self-sorting Stockham stages of
// radix 4 (and one of radix 2 for odd powers); Wn holds exp(-2 pi i t / n)
// for t < n = 2 m (the line's twiddle exp(-2 pi i t / m) is Wn[2 t]).
// Returns the buffer holding the result.  Every lane of the warp calls it.
template <typename Cx, typename R, int SIGN>
__device__ Cx* warp_fft(Cx* a, Cx* b, int m, int ncol, const Cx* Wn) {
    const int lane = threadIdx.x & 31;
    int Ns = 1;
    while (Ns < m) {
        const int rad = (m / Ns) % 4 == 0 ? 4 : 2;
        const int q = m / rad;  // butterflies per line
        const int step = q / Ns;
        const int tot = ncol * q;
        for (int t = lane; t < tot; t += 32) {
            const int col = t / q, j = t - col * q;
            const int jm = j & (Ns - 1);
            const Cx* src = a + col * m;
            Cx v[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (r < rad) {
                    Cx x = src[j + r * q];
                    if (r > 0 && jm > 0) {
                        Cx w = Wn[2 * jm * r * step];
                        if (SIGN > 0) w.y = -w.y;
                        const R xr = x.x * w.x - x.y * w.y;
                        x.y = x.x * w.y + x.y * w.x;
                        x.x = xr;
                    }
                    v[r] = x;
                }
            }
            dft_r<Cx, R, SIGN>(v, rad);
            Cx* dst = b + col * m + (j - jm) * rad + jm;
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (r < rad) dst[r * Ns] = v[r];
        }
        __syncwarp();
        Cx* t = a;
        a = b;
        b = t;
        Ns *= rad;
    }
    return a;
}

template <typename R> struct V2of;
template <> struct V2of<float> { typedef float2 T; };
template <> struct V2of<double> { typedef double2 T; };

// One block: rb consecutive rows (y, z), 8 warps; warp w owns lines
// w * lpw .. (w + 1) * lpw - 1 of the 9 rb (row, field) lines, line
// L = 9 * row + field.  Shared memory: the twiddles (n0), the warps' line
// buffers (2 x 8 lpw lines of m = n0/2 complex) and the real fields of the
// rows (9 x rb x n0).
template <typename R>
__global__ void __launch_bounds__(256) k_xpass(typename Tr<R>::Cx* G, const R* K, const R* phi,
                                               R kres, R invN, SGrid g, FusedX p) {
    typedef typename Tr<R>::Cx Cx;
    extern __shared__ __align__(16) unsigned char dyn[];
    const int n = g.n0, m = n / 2, nh = g.n0h, rb = p.rb, lpw = p.lpw;
    const int row0 = blockIdx.x * rb;
    const int nrow = min(rb, g.n1 * g.n2 - row0);
    const int nline = 9 * nrow;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Cx* Ws = (Cx*)dyn;
    Cx* bufa = Ws + n + (size_t)w * 2 * lpw * m;
    Cx* bufb = bufa + (size_t)lpw * m;
    R* F = (R*)(Ws + n + (size_t)8 * 2 * lpw * m);  // [9][rb][n]
    const Cx* tw = (const Cx*)p.tw;
    for (int i = threadIdx.x; i < n; i += blockDim.x) Ws[i] = tw[i];
    __syncthreads();
    const int L0 = w * lpw;
    const int nl = max(0, min(lpw, nline - L0));  // this warp's lines
    // inverse: Z[k] = (A + B) + i W^-k (A - B), A = X[k], B = conj X[m - k]
    for (int t = lane; t < nl * m; t += 32) {
        const int li = t / m, k = t - li * m;
        const int L = L0 + li, rw = L / 9, c = L - 9 * rw;
        const Cx* X = G + ((size_t)(row0 + rw) * 9 + c) * nh;
        Cx A = X[k], B = X[m - k];
        if (k == 0) {
            A.y = 0;  // real parts only on kx = 0 and the Nyquist entry
            B.y = 0;
        }
        B.y = -B.y;
        const Cx wk = Ws[k];  // exp(-2 pi i k / n); W^-k is its conjugate
        const R dx = A.x - B.x, dy = A.y - B.y;
        // i conj(wk) (dx + i dy)
        const R px = wk.x * dx + wk.y * dy, py = wk.x * dy - wk.y * dx;
        Cx z;
        z.x = A.x + B.x - py;
        z.y = A.y + B.y + px;
        bufa[li * m + k] = z;
    }
    __syncwarp();
    const Cx* zr = warp_fft<Cx, R, +1>(bufa, bufb, m, nl, Ws);
    for (int t = lane; t < nl * m; t += 32) {
        const int li = t / m, k = t - li * m;
        const int L = L0 + li, rw = L / 9, c = L - 9 * rw;
        const Cx z = zr[li * m + k];
        R* f = F + ((size_t)c * rb + rw) * n;
        f[2 * k] = z.x;
        f[2 * k + 1] = z.y;
    }
    __syncthreads();
    // tangent apply, two neighbouring voxels per thread (every K and phi
    // offset is even: 2-wide aligned loads along x)
    typedef typename V2of<R>::T T2;
    const size_t N = g.N;
    for (int t = threadIdx.x; t < nrow * m; t += blockDim.x) {
        const int rw = t / m, x = 2 * (t - rw * m);
        const size_t v = (size_t)(row0 + rw) * n + x;
        R g0[9], g1[9];
#pragma unroll
        for (int b = 0; b < 9; ++b) {
            g0[b] = F[((size_t)b * rb + rw) * n + x];
            g1[b] = F[((size_t)b * rb + rw) * n + x + 1];
        }
        const T2 ph = *reinterpret_cast<const T2*>(phi + v);
        const R o0 = R(1) - ph.x, o1 = R(1) - ph.y;
        const R s0 = (o0 * o0 + kres) * invN, s1 = (o1 * o1 + kres) * invN;
        R r0[9], r1[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            R t0 = 0, t1 = 0;
#pragma unroll
            for (int b = 0; b < 9; ++b) {
                const T2 kk = *reinterpret_cast<const T2*>(K + (size_t)(9 * a + b) * N + v);
                t0 += kk.x * g0[b];
                t1 += kk.y * g1[b];
            }
            r0[a] = s0 * t0;
            r1[a] = s1 * t1;
        }
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            F[((size_t)a * rb + rw) * n + x] = r0[a];
            F[((size_t)a * rb + rw) * n + x + 1] = r1[a];
        }
    }
    __syncthreads();
    // forward: z[k] = tau[2k] + i tau[2k + 1], Z = FFT_m(z),
    // X[k] = (Z[k] + conj Z[m-k]) / 2 - i W^k (Z[k] - conj Z[m-k]) / 2
    for (int t = lane; t < nl * m; t += 32) {
        const int li = t / m, k = t - li * m;
        const int L = L0 + li, rw = L / 9, c = L - 9 * rw;
        const R* f = F + ((size_t)c * rb + rw) * n;
        Cx z;
        z.x = f[2 * k];
        z.y = f[2 * k + 1];
        bufa[li * m + k] = z;
    }
    __syncwarp();
    const Cx* Z = warp_fft<Cx, R, -1>(bufa, bufb, m, nl, Ws);
    for (int t = lane; t < nl * (m + 1); t += 32) {
        const int li = t / (m + 1), k = t - li * (m + 1);
        const int L = L0 + li, rw = L / 9, c = L - 9 * rw;
        const Cx Zk = Z[li * m + (k == m ? 0 : k)];
        Cx Zc = Z[li * m + (k == 0 ? 0 : m - k)];
        Zc.y = -Zc.y;
        const Cx wk = Ws[k];  // exp(-2 pi i k / n), k <= m < n
        const R sx = R(0.5) * (Zk.x + Zc.x), sy = R(0.5) * (Zk.y + Zc.y);
        const R dx = R(0.5) * (Zk.x - Zc.x), dy = R(0.5) * (Zk.y - Zc.y);
        // -i wk (dx + i dy) = (wk.x dy + wk.y dx, -(wk.x dx - wk.y dy))
        Cx X;
        X.x = sx + wk.x * dy + wk.y * dx;
        X.y = sy - (wk.x * dx - wk.y * dy);
        G[((size_t)(row0 + rw) * 9 + c) * nh + k] = X;
    }
}

// ------------------------------------------------------------------- host
template <typename R>
static size_t xpass_smem(int n, int rb) {
    typedef typename Tr<R>::Cx Cx;
    const int lpw = (9 * rb + 7) / 8;
    return sizeof(Cx) * ((size_t)n + (size_t)8 * 2 * lpw * (n / 2)) +
           sizeof(R) * (size_t)9 * rb * n;
}

// Plan of the fused x pass: n0 a power of two in [8, 512]; rows per block
// as many as fit in about 100 KB of shared memory (at most 8).  0 if the
// grid is not supported (the Arnoldi step then uses the library 3-D
// transforms and the separate tangent apply).
template <typename R>
int fused_x_plan(FusedX& p, const SGrid& g) {
    p = FusedX{};
    const int n = g.n0;
    if (n < 8 || n > kFftMaxLen || (n & (n - 1)) != 0) return 0;
    int rb = 8;
    while (rb > 1 && xpass_smem<R>(n, rb) > 100 * 1024) rb /= 2;
    p.rb = rb;
    p.lpw = (9 * rb + 7) / 8;
    p.smem = xpass_smem<R>(n, rb);
    if (p.smem > 200 * 1024 ||
        cudaFuncSetAttribute(k_xpass<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)p.smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    p.ok = 1;
    return 1;
}

// Twiddle table exp(-2 pi i t / n), t < n, in the bulk complex type (host
// memory, n entries of 2 * sizeof(R) bytes).
template <typename R>
void fused_x_twiddles(int n, void* host) {
    typedef typename Tr<R>::Cx Cx;
    Cx* t = (Cx*)host;
    for (int i = 0; i < n; ++i) {
        const double a = -2.0 * M_PI * (double)i / (double)n;
        t[i].x = (R)std::cos(a);
        t[i].y = (R)std::sin(a);
    }
}

template <typename R>
void fused_xpass(const FusedX& p, void* G, const void* K, const void* phi, double kres,
                 const SGrid& g, cudaStream_t s) {
    typedef typename Tr<R>::Cx Cx;
    const unsigned nb = (unsigned)((g.n1 * g.n2 + p.rb - 1) / p.rb);
    k_xpass<R><<<nb, 256, p.smem, s>>>((Cx*)G, (const R*)K, (const R*)phi, (R)kres,
                                       (R)(1.0 / (double)g.N), g, p);
}

template int fused_x_plan<float>(FusedX&, const SGrid&);
template int fused_x_plan<double>(FusedX&, const SGrid&);
template void fused_x_twiddles<float>(int, void*);
template void fused_x_twiddles<double>(int, void*);
template void fused_xpass<float>(const FusedX&, void*, const void*, const void*, double,
                                 const SGrid&, cudaStream_t);
template void fused_xpass<double>(const FusedX&, void*, const void*, const void*, double,
                                  const SGrid&, cudaStream_t);

}  // namespace fatfft
