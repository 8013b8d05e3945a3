// Shared device-side helpers of the fatiguefft library.
#pragma once
#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

namespace fatfft {

// ---- precision traits: R is the bulk real type, Cx the matching complex ----
template <typename R> struct Tr;
template <> struct Tr<double> {
    typedef double2 Cx;
    static constexpr double eps = 2.220446049250313e-16;
};
template <> struct Tr<float> {
    typedef float2 Cx;
    static constexpr double eps = 1.1920928955078125e-7;
};

// ---- launch geometry ----
constexpr int kThreads = 256;
// Reduction kernels run a fixed grid (two blocks per SM of the 152) so that
// their partial sums are combined in a fixed order (deterministic results).
constexpr int kRedBlocks = 304;
// Largest Krylov basis (GMRES restart length) the fused kernels support.
constexpr int kMaxKrylov = 32;
// Partial-sum slots per reduction (values x blocks) in the scratch buffer.
constexpr int kRedSlots = 256;

inline int grid_for(size_t n, int threads = kThreads) {
    size_t b = (n + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

// ---- 3x3 helpers (row-major) ----
template <typename R>
__device__ __forceinline__ void mm3(const R* a, const R* b, R* c) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            c[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
}
// c = a^T b
template <typename R>
__device__ __forceinline__ void mtm3(const R* a, const R* b, R* c) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            c[3 * i + j] = a[i] * b[j] + a[3 + i] * b[3 + j] + a[6 + i] * b[6 + j];
}
// c = a b^T
template <typename R>
__device__ __forceinline__ void mmt3(const R* a, const R* b, R* c) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            c[3 * i + j] = a[3 * i] * b[3 * j] + a[3 * i + 1] * b[3 * j + 1] + a[3 * i + 2] * b[3 * j + 2];
}

// ---- block reductions (double accumulation) ----
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < NT / 32; ++i) s += sh[i];
    return s;  // valid in thread 0
}
template <int NT>
__device__ __forceinline__ double block_max(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < NT / 32; ++i) s = fmax(s, sh[i]);
    return s;
}

// ---- grid-wide multi-value reductions finished by the last block ----
// Every block reduces its per-thread accumulators to one partial per value
// (part[v * gridDim.x + blockIdx.x]; a 2-D grid gives each row of blocks its
// own value, written through part + blockIdx.y * gridDim.x); the last block
// of the whole grid to finish (atomic ticket)
// combines the partials in block order and writes out[v] -- sums scaled by
// `scale`, values whose bit is set in `maxmask` as maxima.  The combination
// order is fixed, so results do not depend on which block finishes last.
struct Red {
    double* part;       // [values][gridDim.x] partials
    unsigned* counter;  // zero between reductions
    double* out;        // [values] results
};

// Per-block partial sums (or maxima, bit v of maxmask) of nv <= NV values:
// warp shuffles and the combine over warps run in the accumulator type T
// (the bulk type: FP64 arithmetic is a narrow pipe on this GPU), and one
// FP64 partial per value is stored at part[v * gridDim.x + blockIdx.x].
template <int NV, int NT, typename T>
__device__ __forceinline__ void block_partials(const T (&acc)[NV], int nv, unsigned maxmask,
                                               double* part) {
    __shared__ T sh[NT / 32][NV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        if (v < nv) {
            T x = acc[v];
            const bool mx = v < 32 && ((maxmask >> v) & 1u);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const T y = __shfl_down_sync(0xffffffffu, x, o);
                x = mx ? (x > y ? x : y) : x + y;
            }
            if (lane == 0) sh[wid][v] = x;
        }
    }
    __syncthreads();
    for (int v = threadIdx.x; v < nv; v += NT) {
        const bool mx = v < 32 && ((maxmask >> v) & 1u);
        T s = 0;
        for (int w = 0; w < NT / 32; ++w) s = mx ? (s > sh[w][v] ? s : sh[w][v]) : s + sh[w][v];
        part[(size_t)v * gridDim.x + blockIdx.x] = (double)s;
        __threadfence();  // publish the partial before the block takes its ticket
    }
}

// Returns true in the block that combined the partials (block-uniform).
// NVMAX bounds nv at compile time: warp w of the last block combines values
// w, w + NT/32, ..., issuing the loads of all its values before reducing
// (one L2 round trip per 32 partials instead of one per value).
template <int NT, int NVMAX>
__device__ __forceinline__ bool grid_finish(const Red& r, int nv, unsigned maxmask, double scale) {
    constexpr int NW = NT / 32;
    constexpr int VPW = (NVMAX + NW - 1) / NW;
    __shared__ unsigned s_last;
    __syncthreads();  // the writers' partials are fenced (block_partials)
    const unsigned total = gridDim.x * gridDim.y;  // 2-D grids: one value per row of blocks
    if (threadIdx.x == 0) s_last = atomicAdd(r.counter, 1u) == total - 1 ? 1u : 0u;
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nb = gridDim.x;
    double s[VPW];
#pragma unroll
    for (int j = 0; j < VPW; ++j) s[j] = 0.0;
#pragma unroll 8
    for (int i = lane; i < nb; i += 32) {
        double x[VPW];
#pragma unroll
        for (int j = 0; j < VPW; ++j) {
            const int v = w + j * NW;
            x[j] = v < nv ? __ldcg(r.part + (size_t)v * nb + i) : 0.0;
        }
#pragma unroll
        for (int j = 0; j < VPW; ++j) {
            const int v = w + j * NW;
            s[j] = ((maxmask >> (v & 31)) & 1u) && v < 32 ? fmax(s[j], x[j]) : s[j] + x[j];
        }
    }
#pragma unroll
    for (int j = 0; j < VPW; ++j) {
        const int v = w + j * NW;
        const bool mx = v < 32 && ((maxmask >> v) & 1u);
        double t = s[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_down_sync(0xffffffffu, t, o);
            t = mx ? fmax(t, y) : t + y;
        }
        if (lane == 0 && v < nv) r.out[v] = mx ? t : t * scale;
    }
    if (threadIdx.x == 0) *r.counter = 0u;
    return true;
}

// Neumaier compensated addition: (s, c) += x.
__device__ __forceinline__ void neumaier(double& s, double& c, double x) {
    const double t = s + x;
    if (fabs(s) >= fabs(x))
        c += (s - t) + x;
    else
        c += (x - t) + s;
    s = t;
}

}  // namespace fatfft
