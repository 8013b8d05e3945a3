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
// Reduction kernels run a fixed grid (a multiple of the 152 SMs) so that
// their partial sums are combined in a fixed order (deterministic results).
constexpr int kRedBlocks = 608;

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
