// Unsigned 32-bit division by a run-time invariant divisor with one
// multiply-high, after Granlund & Montgomery, "Division by invariant integers
// using multiplication" (PLDI 1994), Sec. 4: with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1,
//   q = (t + ((x - t) >> min(l, 1))) >> max(l - 1, 0),  t = mulhi(m, x),
// equals floor(x / d) for every 32-bit x and 1 <= d < 2^32.  The frequency
// decode of the half-spectrum kernels divides by the grid extents this way.
// Plain C++ on the host (also compiled by the CPU test) and CUDA on the device.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define FASTDIV_HD __host__ __device__ __forceinline__
#else
#define FASTDIV_HD inline
#endif

namespace fatfft {

struct FastDiv {
    uint32_t d, m, s1, s2;
};

inline FastDiv make_fastdiv(uint32_t d) {
    uint32_t l = 0;
    while (l < 32 && (1ull << l) < (uint64_t)d) ++l;  // ceil(log2 d)
    FastDiv f;
    f.d = d;
    f.m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 1 ? l - 1 : 0;
    return f;
}

FASTDIV_HD uint32_t fdiv(uint32_t x, const FastDiv& f) {
#if defined(__CUDA_ARCH__)
    const uint32_t t = __umulhi(f.m, x);
#else
    const uint32_t t = (uint32_t)(((uint64_t)f.m * x) >> 32);
#endif
    return (t + ((x - t) >> f.s1)) >> f.s2;
}

}  // namespace fatfft
