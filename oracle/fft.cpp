// Oracle transforms (test infrastructure only).
//
// The paper obtains the Fourier transform of a voxel field with the DFT,
// computed by an FFT (Sec. 3.1).  This file gives the oracle its own
// transforms: a recursive decimation-in-time Cooley-Tukey FFT for any length
// (radix = the smallest prime factor at each level, so lengths 2^a 3^b run in
// O(n log n) and other primes fall back to a direct butterfly) and a naive
// O(N^2) 3-D DFT used to check it.
#include "oracle_internal.hpp"

#include <cmath>
#include <cstring>
#include <vector>

namespace orc {

static int smallest_factor(int n) {
    for (int p = 2; p * p <= n; ++p)
        if (n % p == 0) return p;
    return n;
}

// out[k] = sum_j in[j*stride] * exp(sign*2*pi*i*j*k/n), k = 0..n-1.
// tw[t] = exp(sign*2*pi*i*t/ntop); a length-n sub-problem uses every
// (ntop/n)-th entry.
static void fft_rec(const cplx* in, cplx* out, int n, int stride, const cplx* tw,
                    int ntop, cplx* scratch) {
    if (n == 1) {
        out[0] = in[0];
        return;
    }
    const int p = smallest_factor(n);
    const int m = n / p;
    // p interleaved sub-sequences in[(r + p*j)*stride], each transformed
    // into out[r*m .. r*m+m-1].
    for (int r = 0; r < p; ++r)
        fft_rec(in + (size_t)r * stride, out + (size_t)r * m, m, stride * p, tw, ntop,
                scratch + n);
    // X[k + m*q] = sum_r exp(sign 2 pi i r (k + m q) / n) * Sub_r[k]
    const int step = ntop / n;
    for (int k = 0; k < m; ++k) {
        for (int q = 0; q < p; ++q) {
            const int kk = k + m * q;
            cplx s(0.0, 0.0);
            for (int r = 0; r < p; ++r) {
                const long t = ((long)r * kk) % n;
                s += out[(size_t)r * m + k] * tw[(size_t)t * step];
            }
            scratch[kk] = s;
        }
    }
    for (int k = 0; k < n; ++k) out[k] = scratch[k];
}

void fft1d(cplx* data, int n, int sign) {
    if (n <= 1) return;
    std::vector<cplx> tw(n), in(data, data + n), scratch(4 * (size_t)n + 64);
    const double two_pi = 2.0 * M_PI;
    for (int t = 0; t < n; ++t) {
        const double a = sign * two_pi * (double)t / (double)n;
        tw[t] = cplx(std::cos(a), std::sin(a));
        if ((4L * t) % n == 0) {  // exact values on the quarter turns
            const int q = (int)((4L * t) / n);
            const double re[4] = {1, 0, -1, 0}, im[4] = {0, 1, 0, -1};
            tw[t] = cplx(re[q], sign * im[q]);
        }
    }
    fft_rec(in.data(), data, n, 1, tw.data(), n, scratch.data());
}

// Transform every line along one axis of a 3-D array.
static void transform_axis(const int n[3], cplx* a, int axis, int sign) {
    const int len = n[axis];
    if (len <= 1) return;
    const size_t s0 = 1, s1 = (size_t)n[0], s2 = (size_t)n[0] * n[1];
    const size_t stride = axis == 0 ? s0 : (axis == 1 ? s1 : s2);
    // enumerate the lines: the two other axes
    const int oa = axis == 0 ? 1 : 0;
    const int ob = axis == 2 ? 1 : 2;
    const size_t so[3] = {s0, s1, s2};
    const int nlines = n[oa] * n[ob];
    parallel_for(nlines, [&](int line) {
        const int ia = line % n[oa], ib = line / n[oa];
        const size_t base = ia * so[oa] + ib * so[ob];
        std::vector<cplx> buf(len);
        for (int t = 0; t < len; ++t) buf[t] = a[base + t * stride];
        fft1d(buf.data(), len, sign);
        for (int t = 0; t < len; ++t) a[base + t * stride] = buf[t];
    });
}

// Naive 3-D DFT: X[k] = sum_x f[x] exp(sign 2 pi i sum_d k_d x_d / n_d).
static void dft3d_naive(const int n[3], cplx* a, int sign) {
    const size_t N = (size_t)n[0] * n[1] * n[2];
    std::vector<cplx> in(a, a + N);
    parallel_for((int)N, [&](int kv) {
        const int k0 = kv % n[0], k1 = (kv / n[0]) % n[1], k2 = kv / (n[0] * n[1]);
        cplx s(0.0, 0.0);
        for (int z = 0; z < n[2]; ++z)
            for (int y = 0; y < n[1]; ++y)
                for (int x = 0; x < n[0]; ++x) {
                    // reduce each phase modulo its period before scaling
                    const double ph = (double)((long)k0 * x % n[0]) / n[0] +
                                      (double)((long)k1 * y % n[1]) / n[1] +
                                      (double)((long)k2 * z % n[2]) / n[2];
                    const double ang = sign * 2.0 * M_PI * ph;
                    s += in[x + (size_t)n[0] * (y + (size_t)n[1] * z)] *
                         cplx(std::cos(ang), std::sin(ang));
                }
        a[kv] = s;
    });
}

void fft3d(const int n[3], cplx* a, int sign, bool naive) {
    const size_t N = (size_t)n[0] * n[1] * n[2];
    if (naive) {
        dft3d_naive(n, a, sign);
    } else {
        for (int ax = 0; ax < 3; ++ax) transform_axis(n, a, ax, sign);
    }
    if (sign > 0) {
        const double s = 1.0 / (double)N;
        for (size_t i = 0; i < N; ++i) a[i] *= s;
    }
}

}  // namespace orc

extern "C" void orc_fft3d(const int n[3], double* data, int sign, int naive) {
    orc::fft3d(n, reinterpret_cast<orc::cplx*>(data), sign, naive != 0);
}
