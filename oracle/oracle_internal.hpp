// Internal helpers of the oracle (test infrastructure only).
#pragma once
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstdlib>
#include <functional>
#include <thread>
#include <vector>

#include "oracle.h"

namespace orc {

typedef std::complex<double> cplx;
typedef std::array<double, 9> M3;  // row-major 3x3

// ---------- threading ----------
int n_threads();
void set_threads(int n);
// Run f(i) for i in [0, n) on the configured number of std::threads.
template <class Fn>
void parallel_for(int n, Fn&& f) {
    const int nt = std::max(1, std::min(n_threads(), n));
    if (nt <= 1) {
        for (int i = 0; i < n; ++i) f(i);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(nt);
    for (int t = 0; t < nt; ++t) {
        th.emplace_back([&, t]() {
            const int lo = (int)((long)n * t / nt), hi = (int)((long)n * (t + 1) / nt);
            for (int i = lo; i < hi; ++i) f(i);
        });
    }
    for (auto& x : th) x.join();
}

// ---------- transforms ----------
void fft1d(cplx* data, int n, int sign);
void fft3d(const int n[3], cplx* a, int sign, bool naive);

// ---------- 3x3 algebra ----------
inline M3 eye3() { return M3{1, 0, 0, 0, 1, 0, 0, 0, 1}; }
inline M3 mul(const M3& a, const M3& b) {
    M3 c{};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += a[3 * i + k] * b[3 * k + j];
            c[3 * i + j] = s;
        }
    return c;
}
inline M3 tr(const M3& a) {
    M3 c{};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) c[3 * i + j] = a[3 * j + i];
    return c;
}
inline M3 add(const M3& a, const M3& b) {
    M3 c{};
    for (int i = 0; i < 9; ++i) c[i] = a[i] + b[i];
    return c;
}
inline M3 sub(const M3& a, const M3& b) {
    M3 c{};
    for (int i = 0; i < 9; ++i) c[i] = a[i] - b[i];
    return c;
}
inline M3 scale(const M3& a, double s) {
    M3 c{};
    for (int i = 0; i < 9; ++i) c[i] = a[i] * s;
    return c;
}
inline M3 sym(const M3& a) { return scale(add(a, tr(a)), 0.5); }
inline double ddot(const M3& a, const M3& b) {
    double s = 0;
    for (int i = 0; i < 9; ++i) s += a[i] * b[i];
    return s;
}
inline double det(const M3& a) {
    return a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
           a[2] * (a[3] * a[7] - a[4] * a[6]);
}
inline M3 inv(const M3& a) {
    const double d = det(a);
    M3 c{};
    c[0] = (a[4] * a[8] - a[5] * a[7]) / d;
    c[1] = (a[2] * a[7] - a[1] * a[8]) / d;
    c[2] = (a[1] * a[5] - a[2] * a[4]) / d;
    c[3] = (a[5] * a[6] - a[3] * a[8]) / d;
    c[4] = (a[0] * a[8] - a[2] * a[6]) / d;
    c[5] = (a[2] * a[3] - a[0] * a[5]) / d;
    c[6] = (a[3] * a[7] - a[4] * a[6]) / d;
    c[7] = (a[1] * a[6] - a[0] * a[7]) / d;
    c[8] = (a[0] * a[4] - a[1] * a[3]) / d;
    return c;
}
inline M3 outer(const double* u, const double* v) {
    M3 c{};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) c[3 * i + j] = u[i] * v[j];
    return c;
}
inline M3 from_ptr(const double* p) {
    M3 c{};
    for (int i = 0; i < 9; ++i) c[i] = p[i];
    return c;
}

// Solve the dense n x n system A x = b (row-major A, destroyed) by Gaussian
// elimination with partial pivoting.  Returns false if singular.
bool solve_dense(int n, double* A, double* b);

// Lattice-frame cubic stiffness applied to a symmetric strain: S = C : E.
M3 cubic_apply(const orc_material& m, const M3& E);

}  // namespace orc
