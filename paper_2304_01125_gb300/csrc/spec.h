// Launchers of the Fourier-space, vector and reduction kernels
// (kernels_spec.cu), instantiated for float and double bulk types.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "common.cuh"
#include "fastdiv.h"

namespace fatfft {

// Grid and half-spectrum geometry; tpl_i = 2 pi / L_i (FP64 and FP32); dividers for the
// index decode of half-spectrum entries.
struct SGrid {
    int n0, n1, n2, n0h;
    size_t N, Nh;
    double tpl0, tpl1, tpl2;
    float tpl0f, tpl1f, tpl2f;  // the same in FP32 (the FP64 pipe is narrow on this GPU)
    FastDiv fd_n0h, fd_n1, fd_Nh;
    // derivatives of the mechanical operators: 0 = spectral i xi (Sec. 3.1),
    // 1 = Willot's rotated finite differences (the discrete alternative the
    // paper cites against Gibbs oscillations); 1/h in FP64 and FP32
    int willot;
    double ih;
    float ihf;
};
struct Mat9 {
    double a[9];
};
// Reductions write FP64 results to red.out (see Red in common.cuh).
template <typename R> void add_uniform(void* H, const void* Ht, const double* d, size_t N, cudaStream_t s);
template <typename R> void fp_sample(const void* Hpi, const int32_t* grain, const double* Qg, void* out, size_t N, cudaStream_t s);
template <typename R> void nye(void* F, const SGrid& g, double l2, cudaStream_t s);
template <typename R> void gnd_rho(const void* Lam, const int32_t* grain, const double* Qg, const double* G81, double inv_b, void* rho, size_t N, cudaStream_t s);
template <typename R> void kbar(const void* K, const void* phi, double kres, size_t N, const Red& red, cudaStream_t s);
template <typename R> void degrade(const void* P, const void* phi, double kres, void* out, size_t N, cudaStream_t s);
template <typename R> void residual(const void* Ph, const SGrid& g, void* b, const Red& red, cudaStream_t s);
// il = 1 writes G in the interleaved layout of the fused x pass
template <typename R> void precond_grad(const void* vin, double scale, void* vout, const double* Kbar, const SGrid& g, void* G, int use_pre, cudaStream_t s, int il = 0);
// act (nullable): a device flag; 0 makes the Arnoldi step kernels below return
// at once (a lockstep class member that has left the iteration)
template <typename R> void tangent_apply(void* G, const void* K, const void* phi, double kres, size_t N, cudaStream_t s, const int* act = nullptr);
template <typename R> void contract(const void* T, const SGrid& g, void* w, cudaStream_t s);
// Arnoldi step kernels (DCGS2, see kernels_spec.cu).  Hessenberg columns on
// the device are kHcol doubles apart; the host slot holds the final column
// k-1 at 0, the provisional column k at kSlotProv, nu_k at kSlotNu,
// |c_{k+1}|^2 at kSlotNorm, alpha = |c_k|^2 and |a|^2 (kSlotAlpha,
// kSlotA2) for the solver trace, and the pipelined kernels' error word at
// kSlotErr.
constexpr int kHcol = kMaxKrylov + 1;
constexpr int kSlotProv = 40, kSlotNorm = 80, kSlotNu = 81, kSlotAlpha = 82, kSlotA2 = 83,
              kSlotErr = 84, kSlotLen = 85;
// Resident-CTA budget of the pipelined (bulk-copy) update pass and the
// device error word of its bounded waits; the launchers below take them
// when given (NULL: the register-streaming kernels; the dot pass always
// streams through registers and only reports the error word).
// dcgs_bulk_setup returns 0 if the pipelined kernel cannot be used.
struct BulkCfg {
    int upd_blocks;
    int* err;
};
template <typename R> int dcgs_bulk_setup(BulkCfg& bc);
// one warp's bounded wait on a barrier nothing completes: 1 = gave up, 2 = reported done
int selftest_bounded_wait(unsigned limit);
// the contraction fused with the dot pass: w = -div T stored; alpha, beta,
// |z|^2, a, b reduced and the step coefficients formed (kernels_spec.cu)
// il = 1: T (and, for the update, G) in the interleaved layout of the
// fused x pass
// dot64 = 1: per-thread products and partial sums in FP64 (default: the
// bulk type, FP64 from the block combine on)
template <typename R> void contract_dots(const void* T, const SGrid& g, void* w, const void* c, const void* V, size_t vstride, int k, const Red& red, double* Hd, double* Hp, double* slot, double* coef, const BulkCfg* bc, cudaStream_t s, int il = 0, int dot64 = 0, const int* act = nullptr);
template <typename R> void dcgs_update(void* V, size_t vstride, int k, const void* z, const double* coef, const double* Kbar, const SGrid& g, void* G, const Red& red, const BulkCfg* bc, cudaStream_t s, int il = 0, const int* act = nullptr);
template <typename R> void norm2(const void* v, const SGrid& g, const Red& red, cudaStream_t s);

// Fused x pass of the Arnoldi step (kernels_fft.cu): inverse real
// transform along x of the 9 gradient components, tangent apply and forward
// real transform, per block of rows of the interleaved spectrum layout
// ((9 r + c) n0h + kx for row r = y + n1 z, field c); the transforms along
// y and z are a batched 2-D library transform over that layout.
constexpr int kFftMaxLen = 512;  // longest x line of the fused pass
struct FusedX {
    int ok;          // the grid is supported (else the library 3-D transforms are used)
    int rb, lpw;     // rows per block, (row, field) lines per warp
    size_t smem;     // dynamic shared memory per block
    const void* tw;  // device twiddle table exp(-2 pi i t / n0), t < n0
};
template <typename R> int fused_x_plan(FusedX& p, const SGrid& g);
template <typename R> void fused_x_twiddles(int n, void* host);
template <typename R> void fused_xpass(const FusedX& p, void* G, const void* K, const void* phi, double kres, const SGrid& g, cudaStream_t s);
template <typename R> void xupdate(void* x, const void* V, size_t vstride, int k, const double* y, const double* Kbar, const SGrid& g, cudaStream_t s);
template <typename R> void axpby(void* out, const void* a, const void* b, double alpha, double beta, size_t n, cudaStream_t s);
template <typename R> void fupdate(void* H, const void* G, const void* Ht, size_t N, const Red& red, cudaStream_t s);
template <typename R> void stag_stats(const void* H, const void* Hprev, const void* Ht, const void* P, const void* phi, double kres, size_t N, const Red& red, cudaStream_t s);
template <typename R> void maxval(const void* a, size_t n, const Red& red, cudaStream_t s);
template <typename R> void pf_spec(void* f, const SGrid& g, double l2, int mode, cudaStream_t s);
template <typename R> void pf_init(const void* x, const void* lapx, const void* S, void* r, size_t N, const Red& red, cudaStream_t s);
template <typename R> void rdot(const void* a, const void* b, size_t N, const Red& red, cudaStream_t s);
template <typename R> void pf_q(const void* t, const void* p, const void* S, void* q, size_t N, const Red& red, cudaStream_t s);
template <typename R> void pf_xr(void* x, void* r, const void* p, const void* q, double alpha, size_t N, const Red& red, cudaStream_t s);
template <typename R> void pf_pt(void* p, void* t, const void* z, const void* r, double beta, size_t N, cudaStream_t s);
template <typename R> void pf_clamp(const void* x, const void* phi_t, void* phi, size_t N, const Red& red, cudaStream_t s);
template <typename R> void to_double(const void* src, double* dst, size_t n, size_t N, int add_eye, cudaStream_t s);
template <typename R> void from_double(const double* src, void* dst, size_t n, size_t N, int sub_eye, cudaStream_t s);
template <typename R> void fp_in(const double* Fp, const int32_t* grain, const double* Qg, void* Hpi, size_t N, cudaStream_t s);
void hist_sum(const double* hist, int slot, int comp, int count, double* dst, size_t N, cudaStream_t s);
void hist_set(double* hist, int slot, int comp, int count, const double* src, size_t N, cudaStream_t s);

}  // namespace fatfft
