// Launchers of the Fourier-space, vector and reduction kernels
// (kernels_spec.cu), instantiated for float and double bulk types.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "common.cuh"

namespace fatfft {

// Grid and half-spectrum geometry; tpl_i = 2 pi / L_i.
struct SGrid {
    int n0, n1, n2, n0h;
    size_t N, Nh;
    double tpl0, tpl1, tpl2;
};
struct Mat9 {
    double a[9];
};
// Device-resident Arnoldi position used by the look-ahead GMRES: column
// index k, norm of the last unnormalised Krylov vector, and whether the
// current column took a second Gram-Schmidt pass.
struct GmState {
    int k;
    int reorth;
    double hprev;
};
// Where a GMRES step finds its operands when they come from GmState:
// column 0 reads V (scale 1); column k > 0 reads w scaled by 1/hprev and
// stores the normalised vector as V_k.
struct GmArgs {
    const GmState* st;
    void* V;
    void* w;
    size_t vstride;
};

// Reductions write FP64 results to red.out (see Red in common.cuh).
template <typename R> void add_uniform(void* H, const void* Ht, const double* d, size_t N, cudaStream_t s);
template <typename R> void fp_sample(const void* Hpi, const int32_t* grain, const double* Qg, void* out, size_t N, cudaStream_t s);
template <typename R> void nye(void* F, const SGrid& g, double l2, cudaStream_t s);
template <typename R> void gnd_rho(const void* Lam, const int32_t* grain, const double* Qg, const double* G81, double inv_b, void* rho, size_t N, cudaStream_t s);
template <typename R> void kbar(const void* K, const void* phi, double kres, size_t N, const Red& red, cudaStream_t s);
template <typename R> void degrade(const void* P, const void* phi, double kres, void* out, size_t N, cudaStream_t s);
template <typename R> void residual(const void* Ph, const SGrid& g, void* b, const Red& red, cudaStream_t s);
template <typename R> void precond_grad(const void* vin, double scale, void* vout, const double* Kbar, const SGrid& g, void* G, int use_pre, cudaStream_t s);
template <typename R> void tangent_apply(void* G, const void* K, const void* phi, double kres, size_t N, cudaStream_t s);
template <typename R> void contract_dots(const void* T, const SGrid& g, void* w, const void* V, size_t vstride, int nv, const Red& red, cudaStream_t s, const GmState* st = nullptr);
template <typename R> void gs_update(void* w, const void* V, size_t vstride, int nv, const double* h, int dots, const SGrid& g, const Red& red, cudaStream_t s, const GmState* st = nullptr);
// tiled Krylov vector kernels: out[0] = ||w||^2, out[1 + i] = <V_i, w>; and
// w -= V h with out[0] = ||w||^2.  With need_flag the kernel runs only when
// st->reorth is set.
template <typename R> void contract(const void* T, const SGrid& g, void* w, cudaStream_t s);
template <typename R> void vdots(const void* w, const void* V, size_t vstride, int nv, const SGrid& g, const Red& red, cudaStream_t s, const GmState* st, int need_flag);
template <typename R> void vupdate(void* w, const void* V, size_t vstride, int nv, const double* hin, const SGrid& g, const Red& red, cudaStream_t s, const GmState* st, int need_flag);
template <typename R> void gm_reorth_flag(const double* red, GmState* st, cudaStream_t s);
// look-ahead GMRES helpers
template <typename R> void gm_precond_grad(const GmArgs& a, const double* Kbar, const SGrid& g, void* G, cudaStream_t s);
template <typename R> void gm_reorth(void* w, const void* V, size_t vstride, const double* red, GmState* st, const SGrid& g, const Red& red_dots, const Red& red_norm, cudaStream_t s);
void gm_reset(GmState* st, cudaStream_t s);
void gm_advance(GmState* st, const double* norm2, cudaStream_t s);
template <typename R> void norm2(const void* v, const SGrid& g, const Red& red, cudaStream_t s);
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
