// Host-side launchers of the fatiguefft kernels (one translation unit per
// kernel family; templates instantiated for float and double bulk types).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace fatfft {

// Constitutive parameters in the units of the library (MPa, mm, s).
struct CPParams {
    double C11, C12, C44;
    double tau_c0, mu_b;    // mu * b
    double g0, sT;          // rate prefactor (1/s) and thermal stress kT/dV (MPa)
    double lambda_h, xi_store, G_crit, inv_b;
    double dt;
    double tol_local;
    int max_local;
};

// Device pointers used by the constitutive kernel.  R-typed fields are passed
// as void* and cast inside the kernel of the matching precision.
struct CPFields {
    const void* H;        // R[9][N]  F - I (sample)
    const void* Hpi;      // R[9][N]  committed Fp^-1 - I (lattice)
    const void* rho_gnd;  // R[N]
    const int32_t* grain; // [N]
    const uint8_t* elastic;  // [N] or null
    const double* Qg;     // [9 * n_grains] lattice -> sample rotations
    const double* hist_c; // [32][N] committed history
    double* hist_tr;      // [32][N] trial history (written with history)
    void* P;              // R[9][N]  undegraded P (sample)
    void* K;              // R[81][N] undegraded tangent (sample) or null
    void* Hpi_tr;         // R[9][N]  trial Fp^-1 - I (with history)
    void* drive;          // R[N]     crack driving state function (with history)
    void* We;             // R[N]     W_e+ (with history)
    int* fail_count;      // local-solve failures (atomic)
    size_t N;
};

// history slots (double, slot-major)
enum {
    HIST_RHO = 0,    // (sum, comp)
    HIST_WP = 2,     // (sum, comp)
    HIST_GS = 4,     // (sum, comp)
    HIST_HMAX = 6,
    HIST_WCRIT = 7,
    HIST_GAMMA = 8,  // 12 x (sum, comp)
    HIST_SLOTS = 32
};

void upload_slip_table(cudaStream_t s);
template <typename R>
void launch_constitutive(const CPFields& f, const CPParams& p, bool hist, cudaStream_t s);

}  // namespace fatfft
