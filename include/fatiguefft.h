/*
 * fatiguefft -- GPU solver for the FFT crystal-plasticity phase-field fatigue
 * model of Lucarini, Dunne & Martinez-Paneda ("An FFT-based crystal plasticity
 * phase-field model for micromechanical fatigue cracking based on the stored
 * energy density").  One periodic voxel RVE (representative volume element)
 * per handle, solved on one GPU by the staggered load increment of
 * Algorithm 1:
 *   (a) per-voxel crystal plasticity (Sec. 2.1; history of Sec. 2.3),
 *   (b) Newton-Krylov momentum balance in Fourier space with the Green
 *       preconditioner (Eqs. momentum, fdef, newton, precf, avstiff),
 *   (c) phase-field damage solved in Fourier space (Eqs. strpf, phase,
 *       precph) with the irreversibility clamp of Algorithm 1.
 *
 * Conventions for every call:
 *  - Units MPa, mm, s (energies per volume in MPa, G_crit in N/mm).
 *  - Grid n[0] x n[1] x n[2], x fastest: voxel v = x + n0*(y + n1*z).
 *  - Voxel fields are component-major double arrays: f[c*N + v]; 3x3
 *    tensors row-major (c = 3*i + j), sample frame.
 *  - Orientation per grain: Bunge Euler (phi1, Phi, phi2) in radians,
 *    passive z-x-z; lattice-to-sample rotation Q = (Rz(phi1) Rx(Phi) Rz(phi2)).
 *  - The library owns all device memory of a handle (allocated in
 *    init_rve, released in rve_destroy).  Inputs are copied during the call;
 *    the caller keeps ownership of its buffers.
 *  - All device work runs on the stream given in fft_options.cuda_stream
 *    (0 = legacy default stream).  Calls that return statistics synchronise
 *    that stream.
 *  - Errors: every call returns an fft_status; nothing aborts.  The text of
 *    the last error of a handle is returned by fft_last_error.  On a failed
 *    increment nothing is committed; the handle still accepts fields_out,
 *    apply_increment (restarting from the committed state) and rve_destroy.
 *  - One handle must not be used from two threads at the same time.
 *  - Environment variables read at init_rve (diagnostics and measurement;
 *    the defaults are the tested configuration): FATIGUEFFT_VERBOSE (solver
 *    traces on stderr), FATIGUEFFT_GRAPHS=0 (no per-column CUDA graphs),
 *    FATIGUEFFT_DOT64=1 (FP64 per-thread sums in the Arnoldi dot pass),
 *    FATIGUEFFT_FUSED / FATIGUEFFT_BULK (the kernel-variant bits, see
 *    fft_options.kernel_variant), FATIGUEFFT_PROF_SAMPLE (see rve_profile).
 */
#ifndef FATIGUEFFT_H
#define FATIGUEFFT_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fft_rve_s* fft_rve_t;
typedef struct fft_batch_s* fft_batch_t;

typedef enum {
    FFT_OK = 0,
    FFT_ERR_ARG = -1,            /* invalid argument or size */
    FFT_ERR_OOM = -2,            /* device allocation failed */
    FFT_ERR_CUDA = -3,           /* CUDA runtime error */
    FFT_ERR_CUFFT = -4,          /* cuFFT error */
    FFT_ERR_NOT_CONVERGED = -5,  /* an iteration cap was hit (stats say which) */
    FFT_ERR_NONFINITE = -6,      /* NaN/Inf detected in a residual or norm */
    FFT_ERR_STATE = -7           /* calls made in the wrong order */
} fft_status;

typedef enum { FFT_PREC_FP64 = 0, FFT_PREC_MIXED = 1 } fft_precision;

/* Grid: voxel counts and voxel edge length h (mm); L_i = n_i h.  Each n_i in
 * [1, 4096] and 9 (n0/2 + 1) n1 n2 < 2^31 (32-bit spectral indexing; 512^3
 * fits), else FFT_ERR_ARG. */
typedef struct {
    int n[3];
    double h;
} fft_grid;

/* Material: Table 1 of the paper plus the constants it uses without a value
 * (dV activation volume, mu Taylor shear modulus, xi_store stored-energy
 * fraction, rho_ssd0 initial SSD density), G_crit, ell, ell_Fp (Sec. 4) and
 * the residual stiffness k_res of Eq. deg. */
typedef struct {
    double C11, C12, C44, tau_c0, b, nu_D, k_B, T, dF, rho_m, lambda_h, dV, mu, xi_store,
        rho_ssd0, G_crit, ell, ell_Fp, k_res;
} fft_material;

/* Solver controls.  Tolerances (Sec. 3.1-3.2): tol_stag on the Algorithm 1
 * ratios (each change of an iteration relative to the change over the
 * increment, the latter floored at 1e-12, and for the phase field at 100
 * machine epsilons of the bulk type), tol_newton on ||grad du||inf / ||F - F_t||inf, tol_lin relative
 * GMRES residual, tol_pf relative phase-field CG residual, tol_local the
 * local slip-law residual (MPa).  The Newton update is damped (an
 * extension; the paper takes full steps): from the 4th iteration, an update
 * after which the tol_newton ratio did not fall halves the next update
 * (down to 1/16), one that halved the ratio doubles it back; the ratio is
 * always that of the full correction.  max_* are iteration caps; restart is the
 * GMRES restart length (clamped to [1, 31]).  prec selects FP64 or the mixed
 * path (FP32 fields, transforms and constitutive update; FP64 reductions,
 * dot products, norms and compensated history sums).  max_cutbacks (an
 * extension; the paper's Algorithm 1 has none, 0 = off): when run_increment
 * or run_increment_mixed does not converge, the increment is restarted from
 * the committed state as two halves of the step, each committed: the first
 * to the midpoint of the committed and the requested Fbar (under mixed
 * control, with the stress-controlled components aimed at the midpoint of
 * the committed and the requested stress; the committed stress is the
 * previous increment's target on components it held by stress, its mean
 * <g P> on the others), the second to the request (under mixed control its
 * stress-controlled components of F start from the solved midpoint), dt
 * halved; recursively up to this depth (0..10, else
 * FFT_ERR_ARG at init_rve).  Smaller steps keep Newton within reach of the
 * solution and stiffen the rate-dependent consistent tangent of plastic
 * voxels, which eases the Krylov solves. */
typedef struct {
    double tol_stag, tol_newton, tol_lin, tol_pf, tol_local;
    int max_stag, max_newton, max_lin, max_pf, max_local, restart;
    fft_precision prec;
    void* cuda_stream; /* cudaStream_t */
    int max_cutbacks;
    /* Derivatives of the mechanical operators (gradient, divergence and the
     * Green preconditioner of Eq. precf): 0 = the spectral i xi of Sec. 3.1;
     * 1 = Willot's rotated finite differences, the discrete derivative the
     * paper cites against the Gibbs oscillations of the spectral one:
     * D_j = (e_j - 1)/h prod_{l != j} (1 + e_l)/2, e_l = exp(i xi_l h), in
     * place of i xi_j in the gradient, -conj(D_j) in the divergence, and the
     * Green block [conj(D) . Kbar . D]^-1 (zero where D = 0).  The Nye curl
     * and the phase-field Laplacian stay spectral.  Other values:
     * FFT_ERR_ARG at init_rve. */
    int derivative;
    /* Kernel variants of the Arnoldi step (results agree to the Krylov
     * tolerance; speed differs by grid size): bit 0 = the fused x pass (the
     * inverse real transform along x of the 9 gradient components, the
     * tangent apply and the forward real transform in one kernel, between
     * batched 2-D transforms over (z, y); used where n0 is a power of two
     * in [8, 512]), bit 1 = the register-streaming update pass instead of
     * the pipelined bulk-copy one.  0 is the default; values outside 0..3:
     * FFT_ERR_ARG.  The environment variables FATIGUEFFT_FUSED and
     * FATIGUEFFT_BULK (0 or 1) override the respective bit. */
    int kernel_variant;
} fft_options;

/* Per-increment statistics (accumulated since apply_increment). */
typedef struct {
    int stag_it, newton_it, lin_it_total, pf_it_total, local_fail;
    int converged, skipped_equilibrium;
    double res_F, res_phi; /* last Algorithm 1 ratios */
    double Pbar[9];        /* volume average of g(phi) P at the current iterate */
    long cracked;          /* voxels with phi >= 0.9 */
    int cutbacks;          /* halvings taken (max_cutbacks), either control */
    int mixed_it;          /* outer rounds of the mixed stress/strain control */
    double Fbar[9];        /* macroscopic F (row-major) after the last damage update */
} fft_stats;

/* Field identifiers for fields_out / fields_in (component count). */
enum {
    FFT_FIELD_F = 0,        /* 9  current deformation gradient F */
    FFT_FIELD_P = 1,        /* 9  degraded first Piola-Kirchhoff stress g(phi) P */
    FFT_FIELD_PHI = 2,      /* 1  current phase field */
    FFT_FIELD_FP = 3,       /* 9  committed plastic deformation gradient F_p */
    FFT_FIELD_RHO_SSD = 4,  /* 1  committed SSD density, 1/mm^2 */
    FFT_FIELD_RHO_GND = 5,  /* 1  GND density from the committed F_p */
    FFT_FIELD_WP = 6,       /* 1  committed plastic work, MPa */
    FFT_FIELD_GS = 7,       /* 1  committed stored energy density G_s, N/mm */
    FFT_FIELD_HMAX = 8,     /* 1  committed max over time of W_e+ */
    FFT_FIELD_WCRIT = 9,    /* 1  committed W_crit (0 = not yet reached) */
    FFT_FIELD_DRIVE = 10,   /* 1  crack driving state function S (Eq. zeta) */
    FFT_FIELD_GAMMA = 11,   /* 12 committed accumulated slip per system */
    FFT_FIELD_FT = 12,      /* 9  committed F */
    FFT_FIELD_PHI_T = 13,   /* 1  committed phase field */
    FFT_FIELD_WE = 14,      /* 1  W_e+ at the last constitutive evaluation */
    FFT_FIELD_K = 15,       /* 81 undegraded consistent tangent dP/dF, K[9*(3i+j)+3k+l] */
    FFT_FIELD_PU = 16       /* 9  undegraded P at the last constitutive evaluation */
};

/* Create a handle.  grain_ids: n0*n1*n2 int32 in [0, n_grains), host.
 * euler: 3*n_grains doubles, host.  phi0: optional initial (committed) phase
 * field, N doubles, host (NULL = 0).  elastic_only: optional N bytes, nonzero
 * = no slip in that voxel (the paper's soft pre-crack region), host.
 * Initial state: F = F_p = I, rho_ssd = rho_ssd0, all other history 0. */
fft_status init_rve(fft_rve_t* out, const fft_grid* grid, const int32_t* grain_ids,
                    int n_grains, const double* euler, const fft_material* mat,
                    const fft_options* opt, const double* phi0, const uint8_t* elastic_only);

/* Start a load increment (Algorithm 1 data): commits the previous increment
 * if it converged, sets F_0 = F_t + (Fbar_target - Fbar_t) uniformly,
 * phi^0 = phi_t, the step dt (s), and computes rho_GND from the committed
 * F_p (Nye tensor, Eq. nyeindexfourier, with the F_p regularisation).
 * A non-finite target component or dt, or dt < 0: FFT_ERR_ARG before
 * anything runs (the same for every call below that takes targets,
 * including the batch calls).  A non-finite value that arises in the solve
 * (from a state set with fields_in, say) stops it with FFT_ERR_NONFINITE. */
fft_status apply_increment(fft_rve_t r, const double Fbar_target[9], double dt);

/* One "solve Eq. momentum" line of Algorithm 1: Newton-Krylov at the current
 * phase field phi_{i-1}.  Skipped (F_i = F_{i-1}) when phi has not changed
 * since the previous solve of this increment.  Accumulates into st. */
/* Mixed stress/strain control (the paper's mixed-control extension of the
 * FFT solver, Sec. 3.1; the outer iteration is this library's reading):
 * mask[c] != 0 prescribes component c (row-major) of the volume-averaged
 * degraded first Piola stress, <g(phi) P>_c = Pbar[c] (MPa; Pbar may be NULL
 * for zero), and frees that component of the macroscopic F, whose value in
 * Fbar[c] is the initial guess; mask[c] == 0 prescribes Fbar[c] as in
 * apply_increment.  After each converged Newton solve the stress-controlled
 * components are corrected by Kbar_SS dF_S = -(<gP> - Pbar)_S with the
 * averaged tangent Kbar = <g K>, dF added uniformly, until
 * max_S |<gP> - Pbar| <= tol_newton * max(max_c |<gP>_c|, 1 MPa); more than
 * max_newton rounds give FFT_ERR_NOT_CONVERGED.  The solved F is reported in
 * fft_stats.Fbar and committed with the increment.  run_increment_mixed is
 * run_increment with this control (with cut-back, max_cutbacks).  For
 * uniaxial stress prefer prescribing the lateral normal stresses and the
 * off-diagonal F (no shear, no rotation): prescribed shear stresses leave the
 * rigid rotation to the weak geometric stiffness, so the stress tolerance
 * bounds it only loosely. */
fft_status apply_increment_mixed(fft_rve_t r, const double Fbar[9], const double Pbar[9],
                                 const int32_t mask[9], double dt);
fft_status run_increment_mixed(fft_rve_t r, const double Fbar[9], const double Pbar[9],
                               const int32_t mask[9], double dt, fft_stats* st);

fft_status solve_equilibrium(fft_rve_t r, fft_stats* st);

/* The "solve Eq. phase" and clamp lines of Algorithm 1 at F_i: evaluates the
 * constitutive update and driving force at F_i, solves the phase field,
 * clamps phi >= phi_t and evaluates the two convergence ratios
 * (st->converged).  Accumulates into st. */
fft_status update_damage(fft_rve_t r, fft_stats* st);

/* Accept the current (converged) iterate as the state at t + dt. */
fft_status commit_increment(fft_rve_t r);

/* apply_increment + repeated solve_equilibrium/update_damage until the
 * Algorithm 1 ratios are below tol_stag, then commit.  Resets st. */
fft_status run_increment(fft_rve_t r, const double Fbar_target[9], double dt, fft_stats* st);

/* Copy a field (double, component-major, sample frame) to dst: a host
 * pointer (dst_is_device = 0) or a device pointer on the handle's GPU
 * (dst_is_device = 1).  bytes must be at least ncomp*N*8. */
fft_status fields_out(fft_rve_t r, int field, void* dst, size_t bytes, int dst_is_device);

/* Overwrite a state field from a host double array (F, FT, FP, PHI, PHI_T,
 * RHO_SSD, WP, GS, HMAX, WCRIT, GAMMA, DRIVE).  For testing and restarts;
 * history sums restart with a zero compensation term. */
fft_status fields_in(fft_rve_t r, int field, const double* src, size_t bytes);

/* Checkpoint of the committed state (not in the paper; the state Algorithm 1
 * carries from one increment to the next): F_t, F_p (lattice-frame inverse),
 * phi_t and the FP64 history with its compensation terms, in the handle's
 * precision, plus the committed macroscopic F.  Grain ids, orientations,
 * material and options are not included: a checkpoint is loaded into a
 * handle created with the same ones.
 * state_save: dst == NULL sets *bytes to the size needed; otherwise *bytes
 * is the capacity of dst (host memory, caller-owned), the checkpoint is
 * written, *bytes set to its size and the stream synchronised.  A converged
 * but uncommitted increment of the stage calls is not included.
 * FFT_ERR_ARG: NULL handle or bytes, or capacity too small.
 * state_load: restores a checkpoint of a handle with the same grid,
 * precision, grain ids, orientations, soft-region mask and material (the
 * checkpoint carries a hash of these; else FFT_ERR_ARG) as the committed
 * state and the current iterate; the next increment then reproduces, bit for bit, the run the
 * checkpoint was taken from.  Any earlier failed or uncommitted increment is
 * discarded. */
fft_status state_save(fft_rve_t r, void* dst, size_t* bytes);
fft_status state_load(fft_rve_t r, const void* src, size_t bytes);

/* Stage entry points (same kernels as the increment uses), for checking one
 * stage at a time.  eval_constitutive: constitutive update at the current F
 * with the committed history; with_history = 1 also evaluates W_e+, the
 * driving force and the trial history.  eval_gnd: rho_GND from the committed
 * F_p.  solve_phase_field: the phase-field solve and clamp with the driving
 * force of the last eval_constitutive(with_history = 1). */
fft_status eval_constitutive(fft_rve_t r, double dt, int with_history, int* local_fail);
fft_status eval_gnd(fft_rve_t r);
fft_status solve_phase_field(fft_rve_t r, int* iters);

/* Opt-in kernel timing.  mask selects kernel families by bit (0 constitutive,
 * 1 tangent apply, 2 preconditioner + gradient, 3 divergence, 4 GMRES dot
 * products, 5 Gram-Schmidt update, 6 GMRES solution update, 7 averaged
 * tangent, 8 residual, 9 F update, 10 phase field, 11 GND, 12 cuFFT
 * 9-field transforms, 13 cuFFT scalar transforms, 14 reductions, 15 other);
 * each selected launch is bracketed by CUDA events on the handle's stream.
 * GMRES steps replayed from CUDA graphs (handles with a stream) are timed
 * on every S-th replay only (S from the environment variable
 * FATIGUEFFT_PROF_SAMPLE at init_rve, default 8), the others replaying a
 * graph without event nodes; counts report the timed launches.
 * 0 switches timing off.  rve_profile_read returns the accumulated device
 * milliseconds, launch counts and algorithmic bytes (the minimum HBM traffic
 * of the timed launches; bytes may be NULL) per family (16 entries each,
 * caller-owned arrays), synchronising the stream first; reset = 1 clears
 * them. */
fft_status rve_profile(fft_rve_t r, unsigned mask);
fft_status rve_profile_read(fft_rve_t r, double* ms, long long* counts, double* bytes,
                            int reset);

/* Allocation-free reduction, for callers that may not call cudaMalloc (a
 * host framework that owns all device memory, a pre-sized pool, or code
 * that must not allocate or synchronise once a run has started).  The
 * paper has no counterpart: this is a standalone copy of the library's
 * degraded volume average, out[c] = (1/N) sum_v ((1 - phi_v)^2 + k_res)
 * X[c*N + v] for c < ncomp, the reduction behind the averaged tangent and
 * the reported mean stress.
 *   X: device, ncomp*N doubles, component-major; phi: device, N doubles;
 *   out: device, ncomp doubles (written); cuda_stream: cudaStream_t (0 =
 *   legacy default stream).  The call only enqueues work on that stream.
 * It allocates nothing: the per-block partial sums go to one fixed array of
 * device memory inside the library (kept by every GPU that loads it until
 * the process exits), sized for ncomp <= 81; a larger ncomp, N = 0 or a null
 * pointer returns FFT_ERR_ARG without launching anything.  The first call on
 * each device (with that device current) looks up the array's device
 * address, so make that first call before any stream capture.  The address
 * is kept until the process exits: do not call this function again on a
 * device after resetting it (cudaDeviceReset or a re-created primary
 * context), since the array then lives elsewhere.  All calls on
 * a device share the array: calls whose work overlaps on the GPU (other
 * streams, other threads) race and must be serialised by the caller.  Each
 * call overwrites every partial it later reads, so no clearing is needed. */
fft_status degraded_average_noalloc(const double* X, int ncomp, const double* phi, size_t N,
                                    double k_res, double* out, void* cuda_stream);

/* Size in bytes of the device memory the handle holds. */
size_t rve_device_bytes(fft_rve_t r);
/* Release the handle and its device memory.  A handle still in a batch is
 * left alive (its last error says so): destroy the batch first. */
void rve_destroy(fft_rve_t r);
const char* fft_last_error(fft_rve_t r);

/* Batched RVEs (many independent problems of uneven size, one GPU; the
 * paper solves one RVE at a time).  batch_create groups n existing handles,
 * which must be distinct, each created with its own non-default
 * cuda_stream and in no other batch that has not been destroyed
 * (FFT_ERR_ARG otherwise, with nothing changed); the caller keeps ownership of the
 * handles and must not use them from other threads while the batch runs.
 * n_threads host threads (<= 0: the hardware concurrency; at most n) drive
 * the handles' increments concurrently, largest grid first.  While grouped,
 * a handle's host waits poll its stream and yield the core between polls
 * (instead of spinning), so that more threads than host cores can drive
 * handles; batch_destroy restores the spinning waits.
 * batch_run_increment = run_increment on every handle: Fbar 9n doubles
 * (row-major per handle), dt n doubles, stats n entries (may be NULL),
 * status n ints (may be NULL) receive each handle's own result; returns
 * FFT_OK or the first failing handle's status (the others still ran).
 * A failed handle behaves as after its own failed run_increment.  Calls on
 * one batch from several host threads are serialised (each waits for the
 * previous one to finish).
 * batch_run_increment_mixed = run_increment_mixed on every handle, with the
 * same layouts plus Pbar 9n doubles (may be NULL: zero targets) and mask 9n
 * int32 (per handle as in run_increment_mixed; NULL: FFT_ERR_ARG).
 *
 * Lockstep classes: batch_create groups the handles of one size class (same
 * device, precision, grid and fft_options; the unfused Arnoldi step, CUDA
 * graphs on; by default grids of at most 2^16 voxels, e.g. 40^3, where a
 * GMRES step is latency-bound) into classes of up to 64 members.  A class's
 * increments (batch_run_increment, batch_run_increment_mixed) run together:
 * the Newton, mixed-control and GMRES iterations in lockstep over the
 * members still iterating, each Krylov column of the whole class one CUDA
 * graph launch with one batched library transform per direction over the
 * class's 9 x members fields; the damage updates and the cut-backs of a
 * member whose increment did not converge run per member.  Each member's
 * arithmetic is that of its own run_increment(_mixed).
 * The class holds the members' Arnoldi-step scratch and reduction buffers
 * in arenas while the batch exists (18 real-field components per voxel, in
 * the handle's precision, plus 2 KB per member; the members' own buffers
 * stay allocated and are used again after batch_destroy).  The handles stay
 * usable on their own, from the thread that owns the batch, between batch
 * calls; destroy the batch before any of its handles.  batch_create_ex flags: bit 0 = classes
 * of grids up to 2^16 voxels, bit 1 = classes at any grid size, 0 = no
 * classes (other bits: FFT_ERR_ARG); batch_create = batch_create_ex with
 * flags 1.  batch_classes returns the number of classes and, per class,
 * its member count, the column graphs launched so far and, while timing is
 * on, the device milliseconds of those launches (CUDA events on the class's
 * stream) and their algorithmic bytes (the two 9-field transforms, tangent
 * apply, contraction with the dot pass and update of every member); timing
 * = 1 or 0 switches the timing on or off and zeroes the sums after reading
 * them, -1 leaves both (every array may be NULL; room for batch_size
 * entries suffices). */
fft_status batch_create(fft_batch_t* out, fft_rve_t const* rves, int n, int n_threads);
fft_status batch_create_ex(fft_batch_t* out, fft_rve_t const* rves, int n, int n_threads,
                           int flags);
int batch_classes(fft_batch_t b, int timing, int* sizes, long long* graph_launches,
                  double* graph_ms, double* graph_bytes);
fft_status batch_run_increment(fft_batch_t b, const double* Fbar, const double* dt,
                               fft_stats* stats, int* status);
fft_status batch_run_increment_mixed(fft_batch_t b, const double* Fbar, const double* Pbar,
                                     const int32_t* mask, const double* dt, fft_stats* stats,
                                     int* status);
int batch_size(fft_batch_t b);
void batch_destroy(fft_batch_t b);
/* Kernel launches issued by this handle since creation (for accounting). */
long long rve_kernel_launches(fft_rve_t r);

/* Library self-test (no counterpart in the paper): the bounded mbarrier
 * wait that guards the pipelined Krylov update pass, run on a barrier that
 * nothing completes with a limit of `rounds` try-wait rounds (1..65536).
 * Returns 1 when the wait gave up as it must (the kernel then records an
 * error instead of spinning), 2 if it wrongly reported completion, -1 on a
 * CUDA error, -2 for a bad argument.  Uses the current device and stream 0;
 * allocates one int. */
int fft_selftest_bounded_wait(unsigned rounds);

#ifdef __cplusplus
}
#endif
#endif
