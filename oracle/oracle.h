/*
 * Oracle for the FFT crystal-plasticity phase-field fatigue solver
 * (Lucarini, Dunne & Martinez-Paneda, "An FFT-based crystal plasticity
 * phase-field model for micromechanical fatigue cracking based on the stored
 * energy density").
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, FP64 CPU restatement of
 * the paper's equations, written to check the GPU library against.  Only the
 * test-suite, the package smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or helper with the
 * GPU library: its own FFT (mixed radix 2/3 with a generic-prime fallback,
 * plus a naive O(N^2) DFT), its own slip-system tables and its own solvers.
 *
 * Conventions (each is a reading of the paper, recorded with the design):
 *  - Units: MPa, mm, s; energies per volume in MPa; G_s and G_crit in N/mm.
 *  - Grid n[0] x n[1] x n[2] voxels, x fastest: v = x + n0*(y + n1*z).
 *  - Voxel fields are component-major: f[c*N + v].  3x3 tensors are row-major
 *    (c = 3*i + j).  Tensors given to / returned by the API are in the sample
 *    frame unless the name ends in _L (lattice frame).
 *  - Orientation: Bunge (phi1, Phi, phi2), passive; the matrix Q maps lattice
 *    to sample coordinates (sample = Q * lattice).
 *  - Forward FFT unnormalised, inverse scaled by 1/N.
 *
 * Parity status per function is listed in the test-suite; the full coupled
 * polycrystal trajectory against the paper's reported cycle counts is
 * "parity unpinned" (the paper's microstructures and several constants are not
 * given).
 */
#ifndef FATIGUE_ORACLE_H
#define FATIGUE_ORACLE_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Material data: Table 1 of the paper plus the constants the paper uses but
 * does not list (dV, mu, xi_store, rho_ssd0), Sec. 2.1-2.3 and Sec. 4. */
typedef struct {
    double C11, C12, C44;   /* cubic elastic constants, MPa */
    double tau_c0;          /* initial CRSS, MPa */
    double b;               /* Burgers vector, mm */
    double nu_D;            /* attempt frequency, 1/s */
    double k_B;             /* Boltzmann constant, J/K */
    double T;               /* temperature, K */
    double dF;              /* activation energy, J */
    double rho_m;           /* mobile dislocation density, 1/mm^2 */
    double lambda_h;        /* SSD hardening coefficient, 1/mm^2 */
    double dV;              /* activation volume, mm^3 */
    double mu;              /* shear modulus in the Taylor term, MPa */
    double xi_store;        /* stored-energy fraction (dimensionless) */
    double rho_ssd0;        /* initial SSD density, 1/mm^2 */
    double G_crit;          /* critical stored energy density, N/mm */
    double ell;             /* phase-field length scale, mm */
    double ell_Fp;          /* F_p regularisation length, mm */
    double k_res;           /* residual stiffness in g(phi) */
} orc_material;

typedef struct {
    double tol_stag, tol_newton, tol_lin, tol_pf, tol_local;
    int max_stag, max_newton, max_lin, max_pf, max_local;
    int restart;            /* GMRES restart length */
    int use_naive_dft;      /* 1: every transform is the O(N^2) DFT */
    int n_threads;          /* 0: hardware concurrency */
    int max_cutbacks;       /* 0: off; else a non-converged increment is redone as two
                               halves from the committed state, down to this depth */
    int derivative;         /* mechanical derivatives: 0 spectral (i xi, Sec. 3.1),
                               1 Willot's rotated finite differences */
} orc_options;

typedef struct {
    int stag_it, newton_it, lin_it_total, pf_it_total, local_fail;
    int converged, skipped_equilibrium;
    double res_F, res_phi;
    double Pbar[9];
    long cracked;
    int mixed_it;     /* outer rounds of the mixed stress/strain control */
    double Fbar[9];   /* macroscopic F at the end of the last damage update */
    int cutbacks;     /* halvings taken (max_cutbacks) */
} orc_stats;

/* Per-voxel constitutive result (Sec. 2.1, 2.3). */
typedef struct {
    double P[9];        /* undegraded first Piola-Kirchhoff stress, sample */
    double K[81];       /* undegraded dP/dF, sample, K[9*(3i+j) + 3k+l] */
    double S_L[6];      /* 2nd PK stress in the lattice frame (11,22,33,23,13,12) */
    double Fp_L[9];     /* updated plastic deformation gradient, lattice */
    double dgamma[12];  /* slip increments */
    double tau[12];     /* resolved shear stresses */
    double tau_c;       /* CRSS used */
    double dWp;         /* plastic work increment sum tau*dgamma, MPa */
    double drho_ssd;    /* SSD increment, 1/mm^2 */
    double We_plus;     /* tensile elastic energy 1/2 eps+ : C : eps+, MPa */
    int iters;          /* local Newton iterations */
    int fail;           /* 1 if the local Newton did not converge */
} orc_cp_result;

/* ---------------- transforms ---------------- */
/* In-place 3-D complex transform of data[2*v] (re), data[2*v+1] (im).
 * sign = -1 forward (unnormalised), +1 inverse (scaled by 1/N). */
void orc_fft3d(const int n[3], double* data, int sign, int naive);

/* ---------------- tables and point functions ---------------- */
void orc_material_paper(orc_material* m);   /* Table 1 as printed + readings */
void orc_euler_to_Q(const double euler[3], double Q[9]);
/* FCC {111}<110>: unit slip directions s[12][3] and plane normals n[12][3]. */
void orc_fcc_systems(double s[36], double n[36]);
/* 9x18 GND basis (12 edge b(x)t, 6 screw b(x)b, unit dyads, row-major 9x18)
 * and its Moore-Penrose pseudo-inverse (18x9). */
void orc_gnd_basis(double A[162], double Apinv[162]);

int orc_cp_point(const orc_material* m, const double Q[9], const double F[9],
                 const double Fp_L[9], double rho_ssd_n, double rho_gnd,
                 double dt, int elastic_only, double tol_local, int max_local,
                 int want_tangent, orc_cp_result* out);

/* Tensile elastic energy of a lattice-frame elastic deformation gradient. */
double orc_we_plus(const orc_material* m, const double Fe_L[9]);
/* Symmetric 3x3 eigen-decomposition by cyclic Jacobi: A = V diag(w) V^T,
 * eigenvectors in the columns of V. */
void orc_sym_eig3(const double A[9], double w[3], double V[9]);

/* Green-operator preconditioner of Eq. precf at one frequency:
 * out = [xi . Kbar . xi]^-1 in (3x3) or 0 where xi = 0. */
void orc_green_precond(const double Kbar[81], const double xi[3], double Minv[9]);

/* ---------------- field-level stages ---------------- */
/* Nye tensor and GND density over the whole domain (Eq. nyeindexfourier,
 * F_p regularisation, Eq. nye1 min-norm split).  Fp: sample-frame F_p (9*N);
 * outputs Lambda (9*N, sample) and rho_gnd (N). */
void orc_gnd_field(const int n[3], double h, const orc_material* m,
                   const double* Q_per_voxel, const double* Fp, int naive,
                   double* Lambda, double* rho_gnd);

/* Phase-field solve (Eq. phase) with the Krylov solver and the M_phi
 * preconditioner; x0 and clamp as in Algorithm 1. */
int orc_phase_field(const int n[3], double h, double ell, const double* S,
                    const double* phi_prev, const double* phi_t, double tol,
                    int max_it, int naive, double* phi_out, int* iters);

/* ---------------- RVE solver (Algorithm 1) ---------------- */
typedef struct orc_rve orc_rve;

orc_rve* orc_rve_create(const int n[3], double h, const int32_t* grain_ids,
                        int n_grains, const double* euler,
                        const orc_material* m, const orc_options* o,
                        const double* phi0, const uint8_t* elastic_only);
void orc_rve_destroy(orc_rve* r);
int orc_apply_increment(orc_rve* r, const double Fbar[9], double dt);
int orc_solve_equilibrium(orc_rve* r, orc_stats* st);
int orc_update_damage(orc_rve* r, orc_stats* st);
int orc_commit(orc_rve* r);
int orc_run_increment(orc_rve* r, const double Fbar[9], double dt, orc_stats* st);
/* Mixed stress/strain control (the paper's mixed-control extension, Sec. 3.1;
 * reading: an outer Newton on the stress-controlled macroscopic components):
 * mask[c] = 1 makes component c of Pbar prescribed (Pstar[c]) and that
 * component of Fbar free (Fbar[c] is its initial value); mask[c] = 0
 * prescribes Fbar[c] as in orc_apply_increment.  After each converged
 * Newton solve, Kbar_SS dF_S = -(<gP> - Pstar)_S with Kbar = <g K> is solved
 * and dF added uniformly, until max_S |<gP> - Pstar| <= tol_newton *
 * max(max|<gP>|, 1 MPa) (at most max_newton rounds). */
int orc_apply_increment_mixed(orc_rve* r, const double Fbar[9], const double Pstar[9],
                              const int mask[9], double dt);
int orc_run_increment_mixed(orc_rve* r, const double Fbar[9], const double Pstar[9],
                            const int mask[9], double dt, orc_stats* st);

/* field ids shared in meaning (not in code) with the GPU library */
enum {
    ORC_FIELD_F = 0,        /* 9: current F (sample) */
    ORC_FIELD_P = 1,        /* 9: degraded P at the current iterate g(phi)P */
    ORC_FIELD_PHI = 2,      /* 1: current phase field */
    ORC_FIELD_FP = 3,       /* 9: committed F_p, sample frame */
    ORC_FIELD_RHO_SSD = 4,  /* 1: committed */
    ORC_FIELD_RHO_GND = 5,  /* 1: from the committed F_p */
    ORC_FIELD_WP = 6,       /* 1: committed plastic work */
    ORC_FIELD_GS = 7,       /* 1: committed stored energy density */
    ORC_FIELD_HMAX = 8,     /* 1: committed max W_e+ */
    ORC_FIELD_WCRIT = 9,    /* 1: committed W_crit (0 = unset) */
    ORC_FIELD_DRIVE = 10,   /* 1: crack driving state function S */
    ORC_FIELD_GAMMA = 11,   /* 12: committed accumulated slip per system */
    ORC_FIELD_FT = 12,      /* 9: committed F */
    ORC_FIELD_PHI_T = 13,   /* 1: committed phase field */
    ORC_FIELD_WE = 14       /* 1: W_e+ at the last constitutive evaluation */
};
int orc_fields_out(const orc_rve* r, int field, double* dst);
int orc_fields_in(orc_rve* r, int field, const double* src);

#ifdef __cplusplus
}
#endif
#endif
