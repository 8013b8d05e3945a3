// Host driver and C ABI of the fatiguefft library: the load increment of
// Algorithm 1 (staggered alternating minimisation), the Newton-Krylov
// momentum solve (Eqs. momentum, fdef, newton with the Green preconditioner
// of Eqs. precf, avstiff) and the phase-field solve (Eqs. phase, precph),
// all on one CUDA stream.  Only convergence decisions cross to the host.
#include <mutex>

#include "rve_impl.cuh"

// ------------------------------------------------------- host-side tables
// Lattice-to-sample rotation from Bunge angles: Q = Rz(phi1) Rx(Phi) Rz(phi2).
static void bunge_Q(const double* e, double* Q) {
    auto rz = [](double a, double* m) {
        const double c = std::cos(a), s = std::sin(a);
        const double t[9] = {c, -s, 0, s, c, 0, 0, 0, 1};
        std::memcpy(m, t, sizeof(t));
    };
    double A[9], B[9], C[9], T[9];
    rz(e[0], A);
    const double c = std::cos(e[1]), s = std::sin(e[1]);
    const double X[9] = {1, 0, 0, 0, c, -s, 0, s, c};
    std::memcpy(B, X, sizeof(X));
    rz(e[2], C);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            T[3 * i + j] = 0;
            for (int k = 0; k < 3; ++k) T[3 * i + j] += A[3 * i + k] * B[3 * k + j];
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            Q[3 * i + j] = 0;
            for (int k = 0; k < 3; ++k) Q[3 * i + j] += T[3 * i + k] * C[3 * k + j];
        }
}

// (A A^T)^-1 for the GND dyad basis of Eq. nye1 (12 edge b(x)t, t = n x b;
// the distinct screw b(x)b), assembled from the slip table.
static void gnd_metric(double* G) {
    const int pl[4][3] = {{1, 1, 1}, {-1, 1, 1}, {1, -1, 1}, {1, 1, -1}};
    const int dr[12][3] = {{0, 1, -1}, {1, 0, -1}, {1, -1, 0}, {0, 1, -1}, {1, 0, 1}, {1, 1, 0},
                           {0, 1, 1},  {1, 0, -1}, {1, 1, 0},  {0, 1, 1},  {1, 0, 1}, {1, -1, 0}};
    std::vector<std::vector<double>> cols;
    std::vector<std::vector<int>> screws;
    for (int a = 0; a < 12; ++a) {
        double b[3], n[3], t[3];
        for (int i = 0; i < 3; ++i) {
            b[i] = dr[a][i] / std::sqrt(2.0);
            n[i] = pl[a / 3][i] / std::sqrt(3.0);
        }
        t[0] = n[1] * b[2] - n[2] * b[1];
        t[1] = n[2] * b[0] - n[0] * b[2];
        t[2] = n[0] * b[1] - n[1] * b[0];
        std::vector<double> c(9);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) c[3 * i + j] = b[i] * t[j];
        cols.push_back(c);
        // screw directions, distinct up to sign
        std::vector<int> d = {dr[a][0], dr[a][1], dr[a][2]};
        std::vector<int> m = {-d[0], -d[1], -d[2]};
        bool seen = false;
        for (auto& q : screws) seen = seen || q == d || q == m;
        if (!seen) screws.push_back(d);
    }
    for (auto& d : screws) {
        std::vector<double> c(9);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) c[3 * i + j] = d[i] * d[j] / 2.0;
        cols.push_back(c);
    }
    double M[81], I[81];
    for (int r = 0; r < 9; ++r)
        for (int c = 0; c < 9; ++c) {
            double s = 0;
            for (auto& col : cols) s += col[r] * col[c];
            M[9 * r + c] = s;
            I[9 * r + c] = r == c ? 1.0 : 0.0;
        }
    // Gauss-Jordan inverse with partial pivoting
    for (int c = 0; c < 9; ++c) {
        int p = c;
        for (int r = c + 1; r < 9; ++r)
            if (std::fabs(M[9 * r + c]) > std::fabs(M[9 * p + c])) p = r;
        for (int k = 0; k < 9; ++k) {
            std::swap(M[9 * c + k], M[9 * p + k]);
            std::swap(I[9 * c + k], I[9 * p + k]);
        }
        const double d = M[9 * c + c];
        for (int k = 0; k < 9; ++k) {
            M[9 * c + k] /= d;
            I[9 * c + k] /= d;
        }
        for (int r = 0; r < 9; ++r) {
            if (r == c) continue;
            const double f = M[9 * r + c];
            for (int k = 0; k < 9; ++k) {
                M[9 * r + k] -= f * M[9 * c + k];
                I[9 * r + k] -= f * I[9 * c + k];
            }
        }
    }
    std::memcpy(G, I, sizeof(I));
}


// ------------------------------------------------------------------ C ABI
#define DISPATCH(r, call) ((r)->prec == FFT_PREC_FP64 ? Impl<double>::call : Impl<float>::call)

static void release(fft_rve_s* r) {
    for (auto& p : r->prof_pending)
        if (!p.owned) {
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
        }
    r->prof_pending.clear();
    for (auto e : r->prof_pool) cudaEventDestroy(e);
    r->prof_pool.clear();
    drop_graphs(r);
    if (r->yz_plan) cufftDestroy(r->yz);
    if (r->plans) {
        cufftDestroy(r->r2c9);
        cufftDestroy(r->c2r9);
        cufftDestroy(r->r2c1);
        cufftDestroy(r->c2r1);
    }
    for (void* p : r->allocs) cudaFree(p);
    if (r->stage) cudaFree(r->stage);
    if (r->hred) cudaFreeHost(r->hred);
    if (r->hy) cudaFreeHost(r->hy);
    if (r->hslot) cudaFreeHost(r->hslot);
    for (auto e : r->slot_ev)
        if (e) cudaEventDestroy(e);
    if (r->sync_ev) cudaEventDestroy(r->sync_ev);
}

// Staging buffer for host-side field copies, grown on demand (field copies
// are not on the increment's path).
static fft_status ensure_stage(fft_rve_s* r, size_t bytes) {
    if (r->stage_bytes >= bytes) return FFT_OK;
    if (r->stage) {
        cudaStreamSynchronize(r->st);
        cudaFree(r->stage);
        r->bytes -= r->stage_bytes;
        r->stage = nullptr;
        r->stage_bytes = 0;
    }
    if (cudaMalloc((void**)&r->stage, bytes) != cudaSuccess) {
        r->stage = nullptr;
        FAIL(r, FFT_ERR_OOM, "field staging buffer (%zu bytes)", bytes);
    }
    r->stage_bytes = bytes;
    r->bytes += bytes;
    return FFT_OK;
}

// Checkpoint layout (state_save / state_load): a fixed header, then the
// committed fields in the handle's bulk type (F_t 9N, the lattice-frame
// F_p^-1 9N, phi_t N) and the FP64 history with its compensation terms
// (HIST_SLOTS N).  These fix the next increment completely: the trial
// history and F_p^-1 are rewritten before they are read, GMRES starts from
// zero, the phase field from phi_t and rho_GND is recomputed from F_p.
namespace {
struct CkptHeader {
    char magic[8];
    int32_t version, prec, n[3], esz;
    uint64_t N;
    double Fbar_t[9];
    double Pbar_t[9];     // committed macroscopic stress (cut-back under mixed control)
    uint64_t setup_hash;  // grain ids, orientations, soft regions, material
};
constexpr char kCkptMagic[8] = {'F', 'F', 'T', 'C', 'K', 'P', 'T', '1'};
constexpr int32_t kCkptVersion = 2;
// 64-bit FNV-1a over a byte range, chained through h
uint64_t fnv1a(uint64_t h, const void* p, size_t n) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}
size_t ckpt_bytes(const fft_rve_s* r) {
    const size_t N = r->g.N;
    return sizeof(CkptHeader) + 19 * N * r->esz + (size_t)HIST_SLOTS * N * sizeof(double);
}
struct CkptPart {
    void* dev;
    size_t bytes;
};
void ckpt_parts(fft_rve_s* r, CkptPart out[4]) {
    const size_t N = r->g.N;
    out[0] = {r->Ht, 9 * N * r->esz};
    out[1] = {r->Hpi_t, 9 * N * r->esz};
    out[2] = {r->phi_t, N * r->esz};
    out[3] = {r->hist_c, (size_t)HIST_SLOTS * N * sizeof(double)};
}
}  // namespace

// a macroscopic target (9 values; nullptr: none) is finite, and dt is
// finite and non-negative
static bool finite_targets(const double* a, const double* b, double dt) {
    if (!(dt >= 0) || !std::isfinite(dt)) return false;
    for (int c = 0; c < 9; ++c)
        if ((a && !std::isfinite(a[c])) || (b && !std::isfinite(b[c]))) return false;
    return true;
}

extern "C" {

fft_status init_rve(fft_rve_t* out, const fft_grid* grid, const int32_t* grain_ids, int n_grains,
                    const double* euler, const fft_material* mat, const fft_options* opt,
                    const double* phi0, const uint8_t* elastic_only) {
    if (!out || !grid || !grain_ids || !euler || !mat || !opt || n_grains <= 0)
        return FFT_ERR_ARG;
    *out = nullptr;
    for (int d = 0; d < 3; ++d)
        if (grid->n[d] < 1 || grid->n[d] > 4096) return FFT_ERR_ARG;
    {
        // spectral kernels index 9 half-spectrum components with 32 bits
        const uint64_t nh = (uint64_t)(grid->n[0] / 2 + 1) * grid->n[1] * grid->n[2];
        if (9 * nh >= (1ull << 31)) return FFT_ERR_ARG;
    }
    if (!(grid->h > 0) || (opt->prec != FFT_PREC_FP64 && opt->prec != FFT_PREC_MIXED))
        return FFT_ERR_ARG;
    if (opt->max_cutbacks < 0 || opt->max_cutbacks > 10) return FFT_ERR_ARG;
    if (opt->derivative != 0 && opt->derivative != 1) return FFT_ERR_ARG;
    if (opt->kernel_variant < 0 || opt->kernel_variant > 3) return FFT_ERR_ARG;
    fft_rve_s* r = new fft_rve_s();
    r->prec = opt->prec;
    r->esz = opt->prec == FFT_PREC_FP64 ? 8 : 4;
    r->verbose = std::getenv("FATIGUEFFT_VERBOSE") != nullptr;
    {
        const char* dv = std::getenv("FATIGUEFFT_DOT64");
        r->dot64 = dv && dv[0] == '1';
    }
    {
        const char* gv = std::getenv("FATIGUEFFT_GRAPHS");
        r->graphs = !(gv && gv[0] == '0');
        const char* ps = std::getenv("FATIGUEFFT_PROF_SAMPLE");
        if (ps && std::atoi(ps) >= 1) r->prof_sample = std::atoi(ps);
    }
    r->mat = *mat;
    r->opt = *opt;
    r->h = grid->h;
    r->ngr = n_grains;
    r->st = (cudaStream_t)opt->cuda_stream;
    cudaGetDevice(&r->dev);
    SGrid& g = r->g;
    g.n0 = grid->n[0];
    g.n1 = grid->n[1];
    g.n2 = grid->n[2];
    g.n0h = g.n0 / 2 + 1;
    g.N = (size_t)g.n0 * g.n1 * g.n2;
    g.Nh = (size_t)g.n0h * g.n1 * g.n2;
    g.tpl0 = 2 * M_PI / (g.n0 * grid->h);
    g.tpl1 = 2 * M_PI / (g.n1 * grid->h);
    g.tpl2 = 2 * M_PI / (g.n2 * grid->h);
    g.tpl0f = (float)g.tpl0;
    g.tpl1f = (float)g.tpl1;
    g.tpl2f = (float)g.tpl2;
    g.fd_n0h = make_fastdiv((uint32_t)g.n0h);
    g.fd_n1 = make_fastdiv((uint32_t)g.n1);
    g.fd_Nh = make_fastdiv((uint32_t)g.Nh);
    g.willot = opt->derivative;
    g.ih = 1.0 / grid->h;
    g.ihf = (float)g.ih;
    const size_t N = g.N, Nh = g.Nh;
    for (size_t v = 0; v < N; ++v)
        if (grain_ids[v] < 0 || grain_ids[v] >= n_grains) {
            delete r;
            return FFT_ERR_ARG;
        }
    {
        uint64_t hs = 14695981039346656037ull;
        hs = fnv1a(hs, grain_ids, N * sizeof(int32_t));
        hs = fnv1a(hs, euler, 3 * (size_t)n_grains * sizeof(double));
        hs = fnv1a(hs, mat, sizeof(*mat));
        const uint8_t none = 0xff;
        hs = elastic_only ? fnv1a(hs, elastic_only, N) : fnv1a(hs, &none, 1);
        r->setup_hash = hs;
    }
    // constitutive constants (MPa, mm, s); tau*dV in N mm = 1e-3 J
    const double kT = mat->k_B * mat->T;
    r->cpp.C11 = mat->C11;
    r->cpp.C12 = mat->C12;
    r->cpp.C44 = mat->C44;
    r->cpp.tau_c0 = mat->tau_c0;
    r->cpp.mu_b = mat->mu * mat->b;
    r->cpp.g0 = mat->rho_m * mat->b * mat->b * mat->nu_D * std::exp(-mat->dF / kT);
    r->cpp.sT = kT / (mat->dV * 1e-3);
    r->cpp.lambda_h = mat->lambda_h;
    r->cpp.xi_store = mat->xi_store;
    r->cpp.G_crit = mat->G_crit;
    r->cpp.inv_b = 1.0 / mat->b;
    r->cpp.tol_local = opt->tol_local;
    r->cpp.max_local = opt->max_local;
    const double I9[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    std::memcpy(r->Fbar_t, I9, sizeof(I9));
    std::memcpy(r->Fbar, I9, sizeof(I9));
    const size_t es = r->esz, cs = 2 * r->esz;
    const int m = std::max(1, std::min(opt->restart, kMaxKrylov - 1));
    fft_status s = FFT_OK;
#define AL(ptr, bytes)                                    \
    do {                                                  \
        s = dalloc(r, (void**)&(ptr), (bytes));           \
        if (s != FFT_OK) {                                \
            release(r);                                   \
            delete r;                                     \
            return s;                                     \
        }                                                 \
    } while (0)
    AL(r->H, 9 * N * es);
    AL(r->Ht, 9 * N * es);
    AL(r->Hprev, 9 * N * es);
    AL(r->Hpi_t, 9 * N * es);
    AL(r->Hpi_tr, 9 * N * es);
    AL(r->P, 9 * N * es);
    AL(r->K, 81 * N * es);
    AL(r->rho_gnd, N * es);
    AL(r->phi, N * es);
    AL(r->phi_t, N * es);
    AL(r->drive, N * es);
    AL(r->We, N * es);
    AL(r->hist_c, HIST_SLOTS * N * sizeof(double));
    AL(r->hist_tr, HIST_SLOTS * N * sizeof(double));
    AL(r->grain, N * sizeof(int32_t));
    AL(r->Qg, 9 * (size_t)n_grains * sizeof(double));
    AL(r->G81, 81 * sizeof(double));
    AL(r->Kbar, 81 * sizeof(double));
    AL(r->rb9, 9 * N * es);
    AL(r->cb9, 9 * Nh * cs);
    AL(r->V, (size_t)(m + 1) * 3 * Nh * cs);
    AL(r->x, 3 * Nh * cs);
    AL(r->b, 3 * Nh * cs);
    AL(r->w, 3 * Nh * cs);
    AL(r->pfx, N * es);
    AL(r->pfr, N * es);
    AL(r->pfz, N * es);
    AL(r->pfp, N * es);
    AL(r->pft, N * es);
    AL(r->pfq, N * es);
    AL(r->part, (size_t)kRedSlots * kRedBlocks * sizeof(double));
    AL(r->red, kRedSlots * sizeof(double));
    AL(r->Hd, ((size_t)2 * kMaxKrylov * kHcol + 2 * kMaxKrylov + 2) * sizeof(double));
    AL(r->dy, kMaxRestart * sizeof(double));
    AL(r->dzero, kMaxRestart * sizeof(double));
    AL(r->counter, sizeof(unsigned));
    AL(r->dfail, sizeof(int));
    AL(r->bulk.err, sizeof(int));
    if (elastic_only) AL(r->elastic, N);
#undef AL
    if (cudaMallocHost((void**)&r->hred, kRedSlots * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void**)&r->hy, kMaxRestart * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void**)&r->hslot, 2 * kSlot * sizeof(double)) != cudaSuccess ||
        cudaEventCreateWithFlags(&r->slot_ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&r->slot_ev[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&r->sync_ev, cudaEventDisableTiming) != cudaSuccess) {
        release(r);
        delete r;
        return FFT_ERR_OOM;
    }
    std::vector<double> Q(9 * (size_t)n_grains);
    for (int gi = 0; gi < n_grains; ++gi) bunge_Q(euler + 3 * gi, Q.data() + 9 * gi);
    double G81[81];
    gnd_metric(G81);
    cudaMemcpyAsync(r->grain, grain_ids, N * sizeof(int32_t), cudaMemcpyHostToDevice, r->st);
    cudaMemcpyAsync(r->Qg, Q.data(), Q.size() * sizeof(double), cudaMemcpyHostToDevice, r->st);
    cudaMemcpyAsync(r->G81, G81, sizeof(G81), cudaMemcpyHostToDevice, r->st);
    if (elastic_only)
        cudaMemcpyAsync(r->elastic, elastic_only, N, cudaMemcpyHostToDevice, r->st);
    cudaMemsetAsync(r->dzero, 0, kMaxRestart * sizeof(double), r->st);
    cudaMemsetAsync(r->counter, 0, sizeof(unsigned), r->st);
    cudaMemsetAsync(r->bulk.err, 0, sizeof(int), r->st);
    {
        // the register-streaming Arnoldi update pass: kernel_variant bit 1,
        // or FATIGUEFFT_BULK=0 (FATIGUEFFT_BULK=1 forces the pipelined one)
        const char* bv = std::getenv("FATIGUEFFT_BULK");
        const bool want = bv ? bv[0] != '0' : !(opt->kernel_variant & 2);
        r->use_bulk = want && (r->prec == FFT_PREC_FP64 ? dcgs_bulk_setup<double>(r->bulk)
                                                        : dcgs_bulk_setup<float>(r->bulk));
    }
    {
        // the fused x pass in the Arnoldi step: kernel_variant bit 0, or
        // FATIGUEFFT_FUSED=1 (FATIGUEFFT_FUSED=0 forbids it); measured slower
        // than the library 3-D transforms with the separate tangent apply at
        // 64^3 (the strided batched 2-D transforms cost more than the
        // transform passes they replace).  Grids whose n0 is not a power of
        // two (or with n1 = n2 = 1) always use the library path
        const char* fv = std::getenv("FATIGUEFFT_FUSED");
        const bool want = (fv ? fv[0] == '1' : (opt->kernel_variant & 1) != 0) &&
                          (g.n1 > 1 || g.n2 > 1);
        const bool f64 = r->prec == FFT_PREC_FP64;
        if (want && (f64 ? fused_x_plan<double>(r->fx, g) : fused_x_plan<float>(r->fx, g))) {
            void* tw = nullptr;
            s = dalloc(r, &tw, (size_t)g.n0 * cs);
            if (s != FFT_OK) {
                release(r);
                delete r;
                return s;
            }
            std::vector<unsigned char> host((size_t)g.n0 * cs);
            if (f64)
                fused_x_twiddles<double>(g.n0, host.data());
            else
                fused_x_twiddles<float>(g.n0, host.data());
            cudaMemcpy(tw, host.data(), host.size(), cudaMemcpyHostToDevice);
            r->fx.tw = tw;
            // batched 2-D transform over (z, y) of the interleaved layout:
            // batch b = 9 kx-runs of n0h, element stride 9 n0h
            int n2d[2] = {g.n2, g.n1};
            const int lead2 = g.n2 == 1 ? 1 : 0;
            const int st9 = 9 * g.n0h;
            if (cufftPlanMany(&r->yz, 2 - lead2, n2d + lead2, n2d + lead2, st9, 1, n2d + lead2,
                              st9, 1, f64 ? CUFFT_Z2Z : CUFFT_C2C, st9) == CUFFT_SUCCESS) {
                r->yz_plan = true;
                cufftSetStream(r->yz, r->st);
                r->use_fused = true;
            }
        }
    }
    upload_slip_table(r->st);
    // cuFFT plans: dims slowest-first (n2, n1, n0); 9-field batches use the
    // contiguous component-major layout.  Leading unit extents are dropped
    // (a 2-D plate n2 = 1 gets a rank-2 plan over the same layout).
    int dims3[3] = {g.n2, g.n1, g.n0};
    int lead = 0;
    while (lead < 2 && dims3[lead] == 1) ++lead;
    int* dims = dims3 + lead;
    const int rank = 3 - lead;
    const cufftType tf = r->prec == FFT_PREC_FP64 ? CUFFT_D2Z : CUFFT_R2C;
    const cufftType ti = r->prec == FFT_PREC_FP64 ? CUFFT_Z2D : CUFFT_C2R;
    if (cufftPlanMany(&r->r2c9, rank, dims, nullptr, 1, (int)N, nullptr, 1, (int)Nh, tf, 9) !=
            CUFFT_SUCCESS ||
        cufftPlanMany(&r->c2r9, rank, dims, nullptr, 1, (int)Nh, nullptr, 1, (int)N, ti, 9) !=
            CUFFT_SUCCESS ||
        cufftPlanMany(&r->r2c1, rank, dims, nullptr, 1, (int)N, nullptr, 1, (int)Nh, tf, 1) !=
            CUFFT_SUCCESS ||
        cufftPlanMany(&r->c2r1, rank, dims, nullptr, 1, (int)Nh, nullptr, 1, (int)N, ti, 1) !=
            CUFFT_SUCCESS) {
        release(r);
        delete r;
        return FFT_ERR_CUFFT;
    }
    r->plans = true;
    cufftSetStream(r->r2c9, r->st);
    cufftSetStream(r->c2r9, r->st);
    cufftSetStream(r->r2c1, r->st);
    cufftSetStream(r->c2r1, r->st);
    s = DISPATCH(r, init_state(r, phi0));
    if (s == FFT_OK && cudaStreamSynchronize(r->st) != cudaSuccess) s = FFT_ERR_CUDA;
    if (s != FFT_OK) {
        release(r);
        delete r;
        return s;
    }
    *out = r;
    return FFT_OK;
}

fft_status apply_increment(fft_rve_t r, const double Fbar_target[9], double dt) {
    if (!r || !Fbar_target || !finite_targets(Fbar_target, nullptr, dt)) return FFT_ERR_ARG;
    return DISPATCH(r, apply_increment(r, Fbar_target, dt));
}

fft_status apply_increment_mixed(fft_rve_t r, const double Fbar[9], const double Pbar[9],
                                 const int32_t mask[9], double dt) {
    if (!r || !Fbar || !mask || !finite_targets(Fbar, Pbar, dt)) return FFT_ERR_ARG;
    return DISPATCH(r, apply_increment_mixed(r, Fbar, Pbar, mask, dt));
}

fft_status run_increment_mixed(fft_rve_t r, const double Fbar[9], const double Pbar[9],
                               const int32_t mask[9], double dt, fft_stats* st) {
    if (!r || !Fbar || !mask || !finite_targets(Fbar, Pbar, dt)) return FFT_ERR_ARG;
    if (st) std::memset(st, 0, sizeof(*st));
    fft_status s = DISPATCH(r, run_increment(r, Fbar, Pbar, mask, dt, st));
    if (s == FFT_OK && host_wait(r) != cudaSuccess) return FFT_ERR_CUDA;
    return s;
}

fft_status solve_equilibrium(fft_rve_t r, fft_stats* st) {
    if (!r) return FFT_ERR_ARG;
    return DISPATCH(r, solve_equilibrium(r, st));
}

fft_status update_damage(fft_rve_t r, fft_stats* st) {
    if (!r) return FFT_ERR_ARG;
    return DISPATCH(r, update_damage(r, st));
}

fft_status commit_increment(fft_rve_t r) {
    if (!r) return FFT_ERR_ARG;
    fft_status s = DISPATCH(r, commit(r));
    if (s == FFT_OK && cudaStreamSynchronize(r->st) != cudaSuccess) return FFT_ERR_CUDA;
    return s;
}

fft_status run_increment(fft_rve_t r, const double Fbar_target[9], double dt, fft_stats* st) {
    if (!r || !Fbar_target || !finite_targets(Fbar_target, nullptr, dt)) return FFT_ERR_ARG;
    if (st) std::memset(st, 0, sizeof(*st));
    fft_status s = DISPATCH(r, run_increment(r, Fbar_target, nullptr, nullptr, dt, st));
    if (s == FFT_OK && host_wait(r) != cudaSuccess) return FFT_ERR_CUDA;
    return s;
}

fft_status fields_out(fft_rve_t r, int field, void* dst, size_t bytes, int dst_is_device) {
    if (!r || !dst) return FFT_ERR_ARG;
    int nc = 1;
    if (field == FFT_FIELD_F || field == FFT_FIELD_FT || field == FFT_FIELD_P ||
        field == FFT_FIELD_PU || field == FFT_FIELD_FP)
        nc = 9;
    else if (field == FFT_FIELD_GAMMA)
        nc = 12;
    else if (field == FFT_FIELD_K)
        nc = 81;
    const size_t need = (size_t)nc * r->g.N * sizeof(double);
    if (bytes < need) FAIL(r, FFT_ERR_ARG, "fields_out: %zu bytes < %zu", bytes, need);
    double* d = (double*)dst;
    if (!dst_is_device) {
        fft_status a = ensure_stage(r, need);
        if (a != FFT_OK) return a;
        d = r->stage;
    }
    fft_status s = DISPATCH(r, fields_out(r, field, d));
    if (s == FFT_OK && !dst_is_device)
        if (cudaMemcpyAsync(dst, d, need, cudaMemcpyDeviceToHost, r->st) != cudaSuccess)
            s = FFT_ERR_CUDA;
    if (cudaStreamSynchronize(r->st) != cudaSuccess && s == FFT_OK) s = FFT_ERR_CUDA;
    return s;
}

fft_status fields_in(fft_rve_t r, int field, const double* src, size_t bytes) {
    if (!r || !src) return FFT_ERR_ARG;
    int nc = 1;
    if (field == FFT_FIELD_F || field == FFT_FIELD_FT || field == FFT_FIELD_FP)
        nc = 9;
    else if (field == FFT_FIELD_GAMMA)
        nc = 12;
    const size_t need = (size_t)nc * r->g.N * sizeof(double);
    if (bytes < need) FAIL(r, FFT_ERR_ARG, "fields_in: %zu bytes < %zu", bytes, need);
    fft_status s = ensure_stage(r, need);
    if (s != FFT_OK) return s;
    if (cudaMemcpyAsync(r->stage, src, need, cudaMemcpyHostToDevice, r->st) != cudaSuccess)
        s = FFT_ERR_CUDA;
    if (s == FFT_OK) s = DISPATCH(r, fields_in(r, field, r->stage));
    if (cudaStreamSynchronize(r->st) != cudaSuccess && s == FFT_OK) s = FFT_ERR_CUDA;
    return s;
}

fft_status state_save(fft_rve_t r, void* dst, size_t* bytes) {
    if (!r || !bytes) return FFT_ERR_ARG;
    const size_t need = ckpt_bytes(r);
    if (!dst) {
        *bytes = need;
        return FFT_OK;
    }
    if (*bytes < need) FAIL(r, FFT_ERR_ARG, "state_save: %zu bytes < %zu", *bytes, need);
    CkptHeader h{};
    std::memcpy(h.magic, kCkptMagic, sizeof(h.magic));
    h.version = kCkptVersion;
    h.prec = r->prec;
    h.n[0] = r->g.n0;
    h.n[1] = r->g.n1;
    h.n[2] = r->g.n2;
    h.esz = (int32_t)r->esz;
    h.N = r->g.N;
    std::memcpy(h.Fbar_t, r->Fbar_t, sizeof(h.Fbar_t));
    std::memcpy(h.Pbar_t, r->Pbar_t, sizeof(h.Pbar_t));
    h.setup_hash = r->setup_hash;
    std::memcpy(dst, &h, sizeof(h));
    char* p = (char*)dst + sizeof(h);
    CkptPart parts[4];
    ckpt_parts(r, parts);
    for (const CkptPart& c : parts) {
        CK(r, cudaMemcpyAsync(p, c.dev, c.bytes, cudaMemcpyDeviceToHost, r->st));
        p += c.bytes;
    }
    CK(r, cudaStreamSynchronize(r->st));
    *bytes = need;
    return FFT_OK;
}

fft_status state_load(fft_rve_t r, const void* src, size_t bytes) {
    if (!r || !src) return FFT_ERR_ARG;
    CkptHeader h;
    if (bytes < sizeof(h)) FAIL(r, FFT_ERR_ARG, "state_load: %zu bytes is no checkpoint", bytes);
    std::memcpy(&h, src, sizeof(h));
    if (std::memcmp(h.magic, kCkptMagic, sizeof(h.magic)) != 0 || h.version != kCkptVersion)
        FAIL(r, FFT_ERR_ARG, "state_load: not a checkpoint of this library");
    if (h.prec != r->prec || h.esz != (int32_t)r->esz || h.n[0] != r->g.n0 ||
        h.n[1] != r->g.n1 || h.n[2] != r->g.n2 || h.N != (uint64_t)r->g.N)
        FAIL(r, FFT_ERR_ARG, "state_load: checkpoint of another grid or precision");
    if (h.setup_hash != r->setup_hash)
        FAIL(r, FFT_ERR_ARG,
             "state_load: checkpoint of another microstructure or material (grain ids, "
             "orientations, soft regions or material constants differ)");
    const size_t need = ckpt_bytes(r);
    if (bytes < need) FAIL(r, FFT_ERR_ARG, "state_load: %zu bytes < %zu", bytes, need);
    const char* p = (const char*)src + sizeof(h);
    CkptPart parts[4];
    ckpt_parts(r, parts);
    for (const CkptPart& c : parts) {
        CK(r, cudaMemcpyAsync(c.dev, p, c.bytes, cudaMemcpyHostToDevice, r->st));
        p += c.bytes;
    }
    // the current iterate restarts at the committed state
    CK(r, cudaMemcpyAsync(r->H, r->Ht, 9 * r->g.N * r->esz, cudaMemcpyDeviceToDevice, r->st));
    CK(r, cudaMemcpyAsync(r->phi, r->phi_t, r->g.N * r->esz, cudaMemcpyDeviceToDevice, r->st));
    CK(r, cudaStreamSynchronize(r->st));
    std::memcpy(r->Fbar_t, h.Fbar_t, sizeof(r->Fbar_t));
    std::memcpy(r->Fbar, h.Fbar_t, sizeof(r->Fbar));
    std::memcpy(r->Pbar_t, h.Pbar_t, sizeof(r->Pbar_t));
    r->state = ST_COMMITTED;
    r->converged = false;
    r->cp_valid = false;
    r->mixed = false;
    r->stag_it = 0;
    return FFT_OK;
}

fft_status eval_constitutive(fft_rve_t r, double dt, int with_history, int* local_fail) {
    if (!r || !(dt >= 0)) return FFT_ERR_ARG;
    r->dt = dt;
    return DISPATCH(r, cp(r, with_history != 0, local_fail));
}

fft_status eval_gnd(fft_rve_t r) {
    if (!r) return FFT_ERR_ARG;
    fft_status s = DISPATCH(r, gnd(r));
    if (s == FFT_OK && cudaStreamSynchronize(r->st) != cudaSuccess) return FFT_ERR_CUDA;
    return s;
}

fft_status solve_phase_field(fft_rve_t r, int* iters) {
    if (!r) return FFT_ERR_ARG;
    double o4[4];
    int it = 0;
    fft_status s = DISPATCH(r, phase_field(r, &it, o4));
    if (iters) *iters = it;
    return s;
}

size_t rve_device_bytes(fft_rve_t r) { return r ? r->bytes : 0; }

fft_status rve_profile(fft_rve_t r, unsigned mask) {
    if (!r) return FFT_ERR_ARG;
    mask &= 0xffffu;
    if (mask != r->prof_mask) {
        // the step graphs carry the old mask's timing events: rebuild them
        if (cudaStreamSynchronize(r->st) != cudaSuccess) return FFT_ERR_CUDA;
        prof_collect(r);
        drop_graphs(r);
    }
    r->prof_mask = mask;
    return FFT_OK;
}

fft_status rve_profile_read(fft_rve_t r, double* ms, long long* counts, double* bytes,
                            int reset) {
    if (!r || !ms || !counts) return FFT_ERR_ARG;
    if (cudaStreamSynchronize(r->st) != cudaSuccess) return FFT_ERR_CUDA;
    prof_collect(r);
    for (int i = 0; i < 16; ++i) {
        ms[i] = r->prof_ms[i];
        counts[i] = r->prof_cnt[i];
        if (bytes) bytes[i] = r->prof_bytes[i];
        if (reset) {
            r->prof_ms[i] = 0;
            r->prof_cnt[i] = 0;
            r->prof_bytes[i] = 0;
        }
    }
    return FFT_OK;
}

long long rve_kernel_launches(fft_rve_t r) { return r ? r->launches : 0; }

int fft_selftest_bounded_wait(unsigned rounds) {
    if (rounds == 0 || rounds > (1u << 16)) return -2;
    return fatfft::selftest_bounded_wait(rounds);
}

}  // extern "C"

// Library-internal accessors for the batch driver (batch.cu).
int fatfft_rve_device(fft_rve_t r) { return r ? r->dev : -1; }
void* fatfft_rve_stream(fft_rve_t r) { return r ? (void*)r->st : nullptr; }
size_t fatfft_rve_voxels(fft_rve_t r) { return r ? r->g.N : 0; }
void fatfft_rve_set_poll(fft_rve_t r, bool on) {
    if (r) r->poll = on;
}
// membership of a batch: claim fails if the handle already belongs to one
static std::mutex g_batch_claim;
bool fatfft_rve_claim(fft_rve_t r, void* batch) {
    std::lock_guard<std::mutex> lk(g_batch_claim);
    if (!r || r->batch) return false;
    r->batch = batch;
    return true;
}
void fatfft_rve_unclaim(fft_rve_t r, void* batch) {
    std::lock_guard<std::mutex> lk(g_batch_claim);
    if (r && r->batch == batch) r->batch = nullptr;
}

extern "C" {

void rve_destroy(fft_rve_t r) {
    if (!r) return;
    {
        // a handle still in a batch keeps part of its buffers in the
        // batch's class arenas: it stays alive until the batch is destroyed
        std::lock_guard<std::mutex> lk(g_batch_claim);
        if (r->batch) {
            r->err = "rve_destroy: the handle is still in a batch (destroy the batch first)";
            return;
        }
    }
    cudaStreamSynchronize(r->st);
    release(r);
    delete r;
}

const char* fft_last_error(fft_rve_t r) { return r ? r->err.c_str() : "null handle"; }

}  // extern "C"
