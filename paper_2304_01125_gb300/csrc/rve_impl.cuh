// Internals of the fatiguefft driver shared by the single-handle driver
// (rve.cu) and the lockstep class driver (gang.cu): the handle, the
// host-side helpers and the stage functions of Algorithm 1 (Impl).
#pragma once
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "fatiguefft.h"
#include "launch.h"
#include "spec.h"

using namespace fatfft;


namespace {
enum { ST_NEW = 0, ST_APPLIED = 1, ST_EQUIL = 2, ST_DAMAGE = 3, ST_COMMITTED = 4 };
constexpr int kMaxRestart = 64;
constexpr int kSlot = 96;    // doubles per look-ahead slot (kSlotLen used)
constexpr int kDslot = 128;  // device copy of the slot: red + kDslot
static_assert(kSlotLen <= kSlot, "host slot too small");
static_assert(kDslot + kSlotLen <= kRedSlots, "device slot outside the reduction buffer");
static_assert(3 + 2 * (kMaxKrylov - 1) <= kDslot, "Arnoldi dots overlap the device slot");
}  // namespace

namespace {
// NVTX range over one stage of Algorithm 1, in the library's own domain
// ("fatiguefft"), so that profilers show the stages without touching the
// caller's default-domain ranges; a no-op without a tool attached.
static nvtxDomainHandle_t nvtx_domain() {
    static nvtxDomainHandle_t d = nvtxDomainCreateA("fatiguefft");
    return d;
}
struct NvtxRange {
    explicit NvtxRange(const char* name) {
        nvtxEventAttributes_t a = {};
        a.version = NVTX_VERSION;
        a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        a.messageType = NVTX_MESSAGE_TYPE_ASCII;
        a.message.ascii = name;
        nvtxDomainRangePushEx(nvtx_domain(), &a);
    }
    ~NvtxRange() { nvtxDomainRangePop(nvtx_domain()); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace

struct fft_rve_s {
    int prec = 0;
    size_t esz = 8;  // bytes of the bulk real type
    SGrid g{};
    double h = 0;
    int ngr = 0;
    fft_material mat{};
    fft_options opt{};
    CPParams cpp{};
    cudaStream_t st = 0;
    int dev = 0;  // the device current at init_rve
    cufftHandle r2c9 = 0, c2r9 = 0, r2c1 = 0, c2r1 = 0;
    bool plans = false;
    // device state (bulk type unless noted)
    void *H = nullptr, *Ht = nullptr, *Hprev = nullptr, *Hpi_t = nullptr, *Hpi_tr = nullptr;
    void *P = nullptr, *K = nullptr, *rho_gnd = nullptr, *phi = nullptr, *phi_t = nullptr;
    void *drive = nullptr, *We = nullptr;
    double *hist_c = nullptr, *hist_tr = nullptr;
    int32_t* grain = nullptr;
    uint8_t* elastic = nullptr;
    double *Qg = nullptr, *G81 = nullptr, *Kbar = nullptr;
    double* Hd = nullptr;  // Hessenberg columns, final then provisional (kMaxKrylov x kHcol
                           // each), then the DCGS2 step coefficients
    // work buffers
    void *rb9 = nullptr, *cb9 = nullptr;                      // real 9N, complex 9Nh
    void *V = nullptr, *x = nullptr, *b = nullptr, *w = nullptr;  // GMRES (complex)
    void *pfx = nullptr, *pfr = nullptr, *pfz = nullptr, *pfp = nullptr, *pft = nullptr,
         *pfq = nullptr;
    double *part = nullptr, *red = nullptr, *dy = nullptr, *dzero = nullptr;
    unsigned* counter = nullptr;  // ticket of the last-block reductions
    double *hred = nullptr, *hy = nullptr;  // pinned host
    double* hslot = nullptr;                // pinned look-ahead slots, 2 x kSlot doubles
    cudaEvent_t slot_ev[2] = {nullptr, nullptr};
    // host waits: a blocking (spinning) synchronisation by default; with
    // poll set (a batch drives the handle, its host threads may outnumber
    // the cores) the event is polled and the core yielded between polls
    cudaEvent_t sync_ev = nullptr;
    bool poll = false;
    // the batch the handle belongs to (at most one: a lockstep class takes
    // over the handle's Arnoldi scratch until its batch is destroyed)
    void* batch = nullptr;
    // one CUDA graph per Arnoldi column j (the step's pointers and grid
    // shapes depend on j only), captured on first use; off on the legacy
    // default stream, while the kernel profiler runs, or with
    // FATIGUEFFT_GRAPHS=0
    cudaGraphExec_t step_exec[kMaxKrylov] = {};
    long long step_launches[kMaxKrylov] = {};
    bool graphs = true;
    // with the profiler on, a second graph per column carries the timing
    // event nodes and replaces the plain one on every prof_sample-th replay
    // (FATIGUEFFT_PROF_SAMPLE, default 8), so timing perturbs few replays
    cudaGraphExec_t step_exec_prof[kMaxKrylov] = {};
    int prof_sample = 8;
    long long prof_tick = 0;
    int* dfail = nullptr;
    // pipelined Arnoldi kernels (bulk copies into a shared-memory ring):
    // resident-CTA budgets and the device error word of their bounded waits
    BulkCfg bulk{};
    bool use_bulk = false;
    // fused x pass of the Arnoldi step (inverse real transform along x,
    // tangent apply, forward real transform in one kernel) between batched
    // 2-D transforms over (z, y) of the interleaved spectrum layout; off
    // for grids it does not support or with FATIGUEFFT_FUSED=0
    FusedX fx{};
    bool use_fused = false;
    cufftHandle yz = 0;
    bool yz_plan = false;
    double* stage = nullptr;  // device staging for host fields_out / fields_in
    size_t stage_bytes = 0;
    std::vector<void*> allocs;
    size_t bytes = 0;
    long long launches = 0;
    // opt-in kernel timing per family (CUDA events on the handle's stream)
    unsigned prof_mask = 0;
    struct ProfEv {
        cudaEvent_t a, b;
        int fam;
        double bytes;
        bool owned;  // recorded by a step graph's event nodes; kept by the graph
    };
    std::vector<ProfEv> prof_pending;
    bool capturing = false;                      // a step graph is being captured
    std::vector<ProfEv> cap_prof;                // its profiler event pairs
    std::vector<ProfEv> step_prof[kMaxKrylov];   // per column, replayed with it
    std::vector<cudaEvent_t> prof_pool;
    double prof_ms[16] = {0};
    double prof_bytes[16] = {0};
    long long prof_cnt[16] = {0};
    // Algorithm 1 bookkeeping
    double Fbar_t[9], Fbar[9], dt = 0;
    // mixed stress/strain control (apply_increment_mixed)
    bool mixed = false;
    int mask[9] = {0};
    double Pstar[9] = {0};
    // mean degraded stress <g P> at the last damage update, and the committed
    // macroscopic stress: the target on stress-controlled components, the
    // mean on the others (the start of a halved stress path under cut-back)
    double Pbar_cur[9] = {0}, Pbar_t[9] = {0};
    // hash of the grain ids, orientations, soft-region mask and material
    // (a checkpoint loads only into a handle with the same set-up)
    uint64_t setup_hash = 0;
    int state = ST_NEW, stag_it = 0;
    bool phi_changed = true, skipped = false, converged = false, cp_valid = false;
    bool verbose = false;  // FATIGUEFFT_VERBOSE: solver traces on stderr
    // FATIGUEFFT_DOT64=1: the Arnoldi dot pass forms its per-thread products
    // and partial sums in FP64 (a measurement of the FP32 partials' effect)
    bool dot64 = false;
    std::string err;
};


#define FAIL(r, code, ...)                                          \
    do {                                                            \
        char _b[512];                                               \
        std::snprintf(_b, sizeof(_b), __VA_ARGS__);                 \
        (r)->err = _b;                                              \
        return code;                                                \
    } while (0)
#define CK(r, x)                                                                           \
    do {                                                                                   \
        cudaError_t _e = (x);                                                              \
        if (_e != cudaSuccess) FAIL(r, FFT_ERR_CUDA, "%s: %s", #x, cudaGetErrorString(_e)); \
    } while (0)
#define CKF(r, x)                                                                 \
    do {                                                                          \
        cufftResult _e = (x);                                                     \
        if (_e != CUFFT_SUCCESS) FAIL(r, FFT_ERR_CUFFT, "%s: cufft error %d", #x, (int)_e); \
    } while (0)
#define TRY(x)                        \
    do {                              \
        fft_status _s = (x);          \
        if (_s != FFT_OK) return _s;  \
    } while (0)

namespace {

static Red red_at(fft_rve_s* r, double* out) { return Red{r->part, r->counter, out}; }

// The host waits for an event (for the whole stream with e = nullptr: an
// event recorded on it now), spinning or, with r->poll, polling and yielding.
static cudaError_t host_wait(fft_rve_s* r, cudaEvent_t e = nullptr) {
    if (!r->poll) return e ? cudaEventSynchronize(e) : cudaStreamSynchronize(r->st);
    if (!e) {
        e = r->sync_ev;
        const cudaError_t re = cudaEventRecord(e, r->st);
        if (re != cudaSuccess) return re;
    }
    for (;;) {
        const cudaError_t q = cudaEventQuery(e);
        if (q != cudaErrorNotReady) return q;
        std::this_thread::yield();
    }
}

// kernel families for the opt-in timing
enum {
    KF_CP = 0, KF_TANGENT = 1, KF_PRECOND = 2, KF_CONTRACT = 3, KF_MDOT = 4, KF_GSUPD = 5,
    KF_XUPD = 6, KF_KBAR = 7, KF_RESID = 8, KF_FUPD = 9, KF_PF = 10, KF_GND = 11, KF_FFT9 = 12,
    KF_FFT1 = 13, KF_FIN = 14, KF_OTHER = 15
};
// Event for the profiler: from the pool, or (while a step graph is captured)
// a new one owned by that graph and recorded through an event node.
static cudaEvent_t prof_event(fft_rve_s* r) {
    cudaEvent_t e = nullptr;
    if (r->capturing || r->prof_pool.empty()) {
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    } else {
        e = r->prof_pool.back();
        r->prof_pool.pop_back();
    }
    const cudaError_t ce = r->capturing
                               ? cudaEventRecordWithFlags(e, r->st, cudaEventRecordExternal)
                               : cudaEventRecord(e, r->st);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e);
        return nullptr;
    }
    return e;
}
static cudaEvent_t prof_begin(fft_rve_s* r, int fam) {
    if (!(r->prof_mask >> fam & 1u)) return nullptr;
    return prof_event(r);
}
// bytes: the algorithmic HBM traffic of the bracketed launch(es)
static void prof_end(fft_rve_s* r, int fam, cudaEvent_t a, double bytes = 0.0) {
    if (!a) return;
    cudaEvent_t b = prof_event(r);
    if (!b) return;
    if (r->capturing)
        r->cap_prof.push_back({a, b, fam, bytes, true});
    else
        r->prof_pending.push_back({a, b, fam, bytes, false});
}
static void prof_release(fft_rve_s* r, const fft_rve_s::ProfEv& p) {
    if (p.owned) return;
    r->prof_pool.push_back(p.a);
    r->prof_pool.push_back(p.b);
}
// after a stream synchronisation: fold the recorded pairs into the totals
static void prof_collect(fft_rve_s* r) {
    for (auto& p : r->prof_pending) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            r->prof_ms[p.fam] += ms;
            r->prof_bytes[p.fam] += p.bytes;
            r->prof_cnt[p.fam] += 1;
        }
        prof_release(r, p);
    }
    r->prof_pending.clear();
}

// fold in the recorded pairs whose end event has completed (no waiting)
static void prof_collect_if_done(fft_rve_s* r) {
    if (r->prof_pending.empty()) return;
    std::vector<fft_rve_s::ProfEv> keep;
    for (auto& p : r->prof_pending) {
        if (cudaEventQuery(p.b) != cudaSuccess) {
            keep.push_back(p);
            continue;
        }
        float ms = 0;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            r->prof_ms[p.fam] += ms;
            r->prof_bytes[p.fam] += p.bytes;
            r->prof_cnt[p.fam] += 1;
        }
        prof_release(r, p);
    }
    r->prof_pending.swap(keep);
    cudaGetLastError();  // cudaEventQuery's cudaErrorNotReady is not an error here
}

// Destroy the cached step graphs and their timing events (call with the
// stream idle and the profiler's pending list folded in).
static void drop_graphs(fft_rve_s* r) {
    std::vector<fft_rve_s::ProfEv> keep;  // forget replays not yet folded in
    for (auto& p : r->prof_pending)
        if (!p.owned) keep.push_back(p);
    r->prof_pending.swap(keep);
    for (int j = 0; j < kMaxKrylov; ++j) {
        if (r->step_exec[j]) cudaGraphExecDestroy(r->step_exec[j]);
        r->step_exec[j] = nullptr;
        if (r->step_exec_prof[j]) cudaGraphExecDestroy(r->step_exec_prof[j]);
        r->step_exec_prof[j] = nullptr;
        for (auto& p : r->step_prof[j]) {
            cudaEventDestroy(p.a);
            cudaEventDestroy(p.b);
        }
        r->step_prof[j].clear();
    }
}

static fft_status dalloc(fft_rve_s* r, void** p, size_t bytes) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        FAIL(r, FFT_ERR_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    r->allocs.push_back(*p);
    r->bytes += bytes;
    return FFT_OK;
}

// ---------------------------------------------------------------- cuFFT
template <typename R> struct FFT;
template <> struct FFT<float> {
    static constexpr cufftType R2C = CUFFT_R2C, C2R = CUFFT_C2R, C2C = CUFFT_C2C;
    static cufftResult c2c(cufftHandle p, void* io, int dir) {
        return cufftExecC2C(p, (cufftComplex*)io, (cufftComplex*)io, dir);
    }
    static cufftResult fwd(cufftHandle p, void* i, void* o) {
        return cufftExecR2C(p, (cufftReal*)i, (cufftComplex*)o);
    }
    static cufftResult inv(cufftHandle p, void* i, void* o) {
        return cufftExecC2R(p, (cufftComplex*)i, (cufftReal*)o);
    }
};
template <> struct FFT<double> {
    static constexpr cufftType R2C = CUFFT_D2Z, C2R = CUFFT_Z2D, C2C = CUFFT_Z2Z;
    static cufftResult c2c(cufftHandle p, void* io, int dir) {
        return cufftExecZ2Z(p, (cufftDoubleComplex*)io, (cufftDoubleComplex*)io, dir);
    }
    static cufftResult fwd(cufftHandle p, void* i, void* o) {
        return cufftExecD2Z(p, (cufftDoubleReal*)i, (cufftDoubleComplex*)o);
    }
    static cufftResult inv(cufftHandle p, void* i, void* o) {
        return cufftExecZ2D(p, (cufftDoubleComplex*)i, (cufftDoubleReal*)o);
    }
};

// ------------------------------------------------------- stage helpers
template <typename R>
struct Impl {
    typedef typename Tr<R>::Cx Cx;

    // reduction results red[0, n) to the host: the copy enqueued, then read
    // (the two halves let a driver of several handles overlap them)
    static fft_status fetch_enq(fft_rve_s* r, int n) {
        CK(r, cudaMemcpyAsync(r->hred, r->red, n * sizeof(double), cudaMemcpyDeviceToHost, r->st));
        return FFT_OK;
    }
    static fft_status fetch_get(fft_rve_s* r, int n) {
        CK(r, host_wait(r));
        prof_collect(r);
        for (int i = 0; i < n; ++i)
            if (!std::isfinite(r->hred[i]))
                FAIL(r, FFT_ERR_NONFINITE, "non-finite reduction value (slot %d)", i);
        return FFT_OK;
    }
    static fft_status fetch(fft_rve_s* r, int n) {
        TRY(fetch_enq(r, n));
        return fetch_get(r, n);
    }
    static fft_status fwd9(fft_rve_s* r) {
        cudaEvent_t e = prof_begin(r, KF_FFT9);
        CKF(r, FFT<R>::fwd(r->r2c9, r->rb9, r->cb9));
        prof_end(r, KF_FFT9, e);
        return FFT_OK;
    }
    static fft_status inv9(fft_rve_s* r) {
        cudaEvent_t e = prof_begin(r, KF_FFT9);
        CKF(r, FFT<R>::inv(r->c2r9, r->cb9, r->rb9));
        prof_end(r, KF_FFT9, e);
        return FFT_OK;
    }
    static fft_status fwd1(fft_rve_s* r, void* in) {
        cudaEvent_t e = prof_begin(r, KF_FFT1);
        CKF(r, FFT<R>::fwd(r->r2c1, in, r->cb9));
        prof_end(r, KF_FFT1, e);
        return FFT_OK;
    }
    static fft_status inv1(fft_rve_s* r, void* out) {
        cudaEvent_t e = prof_begin(r, KF_FFT1);
        CKF(r, FFT<R>::inv(r->c2r1, r->cb9, out));
        prof_end(r, KF_FFT1, e);
        return FFT_OK;
    }

    // rho_GND from the committed F_p (Eq. nyeindexfourier + regularisation)
    static fft_status gnd(fft_rve_s* r) {
        const size_t N = r->g.N;
        fp_sample<R>(r->Hpi_t, r->grain, r->Qg, r->rb9, N, r->st);
        TRY(fwd9(r));
        nye<R>(r->cb9, r->g, r->mat.ell_Fp * r->mat.ell_Fp, r->st);
        TRY(inv9(r));
        gnd_rho<R>(r->rb9, r->grain, r->Qg, r->G81, 1.0 / r->mat.b, r->rho_gnd, N, r->st);
        r->launches += 3;
        CK(r, cudaGetLastError());
        return FFT_OK;
    }

    static fft_status cp(fft_rve_s* r, bool hist, int* fails) {
        TRY(cp_enq(r, hist));
        return cp_get(r, fails);
    }
    // the constitutive update enqueued (with the copy of its failure count)
    static fft_status cp_enq(fft_rve_s* r, bool hist) {
        NvtxRange nvtx_("constitutive");
        CPFields f;
        f.H = r->H;
        f.Hpi = r->Hpi_t;
        f.rho_gnd = r->rho_gnd;
        f.grain = r->grain;
        f.elastic = r->elastic;
        f.Qg = r->Qg;
        f.hist_c = r->hist_c;
        f.hist_tr = r->hist_tr;
        f.P = r->P;
        f.K = r->K;
        f.Hpi_tr = r->Hpi_tr;
        f.drive = r->drive;
        f.We = r->We;
        f.fail_count = r->dfail;
        f.N = r->g.N;
        CPParams p = r->cpp;
        p.dt = r->dt;
        CK(r, cudaMemsetAsync(r->dfail, 0, sizeof(int), r->st));
        cudaEvent_t e = prof_begin(r, KF_CP);
        launch_constitutive<R>(f, p, hist, r->st);
        // H, Hpi, rho_gnd, grain, rho history in; P, K out; with history also
        // the 32-slot FP64 history in and out, Hpi_tr, drive, W_e+ out
        const double N = (double)r->g.N, es = (double)sizeof(R);
        prof_end(r, KF_CP, e,
                 N * (es * (9 + 9 + 1 + 9 + 81) + 4 + 16 +
                      (hist ? 2.0 * HIST_SLOTS * 8 + es * 11 : 0.0)));
        r->launches += 1;
        CK(r, cudaGetLastError());
        CK(r, cudaMemcpyAsync(r->hy, r->dfail, sizeof(int), cudaMemcpyDeviceToHost, r->st));
        return FFT_OK;
    }
    // waits for it: local-solve failure count, the tangent valid
    static fft_status cp_get(fft_rve_s* r, int* fails) {
        int nf = 0;
        CK(r, host_wait(r));
        prof_collect(r);
        std::memcpy(&nf, r->hy, sizeof(int));
        if (fails) *fails = nf;
        r->cp_valid = true;
        return FFT_OK;
    }

    // w = A u with A u = -F{g K : F^-1{u (x) i xi}} . i xi, projected onto
    // real fields; use_pre applies the Green preconditioner to u first
    // (u scaled by scale, optionally stored to vout).
    static fft_status apply_op(fft_rve_s* r, const void* u, double scale, void* vout, int use_pre,
                               void* w, int nv) {
        const double N = (double)r->g.N, Nh = (double)r->g.Nh, es = (double)sizeof(R);
        cudaEvent_t e = prof_begin(r, KF_PRECOND);
        precond_grad<R>(u, scale, vout, r->Kbar, r->g, r->cb9, use_pre, r->st);
        prof_end(r, KF_PRECOND, e, Nh * 2 * es * (3 + 9 + (vout ? 3 : 0)));
        TRY(inv9(r));
        e = prof_begin(r, KF_TANGENT);
        tangent_apply<R>(r->rb9, r->K, r->phi, r->mat.k_res, r->g.N, r->st);
        prof_end(r, KF_TANGENT, e, N * es * (9 + 81 + 1 + 9));
        TRY(fwd9(r));
        e = prof_begin(r, KF_CONTRACT);
        contract<R>(r->cb9, r->g, w, r->st);
        prof_end(r, KF_CONTRACT, e, Nh * 2 * es * (9 + 3));
        r->launches += 3;
        (void)nv;
        return FFT_OK;
    }

    // One Arnoldi step j.  Krylov slot j holds the unnormalised vector w^_j
    // (for j = 0 it is formed here as src * scale, normalised) and cb9 the
    // spectrum of grad(M w^_j), written by the previous step's update.  The
    // step forms w = A M V_j with V_j = w^_j / ||w^_j|| (the norm from
    // red[64], applied in the tangent apply; slot j is normalised by the
    // contraction), red[0] = ||w||^2, red[1 + i] = <V_i, w>, the Gram-Schmidt
    // update w^_{j+1} into slot j + 1 with red[64] = ||w^_{j+1}||^2 and the
    // next gradient spectrum, and the optional second pass (red[95] = 1,
    // red[97 + i]); red[0, 130) is then copied to host slot j % 2.
    static fft_status enqueue_step(fft_rve_s* r, int j, const void* src, double scale) {
        if (j == 0) {
            const double Nh = (double)r->g.Nh, es = (double)sizeof(R);
            cudaEvent_t e = prof_begin(r, KF_PRECOND);
            precond_grad<R>(src, scale, r->V, r->Kbar, r->g, r->cb9, 1, r->st,
                            r->use_fused ? 1 : 0);
            prof_end(r, KF_PRECOND, e, Nh * 2 * es * (3 + 3 + 9));
            r->launches += 1;
        }
        if (r->graphs && r->st) {
            const bool timed = r->prof_mask && (r->prof_tick++ % r->prof_sample) == 0;
            cudaGraphExec_t& ex = timed ? r->step_exec_prof[j] : r->step_exec[j];
            if (!ex) {
                const long long l0 = r->launches;
                const unsigned mask = r->prof_mask;
                if (!timed) r->prof_mask = 0;  // the plain graph has no event nodes
                CK(r, cudaStreamBeginCapture(r->st, cudaStreamCaptureModeThreadLocal));
                r->capturing = true;
                r->cap_prof.clear();
                const fft_status sb = step_body(r, j);
                r->capturing = false;
                r->prof_mask = mask;
                cudaGraph_t gr = nullptr;
                const cudaError_t ce = cudaStreamEndCapture(r->st, &gr);
                if (timed) r->step_prof[j].swap(r->cap_prof);
                for (auto& p : r->cap_prof) {
                    cudaEventDestroy(p.a);
                    cudaEventDestroy(p.b);
                }
                r->cap_prof.clear();
                cudaError_t ie = ce;
                if (sb == FFT_OK && ce == cudaSuccess) ie = cudaGraphInstantiate(&ex, gr, 0);
                if (gr) cudaGraphDestroy(gr);
                const long long nl = r->launches - l0;  // this column's own kernels
                r->launches = l0;
                if (sb != FFT_OK || ie != cudaSuccess) {
                    // capture unsupported here: run this handle without graphs
                    // (a genuine error then surfaces from the direct launch)
                    cudaGetLastError();
                    ex = nullptr;
                    drop_graphs(r);
                    r->graphs = false;
                    if (r->verbose)
                        std::fprintf(stderr, "  step graph capture failed (%s, %s); graphs off\n",
                                     cudaGetErrorString(ie), r->err.c_str());
                    TRY(step_body(r, j));
                    CK(r, cudaEventRecord(r->slot_ev[j % 2], r->st));
                    return FFT_OK;
                }
                r->step_launches[j] = nl;
            }
            CK(r, cudaGraphLaunch(ex, r->st));
            r->launches += r->step_launches[j];
            // the graph's timing events; folded in before it is launched again
            // (every GMRES cycle ends with a stream synchronisation)
            if (timed)
                for (auto& p : r->step_prof[j]) r->prof_pending.push_back(p);
        } else {
            TRY(step_body(r, j));
        }
        CK(r, cudaEventRecord(r->slot_ev[j % 2], r->st));
        return FFT_OK;
    }

    // The body of Arnoldi step j after its first-column set-up (see
    // enqueue_step); captured into the column's graph when graphs are on.
    static fft_status step_body(fft_rve_s* r, int k) {
        const double N = (double)r->g.N, Nh = (double)r->g.Nh, es = (double)sizeof(R);
        const size_t vs = 3 * r->g.Nh;
        Cx* V = (Cx*)r->V;
        double* dslot = r->red + kDslot;
        cudaEvent_t e;
        double* Hp = r->Hd + (size_t)kMaxKrylov * kHcol;
        double* coef = Hp + (size_t)kMaxKrylov * kHcol;
        const BulkCfg* bc = r->use_bulk ? &r->bulk : nullptr;
        if (r->use_fused) {
            // the gradient spectrum (interleaved layout) to (kx, y, z) by the
            // batched 2-D inverse transform, then the fused x pass (inverse
            // real transform, tangent apply, forward real transform), then
            // the batched 2-D forward transform
            e = prof_begin(r, KF_FFT9);
            CKF(r, FFT<R>::c2c(r->yz, r->cb9, CUFFT_INVERSE));
            prof_end(r, KF_FFT9, e);
            e = prof_begin(r, KF_TANGENT);
            fused_xpass<R>(r->fx, r->cb9, r->K, r->phi, r->mat.k_res, r->g, r->st);
            prof_end(r, KF_TANGENT, e, Nh * 2 * es * 18 + N * es * 82);
            e = prof_begin(r, KF_FFT9);
            CKF(r, FFT<R>::c2c(r->yz, r->cb9, CUFFT_FORWARD));
            prof_end(r, KF_FFT9, e);
            // z = -div T (stored to w) and, in the same pass over c_k and
            // q_0 .. q_{k-1}: alpha, beta, a, b and the step's coefficients
            e = prof_begin(r, KF_MDOT);
            contract_dots<R>(r->cb9, r->g, r->w, V + (size_t)k * vs, V, vs, k,
                             red_at(r, r->red), r->Hd, Hp, dslot, coef, bc, r->st, 1);
            prof_end(r, KF_MDOT, e, Nh * 2 * es * (9 + 3 + 3 * (k + 1)));
            // q_k final, c_{k+1} and the next gradient spectrum
            e = prof_begin(r, KF_GSUPD);
            dcgs_update<R>(V, vs, k, r->w, coef, r->Kbar, r->g, r->cb9,
                           red_at(r, dslot + kSlotNorm), bc, r->st, 1);
            prof_end(r, KF_GSUPD, e, Nh * 2 * es * 3 * (k + 2 + 2 + 3));
        } else {
            TRY(inv9(r));
            e = prof_begin(r, KF_TANGENT);
            tangent_apply<R>(r->rb9, r->K, r->phi, r->mat.k_res, r->g.N, r->st);
            prof_end(r, KF_TANGENT, e, N * es * (9 + 81 + 1 + 9));
            TRY(fwd9(r));
            // z = -div T (stored to w) and, in the same pass over c_k and
            // q_0 .. q_{k-1}: alpha, beta, a, b and the step's coefficients
            e = prof_begin(r, KF_MDOT);
            contract_dots<R>(r->cb9, r->g, r->w, V + (size_t)k * vs, V, vs, k,
                             red_at(r, r->red), r->Hd, Hp, dslot, coef, bc, r->st, 0,
                             r->dot64 ? 1 : 0);
            prof_end(r, KF_MDOT, e, Nh * 2 * es * (9 + 3 + 3 * (k + 1)));
            // q_k final, c_{k+1} and the next gradient spectrum
            e = prof_begin(r, KF_GSUPD);
            dcgs_update<R>(V, vs, k, r->w, coef, r->Kbar, r->g, r->cb9,
                           red_at(r, dslot + kSlotNorm), bc, r->st);
            prof_end(r, KF_GSUPD, e, Nh * 2 * es * 3 * (k + 2 + 2 + 3));
        }
        double* slot = r->hslot + (size_t)(k % 2) * kSlot;
        CK(r, cudaMemcpyAsync(slot, dslot, kSlotLen * sizeof(double), cudaMemcpyDeviceToHost,
                              r->st));
        r->launches += 3;
        return FFT_OK;
    }

    // Least squares of restarted GMRES over columns 0 .. kc-1 of the host
    // Hessenberg copy (row stride m): Givens QR from scratch (kc <= 31, so
    // this is cheap and lets the last column be replaced by its final value),
    // residual |g_kc| returned; with y, the back substitution.
    static double hess_lsq(const std::vector<double>& Hm, int m, int kc, double beta, double* y) {
        std::vector<double> Rm((size_t)(kc + 1) * kc), g(kc + 1, 0.0), cs(kc), sn(kc);
        for (int i = 0; i <= kc; ++i)
            for (int c = 0; c < kc; ++c) Rm[(size_t)i * kc + c] = Hm[(size_t)i * m + c];
        g[0] = beta;
        for (int c = 0; c < kc; ++c) {
            for (int i = 0; i < c; ++i) {
                const double a = Rm[(size_t)i * kc + c], b = Rm[(size_t)(i + 1) * kc + c];
                Rm[(size_t)i * kc + c] = cs[i] * a + sn[i] * b;
                Rm[(size_t)(i + 1) * kc + c] = -sn[i] * a + cs[i] * b;
            }
            const double a = Rm[(size_t)c * kc + c], b = Rm[(size_t)(c + 1) * kc + c];
            const double den = std::hypot(a, b);
            cs[c] = den > 0 ? a / den : 1.0;
            sn[c] = den > 0 ? b / den : 0.0;
            Rm[(size_t)c * kc + c] = den;
            Rm[(size_t)(c + 1) * kc + c] = 0.0;
            g[c + 1] = -sn[c] * g[c];
            g[c] = cs[c] * g[c];
        }
        if (y)
            for (int i = kc - 1; i >= 0; --i) {
                double s = g[i];
                for (int j = i + 1; j < kc; ++j) s -= Rm[(size_t)i * kc + j] * y[j];
                y[i] = Rm[(size_t)i * kc + i] != 0.0 ? s / Rm[(size_t)i * kc + i] : 0.0;
            }
        return std::fabs(g[kc]);
    }

    // Restarted GMRES, right-preconditioned by the Green operator, with the
    // DCGS2 Arnoldi step above (two passes over the basis per step);
    // Hermitian-weighted FP64 dot products.  The host solves the Hessenberg
    // least squares one step behind the GPU (step j runs while the results
    // of step j - 1 are processed, so the device never waits for the host;
    // the step after convergence is discarded).  After step k the columns
    // 0 .. k-1 are final and column k is provisional: its reorthogonalisation
    // correction arrives with step k + 1 and is of the order of the FP
    // rounding of the first projection.
    static fft_status gmres(fft_rve_s* r, double bn, double pn, int* its) {
        NvtxRange nvtx_("gmres");
        const size_t Nh = r->g.Nh, n3 = 3 * Nh;
        const double es = (double)sizeof(R);
        // round-off floor relative to the scale of the terms summed into b
        const double eta = sizeof(R) == 8 ? 1e-12 : 5e-7;
        const double target = std::max(r->opt.tol_lin * bn, eta * pn);
        CK(r, cudaMemsetAsync(r->x, 0, n3 * sizeof(Cx), r->st));
        *its = 0;
        if (bn <= target) return FFT_OK;
        const int m = std::max(1, std::min(r->opt.restart, kMaxKrylov - 1));
        const size_t vs = n3;  // stride between Krylov vectors (elements)
        Cx* V = (Cx*)r->V;
        std::vector<double> Hm((size_t)(m + 1) * m), y(m);
        bool first = true, ok = false;
        int lin = 0;
        while (lin < r->opt.max_lin && !ok) {
            double beta;
            const void* src = r->b;
            if (first) {
                beta = bn;
            } else {
                TRY(apply_op(r, r->x, 1.0, nullptr, 0, r->w, 0));
                axpby<R>(r->w, r->b, r->w, 1.0, -1.0, n3, r->st);
                norm2<R>(r->w, r->g, red_at(r, r->red), r->st);
                r->launches += 2;
                TRY(fetch(r, 1));
                beta = std::sqrt(r->hred[0]);
                if (r->verbose)
                    std::fprintf(stderr, "  gmres restart: true |r|/|b| %.3e\n", beta / bn);
                if (beta <= target) {
                    ok = true;
                    break;
                }
                src = r->w;
            }
            first = false;
            std::fill(Hm.begin(), Hm.end(), 0.0);
            int kcols = 0;
            // residual estimates of the last two processed steps: when the
            // next one is predicted to converge (geometric extrapolation),
            // the following step is enqueued only after it has been read,
            // instead of ahead of it (it would be discarded)
            double res1 = -1.0, res2 = -1.0;
            for (int j = 0;; ++j) {
                const bool enq = j < m && lin + j < r->opt.max_lin;
                const bool defer = enq && j >= 2 && res2 > 0.0 && res1 > 0.0 &&
                                   res1 * (res1 / res2) <= target;
                if (enq && !defer) TRY(enqueue_step(r, j, src, 1.0 / beta));
                if (j == 0) {
                    if (!enq) break;
                    continue;
                }
                // results of step k = j - 1
                const int k = j - 1;
                CK(r, host_wait(r, r->slot_ev[k % 2]));
                prof_collect_if_done(r);
                const double* slot = r->hslot + (size_t)(k % 2) * kSlot;
                if (slot[kSlotErr] != 0.0)
                    FAIL(r, FFT_ERR_CUDA, "a bulk-copy wait in the Arnoldi step timed out");
                for (int i = 0; i < kSlotLen; ++i)
                    if (!std::isfinite(slot[i]))
                        FAIL(r, FFT_ERR_NONFINITE, "non-finite Krylov coefficient (step %d)",
                             lin + 1);
                if (k >= 1)
                    for (int l = 0; l <= k; ++l) Hm[(size_t)l * m + k - 1] = slot[l];
                for (int l = 0; l <= k; ++l) Hm[(size_t)l * m + k] = slot[kSlotProv + l];
                const double hn = std::sqrt(std::max(slot[kSlotNorm], 0.0));
                Hm[(size_t)(k + 1) * m + k] = hn;
                ++lin;
                kcols = k + 1;
                if (k >= 1 && slot[kSlotNu] == 0.0) {
                    // c_k lay in the span of q_0 .. q_{k-1}: column k - 1 is exact
                    kcols = k;
                    ok = true;
                    break;
                }
                const double res = hess_lsq(Hm, m, kcols, beta, nullptr);
                if (r->verbose)
                    std::fprintf(stderr,
                                 "  gmres it %d |r|/|b| %.3e (|b| %.3e, h %.3e, nu %.3e, "
                                 "|a|/|c| %.3e)\n",
                                 lin, res / bn, bn, hn, slot[kSlotNu],
                                 std::sqrt(std::max(slot[kSlotA2], 0.0) /
                                           std::max(slot[kSlotAlpha], 1e-300)));
                if (res <= target || hn == 0.0) {
                    ok = true;
                    break;
                }
                if (!enq) break;
                if (defer) TRY(enqueue_step(r, j, src, 1.0 / beta));
                res2 = res1;
                res1 = res;
            }
            const int k = kcols;
            hess_lsq(Hm, m, k, beta, y.data());
            CK(r, host_wait(r));  // a discarded look-ahead step, hy reuse
            prof_collect(r);
            if (k > 0) {
                std::memcpy(r->hy, y.data(), k * sizeof(double));
                CK(r, cudaMemcpyAsync(r->dy, r->hy, k * sizeof(double), cudaMemcpyHostToDevice,
                                      r->st));
                cudaEvent_t e = prof_begin(r, KF_XUPD);
                xupdate<R>(r->x, V, vs, k, r->dy, r->Kbar, r->g, r->st);
                prof_end(r, KF_XUPD, e, (double)Nh * 2 * es * 3 * (k + 2));
                r->launches += 1;
                CK(r, host_wait(r));  // hy is reused by the next fetch
                prof_collect(r);
            }
        }
        *its = lin;
        CK(r, cudaGetLastError());
        if (r->use_bulk) {
            int e = 0;
            CK(r, cudaMemcpy(&e, r->bulk.err, sizeof(int), cudaMemcpyDeviceToHost));
            if (e) FAIL(r, FFT_ERR_CUDA, "a bulk-copy wait in the Arnoldi step timed out");
        }
        if (!ok) FAIL(r, FFT_ERR_NOT_CONVERGED, "GMRES reached max_lin = %d", r->opt.max_lin);
        return FFT_OK;
    }

    static fft_status solve_equilibrium(fft_rve_s* r, fft_stats* st) {
        NvtxRange nvtx_("equilibrium");
        if (r->state != ST_APPLIED && r->state != ST_DAMAGE)
            FAIL(r, FFT_ERR_STATE, "solve_equilibrium before apply_increment");
        const size_t N = r->g.N;
        CK(r, cudaMemcpyAsync(r->Hprev, r->H, 9 * N * sizeof(R), cudaMemcpyDeviceToDevice, r->st));
        r->skipped = false;
        r->state = ST_EQUIL;
        if (r->stag_it >= 1 && !r->phi_changed) {
            r->skipped = true;
            if (st) st->skipped_equilibrium = 1;
            return FFT_OK;
        }
        for (int outer = 0;; ++outer) {
            TRY(newton_solve(r, st));
            if (!r->mixed) return FFT_OK;
            bool done = false;
            TRY(mixed_step(r, st, outer, &done));
            if (done) return FFT_OK;
        }
    }

    // Mixed control, one outer round after a converged Newton solve: the
    // mean degraded stress <gP> and Kbar = <gK> at the current F, then
    // Kbar_SS dF_S = -(<gP> - P*)_S on the stress-controlled components S
    // (solved on the host) and dF added uniformly to F.  done when
    // max_S |<gP> - P*| <= tol_newton max(max|<gP>|, 1 MPa).
    static fft_status mixed_step(fft_rve_s* r, fft_stats* st, int outer, bool* done) {
        NvtxRange nvtx_("mixed_control");
        const size_t N = r->g.N;
        int nf = 0;
        TRY(cp(r, false, &nf));
        if (st) st->local_fail += nf;
        kbar<R>(r->K, r->phi, r->mat.k_res, N, red_at(r, r->Kbar), r->st);
        stag_stats<R>(r->H, r->Hprev, r->Ht, r->P, r->phi, r->mat.k_res, N, red_at(r, r->red),
                      r->st);
        r->launches += 2;
        CK(r, cudaMemcpyAsync(r->hred + 16, r->Kbar, 81 * sizeof(double),
                              cudaMemcpyDeviceToHost, r->st));
        TRY(fetch(r, 11));
        const double* Pb = r->hred + 2;  // <gP>, from the statistics kernel
        const double* Kb = r->hred + 16;
        for (int c = 0; c < 81; ++c)
            if (!std::isfinite(Kb[c]))
                FAIL(r, FFT_ERR_NONFINITE,
                     "mixed control: non-finite averaged tangent entry %d (Kbar = <g K>)", c);
        double pmax = 0, res = 0;
        int S[9], ns = 0;
        for (int c = 0; c < 9; ++c) {
            pmax = std::max(pmax, std::fabs(Pb[c]));
            if (r->mask[c]) {
                S[ns++] = c;
                res = std::max(res, std::fabs(Pb[c] - r->Pstar[c]));
            }
        }
        if (st) st->mixed_it = outer + 1;
        if (r->verbose)
            std::fprintf(stderr, "  mixed %d |<gP> - P*|_S %.3e (max|<gP>| %.3e)\n", outer, res,
                         pmax);
        if (res <= r->opt.tol_newton * std::max(pmax, 1.0)) {
            *done = true;
            return FFT_OK;
        }
        if (outer + 1 >= r->opt.max_newton)
            FAIL(r, FFT_ERR_NOT_CONVERGED, "mixed control reached max_newton = %d rounds",
                 r->opt.max_newton);
        // Gauss-Jordan with partial pivoting on [Kbar_SS | -(<gP> - P*)_S]
        double A[9][10];
        for (int a = 0; a < ns; ++a) {
            for (int b = 0; b < ns; ++b) A[a][b] = Kb[9 * S[a] + S[b]];
            A[a][ns] = r->Pstar[S[a]] - Pb[S[a]];
        }
        for (int c = 0; c < ns; ++c) {
            int p = c;
            for (int a = c + 1; a < ns; ++a)
                if (std::fabs(A[a][c]) > std::fabs(A[p][c])) p = a;
            if (!(std::fabs(A[p][c]) > 0))
                FAIL(r, FFT_ERR_NONFINITE, "mixed control: singular averaged tangent block");
            if (p != c)
                for (int b = 0; b <= ns; ++b) std::swap(A[c][b], A[p][b]);
            for (int a = 0; a < ns; ++a) {
                if (a == c) continue;
                const double m = A[a][c] / A[c][c];
                for (int b = c; b <= ns; ++b) A[a][b] -= m * A[c][b];
            }
        }
        double d[9] = {0};
        for (int a = 0; a < ns; ++a) {
            d[S[a]] = A[a][ns] / A[a][a];
            r->Fbar[S[a]] += d[S[a]];
        }
        add_uniform<R>(r->H, r->H, d, N, r->st);
        r->launches += 1;
        r->cp_valid = false;
        return FFT_OK;
    }

    // Newton iteration on the fluctuation at the current macroscopic F
    // (Eq. newton with GMRES, Sec. 3.1).  Damping (an extension; the paper's
    // Newton takes full steps): from the kDampFrom-th iteration on, an update
    // after which the ratio of the Newton test did not fall halves the length
    // of the next (down to 1/16); one that halved the ratio doubles it back
    // (up to a full step).  This breaks the two-cycles a kink in the slip
    // law's tangent can trap Newton in; an iteration whose ratio keeps
    // falling is untouched.  The test itself uses the full correction.
    static constexpr int kDampFrom = 4;
    static fft_status newton_solve(fft_rve_s* r, fft_stats* st) {
        const size_t N = r->g.N;
        double alpha = 1.0, prev_ratio = 0.0;
        for (int it = 0; it < r->opt.max_newton; ++it) {
            if (!r->cp_valid) {
                int nf = 0;
                TRY(cp(r, false, &nf));
                if (st) st->local_fail += nf;
            }
            if (st) st->newton_it += 1;
            cudaEvent_t e = prof_begin(r, KF_KBAR);
            kbar<R>(r->K, r->phi, r->mat.k_res, N, red_at(r, r->Kbar), r->st);
            prof_end(r, KF_KBAR, e, (double)N * sizeof(R) * 82);
            e = prof_begin(r, KF_RESID);
            degrade<R>(r->P, r->phi, r->mat.k_res, r->rb9, N, r->st);
            prof_end(r, KF_RESID, e, (double)N * sizeof(R) * 19);
            TRY(fwd9(r));
            e = prof_begin(r, KF_RESID);
            residual<R>(r->cb9, r->g, r->b, red_at(r, r->red), r->st);
            prof_end(r, KF_RESID, e, (double)r->g.Nh * 2 * sizeof(R) * 12);
            r->launches += 3;
            TRY(fetch(r, 2));
            const double bn = std::sqrt(r->hred[0]), pn = std::sqrt(r->hred[1]);
            int lin = 0;
            const fft_status s = gmres(r, bn, pn, &lin);
            if (st) st->lin_it_total += lin;
            if (s != FFT_OK) return s;
            e = prof_begin(r, KF_PRECOND);
            precond_grad<R>(r->x, alpha, nullptr, r->Kbar, r->g, r->cb9, 0, r->st);
            prof_end(r, KF_PRECOND, e, (double)r->g.Nh * 2 * sizeof(R) * 12);
            TRY(inv9(r));
            e = prof_begin(r, KF_FUPD);
            fupdate<R>(r->H, r->rb9, r->Ht, N, red_at(r, r->red), r->st);
            prof_end(r, KF_FUPD, e, (double)N * sizeof(R) * 36);
            r->launches += 2;
            TRY(fetch(r, 2));
            r->cp_valid = false;
            // the applied update is alpha grad(du) (alpha a power of two)
            const double gmax = r->hred[0] / alpha, dFt = std::max(r->hred[1], 1e-30);
            const double ratio = gmax / dFt;
            if (r->verbose)
                std::fprintf(stderr,
                             "newton %d |b| %.3e |Phat| %.3e lin %d gmax %.3e ratio %.3e alpha %.4f\n",
                             it, bn, pn, lin, gmax, ratio, alpha);
            if (ratio < r->opt.tol_newton) return FFT_OK;
            if (it + 1 >= kDampFrom && ratio >= prev_ratio)
                alpha = std::max(0.5 * alpha, 1.0 / 16);
            else if (ratio < 0.5 * prev_ratio)
                alpha = std::min(2.0 * alpha, 1.0);
            prev_ratio = ratio;
        }
        FAIL(r, FFT_ERR_NOT_CONVERGED, "Newton reached max_newton = %d", r->opt.max_newton);
    }

    // PCG on (1 + 2S) phi - ell^2 lap phi = 2S with M_phi, x0 = current phi;
    // A p through the recurrence t = M^-1 p = r + beta t (one transform pair
    // per iteration).  Result in pfx (unclamped).
    static fft_status pcg_phase(fft_rve_s* r, int* iters) {
        const size_t N = r->g.N;
        const double l2 = r->mat.ell * r->mat.ell;
        // algorithmic bytes: a real field, a half-spectrum scalar field
        const double fb = (double)N * sizeof(R), sb = (double)r->g.Nh * 2 * sizeof(R);
        *iters = 0;
        CK(r, cudaMemcpyAsync(r->pfx, r->phi, N * sizeof(R), cudaMemcpyDeviceToDevice, r->st));
        TRY(fwd1(r, r->pfx));
        cudaEvent_t e = prof_begin(r, KF_PF);
        pf_spec<R>(r->cb9, r->g, l2, 0, r->st);
        prof_end(r, KF_PF, e, 2 * sb);
        TRY(inv1(r, r->pfq));
        e = prof_begin(r, KF_PF);
        pf_init<R>(r->pfx, r->pfq, r->drive, r->pfr, N, red_at(r, r->red), r->st);
        prof_end(r, KF_PF, e, 4 * fb);
        r->launches += 2;
        TRY(fetch(r, 2));
        const double bn = std::sqrt(r->hred[1]);
        if (std::sqrt(r->hred[0]) <= r->opt.tol_pf * bn) return FFT_OK;
        auto precond = [&]() -> fft_status {
            TRY(fwd1(r, r->pfr));
            cudaEvent_t e1 = prof_begin(r, KF_PF);
            pf_spec<R>(r->cb9, r->g, l2, 1, r->st);
            prof_end(r, KF_PF, e1, 2 * sb);
            TRY(inv1(r, r->pfz));
            e1 = prof_begin(r, KF_PF);
            rdot<R>(r->pfr, r->pfz, N, red_at(r, r->red), r->st);
            prof_end(r, KF_PF, e1, 2 * fb);
            r->launches += 2;
            return fetch(r, 1);
        };
        TRY(precond());
        double rz = r->hred[0];
        CK(r, cudaMemcpyAsync(r->pfp, r->pfz, N * sizeof(R), cudaMemcpyDeviceToDevice, r->st));
        CK(r, cudaMemcpyAsync(r->pft, r->pfr, N * sizeof(R), cudaMemcpyDeviceToDevice, r->st));
        for (int it = 1; it <= r->opt.max_pf; ++it) {
            *iters = it;
            e = prof_begin(r, KF_PF);
            pf_q<R>(r->pft, r->pfp, r->drive, r->pfq, N, red_at(r, r->red), r->st);
            prof_end(r, KF_PF, e, 4 * fb);
            TRY(fetch(r, 1));
            const double alpha = rz / r->hred[0];
            e = prof_begin(r, KF_PF);
            pf_xr<R>(r->pfx, r->pfr, r->pfp, r->pfq, alpha, N, red_at(r, r->red), r->st);
            prof_end(r, KF_PF, e, 6 * fb);
            r->launches += 2;
            TRY(fetch(r, 1));
            if (std::sqrt(r->hred[0]) <= r->opt.tol_pf * bn) return FFT_OK;
            TRY(precond());
            const double beta = r->hred[0] / rz;
            rz = r->hred[0];
            e = prof_begin(r, KF_PF);
            pf_pt<R>(r->pfp, r->pft, r->pfz, r->pfr, beta, N, r->st);
            prof_end(r, KF_PF, e, 6 * fb);
            r->launches += 1;
        }
        FAIL(r, FFT_ERR_NOT_CONVERGED, "phase-field CG reached max_pf = %d", r->opt.max_pf);
    }

    // phase-field solve (or phi = phi_t when S = 0 everywhere) and clamp;
    // out: max|phi_new - phi_old|, max|phi_new - phi_t|, changed, cracked.
    static fft_status phase_field(fft_rve_s* r, int* iters, double* out4) {
        NvtxRange nvtx_("phase_field");
        const size_t N = r->g.N;
        maxval<R>(r->drive, N, red_at(r, r->red), r->st);
        r->launches += 1;
        TRY(fetch(r, 1));
        *iters = 0;
        if (r->hred[0] == 0.0) {
            CK(r, cudaMemcpyAsync(r->pfx, r->phi_t, N * sizeof(R), cudaMemcpyDeviceToDevice, r->st));
        } else {
            TRY(pcg_phase(r, iters));
        }
        cudaEvent_t e = prof_begin(r, KF_PF);
        pf_clamp<R>(r->pfx, r->phi_t, r->phi, N, red_at(r, r->red), r->st);
        prof_end(r, KF_PF, e, 4.0 * N * sizeof(R));
        r->launches += 1;
        TRY(fetch(r, 4));
        for (int i = 0; i < 4; ++i) out4[i] = r->hred[i];
        return FFT_OK;
    }

    static fft_status update_damage(fft_rve_s* r, fft_stats* st) {
        NvtxRange nvtx_("damage");
        if (r->state != ST_EQUIL) FAIL(r, FFT_ERR_STATE, "update_damage before solve_equilibrium");
        const size_t N = r->g.N;
        r->stag_it += 1;
        r->state = ST_DAMAGE;
        if (st) st->stag_it = r->stag_it;
        if (r->skipped) {
            r->converged = true;
            if (st) {
                st->res_F = st->res_phi = 0;
                st->converged = 1;
            }
            return FFT_OK;
        }
        int nf = 0;
        TRY(cp(r, true, &nf));
        if (st) st->local_fail += nf;
        int pf_it = 0;
        double o4[4];
        TRY(phase_field(r, &pf_it, o4));
        if (st) st->pf_it_total += pf_it;
        stag_stats<R>(r->H, r->Hprev, r->Ht, r->P, r->phi, r->mat.k_res, N, red_at(r, r->red),
                      r->st);
        r->launches += 1;
        TRY(fetch(r, 11));
        const double dF = r->hred[0], dFt = r->hred[1];
        const double dphi = o4[0], dphit = o4[1];
        r->phi_changed = o4[2] > 0;
        const double tol = r->opt.tol_stag;
        // the phase-field ratio of Algorithm 1 is 0/0 when phi does not
        // change over the increment; its denominator is kept above the
        // resolution of phi in the bulk type (100 eps: 1.2e-5 in FP32, the
        // 1e-12 floor in FP64), below which the iterations' changes are
        // round-off of the phase-field solve
        const double phi_floor = std::max(1e-12, 100.0 * Tr<R>::eps);
        r->converged =
            dF <= tol * std::max(dFt, 1e-12) && dphi <= tol * std::max(dphit, phi_floor);
        for (int c = 0; c < 9; ++c) r->Pbar_cur[c] = r->hred[2 + c];
        if (st) {
            st->res_F = dF / std::max(dFt, 1e-12);
            st->res_phi = dphi / std::max(dphit, phi_floor);
            st->converged = r->converged;
            for (int c = 0; c < 9; ++c) st->Pbar[c] = r->hred[2 + c];
            st->cracked = (long)o4[3];
            std::memcpy(st->Fbar, r->Fbar, sizeof(r->Fbar));
        }
        return FFT_OK;
    }

    static fft_status apply_increment_mixed(fft_rve_s* r, const double* Fbar,
                                            const double* Pstar, const int32_t* mask,
                                            double dt) {
        TRY(apply_increment(r, Fbar, dt));
        int ns = 0;
        for (int c = 0; c < 9; ++c) {
            r->mask[c] = mask[c] ? 1 : 0;
            r->Pstar[c] = Pstar ? Pstar[c] : 0.0;
            ns += r->mask[c];
        }
        r->mixed = ns > 0;
        return FFT_OK;
    }

    static fft_status apply_increment(fft_rve_s* r, const double* Fbar, double dt) {
        NvtxRange nvtx_("apply_increment");
        if (r->state == ST_DAMAGE && r->converged) TRY(commit(r));
        r->mixed = false;
        double d[9];
        for (int c = 0; c < 9; ++c) {
            d[c] = Fbar[c] - r->Fbar_t[c];
            r->Fbar[c] = Fbar[c];
        }
        const size_t N = r->g.N;
        add_uniform<R>(r->H, r->Ht, d, N, r->st);
        r->launches += 1;
        CK(r, cudaMemcpyAsync(r->phi, r->phi_t, N * sizeof(R), cudaMemcpyDeviceToDevice, r->st));
        r->dt = dt;
        TRY(gnd(r));
        r->stag_it = 0;
        r->phi_changed = true;
        r->converged = false;
        r->cp_valid = false;
        r->state = ST_APPLIED;
        return FFT_OK;
    }

    static fft_status commit(fft_rve_s* r) {
        NvtxRange nvtx_("commit");
        if (r->state != ST_DAMAGE || !r->converged)
            FAIL(r, FFT_ERR_STATE, "commit without a converged increment");
        const size_t N = r->g.N;
        std::swap(r->hist_c, r->hist_tr);
        std::swap(r->Hpi_t, r->Hpi_tr);
        CK(r, cudaMemcpyAsync(r->Ht, r->H, 9 * N * sizeof(R), cudaMemcpyDeviceToDevice, r->st));
        CK(r, cudaMemcpyAsync(r->phi_t, r->phi, N * sizeof(R), cudaMemcpyDeviceToDevice, r->st));
        std::memcpy(r->Fbar_t, r->Fbar, sizeof(r->Fbar));
        for (int c = 0; c < 9; ++c)
            r->Pbar_t[c] = (r->mixed && r->mask[c]) ? r->Pstar[c] : r->Pbar_cur[c];
        r->state = ST_COMMITTED;
        r->cp_valid = false;
        return FFT_OK;
    }

    // Algorithm 1 for one increment, committed when converged; mask = nullptr
    // is strain control, otherwise the mixed control of apply_increment_mixed.
    static fft_status run_once(fft_rve_s* r, const double* Fbar, const double* Pstar,
                               const int32_t* mask, double dt, fft_stats* st) {
        if (mask)
            TRY(apply_increment_mixed(r, Fbar, Pstar, mask, dt));
        else
            TRY(apply_increment(r, Fbar, dt));
        return stag_loop(r, st);
    }
    static fft_status stag_loop(fft_rve_s* r, fft_stats* st) {
        for (int i = 0; i < r->opt.max_stag; ++i) {
            TRY(solve_equilibrium(r, st));
            TRY(update_damage(r, st));
            if (r->converged) return commit(r);
        }
        FAIL(r, FFT_ERR_NOT_CONVERGED, "staggered loop reached max_stag = %d", r->opt.max_stag);
    }

    // The increment as two halves from the committed state (a failed
    // attempt leaves it untouched: apply_increment restarts from F_t, phi_t
    // and the committed history), each halved again on failure down to
    // depth max_cutbacks.  Each half takes half of the load change: the
    // first goes to the midpoint of the committed and the requested
    // macroscopic F and, on stress-controlled components, to the midpoint
    // of the committed and the requested stress; the second to the request,
    // its stress-controlled components of F started from the solved
    // midpoint.
    static fft_status run_halves(fft_rve_s* r, const double* Fbar, const double* Pstar,
                                 const int32_t* mask, double dt, fft_stats* st, int depth) {
        if (st) st->cutbacks += 1;
        double tgt[2][9], Ptgt[2][9];
        for (int c = 0; c < 9; ++c) {
            tgt[0][c] = 0.5 * (r->Fbar_t[c] + Fbar[c]);
            Ptgt[1][c] = Pstar ? Pstar[c] : 0.0;
            Ptgt[0][c] = (mask && mask[c]) ? 0.5 * (r->Pbar_t[c] + Ptgt[1][c]) : Ptgt[1][c];
        }
        for (int h = 0; h < 2; ++h) {
            if (h == 1)
                for (int c = 0; c < 9; ++c) tgt[1][c] = (mask && mask[c]) ? r->Fbar_t[c] : Fbar[c];
            fft_status s = run_once(r, tgt[h], Ptgt[h], mask, 0.5 * dt, st);
            if (s == FFT_ERR_NOT_CONVERGED && depth < r->opt.max_cutbacks)
                s = run_halves(r, tgt[h], Ptgt[h], mask, 0.5 * dt, st, depth + 1);
            if (s != FFT_OK) return s;
        }
        return FFT_OK;
    }

    static fft_status run_increment(fft_rve_s* r, const double* Fbar, const double* Pstar,
                                    const int32_t* mask, double dt, fft_stats* st) {
        const fft_status s = run_once(r, Fbar, Pstar, mask, dt, st);
        if (s != FFT_ERR_NOT_CONVERGED || r->opt.max_cutbacks <= 0) return s;
        if (r->verbose) std::fprintf(stderr, "  increment not converged: cutting back\n");
        return run_halves(r, Fbar, Pstar, mask, dt, st, 1);
    }

    static fft_status fields_out(fft_rve_s* r, int field, double* d) {
        const size_t N = r->g.N;
        cudaStream_t s = r->st;
        switch (field) {
            case FFT_FIELD_F: to_double<R>(r->H, d, 9 * N, N, 1, s); break;
            case FFT_FIELD_FT: to_double<R>(r->Ht, d, 9 * N, N, 1, s); break;
            case FFT_FIELD_P:
                degrade<R>(r->P, r->phi, r->mat.k_res, r->rb9, N, s);
                to_double<R>(r->rb9, d, 9 * N, N, 0, s);
                break;
            case FFT_FIELD_PU: to_double<R>(r->P, d, 9 * N, N, 0, s); break;
            case FFT_FIELD_K: to_double<R>(r->K, d, 81 * N, N, 0, s); break;
            case FFT_FIELD_PHI: to_double<R>(r->phi, d, N, N, 0, s); break;
            case FFT_FIELD_PHI_T: to_double<R>(r->phi_t, d, N, N, 0, s); break;
            case FFT_FIELD_DRIVE: to_double<R>(r->drive, d, N, N, 0, s); break;
            case FFT_FIELD_WE: to_double<R>(r->We, d, N, N, 0, s); break;
            case FFT_FIELD_RHO_GND: to_double<R>(r->rho_gnd, d, N, N, 0, s); break;
            case FFT_FIELD_FP:
                fp_sample<R>(r->Hpi_t, r->grain, r->Qg, r->rb9, N, s);
                to_double<R>(r->rb9, d, 9 * N, N, 1, s);
                break;
            case FFT_FIELD_RHO_SSD: hist_sum(r->hist_c, HIST_RHO, 1, 1, d, N, s); break;
            case FFT_FIELD_WP: hist_sum(r->hist_c, HIST_WP, 1, 1, d, N, s); break;
            case FFT_FIELD_GS: hist_sum(r->hist_c, HIST_GS, 1, 1, d, N, s); break;
            case FFT_FIELD_HMAX: hist_sum(r->hist_c, HIST_HMAX, 0, 1, d, N, s); break;
            case FFT_FIELD_WCRIT: hist_sum(r->hist_c, HIST_WCRIT, 0, 1, d, N, s); break;
            case FFT_FIELD_GAMMA: hist_sum(r->hist_c, HIST_GAMMA, 1, 12, d, N, s); break;
            default: FAIL(r, FFT_ERR_ARG, "unknown field %d", field);
        }
        r->launches += 1;
        CK(r, cudaGetLastError());
        return FFT_OK;
    }

    static fft_status fields_in(fft_rve_s* r, int field, const double* d) {
        const size_t N = r->g.N;
        cudaStream_t s = r->st;
        switch (field) {
            case FFT_FIELD_F: from_double<R>(d, r->H, 9 * N, N, 1, s); break;
            case FFT_FIELD_FT: from_double<R>(d, r->Ht, 9 * N, N, 1, s); break;
            case FFT_FIELD_PHI: from_double<R>(d, r->phi, N, N, 0, s); break;
            case FFT_FIELD_PHI_T: from_double<R>(d, r->phi_t, N, N, 0, s); break;
            case FFT_FIELD_FP: fp_in<R>(d, r->grain, r->Qg, r->Hpi_t, N, s); break;
            case FFT_FIELD_RHO_SSD: hist_set(r->hist_c, HIST_RHO, 1, 1, d, N, s); break;
            case FFT_FIELD_WP: hist_set(r->hist_c, HIST_WP, 1, 1, d, N, s); break;
            case FFT_FIELD_GS: hist_set(r->hist_c, HIST_GS, 1, 1, d, N, s); break;
            case FFT_FIELD_HMAX: hist_set(r->hist_c, HIST_HMAX, 0, 1, d, N, s); break;
            case FFT_FIELD_WCRIT: hist_set(r->hist_c, HIST_WCRIT, 0, 1, d, N, s); break;
            case FFT_FIELD_GAMMA: hist_set(r->hist_c, HIST_GAMMA, 1, 12, d, N, s); break;
            case FFT_FIELD_DRIVE: from_double<R>(d, r->drive, N, N, 0, s); break;
            default: FAIL(r, FFT_ERR_ARG, "field %d cannot be set", field);
        }
        r->launches += 1;
        r->cp_valid = false;
        CK(r, cudaGetLastError());
        return FFT_OK;
    }

    static fft_status init_state(fft_rve_s* r, const double* phi0) {
        const size_t N = r->g.N;
        cudaStream_t s = r->st;
        for (void* p : {r->H, r->Ht, r->Hprev, r->Hpi_t, r->Hpi_tr})
            CK(r, cudaMemsetAsync(p, 0, 9 * N * sizeof(R), s));
        for (void* p : {r->P, r->rb9}) CK(r, cudaMemsetAsync(p, 0, 9 * N * sizeof(R), s));
        CK(r, cudaMemsetAsync(r->K, 0, 81 * N * sizeof(R), s));
        for (void* p : {r->rho_gnd, r->phi, r->phi_t, r->drive, r->We})
            CK(r, cudaMemsetAsync(p, 0, N * sizeof(R), s));
        CK(r, cudaMemsetAsync(r->hist_c, 0, HIST_SLOTS * N * sizeof(double), s));
        CK(r, cudaMemsetAsync(r->hist_tr, 0, HIST_SLOTS * N * sizeof(double), s));
        std::vector<double> rho(N, r->mat.rho_ssd0);
        double* tmp = nullptr;
        CK(r, cudaMalloc(&tmp, N * sizeof(double)));
        cudaMemcpyAsync(tmp, rho.data(), N * sizeof(double), cudaMemcpyHostToDevice, s);
        hist_set(r->hist_c, HIST_RHO, 1, 1, tmp, N, s);
        hist_set(r->hist_tr, HIST_RHO, 1, 1, tmp, N, s);
        if (phi0) {
            cudaMemcpyAsync(tmp, phi0, N * sizeof(double), cudaMemcpyHostToDevice, s);
            from_double<R>(tmp, r->phi_t, N, N, 0, s);
            from_double<R>(tmp, r->phi, N, N, 0, s);
        }
        cudaStreamSynchronize(s);
        cudaFree(tmp);
        CK(r, cudaGetLastError());
        return FFT_OK;
    }
};

}  // namespace
