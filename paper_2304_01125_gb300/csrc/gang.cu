// Lockstep class driver: the RVEs of one size class (same grid, precision
// and solver options) advanced through the load increment of Algorithm 1
// together, so that the Arnoldi steps of all of them are one graph launch.
//
// Each member keeps its handle, stream, state and per-member kernels.  The
// class owns the 9-field scratch of the Arnoldi step for all members in one
// arena (member i at offset i x 9N real / 9Nh complex), so that one batched
// library transform per direction (a plan over 9 B fields) serves the whole
// class, and one CUDA graph per Krylov column j: the batched inverse
// transform, the members' tangent applies as parallel branches, the batched
// forward transform, then per member the contraction with its dot pass, the
// Gram-Schmidt update and the copy of its step coefficients to the host.
// The Newton and GMRES loops run in lockstep over the members still
// iterating: a member that has converged leaves the loop, and a device flag
// makes its step kernels in the remaining columns of the cycle return at
// once; once fewer than half the members iterate, the rest of the cycle runs
// their own step graphs instead (the batched transforms would mostly
// transform idle members).  The per-member
// arithmetic is that of the single-handle driver step for step; only the
// order in which the host reads the results differs.  The staggered loop's
// damage updates run per member; a member whose increment does not converge
// is cut back on its own, by the single-handle driver.  The per-member host
// work (enqueueing a member's stages, waiting for and reading its results)
// is spread over a few helper threads of the class.
#include <atomic>
#include <condition_variable>
#include <functional>
#include <mutex>

#include "rve_impl.cuh"

namespace {

constexpr int kGangMax = 64;
// Sparse mode (see the GMRES cycle) starts once kSparse x (members still
// iterating) < members; 0 never starts it.
#ifndef FATIGUEFFT_SPARSE_FACTOR
#define FATIGUEFFT_SPARSE_FACTOR 2
#endif
constexpr int kSparse = FATIGUEFFT_SPARSE_FACTOR;
constexpr int kGangHelpers = 7;  // host threads besides the caller per class

// Fork-join helper threads of a class: run(n, f) calls f(0) .. f(n-1), the
// items taken in order by the caller and the helpers, and returns when all
// are done.  The members' per-member host work (enqueueing their stages,
// waiting for and reading their results) is independent from member to
// member, so that one host thread does not serialise it for the class.
struct ParFor {
    std::vector<std::thread> th;
    std::mutex m;
    std::condition_variable cv, cv_done;
    std::function<void(int)> fn;
    std::atomic<int> next{0};
    int n = 0, busy = 0;
    long long gen = 0;
    bool quit = false;

    void start(int helpers, int dev) {
        for (int t = 0; t < helpers; ++t)
            th.emplace_back([this, dev] {
                cudaSetDevice(dev);
                long long seen = 0;
                std::unique_lock<std::mutex> lk(m);
                for (;;) {
                    cv.wait(lk, [&] { return quit || gen != seen; });
                    if (quit) return;
                    seen = gen;
                    lk.unlock();
                    work();
                    lk.lock();
                    if (--busy == 0) cv_done.notify_all();
                }
            });
    }
    void work() {
        for (;;) {
            const int i = next.fetch_add(1);
            if (i >= n) return;
            fn(i);
        }
    }
    void run(int count, const std::function<void(int)>& f) {
        if (th.empty() || count <= 1) {
            for (int i = 0; i < count; ++i) f(i);
            return;
        }
        {
            std::lock_guard<std::mutex> lk(m);
            fn = f;
            n = count;
            next = 0;
            busy = (int)th.size();
            ++gen;
        }
        cv.notify_all();
        work();
        std::unique_lock<std::mutex> lk(m);
        cv_done.wait(lk, [&] { return busy == 0; });
    }
    void stop() {
        {
            std::lock_guard<std::mutex> lk(m);
            quit = true;
        }
        cv.notify_all();
        for (auto& t : th) t.join();
        th.clear();
    }
};

struct GangBase {
    std::vector<fft_rve_s*> m;
    int B = 0;
    cudaStream_t st = nullptr;
    cufftHandle r2c = 0, c2r = 0;
    bool plans = false;
    void *rb9 = nullptr, *cb9 = nullptr;
    // per member: nonzero while it iterates in the current GMRES cycle (its
    // step kernels return at once otherwise); set by memsets on the class
    // stream, in order with the column graphs
    int* act = nullptr;
    std::vector<void*> rb9_own, cb9_own;  // the members' own scratch, restored at destroy
    // the members' reduction buffers (kRedSlots doubles each) in one arena,
    // so that one strided copy per column brings every member's step
    // coefficients to the host (hslots: 2 x B x kSlot, pinned)
    double* red = nullptr;
    std::vector<double*> red_own;
    double* hslots = nullptr;
    cudaGraphExec_t col[kMaxKrylov] = {};
    cudaEvent_t ev_a = nullptr, slot_ev[2] = {nullptr, nullptr}, done_ev = nullptr;
    std::vector<cudaEvent_t> ev_m;  // per member: fork/join of the column graphs
    long long graph_launches = 0;
    // optional timing of the column graphs (CUDA events on the class
    // stream around each launch) with their algorithmic bytes
    bool timing = false;
    std::vector<cudaEvent_t> tpool;
    std::vector<std::pair<std::pair<cudaEvent_t, cudaEvent_t>, double>> tpend;
    double graph_ms = 0.0, graph_bytes = 0.0;
    ParFor pool;
    std::string err;
};

// f(i) for every member index in idx, spread over the class's host threads
static void for_members(GangBase* g, const std::vector<int>& idx,
                        const std::function<void(int)>& f) {
    g->pool.run((int)idx.size(), [&](int t) { f(idx[t]); });
}

// one host wait on the class stream (polling: the batch's threads may
// outnumber the host cores)
static cudaError_t gang_wait(GangBase* g, cudaEvent_t e) {
    (void)g;
    for (;;) {
        const cudaError_t q = cudaEventQuery(e);
        if (q != cudaErrorNotReady) return q;
        std::this_thread::yield();
    }
}

static cudaEvent_t gang_tevent(GangBase* g) {
    if (!g->tpool.empty()) {
        cudaEvent_t e = g->tpool.back();
        g->tpool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// fold the timed launches in (the class stream is idle)
static void gang_tcollect(GangBase* g) {
    for (auto& p : g->tpend) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.first.first, p.first.second) == cudaSuccess) {
            g->graph_ms += ms;
            g->graph_bytes += p.second;
        }
        g->tpool.push_back(p.first.first);
        g->tpool.push_back(p.first.second);
    }
    g->tpend.clear();
}

template <typename R>
struct Gang {
    typedef typename Tr<R>::Cx Cx;
    typedef Impl<R> I;

    // Arnoldi column k for every member (the body of the single-handle
    // step, non-fused), captured once into a graph on the class stream.
    static fft_status capture_col(GangBase* g, int k) {
        fft_rve_s* r0 = g->m[0];
        const size_t vs = 3 * r0->g.Nh;
        CK(g->m[0], cudaStreamBeginCapture(g->st, cudaStreamCaptureModeThreadLocal));
        bool ok = FFT<R>::inv(g->c2r, g->cb9, g->rb9) == CUFFT_SUCCESS;
        ok = ok && cudaEventRecord(g->ev_a, g->st) == cudaSuccess;
        for (int i = 0; ok && i < g->B; ++i) {
            fft_rve_s* r = g->m[i];
            ok = cudaStreamWaitEvent(r->st, g->ev_a, 0) == cudaSuccess;
            tangent_apply<R>(r->rb9, r->K, r->phi, r->mat.k_res, r->g.N, r->st, g->act + i);
            ok = ok && cudaEventRecord(g->ev_m[i], r->st) == cudaSuccess;
        }
        for (int i = 0; ok && i < g->B; ++i)
            ok = cudaStreamWaitEvent(g->st, g->ev_m[i], 0) == cudaSuccess;
        ok = ok && FFT<R>::fwd(g->r2c, g->rb9, g->cb9) == CUFFT_SUCCESS;
        ok = ok && cudaEventRecord(g->ev_a, g->st) == cudaSuccess;
        for (int i = 0; ok && i < g->B; ++i) {
            fft_rve_s* r = g->m[i];
            Cx* V = (Cx*)r->V;
            double* dslot = r->red + kDslot;
            double* Hp = r->Hd + (size_t)kMaxKrylov * kHcol;
            double* coef = Hp + (size_t)kMaxKrylov * kHcol;
            const BulkCfg* bc = r->use_bulk ? &r->bulk : nullptr;
            ok = cudaStreamWaitEvent(r->st, g->ev_a, 0) == cudaSuccess;
            contract_dots<R>(r->cb9, r->g, r->w, V + (size_t)k * vs, V, vs, k,
                             red_at(r, r->red), r->Hd, Hp, dslot, coef, bc, r->st, 0,
                             r->dot64 ? 1 : 0, g->act + i);
            dcgs_update<R>(V, vs, k, r->w, coef, r->Kbar, r->g, r->cb9,
                           red_at(r, dslot + kSlotNorm), bc, r->st, 0, g->act + i);
            ok = ok && cudaEventRecord(g->ev_m[i], r->st) == cudaSuccess;
        }
        for (int i = 0; ok && i < g->B; ++i)
            ok = cudaStreamWaitEvent(g->st, g->ev_m[i], 0) == cudaSuccess;
        // every member's step coefficients in one copy
        ok = ok && cudaMemcpy2DAsync(g->hslots + (size_t)(k % 2) * g->B * kSlot,
                                     kSlot * sizeof(double), g->red + kDslot,
                                     kRedSlots * sizeof(double), kSlotLen * sizeof(double),
                                     g->B, cudaMemcpyDeviceToHost, g->st) == cudaSuccess;
        cudaGraph_t gr = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(g->st, &gr);
        cudaError_t ie = ce;
        if (ok && ce == cudaSuccess) ie = cudaGraphInstantiate(&g->col[k], gr, 0);
        if (gr) cudaGraphDestroy(gr);
        if (!ok || ie != cudaSuccess) {
            cudaGetLastError();
            g->col[k] = nullptr;
            FAIL(r0, FFT_ERR_CUDA, "class graph capture of Krylov column %d failed (%s)", k,
                 cudaGetErrorString(ie));
        }
        return FFT_OK;
    }

    // algorithmic bytes of column k for the whole class: the two 9-field
    // transforms, the tangent apply, the contraction with its dot pass over
    // c_k and q_0 .. q_{k-1}, the update pass
    static double col_bytes(GangBase* g, int k) {
        const fft_rve_s* r = g->m[0];
        const double N = (double)r->g.N, Nh = (double)r->g.Nh, es = (double)sizeof(R);
        const double fft = 9 * N * es + 9 * Nh * 2 * es;
        return g->B * (2 * fft + N * es * 100 + Nh * 2 * es * (9 + 3 + 3 * (k + 1)) +
                       Nh * 2 * es * 3 * (k + 2 + 2 + 3));
    }

    static fft_status launch_col(GangBase* g, int k) {
        if (!g->col[k]) TRY(capture_col(g, k));
        cudaEvent_t ta = nullptr, tb = nullptr;
        if (g->timing) {
            ta = gang_tevent(g);
            tb = gang_tevent(g);
            if (!ta || !tb) {
                if (ta) g->tpool.push_back(ta);
                if (tb) g->tpool.push_back(tb);
                ta = tb = nullptr;
            } else {
                CK(g->m[0], cudaEventRecord(ta, g->st));
            }
        }
        CK(g->m[0], cudaGraphLaunch(g->col[k], g->st));
        if (ta && tb) {
            CK(g->m[0], cudaEventRecord(tb, g->st));
            g->tpend.push_back({{ta, tb}, col_bytes(g, k)});
        }
        CK(g->m[0], cudaEventRecord(g->slot_ev[k % 2], g->st));
        g->graph_launches += 1;
        for (fft_rve_s* r : g->m) r->launches += 3;
        return FFT_OK;
    }

    static fft_status wait_stream(GangBase* g) {
        CK(g->m[0], cudaEventRecord(g->done_ev, g->st));
        CK(g->m[0], gang_wait(g, g->done_ev));
        gang_tcollect(g);
        return FFT_OK;
    }

    // Restarted GMRES (the single-handle driver's, see Impl::gmres) for the
    // members in E with right-hand-side norms bn and stress scales pn; the
    // Arnoldi steps in lockstep.  its[i] = the member's processed steps,
    // st[i] its status.
    static void gmres(GangBase* g, const std::vector<int>& E, const double* bn,
                      const double* pn, int* its, fft_status* st) {
        fft_rve_s* r0 = g->m[0];
        const size_t Nh = r0->g.Nh, n3 = 3 * Nh, vs = n3;
        const double es = (double)sizeof(R);
        const double eta = sizeof(R) == 8 ? 1e-12 : 5e-7;
        const int mres = std::max(1, std::min(r0->opt.restart, kMaxKrylov - 1));
        const int max_lin = r0->opt.max_lin;
        const int B = g->B;
        std::vector<double> target(B), beta(B);
        std::vector<std::vector<double>> Hm(B), y(B);
        std::vector<int> kcols(B, 0), lin_i(B, 0);
        std::vector<char> ok(B, 0), first(B, 1), in_cycle(B, 0), was_in(B, 0);
        std::vector<double> res1(B), res2(B);
        std::vector<const void*> src(B);
        std::vector<int> C;
        auto fail = [&](int i, fft_status s) {
            st[i] = s;
            in_cycle[i] = 0;
        };
        for (int i : E) {
            fft_rve_s* r = g->m[i];
            target[i] = std::max(r->opt.tol_lin * bn[i], eta * pn[i]);
            its[i] = 0;
            Hm[i].assign((size_t)(mres + 1) * mres, 0.0);
            y[i].assign(mres, 0.0);
            if (cudaMemsetAsync(r->x, 0, n3 * sizeof(Cx), r->st) != cudaSuccess) {
                r->err = "cudaMemsetAsync of the GMRES solution failed";
                st[i] = FFT_ERR_CUDA;
                continue;
            }
            if (bn[i] > target[i]) C.push_back(i);
        }
        int lin = 0;  // steps processed by every member still iterating
        auto alive = [&](int i) { return st[i] == FFT_OK && !ok[i]; };
        while (lin < max_lin) {
            std::vector<int> cur;
            for (int i : C)
                if (alive(i)) cur.push_back(i);
            C.swap(cur);
            if (C.empty()) break;
            // restart residuals r = b - A M x of the members past their first cycle
            for_members(g, C, [&](int i) {
                fft_rve_s* r = g->m[i];
                if (st[i] != FFT_OK) return;
                if (first[i]) {
                    beta[i] = bn[i];
                    src[i] = r->b;
                    first[i] = 0;
                    return;
                }
                fft_status s = I::apply_op(r, r->x, 1.0, nullptr, 0, r->w, 0);
                if (s == FFT_OK) {
                    axpby<R>(r->w, r->b, r->w, 1.0, -1.0, n3, r->st);
                    norm2<R>(r->w, r->g, red_at(r, r->red), r->st);
                    r->launches += 2;
                    s = I::fetch(r, 1);
                }
                if (s != FFT_OK) {
                    st[i] = s;
                    return;
                }
                beta[i] = std::sqrt(r->hred[0]);
                if (r->verbose)
                    std::fprintf(stderr, "  gmres restart: true |r|/|b| %.3e\n", beta[i] / bn[i]);
                if (beta[i] <= target[i]) {
                    ok[i] = 1;
                    return;
                }
                src[i] = r->w;
            });
            cur.clear();
            for (int i : C)
                if (alive(i)) cur.push_back(i);
            C.swap(cur);
            if (C.empty()) break;
            // Sparse mode: once fewer than half the members iterate, the
            // batched transforms would mostly transform idle members, so the
            // rest of the cycle runs each member's own step graph (the
            // single-handle driver's, on its stream and its arena slot).
            bool sparse = kSparse * (int)C.size() < B;
            std::vector<char> col_sparse(mres + 1, 0);
            // first column of the cycle: V_0 = src / beta and its gradient
            // spectrum, per member, before the class stream's column graphs
            // (in sparse mode enqueue_step forms it)
            for (int i : C) {
                fft_rve_s* r = g->m[i];
                std::fill(Hm[i].begin(), Hm[i].end(), 0.0);
                kcols[i] = 0;
                res1[i] = res2[i] = -1.0;
                in_cycle[i] = 1;
                if (sparse) continue;
                precond_grad<R>(src[i], 1.0 / beta[i], r->V, r->Kbar, r->g, r->cb9, 1, r->st, 0);
                r->launches += 1;
                if (cudaEventRecord(g->ev_m[i], r->st) != cudaSuccess ||
                    cudaStreamWaitEvent(g->st, g->ev_m[i], 0) != cudaSuccess) {
                    r->err = "class stream fork failed";
                    fail(i, FFT_ERR_CUDA);
                }
            }
            // the cycle's members iterate: their flags on, the others off
            fft_status gs = FFT_OK;
            if (cudaMemsetAsync(g->act, 0, (size_t)B * sizeof(int), g->st) != cudaSuccess)
                gs = FFT_ERR_CUDA;
            for (int i : C)
                if (in_cycle[i] && gs == FFT_OK &&
                    cudaMemsetAsync(g->act + i, 1, sizeof(int), g->st) != cudaSuccess)
                    gs = FFT_ERR_CUDA;
            auto any_in_cycle = [&]() {
                for (int i : C)
                    if (in_cycle[i]) return true;
                return false;
            };
            if (gs != FFT_OK) r0->err = "class stream memset failed";
            // column j for the members still in the cycle
            auto launch = [&](int j) -> fft_status {
                int na = 0;
                for (int i : C) na += in_cycle[i] ? 1 : 0;
                if (!sparse && j >= 1 && kSparse * na < B) {
                    // switch: the members' streams follow the class stream
                    sparse = true;
                    CK(r0, cudaEventRecord(g->ev_a, g->st));
                    for (int i : C)
                        if (in_cycle[i]) CK(g->m[i], cudaStreamWaitEvent(g->m[i]->st, g->ev_a, 0));
                }
                col_sparse[j] = sparse;
                if (!sparse) return launch_col(g, j);
                for (int i : C)
                    if (in_cycle[i]) {
                        const fft_status s1 = I::enqueue_step(g->m[i], j, src[i], 1.0 / beta[i]);
                        if (s1 != FFT_OK) fail(i, s1);
                    }
                return FFT_OK;
            };
            for (int j = 0; gs == FFT_OK; ++j) {
                const bool enq = j < mres && lin + j < max_lin;
                // defer the look-ahead step when every member still in the
                // cycle predicts convergence at the step being read
                bool defer = enq && j >= 2;
                for (int i : C)
                    if (in_cycle[i] && !(res2[i] > 0.0 && res1[i] > 0.0 &&
                                         res1[i] * (res1[i] / res2[i]) <= target[i]))
                        defer = false;
                if (enq && !defer) {
                    gs = launch(j);
                    if (gs != FFT_OK) break;
                }
                if (j == 0) {
                    if (!enq) break;
                    continue;
                }
                const int k = j - 1;
                for (int i : C) was_in[i] = in_cycle[i];
                if (!col_sparse[k]) {
                    const cudaError_t we = gang_wait(g, g->slot_ev[k % 2]);
                    if (we != cudaSuccess) {
                        r0->err = std::string("class stream: ") + cudaGetErrorString(we);
                        gs = FFT_ERR_CUDA;
                        break;
                    }
                }
                for (int i : C) {
                    if (!in_cycle[i]) continue;
                    fft_rve_s* r = g->m[i];
                    if (col_sparse[k] && host_wait(r, r->slot_ev[k % 2]) != cudaSuccess) {
                        r->err = "stream synchronisation in the Arnoldi step failed";
                        fail(i, FFT_ERR_CUDA);
                        continue;
                    }
                    const double* slot =
                        col_sparse[k] ? r->hslot + (size_t)(k % 2) * kSlot
                                      : g->hslots + ((size_t)(k % 2) * B + i) * kSlot;
                    if (slot[kSlotErr] != 0.0) {
                        r->err = "a bulk-copy wait in the Arnoldi step timed out";
                        fail(i, FFT_ERR_CUDA);
                        continue;
                    }
                    bool fin = true;
                    for (int q = 0; q < kSlotLen; ++q) fin = fin && std::isfinite(slot[q]);
                    if (!fin) {
                        char b[128];
                        std::snprintf(b, sizeof(b), "non-finite Krylov coefficient (step %d)",
                                      lin_i[i] + 1);
                        r->err = b;
                        fail(i, FFT_ERR_NONFINITE);
                        continue;
                    }
                    std::vector<double>& H = Hm[i];
                    if (k >= 1)
                        for (int l = 0; l <= k; ++l) H[(size_t)l * mres + k - 1] = slot[l];
                    for (int l = 0; l <= k; ++l) H[(size_t)l * mres + k] = slot[kSlotProv + l];
                    const double hn = std::sqrt(std::max(slot[kSlotNorm], 0.0));
                    H[(size_t)(k + 1) * mres + k] = hn;
                    ++lin_i[i];
                    kcols[i] = k + 1;
                    if (k >= 1 && slot[kSlotNu] == 0.0) {
                        kcols[i] = k;
                        ok[i] = 1;
                        in_cycle[i] = 0;
                        continue;
                    }
                    const double res = I::hess_lsq(H, mres, kcols[i], beta[i], nullptr);
                    if (r->verbose)
                        std::fprintf(stderr, "  gmres it %d |r|/|b| %.3e (class member %d)\n",
                                     lin_i[i], res / bn[i], i);
                    if (res <= target[i] || hn == 0.0) {
                        ok[i] = 1;
                        in_cycle[i] = 0;
                        continue;
                    }
                    res2[i] = res1[i];
                    res1[i] = res;
                }
                // members that left: their kernels in the steps still to be
                // launched return at once
                for (int i : C)
                    if (was_in[i] && !in_cycle[i] &&
                        cudaMemsetAsync(g->act + i, 0, sizeof(int), g->st) != cudaSuccess) {
                        r0->err = "class stream memset failed";
                        gs = FFT_ERR_CUDA;
                    }
                if (gs != FFT_OK) break;
                ++lin;
                if (!any_in_cycle() || !enq) break;
                if (defer) {
                    gs = launch(j);
                    if (gs != FFT_OK) break;
                }
            }
            // the class stream and the members' streams idle (a discarded
            // look-ahead step), then the solution update of every member
            if (gs == FFT_OK) gs = wait_stream(g);
            if (sparse)
                for (int i : C)
                    if (st[i] == FFT_OK && host_wait(g->m[i]) != cudaSuccess) {
                        g->m[i]->err = "stream synchronisation after the Arnoldi steps failed";
                        st[i] = FFT_ERR_CUDA;
                    }
            if (gs != FFT_OK) {
                for (int i : C)
                    if (st[i] == FFT_OK) {
                        g->m[i]->err = r0->err;
                        st[i] = gs;
                    }
                break;
            }
            for_members(g, C, [&](int i) {
                in_cycle[i] = 0;
                if (st[i] != FFT_OK) return;
                fft_rve_s* r = g->m[i];
                const int k = kcols[i];
                I::hess_lsq(Hm[i], mres, k, beta[i], y[i].data());
                if (k > 0) {
                    std::memcpy(r->hy, y[i].data(), k * sizeof(double));
                    if (cudaMemcpyAsync(r->dy, r->hy, k * sizeof(double), cudaMemcpyHostToDevice,
                                        r->st) != cudaSuccess) {
                        r->err = "GMRES coefficient upload failed";
                        st[i] = FFT_ERR_CUDA;
                        return;
                    }
                    cudaEvent_t e = prof_begin(r, KF_XUPD);
                    xupdate<R>(r->x, r->V, vs, k, r->dy, r->Kbar, r->g, r->st);
                    prof_end(r, KF_XUPD, e, (double)Nh * 2 * es * 3 * (k + 2));
                    r->launches += 1;
                }
                if (host_wait(r) != cudaSuccess) {
                    r->err = "stream synchronisation after the GMRES update failed";
                    st[i] = FFT_ERR_CUDA;
                }
            });
            lin = 0;
            for (int i : C)
                if (alive(i)) lin = std::max(lin, lin_i[i]);
        }
        for (int i : E) {
            its[i] = lin_i[i];
            if (st[i] != FFT_OK) continue;
            fft_rve_s* r = g->m[i];
            if (r->use_bulk) {
                int e = 0;
                if (cudaMemcpy(&e, r->bulk.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
                    r->err = "reading the bulk-copy error word failed";
                    st[i] = FFT_ERR_CUDA;
                    continue;
                }
                if (e) {
                    r->err = "a bulk-copy wait in the Arnoldi step timed out";
                    st[i] = FFT_ERR_CUDA;
                    continue;
                }
            }
            if (!ok[i] && bn[i] > target[i]) {
                char b[96];
                std::snprintf(b, sizeof(b), "GMRES reached max_lin = %d", max_lin);
                r->err = b;
                st[i] = FFT_ERR_NOT_CONVERGED;
            }
        }
    }

    // Newton's method (Impl::newton_solve) for the members in E in lockstep.
    static void newton(GangBase* g, std::vector<int> E, fft_stats** stats, fft_status* st) {
        const int B = g->B;
        std::vector<double> alpha(B, 1.0), prev(B, 0.0), bn(B), pn(B);
        std::vector<int> its(B, 0);
        std::vector<char> cp_pending(B, 0), go(B, 0);
        const int max_newton = g->m[0]->opt.max_newton;
        for (int it = 0; it < max_newton && !E.empty(); ++it) {
            // residual of every member (Impl::newton_solve's opening), enqueued
            for_members(g, E, [&](int i) {
                fft_rve_s* r = g->m[i];
                const size_t N = r->g.N;
                fft_status s = FFT_OK;
                cp_pending[i] = 0;
                if (!r->cp_valid) {
                    s = I::cp_enq(r, false);
                    cp_pending[i] = s == FFT_OK;
                }
                if (s == FFT_OK) {
                    if (stats[i]) stats[i]->newton_it += 1;
                    cudaEvent_t e = prof_begin(r, KF_KBAR);
                    kbar<R>(r->K, r->phi, r->mat.k_res, N, red_at(r, r->Kbar), r->st);
                    prof_end(r, KF_KBAR, e, (double)N * sizeof(R) * 82);
                    e = prof_begin(r, KF_RESID);
                    degrade<R>(r->P, r->phi, r->mat.k_res, r->rb9, N, r->st);
                    prof_end(r, KF_RESID, e, (double)N * sizeof(R) * 19);
                    s = I::fwd9(r);
                }
                if (s == FFT_OK) {
                    cudaEvent_t e = prof_begin(r, KF_RESID);
                    residual<R>(r->cb9, r->g, r->b, red_at(r, r->red), r->st);
                    prof_end(r, KF_RESID, e, (double)r->g.Nh * 2 * sizeof(R) * 12);
                    r->launches += 3;
                    s = I::fetch_enq(r, 2);
                }
                st[i] = s;
            });
            // ... and read
            for_members(g, E, [&](int i) {
                fft_rve_s* r = g->m[i];
                go[i] = 0;
                if (st[i] != FFT_OK) return;
                if (cp_pending[i]) {
                    int nf = 0;
                    st[i] = I::cp_get(r, &nf);
                    if (st[i] != FFT_OK) return;
                    if (stats[i]) stats[i]->local_fail += nf;
                }
                st[i] = I::fetch_get(r, 2);
                if (st[i] != FFT_OK) return;
                bn[i] = std::sqrt(r->hred[0]);
                pn[i] = std::sqrt(r->hred[1]);
                go[i] = 1;
            });
            std::vector<int> L;
            for (int i : E)
                if (go[i]) L.push_back(i);
            gmres(g, L, bn.data(), pn.data(), its.data(), st);
            // the Newton update F += alpha grad(M x) of every member
            for_members(g, L, [&](int i) {
                fft_rve_s* r = g->m[i];
                go[i] = 0;
                if (stats[i]) stats[i]->lin_it_total += its[i];
                if (st[i] != FFT_OK) return;
                const size_t N = r->g.N;
                cudaEvent_t e = prof_begin(r, KF_PRECOND);
                precond_grad<R>(r->x, alpha[i], nullptr, r->Kbar, r->g, r->cb9, 0, r->st);
                prof_end(r, KF_PRECOND, e, (double)r->g.Nh * 2 * sizeof(R) * 12);
                fft_status s = I::inv9(r);
                if (s == FFT_OK) {
                    e = prof_begin(r, KF_FUPD);
                    fupdate<R>(r->H, r->rb9, r->Ht, N, red_at(r, r->red), r->st);
                    prof_end(r, KF_FUPD, e, (double)N * sizeof(R) * 36);
                    r->launches += 2;
                    s = I::fetch_enq(r, 2);
                }
                st[i] = s;
                if (s != FFT_OK) return;
                // the convergence test and the damping of Impl::newton_solve
                st[i] = I::fetch_get(r, 2);
                if (st[i] != FFT_OK) return;
                r->cp_valid = false;
                const double gmax = r->hred[0] / alpha[i], dFt = std::max(r->hred[1], 1e-30);
                const double ratio = gmax / dFt;
                if (r->verbose)
                    std::fprintf(stderr, "newton %d (class member %d) |b| %.3e lin %d ratio %.3e\n",
                                 it, i, bn[i], its[i], ratio);
                if (ratio < r->opt.tol_newton) return;  // converged
                if (it + 1 >= I::kDampFrom && ratio >= prev[i])
                    alpha[i] = std::max(0.5 * alpha[i], 1.0 / 16);
                else if (ratio < 0.5 * prev[i])
                    alpha[i] = std::min(2.0 * alpha[i], 1.0);
                prev[i] = ratio;
                go[i] = 1;
            });
            std::vector<int> next;
            for (int i : L)
                if (go[i]) next.push_back(i);
            E.swap(next);
        }
        for (int i : E) {
            char b[96];
            std::snprintf(b, sizeof(b), "Newton reached max_newton = %d", max_newton);
            g->m[i]->err = b;
            st[i] = FFT_ERR_NOT_CONVERGED;
        }
    }

    // One load increment for every member (run_increment of the
    // single-handle driver, under strain or mixed control): the staggered
    // loop in lockstep, then cut-backs of the members that did not converge,
    // each on its own host thread.
    static void run_increment(GangBase* g, const double* const* Fbar, const double* const* Pstar,
                              const int32_t* const* mask, const double* dt, fft_stats** stats,
                              fft_status* st) {
        const int B = g->B;
        std::vector<int> all(B), A;
        for (int i = 0; i < B; ++i) all[i] = i;
        for_members(g, all, [&](int i) {
            if (stats[i]) std::memset(stats[i], 0, sizeof(fft_stats));
            st[i] = mask ? I::apply_increment_mixed(g->m[i], Fbar[i], Pstar ? Pstar[i] : nullptr,
                                                    mask[i], dt[i])
                         : I::apply_increment(g->m[i], Fbar[i], dt[i]);
        });
        for (int i = 0; i < B; ++i)
            if (st[i] == FFT_OK) A.push_back(i);
        std::vector<char> more(B, 0);
        const int max_stag = g->m[0]->opt.max_stag;
        for (int it = 0; it < max_stag && !A.empty(); ++it) {
            std::vector<int> E;
            for (int i : A) {
                fft_rve_s* r = g->m[i];
                // the opening of Impl::solve_equilibrium
                if (r->state != ST_APPLIED && r->state != ST_DAMAGE) {
                    r->err = "solve_equilibrium before apply_increment";
                    st[i] = FFT_ERR_STATE;
                    continue;
                }
                if (cudaMemcpyAsync(r->Hprev, r->H, 9 * r->g.N * sizeof(R),
                                    cudaMemcpyDeviceToDevice, r->st) != cudaSuccess) {
                    r->err = "cudaMemcpyAsync of F failed";
                    st[i] = FFT_ERR_CUDA;
                    continue;
                }
                r->skipped = false;
                r->state = ST_EQUIL;
                if (r->stag_it >= 1 && !r->phi_changed) {
                    r->skipped = true;
                    if (stats[i]) stats[i]->skipped_equilibrium = 1;
                    continue;
                }
                E.push_back(i);
            }
            // Newton, then under mixed control the outer rounds of
            // Impl::mixed_step, until every member's stress targets hold
            for (int outer = 0; !E.empty(); ++outer) {
                newton(g, E, stats, st);
                for_members(g, E, [&](int i) {
                    more[i] = 0;
                    fft_rve_s* r = g->m[i];
                    if (st[i] != FFT_OK || !r->mixed) return;
                    bool done = false;
                    st[i] = I::mixed_step(r, stats[i], outer, &done);
                    more[i] = st[i] == FFT_OK && !done;
                });
                std::vector<int> again;
                for (int i : E)
                    if (more[i]) again.push_back(i);
                E.swap(again);
            }
            // the damage update of every member, each with its own host
            // round trips (phase-field CG, staggered test), side by side
            for_members(g, A, [&](int i) {
                more[i] = 0;
                if (st[i] != FFT_OK) return;
                fft_rve_s* r = g->m[i];
                st[i] = I::update_damage(r, stats[i]);
                if (st[i] != FFT_OK) return;
                if (r->converged)
                    st[i] = I::commit(r);
                else
                    more[i] = 1;
            });
            std::vector<int> next;
            for (int i : A)
                if (more[i]) next.push_back(i);
            A.swap(next);
        }
        for (int i : A) {
            char b[96];
            std::snprintf(b, sizeof(b), "staggered loop reached max_stag = %d", max_stag);
            g->m[i]->err = b;
            st[i] = FFT_ERR_NOT_CONVERGED;
        }
        // cut-backs: each failed member on its own host thread (the members'
        // streams and state are independent; the cut-backs diverge)
        std::vector<std::thread> cut;
        for (int i = 0; i < B; ++i) {
            fft_rve_s* r = g->m[i];
            if (st[i] != FFT_ERR_NOT_CONVERGED || r->opt.max_cutbacks <= 0) continue;
            if (r->verbose)
                std::fprintf(stderr, "  class member %d not converged: cutting back\n", i);
            cut.emplace_back([=] {
                st[i] = cudaSetDevice(r->dev) != cudaSuccess
                            ? FFT_ERR_CUDA
                            : I::run_halves(r, Fbar[i], Pstar && mask ? Pstar[i] : nullptr,
                                            mask ? mask[i] : nullptr, dt[i], stats[i], 1);
            });
        }
        for (auto& t : cut) t.join();
        for (int i = 0; i < B; ++i)
            if (st[i] == FFT_OK && host_wait(g->m[i]) != cudaSuccess) st[i] = FFT_ERR_CUDA;
    }
};

static void gang_release(GangBase* g) {
    g->pool.stop();
    for (auto& e : g->col)
        if (e) {
            cudaGraphExecDestroy(e);
            e = nullptr;
        }
    for (size_t i = 0; i < g->rb9_own.size(); ++i) {
        fft_rve_s* r = g->m[i];
        drop_graphs(r);  // the members' own step graphs used the arena
        r->rb9 = g->rb9_own[i];
        r->cb9 = g->cb9_own[i];
        if (i < g->red_own.size()) r->red = g->red_own[i];
        r->poll = false;
    }
    if (g->plans) {
        cufftDestroy(g->r2c);
        cufftDestroy(g->c2r);
    }
    if (g->rb9) cudaFree(g->rb9);
    if (g->red) cudaFree(g->red);
    if (g->hslots) cudaFreeHost(g->hslots);
    if (g->act) cudaFree(g->act);
    if (g->cb9) cudaFree(g->cb9);
    for (cudaEvent_t e : g->ev_m)
        if (e) cudaEventDestroy(e);
    gang_tcollect(g);
    for (cudaEvent_t e : g->tpool) cudaEventDestroy(e);
    for (cudaEvent_t e : {g->ev_a, g->slot_ev[0], g->slot_ev[1], g->done_ev})
        if (e) cudaEventDestroy(e);
    if (g->st) cudaStreamDestroy(g->st);
}

}  // namespace

// ------------------------------------------------------------ class entry points
// (internal to the library; the batch driver forms the classes)

// the solver options that the lockstep loops share (all but the stream)
static bool same_options(const fft_options& a, const fft_options& b) {
    return a.tol_stag == b.tol_stag && a.tol_newton == b.tol_newton && a.tol_lin == b.tol_lin &&
           a.tol_pf == b.tol_pf && a.tol_local == b.tol_local && a.max_stag == b.max_stag &&
           a.max_newton == b.max_newton && a.max_lin == b.max_lin && a.max_pf == b.max_pf &&
           a.max_local == b.max_local && a.restart == b.restart && a.prec == b.prec &&
           a.max_cutbacks == b.max_cutbacks && a.derivative == b.derivative &&
           a.kernel_variant == b.kernel_variant;
}

// 1 when b can run in lockstep with a: same device, precision, grid, solver
// options (but the stream); the unfused Arnoldi step with graphs.
int fatfft_gang_compatible(fft_rve_t a, fft_rve_t b) {
    if (!a || !b) return 0;
    return a->dev == b->dev && a->prec == b->prec && a->g.n0 == b->g.n0 &&
           a->g.n1 == b->g.n1 && a->g.n2 == b->g.n2 && same_options(a->opt, b->opt) &&
           !a->use_fused && !b->use_fused && a->graphs && b->graphs && a->st && b->st;
}

fft_status fatfft_gang_create(fft_rve_t const* members, int n, void** out) {
    if (!out || !members || n < 2 || n > kGangMax) return FFT_ERR_ARG;
    *out = nullptr;
    for (int i = 1; i < n; ++i)
        if (!fatfft_gang_compatible(members[0], members[i])) return FFT_ERR_ARG;
    GangBase* g = new GangBase();
    g->m.assign(members, members + n);
    g->B = n;
    fft_rve_s* r0 = members[0];
    const size_t N = r0->g.N, Nh = r0->g.Nh, es = r0->esz;
    auto bad = [&](fft_status s) {
        gang_release(g);
        delete g;
        return s;
    };
    if (cudaSetDevice(r0->dev) != cudaSuccess ||
        cudaStreamCreateWithFlags(&g->st, cudaStreamNonBlocking) != cudaSuccess)
        return bad(FFT_ERR_CUDA);
    g->ev_m.assign(n, nullptr);
    for (int i = 0; i < n; ++i)
        if (cudaEventCreateWithFlags(&g->ev_m[i], cudaEventDisableTiming) != cudaSuccess)
            return bad(FFT_ERR_CUDA);
    if (cudaEventCreateWithFlags(&g->ev_a, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->slot_ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->slot_ev[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&g->done_ev, cudaEventDisableTiming) != cudaSuccess)
        return bad(FFT_ERR_CUDA);
    if (cudaMalloc(&g->rb9, (size_t)n * 9 * N * es) != cudaSuccess ||
        cudaMalloc(&g->cb9, (size_t)n * 9 * Nh * 2 * es) != cudaSuccess ||
        cudaMalloc((void**)&g->act, (size_t)n * sizeof(int)) != cudaSuccess ||
        cudaMalloc((void**)&g->red, (size_t)n * kRedSlots * sizeof(double)) != cudaSuccess ||
        cudaMallocHost((void**)&g->hslots, (size_t)2 * n * kSlot * sizeof(double)) != cudaSuccess)
        return bad(FFT_ERR_OOM);
    // the member plans' layout, batched over the class: 9 n fields
    int dims3[3] = {r0->g.n2, r0->g.n1, r0->g.n0};
    int lead = 0;
    while (lead < 2 && dims3[lead] == 1) ++lead;
    const cufftType tf = r0->prec == FFT_PREC_FP64 ? CUFFT_D2Z : CUFFT_R2C;
    const cufftType ti = r0->prec == FFT_PREC_FP64 ? CUFFT_Z2D : CUFFT_C2R;
    if (cufftPlanMany(&g->r2c, 3 - lead, dims3 + lead, nullptr, 1, (int)N, nullptr, 1, (int)Nh,
                      tf, 9 * n) != CUFFT_SUCCESS)
        return bad(FFT_ERR_CUFFT);
    if (cufftPlanMany(&g->c2r, 3 - lead, dims3 + lead, nullptr, 1, (int)Nh, nullptr, 1, (int)N,
                      ti, 9 * n) != CUFFT_SUCCESS) {
        cufftDestroy(g->r2c);
        return bad(FFT_ERR_CUFFT);
    }
    g->plans = true;
    cufftSetStream(g->r2c, g->st);
    cufftSetStream(g->c2r, g->st);
    // the members' step scratch moves into the arena (their step graphs,
    // captured on the old buffers, are dropped)
    for (int i = 0; i < n; ++i) {
        fft_rve_s* r = members[i];
        if (cudaStreamSynchronize(r->st) != cudaSuccess) return bad(FFT_ERR_CUDA);
        drop_graphs(r);
        g->rb9_own.push_back(r->rb9);
        g->cb9_own.push_back(r->cb9);
        r->rb9 = (char*)g->rb9 + (size_t)i * 9 * N * es;
        r->cb9 = (char*)g->cb9 + (size_t)i * 9 * Nh * 2 * es;
        double* red_i = g->red + (size_t)i * kRedSlots;
        if (cudaMemcpy(red_i, r->red, kRedSlots * sizeof(double), cudaMemcpyDeviceToDevice) !=
            cudaSuccess)
            return bad(FFT_ERR_CUDA);
        g->red_own.push_back(r->red);
        r->red = red_i;
        r->poll = true;
    }
    g->pool.start(std::min(kGangHelpers, n - 1), r0->dev);
    *out = g;
    return FFT_OK;
}

// One increment for every member: Fbar[i] (9 doubles) and dt[i] of member
// i; with mask (nullable: strain control) the mixed control of
// run_increment_mixed, mask[i] (9 flags) and Pstar[i] (nullable arrays);
// stats[i] nullable, status[i] per member.
fft_status fatfft_gang_run(void* gp, const double* const* Fbar, const double* const* Pstar,
                           const int32_t* const* mask, const double* dt, fft_stats** stats,
                           int* status) {
    GangBase* g = (GangBase*)gp;
    if (!g) return FFT_ERR_ARG;
    if (cudaSetDevice(g->m[0]->dev) != cudaSuccess) return FFT_ERR_CUDA;
    std::vector<fft_status> st(g->B, FFT_OK);
    if (g->m[0]->prec == FFT_PREC_FP64)
        Gang<double>::run_increment(g, Fbar, Pstar, mask, dt, stats, st.data());
    else
        Gang<float>::run_increment(g, Fbar, Pstar, mask, dt, stats, st.data());
    fft_status worst = FFT_OK;
    for (int i = 0; i < g->B; ++i) {
        status[i] = (int)st[i];
        if (st[i] != FFT_OK && worst == FFT_OK) worst = st[i];
    }
    return worst;
}

int fatfft_gang_size(void* gp) { return gp ? ((GangBase*)gp)->B : 0; }
fft_rve_t fatfft_gang_member(void* gp, int i) {
    GangBase* g = (GangBase*)gp;
    return g && i >= 0 && i < g->B ? g->m[i] : nullptr;
}
long long fatfft_gang_graph_launches(void* gp) {
    return gp ? ((GangBase*)gp)->graph_launches : 0;
}
void fatfft_gang_timing(void* gp, int on, double* ms, double* bytes) {
    GangBase* g = (GangBase*)gp;
    if (!g) return;
    if (ms) *ms = g->graph_ms;
    if (bytes) *bytes = g->graph_bytes;
    if (on >= 0) {
        g->timing = on != 0;
        g->graph_ms = g->graph_bytes = 0.0;
    }
}

void fatfft_gang_destroy(void* gp) {
    GangBase* g = (GangBase*)gp;
    if (!g) return;
    cudaSetDevice(g->m[0]->dev);
    if (g->st) cudaStreamSynchronize(g->st);
    for (fft_rve_s* r : g->m) cudaStreamSynchronize(r->st);
    gang_release(g);
    delete g;
}
