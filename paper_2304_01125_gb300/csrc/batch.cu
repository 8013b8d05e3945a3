// Batched RVEs: run_increment over many independent handles at once.
//
// Each handle keeps its own stream and device buffers.  Handles of one size
// class (same grid, precision and solver options) form a lockstep class
// (gang.cu): under strain or mixed control their increments run together, every
// Krylov column of the whole class one graph launch with one batched
// transform per direction.  A pool of host threads (native, persistent
// across increments) drives the classes and the remaining single handles
// concurrently, largest work first, so that small grids that cannot fill the
// GPU alone share it.  The handles never wait on one another (independent
// problems, no data exchange).  While in a batch, a handle's host waits poll
// and yield instead of spinning: the pool's threads may outnumber the host
// cores.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "fatiguefft.h"

int fatfft_rve_device(fft_rve_t r);
void* fatfft_rve_stream(fft_rve_t r);
size_t fatfft_rve_voxels(fft_rve_t r);
void fatfft_rve_set_poll(fft_rve_t r, bool on);
bool fatfft_rve_claim(fft_rve_t r, void* batch);
void fatfft_rve_unclaim(fft_rve_t r, void* batch);
int fatfft_gang_compatible(fft_rve_t a, fft_rve_t b);
fft_status fatfft_gang_create(fft_rve_t const* members, int n, void** out);
fft_status fatfft_gang_run(void* g, const double* const* Fbar, const double* const* Pstar,
                           const int32_t* const* mask, const double* dt, fft_stats** stats,
                           int* status);
long long fatfft_gang_graph_launches(void* g);
void fatfft_gang_timing(void* g, int on, double* ms, double* bytes);
void fatfft_gang_destroy(void* g);

namespace {
constexpr int kClassMax = 64;  // members of one lockstep class
// Classes form by default only for grids of at most 2^16 voxels (40^3):
// there a GMRES step is mostly launch and synchronisation latency (about
// 0.09 ms per step from 16^3 to 32^3 on GB300), which one graph launch for
// the class amortises (32 RVEs of 32^3: 49.1 M against 40.4 M
// voxel-increments/s on their own streams; of 16^3: 12.2 M against 10.0 M);
// from 48^3 on a step is increasingly bandwidth-bound and lockstep gains
// nothing over concurrent streams (16 of 48^3: 43.0 M against 43.7 M), it
// only adds the wait for the slowest member.  Flags bit 1 forms classes at
// any size.
constexpr size_t kClassMaxVoxels = 1 << 16;
// a unit of work for one pool thread: a lockstep class or a single handle
struct Unit {
    std::vector<int> idx;  // batch indices
    void* gang = nullptr;
    size_t voxels = 0;
};
}  // namespace

struct fft_batch_s {
    std::vector<fft_rve_t> rves;
    std::vector<int> dev;
    std::vector<int> order;  // indices, largest grid first
    std::vector<Unit> units;  // strain control: classes and single handles, largest first
    std::vector<std::thread> pool;
    std::mutex call;  // one batch call at a time (the job fields below are shared)
    std::mutex m;
    std::condition_variable cv_work, cv_done;
    // the current job
    const double* Fbar = nullptr;
    const double* Pbar = nullptr;   // mixed control: nullable targets (9 per RVE)
    const int32_t* mask = nullptr;  // mixed control: 9 flags per RVE; null = strain control
    const double* dt = nullptr;
    fft_stats* stats = nullptr;
    int* status = nullptr;
    int next = 0, done = 0;
    long long gen = 0;
    bool quit = false;

    // the units of a call: the classes and the single handles
    bool use_units = false;
    int njobs() const { return use_units ? (int)units.size() : (int)rves.size(); }

    void run_one(int i) {
        int s = (int)FFT_ERR_CUDA;
        if (cudaSetDevice(dev[i]) == cudaSuccess)
            s = mask ? (int)run_increment_mixed(rves[i], Fbar + 9 * (size_t)i,
                                                Pbar ? Pbar + 9 * (size_t)i : nullptr,
                                                mask + 9 * (size_t)i, dt[i],
                                                stats ? stats + i : nullptr)
                     : (int)run_increment(rves[i], Fbar + 9 * (size_t)i, dt[i],
                                          stats ? stats + i : nullptr);
        status[i] = s;
    }
    void run_unit(const Unit& u) {
        if (!u.gang) {
            run_one(u.idx[0]);
            return;
        }
        const size_t n = u.idx.size();
        std::vector<const double*> F(n), P(n);
        std::vector<const int32_t*> M(n);
        std::vector<double> d(n);
        std::vector<fft_stats*> sp(n);
        std::vector<int> st(n, (int)FFT_ERR_CUDA);
        for (size_t k = 0; k < n; ++k) {
            const int i = u.idx[k];
            F[k] = Fbar + 9 * (size_t)i;
            P[k] = Pbar ? Pbar + 9 * (size_t)i : nullptr;
            M[k] = mask ? mask + 9 * (size_t)i : nullptr;
            d[k] = dt[i];
            sp[k] = stats ? stats + i : nullptr;
        }
        fatfft_gang_run(u.gang, F.data(), mask ? P.data() : nullptr, mask ? M.data() : nullptr,
                        d.data(), sp.data(), st.data());
        for (size_t k = 0; k < n; ++k) status[u.idx[k]] = st[k];
    }

    void worker() {
        std::unique_lock<std::mutex> lk(m);
        long long seen = 0;
        for (;;) {
            cv_work.wait(lk, [&] { return quit || (gen != seen && next < njobs()); });
            if (quit) return;
            seen = gen;
            while (next < njobs()) {
                const int j = next++;
                lk.unlock();
                if (use_units)
                    run_unit(units[j]);
                else
                    run_one(order[j]);
                lk.lock();
                if (++done == njobs()) cv_done.notify_all();
            }
        }
    }
};

extern "C" {

fft_status batch_create_ex(fft_batch_t* out, fft_rve_t const* rves, int n, int n_threads,
                           int flags) {
    if (!out || !rves || n < 1 || (flags & ~3)) return FFT_ERR_ARG;
    *out = nullptr;
    std::set<fft_rve_t> seen;
    std::set<void*> streams;
    for (int i = 0; i < n; ++i) {
        // distinct handles on distinct, non-default streams: each handle's
        // work (and its graph captures) stays on its own stream
        if (!rves[i]) return FFT_ERR_ARG;
        void* st = fatfft_rve_stream(rves[i]);
        if (!st || !seen.insert(rves[i]).second || !streams.insert(st).second)
            return FFT_ERR_ARG;
    }
    fft_batch_s* b = new fft_batch_s();
    // a handle belongs to one batch at a time (a class takes over its
    // Arnoldi scratch until the batch is destroyed)
    for (int i = 0; i < n; ++i)
        if (!fatfft_rve_claim(rves[i], b)) {
            for (int j = 0; j < i; ++j) fatfft_rve_unclaim(rves[j], b);
            delete b;
            return FFT_ERR_ARG;
        }
    b->rves.assign(rves, rves + n);
    for (int i = 0; i < n; ++i) fatfft_rve_set_poll(rves[i], true);
    for (int i = 0; i < n; ++i) b->dev.push_back(fatfft_rve_device(rves[i]));
    b->order.resize(n);
    for (int i = 0; i < n; ++i) b->order[i] = i;
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
        return fatfft_rve_voxels(rves[x]) > fatfft_rve_voxels(rves[y]);
    });
    // lockstep classes (flags bit 0): handles compatible with a class's
    // first member join it, up to kClassMax members
    std::vector<char> taken(n, 0);
    for (int a : b->order) {
        if (taken[a]) continue;
        Unit u;
        u.idx.push_back(a);
        taken[a] = 1;
        const bool sized = (flags & 2) || fatfft_rve_voxels(rves[a]) <= kClassMaxVoxels;
        if ((flags & 3) && sized)
            for (int c : b->order)
                if (!taken[c] && (int)u.idx.size() < kClassMax &&
                    fatfft_gang_compatible(rves[a], rves[c])) {
                    u.idx.push_back(c);
                    taken[c] = 1;
                }
        for (int i : u.idx) u.voxels += fatfft_rve_voxels(rves[i]);
        if (u.idx.size() > 1) {
            std::vector<fft_rve_t> mem;
            for (int i : u.idx) mem.push_back(rves[i]);
            const fft_status s = fatfft_gang_create(mem.data(), (int)mem.size(), &u.gang);
            if (s != FFT_OK) {
                for (Unit& v : b->units)
                    if (v.gang) fatfft_gang_destroy(v.gang);
                for (int i = 0; i < n; ++i) {
                    fatfft_rve_set_poll(rves[i], false);
                    fatfft_rve_unclaim(rves[i], b);
                }
                delete b;
                return s;
            }
        }
        b->units.push_back(std::move(u));
    }
    std::stable_sort(b->units.begin(), b->units.end(),
                     [](const Unit& x, const Unit& y) { return x.voxels > y.voxels; });
    int t = n_threads > 0 ? n_threads : (int)std::thread::hardware_concurrency();
    t = std::max(1, std::min(t, n));
    for (int i = 0; i < t; ++i) b->pool.emplace_back([b] { b->worker(); });
    *out = b;
    return FFT_OK;
}

fft_status batch_create(fft_batch_t* out, fft_rve_t const* rves, int n, int n_threads) {
    return batch_create_ex(out, rves, n, n_threads, 1);
}

static fft_status run_job(fft_batch_t b, const double* Fbar, const double* Pbar,
                          const int32_t* mask, const double* dt, fft_stats* stats,
                          int* status) {
    if (!b || !Fbar || !dt) return FFT_ERR_ARG;
    const int n = (int)b->rves.size();
    for (int i = 0; i < n; ++i) {
        if (!(dt[i] >= 0) || !std::isfinite(dt[i])) return FFT_ERR_ARG;
        for (int c = 0; c < 9; ++c)
            if (!std::isfinite(Fbar[9 * (size_t)i + c]) ||
                (Pbar && !std::isfinite(Pbar[9 * (size_t)i + c])))
                return FFT_ERR_ARG;
    }
    std::vector<int> st(n, (int)FFT_OK);
    std::lock_guard<std::mutex> serial(b->call);
    {
        std::unique_lock<std::mutex> lk(b->m);
        b->Fbar = Fbar;
        b->Pbar = Pbar;
        b->mask = mask;
        b->dt = dt;
        b->stats = stats;
        b->status = st.data();
        b->next = 0;
        b->done = 0;
        b->use_units = true;
        ++b->gen;
        b->cv_work.notify_all();
        b->cv_done.wait(lk, [&] { return b->done == b->njobs(); });
        b->status = nullptr;
    }
    if (status) std::memcpy(status, st.data(), n * sizeof(int));
    for (int i = 0; i < n; ++i)
        if (st[i] != (int)FFT_OK) return (fft_status)st[i];
    return FFT_OK;
}

fft_status batch_run_increment(fft_batch_t b, const double* Fbar, const double* dt,
                               fft_stats* stats, int* status) {
    return run_job(b, Fbar, nullptr, nullptr, dt, stats, status);
}

fft_status batch_run_increment_mixed(fft_batch_t b, const double* Fbar, const double* Pbar,
                                     const int32_t* mask, const double* dt, fft_stats* stats,
                                     int* status) {
    if (!mask) return FFT_ERR_ARG;
    return run_job(b, Fbar, Pbar, mask, dt, stats, status);
}

int batch_size(fft_batch_t b) { return b ? (int)b->rves.size() : 0; }

int batch_classes(fft_batch_t b, int timing, int* sizes, long long* graph_launches,
                  double* graph_ms, double* graph_bytes) {
    if (!b) return 0;
    std::lock_guard<std::mutex> serial(b->call);
    int k = 0;
    for (const Unit& u : b->units) {
        if (!u.gang) continue;
        if (sizes) sizes[k] = (int)u.idx.size();
        if (graph_launches) graph_launches[k] = fatfft_gang_graph_launches(u.gang);
        fatfft_gang_timing(u.gang, timing, graph_ms ? graph_ms + k : nullptr,
                           graph_bytes ? graph_bytes + k : nullptr);
        ++k;
    }
    return k;
}

void batch_destroy(fft_batch_t b) {
    if (!b) return;
    {
        std::lock_guard<std::mutex> lk(b->m);
        b->quit = true;
    }
    b->cv_work.notify_all();
    for (auto& t : b->pool) t.join();
    for (Unit& u : b->units)
        if (u.gang) fatfft_gang_destroy(u.gang);
    for (fft_rve_t r : b->rves) {
        fatfft_rve_set_poll(r, false);
        fatfft_rve_unclaim(r, b);
    }
    delete b;
}

}  // extern "C"
