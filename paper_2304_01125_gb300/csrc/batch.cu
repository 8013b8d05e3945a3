// Batched RVEs: run_increment over many independent handles at once.
//
// Each handle keeps its own stream, device buffers and per-column GMRES
// graphs; a pool of host threads (native, persistent across increments)
// drives the handles' increments concurrently, largest grid first, so that
// small grids that cannot fill the GPU alone share it.  The handles never
// wait on one another (independent problems, no data exchange).
#include <cuda_runtime.h>

#include <algorithm>
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

struct fft_batch_s {
    std::vector<fft_rve_t> rves;
    std::vector<int> dev;
    std::vector<int> order;  // indices, largest grid first
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

    void worker() {
        std::unique_lock<std::mutex> lk(m);
        long long seen = 0;
        for (;;) {
            cv_work.wait(lk, [&] { return quit || (gen != seen && next < (int)rves.size()); });
            if (quit) return;
            seen = gen;
            while (next < (int)rves.size()) {
                const int i = order[next++];
                lk.unlock();
                int s = (int)FFT_ERR_CUDA;
                if (cudaSetDevice(dev[i]) == cudaSuccess)
                    s = mask ? (int)run_increment_mixed(rves[i], Fbar + 9 * (size_t)i,
                                                        Pbar ? Pbar + 9 * (size_t)i : nullptr,
                                                        mask + 9 * (size_t)i, dt[i],
                                                        stats ? stats + i : nullptr)
                             : (int)run_increment(rves[i], Fbar + 9 * (size_t)i, dt[i],
                                                  stats ? stats + i : nullptr);
                lk.lock();
                status[i] = s;
                if (++done == (int)rves.size()) cv_done.notify_all();
            }
        }
    }
};

extern "C" {

fft_status batch_create(fft_batch_t* out, fft_rve_t const* rves, int n, int n_threads) {
    if (!out || !rves || n < 1) return FFT_ERR_ARG;
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
    b->rves.assign(rves, rves + n);
    for (int i = 0; i < n; ++i) b->dev.push_back(fatfft_rve_device(rves[i]));
    b->order.resize(n);
    for (int i = 0; i < n; ++i) b->order[i] = i;
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
        return fatfft_rve_voxels(rves[x]) > fatfft_rve_voxels(rves[y]);
    });
    int t = n_threads > 0 ? n_threads : (int)std::thread::hardware_concurrency();
    t = std::max(1, std::min(t, n));
    for (int i = 0; i < t; ++i) b->pool.emplace_back([b] { b->worker(); });
    *out = b;
    return FFT_OK;
}

static fft_status run_job(fft_batch_t b, const double* Fbar, const double* Pbar,
                          const int32_t* mask, const double* dt, fft_stats* stats,
                          int* status) {
    if (!b || !Fbar || !dt) return FFT_ERR_ARG;
    const int n = (int)b->rves.size();
    for (int i = 0; i < n; ++i)
        if (!(dt[i] >= 0)) return FFT_ERR_ARG;
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
        ++b->gen;
        b->cv_work.notify_all();
        b->cv_done.wait(lk, [&] { return b->done == n; });
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

void batch_destroy(fft_batch_t b) {
    if (!b) return;
    {
        std::lock_guard<std::mutex> lk(b->m);
        b->quit = true;
    }
    b->cv_work.notify_all();
    for (auto& t : b->pool) t.join();
    delete b;
}

}  // extern "C"
