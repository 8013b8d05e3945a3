// Test probe (not part of the library; built by tests/test_gpu_host_overlap.py
// against the library's internal header): wall time per Arnoldi column of
// restarted GMRES (Sec. 3.2) with the host reading every column's
// coefficients one step behind the device, as the solver does, against the
// same columns enqueued back to back with one synchronisation at the end.
// Equal times show that the host's reads are off the device's critical path.
#include <chrono>

#include "rve_impl.cuh"

extern "C" int hostgap(fft_rve_t r, int ncols, int reps, double* out) {
    typedef Impl<float> I;
    if (r->prec != FFT_PREC_MIXED) return -1;
    const size_t N = r->g.N;
    // a right-hand side: the current residual (as Newton's opening)
    kbar<float>(r->K, r->phi, r->mat.k_res, N, red_at(r, r->Kbar), r->st);
    degrade<float>(r->P, r->phi, r->mat.k_res, r->rb9, N, r->st);
    if (I::fwd9(r) != FFT_OK) return -2;
    residual<float>(r->cb9, r->g, r->b, red_at(r, r->red), r->st);
    if (I::fetch(r, 2) != FFT_OK) return -3;
    double bn = std::sqrt(r->hred[0]);
    if (!(bn > 0)) bn = 1.0;
    double best_a = 1e30, best_b = 1e30;
    for (int rep = 0; rep < reps; ++rep) {
        // (a) back to back
        cudaStreamSynchronize(r->st);
        auto t0 = std::chrono::steady_clock::now();
        for (int j = 0; j < ncols; ++j)
            if (I::enqueue_step(r, j, r->b, 1.0 / bn) != FFT_OK) return -4;
        cudaStreamSynchronize(r->st);
        auto t1 = std::chrono::steady_clock::now();
        best_a = std::min(best_a, std::chrono::duration<double>(t1 - t0).count());
        // (b) the solver's pattern: enqueue j, then wait for and read j - 1
        cudaStreamSynchronize(r->st);
        t0 = std::chrono::steady_clock::now();
        volatile double sink = 0;
        for (int j = 0; j <= ncols; ++j) {
            if (j < ncols && I::enqueue_step(r, j, r->b, 1.0 / bn) != FFT_OK) return -5;
            if (j == 0) continue;
            const int k = j - 1;
            if (host_wait(r, r->slot_ev[k % 2]) != cudaSuccess) return -6;
            const double* slot = r->hslot + (size_t)(k % 2) * kSlot;
            std::vector<double> Hm((size_t)(ncols + 1) * ncols, 0.0);
            for (int l = 0; l <= k; ++l) Hm[(size_t)l * ncols + k] = slot[kSlotProv + l];
            Hm[(size_t)(k + 1) * ncols + k] = std::sqrt(std::max(slot[kSlotNorm], 0.0)) + 1.0;
            sink = sink + I::hess_lsq(Hm, ncols, k + 1, bn, nullptr);
        }
        cudaStreamSynchronize(r->st);
        t1 = std::chrono::steady_clock::now();
        best_b = std::min(best_b, std::chrono::duration<double>(t1 - t0).count());
    }
    out[0] = best_a / ncols * 1e3;
    out[1] = best_b / ncols * 1e3;
    return 0;
}
