// Autotuning of the batched pass-A launch: candidate launch configurations
// (work-item order, class merging, grid split; thr_batch.h) are timed on a
// sample batch and the fastest is stored per batch shape in the index.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <vector>

#include "thr_batch.h"

namespace thr {

uint32_t tune_key(bool multi_class, double mean_n) {
    uint32_t b = 0;
    uint64_t v = uint64_t(mean_n + 0.5);
    while (v) {
        ++b;
        v >>= 1;
    }
    return (multi_class ? 1u : 0u) | (b << 1);
}

uint32_t tune_lookup(const thr_index* idx, uint32_t key) {
    std::lock_guard<std::mutex> lk(idx->tune_mu);
    auto it = idx->tune.find(key);
    return it == idx->tune.end() ? 0u : it->second;
}

thr_status autotune(const thr_index* idx, const BatchInput& in, cudaStream_t st, uint32_t reps,
                    double* times, uint32_t* best, bool share) {
    // flush buffer: every timed run starts with inputs out of L2
    const size_t flush_bytes = size_t(256) << 20;
    void* flush = nullptr;
    cudaError_t e = cudaMallocAsync(&flush, flush_bytes, st);
    if (e != cudaSuccess) return report_error(THR_E_NOMEM, "autotune: flush buffer");
    // room for every result
    const uint64_t cap = uint64_t(in.nq) * (uint64_t(idx->W) + 1);
    uint64_t* pool = nullptr;
    if ((e = cudaMallocAsync(reinterpret_cast<void**>(&pool), 8 * cap, st)) != cudaSuccess) {
        cudaFreeAsync(flush, st);
        return report_error(THR_E_NOMEM, "autotune: result pool");
    }
    std::vector<uint64_t> off(in.nq), len(in.nq);
    uint64_t total = 0;
    double t_best = 1e300;
    uint32_t c_best = 0, key = 0;
    thr_status rs = THR_OK;
    for (uint32_t c = 0; c < kTuneCandidates && rs == THR_OK; ++c) {
        BatchOptions opt;
        opt.graph = true;
        opt.force_tune = int(c);
        opt.share = share;
        std::vector<double> t;
        for (uint32_t k = 0; k < reps + 1 && rs == THR_OK; ++k) {  // first run warms up
            if ((e = cudaMemsetAsync(flush, k & 0xFF, flush_bytes, st)) != cudaSuccess ||
                (e = cudaStreamSynchronize(st)) != cudaSuccess) {
                rs = report_error(THR_E_CUDA, "autotune: flush");
                break;
            }
            BatchStats stats;
            const auto t0 = std::chrono::steady_clock::now();
            rs = run_batch(idx, in, pool, cap, off.data(), len.data(), &total, st, opt, &stats);
            const auto t1 = std::chrono::steady_clock::now();
            key = stats.tune_key;  // the shape as the batch's planning sees it
            if (k) t.push_back(std::chrono::duration<double, std::milli>(t1 - t0).count());
        }
        if (rs != THR_OK) break;
        std::sort(t.begin(), t.end());
        const double med = t.empty() ? 0.0 : t[t.size() / 2];
        if (times) times[c] = med;
        if (med < t_best) {
            t_best = med;
            c_best = c;
        }
    }
    cudaFreeAsync(pool, st);
    cudaFreeAsync(flush, st);
    cudaStreamSynchronize(st);
    if (rs != THR_OK) return rs;
    // store the winner for the shape of the sample's first chunk
    {
        std::lock_guard<std::mutex> lk(idx->tune_mu);
        idx->tune[key] = c_best;
    }
    if (best) *best = c_best;
    return THR_OK;
}

}  // namespace thr
