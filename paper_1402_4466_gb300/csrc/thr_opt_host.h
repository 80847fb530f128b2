// Profiling pass of opt-threshold queries (thr_opt.cuh, thr_opt_host.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/thr.h"

struct thr_index;

namespace thr {
// For each query q of the batch (ids id_off[q] .. id_off[q+1], already
// checked), T[q] = the largest T whose T-overlap result holds at least K[q]
// rows (0 when none does).  Synchronises st; *ms (optional) receives the
// profiling kernels' time; *hist (optional) the per-query count histograms,
// n + 1 bins per query one after another, exact for every count >=
// max(T[q], 1).
thr_status opt_profile(const thr_index* idx, uint32_t nq, const uint32_t* id_off,
                       const uint32_t* ids, const uint64_t* K, uint32_t* T, cudaStream_t st,
                       float* ms, std::vector<unsigned long long>* hist = nullptr);
}  // namespace thr
