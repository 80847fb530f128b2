// Defines the launch and occupancy entry points of one counter width.  The
// kernel's shared state is dynamic shared memory (it exceeds 48 KB for the
// wider counters), so each entry first raises the kernel's limit once.
#pragma once

#include "thr_launch.h"
#include "thr_query_kernel.cuh"

#define THR_DEFINE_WIDTH(S)                                                   \
    static cudaError_t prepare_threshold_##S() {                              \
        static cudaError_t once = cudaFuncSetAttribute(                       \
            k_threshold<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
            int(cta_smem_bytes()));                                        \
        return once;                                                          \
    }                                                                         \
    cudaError_t launch_threshold_##S(const PassAParams& p, int grid,          \
                                     cudaStream_t st) {                       \
        cudaError_t e = prepare_threshold_##S();                              \
        if (e != cudaSuccess) return e;                                       \
        k_threshold<S><<<grid, kNT, cta_smem_bytes(), st>>>(p);            \
        return cudaGetLastError();                                            \
    }                                                                         \
    cudaError_t occupancy_threshold_##S(int* blocks) {                        \
        cudaError_t e = prepare_threshold_##S();                              \
        if (e != cudaSuccess) return e;                                       \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(                 \
            blocks, k_threshold<S>, kNT, cta_smem_bytes());                \
    }
