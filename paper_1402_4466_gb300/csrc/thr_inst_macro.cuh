// Defines the launch and occupancy entry points of one counter width.  The
// kernel's shared state is dynamic shared memory (it exceeds 48 KB for the
// wider counters), so each entry first raises the kernel's limit once.
#pragma once

#include "thr_launch.h"
#include "thr_query_kernel.cuh"
#include "thr_staged.cuh"

// NAME: threshold (grouped decode) or threshold_pos (position-major decode
// of mixed inputs).
#define THR_DEFINE_KERNEL(S, POS, NAME)                                       \
    static cudaError_t prepare_##NAME##_##S() {                               \
        static cudaError_t once = cudaFuncSetAttribute(                       \
            k_threshold<S, POS>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
            int(cta_smem_bytes()));                                           \
        return once;                                                          \
    }                                                                         \
    cudaError_t launch_##NAME##_##S(const PassAParams& p, int grid,           \
                                    cudaStream_t st) {                        \
        cudaError_t e = prepare_##NAME##_##S();                               \
        if (e != cudaSuccess) return e;                                       \
        k_threshold<S, POS><<<grid, kNT, cta_smem_bytes(), st>>>(p);          \
        return cudaGetLastError();                                            \
    }                                                                         \
    cudaError_t occupancy_##NAME##_##S(int* blocks) {                         \
        cudaError_t e = prepare_##NAME##_##S();                               \
        if (e != cudaSuccess) return e;                                       \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(                 \
            blocks, k_threshold<S, POS>, kNT, cta_smem_bytes());              \
    }
#define THR_DEFINE_WIDTH(S) THR_DEFINE_KERNEL(S, kFeedGrouped, threshold)
#define THR_DEFINE_WIDTH_POS(S) THR_DEFINE_KERNEL(S, kFeedPos, threshold_pos)

// The staged carry-save kernel of counter width S (thr_staged.cuh).
#define THR_DEFINE_STAGED(S)                                                  \
    static cudaError_t prepare_staged_##S() {                                 \
        static cudaError_t once = cudaFuncSetAttribute(                       \
            k_staged<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,         \
            int(staged_smem_bytes()));                                        \
        return once;                                                          \
    }                                                                         \
    cudaError_t launch_staged_##S(const PassAParams& p, int grid, cudaStream_t st) { \
        cudaError_t e = prepare_staged_##S();                                 \
        if (e != cudaSuccess) return e;                                       \
        k_staged<S><<<grid, kNT, staged_smem_bytes(), st>>>(p);               \
        return cudaGetLastError();                                            \
    }                                                                         \
    cudaError_t occupancy_staged_##S(int* blocks) {                           \
        cudaError_t e = prepare_staged_##S();                                 \
        if (e != cudaSuccess) return e;                                       \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(                 \
            blocks, k_staged<S>, kNT, staged_smem_bytes());                   \
    }
