// Defines the launch and occupancy entry points of one counter width.
#pragma once

#include "thr_launch.h"
#include "thr_query_kernel.cuh"

#define THR_DEFINE_WIDTH(S)                                                   \
    cudaError_t launch_threshold_##S(const QueryParams& p, int grid,          \
                                     cudaStream_t st) {                       \
        k_threshold<S><<<grid, kNT, 0, st>>>(p);                              \
        return cudaGetLastError();                                            \
    }                                                                         \
    cudaError_t occupancy_threshold_##S(int* blocks) {                        \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(                 \
            blocks, k_threshold<S>, kNT, 0);                                  \
    }
