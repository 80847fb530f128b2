// Launch entry points of the instantiated query kernels (one per counter
// width S), defined in thr_inst_*.cu so that they compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include "thr_device.cuh"

namespace thr {

using LaunchFn = cudaError_t (*)(const PassAParams&, int grid, cudaStream_t);
using OccupancyFn = cudaError_t (*)(int* blocks_per_sm);

struct KernelEntry {
    int S;
    LaunchFn launch;          // grouped decode, every word loaded from global memory
    OccupancyFn occupancy;
    LaunchFn launch_staged;   // staged inputs (thr_staged.cuh)
    OccupancyFn occupancy_staged;
    LaunchFn launch_pos;      // position-major decode of mixed inputs
    OccupancyFn occupancy_pos;
    LaunchFn launch_split;    // inputs split among the CTA's warps (S <= 8), or null
    OccupancyFn occupancy_split;
};

// Pass A with ScanCount counters (thr_scancount.cu), ones only: byte counters
// for n <= 255, 16-bit counters (wide) for n <= 65535.
cudaError_t launch_scancount(bool wide, const PassAParams&, int grid, cudaStream_t);
cudaError_t occupancy_scancount(bool wide, int* blocks_per_sm);

// Pass A with Looped levels (thr_inst_looped.cu), M = 1 .. kLoopedMax.
cudaError_t launch_looped(int M, const PassAParams&, int grid, cudaStream_t);
cudaError_t occupancy_looped(int M, int* blocks_per_sm);

// Instantiated counter widths, ascending; a query uses the first S with
// 2^S >= the largest threshold its counters test.
const KernelEntry* kernel_table(int* count);

#define THR_DECLARE_WIDTH(S)                                                 \
    cudaError_t launch_threshold_##S(const PassAParams&, int, cudaStream_t);     \
    cudaError_t occupancy_threshold_##S(int*);                                   \
    cudaError_t launch_threshold_pos_##S(const PassAParams&, int, cudaStream_t); \
    cudaError_t occupancy_threshold_pos_##S(int*);

#define THR_DECLARE_STAGED(S)                                              \
    cudaError_t launch_staged_##S(const PassAParams&, int, cudaStream_t);     \
    cudaError_t occupancy_staged_##S(int*);

THR_DECLARE_STAGED(1)
THR_DECLARE_STAGED(2)
THR_DECLARE_STAGED(3)
THR_DECLARE_STAGED(4)
THR_DECLARE_STAGED(5)
THR_DECLARE_STAGED(6)
THR_DECLARE_STAGED(7)
THR_DECLARE_STAGED(8)
THR_DECLARE_STAGED(10)
THR_DECLARE_STAGED(12)
THR_DECLARE_STAGED(16)
THR_DECLARE_STAGED(20)

#define THR_DECLARE_SPLIT(S)                                                \
    cudaError_t launch_split_##S(const PassAParams&, int, cudaStream_t);     \
    cudaError_t occupancy_split_##S(int*);

THR_DECLARE_SPLIT(1)
THR_DECLARE_SPLIT(2)
THR_DECLARE_SPLIT(3)
THR_DECLARE_SPLIT(4)
THR_DECLARE_SPLIT(5)
THR_DECLARE_SPLIT(6)
THR_DECLARE_SPLIT(7)
THR_DECLARE_SPLIT(8)

THR_DECLARE_WIDTH(1)
THR_DECLARE_WIDTH(2)
THR_DECLARE_WIDTH(3)
THR_DECLARE_WIDTH(4)
THR_DECLARE_WIDTH(5)
THR_DECLARE_WIDTH(6)
THR_DECLARE_WIDTH(7)
THR_DECLARE_WIDTH(8)
THR_DECLARE_WIDTH(10)
THR_DECLARE_WIDTH(12)
THR_DECLARE_WIDTH(16)
THR_DECLARE_WIDTH(20)

}  // namespace thr
