// Instantiations of the split-input pass-A kernel, counter widths 1..8.
#include "thr_launch.h"
#include "thr_query_kernel.cuh"

#define THR_DEFINE_SPLIT(S)                                                   \
    static cudaError_t prepare_split_##S() {                                  \
        static cudaError_t once = cudaFuncSetAttribute(                       \
            k_threshold_split<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
            int(split_smem_bytes<S>()));                                      \
        return once;                                                          \
    }                                                                         \
    cudaError_t launch_split_##S(const PassAParams& p, int grid, cudaStream_t st) { \
        cudaError_t e = prepare_split_##S();                                  \
        if (e != cudaSuccess) return e;                                       \
        k_threshold_split<S><<<grid, kNT, split_smem_bytes<S>(), st>>>(p);    \
        return cudaGetLastError();                                            \
    }                                                                         \
    cudaError_t occupancy_split_##S(int* blocks) {                            \
        cudaError_t e = prepare_split_##S();                                  \
        if (e != cudaSuccess) return e;                                       \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(                 \
            blocks, k_threshold_split<S>, kNT, split_smem_bytes<S>());        \
    }

namespace thr {
THR_DEFINE_SPLIT(1)
THR_DEFINE_SPLIT(2)
THR_DEFINE_SPLIT(3)
THR_DEFINE_SPLIT(4)
THR_DEFINE_SPLIT(5)
THR_DEFINE_SPLIT(6)
THR_DEFINE_SPLIT(7)
THR_DEFINE_SPLIT(8)
}  // namespace thr
