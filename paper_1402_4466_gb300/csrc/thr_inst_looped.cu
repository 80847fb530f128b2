// Pass-A kernels of the Looped variant, M = 1 .. kLoopedMax levels, and
// their launch and occupancy entry points.
#include "thr_exec.h"
#include "thr_launch.h"
#include "thr_query_kernel.cuh"

namespace thr {

namespace {

template <int M>
cudaError_t prepare_looped() {
    static cudaError_t once = cudaFuncSetAttribute(
        k_looped<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(cta_smem_bytes()));
    return once;
}

template <int M>
cudaError_t launch_m(const PassAParams& p, int grid, cudaStream_t st) {
    cudaError_t e = prepare_looped<M>();
    if (e != cudaSuccess) return e;
    k_looped<M><<<grid, kNT, cta_smem_bytes(), st>>>(p);
    return cudaGetLastError();
}

template <int M>
cudaError_t occupancy_m(int* blocks) {
    cudaError_t e = prepare_looped<M>();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_looped<M>, kNT,
                                                         cta_smem_bytes());
}

static_assert(kLoopedMax == 4, "instantiations below cover M = 1..4");

}  // namespace

cudaError_t launch_looped(int M, const PassAParams& p, int grid, cudaStream_t st) {
    switch (M) {
        case 1: return launch_m<1>(p, grid, st);
        case 2: return launch_m<2>(p, grid, st);
        case 3: return launch_m<3>(p, grid, st);
        case 4: return launch_m<4>(p, grid, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t occupancy_looped(int M, int* blocks) {
    switch (M) {
        case 1: return occupancy_m<1>(blocks);
        case 2: return occupancy_m<2>(blocks);
        case 3: return occupancy_m<3>(blocks);
        case 4: return occupancy_m<4>(blocks);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace thr
