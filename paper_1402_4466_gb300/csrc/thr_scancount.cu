// Pass A with ScanCount counters (Sec. 5.1 of Kaser & Lemire: one counter per
// row, incremented for every set bit of every input, then compared with T),
// partitioned to one 128-word subtile at a time as Sec. 5.1 suggests for a
// bounded number of counters.  Per warp 8192 byte counters (64 rows x 128
// words, byte b * 128 + w) live in shared memory; a ones-fill word adds one to
// all 64 rows of its word and is kept as a per-word count in a register.
// Only words that received increments are compared row by row, and their
// counters are cleared again.  Cost grows with the number of set bits: this
// is the path for very sparse inputs.  Counters are bytes, so the host uses
// it for n <= 255 only, and always counts ones (no zero counting).
#include "thr_launch.h"
#include "thr_query_kernel.cuh"

namespace thr {
namespace {

constexpr uint32_t kRowsPerWord = 64;
constexpr uint32_t kCounterBytes = kRowsPerWord * kGW;  // per warp

struct ScanCount {
    static constexpr bool kSymmetric = false;  // thresholds only
    static constexpr bool kInlineGroups = true;  // never in a group
    unsigned char* cnt;
    uint32_t lane;
    uint32_t cf[kRows];  // ones-fill words seen at the lane's word of row r
    uint32_t touched;    // bit r: the word of row r has counter increments

    __device__ __forceinline__ void begin() {
#pragma unroll
        for (int r = 0; r < kRows; ++r) cf[r] = 0;
        touched = 0;
    }
    __device__ __forceinline__ void add(const uint64_t (&v)[kGroup][kRows], uint32_t nvalid) {
#pragma unroll
        for (int j = 0; j < kGroup; ++j) {
            if (uint32_t(j) >= nvalid) break;
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                uint64_t x = v[j][r];
                if (x == ~0ull) {  // literals are never all ones: a ones fill
                    ++cf[r];
                } else if (x) {
                    touched |= 1u << r;
                    unsigned char* c = cnt + 32 * r + lane;
                    while (x) {  // one increment per set bit
                        const int b = __ffsll(static_cast<long long>(x)) - 1;
                        x &= x - 1;
                        ++c[b * kGW];
                    }
                }
            }
        }
    }
    __device__ __forceinline__ void finish(uint32_t thr, uint32_t, uint64_t (&o)[kRows]) {
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            if (!((touched >> r) & 1u)) {
                o[r] = cf[r] >= thr ? ~0ull : 0ull;
                continue;
            }
            unsigned char* c = cnt + 32 * r + lane;
            uint64_t res = 0;
            for (uint32_t b = 0; b < kRowsPerWord; ++b) {
                const uint32_t k = c[b * kGW];
                if (k + cf[r] >= thr) res |= 1ull << b;
                if (k) c[b * kGW] = 0;
            }
            o[r] = res;
        }
    }
};

__global__ void __launch_bounds__(kNT) k_scancount(const PassAParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CtaSmem& sm = *reinterpret_cast<CtaSmem*>(smem_raw);
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned char* cnt = smem_raw + sizeof(CtaSmem) + wid * kCounterBytes;
    for (uint32_t i = lane; i < kCounterBytes / 16; i += 32)
        reinterpret_cast<uint4*>(cnt)[i] = make_uint4(0, 0, 0, 0);
    __syncwarp();
    ScanCount count{cnt, lane, {0, 0, 0, 0}, 0};
    pass_a(p, sm, count);
}

constexpr size_t scancount_smem() { return sizeof(CtaSmem) + kNW * kCounterBytes; }

cudaError_t prepare() {
    static cudaError_t once = cudaFuncSetAttribute(
        k_scancount, cudaFuncAttributeMaxDynamicSharedMemorySize, int(scancount_smem()));
    return once;
}

}  // namespace

cudaError_t launch_scancount(const PassAParams& p, int grid, cudaStream_t st) {
    cudaError_t e = prepare();
    if (e != cudaSuccess) return e;
    k_scancount<<<grid, kNT, scancount_smem(), st>>>(p);
    return cudaGetLastError();
}

cudaError_t occupancy_scancount(int* blocks) {
    cudaError_t e = prepare();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_scancount, kNT,
                                                         scancount_smem());
}

}  // namespace thr
