// Pass A with ScanCount counters (Sec. 5.1 of Kaser & Lemire: one counter per
// row, incremented for every set bit of every input, then compared with T),
// partitioned to one 128-word subtile at a time as Sec. 5.1 suggests for a
// bounded number of counters.  Per warp 8192 counters (64 rows x 128 words,
// counter b * 128 + w) live in shared memory: bytes for n <= 255 inputs,
// 16-bit for n <= 65535 (the counter-width switch of Sec. 5.1).  A ones-fill
// word adds one to all 64 rows of its word and is kept as a per-word count in
// a register.  The lane also keeps, per word it owns, the OR of the literal
// words added there; only those bit positions are compared (and cleared
// again) at the end, so the cost follows the set bits: this is the path for
// very sparse inputs.  Ones only (no zero counting).
#include "thr_launch.h"
#include "thr_query_kernel.cuh"

namespace thr {
namespace {

constexpr uint32_t kRowsPerWord = 64;
template <class CT>
__host__ __device__ constexpr uint32_t counter_bytes() {  // per warp
    return kRowsPerWord * kGW * sizeof(CT);
}

template <class CT>
struct ScanCount {
    static constexpr bool kSymmetric = false;    // thresholds only
    static constexpr bool kInlineGroups = true;  // never in a group
    CT* cnt;
    uint32_t lane;
    uint32_t cf[kRows];     // ones-fill words seen at the lane's word of row r
    uint64_t seen[kRows];   // OR of the literal words added at that word

    __device__ __forceinline__ void begin() {
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            cf[r] = 0;
            seen[r] = 0;
        }
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
                    seen[r] |= x;
                    CT* c = cnt + 32 * r + lane;
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
            // rows never set in a literal have the ones-fill count alone
            uint64_t res = cf[r] >= thr ? ~seen[r] : 0ull;
            uint64_t x = seen[r];
            CT* c = cnt + 32 * r + lane;
            while (x) {
                const int b = __ffsll(static_cast<long long>(x)) - 1;
                x &= x - 1;
                if (uint32_t(c[b * kGW]) + cf[r] >= thr) res |= 1ull << b;
                c[b * kGW] = 0;
            }
            o[r] = res;
        }
    }
};

template <class CT>
__global__ void __launch_bounds__(kNT) k_scancount(const PassAParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CtaSmem& sm = *reinterpret_cast<CtaSmem*>(smem_raw);
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    CT* cnt = reinterpret_cast<CT*>(smem_raw + sizeof(CtaSmem) + wid * counter_bytes<CT>());
    for (uint32_t i = lane; i < counter_bytes<CT>() / 16; i += 32)
        reinterpret_cast<uint4*>(cnt)[i] = make_uint4(0, 0, 0, 0);
    __syncwarp();
    ScanCount<CT> count{cnt, lane, {0, 0, 0, 0}, {0, 0, 0, 0}};
    pass_a(p, sm, count);
}

template <class CT>
constexpr size_t scancount_smem() {
    return sizeof(CtaSmem) + kNW * counter_bytes<CT>();
}

template <class CT>
cudaError_t prepare() {
    static cudaError_t once = cudaFuncSetAttribute(
        k_scancount<CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(scancount_smem<CT>()));
    return once;
}

template <class CT>
cudaError_t launch(const PassAParams& p, int grid, cudaStream_t st) {
    cudaError_t e = prepare<CT>();
    if (e != cudaSuccess) return e;
    k_scancount<CT><<<grid, kNT, scancount_smem<CT>(), st>>>(p);
    return cudaGetLastError();
}

template <class CT>
cudaError_t occupancy(int* blocks) {
    cudaError_t e = prepare<CT>();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_scancount<CT>, kNT,
                                                         scancount_smem<CT>());
}

}  // namespace

cudaError_t launch_scancount(bool wide, const PassAParams& p, int grid, cudaStream_t st) {
    return wide ? launch<uint16_t>(p, grid, st) : launch<uint8_t>(p, grid, st);
}

cudaError_t occupancy_scancount(bool wide, int* blocks) {
    return wide ? occupancy<uint16_t>(blocks) : occupancy<uint8_t>(blocks);
}

}  // namespace thr
