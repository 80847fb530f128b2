// Opt-threshold queries (Sec. 3.3, last paragraph): T is not given; the
// answer is the largest T whose T-overlap result holds at least K rows
// (K = 1: the largest count any row reaches), and that result.  Sec. 5.1
// gets it from ScanCount's counters (their maximum), Sec. 6.2 from Looped's
// C_i (the largest non-empty one), Sec. 5.2 by trying T = N, N - 1, ...
//
// Here the answer comes from one profiling pass over the carry-save
// counters of the threshold kernels, then one ordinary threshold query at
// that T.  The profiling pass (k_opt_profile<S>) builds, per query, a
// histogram of the counts that can still matter:
//   * lb[q] is a lower bound on the answer, 1 at the start; it only rises
//     to a count c that one subtile alone shows on at least K rows (so the
//     whole result at c holds K rows and the answer is >= c);
//   * a subtile whose counts cannot reach lb (k ones fills + d inputs with
//     literals < lb, or the finer position bound of the threshold kernels)
//     is skipped without counting;
//   * otherwise its counts are compared with c = max, max - 1, ... (the
//     bit-sliced ">= c" of the counters and a popcount), each exact-count
//     bin is added to hist[q][c], and the descent stops at lb or at the
//     first c that the subtile alone shows on K rows (lb rises to c).
// A seeding launch over every 16th subtile first raises lb without
// recording (a bound that one subtile proves holds whatever else is
// counted), so that the recording launch skips most subtiles from the start.
// Every subtile records every row whose count is at least the answer (its
// stopping point and lb never pass the answer), so the histogram's suffix
// sums from the top are exact down to the answer, and the host takes the
// first c (from n down) whose suffix holds K rows; 0 when none does.
// Counters are exact up to 2^S - 1.  The host first runs narrow counters
// (2^S > min(n, 15)); a subtile in which a row reaches 2^S (the sticky
// slice) records nothing and flags its query, which then runs again with
// 2^S > n.
#pragma once

#include "thr_query_kernel.cuh"

namespace thr {

struct OptParams {
    PassAParams a;                   // queries (QDesc sym = kSymProfile), index, list
    unsigned long long* hist;        // exact-count bins, query q at hist + hoff[q]
    const unsigned long long* hoff;  // per query: first bin (n + 1 bins each)
    uint32_t* lb;                    // per query: lower bound on the answer (1 at start)
    const unsigned long long* K;     // per query: rows wanted (>= 1)
    uint32_t stride;                 // subtiles 0, stride, 2 stride, ... of each query
    uint32_t record;                 // 0: only raise the bounds (seeding), 1: also the bins
    uint32_t exact;                  // 1: 2^S > n for every query of the launch
    uint32_t* ovf;                   // per query: set when a count reached 2^S (exact = 0)
};

// Occupancy bound: 4 CTAs per SM up to S = 6 (the narrow first pass runs
// with S <= 4), 3 up to S = 8, 2 beyond.
template <int S>
__global__ void __launch_bounds__(kNT, (S <= 6 ? 4 : (S <= 8 ? 3 : 2)))
    k_opt_profile(const OptParams o) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CtaSmem& sm = *reinterpret_cast<CtaSmem*>(smem_raw);
    const PassAParams& p = o.a;
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WarpSmem& ws = sm.w[wid];
    const QView q{ws, p.ids};
    CsaCount<S> count;
    const uint32_t nwarps = gridDim.x * kNW;
    const uint32_t ng = (p.NG + o.stride - 1) / o.stride;  // subtiles taken per query
    const uint32_t nitems = p.nlist * ng;
    uint32_t cur = ~0u;
    for (uint32_t it = blockIdx.x * kNW + wid; it < nitems; it += nwarps) {
        const uint32_t li = it / ng, g = (it - li * ng) * o.stride;
        const uint32_t s = __ldg(p.list + li);
        uint32_t L = 0;  // the bound as it stands now (other warps raise it)
        if (lane == 0) L = *reinterpret_cast<volatile const uint32_t*>(o.lb + s);
        L = __shfl_sync(~0u, L, 0);
        if (s != cur) {
            const QDesc d = p.qd[s];
            load_query(p, ws, d.ids_off, d.n, L, 0u, L, 0u, kSymProfile, lane);
            cur = s;
        } else {
            __syncwarp();
            if (lane == 0) {
                ws.qT = L;
                ws.qTx = L;
            }
            __syncwarp();
        }
        const uint32_t x0 = g * uint32_t(kGW);
        const uint32_t x1 = min(x0 + uint32_t(kGW), p.W);
        uint32_t k = 0, d = 0;
        count_subtile<CsaCount<S>, kFeedGrouped, false>(p, q, x0, x1, lane, ws, count, k, d);
        if (uint64_t(k) + d < L) continue;  // no row reaches the bound
        // valid rows of the lane's words (half h = 2 r + high word)
        uint32_t vm[8];
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const uint32_t x = x0 + 32 * r + lane;
            uint64_t m = x < p.W ? ~0ull : 0ull;
            if (x == p.W - 1 && p.ragged) m = (1ull << p.ragged) - 1;
            vm[2 * r] = uint32_t(m);
            vm[2 * r + 1] = uint32_t(m >> 32);
        }
        if (!o.exact && d > 0) {  // a count beyond the counters: this query runs again wider
            uint32_t sat = 0;
#pragma unroll
            for (int h = 0; h < 8; ++h) sat |= count.cnt.sticky[h] & vm[h];
            if (__any_sync(~0u, sat != 0)) {
                if (lane == 0) atomicOr(o.ovf + s, 1u);
                continue;
            }
        }
        const unsigned long long K = o.K[s];
        unsigned long long* hist = o.hist + o.hoff[s];
        if (d == 0) {  // every valid row counts k (>= L)
            uint32_t c = 0;
#pragma unroll
            for (int h = 0; h < 8; ++h) c += __popc(vm[h]);
            c = __reduce_add_sync(~0u, c);
            if (lane == 0) {
                if (o.record) atomicAdd(hist + k, (unsigned long long)c);
                if (c >= K) atomicMax(o.lb + s, k);
            }
            continue;
        }
        // the largest active count of a valid row: per half, keep the rows
        // with the highest bits, slice by slice from the top
        uint32_t mx = 0;
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            uint32_t m = vm[h], v = 0;
#pragma unroll
            for (int b = S - 1; b >= 0; --b) {
                const uint32_t t = m & count.cnt.c[b][h];
                if (t) {
                    m = t;
                    v |= 1u << b;
                }
            }
            if (vm[h]) mx = max(mx, v);
        }
        mx = __reduce_max_sync(~0u, mx);
        const uint32_t lo = L > k ? L - k : 0u;  // active counts below lo cannot matter
        uint32_t prev = 0;                        // rows with an active count above c
        for (int64_t c = mx; c >= int64_t(lo); --c) {
            uint32_t cnt = 0;
#pragma unroll
            for (int h = 0; h < 8; ++h)
                cnt += __popc((c == 0 ? ~0u : count.cnt.ge(h, uint32_t(c))) & vm[h]);
            cnt = __reduce_add_sync(~0u, cnt);
            if (lane == 0 && cnt > prev && o.record)
                atomicAdd(hist + k + uint32_t(c), (unsigned long long)(cnt - prev));
            prev = cnt;
            if (cnt >= K) {  // this subtile alone holds K rows counted >= k + c
                if (lane == 0) atomicMax(o.lb + s, k + uint32_t(c));
                break;
            }
        }
    }
}

// Launch entry points of the instantiated widths (thr_opt_a.cu, thr_opt_b.cu).
using OptLaunchFn = cudaError_t (*)(const OptParams&, int grid, cudaStream_t);
using OptOccupancyFn = cudaError_t (*)(int* blocks_per_sm);
struct OptEntry {
    int S;
    OptLaunchFn launch;
    OptOccupancyFn occupancy;
};
// Widths ascending; a query runs with the first S with 2^S > n.
const OptEntry* opt_kernel_table(int* count);

#define THR_DEFINE_OPT(S)                                                         \
    static cudaError_t prepare_opt_##S() {                                        \
        static cudaError_t once = cudaFuncSetAttribute(                           \
            k_opt_profile<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,        \
            int(cta_smem_bytes()));                                               \
        return once;                                                              \
    }                                                                             \
    cudaError_t launch_opt_##S(const OptParams& o, int grid, cudaStream_t st) {   \
        cudaError_t e = prepare_opt_##S();                                        \
        if (e != cudaSuccess) return e;                                           \
        k_opt_profile<S><<<grid, kNT, cta_smem_bytes(), st>>>(o);                 \
        return cudaGetLastError();                                                \
    }                                                                             \
    cudaError_t occupancy_opt_##S(int* blocks) {                                  \
        cudaError_t e = prepare_opt_##S();                                        \
        if (e != cudaSuccess) return e;                                           \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_opt_profile<S>, \
                                                             kNT, cta_smem_bytes()); \
    }

#define THR_DECLARE_OPT(S)                                                  \
    cudaError_t launch_opt_##S(const OptParams&, int, cudaStream_t);        \
    cudaError_t occupancy_opt_##S(int*);

}  // namespace thr
