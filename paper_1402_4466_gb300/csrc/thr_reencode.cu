// Passes B and C of the canonical re-encoding of the results of a chunk of
// queries (slots 0 .. Q-1).
//
// Pass A left, per slot s and 128-word subtile g, the result words in U
// (unless the subtile holds a single fill class) and the aggregate A_g over
// the monoid of thr_device.cuh (heads, literals, last head, boundary
// classes).  Pass B scans each slot's aggregates in order (word 0 of a
// bitmap always starts the first group) into the prefix before every
// subtile and the aggregate of the whole result, whose heads + literals are
// the encoded length; the last CTA of the chunk then scans the lengths over
// the slots, which places each result in the output pool after those of the
// earlier slots and chunks, and writes each result's final marker (the group
// that ends at word W).  Pass C gives every literal and every marker whose
// group ends inside subtile g its position: result offset + heads before +
// literals before.
#include "thr_query_kernel.cuh"

namespace thr {

namespace {


// Word 0 of the bitmap starts a group: the prefix up to and including
// subtile 0 counts it.
__device__ __forceinline__ RangeAgg fix_first(RangeAgg a) {
    a.nh += 1;
    if (!agg_has(a)) {
        a.lh = a.start;
        a.lp = 0;
        a.cls = (a.cls & 0xFu) | (agg_fc(a) << 4) | (1u << 6);
    }
    return a;
}

__device__ __forceinline__ RangeAgg shfl_up_agg(const RangeAgg& a, uint32_t d) {
    RangeAgg b;
    b.start = __shfl_up_sync(~0u, a.start, d);
    b.nh = __shfl_up_sync(~0u, a.nh, d);
    b.nl = __shfl_up_sync(~0u, a.nl, d);
    b.lh = __shfl_up_sync(~0u, a.lh, d);
    b.lp = __shfl_up_sync(~0u, a.lp, d);
    b.cls = __shfl_up_sync(~0u, a.cls, d);
    return b;
}

__device__ __forceinline__ RangeAgg shfl_down_last(const RangeAgg& a, uint32_t src) {
    RangeAgg b;
    b.start = __shfl_sync(~0u, a.start, src);
    b.nh = __shfl_sync(~0u, a.nh, src);
    b.nl = __shfl_sync(~0u, a.nl, src);
    b.lh = __shfl_sync(~0u, a.lh, src);
    b.lp = __shfl_sync(~0u, a.lp, src);
    b.cls = __shfl_sync(~0u, a.cls, src);
    return b;
}

// Inclusive ordered scan over the warp (lanes without a value are skipped).
__device__ __forceinline__ void warp_scan(RangeAgg& v, bool& have, uint32_t lane) {
#pragma unroll
    for (uint32_t d = 1; d < 32; d <<= 1) {
        const RangeAgg u = shfl_up_agg(v, d);
        const bool uh = __shfl_up_sync(~0u, have ? 1u : 0u, d) != 0u;
        if (lane >= d && uh) {
            v = have ? agg_combine(u, v) : u;
            have = true;
        }
    }
}

// Pass B, one launch: every CTA scans kScanBlock consecutive aggregates
// (one per thread) and stores each subtile's exclusive prefix within the
// block plus the block's total; the last CTA to finish (ticket in ctl[4])
// scans the block totals into block prefixes and writes the group that ends
// at word W and the total length.  Pass C joins block prefix and in-block
// prefix.  Empty values carry kEmpty in cls.
constexpr uint32_t kScanBlock = 256;
constexpr uint32_t kEmpty = 1u << 8;

__device__ __forceinline__ RangeAgg load_agg(const WriteParams& w, uint32_t s, uint32_t g) {
    RangeAgg a = agg_load_plain(w.aggs + (uint64_t(s) * w.NG + g) * kAggWords);
    return g == 0 ? fix_first(a) : a;
}

// Exclusive sum over the CTA (kScanBlock threads) and the total.
__device__ __forceinline__ unsigned long long block_exsum(unsigned long long v,
                                                          unsigned long long& total) {
    __shared__ unsigned long long wsum[kScanBlock / 32];
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long t = __shfl_up_sync(~0u, inc, d);
        if (lane >= uint32_t(d)) inc += t;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    unsigned long long before = 0;
    total = 0;
    for (uint32_t k = 0; k < kScanBlock / 32; ++k) {
        if (k < wid) before += wsum[k];
        total += wsum[k];
    }
    __syncthreads();
    return before + inc - v;
}

// Exclusive ordered scan over the CTA (kScanBlock threads); returns the
// exclusive prefix of this thread and the block total (in `total`).
__device__ __forceinline__ RangeAgg block_scan(RangeAgg v, bool vh, bool& eh, RangeAgg& total,
                                               bool& th) {
    __shared__ RangeAgg wagg[kScanBlock / 32];
    __shared__ uint32_t whave[kScanBlock / 32];
    constexpr uint32_t nwarps = kScanBlock / 32;
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    RangeAgg inc = v;
    bool ih = vh;
    warp_scan(inc, ih, lane);
    if (lane == 31) {
        wagg[wid] = inc;
        whave[wid] = ih;
    }
    __syncthreads();
    if (wid == 0) {
        RangeAgg x = lane < nwarps ? wagg[lane] : RangeAgg{};
        bool xh = lane < nwarps && whave[lane] != 0;
        warp_scan(x, xh, lane);
        const RangeAgg ex = shfl_up_agg(x, 1);
        const uint32_t xh_up = __shfl_up_sync(~0u, xh ? 1u : 0u, 1);  // every lane
        const RangeAgg last = shfl_down_last(x, nwarps - 1);
        const uint32_t lasth = __shfl_sync(~0u, xh ? 1u : 0u, nwarps - 1);
        __syncwarp();
        if (lane < nwarps) {
            wagg[lane] = ex;
            whave[lane] = lane > 0 && xh_up != 0u;
        }
        if (lane == 0) {
            wagg[0] = last;  // slot 0's exclusive prefix is empty: reuse it for the total
            whave[0] = lasth ? 2u : 0u;
        }
    }
    __syncthreads();
    total = wagg[0];
    th = (whave[0] & 2u) != 0;
    RangeAgg E = wagg[wid];
    eh = wid > 0 && (whave[wid] & 1u) != 0;
    const RangeAgg le = shfl_up_agg(inc, 1);
    const uint32_t ih_up = __shfl_up_sync(~0u, ih ? 1u : 0u, 1);  // every lane
    if (lane > 0 && ih_up != 0u) {
        E = eh ? agg_combine(E, le) : le;
        eh = true;
    }
    __syncthreads();
    return E;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_aggs(WriteParams w) {
    const uint32_t s = blockIdx.x / w.NB, b = blockIdx.x - s * w.NB;
    const uint32_t g = b * kScanBlock + threadIdx.x;
    RangeAgg a{};
    const bool ah = g < w.NG;
    if (ah) a = load_agg(w, s, g);
    bool eh, th;
    RangeAgg total;
    RangeAgg E = block_scan(a, ah, eh, total, th);
    if (ah) {
        if (!eh) E.cls = kEmpty;
        agg_store_plain(w.pref + (uint64_t(s) * w.NG + g) * kAggWords, E);
    }
    __shared__ bool last_block, last_slot;
    if (threadIdx.x == 0) {
        agg_store_plain(w.bagg + (uint64_t(s) * w.NB + b) * kAggWords, total);
        __threadfence();
        last_block = atomicAdd(w.tick + s, 1u) == w.NB - 1;
    }
    __syncthreads();
    if (!last_block) return;
    __threadfence();
    // the slot's last CTA: exclusive prefixes of its block totals
    RangeAgg carry{};
    bool ch = false;
    for (uint32_t b0 = 0; b0 < w.NB; b0 += kScanBlock) {
        const uint32_t bb = b0 + threadIdx.x;
        RangeAgg x{};
        const bool xh = bb < w.NB;
        if (xh) x = agg_load_plain(w.bagg + (uint64_t(s) * w.NB + bb) * kAggWords);
        bool ebh, cth;
        RangeAgg ctot;
        RangeAgg Eb = block_scan(x, xh, ebh, ctot, cth);
        if (ch) {  // prepend the totals of the earlier block groups
            Eb = ebh ? agg_combine(carry, Eb) : carry;
            ebh = true;
        }
        if (xh) {
            if (!ebh) Eb.cls = kEmpty;
            agg_store_plain(w.bpref + (uint64_t(s) * w.NB + bb) * kAggWords, Eb);
        }
        if (cth) {
            carry = ch ? agg_combine(carry, ctot) : ctot;
            ch = true;
        }
    }
    if (threadIdx.x == 0) {  // carry covers the whole result of slot s
        agg_store_plain(w.full + uint64_t(s) * kAggWords, carry);
        w.tick[s] = 0;
        __threadfence();
        last_slot = atomicAdd(w.gtick, 1u) == w.Q - 1;
    }
    __syncthreads();
    if (!last_slot) return;
    __threadfence();
    // the chunk's last CTA: place the results of its slots in the pool and
    // write the marker of each result's last group
    unsigned long long run = *w.base;
    for (uint32_t s0 = 0; s0 < w.Q; s0 += kScanBlock) {
        const uint32_t t = s0 + threadIdx.x;
        RangeAgg F{};
        unsigned long long len = 0;
        if (t < w.Q) {
            F = agg_load_plain(w.full + uint64_t(t) * kAggWords);
            len = uint64_t(F.nh) + F.nl;
        }
        unsigned long long tot;
        const unsigned long long ex = block_exsum(len, tot);
        if (t < w.Q && THR_CHK(w.chk, uint64_t(w.q0) + t < w.chk_nq, kChkResult,
                               uint64_t(w.q0) + t, w.chk_nq)) {
            const unsigned long long off = run + ex;
            w.res[2 * (uint64_t(w.q0) + t)] = off;
            w.res[2 * (uint64_t(w.q0) + t) + 1] = len;
            const uint64_t L = uint64_t(F.nl) - F.lp;
            const uint64_t Fw = uint64_t(w.W) - F.lh - L;
            const uint64_t bit = (Fw && agg_lhc(F) == 1u) ? 1ull : 0ull;
            const uint64_t pos = off + uint64_t(F.nh) - 1 + F.lp;
            if (pos < w.cap) w.out[pos] = bit | (Fw << 1) | (L << 33);
        }
        run += tot;
    }
    if (threadIdx.x == 0) {
        *w.base = run;
        *w.gtick = 0;
    }
}

// One warp per subtile.
__global__ void __launch_bounds__(kNT) k_write_out(WriteParams w) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t gi = uint64_t(blockIdx.x) * kNW + (threadIdx.x >> 5);
    const uint32_t s = uint32_t(gi / w.NG);
    if (s >= w.Q) return;
    const uint32_t g = uint32_t(gi - uint64_t(s) * w.NG);
    const uint64_t sg = uint64_t(s) * w.NG + g;
    if (!THR_CHK(w.chk, uint64_t(w.q0) + s < w.chk_nq, kChkResult, uint64_t(w.q0) + s,
                 w.chk_nq))
        return;
    const unsigned long long off = w.res[2 * (uint64_t(w.q0) + s)];
    const uint32_t x0 = g * uint32_t(kGW);
    const uint32_t x1 = min(x0 + uint32_t(kGW), w.W);
    const uint32_t xb = x0 + kWPL * lane;
    const RangeAgg A = agg_load_plain(w.aggs + sg * kAggWords);
    // prefix before the subtile, and whether its first word starts a group
    RangeAgg P;
    uint32_t hf;
    const uint32_t fc = agg_fc(A);
    if (g == 0) {
        P.start = P.nh = P.nl = P.lh = P.lp = P.cls = 0;
        hf = 1;
    } else {
        const RangeAgg inb = agg_load_plain(w.pref + sg * kAggWords);
        const uint32_t blk = g / kScanBlock;
        if (blk > 0) {
            const RangeAgg bp =
                agg_load_plain(w.bpref + (uint64_t(s) * w.NB + blk) * kAggWords);
            P = (inb.cls & kEmpty) ? bp : agg_combine(bp, inb);
        } else {
            P = inb;  // g > 0, so subtile 0 is before it in the block
        }
        hf = starts_group(agg_lc(P), fc) ? 1u : 0u;
    }
    if (!(A.nh || A.nl)) {
        // one fill class over the whole subtile: no literal and no group start
        // inside it; only the group that ends at its first word (when that
        // word starts a new group) gets its marker
        if (g > 0 && hf && lane == 0 && agg_has(P)) {
            const uint64_t Lw = uint64_t(P.nl) - P.lp;
            const uint64_t F = uint64_t(x0 - P.lh) - Lw;
            const uint64_t bit = (F && agg_lhc(P) == 1u) ? 1ull : 0ull;
            const uint64_t pos = off + uint64_t(P.nh) - 1 + P.lp;
            if (pos < w.cap) w.out[pos] = bit | (F << 1) | (Lw << 33);
        }
        return;
    }
    uint64_t o[kWPL];
    {
        const ulonglong2* src =
            reinterpret_cast<const ulonglong2*>(w.U + uint64_t(s) * w.NG * kGW + xb);
        const ulonglong2 a = src[0], b = src[1];
        o[0] = a.x;
        o[1] = a.y;
        o[2] = b.x;
        o[3] = b.y;
    }
    const LocalScan L = local_scan(x0, x1, lane, o);
    uint32_t J = P.nh + (lane ? hf : 0u) + L.eh;  // heads before xb
    uint32_t Lc = P.nl + L.el;                    // literals before xb
    uint32_t hp, hcls, lg;
    bool have_hp;
    if (L.ek) {
        hp = x0 + (L.ek >> 16) - 1;
        lg = P.nl + ((L.ek >> 2) & 0x3FFFu);
        hcls = L.ek & 3u;
        have_hp = true;
    } else if (hf && lane) {
        hp = x0;
        lg = P.nl;
        hcls = fc;
        have_hp = true;
    } else {
        hp = P.lh;
        lg = P.lp;
        hcls = agg_lhc(P);
        have_hp = g > 0 && agg_has(P);
    }
#pragma unroll
    for (int q = 0; q < kWPL; ++q) {
        if (xb + q >= x1) continue;
        const uint32_t x = xb + q;
        const uint32_t c = (L.clsbits >> (2 * q)) & 3u;
        const bool h = (lane == 0 && q == 0) ? (hf != 0) : ((L.headbits >> q) & 1u);
        if (h) {
            if (have_hp) {  // the previous group ends here: write its marker
                const uint64_t Lw = Lc - lg;
                const uint64_t F = uint64_t(x - hp) - Lw;
                const uint64_t b = (F && hcls == 1u) ? 1ull : 0ull;
                const uint64_t pos = off + uint64_t(J) - 1 + lg;
                if (pos < w.cap) w.out[pos] = b | (F << 1) | (Lw << 33);
            }
            hp = x;
            lg = Lc;
            hcls = c;
            have_hp = true;
            ++J;
        }
        if (c == 2u) {
            const uint64_t pos = off + uint64_t(J) + Lc;
            if (pos < w.cap) w.out[pos] = o[q];
            ++Lc;
        }
    }
}

}  // namespace

cudaError_t launch_reencode(const WriteParams& w, cudaStream_t st) {
    k_scan_aggs<<<uint64_t(w.Q) * w.NB, kScanBlock, 0, st>>>(w);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const uint64_t warps = uint64_t(w.Q) * w.NG;
    k_write_out<<<(warps + kNW - 1) / kNW, kNT, 0, st>>>(w);
    return cudaGetLastError();
}

}  // namespace thr
