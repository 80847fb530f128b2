// Passes B and C of the canonical re-encoding of the results of a chunk of
// queries (slots 0 .. Q-1).
//
// Pass A left, per slot s and 128-word subtile g, the result words in U
// (unless the subtile holds a single fill class) and the aggregate A_g over
// the monoid of thr_device.cuh (heads, literals, last head, boundary
// classes).  Pass B scans each slot's aggregates in order (word 0 of a
// bitmap always starts the first group) into the prefix before every
// subtile and the aggregate of the whole result, whose heads + literals are
// the encoded length; the last warp of the chunk then scans the lengths over
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

// Pass B, one launch, one warp per scan block of kScanBlock consecutive
// subtiles of a slot: each lane loads its kPer consecutive aggregates at
// once, the lanes' totals are scanned across the warp, and every subtile's
// exclusive prefix within the block (kEmpty in cls for the block's first
// subtile) and the block's total are stored.  The warp that takes the slot's
// last ticket (tick) then scans the slot's block totals into block prefixes
// and the aggregate of the whole result, and the warp that takes the
// chunk's last ticket (gtick) places the chunk's results in the pool and
// writes each one's final marker (the group that ends at word W).  The
// tickets only select who finishes: no warp waits for another.  Pass C
// joins block prefix and in-block prefix.
constexpr uint32_t kScanBlock = 256;
constexpr uint32_t kPer = kScanBlock / 32;  // subtiles per lane
constexpr uint32_t kEmpty = 1u << 8;

__device__ __forceinline__ RangeAgg load_agg(const WriteParams& w, uint32_t s, uint32_t g) {
    RangeAgg a = agg_load_plain(w.aggs + (uint64_t(s) * w.NG + g) * kAggWords);
    return g == 0 ? fix_first(a) : a;
}

// An aggregate another warp of this launch stored: read through L2.
__device__ __forceinline__ RangeAgg agg_load_l2(const uint32_t* p) {
    const uint4 x = __ldcg(reinterpret_cast<const uint4*>(p));
    const uint2 y = __ldcg(reinterpret_cast<const uint2*>(p + 4));
    RangeAgg a;
    a.start = x.x;
    a.nh = x.y;
    a.nl = x.z;
    a.lh = x.w;
    a.lp = y.x;
    a.cls = y.y;
    return a;
}

__global__ void __launch_bounds__(kNT) k_scan_aggs(WriteParams w) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t wi = uint64_t(blockIdx.x) * kNW + (threadIdx.x >> 5);
    const uint32_t NG = w.NG, NB = w.NB;
    if (wi >= uint64_t(w.Q) * NB) return;  // the whole warp
    const uint32_t s = uint32_t(wi / NB), blk = uint32_t(wi - uint64_t(s) * NB);
    const uint32_t g0 = blk * kScanBlock + kPer * lane;
    // 1. the block
    RangeAgg a[kPer];
#pragma unroll
    for (uint32_t i = 0; i < kPer; ++i)
        if (g0 + i < NG) a[i] = load_agg(w, s, g0 + i);
    RangeAgg inc{};
    bool ih = false;
#pragma unroll
    for (uint32_t i = 0; i < kPer; ++i)
        if (g0 + i < NG) {
            inc = ih ? agg_combine(inc, a[i]) : a[i];
            ih = true;
        }
    warp_scan(inc, ih, lane);
    RangeAgg E = shfl_up_agg(inc, 1);
    bool eh = __shfl_up_sync(~0u, ih ? 1u : 0u, 1) != 0u && lane > 0;
#pragma unroll
    for (uint32_t i = 0; i < kPer; ++i)
        if (g0 + i < NG) {
            RangeAgg out = E;
            if (!eh) out.cls = kEmpty;
            agg_store_plain(w.pref + (uint64_t(s) * NG + g0 + i) * kAggWords, out);
            E = eh ? agg_combine(E, a[i]) : a[i];
            eh = true;
        }
    const RangeAgg total = shfl_down_last(inc, 31);
    uint32_t last = 0;
    if (lane == 0) {
        agg_store_plain(w.bagg + (uint64_t(s) * NB + blk) * kAggWords, total);
        __threadfence();
        last = atomicAdd(w.tick + s, 1u) == NB - 1 ? 1u : 0u;
    }
    if (!__shfl_sync(~0u, last, 0)) return;
    __threadfence();
    // 2. the slot's last warp: exclusive prefixes of its block totals, 32 at
    // a time with the earlier ones carried
    RangeAgg carry{};
    bool ch = false;
    for (uint32_t b0 = 0; b0 < NB; b0 += 32) {
        const uint32_t bb = b0 + lane;
        RangeAgg x{};
        bool xh = bb < NB;
        if (xh) x = agg_load_l2(w.bagg + (uint64_t(s) * NB + bb) * kAggWords);
        warp_scan(x, xh, lane);
        const RangeAgg ex = shfl_up_agg(x, 1);
        const bool exh = __shfl_up_sync(~0u, xh ? 1u : 0u, 1) != 0u && lane > 0;
        RangeAgg Eb = carry;
        bool ebh = ch;
        if (exh) {
            Eb = ch ? agg_combine(carry, ex) : ex;
            ebh = true;
        }
        if (bb < NB) {
            if (!ebh) Eb.cls = kEmpty;
            agg_store_plain(w.bpref + (uint64_t(s) * NB + bb) * kAggWords, Eb);
        }
        const RangeAgg tot = shfl_down_last(x, 31);
        if (__shfl_sync(~0u, xh ? 1u : 0u, 31)) {
            carry = ch ? agg_combine(carry, tot) : tot;
            ch = true;
        }
    }
    last = 0;
    if (lane == 0) {  // carry covers the whole result of slot s
        agg_store_plain(w.full + uint64_t(s) * kAggWords, carry);
        w.tick[s] = 0;
        __threadfence();
        last = atomicAdd(w.gtick, 1u) == w.Q - 1 ? 1u : 0u;
    }
    if (!__shfl_sync(~0u, last, 0)) return;
    __threadfence();
    // 3. the chunk's last warp: place the results of its slots in the pool
    // and write the marker of each result's last group
    unsigned long long run = __ldcg(w.base);
    for (uint32_t s0 = 0; s0 < w.Q; s0 += 32) {
        const uint32_t t = s0 + lane;
        RangeAgg F{};
        unsigned long long len = 0;
        if (t < w.Q) {
            F = agg_load_l2(w.full + uint64_t(t) * kAggWords);
            len = uint64_t(F.nh) + F.nl;
        }
        unsigned long long incl = len;
#pragma unroll
        for (uint32_t d = 1; d < 32; d <<= 1) {
            const unsigned long long u = __shfl_up_sync(~0u, incl, d);
            if (lane >= d) incl += u;
        }
        const unsigned long long tot = __shfl_sync(~0u, incl, 31);
        if (t < w.Q && THR_CHK(w.chk, uint64_t(w.q0) + t < w.chk_nq, kChkResult,
                               uint64_t(w.q0) + t, w.chk_nq)) {
            const unsigned long long off = run + incl - len;
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
    if (lane == 0) {
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
    const uint64_t blocks = uint64_t(w.Q) * w.NB;  // one warp each
    k_scan_aggs<<<(blocks + kNW - 1) / kNW, kNT, 0, st>>>(w);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const uint64_t warps = uint64_t(w.Q) * w.NG;
    k_write_out<<<(warps + kNW - 1) / kNW, kNT, 0, st>>>(w);
    return cudaGetLastError();
}

}  // namespace thr
