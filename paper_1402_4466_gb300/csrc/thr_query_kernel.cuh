// Pass A of a batch of threshold queries (see thr_device.cuh for the index
// layout and the outline): the counting kernels k_threshold<S> (carry-save,
// S = counter width; the host picks the smallest instantiated S with 2^S >=
// the threshold the counters test) and, in thr_scancount.cu, k_scancount.
#pragma once

#include "thr_device.cuh"

namespace thr {

// Active inputs decoded together (their loads are issued together).
constexpr int kGroup = 4;
// Rows of 32 words per subtile; lane owns one word of each row.
constexpr int kRows = kGW / 32;

// Per-warp scratch: the records of the active inputs of the current chunk.
// A record is {x, y} = first literal word (one literal run) or mask record
// index (mixed); {z, w} = stream offset of the bitmap (40 bits) | ones-fill
// flag << 62 | mixed flag << 63.
constexpr int kMetaBatch = 32;  // mask records staged per round trip

// What every pass-A kernel keeps per warp (the staged kernel: only this).
struct WarpCore {
    uint4 rec[kCH];
    unsigned long long tw[kGW];    // the subtile's result words, for the scan
    unsigned long long woff[kCH];  // stream offsets of the current query's ids
    uint32_t ids[kCH];             //   and the ids, when n <= kCH
    uint32_t qn, qT, qz, qoff;     // the current query: n, T, zmode, first id
    uint32_t qTx;                  //   largest threshold of its group (qT: the least)
    uint32_t qhi, qsym;            //   range bound and kind (QDesc)
    uint32_t qdir;                 //   QDesc::direct
};
// The direct kernels also stage mask records in shared memory.
struct WarpSmem : WarpCore {
    uint4 meta[kMetaBatch][4];     // mask records of kMetaBatch consecutive inputs
};

struct CtaSmem {
    WarpSmem w[kNW];
};

// The query a warp works on, read from its WarpSmem copy at every use (the
// loads are cheap; keeping the values in registers would spill).  cached:
// n <= kCH and ids / woff of WarpSmem hold its ids and their stream offsets.
struct QView {
    const volatile WarpCore& w;
    const uint32_t* all_ids;
    __device__ __forceinline__ uint32_t n() const { return w.qn; }
    __device__ __forceinline__ uint32_t T() const { return w.qT; }
    __device__ __forceinline__ uint32_t Tmax() const { return w.qTx; }
    __device__ __forceinline__ uint32_t hi() const { return w.qhi; }
    __device__ __forceinline__ uint32_t sym() const { return w.qsym; }
    // Is the subtile decided by k ones fills and d inputs with literals
    // (every row's count lies in [k, k + d]): all ones or all zeros, for
    // every threshold of a group?
    __device__ __forceinline__ bool decided(uint32_t k, uint32_t d) const {
        const uint32_t s = w.qsym;
        const int64_t lo = int64_t(w.qT) - int64_t(k);
        if (s == kSymOdd) return d == 0;
        // profiling pass: nothing reaches the bound, or no input to count
        if (s == kSymProfile) return lo > int64_t(d) || d == 0;
        if (s == kSymRange)
            return int64_t(w.qhi) < int64_t(k) || lo > int64_t(d) ||
                   (lo <= 0 && int64_t(k) + int64_t(d) <= int64_t(w.qhi));
        return int64_t(w.qTx) <= int64_t(k) || lo > int64_t(d);
    }
    __device__ __forceinline__ uint32_t zmode() const { return w.qz; }
    __device__ __forceinline__ const uint32_t* ids() const { return all_ids + w.qoff; }
    __device__ __forceinline__ bool cached() const { return w.qn <= uint32_t(kCH); }
    __device__ __forceinline__ bool direct() const { return w.qdir != 0u; }
};

constexpr size_t cta_smem_bytes() { return sizeof(CtaSmem); }

// How a kernel decodes (the kFeed parameter of pass_a and count_subtile):
// kFeedGrouped four inputs at a time, kFeedPos mixed inputs position-major.
constexpr int kFeedGrouped = 0, kFeedPos = 1;


// Values of up to kGroup active inputs (records r0 ..) at the lane's words
// x0 + 32 r + lane (row r = 0..3).  A literal run is read as four coalesced
// 256-byte rows.  For a mixed input, word x0 + 32 r + lane is a literal iff
// bit `lane` of lm[r] of its 64-byte mask record, and sits at stream index
// base + pre[r] + popc(cm[r] below lane); other words are ones (om bit) or
// zero, and rows without literals or ones are skipped.  The group's mask records are staged in
// shared memory first (one 16-byte load per lane), then every literal load
// of the group is issued.
// A literal word of an input stream: each is read once per query, so it is
// loaded without allocating a line in L1, which keeps the reused packed
// classes, descriptors and mask records there (3-5% faster pass A on the
// many-criteria queries).
__device__ __forceinline__ uint64_t ld_literal(const PassAParams& p, const uint64_t* a) {
    if (!THR_CHK(p.chk, uint64_t(a - p.words) < p.lim.words, kChkLiteral, a - p.words,
                 p.lim.words))
        return 0;
    uint64_t v;
    asm volatile("ld.global.nc.L1::no_allocate.u64 %0, [%1];" : "=l"(v) : "l"(a));
    return v;
}

// Stage the mask records of inputs m0 .. m0 + kMetaBatch - 1 (lane: 16
// bytes of 4 records); literal runs and absent ones-fill masks are skipped.
__device__ __forceinline__ void stage_masks(const PassAParams& p, WarpSmem& ws, uint32_t m0,
                                           uint32_t nrec, uint32_t lane) {
    const uint32_t part = lane & 3;
#pragma unroll
    for (int k = 0; k < kMetaBatch / 8; ++k) {
        const uint32_t j = (lane >> 2) + 8 * k;
        if (m0 + j < nrec) {
            const uint4 rec = ws.rec[m0 + j];
            const uint64_t mi = (uint64_t(rec.y) << 32) | rec.x;
            if ((rec.w >> 31) && (part != 2 || ((rec.w >> 30) & 1u)) &&
                THR_CHK(p.chk, mi < p.lim.masks, kChkMask, mi, p.lim.masks)) {
                const uint4* m = reinterpret_cast<const uint4*>(p.masks + mi);
                ws.meta[j][part] = __ldg(m + part);
            }
        }
    }
    __syncwarp();
}

__device__ __forceinline__ void decode_group(const PassAParams& p, WarpSmem& ws,
                                             uint32_t r0, uint32_t nrec, uint32_t x0,
                                             uint32_t x1, uint32_t lane,
                                             uint64_t (&v)[kGroup][kRows]) {
    const uint32_t bit = 1u << lane;
    const uint32_t lt = bit - 1u;
    const uint32_t mb = r0 % kMetaBatch;  // the group's first slot in the staged batch
    if (!THR_CHK(p.chk, mb + kGroup <= uint32_t(kMetaBatch), kChkMeta, mb, kMetaBatch)) {
#pragma unroll
        for (int j = 0; j < kGroup; ++j)
#pragma unroll
            for (int r = 0; r < kRows; ++r) v[j][r] = 0;
        return;
    }
#pragma unroll
    for (int j = 0; j < kGroup; ++j) {
#pragma unroll
        for (int r = 0; r < kRows; ++r) v[j][r] = 0;
        if (r0 + j >= nrec) continue;
        const uint4 rec = ws.rec[r0 + j];
        const uint64_t ra = (uint64_t(rec.y) << 32) | rec.x;
        if (!(rec.w >> 31)) {  // one literal run covers the subtile
            const uint64_t* src = p.words + ra + lane;
#pragma unroll
            for (int r = 0; r < kRows; ++r)
                if (x0 + 32 * r + lane < x1) v[j][r] = ld_literal(p, src + 32 * r);
            continue;
        }
        const uint4 lmv = ws.meta[mb + j][0], cmv = ws.meta[mb + j][1], bp = ws.meta[mb + j][3];
        const uint64_t* src = p.words + ((uint64_t(rec.w & 0xFFu) << 32) | rec.z) + bp.x;
        const uint32_t lm[4] = {lmv.x, lmv.y, lmv.z, lmv.w};
        const uint32_t cm[4] = {cmv.x, cmv.y, cmv.z, cmv.w};
        if ((rec.w >> 30) & 1u) {  // has ones-fill words in this subtile
            const uint4 omv = ws.meta[mb + j][2];
            const uint32_t om[4] = {omv.x, omv.y, omv.z, omv.w};
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                if ((lm[r] | om[r]) == 0u) continue;  // the row is all zero fill
                const uint32_t off = ((bp.y >> (8 * r)) & 0xFFu) + __popc(cm[r] & lt);
                v[j][r] = (lm[r] & bit) ? ld_literal(p, src + off) : ((om[r] & bit) ? ~0ull : 0ull);
            }
        } else {
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                if (lm[r] == 0u) continue;  // the row is all zero fill
                const uint32_t off = ((bp.y >> (8 * r)) & 0xFFu) + __popc(cm[r] & lt);
                if (lm[r] & bit) v[j][r] = ld_literal(p, src + off);
            }
        }
    }
    __syncwarp();
}

// 32 x 32 bit transpose across the warp: bit j of lane L's result is bit L
// of lane j's x (five rounds of swapping the off-diagonal blocks).
__device__ __forceinline__ uint32_t transpose32(uint32_t x, uint32_t lane) {
    constexpr uint32_t kHi[5] = {0xFFFF0000u, 0xFF00FF00u, 0xF0F0F0F0u, 0xCCCCCCCCu, 0xAAAAAAAAu};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const uint32_t sft = 16u >> k, m = kHi[k];
        const uint32_t y = __shfl_xor_sync(~0u, x, sft);
        x = (lane & sft) ? ((x & m) | ((y & m) >> sft)) : ((x & ~m) | ((y & ~m) << sft));
    }
    return x;
}

// Position-major decode of nb <= 32 mixed inputs (records rec[kCH-1-m0-j],
// j < nb) into the counters, counting ones.  Per row, the literal and
// ones-fill masks of the inputs are transposed so that each lane holds the
// set of inputs with a literal (or a ones-fill word) at its own word of that
// row; every round then takes up to four inputs from each of the lane's four
// sets (16 loads in flight) and the warp adds them.  Rounds = the largest
// set in the warp divided by four, not nb: sparse inputs cost their
// literals, not a full pass each.
template <class Count>
__device__ __forceinline__ void pos_batch(const PassAParams& p, WarpSmem& ws, uint32_t m0,
                                          uint32_t nb, uint32_t lane, Count& count) {
    // stage the batch's 64-byte mask records (skipping absent ones-fill masks)
    const uint32_t part = lane & 3;
#pragma unroll
    for (int k = 0; k < kMetaBatch / 8; ++k) {
        const uint32_t j = (lane >> 2) + 8 * k;
        if (j < nb) {
            const uint4 rec = ws.rec[kCH - 1 - (m0 + j)];
            const uint64_t mi = (uint64_t(rec.y) << 32) | rec.x;
            if ((part != 2 || ((rec.w >> 30) & 1u)) &&
                THR_CHK(p.chk, mi < p.lim.masks, kChkMask, mi, p.lim.masks)) {
                const uint4* m = reinterpret_cast<const uint4*>(p.masks + mi);
                ws.meta[j][part] = __ldg(m + part);
            }
        }
    }
    __syncwarp();
    const bool mine = lane < nb;
    const uint4 myrec = mine ? ws.rec[kCH - 1 - (m0 + lane)] : make_uint4(0, 0, 0, 0);
    const bool has_om = mine && ((myrec.w >> 30) & 1u);
    const bool any_om = __any_sync(~0u, has_om);
    if (mine) {  // stream index of the record's first literal into its pad words
        const uint64_t wb = ((uint64_t(myrec.w & 0xFFu) << 32) | myrec.z) + ws.meta[lane][3].x;
        ws.meta[lane][3].z = uint32_t(wb);
        ws.meta[lane][3].w = uint32_t(wb >> 32);
    }
    uint32_t have[kRows], ones[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const uint32_t lmr = mine ? reinterpret_cast<const uint32_t*>(&ws.meta[lane][0])[r] : 0u;
        const uint32_t omr = has_om ? reinterpret_cast<const uint32_t*>(&ws.meta[lane][2])[r] : 0u;
        ones[r] = any_om ? transpose32(omr, lane) : 0u;
        have[r] = transpose32(lmr, lane) | ones[r];
    }
    __syncwarp();
    const uint32_t lt = (1u << lane) - 1u;
    while (__any_sync(~0u, (have[0] | have[1] | have[2] | have[3]) != 0u)) {
        uint64_t v[kGroup][kRows];
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
#pragma unroll
            for (int k = 0; k < kGroup; ++k) {
                v[k][r] = 0;
                if (have[r]) {
                    const uint32_t j = __ffs(have[r]) - 1;
                    have[r] &= have[r] - 1u;
                    if ((ones[r] >> j) & 1u) {
                        v[k][r] = ~0ull;
                    } else {
                        const uint4 m3 = ws.meta[j][3];
                        const uint32_t cm = reinterpret_cast<const uint32_t*>(&ws.meta[j][1])[r];
                        const uint64_t at = ((uint64_t(m3.w) << 32) | m3.z) +
                                            ((m3.y >> (8 * r)) & 0xFFu) + __popc(cm & lt);
                        v[k][r] = ld_literal(p, p.words + at);
                    }
                }
            }
        }
        count.add(v, kGroup);
    }
    __syncwarp();
}

// Counting policy of the carry-save path: bit-sliced counters in registers
// (Counters<S>), inputs added four at a time, "count >= thr" compared slice
// by slice.
static_assert(kGroup == 2 || kGroup == 4, "inputs are added in fours or twos");

template <int S>
struct CsaCount {
    static constexpr bool kSymmetric = true;  // range and parity tests
    // group members finished inline: below 7 bits the 4-CTA register bound
    // applies anyway; wider counters finish them out of line (finish_group)
    static constexpr bool kInlineGroups = S <= 6;
    Counters<S> cnt;
    // the lowest slice is the parity of the count (never saturated)
    __device__ __forceinline__ void parity(uint64_t (&o)[kRows], uint32_t flip) const {
#pragma unroll
        for (int r = 0; r < kRows; ++r)
            o[r] = (uint64_t(cnt.c[0][2 * r + 1] ^ flip) << 32) | (cnt.c[0][2 * r] ^ flip);
    }
    __device__ __forceinline__ void begin() { cnt.clear(); }
    __device__ __forceinline__ void add(const uint64_t (&v)[kGroup][kRows], uint32_t) {
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            if constexpr (kGroup == 4) {
                cnt.add4(2 * r, uint32_t(v[0][r]), uint32_t(v[1][r]), uint32_t(v[2][r]),
                         uint32_t(v[3][r]));
                cnt.add4(2 * r + 1, uint32_t(v[0][r] >> 32), uint32_t(v[1][r] >> 32),
                         uint32_t(v[2][r] >> 32), uint32_t(v[3][r] >> 32));
            } else {
                cnt.add_pair(2 * r, uint32_t(v[0][r]), uint32_t(v[1][r]));
                cnt.add_pair(2 * r + 1, uint32_t(v[0][r] >> 32), uint32_t(v[1][r] >> 32));
            }
        }
    }
    // 1 <= thr <= 2^S; flip inverts the result (counting zeros)
    __device__ __forceinline__ void finish(uint32_t thr, uint32_t flip, uint64_t (&o)[kRows]) {
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            const uint32_t lo = cnt.ge(2 * r, thr) ^ flip;
            const uint32_t hi = cnt.ge(2 * r + 1, thr) ^ flip;
            o[r] = (uint64_t(hi) << 32) | lo;
        }
    }
};

// Counting policy of the Looped variant (Algorithm 3, Sec. 6.2): M bitmaps
// C_1 .. C_M per 32-bit half word, C_j holding the rows counted at least j
// times so far.  An input x updates C_j |= C_(j-1) & x for j = M .. 2 (one
// LOP3 each), then C_1 |= x; the rows reaching T' <= M are C_(T').  Ones
// only (the host never sets zmode for it); absent inputs of a group are zero
// words, which change nothing.
template <int M>
struct LoopedCount {
    static constexpr bool kSymmetric = false;    // thresholds only
    static constexpr bool kInlineGroups = true;  // never in a group
    uint32_t C[M][8];
    __device__ __forceinline__ void begin() {
#pragma unroll
        for (int j = 0; j < M; ++j)
#pragma unroll
            for (int h = 0; h < 8; ++h) C[j][h] = 0;
    }
    __device__ __forceinline__ void add(const uint64_t (&v)[kGroup][kRows], uint32_t) {
#pragma unroll
        for (int i = 0; i < kGroup; ++i)
#pragma unroll
            for (int h = 0; h < 8; ++h) {
                const uint32_t x = uint32_t(v[i][h >> 1] >> (32 * (h & 1)));
#pragma unroll
                for (int j = M - 1; j >= 1; --j) C[j][h] = lop3<kOrAnd>(C[j][h], C[j - 1][h], x);
                C[0][h] |= x;
            }
    }
    // 1 <= thr <= M; flip inverts the result
    __device__ __forceinline__ void finish(uint32_t thr, uint32_t flip, uint64_t (&o)[kRows]) {
#pragma unroll
        for (int r = 0; r < kRows; ++r) {
            uint32_t lo = 0, hi = 0;
#pragma unroll
            for (int j = 0; j < M; ++j)
                if (uint32_t(j + 1) == thr) {
                    lo = C[j][2 * r];
                    hi = C[j][2 * r + 1];
                }
            o[r] = (uint64_t(hi ^ flip) << 32) | (lo ^ flip);
        }
    }
};

// One warp computes the 128 result words of subtile [x0, x1); lane owns rows
// r = 0..3, words x0 + 32 r + lane (zero past x1).  Count is the counting
// policy (carry-save bit slices, or ScanCount counters).  kPos: mixed inputs
// go through the position-major decode (ones counting; the host never sets
// zmode for these kernels), literal runs through the grouped one.
// The largest number of inputs with a non-zero word at one position of the
// subtile: a literal run counts at every position, a mixed input where its
// literal or ones-fill mask is set (32 inputs' masks bit-transposed across
// the warp per row, then counted).  Records as the classification left
// them (literal runs first and mixed inputs from the back with kPos).
template <bool kPos>
__device__ __forceinline__ uint32_t max_position_count(const PassAParams& p, const WarpSmem& ws,
                                                       uint32_t nrec, uint32_t nrun,
                                                       uint32_t nmix, uint32_t lane) {
    uint32_t c[kRows] = {0, 0, 0, 0};
    uint32_t runs = kPos ? nrun : 0u;
    const uint32_t total = kPos ? nmix : nrec;
    for (uint32_t m0 = 0; m0 < total; m0 += 32) {
        const uint32_t j = m0 + lane;
        uint32_t mk[kRows] = {0, 0, 0, 0};
        bool run = false;
        if (j < total) {
            const uint4 rec = kPos ? ws.rec[kCH - 1 - j] : ws.rec[j];
            const uint64_t mi = (uint64_t(rec.y) << 32) | rec.x;
            if (!(rec.w >> 31)) {
                run = true;
            } else if (THR_CHK(p.chk, mi < p.lim.masks, kChkMask, mi, p.lim.masks)) {
                const uint4* m = reinterpret_cast<const uint4*>(p.masks + mi);
                const uint4 lm = __ldg(m);
                mk[0] = lm.x;
                mk[1] = lm.y;
                mk[2] = lm.z;
                mk[3] = lm.w;
                if ((rec.w >> 30) & 1u) {
                    const uint4 om = __ldg(m + 2);
                    mk[0] |= om.x;
                    mk[1] |= om.y;
                    mk[2] |= om.z;
                    mk[3] |= om.w;
                }
            }
        }
        if (!kPos) runs += __popc(__ballot_sync(~0u, run));
#pragma unroll
        for (int r = 0; r < kRows; ++r) c[r] += __popc(transpose32(mk[r], lane));
    }
    const uint32_t m = max(max(c[0], c[1]), max(c[2], c[3])) + runs;
    return __reduce_max_sync(~0u, m);
}

// Counting part of a subtile's result: classify the query's inputs over the
// subtile, count k (ones fills) and d (inputs with literals) and add the
// active inputs into `count`.  kPart: the inputs are one part of a query
// whose other parts other warps count, so the totals are not known and the
// subtile is never pruned here.
template <class Count, int kFeed = kFeedGrouped, bool kPart = false>
__device__ __forceinline__ void count_subtile(const PassAParams& p, const QView& q,
                                              uint32_t x0, uint32_t x1, uint32_t lane,
                                              WarpSmem& ws, Count& count, uint32_t& k_ones,
                                              uint32_t& d_act) {
    constexpr bool kPos = kFeed == kFeedPos;
    const uint32_t g = x0 / kGW;
    count.begin();
    k_ones = 0;
    d_act = 0;
    const bool one_chunk = q.n() <= uint32_t(kCH);
    bool pruned = false;
    if (!one_chunk && !kPart) {  // classify every input first so that pruning still applies
        for (uint32_t i0 = 0; i0 < q.n(); i0 += 32) {
            const uint32_t i = i0 + lane;
            uint32_t cls = 0;
            if (i < q.n()) {
                const uint64_t ii = uint64_t(q.ids() + i - p.ids);
                const uint32_t b = THR_CHK(p.chk, ii < p.lim.nids, kChkIdIndex, ii, p.lim.nids)
                                       ? __ldg(q.ids() + i)
                                       : 0u;
                if (THR_CHK(p.chk, b < p.lim.nb, kChkIdValue, b, p.lim.nb))
                    cls = uint32_t(__ldg(p.pcls + uint64_t(b) * p.NGW + (g >> 5)) >>
                                   (2 * (g & 31))) & 3u;
            }
            k_ones += __popc(__ballot_sync(~0u, cls == 1));
            d_act += __popc(__ballot_sync(~0u, cls >= 2));
        }
        pruned = q.decided(k_ones, d_act);
    }
    for (uint32_t c0 = 0; c0 < q.n() && !pruned; c0 += kCH) {
        const uint32_t cn = min(uint32_t(kCH), q.n() - c0);
        uint32_t nrec = 0, nrun = 0, nmix = 0;
        // 1. classify, lane per input, from the subtile descriptor: the
        // packed classes of every round of 32 inputs first, then the full
        // descriptors of the inputs with literals, so that each kind of load
        // is in flight for all rounds at once (two dependent round trips
        // per chunk instead of two per round).  A query whose inputs hold
        // literals in most subtiles (QDesc::direct, set by the planner)
        // loads every input's descriptor at once instead, whose low bits
        // are the class: one round trip, at 8 bytes per input and subtile
        // (pass A 2-3% faster on the many-criteria queries; a sparse query
        // would read far more than its packed classes)
        constexpr int kRounds = kCH / 32;
        const bool cached = q.cached();
        const bool direct = q.direct();
        const uint32_t* qids = q.ids() + c0;
        uint32_t cb[kRounds], cc[kRounds];
#pragma unroll
        for (int k = 0; k < kRounds; ++k) {
            const uint32_t i = 32u * k + lane;
            cb[k] = 0;
            cc[k] = 0;  // 0 zero fill, 1 ones fill, 2 literal run, 3 mixed
            if (i < cn) {
                const uint64_t ii = uint64_t(qids + i - p.ids);
                cb[k] = cached ? ws.ids[i]
                               : (THR_CHK(p.chk, ii < p.lim.nids, kChkIdIndex, ii, p.lim.nids)
                                      ? __ldg(qids + i)
                                      : 0u);
                if (THR_CHK(p.chk, cb[k] < p.lim.nb, kChkIdValue, cb[k], p.lim.nb) &&
                    THR_CHK(p.chk, g < p.NG, kChkSubtile, g, p.NG)) {
                    if (direct)
                        cc[k] = 4u;  // the descriptor loaded next holds the class
                    else
                        cc[k] = uint32_t(__ldg(p.pcls + uint64_t(cb[k]) * p.NGW + (g >> 5)) >>
                                         (2 * (g & 31))) & 3u;
                }
            }
        }
        uint64_t sdv[kRounds], wov[kRounds];
#pragma unroll
        for (int k = 0; k < kRounds; ++k) {
            sdv[k] = 0;
            wov[k] = 0;
            if (cc[k] >= 2) {
                sdv[k] = __ldg(p.sdesc + uint64_t(cb[k]) * p.NG + g);
                wov[k] = cached ? ws.woff[32u * k + lane] : p.desc[cb[k]].woff;
            }
            if (cc[k] == 4u) cc[k] = uint32_t(sdv[k] & 3u);
        }
#pragma unroll
        for (int k = 0; k < kRounds; ++k) {
            if (32u * k >= cn) break;
            const uint32_t cls = cc[k];
            uint4 r = make_uint4(0, 0, 0, 0);
            {
                if (cls >= 2) {
                    const uint64_t sd = sdv[k];
                    const uint64_t woff = wov[k];
                    const uint64_t field = sd >> 19;
                    if (cls == 2) {
                        const uint64_t ra = woff + field;
                        r = make_uint4(uint32_t(ra), uint32_t(ra >> 32), 0u, 0u);
                    } else {
                        r = make_uint4(uint32_t(field), uint32_t(field >> 32), uint32_t(woff),
                                       uint32_t(woff >> 32) | (uint32_t(sd & 4u) << 28) |
                                           (1u << 31));
                    }
                }
            }
            if (one_chunk || kPart) k_ones += __popc(__ballot_sync(~0u, cls == 1));
            if constexpr (kPos) {  // literal runs from the front, mixed from the back
                const uint32_t a2 = __ballot_sync(~0u, cls == 2);
                const uint32_t a3 = __ballot_sync(~0u, cls == 3);
                const uint32_t below = (1u << lane) - 1u;
                const uint32_t s2 = nrun + __popc(a2 & below), s3 = nmix + __popc(a3 & below);
                if (cls == 2 && THR_CHK(p.chk, s2 < uint32_t(kCH), kChkRecord, s2, kCH))
                    ws.rec[s2] = r;
                if (cls == 3 && THR_CHK(p.chk, s3 < uint32_t(kCH), kChkRecord, s3, kCH))
                    ws.rec[kCH - 1 - s3] = r;
                nrun += __popc(a2);
                nmix += __popc(a3);
                nrec = nrun + nmix;
            } else {
                const uint32_t act = __ballot_sync(~0u, cls >= 2);
                const uint32_t sr = nrec + __popc(act & ((1u << lane) - 1u));
                if (cls >= 2 && THR_CHK(p.chk, sr < uint32_t(kCH), kChkRecord, sr, kCH))
                    ws.rec[sr] = r;
                nrec += __popc(act);
            }
        }
        __syncwarp();
        if (one_chunk) {  // run-aware pruning (Sec. 6.4 cases 1 and 2)
            d_act = nrec;
            // decided for every threshold of the group: all ones or all zeros
            if (!kPart && q.decided(k_ones, d_act)) break;
            // finer: no word of the subtile is non-zero in T' inputs, so no
            // row reaches T' (checked when T' is a fair share of d)
            const int64_t tp = int64_t(q.T()) - int64_t(k_ones);
            if (!kPart && q.sym() != kSymOdd && tp >= 4 && 4 * tp >= int64_t(d_act) &&
                int64_t(max_position_count<kPos>(p, ws, nrec, nrun, nmix, lane)) < tp) {
                k_ones = 0;  // finish: T > k + d, every row zero
                d_act = 0;
                break;
            }
        } else if (kPart) {
            d_act += nrec;
        }
        if constexpr (kPos) {
            // 2'. literal runs a group at a time, mixed inputs position-major
            for (uint32_t r0 = 0; r0 < nrun; r0 += kGroup) {
                uint64_t v[kGroup][kRows];
                decode_group(p, ws, r0, nrun, x0, x1, lane, v);
                count.add(v, min(uint32_t(kGroup), nrun - r0));
            }
            for (uint32_t m0 = 0; m0 < nmix; m0 += 32) {
                pos_batch(p, ws, m0, min(32u, nmix - m0), lane, count);
                __syncwarp();
            }
            continue;
        }
        // 2. the active inputs into the counters, a group at a time
        for (uint32_t r0 = 0; r0 < nrec; r0 += kGroup) {
            if (r0 % kMetaBatch == 0) {
                __syncwarp();
                stage_masks(p, ws, r0, nrec, lane);
            }
            uint64_t v[kGroup][kRows];
            decode_group(p, ws, r0, nrec, x0, x1, lane, v);
            if (q.zmode()) {  // count the zeros of the active inputs
#pragma unroll
                for (int j = 0; j < kGroup; ++j)
#pragma unroll
                    for (int r = 0; r < kRows; ++r)
                        if (r0 + j < nrec) v[j][r] = ~v[j][r];
            }
            count.add(v, min(uint32_t(kGroup), nrec - r0));
        }
        __syncwarp();
    }
}

// Compare with T' = T - k (or count the zeros against d - T' + 1) and mask
// the words past W: the subtile's result words (row r of the lane in o[r]).
// Range queries test lo' <= c' <= hi' on the active count c' (two compares),
// odd-count queries take the lowest counter slice and the parity of k.
template <class Count>
__device__ __forceinline__ void finish_subtile(const PassAParams& p, uint32_t T, uint32_t zmode,
                                               uint32_t hi, uint32_t sym, uint32_t k_ones,
                                               uint32_t d_act, uint32_t x0, uint32_t lane,
                                               Count& count, uint64_t (&o)[kRows]) {
#pragma unroll
    for (int r = 0; r < kRows; ++r) o[r] = 0;
    const int64_t Tp = int64_t(T) - int64_t(k_ones);
    if constexpr (Count::kSymmetric) {
        if (sym == kSymOdd) {
            count.parity(o, (k_ones & 1u) ? ~0u : 0u);
        } else if (sym == kSymRange) {
            const int64_t Hp = int64_t(hi) - int64_t(k_ones);
            if (Hp >= 0 && Tp <= int64_t(d_act)) {
                uint64_t a[kRows], b[kRows];
                if (Tp <= 0) {
#pragma unroll
                    for (int r = 0; r < kRows; ++r) a[r] = ~0ull;
                } else {
                    count.finish(uint32_t(Tp), 0u, a);
                }
                if (Hp + 1 > int64_t(d_act)) {
#pragma unroll
                    for (int r = 0; r < kRows; ++r) b[r] = 0;
                } else {
                    count.finish(uint32_t(Hp + 1), 0u, b);
                }
#pragma unroll
                for (int r = 0; r < kRows; ++r) o[r] = a[r] & ~b[r];
            }
        }
    }
    if (sym == kSymThreshold) {
        if (Tp <= 0) {
#pragma unroll
            for (int r = 0; r < kRows; ++r) o[r] = ~0ull;
        } else if (Tp <= int64_t(d_act)) {
            const uint32_t thr = zmode ? uint32_t(int64_t(d_act) - Tp + 1) : uint32_t(Tp);
            count.finish(thr, zmode ? ~0u : 0u, o);
        }
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const uint32_t x = x0 + 32 * r + lane;
        if (x >= p.W) o[r] = 0;
        else if (x == p.W - 1 && p.ragged) o[r] &= (1ull << p.ragged) - 1;
    }
}

// Canonical re-encoding, part 1 (per subtile, by its warp).  o[q] is word
// xb + q, xb = x0 + 4 lane.  Word classes (0 zero, 1 ones, 2 literal) give
// the words that start a marker group; warp scans give each lane the heads
// and literals before it and the last head before it, and the subtile's
// aggregate A (the look-back monoid).
struct LocalScan {
    uint32_t clsbits;   // 2 bits per word
    uint32_t headbits;  // bit q: word q starts a group (word x0 excluded)
    uint32_t eh, el;    // heads / literals in the subtile before xb
    uint32_t ek;        // last head before xb: (pos + 1) << 16 | literals before << 2 | class
    RangeAgg A;
};

__device__ __forceinline__ LocalScan local_scan(uint32_t x0, uint32_t x1, uint32_t lane,
                                                const uint64_t (&o)[kWPL]) {
    LocalScan L;
    const uint32_t xb = x0 + kWPL * lane;
    uint32_t cls[kWPL];
    L.clsbits = 0;
#pragma unroll
    for (int q = 0; q < kWPL; ++q) {
        cls[q] = o[q] == 0 ? 0u : (o[q] == ~0ull ? 1u : 2u);
        L.clsbits |= cls[q] << (2 * q);
    }
    const uint32_t pc = __shfl_up_sync(~0u, cls[kWPL - 1], 1);
    uint32_t nh = 0, nl = 0;
    L.headbits = 0;
#pragma unroll
    for (int q = 0; q < kWPL; ++q) {
        if (xb + q >= x1) continue;
        const bool h = (lane == 0 && q == 0) ? false : starts_group(q ? cls[q - 1] : pc, cls[q]);
        if (h) {
            L.headbits |= 1u << q;
            ++nh;
        }
        if (cls[q] == 2u) ++nl;
    }
    const uint32_t packed = (nh << 16) | nl;
    uint32_t incl = packed;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(~0u, incl, d);
        if (lane >= uint32_t(d)) incl += t;
    }
    const uint32_t tot = __shfl_sync(~0u, incl, 31);
    const uint32_t ex = incl - packed;
    L.eh = ex >> 16;
    L.el = ex & 0xFFFFu;
    uint32_t key = 0, lc = L.el;
#pragma unroll
    for (int q = 0; q < kWPL; ++q) {
        if (xb + q >= x1) continue;
        if ((L.headbits >> q) & 1u) key = ((kWPL * lane + q + 1) << 16) | (lc << 2) | cls[q];
        if (cls[q] == 2u) ++lc;
    }
    uint32_t kmax = key;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(~0u, kmax, d);
        if (lane >= uint32_t(d)) kmax = max(kmax, t);
    }
    const uint32_t kall = __shfl_sync(~0u, kmax, 31);
    L.ek = __shfl_up_sync(~0u, kmax, 1);
    if (lane == 0) L.ek = 0;
    const uint32_t fc = __shfl_sync(~0u, cls[0], 0);
    const uint32_t last = x1 - 1 - x0;
    uint32_t lcs = cls[0];
#pragma unroll
    for (int q = 1; q < kWPL; ++q)
        if ((last & 3u) == uint32_t(q)) lcs = cls[q];
    const uint32_t lcls = __shfl_sync(~0u, lcs, last >> 2);
    L.A.start = x0;
    L.A.nh = tot >> 16;
    L.A.nl = tot & 0xFFFFu;
    uint32_t lhc = 0, has = 0;
    L.A.lh = 0;
    L.A.lp = 0;
    if (kall) {
        L.A.lh = x0 + (kall >> 16) - 1;
        L.A.lp = (kall >> 2) & 0x3FFFu;
        lhc = kall & 3u;
        has = 1;
    }
    L.A.cls = fc | (lcls << 2) | (lhc << 4) | (has << 6);
    return L;
}

// The warp's view of a query (or of a part of its inputs): n ids from
// ids_off, its threshold and counting mode; ids and stream offsets are
// cached in the warp's shared memory when n <= kCH.
__device__ __forceinline__ void load_query(const PassAParams& p, WarpCore& ws, uint32_t ids_off,
                                           uint32_t n, uint32_t T, uint32_t zmode,
                                           uint32_t Tmax, uint32_t hi, uint32_t sym,
                                           uint32_t lane, uint32_t direct = 0u) {
    __syncwarp();
    if (lane == 0) {
        ws.qn = n;
        ws.qT = T;
        ws.qz = zmode;
        ws.qoff = ids_off;
        ws.qTx = Tmax;
        ws.qhi = hi;
        ws.qsym = sym;
        ws.qdir = direct;
    }
    if (n <= uint32_t(kCH)) {
        for (uint32_t i = lane; i < n; i += 32) {
            const uint64_t ii = uint64_t(ids_off) + i;
            uint32_t b = THR_CHK(p.chk, ii < p.lim.nids, kChkIdIndex, ii, p.lim.nids)
                             ? __ldg(p.ids + ii)
                             : 0u;
            if (!THR_CHK(p.chk, b < p.lim.nb, kChkIdValue, b, p.lim.nb)) b = 0;
            ws.ids[i] = b;
            ws.woff[i] = p.desc[b].woff;
        }
    }
    __syncwarp();
}

// Re-encoding part 1 of a finished subtile: rows -> 4 consecutive words per
// lane, local scan, the result words (unless one fill class) and the
// aggregate to the slot's scratch.
__device__ __forceinline__ void store_subtile(const PassAParams& p, WarpCore& ws, uint32_t slot,
                                              uint32_t g, uint32_t x0, uint32_t x1,
                                              uint32_t lane, const uint64_t (&orow)[kRows]) {
    if (!THR_CHK(p.chk, slot < p.lim.slots, kChkSlot, slot, p.lim.slots) ||
        !THR_CHK(p.chk, g < p.NG, kChkSubtile, g, p.NG))
        return;
    const uint64_t sg = uint64_t(slot) * p.NG + g;
    // one fill class over all 128 words (words past W are zero): no head and
    // no literal inside, the aggregate follows without the scan
    const uint64_t any = orow[0] | orow[1] | orow[2] | orow[3];
    const uint64_t all = orow[0] & orow[1] & orow[2] & orow[3];
    const bool zeros = __all_sync(~0u, any == 0);
    const bool ones = __all_sync(~0u, all == ~0ull);
    if (zeros || ones) {
        if (lane == 0) {
            const uint32_t c = ones ? 1u : 0u;
            agg_store_plain(p.aggs + sg * kAggWords, RangeAgg{x0, 0, 0, 0, 0, c | (c << 2)});
        }
        return;
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r) ws.tw[32 * r + lane] = orow[r];
    __syncwarp();
    uint64_t o[kWPL];
#pragma unroll
    for (int k = 0; k < kWPL; ++k) o[k] = ws.tw[kWPL * lane + k];
    __syncwarp();
    const LocalScan L = local_scan(x0, x1, lane, o);
    if (L.A.nh || L.A.nl) {
#pragma unroll
        for (int r = 0; r < kRows; ++r) p.U[sg * kGW + 32 * r + lane] = orow[r];
    }
    if (lane == 0) agg_store_plain(p.aggs + sg * kAggWords, L.A);
}

// The members of a group (queries over the same id multiset, counted
// once): every member's compare and re-encoding of the subtile.  Out of
// line, with the counters passed in local memory, so that keeping them
// across the members' re-encodings does not raise the register count (and
// lower the occupancy) of the single-query path that shares the kernel;
// used for counters of 7 bits and more (Count::kInlineGroups).
template <class Count>
__device__ __noinline__ void finish_group(const PassAParams& p, WarpCore& ws, uint2 grp,
                                          uint32_t g, uint32_t x0, uint32_t x1, uint32_t lane,
                                          uint32_t k_ones, uint32_t d_act, Count* count) {
    for (uint32_t i = 0; i < grp.y; ++i) {
        if (!THR_CHK(p.chk, grp.x + i < p.lim.nmemb, kChkMember, grp.x + i, p.lim.nmemb)) break;
        const uint32_t m = __ldg(p.memb + grp.x + i);
        if (!THR_CHK(p.chk, m < p.lim.slots, kChkSlot, m, p.lim.slots)) break;
        uint64_t orow[kRows];
        finish_subtile(p, p.qd[m].T, 0u, 0u, kSymThreshold, k_ones, d_act, x0, lane, *count,
                       orow);
        store_subtile(p, ws, m, g, x0, x1, lane, orow);
    }
}

// Pass A driver: each warp of the persistent grid takes every (grid
// warps)-th work item of the launch, or with a work counter the next free
// one, an item being one (query, subtile) pair: query-major
// (item i = query list[i / NG], subtile i % NG) or subtile-major (subtile
// i / nlist of query list[i % nlist], so that queries sharing inputs read
// them at about the same time).  It computes the subtile's result words with
// the counting policy, stores them in the query's scratch words U (skipped
// when the subtile holds one fill class only) and stores the subtile's
// re-encoding aggregate.  No warp ever waits for another.
template <class Count, int kFeed = kFeedGrouped>
__device__ __forceinline__ void pass_a(const PassAParams& p, CtaSmem& sm, Count& count) {
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WarpSmem& ws = sm.w[wid];
    const uint32_t nwarps = gridDim.x * kNW;
    const uint32_t nitems = p.nlist * p.NG;
    uint32_t cur = ~0u;  // slot whose ids the warp holds
    uint2 grp = make_uint2(0, 1);
    const QView q{ws, p.ids};
    // static striding, or items taken from the launch's counter one at a
    // time (the next one is requested while the current one runs)
    uint32_t it = blockIdx.x * kNW + wid;
    if (p.work) {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(p.work, 1u);
        it = __shfl_sync(~0u, t, 0);
    }
    while (it < nitems) {
        uint32_t next = 0;
        if (p.work && lane == 0) next = atomicAdd(p.work, 1u);
        uint32_t li, g;
        if (p.order) {
            g = it / p.nlist;
            li = it - g * p.nlist;
        } else {
            li = it / p.NG;
            g = it - li * p.NG;
        }
        uint32_t s = __ldg(p.list + li);
        if (!THR_CHK(p.chk, s < p.lim.slots, kChkSlot, s, p.lim.slots)) s = 0;
        if (s != cur) {  // a new query: its parameters, and its ids when they fit
            const QDesc d = p.qd[s];
            load_query(p, ws, d.ids_off, d.n, d.Tlo, d.zmode, d.Thi, d.hi, d.sym, lane, d.direct);
            grp = p.grp[s];
            cur = s;
        }
        const uint32_t x0 = g * uint32_t(kGW);
        const uint32_t x1 = min(x0 + uint32_t(kGW), p.W);
        uint64_t orow[kRows];
        uint32_t k_ones = 0, d_act = 0;
        count_subtile<Count, kFeed, false>(p, q, x0, x1, lane, ws, count, k_ones, d_act);
        if (grp.y <= 1) {
            finish_subtile(p, q.T(), q.zmode(), q.hi(), q.sym(), k_ones, d_act, x0, lane, count,
                           orow);
            store_subtile(p, ws, cur, g, x0, x1, lane, orow);
        } else if constexpr (Count::kInlineGroups) {  // one count, every member's threshold
            for (uint32_t i = 0; i < grp.y; ++i) {
                if (!THR_CHK(p.chk, grp.x + i < p.lim.nmemb, kChkMember, grp.x + i,
                             p.lim.nmemb))
                    break;
                const uint32_t m = __ldg(p.memb + grp.x + i);
                if (!THR_CHK(p.chk, m < p.lim.slots, kChkSlot, m, p.lim.slots)) break;
                finish_subtile(p, p.qd[m].T, 0u, 0u, kSymThreshold, k_ones, d_act, x0, lane,
                               count, orow);
                store_subtile(p, ws, m, g, x0, x1, lane, orow);
            }
        } else {
            Count copy = count;  // the callee reads this copy, count stays in registers
            finish_group(p, ws, grp, g, x0, x1, lane, k_ones, d_act, &copy);
        }
        it = p.work ? __shfl_sync(~0u, next, 0) : it + nwarps;
    }
}

// Pass A with the carry-save counters (S-bit saturating bit slices); kPos
// selects the position-major decode of mixed inputs.  Occupancy bounds
// (measured on the many-criteria queries): 5 CTAs per SM up to S = 4 (96
// registers, few spills: 2-7% faster at T = 2..4 than 6 CTAs with 80
// registers, which in turn beat 8 CTAs with 64 by 7% for the grouped decode
// and 28% for the position-major one; 4% faster at T = 16 than 4 CTAs with
// 126 registers), 4 up to S = 6, 3 up to S = 8 (the
// group members of wider counters finish out of line to stay within it),
// 2 beyond.
template <int S, int kFeed>
__global__ void __launch_bounds__(kNT, (S <= 4 ? 5 : (S <= 6 ? 4 : (S <= 8 ? 3 : 2))))
    k_threshold(const PassAParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CtaSmem& sm = *reinterpret_cast<CtaSmem*>(smem_raw);
    CsaCount<S> count;
    pass_a<CsaCount<S>, kFeed>(p, sm, count);
}

// Pass A with the Looped levels (M thresholds at most).
template <int M>
__global__ void __launch_bounds__(kNT, 6) k_looped(const PassAParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CtaSmem& sm = *reinterpret_cast<CtaSmem*>(smem_raw);
    LoopedCount<M> count;
    pass_a<LoopedCount<M>, false>(p, sm, count);
}

// Pass A with the inputs of every subtile split among the CTA's warps: the
// CTA takes one (query, subtile) item at a time, warp w counts the w-th
// quarter of the query's inputs into its own carry-save counters, and warp 0
// adds the other warps' counter slices (a ripple adder per slice, the sticky
// bits ORed), compares and re-encodes.  Four warps work on one subtile, so
// a query with few subtiles and many inputs finishes in about a quarter of
// the time one warp per subtile needs; with many subtiles the extra
// exchange only costs.  Counter words of warps 1-3 pass through dynamic
// shared memory after CtaSmem.
template <int S>
__global__ void __launch_bounds__(kNT, 4) k_threshold_split(const PassAParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CtaSmem& sm = *reinterpret_cast<CtaSmem*>(smem_raw);
    uint32_t* part = reinterpret_cast<uint32_t*>(smem_raw + sizeof(CtaSmem));
    __shared__ uint32_t kd[kNW][2];
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WarpSmem& ws = sm.w[wid];
    const QView q{ws, p.ids};
    CsaCount<S> count;
    constexpr uint32_t kSliceWords = (S + 1) * 8 * 32;  // one warp's counters
    const uint32_t nitems = p.nlist * p.NG;
    uint32_t cur = ~0u;
    uint32_t T = 0, zmode = 0;
    for (uint32_t it = blockIdx.x; it < nitems; it += gridDim.x) {
        const uint32_t li = it / p.NG, g = it - li * p.NG;
        uint32_t s = __ldg(p.list + li);
        if (!THR_CHK(p.chk, s < p.lim.slots, kChkSlot, s, p.lim.slots)) s = 0;
        if (s != cur) {  // this warp's share of the new query's inputs
            const QDesc d = p.qd[s];
            const uint32_t a = uint32_t(uint64_t(d.n) * wid / kNW);
            const uint32_t b = uint32_t(uint64_t(d.n) * (wid + 1) / kNW);
            load_query(p, ws, d.ids_off + a, b - a, d.T, d.zmode, d.T, d.hi, d.sym, lane,
                       d.direct);
            T = d.T;
            zmode = d.zmode;
            cur = s;
        }
        const uint32_t x0 = g * uint32_t(kGW);
        const uint32_t x1 = min(x0 + uint32_t(kGW), p.W);
        uint32_t k = 0, dd = 0;
        if (q.n() > 0)
            count_subtile<CsaCount<S>, false, true>(p, q, x0, x1, lane, ws, count, k, dd);
        else
            count.begin();
        if (lane == 0) {
            kd[wid][0] = k;
            kd[wid][1] = dd;
        }
        __syncthreads();
        uint32_t K = 0, D = 0;
#pragma unroll
        for (int w = 0; w < kNW; ++w) {
            K += kd[w][0];
            D += kd[w][1];
        }
        const int64_t Tp = int64_t(T) - int64_t(K);
        const bool live = Tp > 0 && Tp <= int64_t(D);
        if (live && wid > 0) count.cnt.store(part + (wid - 1) * kSliceWords, lane);
        __syncthreads();
        if (wid == 0) {
            if (live)
                for (int w = 1; w < kNW; ++w) count.cnt.add_from(part + (w - 1) * kSliceWords, lane);
            uint64_t orow[kRows];
            finish_subtile(p, T, zmode, 0u, kSymThreshold, K, D, x0, lane, count, orow);
            store_subtile(p, ws, cur, g, x0, x1, lane, orow);
        }
        __syncthreads();
    }
}

template <int S>
constexpr size_t split_smem_bytes() {
    return sizeof(CtaSmem) + (kNW - 1) * (S + 1) * 8 * 32 * sizeof(uint32_t);
}

}  // namespace thr
