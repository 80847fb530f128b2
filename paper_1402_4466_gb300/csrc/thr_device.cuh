// Device code of libthr: the threshold (T-overlap) query of Kaser & Lemire
// (arXiv 1402.4466) over word-aligned run-length streams (format: thr.h).
//
// Index layout in HBM (built once by idx_build_rle):
//   words  all streams concatenated, exactly as given (uint64)
//   mtab   per bitmap nmark + 1 entries {pos, ustart | b << 31}: the stream
//          index of every marker word, the uncompressed word where its group
//          starts and its fill bit; the extra entry is {len, W}.  ustart is
//          the segmented exclusive scan of F + L over the marker words
//          (kernel k_marker_scan), so F and L of marker m follow from the
//          entries m and m + 1: L = pos' - pos - 1, F = ustart' - ustart - L.
//   ttab   per bitmap NG + 1 uint32 (NG = ceil(W / 128)): ttab[g] is the
//          marker whose group contains uncompressed word 128 g; ttab[NG] =
//          nmark.  A 128-word subtile g overlaps the markers
//          ttab[g] .. ttab[g + 1] (the last one only if it starts before the
//          subtile ends).
//
// Query kernel (k_threshold<S>): a persistent grid; each CTA takes 512-word
// tiles in order from an atomic counter.  Per 128-word subtile one warp
//   1. looks up, lane per input, which markers cover the subtile and
//      classifies the input there as a fill of zeros, a fill of ones (k of
//      them), one literal run, or mixed; this is the run-aware pruning of the
//      RBMrg/EWAH cases of Sec. 6.4: T <= k gives ones, T > k + d zeros
//      (d = inputs with literals), else T' = T - k over the d active inputs;
//   2. decodes the active inputs (lane owns 4 consecutive words) and adds
//      them into bit-sliced counters with LOP3 full adders (carry-save,
//      Sec. 5.3.1 mentions carry-save and sideways-sum circuits as cheaper
//      ways to form the Hamming weight than BSTM's ripple); counters
//      saturate at 2^S (sticky bit) since only "count >= T'" matters, and
//      when T' is close to d the zeros are counted instead (S bits then
//      bound d - T' + 1);
//   3. compares the bit slices with T' most significant slice first (the
//      O'Neil-Quass comparison BSTM uses, Algorithm 2).
// The CTA then re-encodes its 512 result words canonically: word classes,
// head/literal scans, and a decoupled look-back over the tiles before it
// (bounded spin) give every marker and literal its output position.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace thr {

constexpr int kGW = 128;          // words per subtile (one warp) = ttab granule
constexpr int kNW = 4;            // warps per CTA
constexpr int kNT = 32 * kNW;     // threads per CTA
constexpr int kTW = kGW * kNW;    // words per CTA tile
constexpr int kWPL = 4;           // consecutive words per lane
constexpr int kCH = 128;          // input records per warp and chunk
constexpr int kSMax = 16;         // largest counter width instantiated

// Mask record of a mixed (bitmap, subtile), one 64-byte line.  Bit j of
// word w of lm / cm / om is subtile word x0 + 32 w + j being a literal /
// a literal or the start of a marker group / a ones-fill word (a group
// starts only at a fill word, so a literal never starts one); base = stream
// index (relative to the bitmap's first word) of the first literal at or
// after x0; byte w of pre = literal words + group starts before word 32 w
// (excluding x0, at most 192).  The literal at x0 + 32 w + j then sits at
// stream index base + pre[w] + popc(cm[w] below bit j).
struct MaskRec {
    uint32_t lm[4];
    uint32_t cm[4];
    uint32_t om[4];
    uint32_t base;
    uint32_t pre;
    uint32_t pad[2];
};
static_assert(sizeof(MaskRec) == 64, "mask record is one 64-byte line");

struct BitmapDesc {
    uint64_t woff;   // first word of the stream in `words`
    uint64_t moff;   // first entry of the bitmap in `mtab`
    uint32_t nmark;  // number of markers
    uint32_t len;    // stream length in words
};

// Aggregate of the re-encoding state over a run of words [start, ...):
// heads (words that start a marker group), literal words, the last head and
// the literals before it.  cls packs first class | last class << 2 |
// class of last head << 4 | has-last-head << 6 (class 0 zero, 1 ones, 2 lit).
struct RangeAgg {
    uint32_t start, nh, nl, lh, lp, cls;
};

// Aggregates and prefixes are stored as kAggWords uint32 per subtile.
constexpr int kAggWords = 8;

struct QueryParams {
    const uint64_t* words;
    const uint2* mtab;
    const uint64_t* sdesc;  // subtile descriptors, NG per bitmap
    const MaskRec* masks;   // mask records of the mixed subtiles
    const BitmapDesc* desc;
    const uint32_t* ids;  // device copy of the query's ids
    uint32_t n;
    uint32_t T;
    uint32_t zmode;   // 1: count zeros among the active inputs
    uint32_t W;       // uncompressed words
    uint32_t NG;      // subtiles
    uint32_t ntiles;  // subtiles (= NG)
    uint32_t ragged;  // r % 64
    uint32_t spin_limit;
    uint32_t* ctl;     // [0] subtile counter (zeroed before the launch)
    uint64_t* U;       // scratch: W result words (only non-uniform subtiles stored)
    uint32_t* aggs;    // scratch: per subtile re-encoding aggregate
};

// Passes B and C of the re-encoding (thr_reencode.cu).
struct WriteParams {
    const uint64_t* U;
    const uint32_t* aggs;
    uint32_t* pref;    // per subtile: prefix within its scan block (pass B)
    uint32_t* bagg;    // per scan block: total
    uint32_t* bpref;   // per scan block: prefix before it
    uint64_t* out;     // device output buffer
    uint64_t cap;
    uint32_t W;
    uint32_t NG;
    uint32_t* ctl;     // [2..3] encoded length (pass B), [4] pass B ticket
};
cudaError_t launch_reencode(const WriteParams& w, cudaStream_t st);


// ------------------------------------------------------------ primitives

template <uint32_t LUT>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
    uint32_t d;
    asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
    return d;
}
// truth tables over (a = 0xF0, b = 0xCC, c = 0xAA)
constexpr uint32_t kXor3 = 0x96;  // a ^ b ^ c
constexpr uint32_t kMaj3 = 0xE8;  // majority(a, b, c)
constexpr uint32_t kOr3 = 0xFE;   // a | b | c
constexpr uint32_t kOrAnd = 0xF8; // a | (b & c)
constexpr uint32_t kAndNot = 0x30; // a & ~b  (c unused)

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }


// ---------------------------------------------------- bit-sliced counters
//
// One counter per row: for each 32-bit half of a lane's 4 words, S slices
// c[k] (bit i of c[k] = bit k of row i's count) plus a sticky slice that
// records count >= 2^S.  Adding inputs uses full adders (sum = XOR3,
// carry = MAJ3) in a small carry-save tree.
template <int S>
struct Counters {
    uint32_t c[S][8];
    uint32_t sticky[8];

    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int h = 0; h < 8; ++h) {
#pragma unroll
            for (int k = 0; k < S; ++k) c[k][h] = 0;
            sticky[h] = 0;
        }
    }
    // add x * 2^k: ripple from slice k; overflow goes to sticky
    template <int K>
    __device__ __forceinline__ void add1(int h, uint32_t x) {
#pragma unroll
        for (int j = K; j < S; ++j) {
            const uint32_t t = c[j][h] & x;
            c[j][h] ^= x;
            x = t;
        }
        sticky[h] |= x;
    }
    // add (x + y) * 2^K with one full adder; returns the carry (weight 2^(K+1))
    template <int K>
    __device__ __forceinline__ uint32_t add2(int h, uint32_t x, uint32_t y) {
        if constexpr (K < S) {
            const uint32_t s = lop3<kXor3>(c[K][h], x, y);
            const uint32_t cy = lop3<kMaj3>(c[K][h], x, y);
            c[K][h] = s;
            return cy;
        } else {
            sticky[h] = lop3<kOr3>(sticky[h], x, y);
            return 0u;
        }
    }
    // add four 1-bit inputs: two full adders at weight 1, one at weight 2,
    // then ripple the weight-4 carry
    __device__ __forceinline__ void add4(int h, uint32_t a, uint32_t b, uint32_t cc, uint32_t d) {
        const uint32_t k1 = add2<0>(h, a, b);
        const uint32_t k2 = add2<0>(h, cc, d);
        const uint32_t k3 = add2<1>(h, k1, k2);
        if constexpr (S > 2) add1<2>(h, k3);
        else sticky[h] |= k3;
    }
    // bit-sliced "count >= thr" (thr < 2^S), most significant slice first
    __device__ __forceinline__ uint32_t ge(int h, uint32_t thr) const {
        uint32_t eq = ~0u, gt = 0u;
#pragma unroll
        for (int k = S - 1; k >= 0; --k) {
            if ((thr >> k) & 1u) {
                eq &= c[k][h];
            } else {
                gt = lop3<kOrAnd>(gt, eq, c[k][h]);
                eq = eq & ~c[k][h];
            }
        }
        return gt | eq | sticky[h];
    }
};

// ------------------------------------------------------- re-encode monoid

__device__ __forceinline__ uint32_t agg_fc(const RangeAgg& a) { return a.cls & 3u; }
__device__ __forceinline__ uint32_t agg_lc(const RangeAgg& a) { return (a.cls >> 2) & 3u; }
__device__ __forceinline__ uint32_t agg_lhc(const RangeAgg& a) { return (a.cls >> 4) & 3u; }
__device__ __forceinline__ bool agg_has(const RangeAgg& a) { return (a.cls >> 6) & 1u; }

// Does a word of class `cls` start a marker group after a word of class
// `prev`?  Only fill words do: after a literal, or when the fill changes.
__device__ __forceinline__ bool starts_group(uint32_t prev, uint32_t cls) {
    return cls != 2u && (prev == 2u || prev != cls);
}

// X covers [X.start, Y.start), Y follows it.
__device__ __forceinline__ RangeAgg agg_combine(const RangeAgg& X, const RangeAgg& Y) {
    RangeAgg Z;
    const bool hf = starts_group(agg_lc(X), agg_fc(Y));
    Z.start = X.start;
    Z.nh = X.nh + (hf ? 1u : 0u) + Y.nh;
    Z.nl = X.nl + Y.nl;
    uint32_t lhc, has;
    if (agg_has(Y)) {
        Z.lh = Y.lh;
        Z.lp = X.nl + Y.lp;
        lhc = agg_lhc(Y);
        has = 1;
    } else if (hf) {
        Z.lh = Y.start;
        Z.lp = X.nl;
        lhc = agg_fc(Y);
        has = 1;
    } else {
        Z.lh = X.lh;
        Z.lp = X.lp;
        lhc = agg_lhc(X);
        has = agg_has(X) ? 1u : 0u;
    }
    Z.cls = agg_fc(X) | (agg_lc(Y) << 2) | (lhc << 4) | (has << 6);
    return Z;
}

__device__ __forceinline__ void agg_store_plain(uint32_t* p, const RangeAgg& a) {
    *reinterpret_cast<uint4*>(p) = make_uint4(a.start, a.nh, a.nl, a.lh);
    *reinterpret_cast<uint2*>(p + 4) = make_uint2(a.lp, a.cls);
}
__device__ __forceinline__ RangeAgg agg_load_plain(const uint32_t* p) {
    const uint4 x = *reinterpret_cast<const uint4*>(p);
    const uint2 y = *reinterpret_cast<const uint2*>(p + 4);
    RangeAgg a;
    a.start = x.x;
    a.nh = x.y;
    a.nl = x.z;
    a.lh = x.w;
    a.lp = y.x;
    a.cls = y.y;
    return a;
}

// ------------------------------------------------------------- build (K1)

// Build kernels (thr_build.cu).  Part a: segmented scan of the marker
// extents into mtab, the subtile table ttab (a build temporary) and the
// subtile classes with per-bitmap counts of mixed subtiles.  Part b, once the
// host has placed the mask records: the mask records and final descriptors.
cudaError_t launch_index_build_a(const uint64_t* words, const uint32_t* mpos,
                                 const BitmapDesc* desc, uint2* mtab, uint32_t* ttab,
                                 uint64_t* sdesc, uint32_t* mixed_count,
                                 uint32_t nbitmaps, uint32_t W, uint32_t NG,
                                 cudaStream_t st);
cudaError_t launch_index_build_b(const uint2* mtab, const uint32_t* ttab,
                                 const BitmapDesc* desc, const uint64_t* mixed_base,
                                 uint64_t* sdesc, MaskRec* masks, uint32_t nbitmaps,
                                 uint32_t W, uint32_t NG, cudaStream_t st);

}  // namespace thr
