// Device code of libthr: the threshold (T-overlap) query of Kaser & Lemire
// (arXiv 1402.4466) over word-aligned run-length streams (format: thr.h).
//
// Index layout in HBM (built once by idx_build_rle):
//   words  all streams concatenated, exactly as given (uint64)
//   mtab   per bitmap nmark + 1 entries {pos, ustart | b << 31}: the stream
//          index of every marker word, the uncompressed word where its group
//          starts and its fill bit; the extra entry is {len, W}.  ustart is
//          the segmented exclusive scan of F + L over the marker words
//          (kernel k_marker_scan).
//   sdesc  per bitmap and 128-word subtile one uint64 descriptor: the class
//          of the bitmap over the subtile (zero fill, ones fill, one literal
//          run, mixed) and, for a literal run, the stream index of its first
//          literal, for a mixed subtile the index of its mask record.
//   pcls   the classes of sdesc packed 2 bits each, 32 subtiles per uint64,
//          ceil(NG / 32) words per bitmap: classification reads these and
//          the full descriptor only for inputs with literals.
//   masks  one 64-byte MaskRec per mixed (bitmap, subtile).
//   sseg   per bitmap and subtile one uint64 segment descriptor: the stream
//          index (relative to the bitmap's first word) of the first word the
//          subtile's literals need, | their number of stream words << 32
//          (a literal run: its literals; mixed: the literals and the markers
//          between them, from MaskRec::base on; else 0).  The staged kernel
//          copies exactly these words to shared memory.
//
// A query (or a batch of them) runs in three passes:
//   A  k_threshold<S> / k_scancount: persistent grid; a warp takes a work
//      item (query, m consecutive subtiles) at a time and, per subtile,
//      classifies the query's inputs from sdesc (run-aware pruning of
//      Sec. 6.4: with k ones fills and d inputs holding literals, T <= k
//      gives ones, T > k + d zeros, else T' = T - k over the d inputs),
//      decodes the active inputs, counts per row (carry-save bit slices with
//      LOP3 full adders, or ScanCount byte counters), compares with T', and
//      stores the subtile's result words (only if they are not one fill)
//      and its re-encoding aggregate.
//   B  k_scan_aggs: per query an ordered scan of the aggregates, then a scan
//      of the result lengths over the queries of the chunk that places each
//      result in the output pool and writes its final marker.
//   C  k_write_out: every literal and every marker of a group that ends
//      inside a subtile goes to its place.
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
constexpr int kSMax = 20;         // largest counter width instantiated

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

// One query of a batch.  zmode 1: count the zeros of the active inputs.
// Tlo, Thi: the thresholds pruning considers -- the query's own T, or for
// the leader of a group of queries over the same id multiset (see
// PassAParams::grp), which counts for all of them, the least and the
// largest threshold of the group.
struct QDesc {
    uint32_t ids_off;  // first id in the batch's id array
    uint32_t n;
    uint32_t T;        // threshold, or the lower bound of a range
    uint32_t zmode;
    uint32_t Tlo, Thi;
    uint32_t hi;       // range queries: the upper bound
    uint32_t sym;      // kSymThreshold, kSymRange, kSymOdd (or kSymProfile)
    uint32_t direct;   // 1: classify from the subtile descriptors alone
                       //   (most inputs hold literals in most subtiles)
};
// What a query computes from the count c of a row: c >= T (threshold),
// T <= c <= hi (range: at most, exactly, between), c odd (the XOR).
constexpr uint32_t kSymThreshold = 0, kSymRange = 1, kSymOdd = 2;
// Not a result kind: the profiling pass of opt-threshold queries (thr_opt.cuh),
// whose T is the current lower bound on the answer.
constexpr uint32_t kSymProfile = 3;

// Checked builds (compiled with THR_CHECKED): every global access of
// passes A-C whose index comes from the index arrays or the batch plan (an
// id, a literal or mask-record address, a slot, a group member, a result
// position) and every shared-memory record index is compared with the size
// of what it addresses.  A failing access is skipped and the first one is
// recorded in the batch scratch (CheckRec: site, index, limit, thread and
// block), which the host reports as THR_E_CHECK.  Normal builds compile the
// comparisons away (THR_CHK is true) and never write the record.
struct CheckRec {
    uint32_t site, where;       // CheckSite; threadIdx.x | blockIdx.x << 10
    unsigned long long val, lim;
};
enum CheckSite : uint32_t {
    kChkLiteral = 1,   // a literal word beyond the index's words
    kChkMask = 2,      // a mask record beyond the index's records
    kChkIdIndex = 3,   // an id position beyond the batch's ids
    kChkIdValue = 4,   // an id not below the index's bitmaps
    kChkSubtile = 5,   // a subtile not below NG
    kChkRecord = 6,    // a shared-memory input record beyond kCH
    kChkSlot = 7,      // a slot beyond the chunk's slots or the batch's queries
    kChkMember = 8,    // a group member position beyond the member list
    kChkMeta = 9,      // a staged mask record beyond the staging buffer
    kChkResult = 10,   // a query of pass B or C beyond the batch
};
struct CheckLimits {
    unsigned long long words;  // index words (including the two pad words)
    unsigned long long masks;  // mask records
    uint32_t nb;               // bitmaps
    uint32_t nids;             // ids of the batch
    uint32_t nq;               // queries of the batch
    uint32_t slots;            // slots of a chunk
    uint32_t nmemb;            // group member entries
};
#ifdef THR_CHECKED
__device__ __forceinline__ bool check_access(CheckRec* rec, bool ok, uint32_t site,
                                             unsigned long long v, unsigned long long lim) {
    if (!ok && rec && atomicCAS(&rec->site, 0u, site) == 0u) {
        rec->val = v;
        rec->lim = lim;
        rec->where = threadIdx.x | (blockIdx.x << 10);
    }
    return ok || !rec;
}
#define THR_CHK(rec, cond, site, v, lim) \
    ::thr::check_access((rec), (cond), (site), (unsigned long long)(v), (unsigned long long)(lim))
#else
#define THR_CHK(rec, cond, site, v, lim) true
#endif

// Pass A of one launch: the queries (slots of the chunk) in list[0..nlist),
// one work item per (query, subtile), query-major (order 0) or subtile-major
// (order 1).
struct PassAParams {
    const uint64_t* words;
    const uint64_t* sdesc;  // subtile descriptors, NG per bitmap
    const uint64_t* pcls;   // packed subtile classes, NGW words per bitmap
    const MaskRec* masks;   // mask records of the mixed subtiles
    const uint64_t* sseg;   // segment descriptors, NG per bitmap
    uint32_t* err;          // set to a non-zero code when a kernel gave up waiting
    uint32_t lose;          // test hook: each staged slot expects 16 bytes more than
                            // it is sent, so its wait runs out (THR_TEST_LOST_COPY)
    CheckRec* chk;          // checked builds: the first failed check (null: unchecked)
    CheckLimits lim;        //   and the sizes the checks compare with
    const BitmapDesc* desc;
    const QDesc* qd;        // the chunk's queries, by slot
    const uint32_t* ids;    // every id of the batch
    const uint32_t* list;   // slots taken by this launch
    uint32_t nlist;
    uint32_t order;   // 0 query-major, 1 subtile-major
    uint32_t* work;   // item counter (zeroed before the launch), or null: static striding
    uint32_t W;       // uncompressed words
    uint32_t NG;      // subtiles
    uint32_t NGW;     // packed class words per bitmap, ceil(NG / 32)
    uint32_t ragged;  // r % 64
    uint64_t* U;      // scratch: slot s at U + s NG 128 (only non-uniform subtiles stored)
    uint32_t* aggs;   // scratch: slot s, subtile g at aggs + (s NG + g) kAggWords
    // Queries sharing an id multiset: grp[s] = {first, count} of slot s's
    // group in memb (the member slots; count 1 for a query on its own); the
    // leader's warp counts once and compares for every member's threshold.
    const uint2* grp;
    const uint32_t* memb;
};

// Passes B and C of the re-encoding (thr_reencode.cu), over the Q slots of
// one chunk; slot s holds query q0 + s of the batch.
struct WriteParams {
    CheckRec* chk;      // checked builds: as PassAParams::chk
    uint32_t chk_nq;    //   queries of the batch
    const uint64_t* U;
    const uint32_t* aggs;
    uint32_t* pref;     // per (slot, subtile): prefix within its scan block
    uint32_t* bagg;     // per (slot, scan block): total
    uint32_t* bpref;    // per (slot, scan block): prefix before it
    uint32_t* full;     // per slot: aggregate of the whole result
    uint32_t* tick;     // per slot: pass B ticket (returns to 0)
    uint32_t* gtick;    // chunk ticket (returns to 0)
    unsigned long long* base;  // output words placed by earlier chunks
    unsigned long long* res;   // per query of the batch: {offset, length}
    uint64_t* out;      // output pool
    uint64_t cap;       // its capacity in words
    uint32_t W;
    uint32_t NG;
    uint32_t NB;        // scan blocks per slot
    uint32_t Q;         // slots in the chunk
    uint32_t q0;        // first query of the chunk
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
    // add two 1-bit inputs: one full adder at weight 1, then ripple the
    // weight-2 carry
    __device__ __forceinline__ void add_pair(int h, uint32_t a, uint32_t b) {
        const uint32_t k1 = add2<0>(h, a, b);
        if constexpr (S > 1) add1<1>(h, k1);
        else sticky[h] |= k1;
    }
    // the counters of this lane to dst[(k * 8 + h) * 32 + lane] (slice k,
    // half h; the sticky slice is k = S)
    __device__ __forceinline__ void store(uint32_t* dst, uint32_t lane) const {
#pragma unroll
        for (int h = 0; h < 8; ++h) {
#pragma unroll
            for (int k = 0; k < S; ++k) dst[(k * 8 + h) * 32 + lane] = c[k][h];
            dst[(S * 8 + h) * 32 + lane] = sticky[h];
        }
    }
    // add counters stored by store(): a ripple-carry adder per slice; the
    // carry out of the top slice and the other sticky bit saturate
    __device__ __forceinline__ void add_from(const uint32_t* src, uint32_t lane) {
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            uint32_t cy = 0;
#pragma unroll
            for (int k = 0; k < S; ++k) {
                const uint32_t b = src[(k * 8 + h) * 32 + lane];
                const uint32_t a = c[k][h];
                c[k][h] = lop3<kXor3>(a, b, cy);
                cy = lop3<kMaj3>(a, b, cy);
            }
            sticky[h] = lop3<kOr3>(sticky[h], cy, src[(S * 8 + h) * 32 + lane]);
        }
    }
    // bit-sliced "count >= thr" (thr <= 2^S), most significant slice first;
    // the slices hold the count mod 2^S and the sticky slice "count >= 2^S",
    // so thr = 2^S is the sticky slice alone
    __device__ __forceinline__ uint32_t ge(int h, uint32_t thr) const {
        if (thr >> S) return sticky[h];
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
                                 uint64_t* sdesc, uint64_t* sseg, uint32_t* mixed_count,
                                 uint32_t nbitmaps, uint32_t W, uint32_t NG,
                                 cudaStream_t st);
// Packed classes from the final subtile descriptors (after part b).
cudaError_t launch_pack_classes(const uint64_t* sdesc, uint64_t* pcls, uint32_t nbitmaps,
                                uint32_t NG, cudaStream_t st);
cudaError_t launch_index_build_b(const uint2* mtab, const uint32_t* ttab,
                                 const BitmapDesc* desc, const uint64_t* mixed_base,
                                 uint64_t* sdesc, uint64_t* sseg, MaskRec* masks,
                                 uint32_t nbitmaps, uint32_t W, uint32_t NG, cudaStream_t st);

}  // namespace thr
