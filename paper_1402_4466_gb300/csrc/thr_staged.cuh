// Pass A with staged inputs (k_staged<S>, THR_VARIANT_STAGED).
//
// The counting and the re-encoding are those of k_threshold<S>
// (thr_query_kernel.cuh); what changes is how an input's words reach the
// warp.  The direct kernel loads every literal word from global memory at
// the moment it is added, after a chain of dependent loads (packed class ->
// descriptor -> mask record -> literal).  Here the active inputs of a
// subtile are first classified (packed class, then the segment descriptor
// sseg and, for a mixed input, its descriptor), and their compressed words
// for the subtile -- one contiguous stream segment per input, found at build
// time -- and mask records are copied into shared memory by 1-D bulk copies
// (cp.async.bulk, completion counted in bytes on an mbarrier).  Copies go in
// waves: a wave is as many of the chunk's inputs as fit one kWaveBytes
// buffer (the cut points come from a prefix of the records' sizes computed
// once per chunk); each warp has two buffers, and while it adds the inputs
// of one wave the next wave -- the rest of the chunk, or the first wave of
// its next work item, classified first -- is already on its way.  Every
// word of a segment is read from HBM once, in whole 16-byte units; the
// decode then finds a mixed input's literal at segment word pre[r] +
// popc(cm[r] below the lane) in shared memory.
//
// Measured on the 64 x 2^26 many-criteria bitmaps at T = 2 it is slower than
// the direct kernel (94 vs 75 us): the memory latency is hidden, but one
// bulk copy per input and subtile (about 640 thousand per query, ~300 bytes
// on average) with a wait per wave costs 52 us on its own, without any
// decode or add.  It is a flag-selected variant, not an arm of the
// policies.
//
// A copy starts at an even stream word (16 bytes) and covers whole 16-byte
// units, so it may read one word before the segment and one after it; the
// index keeps two zero words after the last stream.  Waits give up after
// about a second (which only happens if a copy never arrives): the warp
// records a code in p.err (the host then returns THR_E_TIMEOUT), waits --
// bounded again -- for its other buffer's copies, and stops.
#pragma once

#include "thr_query_kernel.cuh"

namespace thr {

constexpr int kWaveBytes = 3840;  // one wave buffer
// the largest input: a mask record and kGW words from an odd stream word,
// in 16-byte units
static_assert(sizeof(MaskRec) + 16 * ((8 * (kGW + 1) + 15) / 16) <= kWaveBytes,
              "a wave holds any one input");
static_assert(kWaveBytes <= (1 << 12), "wave offsets take 12 bits");

struct StageWarp {
    alignas(16) unsigned char buf[2][kWaveBytes];
    unsigned long long bar[2];  // one mbarrier per buffer
    // [unit parity][record]: byte offset of the record's words in its wave's
    // buffer | first word odd << 12 | mixed << 13 | has ones-fill words << 14
    uint32_t dir[2][kCH];
    uint32_t psum[kCH];  // bytes the unit's records take in waves, inclusive prefix
};
struct StagedCta {
    WarpCore w[kNW];
    StageWarp s[kNW];
};

constexpr size_t staged_smem_bytes() { return sizeof(StagedCta); }

// ------------------------------------------------ bulk copies and mbarriers

__device__ __forceinline__ uint32_t smem_addr(const void* ptr) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// orders this thread's earlier shared-memory accesses before later bulk copies
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
// try_wait with a suspend-time hint: the warp sleeps in hardware until the
// phase completes or about `hint_ns` have passed.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of parity `parity` to complete: false after about a
// second (or 2^20 suspended tries) without it.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    constexpr uint32_t kHintNs = 100000;
    if (mbar_try_wait(bar, parity, kHintNs)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 1; i < (1u << 20); ++i) {
        if (mbar_try_wait(bar, parity, kHintNs)) return true;
        if (global_ns() - t0 > 1000000000ull) return false;
    }
    return false;
}

// ------------------------------------------------------------- records

// Records of the staged kernel (ws.rec): x, y & 0xFF = stream index of the
// segment's first word (absolute); y >> 8 & 0x1FF = its words; y bit 30 =
// ones-fill words in the subtile, bit 31 = mixed; z, w = mask record index.
__device__ __forceinline__ uint4 staged_record(uint64_t seg, uint32_t len, bool mixed,
                                               uint32_t ones, uint64_t midx) {
    return make_uint4(uint32_t(seg),
                      uint32_t(seg >> 32) | (len << 8) | (ones << 30) | (mixed ? 1u << 31 : 0u),
                      uint32_t(midx), uint32_t(midx >> 32));
}

// A unit of work: one chunk (at most kCH ids) of a work item (query,
// subtile), with what finishing the item needs.  Warp-uniform registers.
struct Unit {
    uint32_t it;    // work item (>= nitems: none)
    uint32_t c0;    // first id of the chunk
    uint32_t nrec;  // active inputs of the chunk (records in ws.rec)
    uint32_t fill;  // records already sent in waves
    uint32_t k, d;  // ones fills and inputs with literals over the item's ids
    uint32_t flags; // kUCount | kUFirst | kULast | parity << 3 | zmode << 4 | sym << 5
    uint32_t T, hi; // the item's query: threshold (least of a group) and range bound
    uint32_t slot;
    uint2 grp;
};
constexpr uint32_t kUCount = 1u;  // the chunk has inputs to add
constexpr uint32_t kUFirst = 2u;  // first chunk of the item
constexpr uint32_t kULast = 4u;   // last chunk of the item

// The records [begin, end) of the wave in each buffer, 8 bits each: buffer
// b's range at bits 16 b .. 16 b + 15.
__device__ __forceinline__ uint32_t wave_begin(uint32_t w, uint32_t b) {
    return (w >> (16 * b)) & 0xFFu;
}
__device__ __forceinline__ uint32_t wave_end(uint32_t w, uint32_t b) {
    return (w >> (16 * b + 8)) & 0xFFu;
}

// Bytes a record takes in a wave, in 16-byte units: its words, and for a
// mixed input its 64-byte mask record in front of them.
__device__ __forceinline__ uint32_t data_bytes(uint32_t len, uint32_t odd) {
    return (8u * (len + odd) + 15u) & ~15u;
}
__device__ __forceinline__ uint32_t record_bytes(const uint4& rec) {
    const uint32_t len = (rec.y >> 8) & 0x1FFu;
    return data_bytes(len, rec.x & 1u) + ((rec.y >> 31) ? uint32_t(sizeof(MaskRec)) : 0u);
}

// Send the unit's next records, as many as fit buffer b, as one wave: the
// wave's end from the bytes prefix (psum), one arrive with the wave's bytes,
// then the copies (lane per record) and the records' dir entries.  `waves`
// receives the wave's records.
__device__ __forceinline__ void issue_wave(const PassAParams& p, const WarpCore& ws,
                                           StageWarp& sw, Unit& u, uint32_t b, uint32_t lane,
                                           uint32_t& waves) {
    const uint32_t par = (u.flags >> 3) & 1u;
    uint32_t* dir = sw.dir[par];
    const uint32_t r0 = u.fill;
    const uint32_t start = r0 ? sw.psum[r0 - 1] : 0u;
    uint32_t r = r0;
    while (r < u.nrec) {  // the records that fit, 32 at a time
        const uint32_t j = r + lane;
        const bool fits = j < u.nrec && sw.psum[j] - start <= uint32_t(kWaveBytes);
        const uint32_t m = __popc(__ballot_sync(~0u, fits));
        r += m;
        if (m < 32) break;
    }
    const uint32_t used = sw.psum[r - 1] - start;  // r > r0: one record always fits
    const uint32_t bar = smem_addr(&sw.bar[b]);
    fence_proxy_async();
    if (lane == 0) mbar_arrive_expect_tx(bar, used + (p.lose ? 16u : 0u));
    __syncwarp();
    unsigned char* base = sw.buf[b];
    for (uint32_t j = r0 + lane; j < r; j += 32) {  // the copies
        const uint4 rec = ws.rec[j];
        const uint64_t seg = (uint64_t(rec.y & 0xFFu) << 32) | rec.x;
        const uint32_t len = (rec.y >> 8) & 0x1FFu;
        const uint32_t odd = rec.x & 1u, mixed = rec.y >> 31, ones = (rec.y >> 30) & 1u;
        uint32_t off = sw.psum[j] - start - record_bytes(rec);
        if (mixed) {
            bulk_copy(smem_addr(base + off), p.masks + ((uint64_t(rec.w) << 32) | rec.z),
                      uint32_t(sizeof(MaskRec)), bar);
            off += uint32_t(sizeof(MaskRec));
        }
        bulk_copy(smem_addr(base + off), p.words + (seg & ~1ull), data_bytes(len, odd), bar);
        dir[j] = off | (odd << 12) | (mixed << 13) | (ones << 14);
    }
    __syncwarp();
    waves = (waves & ~(0xFFFFu << (16 * b))) | ((r0 | (r << 8)) << (16 * b));
    u.fill = r;
}

// Values of records r0 .. r0 + kGroup - 1 (< rend) at the lane's words
// x0 + 32 r + lane, from the wave buffer: a literal run row by row, a mixed
// input through its mask record (the literal at segment word pre[r] +
// popc(cm[r] below the lane); a ones-fill word from the ones mask; else 0).
__device__ __forceinline__ void staged_decode(const unsigned char* base, const uint32_t* dir,
                                              uint32_t r0, uint32_t rend, uint32_t x0,
                                              uint32_t x1, uint32_t lane,
                                              uint64_t (&v)[kGroup][kRows]) {
    const uint32_t bit = 1u << lane;
    const uint32_t lt = bit - 1u;
#pragma unroll
    for (int j = 0; j < kGroup; ++j) {
#pragma unroll
        for (int r = 0; r < kRows; ++r) v[j][r] = 0;
        if (r0 + j >= rend) continue;
        const uint32_t ej = dir[r0 + j];
        const unsigned char* at = base + (ej & 0xFFFu);
        const uint64_t* data = reinterpret_cast<const uint64_t*>(at) + ((ej >> 12) & 1u);
        if (!((ej >> 13) & 1u)) {  // a literal run: the subtile's words in order
#pragma unroll
            for (int r = 0; r < kRows; ++r)
                if (x0 + 32 * r + lane < x1) v[j][r] = data[32 * r + lane];
            continue;
        }
        const MaskRec* m = reinterpret_cast<const MaskRec*>(at - sizeof(MaskRec));
        const uint4 lmv = *reinterpret_cast<const uint4*>(m->lm);
        const uint4 cmv = *reinterpret_cast<const uint4*>(m->cm);
        const uint32_t pre = m->pre;
        const uint32_t lm[4] = {lmv.x, lmv.y, lmv.z, lmv.w};
        const uint32_t cm[4] = {cmv.x, cmv.y, cmv.z, cmv.w};
        if ((ej >> 14) & 1u) {  // ones-fill words too
            const uint4 omv = *reinterpret_cast<const uint4*>(m->om);
            const uint32_t om[4] = {omv.x, omv.y, omv.z, omv.w};
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                if ((lm[r] | om[r]) == 0u) continue;
                const uint32_t off = ((pre >> (8 * r)) & 0xFFu) + __popc(cm[r] & lt);
                v[j][r] = (lm[r] & bit) ? data[off] : ((om[r] & bit) ? ~0ull : 0ull);
            }
        } else {
#pragma unroll
            for (int r = 0; r < kRows; ++r) {
                if (lm[r] == 0u) continue;
                const uint32_t off = ((pre >> (8 * r)) & 0xFFu) + __popc(cm[r] & lt);
                if (lm[r] & bit) v[j][r] = data[off];
            }
        }
    }
}

// The largest number of inputs with a non-zero word at one position of the
// subtile (as max_position_count, for the staged records).
__device__ __forceinline__ uint32_t staged_max_position_count(const PassAParams& p,
                                                              const WarpCore& ws, uint32_t nrec,
                                                              uint32_t lane) {
    uint32_t c[kRows] = {0, 0, 0, 0};
    uint32_t runs = 0;
    for (uint32_t m0 = 0; m0 < nrec; m0 += 32) {
        const uint32_t j = m0 + lane;
        uint32_t mk[kRows] = {0, 0, 0, 0};
        bool run = false;
        if (j < nrec) {
            const uint4 rec = ws.rec[j];
            if (!(rec.y >> 31)) {
                run = true;
            } else {
                const uint4* m = reinterpret_cast<const uint4*>(
                    p.masks + ((uint64_t(rec.w) << 32) | rec.z));
                const uint4 lm = __ldg(m);
                mk[0] = lm.x;
                mk[1] = lm.y;
                mk[2] = lm.z;
                mk[3] = lm.w;
                if ((rec.y >> 30) & 1u) {
                    const uint4 om = __ldg(m + 2);
                    mk[0] |= om.x;
                    mk[1] |= om.y;
                    mk[2] |= om.z;
                    mk[3] |= om.w;
                }
            }
        }
        runs += __popc(__ballot_sync(~0u, run));
#pragma unroll
        for (int r = 0; r < kRows; ++r) c[r] += __popc(transpose32(mk[r], lane));
    }
    const uint32_t m = max(max(c[0], c[1]), max(c[2], c[3])) + runs;
    return __reduce_max_sync(~0u, m);
}

// Plan the unit of work item `it` whose chunk starts at id c0: for the
// first chunk load the query (unless it is the one in ws) and, for more
// than kCH ids, count k and d over all of them; classify the chunk's ids into
// records; decide the subtile by run-aware pruning (Sec. 6.4 cases 1 and 2,
// and the finer position bound) when it can.  `prev` carries the item's
// values from chunk to chunk.
__device__ __forceinline__ Unit plan_unit(const PassAParams& p, WarpCore& ws, StageWarp& sw,
                                          const QView& q, uint32_t it, uint32_t c0,
                                          const Unit& prev, uint32_t par, uint32_t& loaded,
                                          uint32_t lane) {
    Unit u = prev;
    u.it = it;
    u.c0 = c0;
    u.nrec = 0;
    u.fill = 0;
    if (it >= p.nlist * p.NG) {  // no more work
        u.flags = 0;
        return u;
    }
    uint32_t li, g;
    if (p.order) {
        g = it / p.nlist;
        li = it - g * p.nlist;
    } else {
        li = it / p.NG;
        g = it - li * p.NG;
    }
    if (c0 == 0) {
        const uint32_t s = __ldg(p.list + li);
        if (s != loaded) {
            const QDesc dq = p.qd[s];
            load_query(p, ws, dq.ids_off, dq.n, dq.Tlo, dq.zmode, dq.Thi, dq.hi, dq.sym, lane);
            loaded = s;
        }
        u.slot = s;
        u.grp = p.grp[s];
        u.T = q.T();
        u.hi = q.hi();
        u.flags = kUFirst | (q.zmode() << 4) | (q.sym() << 5);
        u.k = 0;
        u.d = 0;
    } else {
        u.flags &= ~(kUFirst | kUCount | kULast | 8u);
    }
    u.flags |= par << 3;
    const uint32_t n = q.n();
    const bool one_chunk = n <= uint32_t(kCH);
    if (c0 + kCH >= n) u.flags |= kULast;
    if (c0 == 0 && !one_chunk) {  // k and d over every id, so that pruning applies
        for (uint32_t i0 = 0; i0 < n; i0 += 32) {
            const uint32_t i = i0 + lane;
            uint32_t cls = 0;
            if (i < n)
                cls = uint32_t(__ldg(p.pcls + uint64_t(__ldg(q.ids() + i)) * p.NGW + (g >> 5)) >>
                               (2 * (g & 31))) & 3u;
            u.k += __popc(__ballot_sync(~0u, cls == 1));
            u.d += __popc(__ballot_sync(~0u, cls >= 2));
        }
        if (q.decided(u.k, u.d)) {  // decided: no chunk is counted
            u.flags |= kULast;
            return u;
        }
    } else if (c0 > 0 && q.decided(u.k, u.d)) {
        u.flags |= kULast;
        return u;
    }
    // classify the chunk, lane per id: packed class, then the segment (and
    // for a mixed input its descriptor) of inputs with literals
    const uint32_t cn = min(uint32_t(kCH), n - c0);
    uint32_t nrec = 0, k1 = 0;
    for (uint32_t i0 = 0; i0 < cn; i0 += 32) {
        const uint32_t i = i0 + lane;
        uint32_t cls = 0;
        uint4 r = make_uint4(0, 0, 0, 0);
        if (i < cn) {
            const uint32_t b = q.cached() ? ws.ids[i] : __ldg(q.ids() + c0 + i);
            cls = uint32_t(__ldg(p.pcls + uint64_t(b) * p.NGW + (g >> 5)) >> (2 * (g & 31))) & 3u;
            if (cls >= 2) {
                const uint64_t at = uint64_t(b) * p.NG + g;
                const uint64_t sg = __ldg(p.sseg + at);
                const uint64_t sd = cls == 3 ? __ldg(p.sdesc + at) : 0ull;
                const uint64_t woff = q.cached() ? ws.woff[i] : p.desc[b].woff;
                r = staged_record(woff + (sg & 0xFFFFFFFFull), uint32_t(sg >> 32) & 0x1FFu,
                                  cls == 3, uint32_t(sd >> 2) & 1u, sd >> 19);
            }
        }
        k1 += __popc(__ballot_sync(~0u, cls == 1));
        const uint32_t act = __ballot_sync(~0u, cls >= 2);
        if (cls >= 2) ws.rec[nrec + __popc(act & ((1u << lane) - 1u))] = r;
        nrec += __popc(act);
    }
    __syncwarp();
    u.nrec = nrec;
    uint32_t acc = 0;  // bytes prefix of the records (the waves' cut points)
    for (uint32_t j0 = 0; j0 < nrec; j0 += 32) {
        const uint32_t j = j0 + lane;
        uint32_t incl = j < nrec ? record_bytes(ws.rec[j]) : 0u;
#pragma unroll
        for (int dd = 1; dd < 32; dd <<= 1) {
            const uint32_t t = __shfl_up_sync(~0u, incl, dd);
            if (lane >= uint32_t(dd)) incl += t;
        }
        if (j < nrec) sw.psum[j] = acc + incl;
        acc += __shfl_sync(~0u, incl, 31);
    }
    __syncwarp();
    if (one_chunk) {
        u.k = k1;
        u.d = nrec;
        if (q.decided(u.k, u.d)) return u;
        // finer: no word of the subtile is non-zero in T' inputs
        const int64_t tp = int64_t(q.T()) - int64_t(u.k);
        if (q.sym() != kSymOdd && tp >= 4 && 4 * tp >= int64_t(u.d) &&
            int64_t(staged_max_position_count(p, ws, nrec, lane)) < tp) {
            u.k = 0;  // T > k + d: every row zero
            u.d = 0;
            return u;
        }
    }
    if (nrec) u.flags |= kUCount;
    return u;
}

// Add the records [wbeg, wend) of a wave in buffer `base` to the counters.
template <class Count>
__device__ __forceinline__ void add_wave(const unsigned char* base, const uint32_t* dir,
                                         uint32_t wbeg, uint32_t wend, uint32_t zmode,
                                         uint32_t x0, uint32_t x1, uint32_t lane, Count& count) {
    for (uint32_t r0 = wbeg; r0 < wend; r0 += kGroup) {
        uint64_t v[kGroup][kRows];
        staged_decode(base, dir, r0, wend, x0, x1, lane, v);
        if (zmode) {  // count the zeros of the active inputs
#pragma unroll
            for (int j = 0; j < kGroup; ++j)
#pragma unroll
                for (int r = 0; r < kRows; ++r)
                    if (r0 + j < wend) v[j][r] = ~v[j][r];
        }
        count.add(v, min(uint32_t(kGroup), wend - r0));
    }
}

// Finish a work item whose counts are complete: compare and re-encode (for
// every member of its group), as pass_a does.
template <class Count>
__device__ __forceinline__ void finish_unit(const PassAParams& p, WarpCore& ws, const Unit& u,
                                            uint32_t lane, Count& count) {
    const uint32_t g = p.order ? u.it / p.nlist : u.it % p.NG;
    const uint32_t x0 = g * uint32_t(kGW);
    const uint32_t x1 = min(x0 + uint32_t(kGW), p.W);
    uint64_t orow[kRows];
    if (u.grp.y <= 1) {
        finish_subtile(p, u.T, (u.flags >> 4) & 1u, u.hi, u.flags >> 5, u.k, u.d, x0, lane,
                       count, orow);
        store_subtile(p, ws, u.slot, g, x0, x1, lane, orow);
    } else if constexpr (Count::kInlineGroups) {  // one count, every member's threshold
        for (uint32_t i = 0; i < u.grp.y; ++i) {
            const uint32_t m = __ldg(p.memb + u.grp.x + i);
            finish_subtile(p, p.qd[m].T, 0u, 0u, kSymThreshold, u.k, u.d, x0, lane, count,
                           orow);
            store_subtile(p, ws, m, g, x0, x1, lane, orow);
        }
    } else {
        Count copy = count;  // the callee reads this copy, count stays in registers
        finish_group(p, ws, u.grp, g, x0, x1, lane, u.k, u.d, &copy);
    }
}

// Pass A driver of the staged kernel.  The warp's work items come as in
// pass_a (static striding or the launch's counter); each is one unit per
// chunk of kCH ids.  While the last wave of a unit is added, the next unit is
// planned and its first wave sent into the other buffer.
template <class Count>
__device__ __forceinline__ void staged_pass_a(const PassAParams& p, StagedCta& sm, Count& count) {
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WarpCore& ws = sm.w[wid];
    StageWarp& sw = sm.s[wid];
    if (lane == 0) {
        mbar_init(smem_addr(&sw.bar[0]), 1);
        mbar_init(smem_addr(&sw.bar[1]), 1);
        fence_mbar_init();
    }
    __syncwarp();
    const QView q{ws, p.ids};
    const uint32_t nwarps = gridDim.x * kNW;
    const uint32_t nitems = p.nlist * p.NG;
    auto next_item = [&](uint32_t it) -> uint32_t {
        if (!p.work) return it + nwarps;
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(p.work, 1u);
        return __shfl_sync(~0u, t, 0);
    };
    uint32_t first = blockIdx.x * kNW + wid;
    if (p.work) first = next_item(0);
    uint32_t loaded = ~0u;  // slot whose query ws holds
    uint32_t phase = 0;     // per buffer: parity of its next completion
    uint32_t waves = 0;     // records of the wave in each buffer
    Unit cur{};
    cur = plan_unit(p, ws, sw, q, first, 0, cur, 0u, loaded, lane);
    uint32_t b = 0;  // the buffer of cur's next wave
    if (cur.flags & kUCount) issue_wave(p, ws, sw, cur, b, lane, waves);
    while (cur.it < nitems) {
        if (cur.flags & kUFirst) count.begin();
        Unit nxt = cur;
        const uint32_t par = (cur.flags >> 3) & 1u;
        const uint32_t g = p.order ? cur.it / p.nlist : cur.it % p.NG;
        const uint32_t x0 = g * uint32_t(kGW);
        const uint32_t x1 = min(x0 + uint32_t(kGW), p.W);
        bool planned = false;
        if (cur.flags & kUCount) {
            for (;;) {
                const bool more = cur.fill < cur.nrec;
                if (more) {
                    issue_wave(p, ws, sw, cur, b ^ 1u, lane, waves);
                } else {  // the next unit, and its first wave
                    nxt = (cur.flags & kULast)
                              ? plan_unit(p, ws, sw, q, next_item(cur.it), 0, cur, par ^ 1u, loaded,
                                          lane)
                              : plan_unit(p, ws, sw, q, cur.it, cur.c0 + kCH, cur, par ^ 1u,
                                          loaded, lane);
                    planned = true;
                    if (nxt.flags & kUCount)
                        issue_wave(p, ws, sw, nxt, b ^ 1u, lane, waves);
                }
                if (!mbar_wait(smem_addr(&sw.bar[b]), (phase >> b) & 1u)) {
                    if (lane == 0) atomicOr(p.err, 1u);
                    // the other buffer's copies, if any were sent, must land first
                    if (more || (nxt.flags & kUCount))
                        mbar_wait(smem_addr(&sw.bar[b ^ 1u]), (phase >> (b ^ 1u)) & 1u);
                    return;
                }
                phase ^= 1u << b;
                add_wave(sw.buf[b], sw.dir[par], wave_begin(waves, b), wave_end(waves, b),
                         (cur.flags >> 4) & 1u, x0, x1, lane, count);
                __syncwarp();
                b ^= 1u;
                if (!more) break;
            }
        }
        if (cur.flags & kULast) finish_unit(p, ws, cur, lane, count);
        if (!planned) {  // nothing was counted: plan the next unit now
            nxt = (cur.flags & kULast)
                      ? plan_unit(p, ws, sw, q, next_item(cur.it), 0, cur, par ^ 1u, loaded, lane)
                      : plan_unit(p, ws, sw, q, cur.it, cur.c0 + kCH, cur, par ^ 1u, loaded, lane);
            if (nxt.flags & kUCount) issue_wave(p, ws, sw, nxt, b, lane, waves);
        }
        cur = nxt;
    }
}

// The staged carry-save kernel, S-bit counters.
template <int S>
__global__ void __launch_bounds__(kNT, (S <= 4 ? 4 : (S <= 8 ? 3 : 2))) k_staged(const PassAParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StagedCta& sm = *reinterpret_cast<StagedCta*>(smem_raw);
    CsaCount<S> count;
    staged_pass_a<CsaCount<S>>(p, sm, count);
}

}  // namespace thr
