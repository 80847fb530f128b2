// Pass A with staged inputs (k_staged<S>): the default carry-save kernel.
//
// The counting and the re-encoding are those of k_threshold<S>
// (thr_query_kernel.cuh); what changes is how an input's words reach the
// warp.  The direct kernel loads every literal word from global memory at
// the moment it is added, after a chain of dependent loads (packed class ->
// descriptor -> mask record -> literal), so a warp has at most one group of
// inputs in flight and waits on memory most of the time.  Here each active
// input's compressed words for the subtile -- one contiguous stream segment,
// found at build time (sseg) -- and, for a mixed input, its 64-byte mask
// record are copied into a per-warp ring of shared memory by 1-D bulk copies
// (cp.async.bulk, completion counted in bytes on an mbarrier per slot).  The
// ring has kSlots slots; copies run up to kSlots slots ahead of the adds, and
// a slot is refilled as soon as its inputs have been added.  Every word of a
// segment is read from HBM once and in full 16-byte units; the decode then
// finds a mixed input's literal at segment word pre[r] + popc(cm[r] below
// the lane) in shared memory instead of global memory.
//
// A copy always starts at an even stream word (16 bytes) and covers whole
// 16-byte units, so it may read one word before the segment and one after
// it; the index keeps two zero words after the last stream.  Waits on a slot
// give up after about a second (they only end that way if a copy never
// arrives), record a code in p.err (the host returns THR_E_TIMEOUT) and wait,
// again bounded, for the warp's other copies before the warp stops.
#pragma once

#include "thr_query_kernel.cuh"

namespace thr {

constexpr int kSlots = 4;          // ring slots per warp
constexpr int kSlotBytes = 1280;   // one slot
constexpr int kRingBytes = kSlots * kSlotBytes;
// the largest input: a mask record and kGW words from an odd stream word,
// in 16-byte units
static_assert(sizeof(MaskRec) + 16 * ((8 * (kGW + 1) + 15) / 16) <= kSlotBytes,
              "a slot holds any one input");
static_assert(kRingBytes < (1 << 13), "ring offsets take 13 bits");

struct StageWarp {
    alignas(16) unsigned char ring[kRingBytes];
    unsigned long long bar[kSlots];  // one mbarrier per slot
    // per record of the chunk: byte offset of its words in the ring | first
    // word odd << 13 | mixed << 14 | has ones-fill words << 15 | slot << 16
    uint32_t dir[kCH];
};
struct StageSmem {
    StageWarp w[kNW];
};

constexpr size_t staged_smem_bytes() { return sizeof(CtaSmem) + sizeof(StageSmem); }

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
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
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
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of parity `parity` to complete: false after about a
// second (or 2^26 polls) without it.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t i = 1; i < (1u << 26); ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 0u && global_ns() - t0 > 1000000000ull) return false;
    }
    return false;
}

// ------------------------------------------------------------ the ring

// Records of the staged kernel (ws.rec): x, y & 0xFF = stream index of the
// segment's first word (absolute); y >> 8 & 0x1FF = its words; y bit 30 =
// ones-fill words in the subtile, bit 31 = mixed; z, w = mask record index.
__device__ __forceinline__ uint4 staged_record(uint64_t seg, uint32_t len, bool mixed,
                                               uint32_t ones, uint64_t midx) {
    return make_uint4(uint32_t(seg),
                      uint32_t(seg >> 32) | (len << 8) | (ones << 30) | (mixed ? 1u << 31 : 0u),
                      uint32_t(midx), uint32_t(midx >> 32));
}

// Ring state of a warp (warp-uniform): per slot the records [beg, end) of
// its current fill (8 bits each, packed), which slots' fills have been
// waited for, and the next record to copy.
struct RingState {
    uint32_t beg, end;
    uint32_t waited;
    uint32_t fill;
};

// Copy into slot s the records fill, fill + 1, ... of the chunk that fit it
// (at least one: any single record fits an empty slot).  Warp-collective.
__device__ __forceinline__ void stage_slot(const PassAParams& p, const WarpSmem& ws,
                                           StageWarp& sw, uint32_t s, uint32_t nrec,
                                           uint32_t lane, RingState& rs) {
    const uint32_t j = rs.fill + lane;
    uint32_t size = 0, dbytes = 0, shift = 0, mixed = 0, ones = 0;
    uint64_t seg = 0, midx = 0;
    if (j < nrec) {
        const uint4 rec = ws.rec[j];
        seg = (uint64_t(rec.y & 0xFFu) << 32) | rec.x;
        const uint32_t len = (rec.y >> 8) & 0x1FFu;
        mixed = rec.y >> 31;
        ones = (rec.y >> 30) & 1u;
        midx = (uint64_t(rec.w) << 32) | rec.z;
        shift = uint32_t(seg & 1u);
        dbytes = (8u * (len + shift) + 15u) & ~15u;
        size = dbytes + (mixed ? uint32_t(sizeof(MaskRec)) : 0u);
    }
    uint32_t incl = size;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(~0u, incl, d);
        if (lane >= uint32_t(d)) incl += t;
    }
    const bool fits = j < nrec && incl <= uint32_t(kSlotBytes);
    const uint32_t m = __popc(__ballot_sync(~0u, fits));
    const uint32_t bar = smem_addr(&sw.bar[s]);
    if (m) {
        const uint32_t total = __shfl_sync(~0u, incl, m - 1);
        fence_proxy_async();
        if (lane == 0) mbar_expect_tx(bar, total + (p.lose ? 16u : 0u));
        __syncwarp();
        if (fits) {
            uint32_t off = s * uint32_t(kSlotBytes) + incl - size;
            if (mixed) {
                bulk_copy(smem_addr(sw.ring + off), p.masks + midx, uint32_t(sizeof(MaskRec)), bar);
                off += uint32_t(sizeof(MaskRec));
            }
            bulk_copy(smem_addr(sw.ring + off), p.words + (seg & ~1ull), dbytes, bar);
            sw.dir[j] = off | (shift << 13) | (mixed << 14) | (ones << 15) | (s << 16);
        }
    }
    const uint32_t sh = 8 * s;
    rs.beg = (rs.beg & ~(0xFFu << sh)) | (rs.fill << sh);
    rs.fill += m;
    rs.end = (rs.end & ~(0xFFu << sh)) | (rs.fill << sh);
    __syncwarp();
}

// After a failed wait: wait (bounded) for every fill not yet waited for, so
// that no copy is still writing the warp's ring when it stops.
__device__ __forceinline__ void drain_ring(StageWarp& sw, const RingState& rs, uint32_t phase) {
#pragma unroll
    for (uint32_t s = 0; s < uint32_t(kSlots); ++s) {
        const uint32_t b = (rs.beg >> (8 * s)) & 0xFFu, e = (rs.end >> (8 * s)) & 0xFFu;
        if (b != e && !((rs.waited >> s) & 1u)) mbar_wait(smem_addr(&sw.bar[s]), (phase >> s) & 1u);
    }
}

// Values of the group's records r0 .. r0 + kGroup - 1 at the lane's words
// x0 + 32 r + lane, from the ring: a literal run row by row, a mixed input
// through its mask record (the literal at segment word pre[r] + popc(cm[r]
// below the lane), a ones-fill word from the ones mask, else zero).
__device__ __forceinline__ void staged_decode(const StageWarp& sw, const uint32_t (&e)[kGroup],
                                              uint32_t r0, uint32_t nrec, uint32_t x0,
                                              uint32_t x1, uint32_t lane,
                                              uint64_t (&v)[kGroup][kRows]) {
    const uint32_t bit = 1u << lane;
    const uint32_t lt = bit - 1u;
#pragma unroll
    for (int j = 0; j < kGroup; ++j) {
#pragma unroll
        for (int r = 0; r < kRows; ++r) v[j][r] = 0;
        if (r0 + j >= nrec) continue;
        const uint32_t ej = e[j];
        const unsigned char* base = sw.ring + (ej & 0x1FFFu);
        const uint64_t* data = reinterpret_cast<const uint64_t*>(base) + ((ej >> 13) & 1u);
        if (!((ej >> 14) & 1u)) {  // a literal run: the subtile's words in order
#pragma unroll
            for (int r = 0; r < kRows; ++r)
                if (x0 + 32 * r + lane < x1) v[j][r] = data[32 * r + lane];
            continue;
        }
        const MaskRec* m = reinterpret_cast<const MaskRec*>(base - sizeof(MaskRec));
        const uint4 lmv = *reinterpret_cast<const uint4*>(m->lm);
        const uint4 cmv = *reinterpret_cast<const uint4*>(m->cm);
        const uint32_t pre = m->pre;
        const uint32_t lm[4] = {lmv.x, lmv.y, lmv.z, lmv.w};
        const uint32_t cm[4] = {cmv.x, cmv.y, cmv.z, cmv.w};
        if ((ej >> 15) & 1u) {  // ones-fill words too
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

// Add the chunk's nrec records into the counters through the ring: fill
// every slot, then per group of kGroup records wait for their slots, decode,
// add, and refill the slots whose records have all been added.  False when a
// wait gave up (after draining the ring).
template <class Count>
__device__ __forceinline__ bool staged_add(const PassAParams& p, const QView& q,
                                           const WarpSmem& ws, StageWarp& sw, uint32_t nrec,
                                           uint32_t x0, uint32_t x1, uint32_t lane,
                                           uint32_t& phase, Count& count) {
    RingState rs{0u, 0u, 0u, 0u};
    for (uint32_t s = 0; s < uint32_t(kSlots) && rs.fill < nrec; ++s)
        stage_slot(p, ws, sw, s, nrec, lane, rs);
    for (uint32_t r0 = 0; r0 < nrec; r0 += kGroup) {
        uint32_t e[kGroup];
#pragma unroll
        for (int j = 0; j < kGroup; ++j) {
            e[j] = r0 + j < nrec ? sw.dir[r0 + j] : 0u;
            if (r0 + j >= nrec) continue;
            const uint32_t s = (e[j] >> 16) & 3u;
            if (!((rs.waited >> s) & 1u)) {
                if (!mbar_wait(smem_addr(&sw.bar[s]), (phase >> s) & 1u)) {
                    drain_ring(sw, rs, phase);
                    return false;
                }
                phase ^= 1u << s;
                rs.waited |= 1u << s;
            }
        }
        uint64_t v[kGroup][kRows];
        staged_decode(sw, e, r0, nrec, x0, x1, lane, v);
        if (q.zmode()) {  // count the zeros of the active inputs
#pragma unroll
            for (int j = 0; j < kGroup; ++j)
#pragma unroll
                for (int r = 0; r < kRows; ++r)
                    if (r0 + j < nrec) v[j][r] = ~v[j][r];
        }
        count.add(v, min(uint32_t(kGroup), nrec - r0));
        // the values are in registers and added: slots whose records all lie
        // before r0 + kGroup (or that are empty) take the next records
        for (uint32_t s = 0; s < uint32_t(kSlots) && rs.fill < nrec; ++s) {
            const uint32_t b = (rs.beg >> (8 * s)) & 0xFFu, en = (rs.end >> (8 * s)) & 0xFFu;
            if (en <= r0 + kGroup && (b == en || ((rs.waited >> s) & 1u))) {
                rs.waited &= ~(1u << s);
                stage_slot(p, ws, sw, s, nrec, lane, rs);
            }
        }
    }
    return true;
}

// The largest number of inputs with a non-zero word at one position of the
// subtile (as max_position_count, for the staged records).
__device__ __forceinline__ uint32_t staged_max_position_count(const PassAParams& p,
                                                              const WarpSmem& ws, uint32_t nrec,
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

// Counting part of a subtile's result with staged inputs: classification and
// pruning as in count_subtile, then the active inputs through the ring.
// ok = false when a wait gave up.
template <class Count>
__device__ __forceinline__ void staged_count_subtile(const PassAParams& p, const QView& q,
                                                     uint32_t x0, uint32_t x1, uint32_t lane,
                                                     WarpSmem& ws, StageWarp& sw,
                                                     uint32_t& phase, Count& count,
                                                     uint32_t& k_ones, uint32_t& d_act,
                                                     bool& ok) {
    const uint32_t g = x0 / kGW;
    count.begin();
    k_ones = 0;
    d_act = 0;
    ok = true;
    const bool one_chunk = q.n() <= uint32_t(kCH);
    bool pruned = false;
    if (!one_chunk) {  // classify every input first so that pruning still applies
        for (uint32_t i0 = 0; i0 < q.n(); i0 += 32) {
            const uint32_t i = i0 + lane;
            uint32_t cls = 0;
            if (i < q.n())
                cls = uint32_t(__ldg(p.pcls + uint64_t(__ldg(q.ids() + i)) * p.NGW + (g >> 5)) >>
                               (2 * (g & 31))) & 3u;
            k_ones += __popc(__ballot_sync(~0u, cls == 1));
            d_act += __popc(__ballot_sync(~0u, cls >= 2));
        }
        pruned = q.decided(k_ones, d_act);
    }
    for (uint32_t c0 = 0; c0 < q.n() && !pruned; c0 += kCH) {
        const uint32_t cn = min(uint32_t(kCH), q.n() - c0);
        uint32_t nrec = 0;
        // 1. classify, lane per input: packed class, then the segment (and
        //    for a mixed input the mask record) of inputs with literals
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
            if (one_chunk) k_ones += __popc(__ballot_sync(~0u, cls == 1));
            const uint32_t act = __ballot_sync(~0u, cls >= 2);
            if (cls >= 2) ws.rec[nrec + __popc(act & ((1u << lane) - 1u))] = r;
            nrec += __popc(act);
        }
        __syncwarp();
        if (one_chunk) {  // run-aware pruning (Sec. 6.4 cases 1 and 2)
            d_act = nrec;
            if (q.decided(k_ones, d_act)) break;
            // finer: no word of the subtile is non-zero in T' inputs
            const int64_t tp = int64_t(q.T()) - int64_t(k_ones);
            if (q.sym() != kSymOdd && tp >= 4 && 4 * tp >= int64_t(d_act) &&
                int64_t(staged_max_position_count(p, ws, nrec, lane)) < tp) {
                k_ones = 0;  // finish: T > k + d, every row zero
                d_act = 0;
                break;
            }
        }
        // 2. the active inputs into the counters through the ring
        if (!staged_add(p, q, ws, sw, nrec, x0, x1, lane, phase, count)) {
            ok = false;
            return;
        }
        __syncwarp();
    }
}

// Pass A driver of the staged kernel: pass_a with staged counting.  A warp
// whose wait gave up records the code and stops.
template <class Count>
__device__ __forceinline__ void staged_pass_a(const PassAParams& p, CtaSmem& sm, StageSmem& ss,
                                              Count& count) {
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    WarpSmem& ws = sm.w[wid];
    StageWarp& sw = ss.w[wid];
    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < kSlots; ++s) mbar_init(smem_addr(&sw.bar[s]), 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t phase = 0;  // per slot: parity of its next completion
    const uint32_t nwarps = gridDim.x * kNW;
    const uint32_t nitems = p.nlist * p.NG;
    uint32_t cur = ~0u;
    uint2 grp = make_uint2(0, 1);
    const QView q{ws, p.ids};
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
        const uint32_t s = __ldg(p.list + li);
        if (s != cur) {
            const QDesc d = p.qd[s];
            load_query(p, ws, d.ids_off, d.n, d.Tlo, d.zmode, d.Thi, d.hi, d.sym, lane);
            grp = p.grp[s];
            cur = s;
        }
        const uint32_t x0 = g * uint32_t(kGW);
        const uint32_t x1 = min(x0 + uint32_t(kGW), p.W);
        uint64_t orow[kRows];
        uint32_t k_ones = 0, d_act = 0;
        bool ok = true;
        staged_count_subtile(p, q, x0, x1, lane, ws, sw, phase, count, k_ones, d_act, ok);
        if (!ok) {
            if (lane == 0) atomicOr(p.err, 1u);
            return;
        }
        if (grp.y <= 1) {
            finish_subtile(p, q.T(), q.zmode(), q.hi(), q.sym(), k_ones, d_act, x0, lane, count,
                           orow);
            store_subtile(p, ws, cur, g, x0, x1, lane, orow);
        } else if constexpr (Count::kInlineGroups) {
            for (uint32_t i = 0; i < grp.y; ++i) {
                const uint32_t m = __ldg(p.memb + grp.x + i);
                finish_subtile(p, p.qd[m].T, 0u, 0u, kSymThreshold, k_ones, d_act, x0, lane,
                               count, orow);
                store_subtile(p, ws, m, g, x0, x1, lane, orow);
            }
        } else {
            Count copy = count;
            finish_group(p, ws, grp, g, x0, x1, lane, k_ones, d_act, &copy);
        }
        it = p.work ? __shfl_sync(~0u, next, 0) : it + nwarps;
    }
}

// The staged carry-save kernel, S-bit counters.  Four CTAs per SM (the ring
// takes 22 KB of shared memory per CTA besides the warps' records).
template <int S>
__global__ void __launch_bounds__(kNT, (S <= 6 ? 4 : (S <= 8 ? 3 : 2))) k_staged(const PassAParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CtaSmem& sm = *reinterpret_cast<CtaSmem*>(smem_raw);
    StageSmem& ss = *reinterpret_cast<StageSmem*>(smem_raw + sizeof(CtaSmem));
    CsaCount<S> count;
    staged_pass_a<CsaCount<S>>(p, sm, ss, count);
}

}  // namespace thr
