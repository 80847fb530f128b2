// Enqueueing a launch plan: the three passes of every chunk of a batch.
#include "thr_exec.h"

#include <algorithm>
#include <cstdio>
#include <cstdlib>

#include "thr_index.h"
#include "thr_launch.h"

namespace thr {

namespace {

size_t r256(size_t v) { return (v + 255) & ~size_t(255); }

int bits_of(uint64_t v) {
    int n = 0;
    while (v) {
        ++n;
        v >>= 1;
    }
    return n;
}

}  // namespace

// The fewest counter slices (at least 1) that decide "count >= t": 2^S >= t
// (t = 2^S is decided by the sticky slice alone).
int slices_for(uint64_t t) { return t <= 2 ? 1 : bits_of(t - 1); }

namespace {

cudaError_t launch_class(int cls, const PassAParams& p, int grid, cudaStream_t st) {
    if (class_family(cls) == 1) return launch_scancount(cls == kClassScanCount16, p, grid, st);
    if (class_family(cls) == 4)
        return cls < kNumClasses ? launch_looped(cls - kClassLooped + 1, p, grid, st)
                                 : cudaErrorInvalidValue;
    int cnt = 0;
    const KernelEntry* tab = kernel_table(&cnt);
    const int w = class_width(cls);
    if (cls < 0 || cls >= kNumClasses || w >= cnt) return cudaErrorInvalidValue;
    switch (class_family(cls)) {
        case 2: return tab[w].launch_pos(p, grid, st);
        case 3: return tab[w].launch_split ? tab[w].launch_split(p, grid, st)
                                           : cudaErrorInvalidValue;
        case 5: return tab[w].launch_staged(p, grid, st);
        default: return tab[w].launch(p, grid, st);
    }
}

}  // namespace

uint32_t scan_blocks(uint32_t NG) { return (NG + 255) / 256; }

uint32_t test_lost_copy() {
    const char* v = std::getenv("THR_TEST_LOST_COPY");
    return (v && v[0] == '1') ? 1u : 0u;
}

thr_status check_failed(const CheckRec& c) {
    static const char* const names[] = {"?",          "literal word", "mask record",
                                        "id position", "id value",     "subtile",
                                        "input record", "slot",        "group member",
                                        "staged mask record", "result of a query"};
    char msg[192];
    std::snprintf(msg, sizeof msg,
                  "checked build: %s index %llu not below %llu (thread %u, block %u); the "
                  "access was skipped and the results are not valid",
                  c.site < sizeof names / sizeof names[0] ? names[c.site] : "?", c.val, c.lim,
                  c.where & 1023u, c.where >> 10);
    return report_error(THR_E_CHECK, msg);
}

uint64_t scratch_per_slot(uint32_t W, uint32_t NG) {
    const uint64_t NB = scan_blocks(NG);
    return 4 + 32 + 2 * 32 * NB + 2 * 32 * uint64_t(NG) + 8 * uint64_t(NG) * kGW;
}

ScratchLayout scratch_layout(uint64_t Q, uint64_t nq, uint32_t W, uint32_t NG,
                             uint64_t nlaunch) {
    const uint64_t NB = scan_blocks(NG);
    const size_t agg = sizeof(uint32_t) * kAggWords;
    ScratchLayout l{};
    l.gtick = 0;
    l.base = 8;
    l.err = 16;  // a kernel that gave up waiting writes its code here
    l.chk = 32;  // checked builds: the first failed check (CheckRec)
    l.res = 64;  // right after the control words: one read-back covers both
    l.work = r256(l.res + 16 * nq);
    l.tick = l.work + r256(4 * nlaunch);
    l.full = l.tick + r256(4 * Q);
    l.bagg = l.full + r256(agg * Q);
    l.bpref = l.bagg + r256(agg * Q * NB);
    l.aggs = l.bpref + r256(agg * Q * NB);
    l.pref = l.aggs + r256(agg * Q * NG);
    l.U = l.pref + r256(agg * Q * NG);
    l.total = l.U + r256(8 * Q * uint64_t(NG) * kGW);
    return l;
}

void choose_class(uint32_t n, uint32_t T, int* cls, uint32_t* zmode) {
    int cnt = 0;
    const KernelEntry* tab = kernel_table(&cnt);
    uint32_t z = 0;
    int need = 1;
    if (T >= 1 && T <= n) {  // T = 0 and T > n never reach the counters
        const int s1 = slices_for(T), s0 = slices_for(uint64_t(n) - T + 1);
        z = s0 < s1 ? 1u : 0u;
        need = std::min(s1, s0);
    }
    int c = cnt - 1;
    for (int i = 0; i < cnt; ++i)
        if (tab[i].S >= need) {
            c = i;
            break;
        }
    *cls = c;
    *zmode = z;
}

void resolve_variant(uint32_t n, uint32_t T, int v, int* cls, uint32_t* zmode) {
    if (v == kVarLooped && T >= 1 && T <= uint32_t(kLoopedMax) && T <= n) {
        *cls = kClassLooped + int(T) - 1;
        *zmode = 0;
        return;
    }
    if (v == kVarScanCount && n <= 65535) {
        *cls = n <= 255 ? kClassScanCount : kClassScanCount16;
        *zmode = 0;
        return;
    }
    choose_class(n, T, cls, zmode);
    if (v == kVarStaged) {
        *cls += kClassStaged;
        return;
    }
    if (v == kVarSplit) {
        if (*cls < kSplitWidths) *cls += kClassSplit;
        return;
    }
    if (v == kVarPos) {  // ones counting: the first width with 2^S >= T
        int cnt = 0;
        const KernelEntry* tab = kernel_table(&cnt);
        const int need = (T >= 1 && T <= n) ? slices_for(T) : 1;
        int c = cnt - 1;
        for (int i = 0; i < cnt; ++i)
            if (tab[i].S >= need) {
                c = i;
                break;
            }
        *cls = kClassPos + c;
        *zmode = 0;
    }
}

cudaError_t class_occupancy(int cls, int* per_sm) {
    if (class_family(cls) == 1) return occupancy_scancount(cls == kClassScanCount16, per_sm);
    if (class_family(cls) == 4)
        return cls < kNumClasses ? occupancy_looped(cls - kClassLooped + 1, per_sm)
                                 : cudaErrorInvalidValue;
    int cnt = 0;
    const KernelEntry* tab = kernel_table(&cnt);
    const int w = class_width(cls);
    if (cls < 0 || cls >= kNumClasses || w >= cnt) return cudaErrorInvalidValue;
    switch (class_family(cls)) {
        case 2: return tab[w].occupancy_pos(per_sm);
        case 3: return tab[w].occupancy_split ? tab[w].occupancy_split(per_sm)
                                              : cudaErrorInvalidValue;
        case 5: return tab[w].occupancy_staged(per_sm);
        default: return tab[w].occupancy(per_sm);
    }
}

cudaError_t enqueue_plan(const thr_index* idx, const ChunkPlan* chunks, uint32_t nchunks,
                         const Launch* launches, const ExecBufs& b, cudaStream_t st,
                         cudaStream_t* aux, int naux, cudaEvent_t* fork_ev, int nfork_ev,
                         const PassATimer* timer, bool zeroed) {
    const ScratchLayout& l = b.lay;
    unsigned char* s = b.scratch;
    // control words (chunk ticket, running output offset, error word, check
    // record), the per-query results, work counters and slot tickets
    cudaError_t e = zeroed ? cudaSuccess : cudaMemsetAsync(s, 0, l.full, st);
    if (e != cudaSuccess) return e;
    const uint32_t NG = idx->NG;
    PassAParams p{};
    p.words = idx->d_words;
    p.sdesc = idx->d_sdesc;
    p.pcls = idx->d_pcls;
    p.NGW = (NG + 31) / 32;
    p.masks = idx->d_masks;
    p.sseg = idx->d_sseg;
    p.err = reinterpret_cast<uint32_t*>(s + l.err);
    p.lose = test_lost_copy();
#ifdef THR_CHECKED
    p.chk = reinterpret_cast<CheckRec*>(s + l.chk);
    p.lim.words = idx->total_words + 2;
    p.lim.masks = idx->mixed_subtiles;
    p.lim.nb = idx->nbitmaps;
    p.lim.nids = b.nids;
    p.lim.nq = b.nq;
    p.lim.nmemb = b.nmemb;
#endif
    p.desc = idx->d_desc;
    p.ids = b.ids;
    p.W = idx->W;
    p.NG = NG;
    p.ragged = uint32_t(idx->r % 64);
    p.U = reinterpret_cast<uint64_t*>(s + l.U);
    p.aggs = reinterpret_cast<uint32_t*>(s + l.aggs);
    WriteParams w{};
    w.chk = p.chk;
    w.chk_nq = b.nq;
    w.U = p.U;
    w.aggs = p.aggs;
    w.pref = reinterpret_cast<uint32_t*>(s + l.pref);
    w.bagg = reinterpret_cast<uint32_t*>(s + l.bagg);
    w.bpref = reinterpret_cast<uint32_t*>(s + l.bpref);
    w.full = reinterpret_cast<uint32_t*>(s + l.full);
    w.tick = reinterpret_cast<uint32_t*>(s + l.tick);
    w.gtick = reinterpret_cast<uint32_t*>(s + l.gtick);
    w.base = reinterpret_cast<unsigned long long*>(s + l.base);
    w.res = reinterpret_cast<unsigned long long*>(s + l.res);
    w.out = b.out;
    w.cap = b.cap;
    w.W = idx->W;
    w.NG = NG;
    w.NB = scan_blocks(NG);
    for (uint32_t c = 0; c < nchunks; ++c) {
        const ChunkPlan& ch = chunks[c];
        p.qd = b.qd + ch.q0;
        p.grp = b.grp + ch.q0;
        p.memb = b.memb;
        p.lim.slots = ch.Q;
        const uint32_t nl = ch.l1 - ch.l0;
        // several launches run side by side on the aux streams
        const int nside = std::min<int>(int(nl) - 1, std::min(naux, nfork_ev - 1));
        if (timer && timer->ev && (e = cudaEventRecord(timer->ev[2 * c], st)) != cudaSuccess)
            return e;
        if (nside > 0) {
            if ((e = cudaEventRecord(fork_ev[0], st)) != cudaSuccess) return e;
            for (int k = 0; k < nside; ++k)
                if ((e = cudaStreamWaitEvent(aux[k], fork_ev[0], 0)) != cudaSuccess) return e;
        }
        for (uint32_t i = 0; i < nl; ++i) {
            const Launch& L = launches[ch.l0 + i];
            p.list = b.lists + L.list_off;
            p.nlist = L.nlist;
            p.order = L.order;
            p.work = L.dynamic ? reinterpret_cast<uint32_t*>(s + l.work) + ch.l0 + i : nullptr;
            const int slot = nside > 0 ? int(i % uint32_t(nside + 1)) : 0;
            cudaStream_t ls = slot == 0 ? st : aux[slot - 1];
            if ((e = launch_class(L.cls, p, std::max(L.grid, 1), ls)) != cudaSuccess) return e;
        }
        for (int k = 0; k < nside; ++k) {
            if ((e = cudaEventRecord(fork_ev[1 + k], aux[k])) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(st, fork_ev[1 + k], 0)) != cudaSuccess) return e;
        }
        if (timer && timer->ev &&
            (e = cudaEventRecord(timer->ev[2 * c + 1], st)) != cudaSuccess)
            return e;
        w.Q = ch.Q;
        w.q0 = ch.q0;
        if ((e = launch_reencode(w, st)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace thr
