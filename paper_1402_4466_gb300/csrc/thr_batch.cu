// Batches of threshold queries: planning (chunks of queries whose scratch
// fits, and per chunk one pass-A launch per kernel class), execution on a
// stream, optionally as a CUDA graph captured per batch shape and replayed.
//
// Every query of a batch gets a slot of scratch (its result words and
// re-encoding aggregates) in its chunk; the chunks run one after the other,
// the pass-A launches of a chunk side by side.  Pass B of each chunk places
// the chunk's results in the output pool after those of the earlier chunks,
// so the results lie in query order without a host round trip.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <utility>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "../../include/thr.h"
#include "thr_batch.h"
#include "thr_launch.h"

namespace thr {

namespace {

thr_status cuda_error(cudaError_t e, const char* what) {
    char msg[256];
    std::snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString(e));
    return report_error(e == cudaErrorMemoryAllocation ? THR_E_NOMEM : THR_E_CUDA, msg);
}

#define CKB(call, what)                                  \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_error(e_, what); \
    } while (0)

constexpr int kAux = 3;  // side streams for concurrent pass-A launches

// Per host thread: pinned staging, side streams, fork events, the capture
// stream and the cache of instantiated graphs.
struct GraphSlot {
    uint64_t key = 0;
    uint64_t sig = 0;  // every parameter the captured work depends on
    cudaGraphExec_t exec = nullptr;
    uint64_t used = 0;
};

struct ThreadCtx {
    int device = -1;
    unsigned char* pin = nullptr;
    size_t pin_bytes = 0;
    size_t pin_grown = 0;  // size of the last allocation (growth is geometric)
    cudaStream_t aux[kAux] = {};
    cudaEvent_t fork[kAux + 1] = {};
    cudaEvent_t join_in = nullptr;  // orders the capture stream after the caller's
    cudaStream_t cs = nullptr;      // capture stream
    GraphSlot graphs[8];
    uint64_t clock = 0;
    int per_sm[kNumClasses] = {};  // resident CTAs per SM of each kernel class
    bool ok = false;

    cudaError_t init(int dev) {
        if (ok && device == dev) return cudaSuccess;
        release();
        cudaError_t e;
        for (int k = 0; k < kAux; ++k)
            if ((e = cudaStreamCreateWithFlags(&aux[k], cudaStreamNonBlocking)) != cudaSuccess)
                return e;
        for (int k = 0; k <= kAux; ++k)
            if ((e = cudaEventCreateWithFlags(&fork[k], cudaEventDisableTiming)) != cudaSuccess)
                return e;
        if ((e = cudaEventCreateWithFlags(&join_in, cudaEventDisableTiming)) != cudaSuccess)
            return e;
        if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) return e;
        device = dev;
        for (int c = 0; c < kNumClasses; ++c) per_sm[c] = 0;
        ok = true;
        return cudaSuccess;
    }
    void drop_graphs() {
        for (auto& g : graphs)
            if (g.exec) {
                cudaGraphExecDestroy(g.exec);
                g = GraphSlot{};
            }
    }
    void release() {
        if (!ok) return;
        drop_graphs();
        for (int k = 0; k < kAux; ++k) cudaStreamDestroy(aux[k]);
        for (int k = 0; k <= kAux; ++k) cudaEventDestroy(fork[k]);
        cudaEventDestroy(join_in);
        cudaStreamDestroy(cs);
        ok = false;
    }
    cudaError_t pinned(size_t bytes, unsigned char** out) {
        if (pin_bytes < bytes) {
            // Every cached graph copies to and from this buffer, and the
            // copy nodes keep the mapping of the allocation they were made
            // with.  A new allocation can come back at the same address (so
            // a graph's signature would still match), and replaying such a
            // graph would copy through the freed allocation's mapping: a
            // host crash or a GPU fault.  So the graphs go first.  The buffer
            // grows at least twofold, in whole 64 KiB, so that this is rare.
            drop_graphs();
            if (pin) cudaFreeHost(pin);
            pin = nullptr;
            pin_bytes = 0;
            const size_t want = (std::max(bytes, 2 * pin_grown) + 65535) & ~size_t(65535);
            cudaError_t e = cudaMallocHost(&pin, want);
            if (e != cudaSuccess) return e;
            pin_bytes = want;
            pin_grown = want;
        }
        *out = pin;
        return cudaSuccess;
    }
    ~ThreadCtx() {
        // the CUDA runtime may already be shutting down at thread exit;
        // leave the handles to process teardown then
        if (pin) cudaFreeHost(pin);
    }
};
thread_local ThreadCtx g_ctx;

size_t r256(size_t v) { return (v + 255) & ~size_t(255); }

uint64_t fnv(uint64_t h, uint64_t v) {
    for (int i = 0; i < 8; ++i) {
        h ^= (v >> (8 * i)) & 0xFF;
        h *= 1099511628211ull;
    }
    return h;
}


uint64_t env_u64(const char* name, uint64_t dflt) {
    const char* v = std::getenv(name);
    if (!v || !*v) return dflt;
    return std::strtoull(v, nullptr, 10);
}

// Does a query classify its inputs from their subtile descriptors alone
// (QDesc::direct)?  When most of its inputs hold literals in most subtiles:
// an input's share of subtiles with literals is estimated as min(1, stream
// words / subtiles), and the shares must add up to half the inputs.  Else
// the packed classes keep the zero-fill inputs from costing a descriptor
// load each.
bool direct_classification(const thr_index* idx, const uint32_t* ids, uint32_t n) {
    double share = 0;
    for (uint32_t i = 0; i < n; ++i)
        share += std::min(1.0, double(idx->desc[ids[i]].len) / double(idx->NG));
    return 2.0 * share >= double(n);
}

// Groups among the chunk's grouped-carry-save queries over the same id
// multiset: the first member leads, counts ones with enough slices for the
// group's largest threshold and prunes only subtiles decided for every
// member; the others are absorbed (no launch of their own).
void form_groups(const BatchInput& in, uint32_t q0, uint32_t Q, std::vector<QDesc>& qd,
                 std::vector<uint8_t>& qcls, std::vector<uint2>& grp,
                 std::vector<uint32_t>& memb, std::vector<uint8_t>& absorbed) {
    // an order-independent hash of each multiset (a sum of mixed ids), so
    // that only queries whose hashes meet are sorted and compared
    std::vector<std::pair<uint64_t, uint32_t>> keys;  // (hash, slot)
    keys.reserve(Q);
    for (uint32_t s = 0; s < Q; ++s) {
        const uint32_t q = q0 + s;
        if (class_family(qcls[q]) != 0 || qd[q].sym != kSymThreshold) continue;
        uint64_t h = fnv(14695981039346656037ull, in.id_off[q + 1] - in.id_off[q]);
        for (uint32_t i = in.id_off[q]; i < in.id_off[q + 1]; ++i) {
            uint64_t z = uint64_t(in.ids[i]) + 0x9E3779B97F4A7C15ull;  // splitmix64 finaliser
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            h += z ^ (z >> 31);
        }
        keys.emplace_back(h, s);
    }
    std::sort(keys.begin(), keys.end());
    int cnt = 0;
    const KernelEntry* tab = kernel_table(&cnt);
    auto sorted_ids = [&](uint32_t s) {
        std::vector<uint32_t> v(in.ids + in.id_off[q0 + s], in.ids + in.id_off[q0 + s + 1]);
        std::sort(v.begin(), v.end());
        return v;
    };
    for (size_t i = 0; i < keys.size();) {
        size_t j = i + 1;
        while (j < keys.size() && keys[j].first == keys[i].first) ++j;
        if (j - i < 2) {
            i = j;
            continue;
        }
        // exact matches only (hash collisions stay apart)
        const std::vector<uint32_t> lead_ids = sorted_ids(keys[i].second);
        std::vector<uint32_t> mem{keys[i].second};
        for (size_t k = i + 1; k < j; ++k)
            if (sorted_ids(keys[k].second) == lead_ids) mem.push_back(keys[k].second);
        i = j;
        if (mem.size() < 2) continue;
        std::sort(mem.begin(), mem.end());
        const uint32_t n = qd[q0 + mem[0]].n;
        uint32_t tlo = ~0u, thi = 0;
        int need = 1;
        for (uint32_t m : mem) {
            const uint32_t T = qd[q0 + m].T;
            tlo = std::min(tlo, T);
            thi = std::max(thi, T);
            if (T >= 1 && T <= n) need = std::max(need, slices_for(T));
        }
        int c = -1;
        for (int w = 0; w < cnt; ++w)
            if (tab[w].S >= need) {
                c = w;
                break;
            }
        if (c < 0) continue;  // too wide for the counters: no sharing
        const uint32_t lead = q0 + mem[0];
        qd[lead].Tlo = tlo;
        qd[lead].Thi = thi;
        qd[lead].zmode = 0;  // ones are counted for every member
        qcls[lead] = uint8_t(c);
        grp[lead] = make_uint2(uint32_t(memb.size()), uint32_t(mem.size()));
        for (uint32_t m : mem) {
            memb.push_back(m);
            if (q0 + m != lead) absorbed[q0 + m] = 1;
        }
    }
}

}  // namespace

bool trace_time_on() {
    static const bool on = [] {
        const char* v = std::getenv("THR_TRACE_TIME");
        return v && v[0] == '1';
    }();
    return on;
}
double now_us() {
    return std::chrono::duration<double, std::micro>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

thr_status run_batch(const thr_index* idx, const BatchInput& in, uint64_t* dpool, uint64_t cap,
                     uint64_t* h_off, uint64_t* h_len, uint64_t* total, cudaStream_t st,
                     const BatchOptions& opt, BatchStats* stats) {
    const uint32_t nq = in.nq;
    const uint32_t W = idx->W, NG = idx->NG;
    const double t0 = trace_time_on() ? now_us() : 0.0;
    double t_plan = 0, t_stage = 0, t_launch = 0;
    CKB(g_ctx.init(idx->device), "per-thread streams");

    // ---- chunking: as many slots per chunk as the scratch budget allows
    const uint64_t per_slot = scratch_per_slot(W, NG);
    uint64_t budget = opt.scratch_bytes;
    if (!budget) {
        budget = 256ull << 20;  // always granted; more when the device has room
        if (uint64_t(nq) * per_slot > budget) {
            size_t free_b = 0, total_b = 0;
            CKB(cudaMemGetInfo(&free_b, &total_b), "device memory info");
            budget = std::max<uint64_t>(budget, std::min<uint64_t>(8ull << 30, free_b / 4));
        }
    }
    uint64_t Qmax = std::max<uint64_t>(1, budget / per_slot);
    Qmax = std::min<uint64_t>(Qmax, (uint64_t(1) << 31) / NG);  // pass C grid, item counters
    Qmax = std::min<uint64_t>(Qmax, env_u64("THR_MAX_SLOTS", Qmax));
    Qmax = std::max<uint64_t>(Qmax, 1);
    Qmax = std::min<uint64_t>(Qmax, nq);

    // ---- per query: kernel class, zero counting; per chunk: launches
    std::vector<QDesc> qd(nq);
    std::vector<uint8_t> qcls(nq);
    for (uint32_t q = 0; q < nq; ++q) {
        const uint32_t n = in.id_off[q + 1] - in.id_off[q];
        int cls = 0;
        uint32_t z = 0;
        const uint32_t sym = in.sym ? in.sym[q] : kSymThreshold;
        const uint32_t hi = (in.hi && sym == kSymRange) ? in.hi[q] : 0u;
        if (sym == kSymThreshold) {
            resolve_variant(n, in.T[q], in.variant ? in.variant[q] : kVarCsa, &cls, &z);
        } else {  // ranges and parity: carry-save counting ones, 2^S >= min(hi, n) + 1
            const uint64_t top = sym == kSymRange ? std::min<uint64_t>(hi, n) + 1 : 1;
            const int need = slices_for(top);
            int cnt = 0;
            const KernelEntry* tab = kernel_table(&cnt);
            cls = cnt - 1;
            for (int w = 0; w < cnt; ++w)
                if (tab[w].S >= need) {
                    cls = w;
                    break;
                }
            z = 0;
        }
        qd[q] = QDesc{in.id_off[q], n, in.T[q], z, in.T[q], in.T[q], hi, sym, 0u};
        qd[q].direct = direct_classification(idx, in.ids + in.id_off[q], n) ? 1u : 0u;
        qcls[q] = uint8_t(cls);
    }
    // groups of queries over the same id multiset (grouped carry-save, same
    // chunk): one counting pass serves them all (grp / memb, PassAParams)
    std::vector<uint2> grp(nq, make_uint2(0, 1));
    std::vector<uint32_t> memb;
    std::vector<uint8_t> absorbed(nq, 0);
    int* per_sm = g_ctx.per_sm;
    // THR_TUNE_CONFIG=k in the environment forces configuration k (testing)
    const uint64_t env_cfg = env_u64("THR_TUNE_CONFIG", kTuneCandidates);
    std::vector<ChunkPlan> chunks;
    std::vector<Launch> launches;
    std::vector<uint32_t> lists;
    lists.reserve(nq);
    uint64_t key = fnv(14695981039346656037ull, nq > 0 ? 1 : 0);
    uint32_t first_cfg = 0, first_key = 0;
    for (uint32_t q0 = 0; q0 < nq; q0 += uint32_t(Qmax)) {
        const uint32_t Q = uint32_t(std::min<uint64_t>(Qmax, nq - q0));
        ChunkPlan ch{q0, Q, uint32_t(launches.size()), 0};
        if (opt.share) form_groups(in, q0, Q, qd, qcls, grp, memb, absorbed);
        // the chunk's shape and its launch configuration
        uint64_t present = 0;
        double sum_n = 0;
        int widest[kNumFamilies];  // per family
        std::fill(widest, widest + kNumFamilies, -1);
        for (uint32_t s = 0; s < Q; ++s) {
            if (absorbed[q0 + s]) continue;
            const int c = qcls[q0 + s];
            present |= uint64_t(1) << c;
            sum_n += qd[q0 + s].n;
            widest[class_family(c)] = std::max(widest[class_family(c)], c);
        }
        const bool multi = __builtin_popcountll(present) > 1;
        const uint32_t shape = tune_key(multi, sum_n / Q);
        if (q0 == 0) first_key = shape;
        uint32_t cfg = opt.force_tune >= 0 ? uint32_t(opt.force_tune) : tune_lookup(idx, shape);
        if (opt.force_tune < 0 && env_cfg < kTuneCandidates) cfg = uint32_t(env_cfg);
        if (q0 == 0) first_cfg = cfg;
        if (cfg & kTuneMerge) {  // one counter width per carry-save family
            for (uint32_t s = 0; s < Q; ++s) {
                const int fam = class_family(qcls[q0 + s]);
                if (fam != 1) qcls[q0 + s] = uint8_t(widest[fam]);
            }
        }
        double work[kNumClasses] = {};
        double work_all = 0;
        for (uint32_t s = 0; s < Q; ++s) {  // cost ~ inputs x counter slices
            if (absorbed[q0 + s]) continue;
            const int c = qcls[q0 + s];
            const double w =
                double(qd[q0 + s].n) * (class_family(c) == 1 ? 4.0 : 2.0 + class_width(c));
            work[c] += w;
            work_all += w;
        }
        for (int c = 0; c < kNumClasses; ++c) {
            const uint32_t off = uint32_t(lists.size());
            for (uint32_t s = 0; s < Q; ++s)
                if (qcls[q0 + s] == c && !absorbed[q0 + s]) lists.push_back(s);
            const uint32_t cnt = uint32_t(lists.size()) - off;
            if (!cnt) continue;
            if (!per_sm[c]) {  // once per thread and device
                CKB(class_occupancy(c, &per_sm[c]), "occupancy");
                per_sm[c] = std::max(per_sm[c], 1);
            }
            Launch L{c, off, cnt, (cfg & kTuneOrder) ? 1u : 0u, 1,
                     (cfg & kTuneDynamic) ? 1u : 0u};
            const uint64_t items = uint64_t(cnt) * NG;
            double ctas = double(per_sm[c]) * idx->num_sms;
            if ((cfg & kTuneSplit) && work_all > 0) ctas *= work[c] / work_all;
            // a CTA takes kNW items at a time, or one with the inputs split
            const uint64_t per_cta = class_family(c) == 3 ? 1 : kNW;
            L.grid = int(std::max<uint64_t>(
                1, std::min<uint64_t>((items + per_cta - 1) / per_cta, uint64_t(ctas + 0.5))));
            launches.push_back(L);
            key = fnv(key, uint64_t(c) << 8 | 1);
        }
        ch.l1 = uint32_t(launches.size());
        chunks.push_back(ch);
        key = fnv(key, 0xC);
    }
    if (stats) {
        stats->chunks = uint32_t(chunks.size());
        stats->launches = uint32_t(launches.size());
        stats->slots = uint32_t(Qmax);
        stats->tune = first_cfg;
        stats->tune_key = first_key;
    }

    if (t0 > 0) t_plan = now_us();
    // ---- device memory: plan (descriptors, ids, lists) | scratch
    const uint64_t nids = in.id_off[nq];
    const size_t o_qd = 0;
    const size_t o_ids = r256(sizeof(QDesc) * nq);
    const size_t o_lists = o_ids + r256(sizeof(uint32_t) * nids);
    const size_t o_grp = o_lists + r256(sizeof(uint32_t) * lists.size());
    const size_t o_memb = o_grp + r256(sizeof(uint2) * nq);
    const size_t plan_bytes = o_memb + r256(sizeof(uint32_t) * std::max<size_t>(memb.size(), 1));
    const ScratchLayout lay = scratch_layout(Qmax, nq, W, NG, launches.size());
    const size_t res_bytes = (lay.res - lay.base) + 16 * size_t(nq);
    // the plan and, right after it (where the scratch starts on the device),
    // the zeroed control words go up in one copy: no memset node
    const size_t up_bytes = plan_bytes + lay.full;
    unsigned char* pin = nullptr;
    CKB(g_ctx.pinned(r256(up_bytes) + r256(res_bytes), &pin), "pinned staging");
    std::memset(pin + plan_bytes, 0, lay.full);
    std::memcpy(pin + o_qd, qd.data(), sizeof(QDesc) * nq);
    std::memcpy(pin + o_ids, in.ids, sizeof(uint32_t) * nids);
    std::memcpy(pin + o_lists, lists.data(), sizeof(uint32_t) * lists.size());
    std::memcpy(pin + o_grp, grp.data(), sizeof(uint2) * nq);
    if (!memb.empty()) std::memcpy(pin + o_memb, memb.data(), sizeof(uint32_t) * memb.size());
    // read back from base on: total, error word, check record, then the results
    unsigned long long* h_ctl = reinterpret_cast<unsigned long long*>(pin + r256(up_bytes));
    const unsigned long long* h_res = h_ctl + (lay.res - lay.base) / 8;

    if (t0 > 0) t_stage = now_us();
    const bool graph = opt.graph && !opt.profile;
    cudaStream_t xs = graph ? g_ctx.cs : st;  // the stream the work is enqueued on
    if (graph) {  // the capture stream starts after the caller's earlier work
        CKB(cudaEventRecord(g_ctx.join_in, st), "order streams");
        CKB(cudaStreamWaitEvent(xs, g_ctx.join_in, 0), "order streams");
    }
    unsigned char* dmem = nullptr;
    CKB(cudaMallocAsync(reinterpret_cast<void**>(&dmem), plan_bytes + lay.total, xs),
        "batch scratch");
    struct Free {
        unsigned char* p;
        cudaStream_t s;
        ~Free() {
            if (p) cudaFreeAsync(p, s);
        }
    } free_guard{dmem, xs};
    ExecBufs b{};
    b.qd = reinterpret_cast<const QDesc*>(dmem + o_qd);
    b.ids = reinterpret_cast<const uint32_t*>(dmem + o_ids);
    b.lists = reinterpret_cast<const uint32_t*>(dmem + o_lists);
    b.grp = reinterpret_cast<const uint2*>(dmem + o_grp);
    b.memb = reinterpret_cast<const uint32_t*>(dmem + o_memb);
    b.scratch = dmem + plan_bytes;
    b.lay = lay;
    b.out = dpool;
    b.cap = cap;
    b.nids = uint32_t(nids);
    b.nq = nq;
    b.nmemb = uint32_t(memb.size());

    std::vector<cudaEvent_t> tev;
    PassATimer timer{nullptr};
    if (opt.profile) {
        tev.resize(2 * chunks.size());
        for (auto& e : tev) CKB(cudaEventCreate(&e), "profile events");
        timer.ev = tev.data();
    }
    struct EvFree {
        std::vector<cudaEvent_t>& v;
        ~EvFree() {
            for (auto e : v) cudaEventDestroy(e);
        }
    } ev_guard{tev};

    auto enqueue = [&](cudaStream_t s) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(dmem, pin, up_bytes, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
        e = enqueue_plan(idx, chunks.data(), uint32_t(chunks.size()), launches.data(), b, s,
                         g_ctx.aux, kAux, g_ctx.fork, kAux + 1, opt.profile ? &timer : nullptr,
                         true);
        if (e != cudaSuccess) return e;
        return cudaMemcpyAsync(h_ctl, b.scratch + lay.base, res_bytes, cudaMemcpyDeviceToHost,
                               s);
    };

    // the captured work depends on the plan's shape, the launches, the
    // device and pinned buffers and the output: when all of them equal those
    // of a cached executable, it is launched as it is (its copy of the plan
    // reads the pinned staging, which holds this call's plan)
    uint64_t sig = fnv(key, plan_bytes);
    for (size_t v : {o_ids, o_lists, o_grp, o_memb, lay.gtick, lay.base, lay.err, lay.work, lay.tick,
                     lay.res, lay.full, lay.bagg, lay.bpref, lay.aggs, lay.pref, lay.U, lay.total})
        sig = fnv(sig, v);
    sig = fnv(sig, nq);
#ifdef THR_CHECKED
    // the check limits are kernel parameters: a replayed graph must have these
    sig = fnv(sig, nids);
    sig = fnv(sig, memb.size());
#endif
    sig = fnv(sig, reinterpret_cast<uintptr_t>(dmem));
    sig = fnv(sig, reinterpret_cast<uintptr_t>(pin));
    sig = fnv(sig, reinterpret_cast<uintptr_t>(dpool));
    sig = fnv(sig, cap);
    // the index's arrays the kernels read (another index may reuse the same
    // host object address, or the same device addresses with its own data)
    for (const void* ptr : {static_cast<const void*>(idx), static_cast<const void*>(idx->d_words),
                            static_cast<const void*>(idx->d_sdesc),
                            static_cast<const void*>(idx->d_pcls),
                            static_cast<const void*>(idx->d_masks),
                            static_cast<const void*>(idx->d_sseg),
                            static_cast<const void*>(idx->d_desc)})
        sig = fnv(sig, reinterpret_cast<uintptr_t>(ptr));
    sig = fnv(sig, uint64_t(idx->W) << 32 | idx->NG);
    sig = fnv(sig, idx->r);
    sig = fnv(sig, test_lost_copy());
    for (const Launch& L : launches) {
        sig = fnv(sig, uint64_t(uint32_t(L.cls)) << 32 | L.list_off);
        sig = fnv(sig, uint64_t(L.nlist) << 32 | uint64_t(uint32_t(L.grid)));
        sig = fnv(sig, uint64_t(L.order) << 32 | L.dynamic);
    }
    for (const ChunkPlan& c : chunks) {
        sig = fnv(sig, uint64_t(c.q0) << 32 | c.Q);
        sig = fnv(sig, uint64_t(c.l0) << 32 | c.l1);
    }
    GraphSlot* same = nullptr;
    if (graph)
        for (auto& g : g_ctx.graphs)
            if (g.exec && g.key == key && g.sig == sig) same = &g;
    if (same) {
        same->used = ++g_ctx.clock;
        if (stats) stats->graph_reused = 1;
        CKB(cudaGraphLaunch(same->exec, xs), "launch graph");
    } else if (graph) {
        CKB(cudaStreamBeginCapture(xs, cudaStreamCaptureModeThreadLocal), "begin capture");
        const cudaError_t ee = enqueue(xs);
        cudaGraph_t gr = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(xs, &gr);
        if (ee != cudaSuccess) {
            if (gr) cudaGraphDestroy(gr);
            return cuda_error(ee, "enqueue (capture)");
        }
        CKB(ec, "end capture");
        // reuse an executable graph of the same shape (update its parameters)
        GraphSlot* slot = nullptr;
        for (auto& g : g_ctx.graphs)
            if (g.exec && g.key == key) slot = &g;
        bool ready = false;
        if (slot) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(slot->exec, gr, &info) == cudaSuccess) {
                ready = true;
                if (stats) stats->graph_reused = 1;
            } else {
                cudaGetLastError();
                cudaGraphExecDestroy(slot->exec);
                slot->exec = nullptr;
            }
        }
        if (!ready) {
            if (!slot) {  // least recently used slot
                slot = &g_ctx.graphs[0];
                for (auto& g : g_ctx.graphs)
                    if (!g.exec || g.used < slot->used) slot = &g;
                if (slot->exec) cudaGraphExecDestroy(slot->exec);
                slot->exec = nullptr;
            }
            const cudaError_t ei = cudaGraphInstantiate(&slot->exec, gr, 0);
            if (ei != cudaSuccess) {
                cudaGraphDestroy(gr);
                slot->exec = nullptr;
                return cuda_error(ei, "instantiate graph");
            }
            slot->key = key;
            if (stats) stats->graph_reused = 0;
        }
        slot->sig = sig;
        slot->used = ++g_ctx.clock;
        cudaGraphDestroy(gr);
        CKB(cudaGraphLaunch(slot->exec, xs), "launch graph");
    } else {
        CKB(enqueue(xs), "enqueue");
    }
    if (t0 > 0) t_launch = now_us();
    CKB(cudaStreamSynchronize(xs), "batch");
    if (t0 > 0)
        std::fprintf(stderr, "[thr] batch nq=%u plan %.1f stage %.1f launch %.1f wait %.1f us\n",
                     nq, t_plan - t0, t_stage - t_plan, t_launch - t_stage, now_us() - t_launch);
    if (opt.profile) {
        double ms = 0;
        for (size_t c = 0; c < chunks.size(); ++c) {
            float t = 0.f;
            CKB(cudaEventElapsedTime(&t, tev[2 * c], tev[2 * c + 1]), "profile time");
            ms += t;
        }
        if (stats) stats->pass_a_ms = ms;
    }
    if (h_ctl[(lay.err - lay.base) / 8] & 0xFFFFFFFFull)
        return report_error(THR_E_TIMEOUT,
                            "a query kernel gave up waiting for its shared-memory copies");
    {
        CheckRec c;
        std::memcpy(&c, reinterpret_cast<const unsigned char*>(h_ctl) + (lay.chk - lay.base),
                    sizeof c);
        if (c.site) return check_failed(c);
    }
    for (uint32_t q = 0; q < nq; ++q) {
        h_off[q] = h_res[2 * size_t(q)];
        h_len[q] = h_res[2 * size_t(q) + 1];
    }
    *total = h_ctl[0];
    return THR_OK;
}

}  // namespace thr
