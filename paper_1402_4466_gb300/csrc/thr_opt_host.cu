// Host side of opt-threshold queries: the profiling pass of thr_opt.cuh
// over a batch of queries, and each query's answer from its histogram.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "thr_index.h"
#include "thr_opt.cuh"
#include "thr_opt_host.h"

namespace thr {

namespace {

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

thr_status cuda_error(cudaError_t e, const char* what) {
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    return report_error(e == cudaErrorMemoryAllocation ? THR_E_NOMEM : THR_E_CUDA, msg.c_str());
}

// Blocks per SM of each width's kernel on the calling thread's device
// (looked up once per thread and device).
int occupancy(const OptEntry& e, int slot, int device) {
    thread_local int dev = -1;
    thread_local int occ[32];
    if (dev != device) {
        std::fill(occ, occ + 32, 0);
        dev = device;
    }
    if (occ[slot] == 0) {
        int b = 0;
        if (e.occupancy(&b) != cudaSuccess || b < 1) b = 1;
        occ[slot] = b;
    }
    return occ[slot];
}

#define OPT_CK(call, what)                                    \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_error(e_, what);   \
    } while (0)

}  // namespace

// Narrow counters first: exact counts up to this bound, then a second pass
// with 2^S > n for the queries in which some count went beyond it.
constexpr uint32_t kNarrowCounts = 15;

// One profiling pass over the batch; exact: 2^S > n, else narrow counters,
// and ovf[q] (host) tells which queries must run again.
thr_status profile_pass(const thr_index* idx, uint32_t nq, const uint32_t* id_off,
                        const uint32_t* ids, const uint64_t* K, uint32_t* T, cudaStream_t st,
                        float* ms, bool exact, std::vector<uint32_t>* ovf_out,
                        std::vector<unsigned long long>* hist_out) {
    int nt = 0;
    const OptEntry* tab = opt_kernel_table(&nt);
    const uint64_t nids = id_off[nq];
    std::vector<int> width(nq);
    std::vector<uint32_t> per_width(nt, 0);
    uint64_t nbins = 0;
    for (uint32_t q = 0; q < nq; ++q) {
        const uint32_t n = id_off[q + 1] - id_off[q];
        const uint32_t need = exact ? n : std::min(n, kNarrowCounts);
        int w = 0;
        while (w < nt && (uint64_t(1) << tab[w].S) <= need) ++w;
        if (w == nt) return report_error(THR_E_INVAL, "opt-threshold query with too many ids");
        width[q] = w;
        ++per_width[w];
        nbins += uint64_t(n) + 1;
    }
    // one device buffer: queries, K, bin offsets, bounds, list, ids | bins
    const size_t o_K = align16(sizeof(QDesc) * nq);
    const size_t o_hoff = o_K + align16(8ull * nq);
    const size_t o_lb = o_hoff + align16(8ull * nq);
    const size_t o_list = o_lb + align16(4ull * nq);
    const size_t o_ids = o_list + align16(4ull * nq);
    const size_t o_ovf = o_ids + align16(4ull * nids);
    const size_t o_hist = o_ovf + align16(4ull * nq);
    const size_t total = o_hist + 8ull * nbins;
    std::vector<unsigned char> h(o_hist, 0);
    QDesc* qd = reinterpret_cast<QDesc*>(h.data());
    uint64_t* hk = reinterpret_cast<uint64_t*>(h.data() + o_K);
    uint64_t* hoff = reinterpret_cast<uint64_t*>(h.data() + o_hoff);
    uint32_t* lb = reinterpret_cast<uint32_t*>(h.data() + o_lb);
    uint32_t* list = reinterpret_cast<uint32_t*>(h.data() + o_list);
    std::vector<uint32_t> start(nt + 1, 0);
    for (int w = 0; w < nt; ++w) start[w + 1] = start[w] + per_width[w];
    std::vector<uint32_t> fill(start.begin(), start.end() - 1);
    uint64_t bin = 0;
    for (uint32_t q = 0; q < nq; ++q) {
        const uint32_t n = id_off[q + 1] - id_off[q];
        qd[q] = QDesc{id_off[q], n, 1u, 0u, 1u, 1u, 0u, kSymProfile};
        hk[q] = K[q];
        hoff[q] = bin;
        lb[q] = 1;
        list[fill[width[q]]++] = q;
        bin += uint64_t(n) + 1;
    }
    if (nids) std::memcpy(h.data() + o_ids, ids, 4ull * nids);
    unsigned char* d = nullptr;
    OPT_CK(cudaMallocAsync(reinterpret_cast<void**>(&d), total, st), "opt scratch");
    struct Free {
        unsigned char* p;
        cudaStream_t s;
        ~Free() { cudaFreeAsync(p, s); }
    } guard{d, st};
    OPT_CK(cudaMemcpyAsync(d, h.data(), o_hist, cudaMemcpyHostToDevice, st), "opt upload");
    OPT_CK(cudaMemsetAsync(d + o_hist, 0, 8ull * nbins, st), "opt bins");
    struct Events {
        cudaEvent_t e[2] = {nullptr, nullptr};
        ~Events() {
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } evs;
    cudaEvent_t* ev = evs.e;
    if (ms) {
        OPT_CK(cudaEventCreate(&ev[0]), "event");
        OPT_CK(cudaEventCreate(&ev[1]), "event");
        OPT_CK(cudaEventRecord(ev[0], st), "event");
    }
    OptParams o{};
    PassAParams& p = o.a;
    p.words = idx->d_words;
    p.sdesc = idx->d_sdesc;
    p.pcls = idx->d_pcls;
    p.masks = idx->d_masks;
    p.sseg = idx->d_sseg;
    p.desc = idx->d_desc;
    p.qd = reinterpret_cast<const QDesc*>(d);
    p.ids = reinterpret_cast<const uint32_t*>(d + o_ids);
    p.W = idx->W;
    p.NG = idx->NG;
    p.NGW = (idx->NG + 31) / 32;
    p.ragged = uint32_t(idx->r % 64);
    o.hist = reinterpret_cast<unsigned long long*>(d + o_hist);
    o.hoff = reinterpret_cast<const unsigned long long*>(d + o_hoff);
    o.lb = reinterpret_cast<uint32_t*>(d + o_lb);
    o.K = reinterpret_cast<const unsigned long long*>(d + o_K);
    o.exact = exact ? 1u : 0u;
    o.ovf = reinterpret_cast<uint32_t*>(d + o_ovf);
    constexpr uint32_t kSeedStride = 16;
    for (int w = 0; w < nt; ++w) {
        if (!per_width[w] || idx->NG == 0) continue;
        p.list = reinterpret_cast<const uint32_t*>(d + o_list) + start[w];
        p.nlist = per_width[w];
        // seeding over every kSeedStride-th subtile (bounds only), then
        // every subtile with the bins recorded
        for (int pass = idx->NG >= 4 * kSeedStride ? 0 : 1; pass < 2; ++pass) {
            o.stride = pass == 0 ? kSeedStride : 1;
            o.record = uint32_t(pass);
            const uint64_t items =
                uint64_t(p.nlist) * ((idx->NG + o.stride - 1) / o.stride);
            const uint64_t ctas = (items + kNW - 1) / kNW;
            const int grid = int(std::max<uint64_t>(
                1, std::min<uint64_t>(ctas, uint64_t(std::max(idx->num_sms, 1)) *
                                                occupancy(tab[w], w, idx->device))));
            OPT_CK(tab[w].launch(o, grid, st), "opt profiling kernel");
        }
    }
    std::vector<unsigned long long> hist(nbins);
    if (ms) OPT_CK(cudaEventRecord(ev[1], st), "event");
    OPT_CK(cudaMemcpyAsync(hist.data(), d + o_hist, 8ull * nbins, cudaMemcpyDeviceToHost, st),
           "opt bins");
    if (ovf_out) {
        ovf_out->assign(nq, 0);
        OPT_CK(cudaMemcpyAsync(ovf_out->data(), d + o_ovf, 4ull * nq, cudaMemcpyDeviceToHost, st),
               "opt overflow flags");
    }
    OPT_CK(cudaStreamSynchronize(st), "opt profiling");
    if (ms) OPT_CK(cudaEventElapsedTime(ms, ev[0], ev[1]), "profiling time");
    if (hist_out) *hist_out = hist;
    // the first count from the top whose suffix holds K rows
    for (uint32_t q = 0; q < nq; ++q) {
        const uint32_t n = id_off[q + 1] - id_off[q];
        const unsigned long long* b = hist.data() + hoff[q];
        uint64_t atleast = 0;
        T[q] = 0;
        for (uint32_t c = n; c >= 1; --c) {
            atleast += b[c];
            if (atleast >= K[q]) {
                T[q] = c;
                break;
            }
        }
    }
    return THR_OK;
}

thr_status opt_profile(const thr_index* idx, uint32_t nq, const uint32_t* id_off,
                       const uint32_t* ids, const uint64_t* K, uint32_t* T, cudaStream_t st,
                       float* ms, std::vector<unsigned long long>* hist) {
    std::vector<uint32_t> ovf;
    float ms1 = 0.f;
    thr_status s =
        profile_pass(idx, nq, id_off, ids, K, T, st, ms ? &ms1 : nullptr, false, &ovf, hist);
    if (s != THR_OK) return s;
    std::vector<uint32_t> redo;
    for (uint32_t q = 0; q < nq; ++q)
        if (ovf[q]) redo.push_back(q);
    if (!redo.empty()) {  // counts beyond the narrow counters: again with 2^S > n
        std::vector<uint32_t> off2(redo.size() + 1, 0), ids2, T2(redo.size(), 0);
        std::vector<uint64_t> K2(redo.size());
        for (size_t i = 0; i < redo.size(); ++i) {
            const uint32_t q = redo[i];
            ids2.insert(ids2.end(), ids + id_off[q], ids + id_off[q + 1]);
            off2[i + 1] = uint32_t(ids2.size());
            K2[i] = K[q];
        }
        float ms2 = 0.f;
        std::vector<unsigned long long> hist2;
        s = profile_pass(idx, uint32_t(redo.size()), off2.data(), ids2.data(), K2.data(),
                         T2.data(), st, ms ? &ms2 : nullptr, true, nullptr,
                         hist ? &hist2 : nullptr);
        if (s != THR_OK) return s;
        for (size_t i = 0; i < redo.size(); ++i) T[redo[i]] = T2[i];
        if (hist) {  // the exact pass's bins replace those of the narrow one
            std::vector<uint64_t> at(nq + 1, 0);
            for (uint32_t q = 0; q < nq; ++q) at[q + 1] = at[q] + (id_off[q + 1] - id_off[q]) + 1;
            uint64_t a2 = 0;
            for (size_t i = 0; i < redo.size(); ++i) {
                const uint32_t q = redo[i];
                const uint64_t nb = at[q + 1] - at[q];
                std::copy(hist2.begin() + a2, hist2.begin() + a2 + nb, hist->begin() + at[q]);
                a2 += nb;
            }
        }
        ms1 += ms2;
    }
    if (ms) *ms = ms1;
    return THR_OK;
}

}  // namespace thr
