// C ABI of libthr (include/thr.h): index build, threshold queries, batches.
//
// Host responsibilities: argument checks, stream validation (the format's
// marker chain is sequential, so the validating walk that also records every
// marker position runs on the host, one thread per group of bitmaps),
// uploads, scratch allocation (stream-ordered), kernel choice and the final
// device->host read of the result length.  Every step of the query itself
// runs in the kernels of thr_device.cuh / thr_query_kernel.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/thr.h"
#include "rle_host.h"
#include "thr_device.cuh"
#include "thr_index.h"
#include "thr_batch.h"
#include "thr_launch.h"
#include "thr_opt_host.h"

using namespace thr;

namespace {

thread_local std::string g_err;
thread_local double g_kernel_ms = -1.0;
thread_local BatchStats g_last_stats;

// THR_TRACE=1 in the environment: one stderr line per step of a query.
bool trace_on() {
    static const bool on = [] {
        const char* v = std::getenv("THR_TRACE");
        return v && v[0] == '1';
    }();
    return on;
}
#define TRACE(...)                                      \
    do {                                                \
        if (trace_on()) {                               \
            std::fprintf(stderr, "[thr] " __VA_ARGS__); \
            std::fputc('\n', stderr);                  \
            std::fflush(stderr);                        \
        }                                               \
    } while (0)

thr_status fail(thr_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

thr_status cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation)
        return fail(THR_E_NOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(THR_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// RAII for stream-ordered scratch.
struct Scratch {
    cudaStream_t st;
    std::vector<void*> ptrs;
    explicit Scratch(cudaStream_t s) : st(s) {}
    cudaError_t alloc(void** p, size_t bytes) {
        cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 16, st);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    ~Scratch() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
    }
};

// One query, output to a device buffer `dout` of `cap` words.  Returns the
// encoded length in *len (also when it exceeds cap).
thr_status run_query(const thr_index* idx, const uint32_t* ids, uint32_t n,
                     uint32_t T, uint64_t* dout, uint64_t cap, uint64_t* len,
                     cudaStream_t st, bool profile, uint32_t variant) {
    const uint32_t id_off[2] = {0, n};
    const uint8_t var = uint8_t(variant_of_flag(variant));
    BatchInput in{1, id_off, ids, &T, &var};
    BatchOptions opt;
    opt.profile = profile;
    // a query of the same shape as an earlier one on this thread replays
    // that query's CUDA graph (one launch instead of seven stream operations)
    opt.graph = true;
    BatchStats stats;
    uint64_t off = 0, total = 0;
    TRACE("query n=%u T=%u NG=%u", n, T, idx->NG);
    thr_status s = run_batch(idx, in, dout, cap, &off, len, &total, st, opt, &stats);
    if (s != THR_OK) return s;
    if (profile) g_kernel_ms = stats.pass_a_ms;
    return THR_OK;
}

// Is p memory the kernels of device dev may write: device memory of dev
// itself, or managed memory?  Device memory of another GPU is refused: the
// kernels would write it through a peer address, which faults without peer
// access.
bool is_device_ptr(const void* p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

namespace thr {
thr_status report_error(thr_status st, const char* msg) { return fail(st, "%s", msg); }

const KernelEntry* kernel_table(int* count) {
    static const KernelEntry tab[] = {
        {1, launch_threshold_1, occupancy_threshold_1, launch_staged_1,
         occupancy_staged_1, launch_threshold_pos_1,
         occupancy_threshold_pos_1, launch_split_1, occupancy_split_1},
        {2, launch_threshold_2, occupancy_threshold_2, launch_staged_2,
         occupancy_staged_2, launch_threshold_pos_2,
         occupancy_threshold_pos_2, launch_split_2, occupancy_split_2},
        {3, launch_threshold_3, occupancy_threshold_3, launch_staged_3,
         occupancy_staged_3, launch_threshold_pos_3,
         occupancy_threshold_pos_3, launch_split_3, occupancy_split_3},
        {4, launch_threshold_4, occupancy_threshold_4, launch_staged_4,
         occupancy_staged_4, launch_threshold_pos_4,
         occupancy_threshold_pos_4, launch_split_4, occupancy_split_4},
        {5, launch_threshold_5, occupancy_threshold_5, launch_staged_5,
         occupancy_staged_5, launch_threshold_pos_5,
         occupancy_threshold_pos_5, launch_split_5, occupancy_split_5},
        {6, launch_threshold_6, occupancy_threshold_6, launch_staged_6,
         occupancy_staged_6, launch_threshold_pos_6,
         occupancy_threshold_pos_6, launch_split_6, occupancy_split_6},
        {7, launch_threshold_7, occupancy_threshold_7, launch_staged_7,
         occupancy_staged_7, launch_threshold_pos_7,
         occupancy_threshold_pos_7, launch_split_7, occupancy_split_7},
        {8, launch_threshold_8, occupancy_threshold_8, launch_staged_8,
         occupancy_staged_8, launch_threshold_pos_8,
         occupancy_threshold_pos_8, launch_split_8, occupancy_split_8},
        {10, launch_threshold_10, occupancy_threshold_10, launch_staged_10,
         occupancy_staged_10, launch_threshold_pos_10,
         occupancy_threshold_pos_10, nullptr, nullptr},
        {12, launch_threshold_12, occupancy_threshold_12, launch_staged_12,
         occupancy_staged_12, launch_threshold_pos_12,
         occupancy_threshold_pos_12, nullptr, nullptr},
        {16, launch_threshold_16, occupancy_threshold_16, launch_staged_16,
         occupancy_staged_16, launch_threshold_pos_16,
         occupancy_threshold_pos_16, nullptr, nullptr},
        {20, launch_threshold_20, occupancy_threshold_20, launch_staged_20,
         occupancy_staged_20, launch_threshold_pos_20,
         occupancy_threshold_pos_20, nullptr, nullptr},
    };
    *count = int(sizeof tab / sizeof tab[0]);
    return tab;
}
}  // namespace thr

// Argument checks shared by thr_query_batch and thr_autotune; fills the
// kernel class of every query for the policy in flags.
static thr_status check_batch(const thr_index* idx, uint32_t nq, const uint32_t* id_off,
                       const uint32_t* ids, const uint32_t* T, uint32_t flags,
                       std::vector<uint8_t>* cls) {
    if (!idx || !id_off || !T) return fail(THR_E_INVAL, "null argument");
    if (!ids && id_off[nq] > id_off[0]) return fail(THR_E_INVAL, "null ids");
    if (id_off[0] != 0) return fail(THR_E_INVAL, "id_off[0] must be 0");
    const uint32_t policy = flags & THR_POLICY_MASK;
    if (policy != THR_POLICY_PLAIN && policy != THR_POLICY_RULE && policy != THR_POLICY_LEARNED)
        return fail(THR_E_INVAL, "unknown policy");
    const uint32_t variant = flags & THR_VARIANT_MASK;
    if (variant_of_flag(variant) < 0) return fail(THR_E_INVAL, "unknown variant");
    for (uint32_t q = 0; q < nq; ++q) {
        if (id_off[q + 1] < id_off[q]) return fail(THR_E_INVAL, "id_off decreases at %u", q);
        const uint32_t n = id_off[q + 1] - id_off[q];
        if (n == 0 || n > THR_MAX_IDS)
            return fail(THR_E_INVAL, "query %u: n must be in 1..%u", q, THR_MAX_IDS);
    }
    for (uint64_t i = 0; i < id_off[nq]; ++i)
        if (ids[i] >= idx->nbitmaps)
            return fail(THR_E_INVAL, "id %u out of range (%u bitmaps)", ids[i], idx->nbitmaps);
    return choose_variants(idx, nq, id_off, ids, T, policy, variant, cls,
                           !(flags & THR_NO_SHARE));
}

extern "C" {

const char* thr_last_error(void) { return g_err.c_str(); }

double thr_last_kernel_ms(void) { return g_kernel_ms; }

thr_status thr_last_batch_info(uint32_t* chunks, uint32_t* launches, int32_t* graph,
                               uint32_t* config) {
    if (chunks) *chunks = g_last_stats.chunks;
    if (launches) *launches = g_last_stats.launches;
    if (graph) *graph = g_last_stats.graph_reused;
    if (config) *config = g_last_stats.tune;
    return THR_OK;
}

thr_status thr_rle_encode(const uint64_t* words, uint64_t nwords, uint64_t r,
                          uint64_t* out, uint64_t cap, uint64_t* out_len) {
    if (!out_len || (cap > 0 && !out)) return fail(THR_E_INVAL, "null output");
    const int rc = encode_words(words, nwords, r, out, cap, out_len);
    if (rc == 1) return fail(THR_E_INVAL, "need ceil(r/64) words with bits >= r clear");
    if (rc == 4) return fail(THR_E_NOSPACE, "encoded stream needs %llu words",
                             (unsigned long long)*out_len);
    return THR_OK;
}

thr_status thr_rle_encode_rows(const uint64_t* rows, uint64_t nrows, uint64_t r, uint64_t* out,
                               uint64_t cap, uint64_t* out_len) {
    if (!out_len || (cap > 0 && !out) || (nrows > 0 && !rows))
        return fail(THR_E_INVAL, "null argument");
    const int rc = encode_rows(rows, nrows, r, out, cap, out_len);
    if (rc == 1) return fail(THR_E_INVAL, "rows must be ascending and below r (r >= 1)");
    if (rc == 4) return fail(THR_E_NOSPACE, "encoded stream needs %llu words",
                             (unsigned long long)*out_len);
    return THR_OK;
}

thr_status thr_rle_slice(const uint64_t* stream, uint64_t len, uint64_t r, uint64_t w0,
                         uint64_t w1, uint64_t* out, uint64_t cap, uint64_t* out_len) {
    if (!stream || !out_len || (cap > 0 && !out)) return fail(THR_E_INVAL, "null argument");
    if ((r + 63) / 64 > kMaxWords) return fail(THR_E_INVAL, "r too large");
    StreamScan sc;
    std::string why;
    if (scan_stream(stream, len, r, &sc, &why) != 0)
        return fail(THR_E_FORMAT, "%s", why.c_str());
    const int rc = slice_stream(stream, len, r, w0, w1, out, cap, out_len);
    if (rc == 1) return fail(THR_E_INVAL, "need w0 < w1 <= ceil(r/64)");
    if (rc == 4) return fail(THR_E_NOSPACE, "slice needs %llu words", (unsigned long long)*out_len);
    return THR_OK;
}

thr_status thr_rle_stitch(const uint64_t* const* parts, const uint64_t* lens,
                          const uint64_t* rows, uint32_t nparts, uint64_t* out, uint64_t cap,
                          uint64_t* out_len) {
    if (!parts || !lens || !rows || !out_len || (cap > 0 && !out))
        return fail(THR_E_INVAL, "null argument");
    if (nparts == 0) return fail(THR_E_INVAL, "no parts");
    std::vector<uint64_t> words(nparts);
    for (uint32_t k = 0; k < nparts; ++k) {
        if (rows[k] == 0 || (k + 1 < nparts && rows[k] % 64 != 0))
            return fail(THR_E_INVAL, "part %u: rows must be positive, a multiple of 64 but the last", k);
        StreamScan sc;
        std::string why;
        if (scan_stream(parts[k], lens[k], rows[k], &sc, &why) != 0)
            return fail(THR_E_FORMAT, "part %u: %s", k, why.c_str());
        words[k] = (rows[k] + 63) / 64;
    }
    const int rc = stitch_streams(parts, lens, words.data(), nparts, out, cap, out_len);
    if (rc == 1) return fail(THR_E_INVAL, "bad parts");
    if (rc == 4) return fail(THR_E_NOSPACE, "stitched stream needs %llu words",
                             (unsigned long long)*out_len);
    return THR_OK;
}

thr_status thr_rle_validate(const uint64_t* stream, uint64_t len, uint64_t r) {
    if (!stream && len) return fail(THR_E_INVAL, "null stream");
    if ((r + 63) / 64 > kMaxWords) return fail(THR_E_INVAL, "r too large");
    StreamScan sc;
    std::string why;
    if (scan_stream(stream, len, r, &sc, &why) != 0)
        return fail(THR_E_FORMAT, "%s", why.c_str());
    return THR_OK;
}

thr_status idx_build_rle(const uint64_t* words, const uint64_t* offsets,
                         uint32_t nbitmaps, uint64_t r, void* cuda_stream,
                         thr_index** out) {
    if (!out || !offsets || nbitmaps == 0) return fail(THR_E_INVAL, "null argument or no bitmaps");
    if (r == 0) return fail(THR_E_INVAL, "r must be at least 1");
    const uint64_t W = (r + 63) / 64;
    if (W > kMaxWords) return fail(THR_E_INVAL, "r too large (ceil(r/64) > 2^31 - 2)");
    const uint64_t total = offsets[nbitmaps];
    if (offsets[0] != 0) return fail(THR_E_INVAL, "offsets[0] must be 0");
    for (uint32_t b = 0; b < nbitmaps; ++b)
        if (offsets[b + 1] < offsets[b]) return fail(THR_E_INVAL, "offsets decrease at %u", b);
    if (total && !words) return fail(THR_E_INVAL, "null words");
    if (total >= (1ull << 40)) return fail(THR_E_INVAL, "index larger than 2^40 words");
    cudaStream_t st = (cudaStream_t)cuda_stream;

    // validate every stream and record its marker positions (host threads)
    std::vector<StreamScan> scans(nbitmaps);
    std::vector<std::string> whys(nbitmaps);
    std::vector<int> rcs(nbitmaps, 0);
    {
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        const unsigned nt = std::min<unsigned>(hw, std::max<uint32_t>(1, nbitmaps));
        std::atomic<uint32_t> next{0};
        auto worker = [&]() {
            for (;;) {
                const uint32_t b = next.fetch_add(1);
                if (b >= nbitmaps) return;
                rcs[b] = scan_stream(words + offsets[b], offsets[b + 1] - offsets[b], r,
                                     &scans[b], &whys[b]);
            }
        };
        std::vector<std::thread> pool;
        for (unsigned i = 1; i < nt; ++i) pool.emplace_back(worker);
        worker();
        for (auto& th : pool) th.join();
    }
    for (uint32_t b = 0; b < nbitmaps; ++b)
        if (rcs[b]) return fail(THR_E_FORMAT, "bitmap %u: %s", b, whys[b].c_str());

    int device = 0, num_sms = 0;
    CK(cudaGetDevice(&device), "cudaGetDevice");
    CK(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device),
       "device attributes");
    {  // keep query scratch in the device's stream-ordered pool between queries
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
            uint64_t keep = ~0ull;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    thr_index* idx = new (std::nothrow) thr_index;
    if (!idx) return fail(THR_E_NOMEM, "host allocation");
    idx->device = device;
    idx->num_sms = num_sms;
    idx->nbitmaps = nbitmaps;
    idx->r = r;
    idx->W = uint32_t(W);
    idx->NG = uint32_t((W + kGW - 1) / kGW);
    idx->total_words = total;
    idx->desc.resize(nbitmaps);
    idx->set_rows.resize(nbitmaps);
    idx->feat_lw.resize(nbitmaps);
    idx->feat_ld.resize(nbitmaps);
    uint64_t moff = 0;
    for (uint32_t b = 0; b < nbitmaps; ++b) {
        BitmapDesc& d = idx->desc[b];
        d.woff = offsets[b];
        d.moff = moff;
        d.nmark = uint32_t(scans[b].marker_pos.size());
        d.len = uint32_t(offsets[b + 1] - offsets[b]);
        moff += d.nmark + 1;
        idx->set_rows[b] = scans[b].set_rows;
        idx->feat_lw[b] = std::log2(double(d.len) + 1.0);
        idx->feat_ld[b] = std::log10(double(scans[b].set_rows) / double(r) + 1e-7);
    }
    idx->total_markers = moff - nbitmaps;
    std::vector<uint32_t> mpos;
    mpos.reserve(idx->total_markers);
    for (uint32_t b = 0; b < nbitmaps; ++b)
        mpos.insert(mpos.end(), scans[b].marker_pos.begin(), scans[b].marker_pos.end());
    scans.clear();

    auto cleanup = [&](thr_status s) {
        idx_free(idx);
        return s;
    };
    uint32_t* d_mpos = nullptr;
    uint32_t* d_ttab = nullptr;  // build temporary
    const uint64_t ttab_n = uint64_t(idx->NG + 1) * nbitmaps;
    const uint64_t sdesc_n = uint64_t(idx->NG) * nbitmaps;
    cudaError_t e;
    auto free_tmp = [&]() {
        if (d_mpos) cudaFree(d_mpos);
        if (d_ttab) cudaFree(d_ttab);
    };
    // two zero words after the streams: the staged kernel copies whole 16-byte
    // units, which may run one word past a stream's last word
    if ((e = cudaMalloc(&idx->d_words, sizeof(uint64_t) * (total + 2))) != cudaSuccess ||
        (e = cudaMalloc(&idx->d_mtab, sizeof(uint2) * moff)) != cudaSuccess ||
        (e = cudaMalloc(&idx->d_sdesc, sizeof(uint64_t) * sdesc_n)) != cudaSuccess ||
        (e = cudaMalloc(&idx->d_sseg, sizeof(uint64_t) * sdesc_n)) != cudaSuccess ||
        (e = cudaMalloc(&idx->d_desc, sizeof(BitmapDesc) * nbitmaps)) != cudaSuccess ||
        (e = cudaMalloc(&d_ttab, sizeof(uint32_t) * ttab_n)) != cudaSuccess ||
        (e = cudaMalloc(&d_mpos, sizeof(uint32_t) * std::max<uint64_t>(mpos.size(), 1))) != cudaSuccess) {
        free_tmp();
        return cleanup(cuda_fail(e, "index allocation"));
    }
    if ((e = cudaMemsetAsync(idx->d_words + total, 0, 2 * sizeof(uint64_t), st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(idx->d_words, words, sizeof(uint64_t) * total,
                             cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_mpos, mpos.data(), sizeof(uint32_t) * mpos.size(),
                             cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(idx->d_desc, idx->desc.data(), sizeof(BitmapDesc) * nbitmaps,
                             cudaMemcpyHostToDevice, st)) != cudaSuccess) {
        free_tmp();
        return cleanup(cuda_fail(e, "index upload"));
    }
    uint32_t* d_mcount = nullptr;
    uint64_t* d_mbase = nullptr;
    auto free_all_tmp = [&]() {
        free_tmp();
        if (d_mcount) cudaFree(d_mcount);
        if (d_mbase) cudaFree(d_mbase);
    };
    if ((e = cudaMalloc(&d_mcount, sizeof(uint32_t) * nbitmaps)) != cudaSuccess ||
        (e = cudaMalloc(&d_mbase, sizeof(uint64_t) * nbitmaps)) != cudaSuccess) {
        free_all_tmp();
        return cleanup(cuda_fail(e, "index allocation"));
    }
    e = launch_index_build_a(idx->d_words, d_mpos, idx->d_desc, idx->d_mtab, d_ttab,
                             idx->d_sdesc, idx->d_sseg, d_mcount, nbitmaps, idx->W, idx->NG,
                             st);
    std::vector<uint32_t> mcount(nbitmaps);
    std::vector<uint64_t> mbase(nbitmaps);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(mcount.data(), d_mcount, sizeof(uint32_t) * nbitmaps,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
        uint64_t acc = 0;
        for (uint32_t b = 0; b < nbitmaps; ++b) {
            mbase[b] = acc;
            acc += mcount[b];
        }
        idx->mixed_subtiles = acc;
        e = cudaMalloc(&idx->d_masks, sizeof(MaskRec) * std::max<uint64_t>(acc, 1));
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_mbase, mbase.data(), sizeof(uint64_t) * nbitmaps,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_index_build_b(idx->d_mtab, d_ttab, idx->d_desc, d_mbase, idx->d_sdesc,
                                 idx->d_sseg, idx->d_masks, nbitmaps, idx->W, idx->NG, st);
    if (e == cudaSuccess)
        e = cudaMalloc(&idx->d_pcls, sizeof(uint64_t) * uint64_t(nbitmaps) * ((idx->NG + 31) / 32));
    if (e == cudaSuccess) e = launch_pack_classes(idx->d_sdesc, idx->d_pcls, nbitmaps, idx->NG, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    free_all_tmp();
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "index build kernels"));
    *out = idx;
    return THR_OK;
}

void idx_free(thr_index* idx) {
    if (!idx) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(idx->device);
    cudaDeviceSynchronize();
    cudaFree(idx->d_words);
    cudaFree(idx->d_mtab);
    cudaFree(idx->d_sdesc);
    cudaFree(idx->d_pcls);
    cudaFree(idx->d_masks);
    cudaFree(idx->d_sseg);
    cudaFree(idx->d_desc);
    cudaSetDevice(cur);
    delete idx;
}

thr_status idx_info(const thr_index* idx, uint32_t* nbitmaps, uint64_t* r,
                    uint64_t* total_words) {
    if (!idx) return fail(THR_E_INVAL, "null index");
    if (nbitmaps) *nbitmaps = idx->nbitmaps;
    if (r) *r = idx->r;
    if (total_words) *total_words = idx->total_words;
    return THR_OK;
}

thr_status thr_query(const thr_index* idx, const uint32_t* ids, uint32_t n,
                     uint32_t T, uint64_t* out, uint64_t cap, uint64_t* out_len,
                     uint32_t flags, void* cuda_stream) {
    if (!idx || !ids || !out_len || (cap > 0 && !out))
        return fail(THR_E_INVAL, "null argument");
    if (n == 0 || n > THR_MAX_IDS) return fail(THR_E_INVAL, "n must be in 1..%u", THR_MAX_IDS);
    if (flags & ~(THR_OUT_DEVICE | THR_POLICY_MASK | THR_PROFILE | THR_VARIANT_MASK))
        return fail(THR_E_INVAL, "unknown flags");
    const bool profile = flags & THR_PROFILE;
    const uint32_t variant = flags & THR_VARIANT_MASK;
    if (variant_of_flag(variant) < 0) return fail(THR_E_INVAL, "unknown variant");
    for (uint32_t i = 0; i < n; ++i)
        if (ids[i] >= idx->nbitmaps)
            return fail(THR_E_INVAL, "id %u out of range (%u bitmaps)", ids[i], idx->nbitmaps);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const bool dev_out = flags & THR_OUT_DEVICE;
    if (dev_out && cap > 0 && !is_device_ptr(out, idx->device))
        return fail(THR_E_INVAL, "THR_OUT_DEVICE given but out is not device memory of the index's GPU");
    if (dev_out) {
        thr_status s = run_query(idx, ids, n, T, out, cap, out_len, st, profile, variant);
        if (s == THR_OK && *out_len > cap)
            return fail(THR_E_NOSPACE, "result needs %llu words", (unsigned long long)*out_len);
        return s;
    }
    // host output: compute into device scratch, then copy back
    const uint64_t need = uint64_t(idx->W) + 1;
    const uint64_t dcap = std::min<uint64_t>(cap, need);
    uint64_t* dbuf = nullptr;
    {
        Scratch scr(st);
        CK(scr.alloc((void**)&dbuf, sizeof(uint64_t) * std::max<uint64_t>(dcap, 1)),
           "scratch (output)");
        uint64_t len = 0;
        thr_status s = run_query(idx, ids, n, T, dbuf, dcap, &len, st, profile, variant);
        if (s != THR_OK) return s;
        *out_len = len;
        if (len > cap)
            return fail(THR_E_NOSPACE, "result needs %llu words", (unsigned long long)len);
        CK(cudaMemcpyAsync(out, dbuf, sizeof(uint64_t) * len, cudaMemcpyDeviceToHost, st),
           "copy result");
        CK(cudaStreamSynchronize(st), "copy result");
    }
    return THR_OK;
}

thr_status thr_select_variants(const thr_index* idx, uint32_t nq, const uint32_t* id_off,
                               const uint32_t* ids, const uint32_t* T, uint32_t flags,
                               uint8_t* variant) {
    if (!variant && nq) return fail(THR_E_INVAL, "null output");
    if (nq == 0) return THR_OK;
    if (flags & ~(THR_POLICY_MASK | THR_VARIANT_MASK)) return fail(THR_E_INVAL, "unknown flags");
    std::vector<uint8_t> var;
    thr_status ps = check_batch(idx, nq, id_off, ids, T, flags, &var);
    if (ps != THR_OK) return ps;
    for (uint32_t q = 0; q < nq; ++q) {
        const uint32_t n = id_off[q + 1] - id_off[q];
        int cls = 0;
        uint32_t z = 0;
        resolve_variant(n, T[q], var[q], &cls, &z);
        // the variant that actually runs (fallbacks of ScanCount and split)
        const int fam = class_family(cls);
        variant[q] = uint8_t(fam == 0   ? kVarCsa
                             : fam == 1 ? kVarScanCount
                             : fam == 2 ? kVarPos
                             : fam == 3 ? kVarSplit
                             : fam == 4 ? kVarLooped
                                        : kVarStaged);
    }
    return THR_OK;
}

thr_status thr_rule_model(const double* set, double* get) {
    if (set) set_rule_model(set);
    if (get) get_rule_model(get);
    return THR_OK;
}

thr_status thr_autotune(const thr_index* idx, uint32_t nq, const uint32_t* id_off,
                        const uint32_t* ids, const uint32_t* T, uint32_t flags, uint32_t reps,
                        void* cuda_stream, double* times, uint32_t* best) {
    if (nq == 0) return fail(THR_E_INVAL, "empty sample batch");
    if (reps == 0) return fail(THR_E_INVAL, "reps must be at least 1");
    if (flags & ~(THR_POLICY_MASK | THR_VARIANT_MASK | THR_NO_SHARE))
        return fail(THR_E_INVAL, "unknown flags");
    std::vector<uint8_t> cls;
    thr_status ps = check_batch(idx, nq, id_off, ids, T, flags & ~THR_NO_SHARE, &cls);
    if (ps != THR_OK) return ps;
    BatchInput in{nq, id_off, ids, T, cls.data()};
    return autotune(idx, in, (cudaStream_t)cuda_stream, reps, times, best,
                    !(flags & THR_NO_SHARE));
}

thr_status thr_query_sym(const thr_index* idx, const uint32_t* ids, uint32_t n, uint32_t lo,
                         uint32_t hi, uint64_t* out, uint64_t cap, uint64_t* out_len,
                         uint32_t flags, void* cuda_stream) {
    if (!idx || !ids || !out_len || (cap > 0 && !out)) return fail(THR_E_INVAL, "null argument");
    if (n == 0 || n > THR_MAX_IDS) return fail(THR_E_INVAL, "n must be in 1..%u", THR_MAX_IDS);
    if (flags & ~(THR_OUT_DEVICE | THR_SYM_ODD | THR_PROFILE))
        return fail(THR_E_INVAL, "unknown flags");
    for (uint32_t i = 0; i < n; ++i)
        if (ids[i] >= idx->nbitmaps)
            return fail(THR_E_INVAL, "id %u out of range (%u bitmaps)", ids[i], idx->nbitmaps);
    const uint8_t sym = (flags & THR_SYM_ODD) ? uint8_t(kSymOdd) : uint8_t(kSymRange);
    const uint32_t id_off[2] = {0, n};
    const uint8_t var = uint8_t(kVarCsa);
    BatchInput in{1, id_off, ids, &lo, &var, &sym, &hi};
    BatchOptions opt;
    opt.profile = flags & THR_PROFILE;
    BatchStats stats;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    uint64_t off = 0, total = 0;
    if (flags & THR_OUT_DEVICE) {
        if (cap > 0 && !is_device_ptr(out, idx->device))
            return fail(THR_E_INVAL, "THR_OUT_DEVICE given but out is not device memory of the index's GPU");
        thr_status s = run_batch(idx, in, out, cap, &off, out_len, &total, st, opt, &stats);
        if (s != THR_OK) return s;
        if (opt.profile) g_kernel_ms = stats.pass_a_ms;
        if (*out_len > cap)
            return fail(THR_E_NOSPACE, "result needs %llu words", (unsigned long long)*out_len);
        return THR_OK;
    }
    const uint64_t dcap = std::min<uint64_t>(cap, uint64_t(idx->W) + 1);
    Scratch scr(st);
    uint64_t* dbuf = nullptr;
    CK(scr.alloc((void**)&dbuf, sizeof(uint64_t) * std::max<uint64_t>(dcap, 1)),
       "scratch (output)");
    thr_status s = run_batch(idx, in, dbuf, dcap, &off, out_len, &total, st, opt, nullptr);
    if (s != THR_OK) return s;
    if (*out_len > cap)
        return fail(THR_E_NOSPACE, "result needs %llu words", (unsigned long long)*out_len);
    CK(cudaMemcpyAsync(out, dbuf, sizeof(uint64_t) * *out_len, cudaMemcpyDeviceToHost, st),
       "copy result");
    CK(cudaStreamSynchronize(st), "copy result");
    return THR_OK;
}

thr_status thr_query_opt_batch(const thr_index* idx, uint32_t nq, const uint32_t* id_off,
                               const uint32_t* ids, const uint64_t* K, uint32_t* T_out,
                               uint64_t* pool, uint64_t pool_cap, uint64_t* out_off,
                               uint64_t* out_len, uint32_t flags, void* cuda_stream) {
    if (!idx || !id_off || !K || !T_out || !out_off || !out_len || (pool_cap > 0 && !pool))
        return fail(THR_E_INVAL, "null argument");
    if (nq == 0) return THR_OK;
    if (flags & ~(THR_OUT_DEVICE | THR_POLICY_MASK | THR_PROFILE | THR_VARIANT_MASK |
                  THR_NO_GRAPH | THR_NO_SHARE))
        return fail(THR_E_INVAL, "unknown flags");
    if (id_off[0] != 0) return fail(THR_E_INVAL, "id_off[0] must be 0");
    for (uint32_t q = 0; q < nq; ++q) {
        if (id_off[q + 1] < id_off[q]) return fail(THR_E_INVAL, "id_off decreases at %u", q);
        const uint32_t n = id_off[q + 1] - id_off[q];
        if (n == 0 || n > 65535)
            return fail(THR_E_INVAL, "query %u: n must be in 1..65535", q);
        if (K[q] == 0) return fail(THR_E_INVAL, "query %u: K must be >= 1", q);
    }
    if (!ids) return fail(THR_E_INVAL, "null ids");
    for (uint64_t i = 0; i < id_off[nq]; ++i)
        if (ids[i] >= idx->nbitmaps)
            return fail(THR_E_INVAL, "id %u out of range (%u bitmaps)", ids[i], idx->nbitmaps);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    float ms = 0.f;
    thr_status s = opt_profile(idx, nq, id_off, ids, K, T_out, st,
                               (flags & THR_PROFILE) ? &ms : nullptr);
    if (s != THR_OK) return s;
    s = thr_query_batch(idx, nq, id_off, ids, T_out, pool, pool_cap, out_off, out_len,
                        flags & ~THR_PROFILE, cuda_stream);
    if (flags & THR_PROFILE) g_kernel_ms = ms;
    return s;
}

thr_status thr_query_opt(const thr_index* idx, const uint32_t* ids, uint32_t n, uint64_t K,
                         uint32_t* T_out, uint64_t* out, uint64_t cap, uint64_t* out_len,
                         uint32_t flags, void* cuda_stream) {
    if (!idx || !ids || !T_out || !out_len || (cap > 0 && !out))
        return fail(THR_E_INVAL, "null argument");
    if (n == 0 || n > 65535) return fail(THR_E_INVAL, "n must be in 1..65535");
    if (K == 0) return fail(THR_E_INVAL, "K must be >= 1");
    if (flags & ~(THR_OUT_DEVICE | THR_PROFILE | THR_VARIANT_MASK))
        return fail(THR_E_INVAL, "unknown flags");
    if (variant_of_flag(flags & THR_VARIANT_MASK) < 0)
        return fail(THR_E_INVAL, "unknown variant");
    for (uint32_t i = 0; i < n; ++i)
        if (ids[i] >= idx->nbitmaps)
            return fail(THR_E_INVAL, "id %u out of range (%u bitmaps)", ids[i], idx->nbitmaps);
    if ((flags & THR_OUT_DEVICE) && cap > 0 && !is_device_ptr(out, idx->device))
        return fail(THR_E_INVAL, "THR_OUT_DEVICE given but out is not device memory of the index's GPU");
    const uint32_t id_off[2] = {0, n};
    float ms = 0.f;
    thr_status s = opt_profile(idx, 1, id_off, ids, &K, T_out, (cudaStream_t)cuda_stream,
                               (flags & THR_PROFILE) ? &ms : nullptr);
    if (s != THR_OK) return s;
    s = thr_query(idx, ids, n, *T_out, out, cap, out_len, flags & ~THR_PROFILE, cuda_stream);
    if (flags & THR_PROFILE) g_kernel_ms = ms;
    return s;
}

thr_status thr_query_opt_hist(const thr_index* idx, const uint32_t* ids, uint32_t n,
                              uint64_t K, uint32_t* T_out, uint64_t* hist,
                              void* cuda_stream) {
    if (!idx || !ids || !T_out || !hist) return fail(THR_E_INVAL, "null argument");
    if (n == 0 || n > 65535) return fail(THR_E_INVAL, "n must be in 1..65535");
    if (K == 0) return fail(THR_E_INVAL, "K must be >= 1");
    for (uint32_t i = 0; i < n; ++i)
        if (ids[i] >= idx->nbitmaps)
            return fail(THR_E_INVAL, "id %u out of range (%u bitmaps)", ids[i], idx->nbitmaps);
    const uint32_t id_off[2] = {0, n};
    std::vector<unsigned long long> h;
    thr_status s = opt_profile(idx, 1, id_off, ids, &K, T_out, (cudaStream_t)cuda_stream,
                               nullptr, &h);
    if (s != THR_OK) return s;
    for (uint32_t c = 0; c <= n; ++c) hist[c] = h[c];
    hist[0] = 0;  // not counted by the profiling pass
    return THR_OK;
}

thr_status thr_query_batch(const thr_index* idx, uint32_t nq, const uint32_t* id_off,
                           const uint32_t* ids, const uint32_t* T, uint64_t* pool,
                           uint64_t pool_cap, uint64_t* out_off, uint64_t* out_len,
                           uint32_t flags, void* cuda_stream) {
    if (!idx || !id_off || !T || !out_off || !out_len || (pool_cap > 0 && !pool))
        return fail(THR_E_INVAL, "null argument");
    if (nq == 0) return THR_OK;
    if (flags & ~(THR_OUT_DEVICE | THR_POLICY_MASK | THR_PROFILE | THR_VARIANT_MASK |
                  THR_NO_GRAPH | THR_NO_SHARE))
        return fail(THR_E_INVAL, "unknown flags");
    const double t_in = trace_time_on() ? now_us() : 0.0;
    std::vector<uint8_t> cls;
    thr_status ps = check_batch(idx, nq, id_off, ids, T, flags, &cls);
    if (ps != THR_OK) return ps;
    if (t_in > 0) std::fprintf(stderr, "[thr] batch checks and variants %.1f us\n", now_us() - t_in);
    BatchInput in{nq, id_off, ids, T, cls.data()};
    BatchOptions opt;
    opt.graph = !(flags & THR_NO_GRAPH);
    opt.profile = flags & THR_PROFILE;
    opt.share = !(flags & THR_NO_SHARE);
    BatchStats stats;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    uint64_t total = 0;
    if (flags & THR_OUT_DEVICE) {
        const double t_p = trace_time_on() ? now_us() : 0.0;
        if (pool_cap > 0 && !is_device_ptr(pool, idx->device))
            return fail(THR_E_INVAL, "THR_OUT_DEVICE given but pool is not device memory");
        if (t_p > 0) std::fprintf(stderr, "[thr] batch pool check %.1f us\n", now_us() - t_p);
        thr_status s = run_batch(idx, in, pool, pool_cap, out_off, out_len, &total, st, opt,
                                 &stats);
        if (s != THR_OK) return s;
    } else {
        // host pool: results go to a device staging pool first; if they do
        // not fit there but fit the caller's pool, run again with room
        uint64_t dcap = std::min<uint64_t>(pool_cap, uint64_t(nq) * (uint64_t(idx->W) + 1));
        dcap = std::min<uint64_t>(dcap, uint64_t(1) << 27);
        for (int attempt = 0; attempt < 2; ++attempt) {
            Scratch scr(st);
            uint64_t* dbuf = nullptr;
            CK(scr.alloc((void**)&dbuf, sizeof(uint64_t) * std::max<uint64_t>(dcap, 1)),
               "scratch (output pool)");
            thr_status s = run_batch(idx, in, dbuf, dcap, out_off, out_len, &total, st, opt,
                                     &stats);
            if (s != THR_OK) return s;
            if (total > dcap && total <= pool_cap) {
                dcap = total;
                continue;
            }
            if (total <= pool_cap && total > 0) {
                CK(cudaMemcpyAsync(pool, dbuf, sizeof(uint64_t) * total, cudaMemcpyDeviceToHost,
                                   st),
                   "copy results");
                CK(cudaStreamSynchronize(st), "copy results");
            }
            break;
        }
    }
    if (opt.profile) g_kernel_ms = stats.pass_a_ms;
    g_last_stats = stats;
    if (total > pool_cap)
        return fail(THR_E_NOSPACE, "pool needs %llu words", (unsigned long long)total);
    return THR_OK;
}

}  // extern "C"
