// thr_query_static: a threshold query that allocates nothing.
//
// Some callers cannot allocate device memory while they answer a query: a
// process whose GPU memory is owned by another allocator (for example a
// framework's caching allocator that reserves the device up front), or code
// that must not risk an allocation failure, or the device synchronisation an
// allocation or free can cause, in the middle of its work.  This entry point
// runs the same kernels as thr_query, but every piece of scratch memory it
// needs lives in one fixed file-scope device array, g_noalloc_scratch, that
// each GPU loading the library holds until the process exits.  It calls no
// cudaMalloc, cudaMallocAsync, cudaMallocHost or free routine.
//
// Limits: W = ceil(r/64) <= kStaticMaxWords (r <= 2^26 rows) and
// n <= kStaticMaxIds; larger queries are rejected with THR_E_INVAL.
//
// The array is shared by every call: a call overwrites what the previous one
// left there, and calls whose work overlaps on the GPU (other streams, other
// host threads) race on it; callers must not let two such calls run at once.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "thr_index.h"
#include "thr_launch.h"

namespace thr {
namespace {

constexpr uint64_t kStaticMaxWords = 1ull << 20;              // r <= 2^26 rows
constexpr uint64_t kStaticMaxSubtiles = kStaticMaxWords / kGW;
constexpr uint64_t kStaticMaxIds = 65536;
constexpr uint64_t kStaticBlocks = (kStaticMaxSubtiles + 255) / 256;

// fixed layout: control | ids | aggregates | prefixes | block totals |
// block prefixes | result words
constexpr uint64_t kOffIds = 256;
constexpr uint64_t kOffAggs = kOffIds + 4 * kStaticMaxIds;
constexpr uint64_t kOffPref = kOffAggs + 4 * kAggWords * kStaticMaxSubtiles;
constexpr uint64_t kOffBagg = kOffPref + 4 * kAggWords * kStaticMaxSubtiles;
constexpr uint64_t kOffBpref = kOffBagg + 4 * kAggWords * kStaticBlocks;
constexpr uint64_t kOffU = kOffBpref + 4 * kAggWords * kStaticBlocks;
constexpr uint64_t kStaticBytes = kOffU + 8 * kStaticMaxSubtiles * kGW;  // about 8.75 MiB

__device__ __align__(256) unsigned char g_noalloc_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device.  The first
// call on a device looks it up (cudaGetSymbolAddress, with that device
// current); later calls reuse it.
cudaError_t scratch_address(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
    return cudaSuccess;
}

int bits_needed(uint64_t v) {
    int n = 0;
    while (v) {
        ++n;
        v >>= 1;
    }
    return n;
}

thr_status cuda_error(cudaError_t e, const char* what) {
    char msg[256];
    std::snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString(e));
    return report_error(THR_E_CUDA, msg);
}

}  // namespace
}  // namespace thr

using namespace thr;

extern "C" thr_status thr_query_static(const thr_index* idx, const uint32_t* ids, uint32_t n,
                                       uint32_t T, uint64_t* out, uint64_t cap,
                                       uint64_t* out_len, void* cuda_stream) {
    if (!idx || !ids || !out_len || (cap > 0 && !out))
        return report_error(THR_E_INVAL, "null argument");
    if (n == 0) return report_error(THR_E_INVAL, "n must be at least 1");
    if (n > kStaticMaxIds || idx->W > kStaticMaxWords) {
        char msg[200];
        std::snprintf(msg, sizeof msg,
                      "thr_query_static handles at most %llu ids and ceil(r/64) <= %llu "
                      "words (r <= 2^26); got n = %u, ceil(r/64) = %u",
                      (unsigned long long)kStaticMaxIds, (unsigned long long)kStaticMaxWords, n,
                      idx->W);
        return report_error(THR_E_INVAL, msg);
    }
    for (uint32_t i = 0; i < n; ++i)
        if (ids[i] >= idx->nbitmaps) return report_error(THR_E_INVAL, "id out of range");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev != idx->device || dev >= kMaxDevices)
        return report_error(THR_E_INVAL, "the index lives on another device");
    if (cap > 0) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, out) != cudaSuccess ||
            (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return report_error(THR_E_INVAL, "thr_query_static writes to device memory only");
        }
    }
    unsigned char* blk = nullptr;
    if ((e = scratch_address(dev, &blk)) != cudaSuccess) return cuda_error(e, "scratch address");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    uint32_t* d_ctl = reinterpret_cast<uint32_t*>(blk);
    uint32_t* d_ids = reinterpret_cast<uint32_t*>(blk + kOffIds);
    // the control words (work counter, pass B ticket) must start at zero
    if ((e = cudaMemsetAsync(d_ctl, 0, 64, st)) != cudaSuccess) return cuda_error(e, "memset");
    if ((e = cudaMemcpyAsync(d_ids, ids, sizeof(uint32_t) * n, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return cuda_error(e, "upload ids");

    int cnt = 0;
    const KernelEntry* tab = kernel_table(&cnt);
    uint32_t zmode = 0;
    int need = 1;
    if (T >= 1 && T <= n) {
        const int s1 = bits_needed(T), s0 = bits_needed(uint64_t(n) - T + 1);
        zmode = s0 < s1 ? 1u : 0u;
        need = std::min(s1, s0);
    }
    const KernelEntry* k = &tab[cnt - 1];
    for (int i = 0; i < cnt; ++i)
        if (tab[i].S >= need) {
            k = &tab[i];
            break;
        }
    QueryParams p{};
    p.words = idx->d_words;
    p.mtab = idx->d_mtab;
    p.sdesc = idx->d_sdesc;
    p.masks = idx->d_masks;
    p.desc = idx->d_desc;
    p.ids = d_ids;
    p.n = n;
    p.T = T;
    p.zmode = zmode;
    p.W = idx->W;
    p.NG = idx->NG;
    p.ntiles = idx->NG;
    p.ragged = uint32_t(idx->r % 64);
    p.ctl = d_ctl;
    p.U = reinterpret_cast<uint64_t*>(blk + kOffU);
    p.aggs = reinterpret_cast<uint32_t*>(blk + kOffAggs);
    int per_sm = 0;
    if ((e = k->occupancy(&per_sm)) != cudaSuccess) return cuda_error(e, "occupancy");
    const uint64_t grid = std::min<uint64_t>((idx->NG + kNW - 1) / kNW,
                                             uint64_t(std::max(per_sm, 1)) * idx->num_sms);
    if ((e = k->launch(p, int(std::max<uint64_t>(grid, 1)), st)) != cudaSuccess)
        return cuda_error(e, "launch threshold kernel");
    WriteParams w{};
    w.U = p.U;
    w.aggs = p.aggs;
    w.pref = reinterpret_cast<uint32_t*>(blk + kOffPref);
    w.bagg = reinterpret_cast<uint32_t*>(blk + kOffBagg);
    w.bpref = reinterpret_cast<uint32_t*>(blk + kOffBpref);
    w.out = out;
    w.cap = cap;
    w.W = idx->W;
    w.NG = idx->NG;
    w.ctl = d_ctl;
    if ((e = launch_reencode(w, st)) != cudaSuccess) return cuda_error(e, "launch re-encoding");
    uint32_t h[4] = {0, 0, 0, 0};
    if ((e = cudaMemcpyAsync(h, d_ctl, sizeof h, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_error(e, "read result length");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_error(e, "query");
    *out_len = uint64_t(h[2]) | (uint64_t(h[3]) << 32);
    if (*out_len > cap) return report_error(THR_E_NOSPACE, "output buffer too small");
    return THR_OK;
}
