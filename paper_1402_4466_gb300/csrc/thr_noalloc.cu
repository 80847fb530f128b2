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
#include <cstring>
#include <mutex>

#include "thr_index.h"
#include "thr_exec.h"

namespace thr {
namespace {

constexpr uint64_t kStaticMaxWords = 1ull << 20;  // r <= 2^26 rows
constexpr uint64_t kStaticMaxIds = 65536;
// fixed layout: query descriptor | slot list, group record | ids | scratch
// of one slot
// (control words, aggregates, prefixes, result words: about 8.5 MiB at the
// largest r)
constexpr uint64_t kOffList = 256;
constexpr uint64_t kOffIds = 512;
constexpr uint64_t kOffScratch = kOffIds + 4 * kStaticMaxIds;
constexpr uint64_t kStaticBytes = kOffScratch + 9ull * 1024 * 1024;

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
            (a.type != cudaMemoryTypeManaged &&
             (a.type != cudaMemoryTypeDevice || a.device != dev))) {
            cudaGetLastError();
            return report_error(THR_E_INVAL,
                                "thr_query_static writes to device memory of the index's GPU only");
        }
    }
    unsigned char* blk = nullptr;
    if ((e = scratch_address(dev, &blk)) != cudaSuccess) return cuda_error(e, "scratch address");
    const ScratchLayout lay = scratch_layout(1, 1, idx->W, idx->NG, 1);
    if (kOffScratch + lay.total > kStaticBytes)
        return report_error(THR_E_INVAL, "static scratch too small for this index");
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int cls = 0;
    uint32_t zmode = 0;
    choose_class(n, T, &cls, &zmode);
    const QDesc qd{0, n, T, zmode, T, T, 0u, kSymThreshold};
    const uint2 grp1 = make_uint2(0, 1);
    const uint32_t slot0 = 0;
    if ((e = cudaMemcpyAsync(blk, &qd, sizeof qd, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(blk + kOffList, &slot0, sizeof slot0, cudaMemcpyHostToDevice,
                             st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(blk + kOffList + 64, &grp1, sizeof grp1, cudaMemcpyHostToDevice,
                             st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(blk + kOffIds, ids, sizeof(uint32_t) * n, cudaMemcpyHostToDevice,
                             st)) != cudaSuccess)
        return cuda_error(e, "upload query");
    int per_sm = 0;
    if ((e = class_occupancy(cls, &per_sm)) != cudaSuccess) return cuda_error(e, "occupancy");
    Launch L{cls, 0, 1, 0, 1, 1};
    L.grid = int(std::max<uint64_t>(1, std::min<uint64_t>((idx->NG + kNW - 1) / kNW,
                                                          uint64_t(std::max(per_sm, 1)) *
                                                              idx->num_sms)));
    const ChunkPlan ch{0, 1, 0, 1};
    ExecBufs b{};
    b.qd = reinterpret_cast<const QDesc*>(blk);
    b.lists = reinterpret_cast<const uint32_t*>(blk + kOffList);
    b.grp = reinterpret_cast<const uint2*>(blk + kOffList + 64);
    b.memb = reinterpret_cast<const uint32_t*>(blk + kOffList);
    b.ids = reinterpret_cast<const uint32_t*>(blk + kOffIds);
    b.scratch = blk + kOffScratch;
    b.lay = lay;
    b.out = out;
    b.cap = cap;
    b.nids = n;
    b.nq = 1;
    b.nmemb = 1;
    if ((e = enqueue_plan(idx, &ch, 1, &L, b, st, nullptr, 0, nullptr, 0, nullptr)) !=
        cudaSuccess)
        return cuda_error(e, "launch query kernels");
    // one read-back from base: total, error word, check record, {offset, length}
    unsigned long long h[(64 - 8 + 16) / 8] = {};
    if (lay.res - lay.base + 16 > sizeof h) return report_error(THR_E_CUDA, "control layout");
    if ((e = cudaMemcpyAsync(h, b.scratch + lay.base, lay.res - lay.base + 16,
                             cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_error(e, "read result length");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_error(e, "query");
    if (h[(lay.err - lay.base) / 8] & 0xFFFFFFFFull)
        return report_error(THR_E_TIMEOUT,
                            "a query kernel gave up waiting for its shared-memory copies");
    CheckRec chk;
    std::memcpy(&chk, reinterpret_cast<const unsigned char*>(h) + (lay.chk - lay.base),
                sizeof chk);
    if (chk.site) return check_failed(chk);
    *out_len = h[(lay.res - lay.base) / 8 + 1];
    if (*out_len > cap) return report_error(THR_E_NOSPACE, "output buffer too small");
    return THR_OK;
}
