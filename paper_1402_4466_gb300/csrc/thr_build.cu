// Index build kernels (see thr_device.cuh for the layout they produce).
#include "thr_device.cuh"

namespace thr {

// ------------------------------------------------------------- build (K1)

// Segmented exclusive scan of the group extents F + L over the marker words
// of every bitmap (one CTA per bitmap), writing mtab.  `mpos` holds the
// stream index of every marker (found by the host validator), per bitmap at
// desc.moff - b (mtab has one extra entry per bitmap, mpos does not).
__global__ void k_marker_scan(const uint64_t* __restrict__ words,
                              const uint32_t* __restrict__ mpos,
                              const BitmapDesc* __restrict__ desc,
                              uint2* __restrict__ mtab, uint32_t W) {
    const uint32_t b = blockIdx.x;
    const BitmapDesc d = desc[b];
    const uint32_t* mp = mpos + (d.moff - b);
    uint2* mt = mtab + d.moff;
    __shared__ uint32_t warp_sum[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t nwarps = blockDim.x >> 5;
    for (uint32_t base = 0; base < d.nmark; base += blockDim.x) {
        const uint32_t m = base + threadIdx.x;
        uint32_t ext = 0, pos = 0, fb = 0;
        if (m < d.nmark) {
            pos = mp[m];
            const uint64_t mw = words[d.woff + pos];
            fb = uint32_t(mw & 1);
            ext = uint32_t((mw >> 1) & 0xFFFFFFFFull) + uint32_t(mw >> 33);
        }
        uint32_t incl = ext;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= uint32_t(o)) incl += v;
        }
        if (lane == 31) warp_sum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            uint32_t ws = lane < nwarps ? warp_sum[lane] : 0;
            uint32_t wi = ws;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= uint32_t(o)) wi += v;
            }
            if (lane < nwarps) warp_sum[lane] = wi - ws;  // exclusive
        }
        __syncthreads();
        const uint32_t ustart = carry + warp_sum[wid] + incl - ext;
        if (m < d.nmark) mt[m] = make_uint2(pos, ustart | (fb << 31));
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = ustart + ext;
        __syncthreads();
    }
    if (threadIdx.x == 0) mt[d.nmark] = make_uint2(d.len, W);
}

// ttab: for every (bitmap, subtile) the marker containing word 128 g, by
// binary search over the bitmap's ustart column.
__global__ void k_tile_table(const uint2* __restrict__ mtab,
                             const BitmapDesc* __restrict__ desc,
                             uint32_t* __restrict__ ttab, uint32_t nbitmaps,
                             uint32_t NG) {
    const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t per = uint64_t(NG) + 1;
    if (i >= per * nbitmaps) return;
    const uint32_t b = uint32_t(i / per), g = uint32_t(i % per);
    const BitmapDesc d = desc[b];
    if (g == NG) {
        ttab[i] = d.nmark;
        return;
    }
    const uint32_t x = g * uint32_t(kGW);
    uint32_t lo = 0, hi = d.nmark;  // invariant: ustart[lo] <= x < ustart[hi]
    while (hi - lo > 1) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if ((mtab[d.moff + mid].y & 0x7fffffffu) <= x) lo = mid;
        else hi = mid;
    }
    ttab[i] = lo;
}

cudaError_t launch_index_build(const uint64_t* words, const uint32_t* mpos,
                               const BitmapDesc* desc, uint2* mtab,
                               uint32_t* ttab, uint32_t nbitmaps, uint32_t W,
                               uint32_t NG, cudaStream_t st) {
    k_marker_scan<<<nbitmaps, 256, 0, st>>>(words, mpos, desc, mtab, W);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const uint64_t n = (uint64_t(NG) + 1) * nbitmaps;
    const uint64_t blocks = (n + 255) / 256;
    k_tile_table<<<unsigned(blocks), 256, 0, st>>>(mtab, desc, ttab, nbitmaps, NG);
    return cudaGetLastError();
}

}  // namespace thr
