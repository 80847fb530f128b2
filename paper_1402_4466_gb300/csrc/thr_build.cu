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

// Subtile classes.  One CTA per bitmap walks its subtiles in order; for
// every subtile it counts the literal and ones-fill words of the markers that
// overlap it (the RBMrg/EWAH run cases of Sec. 6.4 decided once, at build):
// class 0 all zero fill, 1 all ones fill, 2 one literal run (the subtile's
// words are contiguous literals), 3 mixed.  Mixed subtiles are numbered in
// order (block scan); the descriptor holds class | flags | counts | field
// (field: class 2 = stream index of the first literal, class 3 = the rank,
// replaced by the mask record index in k_subtile_masks).
__global__ void k_subtile_class(const uint2* __restrict__ mtab,
                                const uint32_t* __restrict__ ttab,
                                const BitmapDesc* __restrict__ desc,
                                uint64_t* __restrict__ sdesc,
                                uint64_t* __restrict__ sseg,
                                uint32_t* __restrict__ mixed_count, uint32_t W,
                                uint32_t NG) {
    const uint32_t b = blockIdx.x;
    const BitmapDesc d = desc[b];
    const uint32_t* tt = ttab + uint64_t(b) * (NG + 1);
    __shared__ uint32_t warp_sum[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (uint32_t base = 0; base < NG; base += blockDim.x) {
        const uint32_t g = base + threadIdx.x;
        uint32_t mixed = 0;
        uint64_t word = 0;
        if (g < NG) {
            const uint32_t x0 = g * uint32_t(kGW);
            const uint32_t x1 = min(x0 + uint32_t(kGW), W);
            const uint32_t m0 = tt[g], m1 = tt[g + 1];
            uint32_t mend = d.nmark;
            if (m1 < d.nmark) mend = m1 + (((mtab[d.moff + m1].y & 0x7fffffffu) < x1) ? 1u : 0u);
            uint32_t nl = 0, none = 0;
            for (uint32_t m = m0; m < mend; ++m) {
                const uint2 e0 = mtab[d.moff + m], e1 = mtab[d.moff + m + 1];
                const uint32_t u = e0.y & 0x7fffffffu, ue = e1.y & 0x7fffffffu;
                const uint32_t fe = ue - (e1.x - e0.x - 1);
                const uint32_t la = max(fe, x0), lb = min(ue, x1);
                if (lb > la) nl += lb - la;
                if (e0.y >> 31) {
                    const uint32_t oa = max(u, x0), ob = min(fe, x1);
                    if (ob > oa) none += ob - oa;
                }
            }
            const uint32_t nm = mend - m0, len = x1 - x0;
            const uint2 f0 = mtab[d.moff + m0], f1 = mtab[d.moff + m0 + 1];
            const uint32_t fe0 = (f1.y & 0x7fffffffu) - (f1.x - f0.x - 1);
            uint64_t cls, field = 0;
            if (nl == 0 && none == 0) {
                cls = 0;
            } else if (none == len) {
                cls = 1;
            } else if (nl == len && nm == 1) {
                cls = 2;
                field = uint64_t(f0.x) + 1 + (x0 - fe0);
            } else {
                cls = 3;
                mixed = 1;
            }
            word = cls | (uint64_t(none ? 1 : 0) << 2) | (uint64_t(nl) << 3) |
                   (uint64_t(none) << 11) | (field << 19);
        }
        uint32_t incl = mixed;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= uint32_t(o)) incl += v;
        }
        if (lane == 31) warp_sum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const uint32_t ws = lane < nwarps ? warp_sum[lane] : 0;
            uint32_t wi = ws;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t v = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= uint32_t(o)) wi += v;
            }
            if (lane < nwarps) warp_sum[lane] = wi - ws;
        }
        __syncthreads();
        const uint32_t rank = carry + warp_sum[wid] + incl - mixed;
        if (g < NG) {
            sdesc[uint64_t(b) * NG + g] = mixed ? (word | (uint64_t(rank) << 19)) : word;
            // a literal run: its words are the segment (mixed: k_subtile_masks)
            const uint64_t c = word & 3u;
            sseg[uint64_t(b) * NG + g] =
                c == 2 ? ((word >> 19) | (uint64_t(min(uint32_t(kGW), W - g * uint32_t(kGW))) << 32))
                       : 0ull;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = rank + mixed;
        __syncthreads();
    }
    if (threadIdx.x == 0) mixed_count[b] = carry;
}

// Mask records of the mixed subtiles (layout: MaskRec in thr_device.cuh):
// literal-word mask, literal-or-group-start mask (groups starting strictly
// after the subtile's first word), ones-fill mask, the stream index of the
// first literal at or after the subtile start (base) and the per-32-word
// prefix counts.  The literal at subtile word x then sits at stream index
// base + (literal words in [x0, x)) + (group starts in (x0, x]), because every
// group after the first adds one marker word before its literals.
__global__ void k_subtile_masks(const uint2* __restrict__ mtab,
                                const uint32_t* __restrict__ ttab,
                                const BitmapDesc* __restrict__ desc,
                                const uint64_t* __restrict__ mixed_base,
                                uint64_t* __restrict__ sdesc, uint64_t* __restrict__ sseg,
                                MaskRec* __restrict__ masks, uint32_t nbitmaps,
                                uint32_t W, uint32_t NG) {
    const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= uint64_t(NG) * nbitmaps) return;
    const uint64_t sd = sdesc[i];
    if ((sd & 3u) != 3u) return;
    const uint32_t b = uint32_t(i / NG), g = uint32_t(i % NG);
    const BitmapDesc d = desc[b];
    const uint32_t* tt = ttab + uint64_t(b) * (NG + 1);
    const uint32_t x0 = g * uint32_t(kGW);
    const uint32_t x1 = min(x0 + uint32_t(kGW), W);
    const uint32_t m0 = tt[g], m1 = tt[g + 1];
    uint32_t mend = d.nmark;
    if (m1 < d.nmark) mend = m1 + (((mtab[d.moff + m1].y & 0x7fffffffu) < x1) ? 1u : 0u);
    uint32_t lm[4] = {0, 0, 0, 0}, gm[4] = {0, 0, 0, 0}, om[4] = {0, 0, 0, 0};
    uint32_t base = 0;
    for (uint32_t m = m0; m < mend; ++m) {
        const uint2 e0 = mtab[d.moff + m], e1 = mtab[d.moff + m + 1];
        const uint32_t u = e0.y & 0x7fffffffu, ue = e1.y & 0x7fffffffu;
        const uint32_t fe = ue - (e1.x - e0.x - 1);
        if (m == m0) base = e0.x + 1 + (x0 > fe ? x0 - fe : 0u);
        if (m > m0) {  // u is inside (x0, x1)
            const uint32_t r = u - x0;
            gm[r >> 5] |= 1u << (r & 31);
        }
        for (uint32_t x = max(fe, x0); x < min(ue, x1); ++x) {
            const uint32_t r = x - x0;
            lm[r >> 5] |= 1u << (r & 31);
        }
        if (e0.y >> 31)
            for (uint32_t x = max(u, x0); x < min(fe, x1); ++x) {
                const uint32_t r = x - x0;
                om[r >> 5] |= 1u << (r & 31);
            }
    }
    MaskRec rec;
    uint32_t run = 0;
    rec.pre = 0;
    for (int w = 0; w < 4; ++w) {
        rec.lm[w] = lm[w];
        rec.cm[w] = lm[w] | gm[w];
        rec.om[w] = om[w];
        rec.pre |= run << (8 * w);
        run += __popc(lm[w]) + __popc(gm[w]);
    }
    rec.base = base;
    rec.pad[0] = rec.pad[1] = 0;
    const uint64_t idx = mixed_base[b] + (sd >> 19);
    masks[idx] = rec;
    sdesc[i] = (sd & ((1ull << 19) - 1)) | (idx << 19);
    // the stream words of the subtile's literals and group starts: from the
    // first literal (base) on, `run` of them (at most kGW: each group start
    // takes a fill word of the subtile, each literal a word)
    sseg[i] = uint64_t(base) | (uint64_t(run) << 32);
}

// Thread per (bitmap, word): the classes of 32 consecutive subtiles.
__global__ void k_pack_classes(const uint64_t* __restrict__ sdesc, uint64_t* __restrict__ pcls,
                               uint32_t nbitmaps, uint32_t NG, uint32_t NGW) {
    const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= uint64_t(nbitmaps) * NGW) return;
    const uint64_t b = i / NGW;
    const uint32_t w = uint32_t(i - b * NGW);
    uint64_t word = 0;
    for (uint32_t k = 0; k < 32; ++k) {
        const uint32_t g = 32 * w + k;
        if (g < NG) word |= (sdesc[b * NG + g] & 3ull) << (2 * k);
    }
    pcls[i] = word;
}

cudaError_t launch_pack_classes(const uint64_t* sdesc, uint64_t* pcls, uint32_t nbitmaps,
                                uint32_t NG, cudaStream_t st) {
    const uint32_t NGW = (NG + 31) / 32;
    const uint64_t n = uint64_t(nbitmaps) * NGW;
    k_pack_classes<<<unsigned((n + 255) / 256), 256, 0, st>>>(sdesc, pcls, nbitmaps, NG, NGW);
    return cudaGetLastError();
}

cudaError_t launch_index_build_a(const uint64_t* words, const uint32_t* mpos,
                                 const BitmapDesc* desc, uint2* mtab, uint32_t* ttab,
                                 uint64_t* sdesc, uint64_t* sseg, uint32_t* mixed_count,
                                 uint32_t nbitmaps, uint32_t W, uint32_t NG,
                                 cudaStream_t st) {
    k_marker_scan<<<nbitmaps, 256, 0, st>>>(words, mpos, desc, mtab, W);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const uint64_t n = (uint64_t(NG) + 1) * nbitmaps;
    k_tile_table<<<unsigned((n + 255) / 256), 256, 0, st>>>(mtab, desc, ttab, nbitmaps, NG);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_subtile_class<<<nbitmaps, 256, 0, st>>>(mtab, ttab, desc, sdesc, sseg, mixed_count, W,
                                              NG);
    return cudaGetLastError();
}

cudaError_t launch_index_build_b(const uint2* mtab, const uint32_t* ttab,
                                 const BitmapDesc* desc, const uint64_t* mixed_base,
                                 uint64_t* sdesc, uint64_t* sseg, MaskRec* masks,
                                 uint32_t nbitmaps, uint32_t W, uint32_t NG, cudaStream_t st) {
    const uint64_t ns = uint64_t(NG) * nbitmaps;
    k_subtile_masks<<<unsigned((ns + 255) / 256), 256, 0, st>>>(mtab, ttab, desc, mixed_base,
                                                               sdesc, sseg, masks, nbitmaps, W, NG);
    return cudaGetLastError();
}

}  // namespace thr
