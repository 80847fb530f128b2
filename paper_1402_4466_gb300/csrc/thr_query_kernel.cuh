// The fused threshold kernel k_threshold<S> (see thr_device.cuh for the
// index layout and the outline).  S = counter width; the host picks the
// smallest instantiated S with 2^S > the threshold the counters test.
#pragma once

#include "thr_device.cuh"

namespace thr {

// Per-warp scratch in shared memory.
struct WarpSmem {
    uint4 rec[kCH];                 // active inputs of the current chunk
    uint32_t bu[32], bfe[32], bend[32];  // marker batch: start, fill end, end
    long long boff[32];             // literal address = boff + word index
    unsigned long long bfill[32];   // fill word value
};

struct CtaSmem {
    WarpSmem w[kNW];
    uint32_t lastcls[kNT];
    uint32_t wsum[kNW];
    uint32_t wmax[kNW];
    uint32_t tile;
    uint32_t fc, lc, hf;
    RangeAgg P, I;
};

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t* p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Values of one active input at the lane's 4 words (0 outside [x0, x1)).
// rec: .x/.y = first literal word (one literal run) or first mtab entry
// (mixed); .z/.w = woff | nm << 40, bit 63 set for mixed.
__device__ __forceinline__ void decode_input(const QueryParams& p, uint4 rec,
                                             uint32_t x0, uint32_t x1,
                                             uint32_t lane, WarpSmem& ws,
                                             uint64_t (&v)[kWPL]) {
    const uint64_t ra = (uint64_t(rec.y) << 32) | rec.x;
    const uint32_t xl = x0 + kWPL * lane;
#pragma unroll
    for (int q = 0; q < kWPL; ++q) v[q] = 0;
    if (!(rec.w >> 31)) {  // one literal run covers the subtile
#pragma unroll
        for (int q = 0; q < kWPL; ++q)
            if (xl + q < x1) v[q] = __ldg(p.words + ra + kWPL * lane + q);
        return;
    }
    const uint64_t rb = (uint64_t(rec.w & 0x7fffffffu) << 32) | rec.z;
    const uint64_t woff = rb & ((1ull << 40) - 1);
    const uint32_t nm = uint32_t(rb >> 40);
    for (uint32_t mb = 0; mb < nm; mb += 32) {
        const uint32_t j = mb + lane;
        if (j < nm) {
            const uint2 e0 = __ldg(p.mtab + ra + j);
            const uint2 e1 = __ldg(p.mtab + ra + j + 1);
            const uint32_t u = e0.y & 0x7fffffffu, ue = e1.y & 0x7fffffffu;
            const uint32_t fe = ue - (e1.x - e0.x - 1);  // end of the fill part
            ws.bu[lane] = u;
            ws.bfe[lane] = fe;
            ws.bend[lane] = ue;
            ws.boff[lane] = (long long)(woff + e0.x + 1) - (long long)fe;
            ws.bfill[lane] = (e0.y >> 31) ? ~0ull : 0ull;
        }
        __syncwarp();
        const uint32_t nb = min(32u, nm - mb);
        const uint32_t lo = ws.bu[0], hi = ws.bend[nb - 1];
        if (xl < hi && xl + kWPL > lo) {
            const uint32_t xs = max(xl, lo);
            uint32_t c = 0;
#pragma unroll
            for (uint32_t step = 16; step; step >>= 1)
                if (c + step < nb && ws.bu[c + step] <= xs) c += step;
#pragma unroll
            for (int q = 0; q < kWPL; ++q) {
                const uint32_t x = xl + q;
                if (x < lo || x >= hi || x >= x1) continue;
                while (c + 1 < nb && ws.bend[c] <= x) ++c;
                v[q] = x < ws.bfe[c] ? ws.bfill[c]
                                     : __ldg(p.words + (ws.boff[c] + (long long)x));
            }
        }
        __syncwarp();
    }
}

// One warp computes the 128 result words of subtile [x0, x1) (lane: 4
// consecutive words starting at x0 + 4 lane; zero past x1).
template <int S>
__device__ __forceinline__ void subtile_result(const QueryParams& p, uint32_t x0,
                                               uint32_t x1, uint32_t lane,
                                               WarpSmem& ws,
                                               uint64_t (&o)[kWPL]) {
#pragma unroll
    for (int q = 0; q < kWPL; ++q) o[q] = 0;
    if (x0 >= p.W) return;
    const uint32_t g = x0 / kGW;
    const uint64_t tstride = uint64_t(p.NG) + 1;
    Counters<S> cnt;
    cnt.clear();
    uint32_t k_ones = 0, d_act = 0;
    const bool one_chunk = p.n <= uint32_t(kCH);
    const uint64_t inv = p.zmode ? ~0ull : 0ull;
    for (uint32_t c0 = 0; c0 < p.n; c0 += kCH) {
        const uint32_t cn = min(uint32_t(kCH), p.n - c0);
        uint32_t nrec = 0;
        // 1. lookup and classify, lane per input
        for (uint32_t i0 = 0; i0 < cn; i0 += 32) {
            const uint32_t i = i0 + lane;
            uint32_t type = 0;  // 0 zero fill, 1 ones fill, 2 literal run, 3 mixed
            uint64_t ra = 0, rb = 0;
            if (i < cn) {
                const uint32_t b = __ldg(p.ids + c0 + i);
                const BitmapDesc d = p.desc[b];
                const uint32_t* tt = p.ttab + uint64_t(b) * tstride;
                const uint32_t m0 = __ldg(tt + g), m1 = __ldg(tt + g + 1);
                const uint2 e0 = __ldg(p.mtab + d.moff + m0);
                const uint2 e1 = __ldg(p.mtab + d.moff + m0 + 1);
                uint32_t mend = d.nmark;
                if (m1 < d.nmark) {
                    const uint2 em = __ldg(p.mtab + d.moff + m1);
                    mend = m1 + (((em.y & 0x7fffffffu) < x1) ? 1u : 0u);
                }
                const uint32_t nm = mend - m0;
                const uint32_t fe = (e1.y & 0x7fffffffu) - (e1.x - e0.x - 1);
                if (nm == 1 && x1 <= fe) {
                    type = (e0.y >> 31) ? 1u : 0u;
                } else if (nm == 1 && x0 >= fe) {
                    type = 2;
                    ra = d.woff + e0.x + 1 + (x0 - fe);
                } else {
                    type = 3;
                    ra = d.moff + m0;
                    rb = d.woff | (uint64_t(nm) << 40) | (1ull << 63);
                }
            }
            const uint32_t act = __ballot_sync(~0u, type >= 2);
            k_ones += __popc(__ballot_sync(~0u, type == 1));
            if (type >= 2) {
                const uint32_t slot = nrec + __popc(act & ((1u << lane) - 1u));
                ws.rec[slot] = make_uint4(uint32_t(ra), uint32_t(ra >> 32),
                                          uint32_t(rb), uint32_t(rb >> 32));
            }
            nrec += __popc(act);
        }
        __syncwarp();
        d_act += nrec;
        if (one_chunk) {  // run-aware pruning (Sec. 6.4 cases 1 and 2)
            const int64_t Tp = int64_t(p.T) - int64_t(k_ones);
            if (Tp <= 0 || Tp > int64_t(d_act)) break;
        }
        // 2. count the active inputs, four at a time
        for (uint32_t r0 = 0; r0 < nrec; r0 += 4) {
            uint64_t v[4][kWPL];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (r0 + j < nrec) {
                    decode_input(p, ws.rec[r0 + j], x0, x1, lane, ws, v[j]);
#pragma unroll
                    for (int q = 0; q < kWPL; ++q) v[j][q] ^= inv;
                } else {
#pragma unroll
                    for (int q = 0; q < kWPL; ++q) v[j][q] = 0;
                }
            }
#pragma unroll
            for (int q = 0; q < kWPL; ++q) {
                cnt.add4(2 * q, uint32_t(v[0][q]), uint32_t(v[1][q]),
                         uint32_t(v[2][q]), uint32_t(v[3][q]));
                cnt.add4(2 * q + 1, uint32_t(v[0][q] >> 32), uint32_t(v[1][q] >> 32),
                         uint32_t(v[2][q] >> 32), uint32_t(v[3][q] >> 32));
            }
        }
        __syncwarp();
    }
    // 3. compare with T' = T - k (or the zeros with d - T' + 1)
    const int64_t Tp = int64_t(p.T) - int64_t(k_ones);
    const uint32_t xl = x0 + kWPL * lane;
    if (Tp <= 0) {
#pragma unroll
        for (int q = 0; q < kWPL; ++q) o[q] = ~0ull;
    } else if (Tp <= int64_t(d_act)) {
        const uint32_t thr = p.zmode ? uint32_t(int64_t(d_act) - Tp + 1) : uint32_t(Tp);
        const uint32_t flip = p.zmode ? ~0u : 0u;
#pragma unroll
        for (int q = 0; q < kWPL; ++q) {
            const uint32_t lo = cnt.ge(2 * q, thr) ^ flip;
            const uint32_t hi = cnt.ge(2 * q + 1, thr) ^ flip;
            o[q] = (uint64_t(hi) << 32) | lo;
        }
    }
#pragma unroll
    for (int q = 0; q < kWPL; ++q) {
        const uint32_t x = xl + q;
        if (x >= p.W) o[q] = 0;
        else if (x == p.W - 1 && p.ragged) o[q] &= (1ull << p.ragged) - 1;
    }
}

// Block-wide exclusive scans (sum and max) over kNT threads.
__device__ __forceinline__ uint32_t block_excl_sum(uint32_t v, uint32_t* wsum,
                                                   uint32_t& total) {
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(~0u, incl, o);
        if (lane >= uint32_t(o)) incl += t;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    uint32_t before = 0;
    total = 0;
#pragma unroll
    for (int w = 0; w < kNW; ++w) {
        if (w < int(wid)) before += wsum[w];
        total += wsum[w];
    }
    __syncthreads();
    return before + incl - v;
}
__device__ __forceinline__ uint32_t block_excl_max(uint32_t v, uint32_t* wmax,
                                                   uint32_t& all) {
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(~0u, incl, o);
        if (lane >= uint32_t(o)) incl = max(incl, t);
    }
    uint32_t excl = __shfl_up_sync(~0u, incl, 1);
    if (lane == 0) excl = 0;
    if (lane == 31) wmax[wid] = incl;
    __syncthreads();
    uint32_t before = 0;
    all = 0;
#pragma unroll
    for (int w = 0; w < kNW; ++w) {
        if (w < int(wid)) before = max(before, wmax[w]);
        all = max(all, wmax[w]);
    }
    __syncthreads();
    return max(before, excl);
}

template <int S>
__global__ void __launch_bounds__(kNT) k_threshold(const QueryParams p) {
    __shared__ CtaSmem sm;
    const uint32_t tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (;;) {
        if (tid == 0) sm.tile = atomicAdd(p.ctl + 0, 1u);
        __syncthreads();
        const uint32_t t = sm.tile;
        if (t >= p.ntiles) break;
        const uint32_t w0 = t * uint32_t(kTW);
        const uint32_t w1 = min(w0 + uint32_t(kTW), p.W);
        const uint32_t x0 = w0 + wid * uint32_t(kGW);
        const uint32_t x1 = min(x0 + uint32_t(kGW), p.W);
        uint64_t o[kWPL];
        subtile_result<S>(p, x0, x1, lane, sm.w[wid], o);

        // ---- canonical re-encoding of the tile's words
        const uint32_t xb = w0 + kWPL * tid;  // this thread's first word
        uint32_t cls[kWPL];
        bool valid[kWPL];
#pragma unroll
        for (int q = 0; q < kWPL; ++q) {
            valid[q] = xb + q < w1;
            cls[q] = o[q] == 0 ? 0u : (o[q] == ~0ull ? 1u : 2u);
        }
        sm.lastcls[tid] = cls[kWPL - 1];
        if (tid == 0) sm.fc = cls[0];
#pragma unroll
        for (int q = 0; q < kWPL; ++q)
            if (xb + q == w1 - 1) sm.lc = cls[q];
        __syncthreads();
        const uint32_t pc = tid ? sm.lastcls[tid - 1] : 0u;
        uint32_t headbits = 0, nh = 0, nl = 0;
#pragma unroll
        for (int q = 0; q < kWPL; ++q) {
            if (!valid[q]) continue;
            const bool h = (tid == 0 && q == 0)
                               ? false
                               : starts_group(q ? cls[q - 1] : pc, cls[q]);
            if (h) {
                headbits |= 1u << q;
                ++nh;
            }
            if (cls[q] == 2u) ++nl;
        }
        uint32_t tot;
        const uint32_t ex = block_excl_sum((nh << 16) | nl, sm.wsum, tot);
        const uint32_t eh = ex >> 16, el = ex & 0xFFFFu;
        uint32_t key = 0, lc = el;
#pragma unroll
        for (int q = 0; q < kWPL; ++q) {
            if (!valid[q]) continue;
            if ((headbits >> q) & 1u) key = ((kWPL * tid + q + 1) << 16) | (lc << 2) | cls[q];
            if (cls[q] == 2u) ++lc;
        }
        uint32_t kall;
        const uint32_t ek = block_excl_max(key, sm.wmax, kall);
        const uint32_t fc = sm.fc;

        if (tid == 0) {
            RangeAgg A;
            A.start = w0;
            A.nh = tot >> 16;
            A.nl = tot & 0xFFFFu;
            uint32_t lhc = 0, has = 0;
            A.lh = 0;
            A.lp = 0;
            if (kall) {
                A.lh = w0 + (kall >> 16) - 1;
                A.lp = (kall >> 2) & 0x3FFFu;
                lhc = kall & 3u;
                has = 1;
            }
            A.cls = fc | (sm.lc << 2) | (lhc << 4) | (has << 6);
            uint32_t* st = p.states + uint64_t(t) * kStateWords;
            RangeAgg P, I;
            uint32_t hf;
            if (t == 0) {
                hf = 1;
                P.start = P.nh = P.nl = P.lh = P.lp = P.cls = 0;
                I = A;
                I.nh += 1;
                if (!has) {
                    I.lh = 0;
                    I.lp = 0;
                    I.cls = (A.cls & 0xFu) | (fc << 4) | (1u << 6);
                }
            } else {
                agg_store(st + 1, A);
                __threadfence();
                st_release(st, 1u);
                RangeAgg R{};
                bool haveR = false;
                int64_t j = int64_t(t) - 1;
                uint32_t spins = 0;
                for (;;) {
                    uint32_t* sj = p.states + uint64_t(j) * kStateWords;
                    const uint32_t f = ld_acquire(sj);
                    if (f == 0u) {
                        if (++spins > p.spin_limit) {
                            atomicOr(p.ctl + 1, kErrSpin);
                            P.start = P.nh = P.nl = P.lh = P.lp = P.cls = 0;
                            break;
                        }
                        __nanosleep(32);
                        continue;
                    }
                    if (f == 2u) {
                        const RangeAgg Ij = agg_load(sj + 7);
                        P = haveR ? agg_combine(Ij, R) : Ij;
                        break;
                    }
                    const RangeAgg Aj = agg_load(sj + 1);
                    R = haveR ? agg_combine(Aj, R) : Aj;
                    haveR = true;
                    --j;
                }
                hf = starts_group(agg_lc(P), fc) ? 1u : 0u;
                I = agg_combine(P, A);
            }
            agg_store(st + 7, I);
            __threadfence();
            st_release(st, 2u);
            sm.P = P;
            sm.I = I;
            sm.hf = hf;
            if (t == p.ntiles - 1) {  // the group that ends at word W
                const uint64_t L = uint64_t(I.nl) - I.lp;
                const uint64_t F = uint64_t(p.W) - I.lh - L;
                const uint64_t b = (F && agg_lhc(I) == 1u) ? 1ull : 0ull;
                const uint64_t pos = uint64_t(I.nh) - 1 + I.lp;
                if (pos < p.cap) p.out[pos] = b | (F << 1) | (L << 33);
                *reinterpret_cast<unsigned long long*>(p.ctl + 2) =
                    uint64_t(I.nh) + uint64_t(I.nl);
            }
        }
        __syncthreads();
        const RangeAgg P = sm.P;
        const uint32_t hf = sm.hf;
        uint64_t J = uint64_t(P.nh) + (tid ? hf : 0u) + eh;  // heads before xb
        uint64_t Lc = uint64_t(P.nl) + el;                    // literals before xb
        uint32_t hp, hcls;
        uint64_t lg;
        bool have_hp;
        if (ek) {
            hp = w0 + (ek >> 16) - 1;
            lg = uint64_t(P.nl) + ((ek >> 2) & 0x3FFFu);
            hcls = ek & 3u;
            have_hp = true;
        } else if (hf && tid) {
            hp = w0;
            lg = P.nl;
            hcls = fc;
            have_hp = true;
        } else {
            hp = P.lh;
            lg = P.lp;
            hcls = agg_lhc(P);
            have_hp = t > 0 && agg_has(P);
        }
#pragma unroll
        for (int q = 0; q < kWPL; ++q) {
            if (!valid[q]) continue;
            const uint32_t x = xb + q;
            const bool h = (tid == 0 && q == 0) ? (hf != 0) : ((headbits >> q) & 1u);
            if (h) {
                if (have_hp) {  // the previous group ends here: write its marker
                    const uint64_t L = Lc - lg;
                    const uint64_t F = uint64_t(x - hp) - L;
                    const uint64_t b = (F && hcls == 1u) ? 1ull : 0ull;
                    const uint64_t pos = J - 1 + lg;
                    if (pos < p.cap) p.out[pos] = b | (F << 1) | (L << 33);
                }
                hp = x;
                lg = Lc;
                hcls = cls[q];
                have_hp = true;
                ++J;
            }
            if (cls[q] == 2u) {
                const uint64_t pos = J + Lc;
                if (pos < p.cap) p.out[pos] = o[q];
                ++Lc;
            }
        }
        __syncthreads();
    }
}

}  // namespace thr
