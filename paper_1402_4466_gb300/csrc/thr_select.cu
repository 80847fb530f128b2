// Per-query choice of the counting kernel (thr_query_batch policies).
//
//   THR_POLICY_PLAIN    the variant given in the flags for every query.
//   THR_POLICY_RULE     the rule chooser, in the form of the execution-time
//                       model of Sec. 8.1: each variant's time is predicted
//                       by a linear model in the query's compressed size and
//                       set bits, and the smallest prediction wins (the
//                       hybrid H of Sec. 8.2).
//   THR_POLICY_LEARNED  the learned cost model (thr_mlp.cu) attached to the
//                       index, else the rule chooser: the variant with the
//                       smallest predicted time wins.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <thread>
#include <vector>

#include "thr_batch.h"
#include "thr_mlp.h"

namespace thr {

namespace {

// Predicted pass-A time (ms) of the three counting kernels:
//   carry-save, grouped   a0 + a1 * words + a2 * words * S
//   carry-save, position  c0 + c1 * words + c2 * words * S1
//   ScanCount             b0 + b1 * words + b2 * set bits
//   carry-save, split     s0 + s1 * words + s2 * words * S
// words = compressed words of the query's inputs, S = counter bits of the
// grouped kernel (the smaller of the ones and zeros counts), S1 = counter
// bits when counting ones.  The defaults are placeholders until
// thr_rule_model sets coefficients fitted to measured times.
struct RuleModel {
    double a0 = 0, a1 = 1.0, a2 = 0.25;
    double c0 = 0, c1 = 1.0, c2 = 0.3;
    double b0 = 0, b1 = 1.0, b2 = 0.35;
    double s0 = 0, s1 = 1.0, s2 = 0.3;
};
std::mutex g_rule_mu;
RuleModel g_rule;

int bitlen(uint64_t v) {
    int k = 0;
    while (v) {
        ++k;
        v >>= 1;
    }
    return k;
}

}  // namespace

void set_rule_model(const double* c) {
    std::lock_guard<std::mutex> lk(g_rule_mu);
    g_rule = RuleModel{c[0], c[1], c[2], c[3], c[4], c[5], c[6], c[7], c[8], c[9], c[10], c[11]};
}

void get_rule_model(double* c) {
    std::lock_guard<std::mutex> lk(g_rule_mu);
    const RuleModel& m = g_rule;
    const double v[kRuleCoeffs] = {m.a0, m.a1, m.a2, m.c0, m.c1, m.c2,
                                   m.b0, m.b1, m.b2, m.s0, m.s1, m.s2};
    for (int i = 0; i < kRuleCoeffs; ++i) c[i] = v[i];
}

uint8_t rule_choice(const thr_index* idx, const uint32_t* ids, uint32_t n, uint32_t T) {
    RuleModel m;
    {
        std::lock_guard<std::mutex> lk(g_rule_mu);
        m = g_rule;
    }
    double words = 0, bits = 0;
    for (uint32_t i = 0; i < n; ++i) {
        words += double(idx->desc[ids[i]].len);
        bits += double(idx->set_rows[ids[i]]);
    }
    const bool counted = T >= 1 && T <= n;
    const double S1 = counted ? double(bitlen(T)) : 1.0;
    const double S = counted ? double(std::min(bitlen(T), bitlen(uint64_t(n) - T + 1))) : 1.0;
    const double t[4] = {m.a0 + m.a1 * words + m.a2 * words * S,
                         m.c0 + m.c1 * words + m.c2 * words * S1,
                         m.b0 + m.b1 * words + m.b2 * bits,
                         m.s0 + m.s1 * words + m.s2 * words * S};
    int best = kVarCsa;
    for (int v = 1; v < 4; ++v) {
        if (v == kVarScanCount && n > 65535) continue;
        if (v == kVarSplit && S > 8) continue;
        if (t[v] < t[best]) best = v;
    }
    return uint8_t(best);
}

// The split-input kernel buys parallelism for queries with few subtiles; a
// batch whose (query, subtile) items already outnumber the GPU's resident
// warps several times over gains nothing from it (the costs both choosers
// learned come from queries timed alone), so it is not chosen there.
void drop_split_when_saturated(const thr_index* idx, uint32_t nq, std::vector<uint8_t>* var) {
    const uint64_t items = uint64_t(nq) * idx->NG;
    const uint64_t warps = uint64_t(std::max(idx->num_sms, 1)) * 6 * kNW;  // resident
    if (nq > 1 && items >= 4 * warps)
        for (auto& v : *var)
            if (v == kVarSplit) v = uint8_t(kVarCsa);
}

int variant_of_flag(uint32_t f) {
    switch (f) {
        case THR_VARIANT_CSA: return kVarCsa;
        case THR_VARIANT_POSITION: return kVarPos;
        case THR_VARIANT_SCANCOUNT: return kVarScanCount;
        case THR_VARIANT_SPLIT: return kVarSplit;
        case THR_VARIANT_LOOPED: return kVarLooped;
        case THR_VARIANT_STAGED: return kVarStaged;
        default: return -1;
    }
}

// Queries of a batch over the same id multiset share one counting pass of
// the grouped carry-save kernel (thr_batch.cu): the inputs are read and
// counted once for all of them.  Both choosers price a query alone, so a
// variant they predict faster for one member would cost the batch a second
// pass over the same inputs; such members keep the default.  The multiset
// key is order-independent (n and a sum of mixed ids); a collision only
// keeps a query on the default, which is exact like every variant.
void keep_shared_groups(uint32_t nq, const uint32_t* id_off, const uint32_t* ids,
                        std::vector<uint8_t>* var) {
    if (nq < 2) return;
    std::vector<std::pair<uint64_t, uint32_t>> keys(nq);
    for (uint32_t q = 0; q < nq; ++q) {
        uint64_t h = 0;
        for (uint32_t i = id_off[q]; i < id_off[q + 1]; ++i) {
            uint64_t x = uint64_t(ids[i]) + 0x9E3779B97F4A7C15ull;  // splitmix64 of the id
            x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
            x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
            h += x ^ (x >> 31);
        }
        keys[q] = {h ^ (uint64_t(id_off[q + 1] - id_off[q]) << 40), q};
    }
    std::sort(keys.begin(), keys.end());
    for (uint32_t a = 0; a < nq;) {
        uint32_t b = a + 1;
        while (b < nq && keys[b].first == keys[a].first) ++b;
        if (b - a > 1)
            for (uint32_t k = a; k < b; ++k) (*var)[keys[k].second] = uint8_t(kVarCsa);
        a = b;
    }
}

thr_status choose_variants(const thr_index* idx, uint32_t nq, const uint32_t* id_off,
                           const uint32_t* ids, const uint32_t* T, uint32_t policy,
                           uint32_t variant_flag, std::vector<uint8_t>* cls, bool share) {
    cls->assign(nq, uint8_t(kVarCsa));
    if (policy == THR_POLICY_PLAIN) {
        const int v = variant_of_flag(variant_flag);
        for (uint32_t q = 0; q < nq; ++q) (*cls)[q] = uint8_t(v < 0 ? kVarCsa : v);
        return THR_OK;
    }
    if (policy == THR_POLICY_LEARNED) {
        bool used = false;
        thr_status s = learned_choice(idx, nq, id_off, ids, T, cls, &used);
        if (s != THR_OK) return s;
        if (used) {
            drop_split_when_saturated(idx, nq, cls);
            if (share) keep_shared_groups(nq, id_off, ids, cls);
            return THR_OK;
        }
    }
    for (uint32_t q = 0; q < nq; ++q)
        (*cls)[q] = rule_choice(idx, ids + id_off[q], id_off[q + 1] - id_off[q], T[q]);
    drop_split_when_saturated(idx, nq, cls);
    if (share) keep_shared_groups(nq, id_off, ids, cls);
    return THR_OK;
}

void query_features(const thr_index* idx, const uint32_t* ids, uint32_t n, uint32_t T,
                    float* f) {
    std::vector<double> w(n), d(n);
    double sw = 0, sd = 0;
    const double r = double(idx->r);
    for (uint32_t i = 0; i < n; ++i) {  // log terms precomputed per bitmap at build
        const double words = double(idx->desc[ids[i]].len);
        const double dens = double(idx->set_rows[ids[i]]) / r;
        w[i] = idx->feat_lw[ids[i]];
        d[i] = idx->feat_ld[ids[i]];
        sw += words;
        sd += dens;
    }
    std::sort(w.begin(), w.end());
    std::sort(d.begin(), d.end());
    auto quant = [&](const std::vector<double>& v, double qq) {
        const double pos = qq * double(v.size() - 1);
        const size_t lo = size_t(pos);
        const size_t hi = std::min(lo + 1, v.size() - 1);
        return v[lo] + (pos - double(lo)) * (v[hi] - v[lo]);
    };
    f[0] = float(std::log2(double(n)));
    f[1] = float(std::log2(double(T) + 1.0));
    f[2] = T <= n ? float(std::log2(double(n) - double(T) + 2.0)) : 0.f;
    f[3] = float(std::log2(r));
    const double qs[5] = {0.0, 0.25, 0.5, 0.75, 1.0};
    for (int k = 0; k < 5; ++k) f[4 + k] = float(quant(w, qs[k]));
    f[9] = float(std::log2(sw + 1.0));
    for (int k = 0; k < 5; ++k) f[10 + k] = float(quant(d, qs[k]));
    f[15] = float(sd);
}

constexpr float kSwitchGain = 0.10f;

// The split kernel exists for counter widths up to 8 bits.
bool split_applies(uint32_t n, uint32_t T) {
    int cls = 0;
    uint32_t z = 0;
    choose_class(n, T, &cls, &z);
    return cls < kSplitWidths;
}

// With a cost model attached to the index: features of every query, one
// forward pass for the batch, and per query the variant with the smallest
// predicted time among those it can run (ScanCount needs n <= 65535).
thr_status learned_choice(const thr_index* idx, uint32_t nq, const uint32_t* id_off,
                          const uint32_t* ids, const uint32_t* T, std::vector<uint8_t>* var,
                          bool* used) {
    const Selector* sel = nullptr;
    {
        std::lock_guard<std::mutex> lk(idx->tune_mu);
        sel = idx->selector;
    }
    *used = false;
    if (!sel) return THR_OK;
    std::vector<float> X(size_t(nq) * kSelFeatures), Y(size_t(nq) * kSelVariants);
    auto features = [&](uint32_t q0, uint32_t q1) {
        for (uint32_t q = q0; q < q1; ++q)
            query_features(idx, ids + id_off[q], id_off[q + 1] - id_off[q], T[q],
                           &X[size_t(q) * kSelFeatures]);
    };
    // large batches: the features on a few host threads
    const uint32_t nthreads =
        nq >= 1024 ? std::min<uint32_t>(8, std::max(1u, std::thread::hardware_concurrency()))
                   : 1;
    if (nthreads > 1) {
        std::vector<std::thread> pool;
        for (uint32_t t = 1; t < nthreads; ++t)
            pool.emplace_back(features, uint32_t(uint64_t(nq) * t / nthreads),
                              uint32_t(uint64_t(nq) * (t + 1) / nthreads));
        features(0, uint32_t(nq / nthreads));
        for (auto& th : pool) th.join();
    } else {
        features(0, nq);
    }
    thr_status s = sel->predict_memo(X.data(), nq, Y.data());
    if (s != THR_OK) return s;
    // another variant replaces the default only when it is predicted at
    // least kSwitchGain faster: a marginal switch costs a batch an extra
    // launch and the sharing of reads with the default's queries
    const float margin = std::log(1.0f + kSwitchGain);
    for (uint32_t q = 0; q < nq; ++q) {
        const uint32_t n = id_off[q + 1] - id_off[q];
        const float* y = &Y[size_t(q) * kSelVariants];
        int best = kVarCsa;
        float best_y = y[kVarCsa] - margin;
        for (int v = 0; v < kSelVariants; ++v) {
            if (v == kVarCsa || (v == kVarScanCount && n > 65535)) continue;
            if (v == kVarSplit && !split_applies(n, T[q])) continue;
            if (y[v] < best_y) {
                best = v;
                best_y = y[v];
            }
        }
        (*var)[q] = uint8_t(best);
    }
    *used = true;
    return THR_OK;
}

}  // namespace thr
