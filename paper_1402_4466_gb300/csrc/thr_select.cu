// Per-query choice of the counting kernel (thr_query_batch policies).
//
//   THR_POLICY_PLAIN    the variant given in the flags for every query.
//   THR_POLICY_RULE     the rule chooser, in the form of the execution-time
//                       model of Sec. 8.1: each variant's time is predicted
//                       by a linear model in the query's compressed size and
//                       set bits, and the smallest prediction wins (the
//                       hybrid H of Sec. 8.2).
//   THR_POLICY_LEARNED  the learned cost model when one is loaded, else the
//                       rule chooser.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "thr_batch.h"

namespace thr {

namespace {

// Predicted pass-A time (arbitrary units) of the two counting kernels:
//   carry-save  a0 + a1 * words + a2 * words * S
//   ScanCount   b0 + b1 * words + b2 * set bits
// words = compressed words of the query's inputs, S = counter width.
struct RuleModel {
    double a0 = 0, a1 = 1.0, a2 = 0.25;
    double b0 = 0, b1 = 1.0, b2 = 0.35;
};
std::mutex g_rule_mu;
RuleModel g_rule;

}  // namespace

void set_rule_model(const double* c) {
    std::lock_guard<std::mutex> lk(g_rule_mu);
    g_rule = RuleModel{c[0], c[1], c[2], c[3], c[4], c[5]};
}

void get_rule_model(double* c) {
    std::lock_guard<std::mutex> lk(g_rule_mu);
    const RuleModel& m = g_rule;
    const double v[6] = {m.a0, m.a1, m.a2, m.b0, m.b1, m.b2};
    for (int i = 0; i < 6; ++i) c[i] = v[i];
}

uint8_t rule_choice(const thr_index* idx, const uint32_t* ids, uint32_t n, uint32_t T) {
    if (n > 255) return 0;
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
    int cls = 0;
    uint32_t z = 0;
    choose_class(n, T, &cls, &z);
    const double S = double(std::max(1, int(std::ceil(std::log2(double(std::min(T, n - T + 1)) + 1)))));
    const double t_csa = m.a0 + m.a1 * words + m.a2 * words * S;
    const double t_sc = m.b0 + m.b1 * words + m.b2 * bits;
    return t_sc < t_csa ? uint8_t(kClassScanCount) : uint8_t(0);
}

thr_status choose_variants(const thr_index* idx, uint32_t nq, const uint32_t* id_off,
                           const uint32_t* ids, const uint32_t* T, uint32_t policy,
                           uint32_t variant, std::vector<uint8_t>* cls) {
    cls->assign(nq, 0);
    if (policy == THR_POLICY_PLAIN) {
        if (variant == THR_VARIANT_SCANCOUNT)
            for (uint32_t q = 0; q < nq; ++q) (*cls)[q] = uint8_t(kClassScanCount);
        return THR_OK;
    }
    if (policy == THR_POLICY_LEARNED) {
        bool used = false;
        thr_status s = learned_choice(idx, nq, id_off, ids, T, cls, &used);
        if (s != THR_OK || used) return s;
    }
    for (uint32_t q = 0; q < nq; ++q)
        (*cls)[q] = rule_choice(idx, ids + id_off[q], id_off[q + 1] - id_off[q], T[q]);
    return THR_OK;
}

// Until the learned model is built the learned policy uses the rule.
thr_status learned_choice(const thr_index*, uint32_t, const uint32_t*, const uint32_t*,
                          const uint32_t*, std::vector<uint8_t>*, bool* used) {
    *used = false;
    return THR_OK;
}

}  // namespace thr
