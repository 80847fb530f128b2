// Batched execution of threshold queries (thr_batch.cu) and the launch
// tuning it consults (thr_tune.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/thr.h"
#include "thr_exec.h"
#include "thr_index.h"

namespace thr {

// The queries of a batch (host arrays, validated by the caller).
struct BatchInput {
    uint32_t nq;
    const uint32_t* id_off;  // nq + 1
    const uint32_t* ids;
    const uint32_t* T;
    const uint8_t* variant;  // counting variant per query (kVar*), or null (kVarCsa)
    const uint8_t* sym = nullptr;  // kSym* per query, or null (thresholds)
    const uint32_t* hi = nullptr;  // range upper bounds (kSymRange queries)
};

struct BatchOptions {
    bool graph = false;        // capture the batch as a CUDA graph and replay it
    bool profile = false;      // time the pass-A launches (no graph then)
    uint64_t scratch_bytes = 0;  // scratch budget per batch; 0: from free memory
    int force_tune = -1;       // launch configuration for every chunk (tuner)
    bool share = true;         // one counting pass per group of queries over the same ids
};

struct BatchStats {
    uint32_t chunks = 0, launches = 0, slots = 0;
    uint32_t tune = 0;      // configuration of the first chunk
    uint32_t tune_key = 0;  // its shape key (tune_key)
    int graph_reused = -1;  // 1 updated a cached graph, 0 instantiated, -1 no graph
    double pass_a_ms = -1;  // with profile
};

// Launch configuration of the pass-A launches of a chunk (a small integer,
// the autotuner's candidate index):
//   bit 0  work-item order: subtile-major (1) or query-major (0)
//   bit 1  merge: every carry-save query of the chunk runs in the widest
//          counter width among them, so one launch covers them all
//   bit 2  split: launches that run side by side get CTAs in proportion to
//          their work (each a share of its full occupancy), else each is
//          sized for the whole GPU
//   bit 3  dynamic: warps take work items from a counter as they finish
//          (balances items of uneven cost), else static striding
constexpr uint32_t kTuneOrder = 1, kTuneMerge = 2, kTuneSplit = 4, kTuneDynamic = 8;
constexpr uint32_t kTuneCandidates = 16;
// Shape of a chunk, the key of the tuning table: several kernel classes
// (bit 0) and the bit length of the mean number of inputs per query.
uint32_t tune_key(bool multi_class, double mean_n);
// The configuration stored for a shape (thr_autotune), else the default.
uint32_t tune_lookup(const thr_index* idx, uint32_t key);

// Run a batch with results into the device pool dpool (cap words); h_off,
// h_len receive each query's place and length, *total the words needed.
// Words past cap are not written.  Synchronous.
// THR_TRACE_TIME=1 in the environment: one stderr line per batch call with
// the host time (us) at the end of planning, staging, launch and the wait
// (and, from thr_query_batch, of its argument checks and variant choice).
bool trace_time_on();
double now_us();

thr_status run_batch(const thr_index* idx, const BatchInput& in, uint64_t* dpool, uint64_t cap,
                     uint64_t* h_off, uint64_t* h_len, uint64_t* total, cudaStream_t st,
                     const BatchOptions& opt, BatchStats* stats);

// Time every launch configuration on the sample batch (reps runs each after
// a warm-up, L2 flushed before each) and store the fastest for its shape.
thr_status autotune(const thr_index* idx, const BatchInput& in, cudaStream_t st, uint32_t reps,
                    double* times, uint32_t* best, bool share);

// Counting variant per query for a thr_query_batch policy (thr_select.cu);
// variant_flag: the THR_VARIANT_* of the flags (THR_POLICY_PLAIN).  share:
// queries over one id multiset will share a counting pass (no THR_NO_SHARE),
// so under the RULE and LEARNED policies they keep the grouped carry-save
// variant that shares.
thr_status choose_variants(const thr_index* idx, uint32_t nq, const uint32_t* id_off,
                           const uint32_t* ids, const uint32_t* T, uint32_t policy,
                           uint32_t variant_flag, std::vector<uint8_t>* var,
                           bool share = true);
thr_status learned_choice(const thr_index* idx, uint32_t nq, const uint32_t* id_off,
                          const uint32_t* ids, const uint32_t* T, std::vector<uint8_t>* var,
                          bool* used);
uint8_t rule_choice(const thr_index* idx, const uint32_t* ids, uint32_t n, uint32_t T);
int variant_of_flag(uint32_t variant_flag);
constexpr int kRuleCoeffs = 12;
void set_rule_model(const double* c);
void get_rule_model(double* c);

}  // namespace thr
