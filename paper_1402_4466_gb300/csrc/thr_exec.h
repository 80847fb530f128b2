// Host side of query execution: the launch plan of a batch of queries and
// the code that enqueues it on a stream (thr_exec.cu).  thr_query,
// thr_query_batch and thr_query_static all go through enqueue_plan.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "thr_device.cuh"
#include "thr_index.h"

namespace thr {

// Kernel classes: 0 .. kNumWidths-1 carry-save with the counter width
// kernel_table()[c].S (grouped decode), kClassScanCount the
// ScanCount kernel with byte counters (kClassScanCount + 1: 16-bit counters), kClassPos + c carry-save of width kernel_table()[c].S
// with the position-major decode of mixed inputs, kClassSplit + c carry-save
// with the inputs split among the CTA's warps (widths up to kSplitWidths),
// kClassLooped + M - 1 Looped with M levels (M = 1 .. kLoopedMax),
// kClassStaged + c carry-save of width kernel_table()[c].S with each input's
// words staged in shared memory by bulk copies (thr_staged.cuh).
constexpr int kNumWidths = 12;
constexpr int kSplitWidths = 8;  // S = 1..8
constexpr int kLoopedMax = 4;    // Looped levels (thresholds) instantiated
constexpr int kClassScanCount = kNumWidths;
constexpr int kClassScanCount16 = kNumWidths + 1;
constexpr int kClassPos = kNumWidths + 2;
constexpr int kClassSplit = 2 * kNumWidths + 2;
constexpr int kClassLooped = kClassSplit + kSplitWidths;
constexpr int kClassStaged = kClassLooped + kLoopedMax;
constexpr int kNumClasses = kClassStaged + kNumWidths;
static_assert(kNumClasses <= 64, "class sets are 64-bit masks");
// Family of a class: 0 grouped carry-save, 1 ScanCount, 2 position-major,
// 3 split inputs, 4 Looped, 5 staged carry-save.
constexpr int kNumFamilies = 6;
inline int class_family(int c) {
    return c < kNumWidths
               ? 0
               : (c <= kClassScanCount16
                      ? 1
                      : (c < kClassSplit ? 2
                                         : (c < kClassLooped ? 3 : (c < kClassStaged ? 4 : 5))));
}
// Counter-width index of a carry-save class (levels - 1 for Looped).
inline int class_width(int c) {
    return c < kNumWidths
               ? c
               : (c <= kClassScanCount16
                      ? c - kClassScanCount
                      : (c < kClassSplit
                             ? c - kClassPos
                             : (c < kClassLooped ? c - kClassSplit
                                                 : (c < kClassStaged ? c - kClassLooped
                                                                     : c - kClassStaged))));
}

// One pass-A launch: the slots list[list_off .. list_off + nlist) of its
// chunk, work items in `order` (0 query-major, 1 subtile-major), `grid` CTAs.
struct Launch {
    int cls;
    uint32_t list_off;
    uint32_t nlist;
    uint32_t order;
    int grid;
    uint32_t dynamic;  // 1: warps take items from a counter, 0: static striding
};

// A chunk: queries q0 .. q0 + Q - 1 of the batch in slots 0 .. Q - 1, pass-A
// launches launches[l0 .. l1).
struct ChunkPlan {
    uint32_t q0, Q;
    uint32_t l0, l1;
};

// Byte offsets of the scratch regions for chunks of at most Q slots and
// nlaunch pass-A launches in all.
struct ScratchLayout {
    size_t gtick, base, err, chk, work, tick, res, full, bagg, bpref, aggs, pref, U, total;
};
// After a batch the host reads back, with one copy from base to the end of
// res, the running output total (base), the kernels' error word (err), the
// check record (chk) and every query's {offset, length} (res).
ScratchLayout scratch_layout(uint64_t Q, uint64_t nq, uint32_t W, uint32_t NG,
                             uint64_t nlaunch);
// Scratch bytes per slot (everything that grows with Q).
uint64_t scratch_per_slot(uint32_t W, uint32_t NG);
uint32_t scan_blocks(uint32_t NG);

// Device pointers of one execution.
struct ExecBufs {
    const QDesc* qd;        // nq descriptors
    const uint32_t* ids;    // every id
    const uint32_t* lists;  // slot lists of all launches
    const uint2* grp;       // nq: {first, count} of each query's group in memb
    const uint32_t* memb;   // group member slots
    unsigned char* scratch; // ScratchLayout of the largest chunk
    ScratchLayout lay;
    uint64_t* out;          // output pool
    uint64_t cap;
    uint32_t nids = 0, nq = 0, nmemb = 0;  // sizes of ids, qd and memb (checked builds)
};

// Times of the pass-A launches (THR_PROFILE): an event pair per chunk.
struct PassATimer {
    cudaEvent_t* ev;  // 2 per chunk, or null
};

// Enqueue the whole plan on st: clear the control words, then per chunk its
// pass-A launches (forked onto the aux streams when there are several),
// pass B and pass C.  Results: res (offset, length per query) and base
// (total words) in scratch.  aux: naux streams for the forks (may be 0).
// zeroed: the caller's copy of the plan already zeroed the control words
// (the ScratchLayout up to `full`), so no memset is enqueued.
cudaError_t enqueue_plan(const thr_index* idx, const ChunkPlan* chunks, uint32_t nchunks,
                         const Launch* launches, const ExecBufs& b, cudaStream_t st,
                         cudaStream_t* aux, int naux, cudaEvent_t* fork_ev, int nfork_ev,
                         const PassATimer* timer, bool zeroed = false);

// Counting variants a query can run with (the selector's choices):
//   kVarCsa        carry-save bit slices, inputs decoded in groups of four;
//                  zeros of the active inputs are counted instead of ones
//                  when that needs fewer slices
//   kVarPos        carry-save bit slices counting ones; mixed inputs decoded
//                  position-major (cost follows their literals)
//   kVarScanCount  ScanCount counters (bytes for n <= 255, 16 bits for
//                  n <= 65535; else kVarCsa runs)
//   kVarSplit      grouped carry-save with each subtile's inputs split among
//                  the four warps of a CTA (S <= 8; else kVarCsa runs)
constexpr int kVarCsa = 0, kVarPos = 1, kVarScanCount = 2, kVarSplit = 3;
constexpr int kNumVariants = 4;  // the policies' choices
//   kVarLooped     Looped levels (Sec. 6.2) for 1 <= T <= kLoopedMax, T <= n
//                  (else kVarCsa runs); chosen by flag only
//   kVarStaged     kVarCsa with each input's words copied to shared memory
//                  by bulk copies ahead of the adds; chosen by flag only
constexpr int kVarLooped = 4;
constexpr int kVarStaged = 5;
// Kernel class and zero counting of a query run with variant v.
void resolve_variant(uint32_t n, uint32_t T, int v, int* cls, uint32_t* zmode);

// Counter width and zero counting for a query of n inputs and threshold T:
// counting ones needs 2^S >= T, counting the zeros of the active inputs
// 2^S >= n - T + 1 (a threshold of exactly 2^S is the sticky slice); the
// class is the first instantiated width that fits.
int slices_for(uint64_t t);  // the fewest S >= 1 with 2^S >= t
void choose_class(uint32_t n, uint32_t T, int* cls, uint32_t* zmode);

// THR_TEST_LOST_COPY=1 in the environment (tests only): every staged slot
// waits for 16 bytes that are never sent, so the kernel's bounded wait runs
// out and the call returns THR_E_TIMEOUT.
uint32_t test_lost_copy();

// CTAs per SM of a class's kernel at full occupancy.
cudaError_t class_occupancy(int cls, int* per_sm);

// THR_E_CHECK with the failed check of a checked build (site, index, limit,
// thread and block) as the message.
thr_status check_failed(const CheckRec& c);

}  // namespace thr
