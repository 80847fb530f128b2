/*
 * thr.h -- C ABI of libthr, a GPU (sm_103a) implementation of the threshold
 * (T-overlap) query over run-length-compressed bitmaps described by Kaser &
 * Lemire, "Compressed bitmap indexes: beyond unions and intersections"
 * (arXiv 1402.4466).
 *
 * The query (Sec. 2, "Formulation"): given N bitmaps over the rows [0, r) and
 * a threshold T, return the rows that are set in at least T of the N inputs.
 * T = 1 is a union and T = N an intersection; a bitmap listed twice counts
 * twice; T = 0 returns every row and T > N returns no row.
 *
 * Stream format.  Every bitmap and every result is a stream of 64-bit words
 * in a word-aligned run-length format in the style of EWAH (Sec. 3.1,
 * "Compressed Bitmaps": marker words carry the length of a run of fill words
 * and the number of dirty words that follow; 64-bit EWAH uses a 32-bit fill
 * counter).  The paper defers the exact layout to earlier work; this library
 * fixes it as:
 *   marker word   bit 0       fill bit b (fill words are 0 or ~0)
 *                 bits 1..32  F, number of fill words
 *                 bits 33..63 L, number of literal ("dirty") words after it
 *   stream        [marker, L literals] groups covering exactly
 *                 W = ceil(r/64) uncompressed words; uncompressed word i holds
 *                 rows 64i..64i+63, least-significant bit = smallest row.
 *   canonical     (i) no literal equals 0 or ~0; (ii) fill runs are maximal;
 *                 (iii) a marker starts only where a fill follows a literal,
 *                 the fill value changes, or a counter overflows; (iv) F = 0
 *                 implies b = 0; (v) bits >= r of the last word are 0, so a
 *                 ragged last word whose valid bits are all 1 is a literal;
 *                 (vi) F = 0 only in the first marker or after a marker whose
 *                 literal count overflowed.  Hence a stream has at most W + 1
 *                 words.  Inputs must be canonical; outputs always are.
 *
 * Limits: 1 <= r and W = ceil(r/64) <= 2^31 - 2 (so no counter overflows and
 * word indices fit 31 bits); 1 <= n <= THR_MAX_IDS = 2^20 - 1 bitmap ids per
 * query (a million inputs: the per-row counts then need at most 20 bits);
 * opt-threshold queries take at most 65535.
 *
 * Errors: every call returns a thr_status; no C++ exception crosses the ABI.
 * thr_last_error() describes the last failure of the calling thread.
 * A CUDA failure returns THR_E_CUDA.  No kernel of the library waits on
 * another CTA or launch (cross-CTA scans finish in the last CTA to arrive).
 * The one device-side wait is a warp's wait for its own bulk copies into
 * shared memory (THR_VARIANT_STAGED); it gives up after about a second, and the
 * call then returns THR_E_TIMEOUT (the results are not valid).
 *
 * Checked build: the same library compiled with THR_CHECKED defined
 * (libthr_checked.so; the Python binding loads it when THR_CHECKED=1 is in
 * the environment) compares every index-derived global access of the query
 * kernels of thr_query, thr_query_sym, thr_query_batch, thr_query_static and
 * the server with the size of what it addresses, skips a failing access and
 * returns THR_E_CHECK naming the first one.  The opt-threshold profiling
 * pass and the staged variant's copies are not checked.  Same ABI and
 * results otherwise.
 */
#ifndef THR_H
#define THR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct thr_index thr_index; /* opaque; owns all device memory */

#define THR_MAX_IDS 1048575u /* bitmap ids (with repeats) per query: 2^20 - 1 */

typedef enum {
    THR_OK = 0,
    THR_E_INVAL = 1,   /* bad argument (null pointer, id out of range, n = 0) */
    THR_E_FORMAT = 2,  /* an input stream is not canonical for r rows */
    THR_E_NOMEM = 3,   /* host or device allocation failed */
    THR_E_NOSPACE = 4, /* output buffer too small; required size returned */
    THR_E_CUDA = 5,    /* a CUDA runtime call failed */
    THR_E_TIMEOUT = 6, /* a kernel gave up waiting for its shared-memory copies */
    THR_E_CHECK = 7    /* checked build only: an index out of range (access skipped) */
} thr_status;

/* flags for thr_query / thr_query_batch */
#define THR_OUT_DEVICE 0x1u     /* out / pool are device pointers */
#define THR_POLICY_PLAIN 0x00u  /* batch: one launch per query, fixed variant */
#define THR_POLICY_RULE 0x10u   /* batch: rule-based variant choice */
#define THR_POLICY_LEARNED 0x20u /* batch: learned cost-model choice */
#define THR_POLICY_MASK 0xF0u
#define THR_PROFILE 0x100u      /* time the query kernel with CUDA events */
#define THR_NO_GRAPH 0x1000u    /* batch: launch directly, no CUDA graph */
#define THR_NO_SHARE 0x2000u    /* batch: no shared counting pass for queries
                                   over the same id multiset */
/* Counting kernel of a query (thr_query; thr_query_batch with
 * THR_POLICY_PLAIN uses it for every query):
 *   THR_VARIANT_CSA        carry-save bit-sliced counters in registers
 *                          (default; any n and T), inputs decoded four at a
 *                          time; when T is close to n the zeros of the
 *                          active inputs are counted instead, which needs
 *                          fewer counter bits
 *   THR_VARIANT_POSITION   the same counters counting ones; inputs that mix
 *                          fills and literals inside a 128-word subtile are
 *                          decoded position by position (each lane walks the
 *                          inputs with a literal at its word), so their cost
 *                          follows their literals: for sparse inputs
 *   THR_VARIANT_SCANCOUNT  ScanCount: one counter per row in shared memory
 *                          per subtile (Sec. 5.1), bytes for n <= 255 and
 *                          16 bits for n <= 65535 (else CSA runs); only the
 *                          bit positions some input set are compared, so the
 *                          cost follows the set bits: for very sparse inputs
 *   THR_VARIANT_SPLIT      THR_VARIANT_CSA with each subtile's inputs split
 *                          among the four warps of a CTA, whose counters are
 *                          then added: more parallelism for queries with
 *                          few subtiles (small r) and many inputs; used when
 *                          the counters need at most 8 bits, else CSA runs
 *   THR_VARIANT_LOOPED     Looped (Sec. 6.2, Algorithm 3): T bitmaps C_1..C_T
 *                          per word, C_j = rows counted at least j times so
 *                          far, each input one AND-OR per level; used when
 *                          1 <= T <= 4 and T <= n, else CSA runs.  Not an arm
 *                          of the rule or learned policies.
 *   THR_VARIANT_STAGED     THR_VARIANT_CSA with each input's compressed words
 *                          for a 128-word subtile first copied to shared
 *                          memory by bulk copies, the next inputs' copies in
 *                          flight while the current ones are added (not a
 *                          policy arm) */
#define THR_VARIANT_CSA 0x000u
#define THR_VARIANT_SCANCOUNT 0x200u
#define THR_VARIANT_POSITION 0x400u
#define THR_VARIANT_SPLIT 0x600u
#define THR_VARIANT_LOOPED 0x800u
#define THR_VARIANT_STAGED 0xA00u
#define THR_VARIANT_MASK 0xE00u

/*
 * Build a device-resident index from canonical streams (Sec. 3.1 format
 * above; Sec. 2: the N sets share the universe [0, r)).
 *   words     host array: all streams concatenated
 *   offsets   host array of nbitmaps + 1 word offsets; stream i is
 *             words[offsets[i] .. offsets[i+1])
 *   nbitmaps  >= 1
 *   r         number of rows of every bitmap
 *   cuda_stream  cudaStream_t used for the uploads and build kernels (0 ok)
 *   out       receives the new index on THR_OK, untouched otherwise
 * The input is copied; the caller keeps ownership of words and offsets.
 * Every stream is validated on the host: one that is not canonical for r
 * rows returns THR_E_FORMAT.  The index lives on the device that is current
 * at the call; queries must run with that device current.  Returns after the
 * build work on cuda_stream has completed.
 */
thr_status idx_build_rle(const uint64_t *words, const uint64_t *offsets,
                         uint32_t nbitmaps, uint64_t r, void *cuda_stream,
                         thr_index **out);

/*
 * Threshold query (Sec. 2): the rows set in at least T of the bitmaps
 * ids[0..n), encoded canonically.
 *   idx       index from idx_build_rle
 *   ids       host array of n bitmap ids (< nbitmaps; duplicates count with
 *             multiplicity)
 *   n         1 <= n <= THR_MAX_IDS
 *   T         any value; 0 gives every row, > n gives none
 *   out       caller-owned buffer of cap words: host memory, or device memory
 *             of the index's GPU (or managed memory) when flags has
 *             THR_OUT_DEVICE; device memory of another GPU is THR_E_INVAL
 *   cap       capacity of out in words; cap >= ceil(r/64) + 1 always suffices
 *   out_len   receives the encoded length in words.  When it exceeds cap the
 *             call returns THR_E_NOSPACE and the contents of out are
 *             unspecified (at most cap words are written).
 *   flags     THR_OUT_DEVICE or 0
 *   cuda_stream  cudaStream_t for all work (0 ok)
 * On return the result and *out_len are complete (the call synchronises
 * cuda_stream).  Concurrent queries on one index are allowed.  The work is
 * captured as a CUDA graph kept per calling thread; a later query of the
 * same shape (input count within the same 64, variant, counter width,
 * output buffer) on that thread replays it (not with THR_PROFILE).
 */
thr_status thr_query(const thr_index *idx, const uint32_t *ids, uint32_t n,
                     uint32_t T, uint64_t *out, uint64_t cap,
                     uint64_t *out_len, uint32_t flags, void *cuda_stream);

/*
 * Symmetric-function query: the rows whose count c over the bitmaps
 * ids[0..n) (duplicates counted with multiplicity) satisfies lo <= c <= hi,
 * or, with THR_SYM_ODD in flags, whose c is odd (the XOR of the inputs; lo
 * and hi are then ignored).  The threshold query is the range [T, n]; "at
 * most T" is [0, T] and "exactly k" is [k, k].  Threshold functions are the
 * symmetric Boolean functions the paper studies (Sec. 3.3); these are the
 * other symmetric functions of the same counts.  The carry-save counters
 * of thr_query are reused; only the final compare and the pruning differ
 * (a subtile is zero when [k, k + d] misses [lo, hi] and ones when it lies
 * inside).  Other arguments, output and errors as thr_query.
 */
#define THR_SYM_ODD 0x4000u
thr_status thr_query_sym(const thr_index *idx, const uint32_t *ids, uint32_t n, uint32_t lo,
                         uint32_t hi, uint64_t *out, uint64_t cap, uint64_t *out_len,
                         uint32_t flags, void *cuda_stream);

/*
 * Opt-threshold query (Sec. 3.3, last paragraph; Sec. 5.1 and Sec. 6.2 give
 * it for ScanCount and Looped): T is not given.  *T_out receives
 *   T* = the largest T in 0..n whose T-overlap result over ids[0..n) holds
 *        at least K rows (K = 1: the largest count any row reaches),
 *        or 0 when no T does (only when K > r: the T = 0 result is every row),
 * and out receives that result, as thr_query(ids, n, T*) would write it (for
 * K = 1 exactly the rows whose count is T*).  The generalisation to K rows
 * is the one Sec. 3.3 suggests; ties at T* are all kept (it is not a top-K
 * list).  Two passes on cuda_stream: a profiling pass of the carry-save
 * counters (a histogram of the counts at or above a rising lower bound on
 * T*, skipping subtiles that cannot reach it), a device->host read of the
 * histogram, then the threshold query at T*.
 *   K      >= 1 (THR_E_INVAL otherwise)
 *   n      1..65535
 *   flags  THR_OUT_DEVICE, THR_PROFILE (thr_last_kernel_ms then returns the
 *          profiling pass's time), one THR_VARIANT_* value for the second pass
 * Other arguments, output and errors as thr_query; *T_out is set whenever
 * the profiling pass ran, also when the result does not fit (THR_E_NOSPACE).
 */
thr_status thr_query_opt(const thr_index *idx, const uint32_t *ids, uint32_t n, uint64_t K,
                         uint32_t *T_out, uint64_t *out, uint64_t cap, uint64_t *out_len,
                         uint32_t flags, void *cuda_stream);

/*
 * The profiling pass of thr_query_opt alone, for callers that combine
 * partial answers, such as the row shards of an index split by rows (Sec. 9
 * asks about partitioning the problem): *T_out receives this index's answer
 * T* for K (as thr_query_opt; 0 when no T qualifies) and hist[c], c = 0..n,
 * the number of rows whose count over ids is exactly c, exact for every
 * c >= max(*T_out, 1); bins below may be incomplete and hist[0] is 0 (not
 * computed).  Over shards g with answers T_g, the answer of the whole is at
 * least max_g T_g, and every shard's bins are exact from there up, so the
 * whole's answer is the first c from n down to max(max_g T_g, 1) whose
 * summed suffix hist[c] + .. + hist[n] reaches K (0 if none does).
 *   n      1..65535;  K >= 1;  hist: host array of n + 1 words
 * Synchronous on cuda_stream; errors as thr_query.
 */
thr_status thr_query_opt_hist(const thr_index *idx, const uint32_t *ids, uint32_t n,
                              uint64_t K, uint32_t *T_out, uint64_t *hist,
                              void *cuda_stream);

/*
 * nq opt-threshold queries (as thr_query_opt) in one profiling launch per
 * counter width and one thr_query_batch: K and T_out have nq entries; the
 * other arguments, flags and output as thr_query_batch.  Results equal nq
 * calls of thr_query_opt.
 */
thr_status thr_query_opt_batch(const thr_index *idx, uint32_t nq, const uint32_t *id_off,
                               const uint32_t *ids, const uint64_t *K, uint32_t *T_out,
                               uint64_t *pool, uint64_t pool_cap, uint64_t *out_off,
                               uint64_t *out_len, uint32_t flags, void *cuda_stream);

/*
 * Batch of nq threshold queries (Sec. 2) over one index.
 *   id_off    host array of nq + 1 offsets into ids; query q uses
 *             ids[id_off[q] .. id_off[q+1])
 *   ids, T    host arrays (T has nq entries)
 *   pool      caller-owned output pool of pool_cap words (host, or device
 *             with THR_OUT_DEVICE); query q's result is stored at
 *             pool[out_off[q] .. out_off[q] + out_len[q])
 *   out_off, out_len  host arrays of nq entries, filled on return
 *   flags     THR_OUT_DEVICE | one THR_POLICY_* value (RULE and LEARNED
 *             choose a counting variant per query, except that queries
 *             over the same id multiset keep THR_VARIANT_CSA, whose one
 *             counting pass they share, unless THR_NO_SHARE is given)
 * pool_cap >= nq * (ceil(r/64) + 1) never yields THR_E_NOSPACE; a smaller
 * pool works when the results fit, else THR_E_NOSPACE with out_len holding
 * every query's length.  Results are identical to nq calls of thr_query.
 */
thr_status thr_query_batch(const thr_index *idx, uint32_t nq,
                           const uint32_t *id_off, const uint32_t *ids,
                           const uint32_t *T, uint64_t *pool,
                           uint64_t pool_cap, uint64_t *out_off,
                           uint64_t *out_len, uint32_t flags,
                           void *cuda_stream);

/*
 * The same query as thr_query, for callers that cannot allocate device
 * memory while they answer it (the paper has no counterpart: this is a
 * property of the library).  Examples: a process whose GPU memory is owned
 * by another allocator that reserved the device up front, or code that must
 * not risk an allocation failure, or the device synchronisation an
 * allocation or free can cause, in the middle of its work.  Every scratch
 * buffer the kernels need lives in one fixed device array of about 9.25 MiB
 * inside the library, which each GPU that loads the library holds until the
 * process exits; the call allocates nothing (no cudaMalloc, stream-ordered
 * or pinned allocation).
 *   out       device memory of the index's GPU (or managed memory) only, cap
 *             words; the other arguments and the
 *             result are as for thr_query with THR_OUT_DEVICE
 * Limits: ceil(r/64) <= 2^20 words (r <= 2^26 rows) and n <= 65536;
 * larger queries return THR_E_INVAL.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress, with that device
 * current); make that first call before any stream capture.  Every call
 * reuses the same array, so calls whose work overlaps on the GPU (other
 * streams or host threads) race on it: do not let two such calls run at
 * the same time.  Synchronous like thr_query.
 */
thr_status thr_query_static(const thr_index *idx, const uint32_t *ids, uint32_t n,
                            uint32_t T, uint64_t *out, uint64_t cap,
                            uint64_t *out_len, void *cuda_stream);

/*
 * Serving loop with continuous batching over a resident index.  Requests
 * (thr_server_submit copies ids) wait in one queue; each of `workers` host
 * threads owns a CUDA stream and, when free, takes the oldest waiting
 * requests as one micro-batch: at most max_batch of them, and only as many
 * as fit mem_budget bytes together with the batches already in flight (a
 * request claims the scratch of one query slot plus 8 (ceil(r/64) + 1)
 * bytes for its result; a batch with nothing else in flight always admits
 * its first request).  The micro-batch runs as thr_query_batch would (CUDA
 * graph replay; flags: one THR_POLICY_* and THR_VARIANT_* value), so batches
 * of different workers overlap on the device.  thr_server_wait blocks until
 * the request is done, copies its result (THR_E_NOSPACE if cap is too
 * small, *out_len = its length), gives the time from submit to completion
 * and releases the ticket.  Results equal thr_query's for the same query.
 * Submitting and waiting may go on at the same time from different host
 * threads; a ticket is waited for once (a second concurrent wait on the
 * same ticket returns THR_E_INVAL).
 * thr_server_stats fills 8 counters: queries done, micro-batches run,
 * queries in them, most batches in flight at once, largest batch, most
 * budget bytes claimed at once, requests waiting, batches in flight now.
 * thr_server_free finishes every waiting request, then stops the workers;
 * the index must outlive the server.
 */
typedef struct thr_server thr_server;
thr_status thr_server_create(const thr_index *idx, uint32_t workers, uint32_t max_batch,
                             uint64_t mem_budget, uint32_t flags, thr_server **out);
thr_status thr_server_submit(thr_server *srv, const uint32_t *ids, uint32_t n, uint32_t T,
                             uint64_t *ticket);
thr_status thr_server_wait(thr_server *srv, uint64_t ticket, uint64_t *out, uint64_t cap,
                           uint64_t *out_len, double *latency_ms);
thr_status thr_server_stats(thr_server *srv, uint64_t *stats);
void thr_server_free(thr_server *srv);

/* Release an index (NULL-safe); waits for in-flight work on its device. */
void idx_free(thr_index *idx);

/* Number of bitmaps, rows and total stored words of an index. */
thr_status idx_info(const thr_index *idx, uint32_t *nbitmaps, uint64_t *r,
                    uint64_t *total_words);

/*
 * Host codec.  thr_rle_encode writes the canonical stream of the
 * uncompressed bitmap words[0..nwords) (nwords = ceil(r/64), bits >= r must
 * be 0) into out (cap words), *out_len = its length (THR_E_NOSPACE if it
 * exceeds cap).  thr_rle_validate returns THR_OK for a canonical stream of an
 * r-row bitmap and THR_E_FORMAT otherwise.  Both are host-only.
 */
thr_status thr_rle_encode(const uint64_t *words, uint64_t nwords, uint64_t r,
                          uint64_t *out, uint64_t cap, uint64_t *out_len);
thr_status thr_rle_validate(const uint64_t *stream, uint64_t len, uint64_t r);
/*
 * Row-range sharding (host).  thr_rle_slice writes the canonical stream of
 * the uncompressed words [w0, w1) (rows 64 w0 .. 64 w1 - 1) of a canonical
 * stream of an r-row bitmap: a shard of the rows.  thr_rle_stitch writes the
 * canonical stream of the concatenation of nparts streams of consecutive
 * row ranges (part k covers rows[k] rows, a multiple of 64 except for the
 * last part): a fill that continues a fill of the same value across a seam
 * and literals that follow literals merge into one group, so the threshold
 * results of the shards of a row-sharded index stitch into the result of the
 * whole.  Both validate their inputs (THR_E_FORMAT) and return
 * THR_E_NOSPACE with the needed length when cap is too small.
 */
thr_status thr_rle_slice(const uint64_t *stream, uint64_t len, uint64_t r, uint64_t w0,
                         uint64_t w1, uint64_t *out, uint64_t cap, uint64_t *out_len);
thr_status thr_rle_stitch(const uint64_t *const *parts, const uint64_t *lens,
                          const uint64_t *rows, uint32_t nparts, uint64_t *out,
                          uint64_t cap, uint64_t *out_len);
/* The canonical stream of the r-row bitmap whose set rows are
 * rows[0..nrows) (ascending, repeats allowed, each < r), written like
 * thr_rle_encode but without forming the uncompressed words.  Host-only. */
thr_status thr_rle_encode_rows(const uint64_t *rows, uint64_t nrows, uint64_t r,
                               uint64_t *out, uint64_t cap, uint64_t *out_len);

/*
 * Device time in milliseconds of the counting kernels (pass A) of the last
 * call on this thread that passed THR_PROFILE (thr_query, thr_query_sym,
 * thr_query_batch: CUDA events recorded right before and after the pass-A
 * launches of each chunk, summed; thr_query_opt and thr_query_opt_batch: the
 * profiling pass); -1 if none.
 */
double thr_last_kernel_ms(void);

/*
 * Autotuner of the batched launch.  Runs the sample batch (arguments as for
 * thr_query_batch; flags: a THR_POLICY_* and THR_VARIANT_* value, and
 * THR_NO_SHARE to tune batches that run without shared counting) under
 * each of the 16 launch configurations of pass A, reps times each after one
 * warm-up run, with L2 flushed before every run, and keeps the fastest for
 * the batch's shape (several kernel classes or one; mean inputs per query)
 * in the index: later thr_query and thr_query_batch calls of that shape use
 * it.  A configuration is 4 bits: 1 subtile-major work order (queries that
 * share inputs read them at about the same time; else query-major), 2 merge
 * the counter widths of a chunk into one launch, 4 split the SMs among
 * launches that run side by side in proportion to their work, 8 warps take
 * work items from a counter as they finish (else static striding).
 *   times  optional, 16 entries: median host time in ms of each configuration
 *   best   optional: the configuration kept
 * Results are identical under every configuration; only the time differs.
 */
thr_status thr_autotune(const thr_index *idx, uint32_t nq, const uint32_t *id_off,
                        const uint32_t *ids, const uint32_t *T, uint32_t flags,
                        uint32_t reps, void *cuda_stream, double *times, uint32_t *best);

/*
 * Learned cost model of the variant selector (THR_POLICY_LEARNED).  The
 * paper predicts each algorithm's time with a fitted model and runs the one
 * predicted fastest (Sec. 8.1-8.2); here a multilayer perceptron
 * 16 -> 64 -> 64 -> 4 with ReLU predicts log(pass-A time) of the four
 * counting variants (0 THR_VARIANT_CSA, 1 THR_VARIANT_POSITION,
 * 2 THR_VARIANT_SCANCOUNT, 3 THR_VARIANT_SPLIT) from the 16 features of
 * thr_query_features,
 * normalised as (x - mean) * istd.  Weights are BF16 (FP32 with
 * THR_SEL_FP32) and every sum is accumulated in FP32; training is minibatch
 * Adam on the mean squared error over the (row, variant) pairs whose mask
 * byte is non-zero.  The learned policy runs the variant predicted fastest,
 * but leaves THR_VARIANT_CSA only for a predicted gain of at least 10%.  The forward, backward and update steps are CUDA kernels
 * of this library, on the device current at creation.
 * Parameters (THR_SEL_PARAMS floats): W1[16][64] b1[64] W2[64][64] b2[64]
 * W3[64][4] b3[4], y = W3^T relu(W2^T relu(W1^T x + b1) + b2) + b3.
 * X: rows x 16 floats, T (targets) and Y: rows x 4 floats, M: rows x 4
 * bytes; all host arrays.
 */
typedef struct thr_selector thr_selector;
#define THR_SEL_FEATURES 16
#define THR_SEL_VARIANTS 4
#define THR_SEL_PARAMS 5508
#define THR_SEL_FP32 0x1u
thr_status thr_selector_create(uint64_t seed, uint32_t flags, thr_selector **out);
void thr_selector_free(thr_selector *sel);
thr_status thr_selector_set_params(thr_selector *sel, const float *params);
thr_status thr_selector_get_params(const thr_selector *sel, float *params);
thr_status thr_selector_set_norm(thr_selector *sel, const float *mean, const float *istd);
thr_status thr_selector_train(thr_selector *sel, const float *X, const float *T,
                              const uint8_t *M, uint32_t rows, uint32_t epochs,
                              uint32_t batch, float lr, uint64_t seed, float *loss);
thr_status thr_selector_predict(const thr_selector *sel, const float *X, uint32_t rows,
                                float *Y);
/* Gradient of the loss over all rows (no update) and the loss itself. */
thr_status thr_selector_gradients(thr_selector *sel, const float *X, const float *T,
                                  const uint8_t *M, uint32_t rows, float *grad,
                                  float *loss);
/* Features of a query: log2 n, log2 (T + 1), log2 (n - T + 2) (0 if T > n),
 * log2 r, the quantiles 0, 1/4, 1/2, 3/4, 1 of log2 (compressed words + 1)
 * over the inputs and log2 of their total, the same quantiles of
 * log10 (density + 1e-7) and the sum of the densities. */
thr_status thr_query_features(const thr_index *idx, const uint32_t *ids, uint32_t n,
                              uint32_t T, float *features);
/* Attach a cost model to an index (NULL detaches); THR_POLICY_LEARNED then
 * uses it.  The selector must outlive its use by the index. */
thr_status thr_index_set_selector(thr_index *idx, const thr_selector *sel);

/*
 * The counting variant (0 THR_VARIANT_CSA, 1 THR_VARIANT_POSITION,
 * 2 THR_VARIANT_SCANCOUNT, 3 THR_VARIANT_SPLIT, 4 THR_VARIANT_LOOPED,
 * 5 THR_VARIANT_STAGED) each query of a batch runs with under the policy in
 * flags (arguments as for thr_query_batch), after the fallbacks (ScanCount
 * above 65535 inputs, split above 8 counter bits and Looped above T = 4
 * run the grouped carry-save kernel); nothing is run.
 */
thr_status thr_select_variants(const thr_index *idx, uint32_t nq, const uint32_t *id_off,
                               const uint32_t *ids, const uint32_t *T, uint32_t flags,
                               uint8_t *variant);

/*
 * Coefficients of the rule chooser (THR_POLICY_RULE, and THR_POLICY_LEARNED
 * without a cost model): linear time models in the manner of Sec. 8.1, one
 * per counting variant, the smallest prediction wins (Sec. 8.2):
 *   THR_VARIANT_CSA        c[0] + c[1] * words + c[2] * words * S
 *   THR_VARIANT_POSITION   c[3] + c[4] * words + c[5] * words * S1
 *   THR_VARIANT_SCANCOUNT  c[6] + c[7] * words + c[8] * set bits
 *   THR_VARIANT_SPLIT      c[9] + c[10] * words + c[11] * words * S
 * (words: compressed words of the inputs; S: counter bits of the grouped
 * kernel, S1: counter bits counting ones; set bits: of the inputs), refit
 * by least squares on measured times.  set (12 values) is applied when
 * non-NULL, then the current values go to get when non-NULL.
 */
thr_status thr_rule_model(const double *set, double *get);

/*
 * Shape of the last thr_query_batch call on this thread: chunks (groups of
 * queries whose scratch fits, run one after another), pass-A launches, and
 * graph = 1 if a cached CUDA graph of the same shape was updated and
 * replayed, 0 if a new graph was instantiated, -1 if none was used, and the
 * launch configuration of its first chunk (see thr_autotune).  Any pointer
 * may be NULL.
 */
thr_status thr_last_batch_info(uint32_t *chunks, uint32_t *launches, int32_t *graph,
                               uint32_t *config);

/*
 * Diagnostics read from the environment at first use: THR_TRACE=1 prints a
 * stderr line per step of a query; THR_TRACE_TIME=1 prints, per batch call,
 * the host time of planning, staging, launch and the wait for the device.
 * Testing only: THR_TUNE_CONFIG=k forces pass-A launch configuration k and
 * THR_MAX_SLOTS=m caps the queries per chunk.
 */

/* Message for the last failed call on this thread ("" if none). */
const char *thr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* THR_H */
