/*
 * oracle.c -- plain, slow, obviously correct CPU reference for the threshold
 * (T-overlap) query over word-aligned run-length-compressed bitmaps
 * (Kaser & Lemire, "Compressed bitmap indexes: beyond unions and
 * intersections", arXiv 1402.4466).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  The GPU library never links,
 * includes or calls it, and it shares no code with it.
 *
 * What it computes (Sec. 2, "Formulation"): given N bitmaps over the rows
 * [0, r) and a threshold T, the rows set in at least T of the N inputs.  A
 * bitmap id listed twice in a query counts twice.  T = 0 selects every row and
 * T > N selects none; both follow from the definition.
 *
 * How (ScanCount, Sec. 5.1): decode every input stream into its sorted list of
 * set rows (iterating the 1s of a literal word with a trailing-zero loop, as
 * Sec. 3.1 describes), keep one counter per row, increment the counter of
 * every listed row, and keep the rows whose counter reaches T.  The result
 * rows are packed into 64-bit words, least-significant bit = smallest row
 * (Sec. 3.1, "Uncompressed Bitmaps"), and encoded in the canonical form below.
 *
 * Stream format (Sec. 3.1, "Compressed Bitmaps": fill words, dirty words and
 * marker words that carry both the length of a fill run and the number of
 * dirty words after it; 64-bit EWAH keeps a 32-bit fill counter).  The paper
 * defers the exact layout to earlier work, so this project fixes it:
 *   marker word  bit 0      fill bit b (value of the fill words: 0 or ~0)
 *                bits 1..32 F, the number of fill words        (< 2^32)
 *                bits 33..63 L, the number of literal words that follow (< 2^31)
 *   A stream is a sequence of [marker, L literal words] groups that covers
 *   exactly W = ceil(r/64) uncompressed words.  Canonical form:
 *   (i)   a literal is never 0 or ~0;
 *   (ii)  fill runs are maximal (split only when F would overflow);
 *   (iii) a new marker starts only where a fill follows a literal, where the
 *         fill value changes, or where a counter overflows;
 *   (iv)  F = 0 implies b = 0;
 *   (v)   bits >= r of the last word are 0, so a ragged last word whose valid
 *         bits are all 1 is a literal, never a fill of ones;
 *   (vi)  F = 0 appears only in the first marker or after a marker whose
 *         literal count overflowed;
 *   a marker with F = 0 and L = 0 exists only for r = 0 (the stream [0]).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_E_INVAL 1
#define ORC_E_FORMAT 2
#define ORC_E_NOMEM 3
#define ORC_E_NOSPACE 4

#define ORC_FMAX 0xFFFFFFFFull /* 32-bit fill counter */
#define ORC_LMAX 0x7FFFFFFFull /* 31-bit literal counter */

static uint64_t orc_nwords(uint64_t r) { return (r + 63) / 64; }

static uint64_t orc_marker(uint64_t b, uint64_t F, uint64_t L)
{
    return (b & 1) | (F << 1) | (L << 33);
}

/* Trailing-zero count of a non-zero word, written as a plain loop. */
static int orc_ctz(uint64_t v)
{
    int t = 0;
    while (!(v & 1)) {
        v >>= 1;
        t++;
    }
    return t;
}

static int orc_is_fill(uint64_t v) { return v == 0 || v == ~0ull; }

/*
 * Canonical encoder (format above).  words holds W = ceil(r/64) words with
 * bits >= r cleared.  Writes at most cap words to out; *out_len receives the
 * encoded length even when it exceeds cap (then ORC_E_NOSPACE).
 */
int orc_encode(const uint64_t *words, uint64_t nwords, uint64_t r,
               uint64_t *out, uint64_t cap, uint64_t *out_len)
{
    uint64_t W = orc_nwords(r), i = 0, n = 0;
    if (nwords != W || out_len == NULL || (words == NULL && W > 0))
        return ORC_E_INVAL;
    if (W > 0 && (r % 64) != 0 && (words[W - 1] >> (r % 64)) != 0)
        return ORC_E_INVAL; /* rule (v): bits past r must be zero */
    if (W == 0) {
        if (cap >= 1 && out) out[0] = 0;
        *out_len = 1;
        return cap >= 1 ? ORC_OK : ORC_E_NOSPACE;
    }
    while (i < W) {
        uint64_t b = 0, F = 0, L = 0, lit0;
        if (orc_is_fill(words[i])) {
            uint64_t v = words[i];
            b = (v == ~0ull);
            while (i < W && words[i] == v && F < ORC_FMAX) {
                F++;
                i++;
            }
        }
        lit0 = i;
        while (i < W && !orc_is_fill(words[i]) && L < ORC_LMAX) {
            L++;
            i++;
        }
        if (n < cap && out) out[n] = orc_marker(b, F, L);
        n++;
        for (uint64_t k = 0; k < L; k++) {
            if (n < cap && out) out[n] = words[lit0 + k];
            n++;
        }
    }
    *out_len = n;
    return n <= cap ? ORC_OK : ORC_E_NOSPACE;
}

/*
 * Decoder and validator.  Walks the markers of one stream (Sec. 3.1), checks
 * every canonical rule and, when rows != NULL, lists the set rows in
 * increasing order (fill runs of ones row by row; literal words with the
 * trailing-zero loop).  *nrows receives the number of set rows even when it
 * exceeds cap (then ORC_E_NOSPACE after a complete, valid walk).
 */
int orc_decode(const uint64_t *s, uint64_t len, uint64_t r,
               uint64_t *rows, uint64_t cap, uint64_t *nrows)
{
    uint64_t W = orc_nwords(r), covered = 0, i = 0, cnt = 0;
    uint64_t prevF = 0, prevL = 0, prevb = 0;
    int first = 1;
    if (s == NULL && len > 0) return ORC_E_INVAL;
    if (W == 0) {
        if (len != 1 || s[0] != 0) return ORC_E_FORMAT;
        if (nrows) *nrows = 0;
        return ORC_OK;
    }
    while (covered < W) {
        uint64_t mw, b, F, L;
        if (i >= len) return ORC_E_FORMAT; /* stream ends too early */
        mw = s[i++];
        b = mw & 1;
        F = (mw >> 1) & 0xFFFFFFFFull;
        L = mw >> 33;
        if (F == 0 && L == 0) return ORC_E_FORMAT; /* empty marker */
        if (F == 0 && b) return ORC_E_FORMAT;      /* rule (iv) */
        if (!first) {
            if (F == 0 && prevL != ORC_LMAX) return ORC_E_FORMAT; /* (vi) */
            if (F > 0 && prevL == 0 && prevb == b && prevF != ORC_FMAX)
                return ORC_E_FORMAT; /* (ii): fill run not maximal */
        }
        if (F > W - covered || L > W - covered - F) return ORC_E_FORMAT;
        if (b && (r % 64) != 0 && covered + F == W)
            return ORC_E_FORMAT; /* (v): ones fill over the ragged word */
        if (b) {
            for (uint64_t x = covered * 64; x < (covered + F) * 64; x++) {
                if (rows && cnt < cap) rows[cnt] = x;
                cnt++;
            }
        }
        covered += F;
        for (uint64_t k = 0; k < L; k++) {
            uint64_t v;
            if (i >= len) return ORC_E_FORMAT;
            v = s[i++];
            if (orc_is_fill(v)) return ORC_E_FORMAT; /* rule (i) */
            if (covered == W - 1 && (r % 64) != 0 && (v >> (r % 64)) != 0)
                return ORC_E_FORMAT; /* rule (v) */
            while (v) {
                uint64_t x = covered * 64 + (uint64_t)orc_ctz(v);
                if (rows && cnt < cap) rows[cnt] = x;
                cnt++;
                v &= v - 1;
            }
            covered++;
        }
        prevF = F;
        prevL = L;
        prevb = b;
        first = 0;
    }
    if (i != len) return ORC_E_FORMAT; /* words after the last group */
    if (nrows) *nrows = cnt;
    if (rows && cnt > cap) return ORC_E_NOSPACE;
    return ORC_OK;
}

/* Validation only: orc_decode without a row list. */
int orc_validate(const uint64_t *s, uint64_t len, uint64_t r)
{
    uint64_t nr = 0;
    return orc_decode(s, len, r, NULL, 0, &nr);
}

/*
 * Threshold query by ScanCount (Sec. 5.1).  streams: all bitmaps' streams
 * concatenated; offsets[nbitmaps + 1] delimit them (in words).  ids[0..n)
 * select the inputs (with multiplicity).  The canonical encoding of the
 * result is written to out (cap words); *out_len receives its length.
 */
int orc_threshold(const uint64_t *streams, const uint64_t *offsets,
                  uint32_t nbitmaps, uint64_t r, const uint32_t *ids,
                  uint32_t n, uint32_t T, uint64_t *out, uint64_t cap,
                  uint64_t *out_len)
{
    uint64_t W = orc_nwords(r);
    uint32_t *count = NULL; /* one counter per row */
    uint64_t *rows = NULL, *words = NULL;
    int rc = ORC_OK;
    if (out_len == NULL || (n > 0 && ids == NULL) || offsets == NULL)
        return ORC_E_INVAL;
    for (uint32_t q = 0; q < n; q++)
        if (ids[q] >= nbitmaps) return ORC_E_INVAL;
    count = (uint32_t *)calloc(r > 0 ? r : 1, sizeof(uint32_t));
    rows = (uint64_t *)malloc((r > 0 ? r : 1) * sizeof(uint64_t));
    words = (uint64_t *)calloc(W > 0 ? W : 1, sizeof(uint64_t));
    if (!count || !rows || !words) {
        rc = ORC_E_NOMEM;
        goto done;
    }
    /* one pass per input bitmap: decode it, increment the counters */
    for (uint32_t q = 0; q < n; q++) {
        uint64_t b = ids[q], nr = 0;
        rc = orc_decode(streams + offsets[b], offsets[b + 1] - offsets[b], r,
                        rows, r, &nr);
        if (rc != ORC_OK) goto done;
        for (uint64_t k = 0; k < nr; k++) count[rows[k]]++;
    }
    /* final pass over the counters: keep rows seen at least T times */
    for (uint64_t x = 0; x < r; x++)
        if (count[x] >= T) words[x / 64] |= 1ull << (x % 64);
    rc = orc_encode(words, W, r, out, cap, out_len);
done:
    free(count);
    free(rows);
    free(words);
    return rc;
}

/*
 * The same query, returning the uncompressed result words (W of them) instead
 * of the encoded stream; used to diagnose mismatches row by row.
 */
/* Symmetric functions of the counts (beyond thresholds, Sec. 3.3 and Sec. 5.3
 * discuss them as Boolean functions of the input bits that depend only on
 * how many are set): the rows whose count c over the multiset of ids
 * satisfies lo <= c <= hi, or, with odd != 0, whose c is odd (the XOR of the
 * inputs).  The same ScanCount as orc_threshold, a different final test. */
int orc_symmetric(const uint64_t *streams, const uint64_t *offsets,
                  uint32_t nbitmaps, uint64_t r, const uint32_t *ids,
                  uint32_t n, uint32_t lo, uint32_t hi, int odd, uint64_t *out,
                  uint64_t cap, uint64_t *out_len)
{
    uint64_t W = orc_nwords(r);
    uint32_t *count = NULL;
    uint64_t *rows = NULL, *words = NULL;
    int rc = ORC_OK;
    if (out_len == NULL || (n > 0 && ids == NULL) || offsets == NULL)
        return ORC_E_INVAL;
    for (uint32_t q = 0; q < n; q++)
        if (ids[q] >= nbitmaps) return ORC_E_INVAL;
    count = (uint32_t *)calloc(r > 0 ? r : 1, sizeof(uint32_t));
    rows = (uint64_t *)malloc((r > 0 ? r : 1) * sizeof(uint64_t));
    words = (uint64_t *)calloc(W > 0 ? W : 1, sizeof(uint64_t));
    if (!count || !rows || !words) {
        rc = ORC_E_NOMEM;
        goto done;
    }
    for (uint32_t q = 0; q < n; q++) {
        uint64_t b = ids[q], nr = 0;
        rc = orc_decode(streams + offsets[b], offsets[b + 1] - offsets[b], r,
                        rows, r, &nr);
        if (rc != ORC_OK) goto done;
        for (uint64_t k = 0; k < nr; k++) count[rows[k]]++;
    }
    for (uint64_t x = 0; x < r; x++) {
        const int keep = odd ? (int)(count[x] & 1u) : (count[x] >= lo && count[x] <= hi);
        if (keep) words[x / 64] |= 1ull << (x % 64);
    }
    rc = orc_encode(words, W, r, out, cap, out_len);
done:
    free(count);
    free(rows);
    free(words);
    return rc;
}

/* Opt-threshold query (Sec. 3.3, last paragraph; Sec. 5.1 derives it from
 * ScanCount): T is not given; the answer is the largest T in [0, n] whose
 * T-overlap result holds at least K rows (K = 1: the largest count any row
 * reaches), and that result.  ScanCount's counters as in orc_threshold,
 * then a histogram of the counts, whose suffix sums from n downwards give
 * |result_T| for every T; the first T (from the top) with a suffix of at
 * least K rows is the answer.  When no T qualifies (K > r) the answer is
 * T = 0, every row.  *T_out receives T. */
int orc_opt_threshold(const uint64_t *streams, const uint64_t *offsets,
                      uint32_t nbitmaps, uint64_t r, const uint32_t *ids,
                      uint32_t n, uint64_t K, uint32_t *T_out, uint64_t *out,
                      uint64_t cap, uint64_t *out_len)
{
    uint64_t W = orc_nwords(r);
    uint32_t *count = NULL;
    uint64_t *rows = NULL, *words = NULL, *hist = NULL;
    int rc = ORC_OK;
    if (out_len == NULL || T_out == NULL || (n > 0 && ids == NULL) || offsets == NULL || K == 0)
        return ORC_E_INVAL;
    for (uint32_t q = 0; q < n; q++)
        if (ids[q] >= nbitmaps) return ORC_E_INVAL;
    count = (uint32_t *)calloc(r > 0 ? r : 1, sizeof(uint32_t));
    rows = (uint64_t *)malloc((r > 0 ? r : 1) * sizeof(uint64_t));
    words = (uint64_t *)calloc(W > 0 ? W : 1, sizeof(uint64_t));
    hist = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    if (!count || !rows || !words || !hist) {
        rc = ORC_E_NOMEM;
        goto done;
    }
    for (uint32_t q = 0; q < n; q++) {
        uint64_t b = ids[q], nr = 0;
        rc = orc_decode(streams + offsets[b], offsets[b + 1] - offsets[b], r,
                        rows, r, &nr);
        if (rc != ORC_OK) goto done;
        for (uint64_t k = 0; k < nr; k++) count[rows[k]]++;
    }
    /* hist[c] = rows whose count is exactly c */
    for (uint64_t x = 0; x < r; x++) hist[count[x]]++;
    {
        uint32_t T = 0;
        uint64_t atleast = 0; /* rows whose count is >= c */
        for (uint32_t c = n; c >= 1; c--) {
            atleast += hist[c];
            if (atleast >= K) {
                T = c;
                break;
            }
        }
        *T_out = T;
        for (uint64_t x = 0; x < r; x++)
            if (count[x] >= T) words[x / 64] |= 1ull << (x % 64);
    }
    rc = orc_encode(words, W, r, out, cap, out_len);
done:
    free(count);
    free(rows);
    free(words);
    free(hist);
    return rc;
}

int orc_threshold_words(const uint64_t *streams, const uint64_t *offsets,
                        uint32_t nbitmaps, uint64_t r, const uint32_t *ids,
                        uint32_t n, uint32_t T, uint64_t *words)
{
    uint32_t *count = NULL;
    uint64_t *rows = NULL, W = orc_nwords(r);
    int rc = ORC_OK;
    if ((n > 0 && ids == NULL) || offsets == NULL || (words == NULL && W > 0))
        return ORC_E_INVAL;
    for (uint32_t q = 0; q < n; q++)
        if (ids[q] >= nbitmaps) return ORC_E_INVAL;
    count = (uint32_t *)calloc(r > 0 ? r : 1, sizeof(uint32_t));
    rows = (uint64_t *)malloc((r > 0 ? r : 1) * sizeof(uint64_t));
    if (!count || !rows) {
        rc = ORC_E_NOMEM;
        goto done;
    }
    for (uint32_t q = 0; q < n; q++) {
        uint64_t b = ids[q], nr = 0;
        rc = orc_decode(streams + offsets[b], offsets[b + 1] - offsets[b], r,
                        rows, r, &nr);
        if (rc != ORC_OK) goto done;
        for (uint64_t k = 0; k < nr; k++) count[rows[k]]++;
    }
    memset(words, 0, W * sizeof(uint64_t));
    for (uint64_t x = 0; x < r; x++)
        if (count[x] >= T) words[x / 64] |= 1ull << (x % 64);
done:
    free(count);
    free(rows);
    return rc;
}

/*
 * The same ScanCount partitioned by row range (the multi-core CPU baseline):
 * the W words are cut into `parts` contiguous word ranges; each range keeps
 * its own counters and walks every input stream, counting only the rows that
 * fall inside it (fill runs of ones row by row, literal words bit by bit with
 * the trailing-zero loop), then marks its rows whose count reaches T.  One
 * canonical encoding of all W words follows.  The ranges run on OpenMP
 * threads when the library was compiled with OpenMP (orc_max_threads() > 1),
 * else one after the other; the result does not depend on either.  Streams
 * are validated first (orc_validate), so the range walks trust the format.
 */
static void orc_count_range(const uint64_t *s, uint64_t W, uint64_t w0, uint64_t w1,
                            uint32_t *count)
{
    uint64_t covered = 0, i = 0;
    while (covered < W && covered < w1) {
        uint64_t mw = s[i++];
        uint64_t b = mw & 1, F = (mw >> 1) & 0xFFFFFFFFull, L = mw >> 33;
        if (b) {
            uint64_t a = covered > w0 ? covered : w0;
            uint64_t e = covered + F < w1 ? covered + F : w1;
            for (uint64_t w = a; w < e; w++)
                for (uint64_t x = w * 64; x < w * 64 + 64; x++) count[x - w0 * 64]++;
        }
        covered += F;
        for (uint64_t k = 0; k < L; k++) {
            uint64_t v = s[i++];
            if (covered >= w0 && covered < w1) {
                while (v) {
                    count[covered * 64 + (uint64_t)orc_ctz(v) - w0 * 64]++;
                    v &= v - 1;
                }
            }
            covered++;
        }
    }
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int orc_threshold_parts(const uint64_t *streams, const uint64_t *offsets,
                        uint32_t nbitmaps, uint64_t r, const uint32_t *ids,
                        uint32_t n, uint32_t T, uint32_t parts, uint64_t *out,
                        uint64_t cap, uint64_t *out_len)
{
    uint64_t W = orc_nwords(r);
    uint64_t *words = NULL;
    int rc = ORC_OK, bad = 0;
    if (out_len == NULL || (n > 0 && ids == NULL) || offsets == NULL || parts == 0)
        return ORC_E_INVAL;
    for (uint32_t q = 0; q < n; q++)
        if (ids[q] >= nbitmaps) return ORC_E_INVAL;
    for (uint32_t q = 0; q < n; q++) {
        uint64_t b = ids[q];
        rc = orc_validate(streams + offsets[b], offsets[b + 1] - offsets[b], r);
        if (rc != ORC_OK) return rc;
    }
    words = (uint64_t *)calloc(W > 0 ? W : 1, sizeof(uint64_t));
    if (!words) return ORC_E_NOMEM;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(| : bad)
#endif
    for (int64_t p = 0; p < (int64_t)parts; p++) {
        uint64_t w0 = W * (uint64_t)p / parts, w1 = W * (uint64_t)(p + 1) / parts;
        uint32_t *count;
        if (w1 == w0) continue;
        count = (uint32_t *)calloc((w1 - w0) * 64, sizeof(uint32_t));
        if (!count) {
            bad = 1;
            continue;
        }
        for (uint32_t q = 0; q < n; q++)
            orc_count_range(streams + offsets[ids[q]], W, w0, w1, count);
        for (uint64_t x = w0 * 64; x < w1 * 64 && x < r; x++)
            if (count[x - w0 * 64] >= T) words[x / 64] |= 1ull << (x % 64);
        free(count);
    }
    if (bad) rc = ORC_E_NOMEM;
    else rc = orc_encode(words, W, r, out, cap, out_len);
    free(words);
    return rc;
}

/*
 * The histogram of the counts (Sec. 5.1: ScanCount's counters, then the
 * opt-threshold reasoning of Sec. 3.3 reads them by count): hist[c], c = 0..n,
 * receives the number of rows in [0, r) counted exactly c times over the
 * multiset ids.  The suffix sum hist[T] + .. + hist[n] is the size of the
 * T-overlap result; row shards can add their histograms bin by bin.
 */
int orc_count_histogram(const uint64_t *streams, const uint64_t *offsets,
                        uint32_t nbitmaps, uint64_t r, const uint32_t *ids,
                        uint32_t n, uint64_t *hist)
{
    uint32_t *count = NULL;
    uint64_t *rows = NULL;
    int rc = ORC_OK;
    if ((n > 0 && ids == NULL) || offsets == NULL || hist == NULL) return ORC_E_INVAL;
    for (uint32_t q = 0; q < n; q++)
        if (ids[q] >= nbitmaps) return ORC_E_INVAL;
    count = (uint32_t *)calloc(r > 0 ? r : 1, sizeof(uint32_t));
    rows = (uint64_t *)malloc((r > 0 ? r : 1) * sizeof(uint64_t));
    if (!count || !rows) {
        rc = ORC_E_NOMEM;
        goto done;
    }
    for (uint32_t q = 0; q < n; q++) {
        uint64_t b = ids[q], nr = 0;
        rc = orc_decode(streams + offsets[b], offsets[b + 1] - offsets[b], r,
                        rows, r, &nr);
        if (rc != ORC_OK) goto done;
        for (uint64_t k = 0; k < nr; k++) count[rows[k]]++;
    }
    for (uint32_t c = 0; c <= n; c++) hist[c] = 0;
    for (uint64_t x = 0; x < r; x++) hist[count[x]]++;
done:
    free(count);
    free(rows);
    return rc;
}
