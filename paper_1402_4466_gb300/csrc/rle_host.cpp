// Host codec of the stream format (see rle_host.h and include/thr.h).
#include "rle_host.h"

#include <cstdio>

namespace thr {

namespace {

inline bool is_fill_word(uint64_t v) { return v == 0 || v == ~0ull; }

struct Emitter {
    uint64_t* out;
    uint64_t cap;
    uint64_t n = 0;
    void put(uint64_t v) {
        if (n < cap && out) out[n] = v;
        ++n;
    }
};

}  // namespace

int scan_stream(const uint64_t* s, uint64_t len, uint64_t r, StreamScan* scan,
                std::string* why) {
    auto fail = [&](const char* msg, uint64_t at) {
        if (why) {
            char buf[160];
            std::snprintf(buf, sizeof buf, "%s (stream word %llu)", msg,
                          (unsigned long long)at);
            *why = buf;
        }
        return 2;
    };
    const uint64_t W = (r + 63) / 64;
    const unsigned ragged = unsigned(r % 64);
    scan->marker_pos.clear();
    scan->set_rows = scan->literal_words = scan->ones_fill_words = 0;
    if (W == 0) {
        if (len != 1 || s[0] != 0) return fail("r = 0 requires the stream [0]", 0);
        scan->marker_pos.push_back(0);
        return 0;
    }
    if (len > kMaxWords + 1) return fail("stream longer than W + 1 words", 0);
    uint64_t at = 0, done = 0;  // stream cursor, uncompressed words covered
    bool have_prev = false;
    uint64_t pF = 0, pL = 0, pb = 0;
    while (done < W) {
        if (at >= len) return fail("stream ends before covering ceil(r/64) words", at);
        const uint64_t m = s[at];
        const uint64_t b = marker_fill_bit(m), F = marker_fill_len(m),
                       L = marker_lit_count(m);
        if (F == 0 && L == 0) return fail("marker covers no word", at);
        if (F == 0 && b) return fail("fill bit set on an empty fill", at);
        if (have_prev) {
            if (F == 0 && pL != kLitMax)
                return fail("marker without fill after an unsaturated literal run", at);
            if (F > 0 && pL == 0 && pb == b && pF != kFillMax)
                return fail("fill run split over two markers", at);
        }
        if (F > W - done || L > W - done - F) return fail("marker runs past the last word", at);
        if (b && ragged && done + F == W) return fail("fill of ones over the ragged last word", at);
        scan->marker_pos.push_back(uint32_t(at));
        if (b) {
            scan->set_rows += 64 * F;
            scan->ones_fill_words += F;
        }
        done += F;
        ++at;
        if (L > len - at) return fail("literal run truncated", at);
        for (uint64_t k = 0; k < L; ++k) {
            const uint64_t v = s[at + k];
            if (is_fill_word(v)) return fail("literal word equal to a fill word", at + k);
            if (ragged && done + k == W - 1 && (v >> ragged) != 0)
                return fail("bits past r in the last word", at + k);
            scan->set_rows += uint64_t(__builtin_popcountll(v));
        }
        at += L;
        done += L;
        scan->literal_words += L;
        pF = F;
        pL = L;
        pb = b;
        have_prev = true;
    }
    if (at != len) return fail("words after the last group", at);
    return 0;
}

namespace {

// Canonical group builder: fill words and literal words are fed in order;
// a group [marker, literals] is emitted when a fill word follows literals,
// when the fill value changes, or when a counter would overflow.
struct GroupEncoder {
    Emitter e;
    bool open = false;
    uint64_t gb = 0, gF = 0;
    std::vector<uint64_t> lits;
    void flush() {
        if (!open) return;
        e.put(marker_word(gF ? gb : 0, gF, lits.size()));
        for (uint64_t v : lits) e.put(v);
        lits.clear();
        open = false;
    }
    void fill(uint64_t fb, uint64_t count) {
        while (count) {
            if (open && lits.empty() && gb == fb && gF < kFillMax) {
                const uint64_t take = std::min(count, kFillMax - gF);
                gF += take;
                count -= take;
                continue;
            }
            flush();
            open = true;
            gb = fb;
            gF = 0;
        }
    }
    void literal(uint64_t v) {
        if (open && lits.size() == kLitMax) flush();
        if (!open) {
            open = true;
            gb = 0;
            gF = 0;
        }
        lits.push_back(v);
    }
    void word(uint64_t v) {
        if (is_fill_word(v))
            fill(v ? 1 : 0, 1);
        else
            literal(v);
    }
};

}  // namespace

// Feeds the uncompressed words [w0, w1) of a canonical stream s (W words)
// into g as fills and literals.
void feed_range(const uint64_t* s, uint64_t len, uint64_t w0, uint64_t w1, GroupEncoder* g) {
    uint64_t pos = 0;  // uncompressed word where the current group starts
    for (uint64_t i = 0; i < len && pos < w1;) {
        const uint64_t m = s[i];
        const uint64_t F = marker_fill_len(m), L = marker_lit_count(m), b = marker_fill_bit(m);
        // fill words [pos, pos + F)
        const uint64_t f0 = std::max(pos, w0), f1 = std::min(pos + F, w1);
        if (f1 > f0) g->fill(F ? b : 0, f1 - f0);
        pos += F;
        // literal words [pos, pos + L)
        const uint64_t l0 = std::max(pos, w0), l1 = std::min(pos + L, w1);
        for (uint64_t w = l0; w < l1; ++w) g->literal(s[i + 1 + (w - pos)]);
        pos += L;
        i += 1 + L;
    }
}

int slice_stream(const uint64_t* s, uint64_t len, uint64_t r, uint64_t w0, uint64_t w1,
                 uint64_t* out, uint64_t cap, uint64_t* out_len) {
    const uint64_t W = (r + 63) / 64;
    if (w0 >= w1 || w1 > W) return 1;
    GroupEncoder g{Emitter{out, cap}};
    feed_range(s, len, w0, w1, &g);
    g.flush();
    *out_len = g.e.n;
    return g.e.n <= cap ? 0 : 4;
}

int stitch_streams(const uint64_t* const* parts, const uint64_t* lens, const uint64_t* words,
                   uint32_t nparts, uint64_t* out, uint64_t cap, uint64_t* out_len) {
    if (nparts == 0) return 1;
    GroupEncoder g{Emitter{out, cap}};
    for (uint32_t k = 0; k < nparts; ++k) {
        if (!words[k]) return 1;
        feed_range(parts[k], lens[k], 0, words[k], &g);
    }
    g.flush();
    *out_len = g.e.n;
    return g.e.n <= cap ? 0 : 4;
}

int encode_rows(const uint64_t* rows, uint64_t nrows, uint64_t r, uint64_t* out, uint64_t cap,
                uint64_t* out_len) {
    const uint64_t W = (r + 63) / 64;
    if (W > kMaxWords || r == 0) return 1;
    for (uint64_t i = 0; i < nrows; ++i)
        if (rows[i] >= r || (i && rows[i] < rows[i - 1])) return 1;
    GroupEncoder g{Emitter{out, cap}};
    uint64_t next = 0;  // first word not yet fed
    for (uint64_t i = 0; i < nrows;) {
        const uint64_t w = rows[i] / 64;
        uint64_t v = 0;
        for (; i < nrows && rows[i] / 64 == w; ++i) v |= 1ull << (rows[i] % 64);
        if (w > next) g.fill(0, w - next);
        g.word(v);
        next = w + 1;
    }
    if (W > next) g.fill(0, W - next);
    g.flush();
    *out_len = g.e.n;
    return g.e.n <= cap ? 0 : 4;
}

int encode_words(const uint64_t* words, uint64_t nwords, uint64_t r,
                 uint64_t* out, uint64_t cap, uint64_t* out_len) {
    const uint64_t W = (r + 63) / 64;
    if (nwords != W || !out_len || (W > 0 && !words)) return 1;
    if (W > kMaxWords) return 1;
    if ((r % 64) && (words[W - 1] >> (r % 64)) != 0) return 1;
    Emitter e{out, cap};
    if (W == 0) {
        e.put(0);
        *out_len = e.n;
        return e.n <= cap ? 0 : 4;
    }
    // One pending group [fill run][literal run]; it is emitted when a fill
    // word follows literals, when the fill value changes, or on overflow.
    bool open = false;
    uint64_t gb = 0, gF = 0, gL = 0, gfirst = 0;
    auto flush = [&]() {
        if (!open) return;
        e.put(marker_word(gF ? gb : 0, gF, gL));
        for (uint64_t k = 0; k < gL; ++k) e.put(words[gfirst + k]);
        open = false;
    };
    for (uint64_t i = 0; i < W; ++i) {
        const uint64_t v = words[i];
        if (is_fill_word(v)) {
            const uint64_t fb = v ? 1 : 0;
            if (open && gL == 0 && gb == fb && gF < kFillMax) {
                ++gF;
            } else {
                flush();
                open = true;
                gb = fb;
                gF = 1;
                gL = 0;
            }
        } else {
            if (open && gL == kLitMax) flush();
            if (!open) {
                open = true;
                gb = 0;
                gF = 0;
                gL = 0;
            }
            if (gL == 0) gfirst = i;
            ++gL;
        }
    }
    flush();
    *out_len = e.n;
    return e.n <= cap ? 0 : 4;
}

}  // namespace thr
