// Host side of the stream format: canonical encoder and the validating
// scanner that also records where every marker word sits (the marker table
// the device decoder starts from).  Format: see include/thr.h; it follows the
// marker/fill/dirty-word description of Sec. 3.1 of Kaser & Lemire.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace thr {

constexpr uint64_t kFillMax = 0xFFFFFFFFull;  // 32-bit fill counter
constexpr uint64_t kLitMax = 0x7FFFFFFFull;   // 31-bit literal counter
constexpr uint64_t kMaxWords = (1ull << 31) - 2;  // largest W accepted

inline uint64_t marker_word(uint64_t fill_bit, uint64_t F, uint64_t L) {
    return (fill_bit & 1) | (F << 1) | (L << 33);
}
inline uint64_t marker_fill_bit(uint64_t m) { return m & 1; }
inline uint64_t marker_fill_len(uint64_t m) { return (m >> 1) & kFillMax; }
inline uint64_t marker_lit_count(uint64_t m) { return m >> 33; }

struct StreamScan {
    std::vector<uint32_t> marker_pos;  // stream index of every marker word
    uint64_t set_rows = 0;             // number of set rows
    uint64_t literal_words = 0;        // number of literal words
    uint64_t ones_fill_words = 0;      // uncompressed words inside 1-fills
};

// Validates a stream of an r-row bitmap against the canonical rules and
// fills *scan.  Returns 0 on success; otherwise 2 (THR_E_FORMAT) and a reason.
int scan_stream(const uint64_t* s, uint64_t len, uint64_t r, StreamScan* scan,
                std::string* why);

// Canonical encoding of W = ceil(r/64) uncompressed words.  Returns 0, or
// 1 (bad argument: wrong word count or bits past r), or 4 (out too small;
// *out_len still receives the full length).
int encode_words(const uint64_t* words, uint64_t nwords, uint64_t r,
                 uint64_t* out, uint64_t cap, uint64_t* out_len);

// Canonical encoding of the bitmap whose set rows are rows[0..nrows)
// (ascending, repeats allowed, each < r), without forming the uncompressed
// words.  Returns 0, 1 (bad argument) or 4 (out too small; *out_len still
// receives the full length).
int encode_rows(const uint64_t* rows, uint64_t nrows, uint64_t r, uint64_t* out, uint64_t cap,
                uint64_t* out_len);

// The uncompressed words [w0, w1) of the canonical stream s of an r-row
// bitmap, as a canonical stream of its own (a row-range shard when w0 and w1
// are word boundaries).  The stream must be valid (scan_stream).  Returns 0,
// 1 (bad range) or 4 (out too small; *out_len still receives the length).
int slice_stream(const uint64_t* s, uint64_t len, uint64_t r, uint64_t w0, uint64_t w1,
                 uint64_t* out, uint64_t cap, uint64_t* out_len);

// The canonical stream of the concatenation of nparts valid canonical
// streams covering words[k] uncompressed words each: runs that meet at a
// seam merge (a fill continuing a fill of the same value, literals following
// literals).  Returns 0, 1 (bad argument) or 4 (out too small).
int stitch_streams(const uint64_t* const* parts, const uint64_t* lens, const uint64_t* words,
                   uint32_t nparts, uint64_t* out, uint64_t cap, uint64_t* out_len);

}  // namespace thr
