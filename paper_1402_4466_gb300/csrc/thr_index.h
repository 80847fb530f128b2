// The index object behind the opaque thr_index handle of include/thr.h
// (internal to the library).
#pragma once

#include <cstdint>
#include <map>
#include <mutex>
#include <vector>

#include "../../include/thr.h"
#include "thr_device.cuh"

namespace thr {
struct Selector;
}

struct thr_index {
    int device = 0;
    uint32_t nbitmaps = 0;
    uint64_t r = 0;
    uint32_t W = 0;   // ceil(r / 64)
    uint32_t NG = 0;  // ceil(W / 128)
    uint64_t total_words = 0;
    uint64_t total_markers = 0;
    uint64_t* d_words = nullptr;  // total_words + 2 (zero pad: 16-byte copies may round up)
    uint2* d_mtab = nullptr;
    uint64_t* d_sdesc = nullptr;  // NG subtile descriptors per bitmap
    uint64_t* d_pcls = nullptr;   // their classes, 2 bits each, ceil(NG/32) words per bitmap
    thr::MaskRec* d_masks = nullptr;  // mask records of the mixed subtiles
    uint64_t* d_sseg = nullptr;   // NG segment descriptors per bitmap
    uint64_t mixed_subtiles = 0;
    thr::BitmapDesc* d_desc = nullptr;
    std::vector<thr::BitmapDesc> desc;
    std::vector<uint64_t> set_rows;
    // per bitmap, the selector's feature terms log2(words + 1) and
    // log10(density + 1e-7), computed once at build
    std::vector<double> feat_lw, feat_ld;
    int num_sms = 0;
    // pass-A launch configurations chosen by thr_autotune, per batch shape
    mutable std::mutex tune_mu;
    mutable std::map<uint32_t, uint32_t> tune;
    // cost model of THR_POLICY_LEARNED (not owned; thr_index_set_selector)
    const thr::Selector* selector = nullptr;
};

namespace thr {
// Records msg as the calling thread's thr_last_error() and returns st.
thr_status report_error(thr_status st, const char* msg);
}  // namespace thr
