// The selector's cost model (thr_mlp.cu) and query features (thr_select.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <array>
#include <cstdint>
#include <mutex>
#include <string>
#include <unordered_map>

#include "../../include/thr.h"

struct thr_index;

namespace thr {

constexpr int kSelFeatures = 16;
constexpr int kSelHidden = 64;
constexpr int kSelVariants = 4;
constexpr int kSelParams = kSelFeatures * kSelHidden + kSelHidden + kSelHidden * kSelHidden +
                           kSelHidden + kSelHidden * kSelVariants + kSelVariants;

// MLP F -> 64 -> 64 -> V on the device: FP32 master parameters, BF16
// copies read by the passes (or the FP32 values when bf16 is false), Adam
// state, feature normalisation x' = (x - mean) * istd.
struct Selector {
    int device = 0, num_sms = 1;
    bool bf16 = true;
    float* p = nullptr;  // parameters (layout: W1[F][H] b1[H] W2[H][H] b2[H] W3[H][V] b3[V])
    float* g = nullptr;  // gradients
    float* m = nullptr;  // Adam first moments
    float* v = nullptr;  // Adam second moments
    __nv_bfloat16* q = nullptr;
    float* norm = nullptr;  // mean[F], istd[F]
    float* loss = nullptr;
    float h_norm[2 * kSelFeatures] = {};
    uint64_t step = 0;
    // predict(): buffers kept between calls (grown on demand) and a stream,
    // one caller at a time
    mutable std::mutex pmu;
    mutable float* pdev = nullptr;  // features | predictions
    mutable float* phost = nullptr; // pinned staging of the same
    mutable uint32_t pcap = 0;      // rows
    mutable cudaStream_t pst = nullptr;
    // predictions already made, by feature vector, for the parameters and
    // normalisation of `version` (bumped by every change of either)
    uint64_t version = 0;
    mutable uint64_t memo_version = ~0ull;
    mutable std::unordered_map<std::string, std::array<float, kSelVariants>> memo;

    ~Selector();
    thr_status init(uint64_t seed, bool use_bf16);
    thr_status set_params(const float* host);
    thr_status get_params(float* host) const;
    thr_status set_norm(const float* mean, const float* istd);
    thr_status predict(const float* X, uint32_t rows, float* Y) const;
    // the same predictions, reusing those already made for identical
    // features (the policy's repeated queries skip the forward pass)
    thr_status predict_memo(const float* X, uint32_t rows, float* Y) const;
    thr_status forward_locked(const float* X, uint32_t rows, float* Y) const;  // pmu held
    void bump_version();  // after a change of parameters or normalisation
    thr_status gradients(const float* X, const float* T, const uint8_t* M, uint32_t rows,
                         float* grad, float* loss_out);
    thr_status train(const float* X, const float* T, const uint8_t* M, uint32_t rows,
                     uint32_t epochs, uint32_t batch, float lr, uint64_t seed, float* final_loss);
};

// The features of a query (kSelFeatures floats): log2 n, log2 (T + 1),
// log2 (n - T + 2) (0 when T > n), log2 r; the quantiles 0, 1/4, 1/2, 3/4, 1
// of log2 (compressed words + 1) over its inputs and log2 of their sum; the
// same quantiles of log10 (density + 1e-7) and the sum of the densities.
void query_features(const thr_index* idx, const uint32_t* ids, uint32_t n, uint32_t T,
                    float* f);

}  // namespace thr
