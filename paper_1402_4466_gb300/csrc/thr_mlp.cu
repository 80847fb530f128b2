// The learned cost model of the variant selector: a multilayer perceptron
// F -> H -> H -> V (ReLU between layers) that predicts, from features of a
// query, the log of the pass-A time of each counting variant.  The paper
// fits linear execution-time models per algorithm and picks the smallest
// prediction (Sec. 8.1-8.2); this model replaces the linear fits and keeps
// their role.
//
// Parameters live on the device as FP32 master copies; the forward and
// backward passes read them rounded to BF16 (round to nearest even) or, for
// checking, unrounded.  Activations, gradients and accumulation are FP32.
// Training is minibatch Adam; every kernel is here.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <random>
#include <vector>

#include "../../include/thr.h"
#include "thr_index.h"
#include "thr_mlp.h"

namespace thr {

namespace {

constexpr int F = kSelFeatures, H = kSelHidden, V = kSelVariants;
constexpr int kRowsPerTile = 32;

// parameter offsets (floats) in the flat vector
constexpr int oW1 = 0, ob1 = oW1 + F * H, oW2 = ob1 + H, ob2 = oW2 + H * H, oW3 = ob2 + H,
              ob3 = oW3 + H * V, kParams = ob3 + V;
static_assert(kParams == kSelParams, "parameter count");

// Parameters as the passes read them, staged in shared memory.
struct Weights {
    float w1[F * H], b1[H], w2[H * H], b2[H], w3[H * V], b3[V];
};

__device__ __forceinline__ void load_weights(Weights& w, const float* p, const __nv_bfloat16* q,
                                             bool bf16) {
    float* dst = reinterpret_cast<float*>(&w);
    for (int i = threadIdx.x; i < kParams; i += blockDim.x)
        dst[i] = bf16 ? __bfloat162float(q[i]) : p[i];
}

// Forward pass of rows [r0, r0 + 32) of the minibatch; x normalised in
// place in xs.  Thread u < H computes hidden unit u.
__device__ __forceinline__ void forward_tile(const Weights& w, float (*xs)[F], float (*h1)[H],
                                             float (*h2)[H], float (*y)[V], int nrows) {
    const int u = threadIdx.x;
    for (int r = 0; r < nrows; ++r) {
        float a = w.b1[u];
#pragma unroll
        for (int f = 0; f < F; ++f) a = fmaf(xs[r][f], w.w1[f * H + u], a);
        h1[r][u] = fmaxf(a, 0.f);
    }
    __syncthreads();
    for (int r = 0; r < nrows; ++r) {
        float a = w.b2[u];
#pragma unroll 16
        for (int k = 0; k < H; ++k) a = fmaf(h1[r][k], w.w2[k * H + u], a);
        h2[r][u] = fmaxf(a, 0.f);
    }
    __syncthreads();
    for (int i = u; i < nrows * V; i += H) {
        const int r = i / V, v = i % V;
        float a = w.b3[v];
#pragma unroll 16
        for (int k = 0; k < H; ++k) a = fmaf(h2[r][k], w.w3[k * V + v], a);
        y[r][v] = a;
    }
    __syncthreads();
}

__device__ __forceinline__ void stage_x(const float* X, const float* mean, const float* istd,
                                        int r0, int nrows, float (*xs)[F]) {
    for (int i = threadIdx.x; i < nrows * F; i += blockDim.x) {
        const int r = i / F, f = i % F;
        xs[r][f] = (X[uint64_t(r0 + r) * F + f] - mean[f]) * istd[f];
    }
    __syncthreads();
}

struct SmemTile {
    Weights w;
    float xs[kRowsPerTile][F];
    float h1[kRowsPerTile][H];
    float h2[kRowsPerTile][H];
    float y[kRowsPerTile][V];
    float dy[kRowsPerTile][V];
    float dh2[kRowsPerTile][H];
    float red[H];
};

// Predictions of rows [0, B).
__global__ void __launch_bounds__(H) k_mlp_forward(const float* X, const float* mean,
                                                   const float* istd, const float* p,
                                                   const __nv_bfloat16* q, int bf16, uint32_t B,
                                                   float* Y) {
    extern __shared__ __align__(16) unsigned char raw[];
    SmemTile& s = *reinterpret_cast<SmemTile*>(raw);
    load_weights(s.w, p, q, bf16 != 0);
    __syncthreads();
    for (uint32_t r0 = blockIdx.x * kRowsPerTile; r0 < B; r0 += gridDim.x * kRowsPerTile) {
        const int nrows = int(min(uint32_t(kRowsPerTile), B - r0));
        stage_x(X, mean, istd, int(r0), nrows, s.xs);
        forward_tile(s.w, s.xs, s.h1, s.h2, s.y, nrows);
        for (int i = threadIdx.x; i < nrows * V; i += H) Y[uint64_t(r0) * V + i] = s.y[i / V][i % V];
        __syncthreads();
    }
}

// Loss = sum over valid (row, variant) of (y - t)^2 / count; gradients of
// the rows [0, B) added into g (zeroed by the caller), loss into *loss.
__global__ void __launch_bounds__(H) k_mlp_backward(const float* X, const float* mean,
                                                    const float* istd, const float* Tg,
                                                    const uint8_t* M, const float* p,
                                                    const __nv_bfloat16* q, int bf16, uint32_t B,
                                                    float inv_count, float* g, float* loss) {
    extern __shared__ __align__(16) unsigned char raw[];
    SmemTile& s = *reinterpret_cast<SmemTile*>(raw);
    load_weights(s.w, p, q, bf16 != 0);
    __syncthreads();
    const int u = threadIdx.x;
    float gW2[H];  // column u of dW2: gW2[k] = dW2[k][u]
#pragma unroll
    for (int k = 0; k < H; ++k) gW2[k] = 0.f;
    float gW1[F];  // column u of dW1
#pragma unroll
    for (int f = 0; f < F; ++f) gW1[f] = 0.f;
    float gW3[V];  // row u of dW3
#pragma unroll
    for (int v = 0; v < V; ++v) gW3[v] = 0.f;
    float gb1 = 0.f, gb2 = 0.f, gb3 = 0.f, lsum = 0.f;
    for (uint32_t r0 = blockIdx.x * kRowsPerTile; r0 < B; r0 += gridDim.x * kRowsPerTile) {
        const int nrows = int(min(uint32_t(kRowsPerTile), B - r0));
        stage_x(X, mean, istd, int(r0), nrows, s.xs);
        forward_tile(s.w, s.xs, s.h1, s.h2, s.y, nrows);
        for (int i = u; i < nrows * V; i += H) {
            const int r = i / V, v = i % V;
            const uint64_t gi = uint64_t(r0 + r) * V + v;
            const float d = M[gi] ? s.y[r][v] - Tg[gi] : 0.f;
            s.dy[r][v] = 2.f * d * inv_count;
            lsum += d * d * inv_count;
        }
        __syncthreads();
        // layer 3: dW3 row u, db3, dh2
        for (int r = 0; r < nrows; ++r) {
            float a = 0.f;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                gW3[v] = fmaf(s.h2[r][u], s.dy[r][v], gW3[v]);
                a = fmaf(s.w.w3[u * V + v], s.dy[r][v], a);
            }
            s.dh2[r][u] = s.h2[r][u] > 0.f ? a : 0.f;
        }
        if (u < V)
            for (int r = 0; r < nrows; ++r) gb3 += s.dy[r][u];
        __syncthreads();
        // layer 2: dW2 column u, db2; dh1 (in place of h2, which is no longer needed)
        for (int r = 0; r < nrows; ++r) {
            const float d = s.dh2[r][u];
            gb2 += d;
#pragma unroll
            for (int k = 0; k < H; ++k) gW2[k] = fmaf(s.h1[r][k], d, gW2[k]);
        }
        for (int r = 0; r < nrows; ++r) {
            float a = 0.f;
#pragma unroll 16
            for (int jj = 0; jj < H; ++jj) {  // rotated so the warp's reads hit distinct banks
                const int j = (jj + u) & (H - 1);
                a = fmaf(s.w.w2[u * H + j], s.dh2[r][j], a);
            }
            s.h2[r][u] = s.h1[r][u] > 0.f ? a : 0.f;  // dh1[r][u]
        }
        __syncthreads();
        // layer 1: dW1 column u, db1
        for (int r = 0; r < nrows; ++r) {
            const float d = s.h2[r][u];
            gb1 += d;
#pragma unroll
            for (int f = 0; f < F; ++f) gW1[f] = fmaf(s.xs[r][f], d, gW1[f]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < H; ++k) atomicAdd(g + oW2 + k * H + u, gW2[k]);
#pragma unroll
    for (int f = 0; f < F; ++f) atomicAdd(g + oW1 + f * H + u, gW1[f]);
#pragma unroll
    for (int v = 0; v < V; ++v) atomicAdd(g + oW3 + u * V + v, gW3[v]);
    atomicAdd(g + ob1 + u, gb1);
    atomicAdd(g + ob2 + u, gb2);
    if (u < V) atomicAdd(g + ob3 + u, gb3);
    s.red[u] = lsum;
    __syncthreads();
    if (u == 0) {
        float t = 0.f;
        for (int k = 0; k < H; ++k) t += s.red[k];
        atomicAdd(loss, t);
    }
}

// Adam (Kingma & Ba) on the master copy; refreshes the BF16 copy.
__global__ void k_adam(float* p, const float* g, float* m, float* v, __nv_bfloat16* q, int n,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float step = lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    const float pi = p[i] - step;
    p[i] = pi;
    q[i] = __float2bfloat16_rn(pi);
}

__global__ void k_round(const float* p, __nv_bfloat16* q, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) q[i] = __float2bfloat16_rn(p[i]);
}

constexpr size_t kSmem = sizeof(SmemTile);

thr_status cuda_err(cudaError_t e, const char* what) {
    char msg[256];
    std::snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString(e));
    return report_error(e == cudaErrorMemoryAllocation ? THR_E_NOMEM : THR_E_CUDA, msg);
}

#define CKM(call, what)                                  \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_err(e_, what); \
    } while (0)

cudaError_t prepare_kernels() {
    static cudaError_t once = [] {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_forward,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             int(kSmem));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(kSmem));
        return e;
    }();
    return once;
}

// Device copies of a data set (features, targets, mask).
struct DevData {
    float* X = nullptr;
    float* T = nullptr;
    uint8_t* M = nullptr;
    uint32_t rows = 0;
    ~DevData() {
        cudaFree(X);
        cudaFree(T);
        cudaFree(M);
    }
    cudaError_t upload(const float* x, const float* t, const uint8_t* m, uint32_t n) {
        rows = n;
        cudaError_t e;
        if ((e = cudaMalloc(&X, sizeof(float) * F * std::max<uint32_t>(n, 1))) != cudaSuccess)
            return e;
        if ((e = cudaMemcpy(X, x, sizeof(float) * F * n, cudaMemcpyHostToDevice)) != cudaSuccess)
            return e;
        if (t) {
            if ((e = cudaMalloc(&T, sizeof(float) * V * std::max<uint32_t>(n, 1))) !=
                cudaSuccess)
                return e;
            if ((e = cudaMemcpy(T, t, sizeof(float) * V * n, cudaMemcpyHostToDevice)) !=
                cudaSuccess)
                return e;
            if ((e = cudaMalloc(&M, std::max<uint32_t>(V * n, 1))) != cudaSuccess) return e;
            if ((e = cudaMemcpy(M, m, size_t(V) * n, cudaMemcpyHostToDevice)) != cudaSuccess)
                return e;
        }
        return cudaSuccess;
    }
};

int grid_for(uint32_t rows, int num_sms) {
    const uint32_t tiles = (rows + kRowsPerTile - 1) / kRowsPerTile;
    return int(std::max<uint32_t>(1, std::min<uint32_t>(tiles, uint32_t(num_sms) * 4)));
}

}  // namespace

Selector::~Selector() {
    cudaFree(pdev);
    if (phost) cudaFreeHost(phost);
    if (pst) cudaStreamDestroy(pst);
    cudaFree(p);
    cudaFree(g);
    cudaFree(m);
    cudaFree(v);
    cudaFree(q);
    cudaFree(norm);
    cudaFree(loss);
}

thr_status Selector::init(uint64_t seed, bool use_bf16) {
    bf16 = use_bf16;
    CKM(cudaGetDevice(&device), "device");
    cudaDeviceProp prop;
    CKM(cudaGetDeviceProperties(&prop, device), "device properties");
    num_sms = prop.multiProcessorCount;
    CKM(prepare_kernels(), "MLP kernel attributes");
    CKM(cudaMalloc(&p, sizeof(float) * kParams), "MLP parameters");
    CKM(cudaMalloc(&g, sizeof(float) * kParams), "MLP gradients");
    CKM(cudaMalloc(&m, sizeof(float) * kParams), "Adam state");
    CKM(cudaMalloc(&v, sizeof(float) * kParams), "Adam state");
    CKM(cudaMalloc(&q, sizeof(__nv_bfloat16) * kParams), "BF16 parameters");
    CKM(cudaMalloc(&norm, sizeof(float) * 2 * F), "feature normalisation");
    CKM(cudaMalloc(&loss, sizeof(float)), "loss");
    // He initialisation of the weights, zero biases
    std::vector<float> h(kParams, 0.f);
    std::mt19937_64 rng(seed);
    auto fill = [&](int off, int fan_in, int count) {
        std::normal_distribution<float> nd(0.f, std::sqrt(2.f / float(fan_in)));
        for (int i = 0; i < count; ++i) h[off + i] = nd(rng);
    };
    fill(oW1, F, F * H);
    fill(oW2, H, H * H);
    fill(oW3, H, H * V);
    std::vector<float> nm(2 * F);
    for (int f = 0; f < F; ++f) {
        nm[f] = 0.f;
        nm[F + f] = 1.f;
    }
    CKM(cudaMemcpy(norm, nm.data(), sizeof(float) * 2 * F, cudaMemcpyHostToDevice), "norm");
    return set_params(h.data());
}

thr_status Selector::set_params(const float* host) {
    CKM(cudaMemcpy(p, host, sizeof(float) * kParams, cudaMemcpyHostToDevice), "set parameters");
    CKM(cudaMemset(m, 0, sizeof(float) * kParams), "Adam state");
    CKM(cudaMemset(v, 0, sizeof(float) * kParams), "Adam state");
    step = 0;
    k_round<<<(kParams + 255) / 256, 256>>>(p, q, kParams);
    CKM(cudaGetLastError(), "round parameters");
    CKM(cudaDeviceSynchronize(), "round parameters");
    bump_version();
    return THR_OK;
}

thr_status Selector::get_params(float* host) const {
    CKM(cudaMemcpy(host, p, sizeof(float) * kParams, cudaMemcpyDeviceToHost), "get parameters");
    return THR_OK;
}

thr_status Selector::set_norm(const float* mean, const float* istd) {
    CKM(cudaMemcpy(norm, mean, sizeof(float) * F, cudaMemcpyHostToDevice), "norm");
    CKM(cudaMemcpy(norm + F, istd, sizeof(float) * F, cudaMemcpyHostToDevice), "norm");
    std::memcpy(h_norm, mean, sizeof(float) * F);
    std::memcpy(h_norm + F, istd, sizeof(float) * F);
    bump_version();
    return THR_OK;
}

void Selector::bump_version() {
    std::lock_guard<std::mutex> lk(pmu);
    ++version;
}

thr_status Selector::predict(const float* X, uint32_t rows, float* Y) const {
    if (!rows) return THR_OK;
    std::lock_guard<std::mutex> lk(pmu);
    return forward_locked(X, rows, Y);
}

thr_status Selector::predict_memo(const float* X, uint32_t rows, float* Y) const {
    if (!rows) return THR_OK;
    std::lock_guard<std::mutex> lk(pmu);
    if (memo_version != version || memo.size() > 65536) {
        memo.clear();
        memo_version = version;
    }
    std::vector<uint32_t> miss;
    for (uint32_t i = 0; i < rows; ++i) {
        auto it = memo.find(std::string(reinterpret_cast<const char*>(X + size_t(F) * i),
                                        sizeof(float) * F));
        if (it == memo.end()) {
            miss.push_back(i);
        } else {
            std::memcpy(Y + size_t(V) * i, it->second.data(), sizeof(float) * V);
        }
    }
    if (miss.empty()) return THR_OK;
    std::vector<float> mx(size_t(F) * miss.size()), my(size_t(V) * miss.size());
    for (size_t k = 0; k < miss.size(); ++k)
        std::memcpy(&mx[F * k], X + size_t(F) * miss[k], sizeof(float) * F);
    thr_status s = forward_locked(mx.data(), uint32_t(miss.size()), my.data());
    if (s != THR_OK) return s;
    for (size_t k = 0; k < miss.size(); ++k) {
        std::array<float, kSelVariants> y;
        std::memcpy(y.data(), &my[V * k], sizeof(float) * V);
        std::memcpy(Y + size_t(V) * miss[k], y.data(), sizeof(float) * V);
        memo.emplace(std::string(reinterpret_cast<const char*>(X + size_t(F) * miss[k]),
                                 sizeof(float) * F),
                     y);
    }
    return THR_OK;
}

thr_status Selector::forward_locked(const float* X, uint32_t rows, float* Y) const {
    if (!pst) CKM(cudaStreamCreateWithFlags(&pst, cudaStreamNonBlocking), "predict stream");
    if (pcap < rows) {
        cudaFree(pdev);
        if (phost) cudaFreeHost(phost);
        pdev = nullptr;
        phost = nullptr;
        pcap = 0;
        const uint32_t cap = std::max<uint32_t>(rows, 256);
        CKM(cudaMalloc(&pdev, sizeof(float) * (F + V) * cap), "predict buffers");
        CKM(cudaMallocHost(&phost, sizeof(float) * (F + V) * cap), "predict staging");
        pcap = cap;
    }
    float* dX = pdev;
    float* dY = pdev + size_t(F) * pcap;
    float* hX = phost;
    float* hY = phost + size_t(F) * pcap;
    std::memcpy(hX, X, sizeof(float) * F * rows);
    CKM(cudaMemcpyAsync(dX, hX, sizeof(float) * F * rows, cudaMemcpyHostToDevice, pst),
        "upload features");
    k_mlp_forward<<<grid_for(rows, num_sms), H, kSmem, pst>>>(dX, norm, norm + F, p, q,
                                                                bf16 ? 1 : 0, rows, dY);
    CKM(cudaGetLastError(), "MLP forward");
    CKM(cudaMemcpyAsync(hY, dY, sizeof(float) * V * rows, cudaMemcpyDeviceToHost, pst),
        "read predictions");
    CKM(cudaStreamSynchronize(pst), "MLP forward");
    std::memcpy(Y, hY, sizeof(float) * V * rows);
    return THR_OK;
}

thr_status Selector::gradients(const float* X, const float* Tg, const uint8_t* M, uint32_t rows,
                               float* grad, float* loss_out) {
    DevData d;
    CKM(d.upload(X, Tg, M, rows), "upload training data");
    uint64_t cnt = 0;
    for (uint64_t i = 0; i < uint64_t(rows) * V; ++i) cnt += M[i] ? 1 : 0;
    CKM(cudaMemset(g, 0, sizeof(float) * kParams), "zero gradients");
    CKM(cudaMemset(loss, 0, sizeof(float)), "zero loss");
    k_mlp_backward<<<grid_for(rows, num_sms), H, kSmem>>>(
        d.X, norm, norm + F, d.T, d.M, p, q, bf16 ? 1 : 0, rows,
        cnt ? 1.f / float(cnt) : 0.f, g, loss);
    CKM(cudaGetLastError(), "MLP backward");
    CKM(cudaMemcpy(grad, g, sizeof(float) * kParams, cudaMemcpyDeviceToHost), "gradients");
    CKM(cudaMemcpy(loss_out, loss, sizeof(float), cudaMemcpyDeviceToHost), "loss");
    return THR_OK;
}

thr_status Selector::train(const float* X, const float* Tg, const uint8_t* M, uint32_t rows,
                           uint32_t epochs, uint32_t batch, float lr, uint64_t seed,
                           float* final_loss) {
    if (!rows || !batch) return report_error(THR_E_INVAL, "empty training set or batch");
    std::vector<uint32_t> perm(rows);
    for (uint32_t i = 0; i < rows; ++i) perm[i] = i;
    std::mt19937_64 rng(seed);
    std::vector<float> xs(size_t(rows) * F), ts(size_t(rows) * V);
    std::vector<uint8_t> ms(size_t(rows) * V);
    std::vector<uint32_t> cnt_prefix(rows + 1, 0);  // valid targets before row i
    DevData d;
    CKM(d.upload(X, Tg, M, rows), "upload training data");
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    batch = std::min(batch, rows);
    const uint32_t nbatches = (rows + batch - 1) / batch;
    float last = 0.f;
    for (uint32_t ep = 0; ep < epochs; ++ep) {
        // a new order every epoch, then contiguous minibatches
        std::shuffle(perm.begin(), perm.end(), rng);
        for (uint32_t i = 0; i < rows; ++i) {
            std::memcpy(&xs[size_t(i) * F], X + size_t(perm[i]) * F, sizeof(float) * F);
            std::memcpy(&ts[size_t(i) * V], Tg + size_t(perm[i]) * V, sizeof(float) * V);
            std::memcpy(&ms[size_t(i) * V], M + size_t(perm[i]) * V, V);
            uint32_t c = 0;
            for (int k = 0; k < V; ++k) c += ms[size_t(i) * V + k] ? 1 : 0;
            cnt_prefix[i + 1] = cnt_prefix[i] + c;
        }
        CKM(cudaMemcpy(d.X, xs.data(), sizeof(float) * F * rows, cudaMemcpyHostToDevice),
            "upload features");
        CKM(cudaMemcpy(d.T, ts.data(), sizeof(float) * V * rows, cudaMemcpyHostToDevice),
            "upload targets");
        CKM(cudaMemcpy(d.M, ms.data(), size_t(V) * rows, cudaMemcpyHostToDevice), "upload mask");
        CKM(cudaMemset(loss, 0, sizeof(float)), "zero loss");
        for (uint32_t a = 0; a < rows; a += batch) {
            const uint32_t nb = std::min(batch, rows - a);
            const uint32_t cnt = cnt_prefix[a + nb] - cnt_prefix[a];
            CKM(cudaMemsetAsync(g, 0, sizeof(float) * kParams, 0), "zero gradients");
            k_mlp_backward<<<grid_for(nb, num_sms), H, kSmem>>>(
                d.X + size_t(a) * F, norm, norm + F, d.T + size_t(a) * V, d.M + size_t(a) * V, p,
                q, bf16 ? 1 : 0, nb, cnt ? 1.f / float(cnt) : 0.f, g, loss);
            CKM(cudaGetLastError(), "MLP backward");
            ++step;
            const float c1 = 1.f - std::pow(b1, float(step));
            const float c2 = 1.f - std::pow(b2, float(step));
            k_adam<<<(kParams + 255) / 256, 256>>>(p, g, m, v, q, kParams, lr, b1, b2, eps, c1,
                                                    c2);
            CKM(cudaGetLastError(), "Adam");
        }
        float l = 0.f;
        CKM(cudaMemcpy(&l, loss, sizeof(float), cudaMemcpyDeviceToHost), "loss");
        last = l / float(nbatches);  // mean of the minibatch losses
    }
    if (final_loss) *final_loss = last;
    bump_version();
    return THR_OK;
}

}  // namespace thr

// ------------------------------------------------------------------ C ABI

struct thr_selector {
    thr::Selector s;
};

using thr::report_error;

extern "C" {

thr_status thr_selector_create(uint64_t seed, uint32_t flags, thr_selector** out) {
    if (!out) return report_error(THR_E_INVAL, "null output");
    if (flags & ~THR_SEL_FP32) return report_error(THR_E_INVAL, "unknown flags");
    thr_selector* h = new (std::nothrow) thr_selector;
    if (!h) return report_error(THR_E_NOMEM, "selector");
    const thr_status st = h->s.init(seed, !(flags & THR_SEL_FP32));
    if (st != THR_OK) {
        delete h;
        return st;
    }
    *out = h;
    return THR_OK;
}

void thr_selector_free(thr_selector* h) { delete h; }

thr_status thr_selector_set_params(thr_selector* h, const float* params) {
    if (!h || !params) return report_error(THR_E_INVAL, "null argument");
    return h->s.set_params(params);
}

thr_status thr_selector_get_params(const thr_selector* h, float* params) {
    if (!h || !params) return report_error(THR_E_INVAL, "null argument");
    return h->s.get_params(params);
}

thr_status thr_selector_set_norm(thr_selector* h, const float* mean, const float* istd) {
    if (!h || !mean || !istd) return report_error(THR_E_INVAL, "null argument");
    return h->s.set_norm(mean, istd);
}

thr_status thr_selector_train(thr_selector* h, const float* X, const float* T, const uint8_t* M,
                              uint32_t rows, uint32_t epochs, uint32_t batch, float lr,
                              uint64_t seed, float* loss) {
    if (!h || !X || !T || !M) return report_error(THR_E_INVAL, "null argument");
    return h->s.train(X, T, M, rows, epochs, batch, lr, seed, loss);
}

thr_status thr_selector_predict(const thr_selector* h, const float* X, uint32_t rows, float* Y) {
    if (!h || (rows && (!X || !Y))) return report_error(THR_E_INVAL, "null argument");
    return h->s.predict(X, rows, Y);
}

thr_status thr_selector_gradients(thr_selector* h, const float* X, const float* T,
                                  const uint8_t* M, uint32_t rows, float* grad, float* loss) {
    if (!h || !X || !T || !M || !grad || !loss) return report_error(THR_E_INVAL, "null argument");
    if (!rows) return report_error(THR_E_INVAL, "no rows");
    return h->s.gradients(X, T, M, rows, grad, loss);
}

thr_status thr_query_features(const thr_index* idx, const uint32_t* ids, uint32_t n, uint32_t T,
                              float* f) {
    if (!idx || !ids || !f) return report_error(THR_E_INVAL, "null argument");
    if (n == 0) return report_error(THR_E_INVAL, "n must be at least 1");
    for (uint32_t i = 0; i < n; ++i)
        if (ids[i] >= idx->nbitmaps) return report_error(THR_E_INVAL, "id out of range");
    thr::query_features(idx, ids, n, T, f);
    return THR_OK;
}

thr_status thr_index_set_selector(thr_index* idx, const thr_selector* h) {
    if (!idx) return report_error(THR_E_INVAL, "null index");
    std::lock_guard<std::mutex> lk(idx->tune_mu);
    idx->selector = h ? &h->s : nullptr;
    return THR_OK;
}

}  // extern "C"
