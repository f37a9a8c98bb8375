// Learned refinement proposal: per-patch features of the wavelet coefficients, a
// two-layer perceptron (BF16 weights, FP32 accumulation) that proposes patches for
// the next mask, and its training kernels (loss gradient and Adam).  The exact
// threshold rules still build the mask; a proposed patch only adds its nodes to
// the set T before the graded closure, so the plain criterion keeps the last word.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "sww_core.cuh"
#include "sww_kernels.h"
#include "sww_internal.h"
#include "sww_learn.h"

namespace sww {

namespace {

__device__ __forceinline__ int64_t lgid() { return int64_t(blockIdx.x) * blockDim.x + threadIdx.x; }



__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// ------------------------------------------------------------------ training

__device__ __forceinline__ void load_weights(const float* __restrict__ params, MlpWeights& w) {
    for (int k = 0; k < NF * NH; ++k) w.w1[k] = __float2bfloat16_rn(params[k]);
    for (int h = 0; h < NH; ++h) w.b1[h] = params[NF * NH + h];
    for (int h = 0; h < NH; ++h) w.w2[h] = __float2bfloat16_rn(params[NF * NH + NH + h]);
    w.b2 = params[NF * NH + 2 * NH];
}

constexpr int CHUNK = 128;

// Per-block partial sums of the weighted binary cross-entropy and its gradient with
// respect to the FP32 master parameters (the BF16 rounding is passed straight
// through): chunks of CHUNK samples, one thread per sample for the forward pass,
// then one thread per parameter summing the chunk in sample order.
__global__ void k_mlp_grad(const float* __restrict__ X, const float* __restrict__ y, int64_t n,
                           const float* __restrict__ params, float pos_w, float* __restrict__ part) {
    __shared__ MlpWeights w;
    __shared__ float xs[CHUNK][NF], as[CHUNK][NH], dz[CHUNK][NH], gs[CHUNK], ls[CHUNK];
    if (threadIdx.x == 0) load_weights(params, w);
    __syncthreads();
    constexpr int NP = MLP_PARAMS + 1;
    constexpr int PER = (NP + CHUNK - 1) / CHUNK;
    float acc[PER];
#pragma unroll
    for (int r = 0; r < PER; ++r) acc[r] = 0.f;
    for (int64_t c0 = int64_t(blockIdx.x) * CHUNK; c0 < n; c0 += int64_t(gridDim.x) * CHUNK) {
        const int s = threadIdx.x;
        const int64_t i = c0 + s;
        if (i < n) {
            for (int f = 0; f < NF; ++f) xs[s][f] = X[i * NF + f];
            float z[NH];
            const float logit = mlp_logit(w, xs[s], as[s], z);
            const float t = y[i];
            const float p = 1.f / (1.f + expf(-logit));
            const float g = pos_w * t * (p - 1.f) + (1.f - t) * p;   // d loss / d logit
            const float sp_pos = logit > 0 ? logit + log1pf(expf(-logit)) : log1pf(expf(logit));   // softplus
            ls[s] = pos_w * t * (sp_pos - logit) + (1.f - t) * sp_pos;
            gs[s] = g;
            for (int h = 0; h < NH; ++h) dz[s][h] = z[h] > 0.f ? g * __bfloat162float(w.w2[h]) : 0.f;
        } else {
            gs[s] = 0.f, ls[s] = 0.f;
            for (int f = 0; f < NF; ++f) xs[s][f] = 0.f;
            for (int h = 0; h < NH; ++h) as[s][h] = 0.f, dz[s][h] = 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int k = threadIdx.x + r * CHUNK;
            if (k >= NP) continue;
            float sum = 0.f;
            if (k < NF * NH) {
                const int f = k / NH, h = k % NH;
                for (int q = 0; q < CHUNK; ++q) sum = fmaf(dz[q][h], xs[q][f], sum);
            } else if (k < NF * NH + NH) {
                const int h = k - NF * NH;
                for (int q = 0; q < CHUNK; ++q) sum += dz[q][h];
            } else if (k < NF * NH + 2 * NH) {
                const int h = k - NF * NH - NH;
                for (int q = 0; q < CHUNK; ++q) sum = fmaf(gs[q], as[q][h], sum);
            } else if (k == MLP_PARAMS - 1) {
                for (int q = 0; q < CHUNK; ++q) sum += gs[q];
            } else {
                for (int q = 0; q < CHUNK; ++q) sum += ls[q];
            }
            acc[r] += sum;
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const int k = threadIdx.x + r * CHUNK;
        if (k < NP) part[int64_t(blockIdx.x) * NP + k] = acc[r];
    }
}

__global__ void k_mlp_grad_final(const float* __restrict__ part, int nblk, int64_t n, float* __restrict__ out) {
    constexpr int NP = MLP_PARAMS + 1;
    const int k = int(lgid());
    if (k >= NP) return;
    double s = 0;
    for (int b = 0; b < nblk; ++b) s += part[int64_t(b) * NP + k];
    out[k] = float(s / double(n > 0 ? n : 1));
}

__global__ void k_adam(float* __restrict__ params, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, int t, float lr, float b1, float b2, float eps) {
    const int k = int(lgid());
    if (k >= MLP_PARAMS) return;
    const float g = grad[k];
    m[k] = b1 * m[k] + (1.f - b1) * g;
    v[k] = b2 * v[k] + (1.f - b2) * g * g;
    const float mh = m[k] / (1.f - powf(b1, float(t)));
    const float vh = v[k] / (1.f - powf(b2, float(t)));
    params[k] -= lr * mh / (sqrtf(vh) + eps);
}

__global__ void k_mlp_predict(const float* __restrict__ X, int64_t n, const float* __restrict__ params,
                              float* __restrict__ out) {
    __shared__ MlpWeights w;
    if (threadIdx.x == 0) load_weights(params, w);
    __syncthreads();
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = lgid(); i < n; i += stride) {
        float x[NF];
#pragma unroll
        for (int f = 0; f < NF; ++f) x[f] = X[i * NF + f];
        out[i] = 1.f / (1.f + expf(-mlp_logit(w, x, nullptr, nullptr)));
    }
}

}  // namespace

MlpWeights mlp_weights(const float* params) {
    MlpWeights w{};
    for (int k = 0; k < NF * NH; ++k) w.w1[k] = __float2bfloat16_rn(params[k]);
    for (int h = 0; h < NH; ++h) w.b1[h] = params[NF * NH + h];
    for (int h = 0; h < NH; ++h) w.w2[h] = __float2bfloat16_rn(params[NF * NH + NH + h]);
    w.b2 = params[NF * NH + 2 * NH];
    return w;
}

void launch_mlp_grad(const float* X, const float* y, int64_t n, const float* params, float pos_w, float* work,
                     float* out, cudaStream_t s) {
    count_launch(2);
    k_mlp_grad<<<MLP_GRAD_BLOCKS, CHUNK, 0, s>>>(X, y, n, params, pos_w, work);
    k_mlp_grad_final<<<blocks_for(MLP_PARAMS + 1, 128), 128, 0, s>>>(work, MLP_GRAD_BLOCKS, n, out);
}

void launch_adam(float* params, const float* grad, float* m, float* v, int t, float lr, cudaStream_t s) {
    count_launch(1);
    k_adam<<<blocks_for(MLP_PARAMS, 128), 128, 0, s>>>(params, grad, m, v, t, lr, 0.9f, 0.999f, 1e-8f);
}

void launch_mlp_predict(const float* X, int64_t n, const float* params, float* out, cudaStream_t s) {
    if (n <= 0) return;
    count_launch(1);
    k_mlp_predict<<<unsigned(std::min<int64_t>(blocks_for(n, 256), 4096)), 256, 0, s>>>(X, n, params, out);
}

}  // namespace sww

// ------------------------------------------------------------------ C ABI (training)

namespace {
int learn_fail(int code, const char* msg) { return sww::set_error(code, msg); }
}  // namespace

extern "C" int sww_mlp_loss_grad(const float* X, const float* y, int64_t n, const float* params, float pos_weight,
                                 float* work, float* out, void* stream) {
    if (!X || !y || !params || !work || !out || n < 0) return learn_fail(SWW_E_ARG, "sww_mlp_loss_grad: bad argument");
    sww::launch_mlp_grad(X, y, n, params, pos_weight, work, out, static_cast<cudaStream_t>(stream));
    if (cudaGetLastError() != cudaSuccess) return learn_fail(SWW_E_CUDA, "sww_mlp_loss_grad: launch failed");
    return SWW_OK;
}

extern "C" int sww_mlp_adam(float* params, const float* grad, float* m, float* v, int t, float lr, void* stream) {
    if (!params || !grad || !m || !v || t < 1) return learn_fail(SWW_E_ARG, "sww_mlp_adam: bad argument");
    sww::launch_adam(params, grad, m, v, t, lr, static_cast<cudaStream_t>(stream));
    if (cudaGetLastError() != cudaSuccess) return learn_fail(SWW_E_CUDA, "sww_mlp_adam: launch failed");
    return SWW_OK;
}

extern "C" int sww_mlp_predict(const float* X, int64_t n, const float* params, float* out, void* stream) {
    if (!X || !params || !out || n < 0) return learn_fail(SWW_E_ARG, "sww_mlp_predict: bad argument");
    sww::launch_mlp_predict(X, n, params, out, static_cast<cudaStream_t>(stream));
    if (cudaGetLastError() != cudaSuccess) return learn_fail(SWW_E_CUDA, "sww_mlp_predict: launch failed");
    return SWW_OK;
}

namespace sww {

}  // namespace sww
