// Learned refinement proposal: launchers (sww_learn.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "sww_core.cuh"
#include "sww_kernels.h"

namespace sww {

// Perceptron weights as the kernels use them: BF16 W1[NF][NH] and w2[NH], FP32 biases.
struct MlpWeights {
    __nv_bfloat16 w1[NF * NH];
    float b1[NH];
    __nv_bfloat16 w2[NH];
    float b2;
};

// perceptron logit of one feature vector x[NF] (weights already BF16-rounded)
__device__ __forceinline__ float mlp_logit(const MlpWeights& w, const float* x, float* a_out, float* z_out) {
    float out = w.b2;
    for (int h = 0; h < NH; ++h) {
        float z = w.b1[h];
#pragma unroll
        for (int f = 0; f < NF; ++f) z = fmaf(x[f], __bfloat162float(w.w1[f * NH + h]), z);
        const float a = z > 0.f ? z : 0.f;
        if (a_out) a_out[h] = a, z_out[h] = z;
        out = fmaf(a, __bfloat162float(w.w2[h]), out);
    }
    return out;
}

// Blocks of the gradient kernel; the caller's work buffer holds
// MLP_GRAD_BLOCKS * (MLP_PARAMS + 1) floats.
constexpr int MLP_GRAD_BLOCKS = 256;

// BF16-rounded weights of FP32 master parameters (W1, b1, w2, b2 in that order).
MlpWeights mlp_weights(const float* params);

// out[0..MLP_PARAMS) = mean gradient, out[MLP_PARAMS] = mean loss
void launch_mlp_grad(const float* X, const float* y, int64_t n, const float* params, float pos_w, float* work,
                     float* out, cudaStream_t s);
void launch_adam(float* params, const float* grad, float* m, float* v, int t, float lr, cudaStream_t s);
void launch_mlp_predict(const float* X, int64_t n, const float* params, float* out, cudaStream_t s);

}  // namespace sww
