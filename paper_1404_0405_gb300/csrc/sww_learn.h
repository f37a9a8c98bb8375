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

// Blocks of the gradient kernel; the caller's work buffer holds
// MLP_GRAD_BLOCKS * (MLP_PARAMS + 1) floats.
constexpr int MLP_GRAD_BLOCKS = 256;

// BF16-rounded weights of FP32 master parameters (W1, b1, w2, b2 in that order).
MlpWeights mlp_weights(const float* params);

// features of the patches of patches_f's levels (levels above Jmin)
// (active, active_count: the all-level active list; grid: blocks of 256 for it)
template <class R>
void launch_features(const DevLevelT<R>* lvs, const Span& patches_f, const double* thr, int jmin, int jmax,
                     const int32_t* active, const int32_t* active_count, unsigned grid, cudaStream_t s);
// prop[P] = sigmoid(logit) > tau on the same patches
template <class R>
void launch_propose(const DevLevelT<R>* lvs, const Span& patches_f, const MlpWeights& w, float tau, cudaStream_t s);
// post == 0 (before a mask): pexact <- 0 and any[j - 1] <- 1 for every level j with a
// proposed patch; post == 1 (after it): prop_prev <- prop, prop <- 0
template <class R>
void launch_prop_roll(const DevLevelT<R>* lvs, const Span& patches, int post, int32_t* any, cudaStream_t s);

// out[0..MLP_PARAMS) = mean gradient, out[MLP_PARAMS] = mean loss
void launch_mlp_grad(const float* X, const float* y, int64_t n, const float* params, float pos_w, float* work,
                     float* out, cudaStream_t s);
void launch_adam(float* params, const float* grad, float* m, float* v, int t, float lr, cudaStream_t s);
void launch_mlp_predict(const float* X, int64_t n, const float* params, float* out, cudaStream_t s);

}  // namespace sww
