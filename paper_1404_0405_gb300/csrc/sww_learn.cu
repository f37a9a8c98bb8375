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

__device__ __forceinline__ bool lfind(const Span& sp, int64_t t, int& j, int64_t& i) {
    for (j = sp.ja; j <= sp.jb; ++j)
        if (t < sp.off[j + 1 - sp.ja]) {
            i = t - sp.off[j - sp.ja];
            return true;
        }
    return false;
}

__device__ __forceinline__ float feat_log(double x) { return float(log2(1.0 + x)); }

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Own features of a patch: log2(1 + max|h~|/eps_h) over its live odd nodes,
// log2(1 + max|u~|/eps_u) over its live interior edges and the pair coefficients of
// the coarse edges under its even nodes, and the fraction of its nodes that are
// live.  An inactive patch has no live point: all three are 0 (k_feat_clear, one
// thread per patch; the pole entry is cleared too and recomputed when listed).
// The active patches of levels ja..jb come from the active list, one warp per
// entry (one lane per node of the patch).
template <class R>
__global__ void k_feat_clear(const DevLevelT<R>* __restrict__ lvs, Span sp) {
    int j;
    int64_t P;
    if (!lfind(sp, lgid(), j, P)) return;
    const DevLevelT<R>& L = lvs[j];
    const int64_t np1 = L.npatch + 1;
    if (P == L.npatch || !L.pflag[P]) L.pfeat[0 * np1 + P] = 0.f, L.pfeat[1 * np1 + P] = 0.f, L.pfeat[6 * np1 + P] = 0.f;
}

template <class R>
__global__ void k_feat_own(const DevLevelT<R>* __restrict__ lvs, int ja, int jb, const int32_t* __restrict__ list,
                           const int32_t* __restrict__ count, const double* __restrict__ thr) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t w = lgid() >> 5; w < *count; w += nw) {
        const int32_t ent = list[w];
        const int j = ent >> LVL_SHIFT;
        if (j < ja || j > jb) continue;
        const int64_t P = ent & PATCH_MASK;
        const DevLevelT<R>& L = lvs[j];
        const DevLevelT<R>& C = lvs[j - 1];
        const int64_t pp = L.p * L.p, np1 = L.npatch + 1;
        const bool pole = P == L.npatch;
        R mh = R(0), mu = R(0);
        int live = 0;
        const int64_t nn = pole ? 2 : pp;
        for (int64_t l = lane; l < nn; l += 32) {
            const int64_t v = pole ? L.nelem + l : P * pp + l;
            const uint8_t f = L.nflag[v];
            live += (f & LIVE) ? 1 : 0;
            if ((f & LIVE) && L.f2c[v] < 0) mh = fmax(mh, fabs(L.hdet[v]));
            if (pole) continue;
            for (int o = 0; o < 3; ++o) {
                const int64_t e = o * L.nelem + v;
                if ((L.eflag[e] & LIVE) && L.fe_kind[e] == 2) mu = fmax(mu, fabs(L.ui[e]));
            }
            const int32_t ce = L.f2c[v];
            if (ce >= 0 && ce < C.nelem) {
                for (int o = 0; o < 3; ++o) {
                    const int64_t E = o * C.nelem + ce;
                    const int32_t h0 = C.half[E], h1 = C.half[C.E + E];
                    if ((L.eflag[h0] | L.eflag[h1]) & LIVE) mu = fmax(mu, fabs(L.ue[E]));
                }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            mh = fmax(mh, __shfl_xor_sync(0xffffffffu, mh, o));
            mu = fmax(mu, __shfl_xor_sync(0xffffffffu, mu, o));
            live += __shfl_xor_sync(0xffffffffu, live, o);
        }
        if (lane == 0) {
            const double eh = thr[0] > 0 ? thr[0] : 1.0, eu = thr[1] > 0 ? thr[1] : 1.0;
            L.pfeat[0 * np1 + P] = feat_log(double(mh) / eh);
            L.pfeat[1 * np1 + P] = feat_log(double(mu) / eu);
            L.pfeat[6 * np1 + P] = float(live) / float(nn);
        }
    }
}

// Context features (one thread per patch): the coarse patch's own features (zero on
// the level above Jmin, which carries no coefficients), the maxima over the
// neighbour patches, and the level's depth in Jmin..Jmax.
template <class R>
__global__ void k_feat_ctx(const DevLevelT<R>* __restrict__ lvs, Span sp, int jmin, int jmax) {
    int j;
    int64_t P;
    if (!lfind(sp, lgid(), j, P)) return;
    const DevLevelT<R>& L = lvs[j];
    const DevLevelT<R>& C = lvs[j - 1];
    const int64_t np1 = L.npatch + 1, cnp1 = C.npatch + 1;
    float f2 = 0, f3 = 0, f4 = 0, f5 = 0;
    const int32_t cp = L.ppar[P];
    if (j - 1 > jmin && cp >= 0) f2 = C.pfeat[0 * cnp1 + cp], f3 = C.pfeat[1 * cnp1 + cp];
    for (int k = 0; k < NB; ++k) {
        const int32_t Q = L.pnbr[k * np1 + P];
        if (Q < 0) break;
        f4 = fmaxf(f4, L.pfeat[0 * np1 + Q]);
        f5 = fmaxf(f5, L.pfeat[1 * np1 + Q]);
    }
    L.pfeat[2 * np1 + P] = f2;
    L.pfeat[3 * np1 + P] = f3;
    L.pfeat[4 * np1 + P] = f4;
    L.pfeat[5 * np1 + P] = f5;
    L.pfeat[7 * np1 + P] = float(j - jmin) / float(jmax > jmin ? jmax - jmin : 1);
}

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

template <class R>
__global__ void k_propose(const DevLevelT<R>* __restrict__ lvs, Span sp, MlpWeights wp, float logit_tau) {
    __shared__ MlpWeights w;   // staged once per block (indexed loads from the parameter would go to local memory)
    if (threadIdx.x == 0) w = wp;
    __syncthreads();
    int j;
    int64_t P;
    if (!lfind(sp, lgid(), j, P)) return;
    const DevLevelT<R>& L = lvs[j];
    const int64_t np1 = L.npatch + 1;
    // only patches that are not active yet: an active patch stays under the exact rules
    const bool active = P < L.npatch ? L.pflag[P] != 0 : L.pfeat[6 * np1 + P] > 0.f;
    float x[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) x[f] = L.pfeat[f * np1 + P];
    L.prop[P] = (!active && mlp_logit(w, x, nullptr, nullptr) > logit_tau) ? 1 : 0;
}

// before a mask (post == 0): clear the exact-set flags and mark every level with a
// proposed patch as able to gain points (any[j - 1], the flag a tail level checks);
// after it (post == 1): the proposal it applied becomes the previous one
template <class R>
__global__ void k_prop_roll(const DevLevelT<R>* __restrict__ lvs, Span sp, int post, int32_t* any) {
    int j;
    int64_t P;
    if (!lfind(sp, lgid(), j, P)) return;
    const DevLevelT<R>& L = lvs[j];
    if (post) {
        L.prop_prev[P] = L.prop[P];
        L.prop[P] = 0;
    } else {
        L.pexact[P] = 0;
        if (L.prop[P]) any[j - 1] = 1;
    }
}

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

template <class R>
void launch_features(const DevLevelT<R>* lvs, const Span& patches_f, const double* thr, int jmin, int jmax,
                     const int32_t* active, const int32_t* active_count, unsigned grid, cudaStream_t s) {
    const int64_t n = patches_f.off[patches_f.jb + 1 - patches_f.ja];
    if (n <= 0) return;
    count_launch(3);
    k_feat_clear<R><<<blocks_for(n, 256), 256, 0, s>>>(lvs, patches_f);
    k_feat_own<R><<<grid, 256, 0, s>>>(lvs, patches_f.ja, patches_f.jb, active, active_count, thr);
    k_feat_ctx<R><<<blocks_for(n, 256), 256, 0, s>>>(lvs, patches_f, jmin, jmax);
}

template <class R>
void launch_propose(const DevLevelT<R>* lvs, const Span& patches_f, const MlpWeights& w, float tau, cudaStream_t s) {
    const int64_t n = patches_f.off[patches_f.jb + 1 - patches_f.ja];
    if (n <= 0) return;
    count_launch(1);
    const float logit_tau = std::log(tau / (1.f - tau));
    k_propose<R><<<blocks_for(n, 256), 256, 0, s>>>(lvs, patches_f, w, logit_tau);
}

template <class R>
void launch_prop_roll(const DevLevelT<R>* lvs, const Span& patches, int post, int32_t* any, cudaStream_t s) {
    const int64_t n = patches.off[patches.jb + 1 - patches.ja];
    if (n <= 0) return;
    count_launch(1);
    k_prop_roll<R><<<blocks_for(n, 256), 256, 0, s>>>(lvs, patches, post, any);
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

template void launch_features<double>(const DevLevelT<double>*, const Span&, const double*, int, int, const int32_t*,
                                      const int32_t*, unsigned, cudaStream_t);
template void launch_features<float>(const DevLevelT<float>*, const Span&, const double*, int, int, const int32_t*,
                                     const int32_t*, unsigned, cudaStream_t);
template void launch_propose<double>(const DevLevelT<double>*, const Span&, const MlpWeights&, float, cudaStream_t);
template void launch_propose<float>(const DevLevelT<float>*, const Span&, const MlpWeights&, float, cudaStream_t);
template void launch_prop_roll<double>(const DevLevelT<double>*, const Span&, int, int32_t*, cudaStream_t);
template void launch_prop_roll<float>(const DevLevelT<float>*, const Span&, int, int32_t*, cudaStream_t);

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
