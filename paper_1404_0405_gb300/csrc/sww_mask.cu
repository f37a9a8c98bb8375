// List-based mask construction (Sec. 2.3): the passes of the mask over candidate
// patches instead of whole levels, so that their cost follows the active grid.
//
// Candidates of the live set at level j: the patches within one ring (every patch
// with a node within p hops; two rings for p = 4) of the seeds -- the active patches
// of level j, the patches over those of level j-1 that hold a significant
// coefficient, and the patches under the candidates of level j+1 (built from the
// top level down).  Every point the rules can add lies within five hops of a seed:
// a significant point is within one hop of a live coefficient, its neighbours and
// children within two more, the closure's parents within two more, and a point
// the closure brings down from level j+1 sits under a candidate of level j+1.
// Candidates of the ghost band: one ring (two for p = 4) around the patches that
// hold a live node, since the band reaches five hops.  Scratch bytes are zero
// outside the candidates when a mask starts: band0/band1 are cleared after use,
// the significance bytes at the start of the next mask (over the previous
// candidates); flags outside the candidates are already right (a point live or
// ghost before lies in an active patch, which is a seed).
//
// Every launch covers the members of a MaskBatch: blockIdx.y is the member, and
// blockIdx.x strides over that member's items; a member whose levels end below a
// per-level launch's level leaves at once.  A handle stepping alone is a batch of
// one.  The learned proposal's features and perceptron run in the same way
// (Sec. 2.3 extension: the exact rules keep the last word).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <stdexcept>

#include "sww_core.cuh"
#include "sww_kernels.h"
#include "sww_mask.h"

namespace sww {

namespace {

#include "sww_bodies.cuh"

constexpr int TPB = 256;

#define MEMBER const MaskMember<R>& M = B.m[blockIdx.y]

constexpr int MAXL = 12;

// The member's level records ja..jb copied into shared memory by every thread of
// the block (then a block barrier), so that the item bodies take their field
// addresses from shared memory; returns the staged array (indexed by level).  The
// mask kernels stage every level Jmin..Jmax of the member: a list left by the
// previous mask (its candidates) may name levels above this mask's top.
template <class R>
__device__ __forceinline__ const DevLevelT<R>* stage_levels(DevLevelT<R>* sl, const DevLevelT<R>* lvs, int ja, int jb) {
    const int words = int((jb - ja + 1) * sizeof(DevLevelT<R>) / sizeof(int));
    const int* src = reinterpret_cast<const int*>(lvs + ja);
    int* dst = reinterpret_cast<int*>(sl + ja);
    for (int k = threadIdx.x; k < words; k += blockDim.x) dst[k] = src[k];
    __syncthreads();
    return sl;
}
#define STAGE_LEVELS                \
    __shared__ DevLevelT<R> sl_[MAXL]; \
    const DevLevelT<R>* lvs = stage_levels(sl_, M.lvs, B.ja, M.jmax)

template <class Lv>
__device__ __forceinline__ int64_t patch_of(const Lv& L, int64_t x) {
    return x < L.nelem ? x / (L.p * L.p) : L.npatch;
}

__device__ __forceinline__ bool span_find(const Span& sp, int64_t t, int& j, int64_t& i) {
    for (j = sp.ja; j <= sp.jb; ++j)
        if (t < sp.off[j + 1 - sp.ja]) {
            i = t - sp.off[j - sp.ja];
            return true;
        }
    return false;
}

// log2(1 + x) of a feature ratio, in FP32 (the features are FP32 values)
__device__ __forceinline__ float feat_log(float x) { return log2f(1.0f + x); }

// ------------------------------------------------------------------ learned proposal

// before a mask (post == 0): the sig_any words cleared, the exact-set flags
// cleared and every level with a proposed patch marked as able to gain points
// (sig_any[j - 1]); after it (post == 1): the proposal it applied becomes the
// previous one.  Levels Jmin+1..jmax of the member.
template <class R, int CAP>
__global__ void k_prop_roll(const __grid_constant__ MaskBatch<R, CAP> B, int post) {
    MEMBER;
    int j;
    int64_t P;
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (!post && t < M.jmax + 2 && t >= 0) M.sig_any[t] = 0;
    if (!span_find(B.props, t, j, P) || j > M.jmax) return;
    const DevLevelT<R>& L = M.lvs[j];
    if (post) {
        L.prop_prev[P] = L.prop[P];
        L.prop[P] = 0;
    } else {
        L.pexact[P] = 0;
    }
}

// after the clear above: sig_any[j - 1] for every level j with a proposed patch
template <class R, int CAP>
__global__ void k_prop_any(const __grid_constant__ MaskBatch<R, CAP> B) {
    MEMBER;
    int j;
    int64_t P;
    if (!span_find(B.props, int64_t(blockIdx.x) * blockDim.x + threadIdx.x, j, P) || j > M.jmax) return;
    if (M.lvs[j].prop[P]) M.sig_any[j - 1] = 1;
}

// Own features of a patch: log2(1 + max|h~|/eps_h) over its live odd nodes,
// log2(1 + max|u~|/eps_u) over its live interior edges and the pair coefficients of
// the coarse edges under its even nodes, and the fraction of its nodes that are
// live.  An inactive patch has no live point: all three are 0 (k_feat_clear, one
// thread per patch; the pole entry is cleared too and recomputed when listed).
// The active patches of levels Jmin+1..jb come from the active list, one warp per
// entry (one lane per node of the patch).
template <class R, int CAP>
__global__ void k_feat_clear(const __grid_constant__ MaskBatch<R, CAP> B) {
    MEMBER;
    int j;
    int64_t P;
    if (!M.learn || !span_find(B.patches_f, int64_t(blockIdx.x) * blockDim.x + threadIdx.x, j, P) || j > M.jb)
        return;
    const DevLevelT<R>& L = M.lvs[j];
    const int64_t np1 = L.npatch + 1;
    if (P == L.npatch || !L.pflag[P]) L.pfeat[0 * np1 + P] = 0.f, L.pfeat[1 * np1 + P] = 0.f, L.pfeat[6 * np1 + P] = 0.f;
}

template <class R, int CAP>
__global__ void k_feat_own(const __grid_constant__ MaskBatch<R, CAP> B) {
    MEMBER;
    if (!M.learn) return;
    STAGE_LEVELS;
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
    // the thresholds once per thread, in FP32
    const float eh = float(M.thr[0] > 0 ? M.thr[0] : 1.0), eu = float(M.thr[1] > 0 ? M.thr[1] : 1.0);
    for (int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; w < *M.active_count; w += nw) {
        const int32_t ent = M.active[w];
        const int j = ent >> LVL_SHIFT;
        if (j <= B.ja || j > M.jb) continue;
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
            L.pfeat[0 * np1 + P] = feat_log(float(mh) / eh);
            L.pfeat[1 * np1 + P] = feat_log(float(mu) / eu);
            L.pfeat[6 * np1 + P] = float(live) / float(nn);
        }
    }
}

// Context features (one thread per patch): the coarse patch's own features (zero on
// the level above Jmin, which carries no coefficients), the maxima over the
// neighbour patches, and the level's depth in Jmin..Jmax.
template <class R, int CAP>
__global__ void k_feat_ctx(const __grid_constant__ MaskBatch<R, CAP> B) {
    MEMBER;
    int j;
    int64_t P;
    if (!M.learn || !span_find(B.patches_f, int64_t(blockIdx.x) * blockDim.x + threadIdx.x, j, P) || j > M.jb)
        return;
    const DevLevelT<R>& L = M.lvs[j];
    const DevLevelT<R>& C = M.lvs[j - 1];
    const int64_t np1 = L.npatch + 1, cnp1 = C.npatch + 1;
    float f2 = 0, f3 = 0, f4 = 0, f5 = 0;
    const int32_t cp = L.ppar[P];
    if (j - 1 > B.ja && cp >= 0) f2 = C.pfeat[0 * cnp1 + cp], f3 = C.pfeat[1 * cnp1 + cp];
    // the neighbours eight at a time, each group's loads issued together (max is
    // order-independent)
#pragma unroll
    for (int k0 = 0; k0 < NB; k0 += 8) {
        int32_t Q[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) Q[k] = L.pnbr[(k0 + k) * np1 + P];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (Q[k] >= 0) {
                f4 = fmaxf(f4, L.pfeat[0 * np1 + Q[k]]);
                f5 = fmaxf(f5, L.pfeat[1 * np1 + Q[k]]);
            }
        if (Q[7] < 0) break;
    }
    L.pfeat[2 * np1 + P] = f2;
    L.pfeat[3 * np1 + P] = f3;
    L.pfeat[4 * np1 + P] = f4;
    L.pfeat[5 * np1 + P] = f5;
    L.pfeat[7 * np1 + P] = float(j - B.ja) / float(M.jmax > B.ja ? M.jmax - B.ja : 1);
}

// the proposal: a patch that is not active yet and whose logit passes the member's
// threshold (an active patch stays under the exact rules)
template <class R, int CAP>
__global__ void k_propose(const __grid_constant__ MaskBatch<R, CAP> B) {
    MEMBER;
    __shared__ MlpWeights w;   // staged once per block
    if (M.learn < 2) return;
    for (int k = threadIdx.x; k < int(sizeof(MlpWeights) / 4); k += blockDim.x)
        reinterpret_cast<int*>(&w)[k] = reinterpret_cast<const int*>(M.net)[k];
    __syncthreads();
    int j;
    int64_t P;
    if (!span_find(B.patches_f, int64_t(blockIdx.x) * blockDim.x + threadIdx.x, j, P) || j > M.jb) return;
    const DevLevelT<R>& L = M.lvs[j];
    const int64_t np1 = L.npatch + 1;
    const bool active = P < L.npatch ? L.pflag[P] != 0 : L.pfeat[6 * np1 + P] > 0.f;
    float x[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) x[f] = L.pfeat[f * np1 + P];
    L.prop[P] = (!active && mlp_logit(w, x, nullptr, nullptr) > M.logit_tau) ? 1 : 0;
}

// ------------------------------------------------------------------ mask passes

// all candidate flags of the member's levels ja..jb to zero
template <class R, int CAP>
__global__ void k_clear_flags(const __grid_constant__ MaskBatch<R, CAP> B) {
    MEMBER;
    int j;
    int64_t P;
    if (!span_find(B.patches, int64_t(blockIdx.x) * blockDim.x + threadIdx.x, j, P) || j > M.jb) return;
    const DevLevelT<R>& L = M.lvs[j];
    L.zflag[P] = 0, L.sflag[P] = 0, L.cflag[P] = 0, L.lflag[P] = 0, L.gflag[P] = 0;
}

// the significance bytes of the previous mask, over its candidates (they stay
// readable until the next mask)
template <class R, int CAP>
__global__ void k_clear_sig_list(const __grid_constant__ MaskBatch<R, CAP> B) {
    MEMBER;
    STAGE_LEVELS;
    DevLevelT<R> none{};
    ITEMS(K_NODE, lvs, none, M.cand, M.cand_count, B.P) { L.sig[id] = 0; });
}

// significance over the items of the active patches above Jmin; the patch of each
// significant coefficient is recorded
template <class R, int CAP>
__global__ void k_sig_list(const __grid_constant__ MaskBatch<R, CAP> B) {
    MEMBER;
    STAGE_LEVELS;
    DevLevelT<R> none{};
    const R eh = sig_thr<R>(M.thr[0]), eu = sig_thr<R>(M.thr[1]);
    int32_t* sig_any = M.sig_any;
    ITEMS(K_NODE | K_EDGE | K_CEDGE, lvs, none, M.active, M.active_count, B.P) {
        if (L.J == B.ja) return;
        const DevLevelT<R>& C = lvs[L.J - 1];
        bool any;
        if (kind == K_NODE) {
            any = sig_node(L, id, eh);
        } else if (kind == K_EDGE) {
            any = sig_edge(L, id, eu);
        } else {
            const int32_t ce = L.f2c[el];
            if (ce < 0) return;
            any = sig_cedge(L, C, id * C.nelem + ce, eu);
        }
        if (any) {
            sig_any[L.J] = 1;
            L.sflag[el < 0 ? L.npatch : el / (L.p * L.p)] = 1;
        }
    });
}

// seeds: every active patch, and the patches over an active patch holding a
// significant coefficient (one thread per list entry)
template <class R, int CAP>
__global__ void k_seed(const __grid_constant__ MaskBatch<R, CAP> B) {
    MEMBER;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < *M.active_count; t += stride) {
        const int32_t ent = M.active[t];
        const int j = ent >> LVL_SHIFT;
        const int64_t P = ent & PATCH_MASK;
        const DevLevelT<R>& L = M.lvs[j];
        L.zflag[P] = 1;
        if (j < M.jb && L.sflag[P]) {
            const DevLevelT<R>& F = M.lvs[j + 1];
            for (int q = 0; q < 4; ++q) {
                const int32_t c = L.pchild[q * (L.npatch + 1) + P];
                if (c >= 0) F.zflag[c] = 1;
            }
        }
    }
}

// whether a neighbour patch of P (pnbr, -1 padded) has its byte set in `in` (bytes
// 0 or 1): the neighbours read eight at a time, each group's loads issued together
template <class Lv>
__device__ __forceinline__ uint8_t nbr_any(const Lv& L, int64_t P, int64_t np1, const uint8_t* in) {
    static_assert(NB % 8 == 0, "neighbour groups");
    uint8_t c = 0;
#pragma unroll
    for (int k0 = 0; k0 < NB; k0 += 8) {
        int32_t Q[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) Q[k] = L.pnbr[(k0 + k) * np1 + P];
#pragma unroll
        for (int k = 0; k < 8; ++k)
            if (Q[k] >= 0) c |= in[Q[k]];
        if (c || Q[7] < 0) break;
    }
    return c;
}

// one ring around the flagged patches of level j: out = in + neighbours of in.  The
// final pass writes the candidates and marks the patch under each candidate as a
// seed of level j-1.  `all`: every patch is a candidate.
template <class R, int CAP>
__global__ void k_ring(const __grid_constant__ MaskBatch<R, CAP> B, int j, int src, int final_pass, int push, int all) {
    MEMBER;
    if (j > M.jb) return;
    const DevLevelT<R>& L = M.lvs[j];
    const int64_t P = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (P > L.npatch) return;
    const int64_t np1 = L.npatch + 1;
    const uint8_t* in = src == 0 ? L.zflag : L.gflag;
    uint8_t c = all ? 1 : in[P];
    if (!c) c = nbr_any(L, P, np1, in);
    if (final_pass) {
        L.cflag[P] = c;
        if (c && push && L.ppar[P] >= 0) M.lvs[j - 1].zflag[L.ppar[P]] = 1;
    } else {
        L.gflag[P] = c;
    }
}

// ghost candidates: one ring around the patches with a live node; with two rings
// the first pass goes through cflag (no longer needed once the candidate lists are
// built).  Jmin: every patch.
template <class R, int CAP>
__global__ void k_gring(const __grid_constant__ MaskBatch<R, CAP> B, int pass) {
    MEMBER;
    int j;
    int64_t P;
    if (!span_find(B.patches, int64_t(blockIdx.x) * blockDim.x + threadIdx.x, j, P) || j > M.jb) return;
    const DevLevelT<R>& L = M.lvs[j];
    const int64_t np1 = L.npatch + 1;
    const uint8_t* in = pass == 0 ? L.lflag : L.cflag;
    uint8_t c = j == B.ja ? 1 : in[P];
    if (!c) c = nbr_any(L, P, np1, in);
    (pass == 0 && B.rings == 2 ? L.cflag : L.gflag)[P] = c;
}

// compact flags of every level (one block per level) into level-tagged lists:
// which 1 candidates (cflag -> cand), 2 ghost candidates (gflag -> gcand)
template <class R, int CAP>
__global__ void k_flag_scan(const __grid_constant__ MaskBatch<R, CAP> B, int which) {
    MEMBER;
    const int j = B.ja + int(blockIdx.x);
    if (j > M.jb) return;
    const DevLevelT<R>& L = M.lvs[j];
    const uint8_t* flag = which == 1 ? L.cflag : L.gflag;
    int32_t* out = which == 1 ? L.cand : L.gcand;
    int32_t* nout = which == 1 ? L.ncand : L.ngcand;
    const int n = compact_flags(flag, L.npatch + 1, int32_t(L.J) << LVL_SHIFT, out);
    if (threadIdx.x == 0) *nout = n;
}

// concatenation of the candidate lists of the member's levels ja..jb (one block)
template <class R, int CAP>
__global__ void k_cat(const __grid_constant__ MaskBatch<R, CAP> B, int which) {
    MEMBER;
    int32_t* all = which == 1 ? M.cand : M.gcand;
    int32_t* count = which == 1 ? M.cand_count : M.gcand_count;
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int j = B.ja; j <= M.jb; ++j) {
        const DevLevelT<R>& L = M.lvs[j];
        const int32_t* src = which == 1 ? L.cand : L.gcand;
        const int n = which == 1 ? *L.ncand : *L.ngcand;
        for (int i = threadIdx.x; i < n; i += blockDim.x) all[base + i] = src[i];
        __syncthreads();
        if (threadIdx.x == 0) base += n;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = base;
}

template <class R, int CAP>
__global__ void k_adjacent_list(const __grid_constant__ MaskBatch<R, CAP> B) {
    MEMBER;
    STAGE_LEVELS;
    DevLevelT<R> none{};
    ITEMS(K_NODE, lvs, none, M.cand, M.cand_count, B.P) {
        if (L.J == B.ja) return;
        adjacent_node(L, lvs[L.J - 1], L.J - 1 > B.ja, id);
    });
}

// graded closure at level j (from the top level down)
template <class R, int CAP>
__global__ void k_close_list(const __grid_constant__ MaskBatch<R, CAP> B, int j) {
    MEMBER;
    if (j > M.jb) return;
    STAGE_LEVELS;
    const DevLevelT<R>& F = lvs[j];
    const bool has_finer = j < M.jb;
    const DevLevelT<R>& Fp = lvs[has_finer ? j + 1 : j];
    ITEMS(K_NODE, (const DevLevelT<R>*)nullptr, F, F.cand, F.ncand, B.P) { close_node(L, Fp, has_finer, id); });
}

template <class R, int CAP>
__global__ void k_live_list(const __grid_constant__ MaskBatch<R, CAP> B) {
    MEMBER;
    STAGE_LEVELS;
    DevLevelT<R> none{};
    ITEMS(K_NODE, lvs, none, M.cand, M.cand_count, B.P) {
        if (live_node(L, id, L.J == B.ja)) L.lflag[patch_of(L, id)] = 1;
    });
}

template <class R, int CAP>
__global__ void k_live_edges_list(const __grid_constant__ MaskBatch<R, CAP> B) {
    MEMBER;
    STAGE_LEVELS;
    DevLevelT<R> none{};
    ITEMS(K_EDGE, lvs, none, M.cand, M.cand_count, B.P) { live_edge(L, id); });
}

template <class R, int CAP>
__global__ void k_dilate_list(const __grid_constant__ MaskBatch<R, CAP> B, int forward) {
    MEMBER;
    if (M.jb == B.ja) return;
    STAGE_LEVELS;
    DevLevelT<R> none{};
    ITEMS(K_NODE, lvs, none, M.gcand, M.gcand_count, B.P) {
        if (L.J == B.ja) return;
        dilate_node(L, id, forward != 0);
    });
}

template <class R, int CAP>
__global__ void k_ghost_list(const __grid_constant__ MaskBatch<R, CAP> B, int in_band1) {
    MEMBER;
    if (M.jb == B.ja) return;
    STAGE_LEVELS;
    DevLevelT<R> none{};
    ITEMS(K_NODE | K_EDGE, lvs, none, M.gcand, M.gcand_count, B.P) {
        if (L.J == B.ja) return;
        const uint8_t* band = in_band1 ? L.band1 : L.band0;
        if (kind == K_NODE)
            ghost_node(L, id, band);
        else
            ghost_edge(L, id, band);
    });
}

template <class R, int CAP>
__global__ void k_covered_list(const __grid_constant__ MaskBatch<R, CAP> B) {
    MEMBER;
    if (M.jb == B.ja) return;
    STAGE_LEVELS;
    DevLevelT<R> none{};
    const int jtop = M.jb;
    ITEMS(K_NODE, lvs, none, M.cand, M.cand_count, B.P) {
        if (L.J >= jtop) return;
        covered_node(L, lvs[L.J + 1], id);
    });
}

// before the new patch flags: the learned proposal's counts (misses, over-refined,
// proposed; levels above Jmin) and the old flags cleared, over the candidates (a
// superset of the old active patches and of the exact set)
template <class R, int CAP>
__global__ void k_pre_flags(const __grid_constant__ MaskBatch<R, CAP> B) {
    MEMBER;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < *M.cand_count; t += stride) {
        const int32_t ent = M.cand[t];
        const int j = ent >> LVL_SHIFT;
        const int64_t P = ent & PATCH_MASK;
        const DevLevelT<R>& L = M.lvs[j];
        if (P >= L.npatch) continue;
        if (M.lstat && j > B.ja) {
            if (L.pexact[P] && !L.pflag[P]) atomicAdd(&M.lstat[0], 1ull);
            if (L.prop_prev[P] && !L.pexact[P]) atomicAdd(&M.lstat[1], 1ull);
            if (L.prop[P]) atomicAdd(&M.lstat[2], 1ull);
        }
        L.pflag[P] = 0;
    }
}

// patch flags over the ghost candidates (every patch with a live or ghost point is
// one), and the band bytes of their nodes cleared; a block per entry
template <class R, int CAP>
__global__ void k_flags_list(const __grid_constant__ MaskBatch<R, CAP> B) {
    MEMBER;
    for (int64_t t = blockIdx.x; t < *M.gcand_count; t += gridDim.x) {
        const int32_t ent = M.gcand[t];
        const int j = ent >> LVL_SHIFT;
        const int64_t P = ent & PATCH_MASK;
        const DevLevelT<R>& L = M.lvs[j];
        if (P == L.npatch) {
            if (threadIdx.x < 2) {
                const int64_t v = L.nelem + threadIdx.x;
                L.band0[v] = 0, L.band1[v] = 0;
            }
            continue;
        }
        const int64_t pp = L.p * L.p;
        int any = 0;
        for (int64_t l = threadIdx.x; l < pp; l += blockDim.x) {
            const int64_t e = P * pp + l;
            if ((L.nflag[e] | L.eflag[e] | L.eflag[L.nelem + e] | L.eflag[2 * L.nelem + e]) & AVAIL) any = 1;
            L.band0[e] = 0, L.band1[e] = 0;
        }
        any = __syncthreads_or(any);
        if (threadIdx.x == 0) L.pflag[P] = uint8_t(any);
    }
}

// the ascending patch list of each of the member's levels ja..jb (one block per level)
template <class R, int CAP>
__global__ void k_patch_scan_b(const __grid_constant__ MaskBatch<R, CAP> B) {
    MEMBER;
    const int j = B.ja + int(blockIdx.x);
    if (j > M.jb) return;
    patch_scan_level(M.lvs[j]);
}

// the member's all-level and irregular lists (one block per member)
template <class R, int CAP>
__global__ void k_concat_b(const __grid_constant__ MaskBatch<R, CAP> B) {
    MEMBER;
    concat_lists(M.lvs, B.ja, M.jmax, M.all, M.all_count, M.irr, M.irr_count);
}

// the point work lists of the member's levels from its all-level list
template <class R, int CAP>
__global__ void k_wl_build_b(const __grid_constant__ MaskBatch<R, CAP> B) {
    MEMBER;
    STAGE_LEVELS;
    DevLevelT<R> none{};
    ITEMS(K_NODE | K_EDGE, lvs, none, M.all, M.all_count, B.P) { wl_item(L, kind, id); });
}

}  // namespace

namespace {
// one launch of `kernel` over gx blocks per member (threads: TPB unless given)
template <class K, class... A>
void go(K kernel, unsigned gx, unsigned nm, unsigned threads, cudaStream_t s, const A&... args) {
    count_launch(1);
    kernel<<<dim3(std::max(gx, 1u), nm), threads, 0, s>>>(args...);
}
}  // namespace

template <class R, int CAP>
void launch_proposal_batch(const MaskBatch<R, CAP>& b, unsigned grid, int post, cudaStream_t s) {
    if (b.nm < 1 || b.nm > CAP) throw std::runtime_error("mask batch size");
    const int64_t np = b.props.off[b.props.jb + 1 - b.props.ja];
    bool learn = false;
    for (int i = 0; i < b.nm; ++i) learn = learn || b.m[i].learn > 0;
    if (post) {
        if (np > 0) go(k_prop_roll<R, CAP>, blocks_for(np, TPB), unsigned(b.nm), TPB, s, b, 1);
        return;
    }
    // the sig_any words are cleared in the same launch (at least one block per member)
    go(k_prop_roll<R, CAP>, std::max<unsigned>(1, blocks_for(np, TPB)), unsigned(b.nm), TPB, s, b, 0);
    const int64_t nf = b.patches_f.off[b.patches_f.jb + 1 - b.patches_f.ja];
    if (learn && b.jb_max > b.ja && nf > 0) {
        go(k_feat_clear<R, CAP>, blocks_for(nf, TPB), unsigned(b.nm), TPB, s, b);
        go(k_feat_own<R, CAP>, grid, unsigned(b.nm), TPB, s, b);
        go(k_feat_ctx<R, CAP>, blocks_for(nf, TPB), unsigned(b.nm), TPB, s, b);
        go(k_propose<R, CAP>, blocks_for(nf, TPB), unsigned(b.nm), TPB, s, b);
    }
    if (np > 0) go(k_prop_any<R, CAP>, blocks_for(np, TPB), unsigned(b.nm), TPB, s, b);
}

template <class R, int CAP>
void launch_mask_batch(const MaskBatch<R, CAP>& b, unsigned grid, cudaStream_t s) {
    if (b.nm < 1 || b.nm > CAP) throw std::runtime_error("mask batch size");
    const int ja = b.ja, jb = b.jb_max;
    const int64_t npatches = b.patches.off[jb + 1 - ja];
    // seeds
    go(k_clear_flags<R, CAP>, blocks_for(npatches, TPB), unsigned(b.nm), TPB, s, b);
    go(k_clear_sig_list<R, CAP>, grid, unsigned(b.nm), TPB, s, b);
    go(k_sig_list<R, CAP>, grid, unsigned(b.nm), TPB, s, b);
    go(k_seed<R, CAP>, grid, unsigned(b.nm), TPB, s, b);
    // candidates, from the top level down (Jmin and whole-lozenge levels: every patch)
    for (int j = jb; j >= ja; --j) {
        const int64_t np1 = b.patches.off[j + 1 - ja] - b.patches.off[j - ja];
        const int all = (j == ja || np1 <= 11) ? 1 : 0;
        const int push = j - 1 > ja ? 1 : 0;
        const unsigned g = blocks_for(np1, TPB);
        if (b.rings == 2 && !all) {
            go(k_ring<R, CAP>, g, unsigned(b.nm), TPB, s, b, j, 0, 0, 0, 0);
            go(k_ring<R, CAP>, g, unsigned(b.nm), TPB, s, b, j, 1, 1, push, 0);
        } else {
            go(k_ring<R, CAP>, g, unsigned(b.nm), TPB, s, b, j, 0, 1, push, all);
        }
    }
    go(k_flag_scan<R, CAP>, unsigned(jb - ja + 1), unsigned(b.nm), 1024, s, b, 1);
    go(k_cat<R, CAP>, 1u, unsigned(b.nm), 1024, s, b, 1);
    // the set T, its closure from the top level down, live flags
    go(k_adjacent_list<R, CAP>, grid, unsigned(b.nm), TPB, s, b);
    for (int j = jb; j > ja; --j) go(k_close_list<R, CAP>, grid, unsigned(b.nm), TPB, s, b, j);
    go(k_live_list<R, CAP>, grid, unsigned(b.nm), TPB, s, b);
    go(k_live_edges_list<R, CAP>, grid, unsigned(b.nm), TPB, s, b);
    // ghost candidates (every patch of Jmin), ghost band, covered nodes
    go(k_gring<R, CAP>, blocks_for(npatches, TPB), unsigned(b.nm), TPB, s, b, 0);
    if (b.rings == 2) go(k_gring<R, CAP>, blocks_for(npatches, TPB), unsigned(b.nm), TPB, s, b, 1);
    go(k_flag_scan<R, CAP>, unsigned(jb - ja + 1), unsigned(b.nm), 1024, s, b, 2);
    go(k_cat<R, CAP>, 1u, unsigned(b.nm), 1024, s, b, 2);
    if (jb > ja) {
        for (int h = 0; h < b.hops; ++h) go(k_dilate_list<R, CAP>, grid, unsigned(b.nm), TPB, s, b, h % 2 == 0 ? 1 : 0);
        go(k_ghost_list<R, CAP>, grid, unsigned(b.nm), TPB, s, b, b.hops % 2 == 1 ? 1 : 0);
        go(k_covered_list<R, CAP>, grid, unsigned(b.nm), TPB, s, b);
    }
    // patch flags: the old ones cleared over the candidates (a superset of the old
    // active patches), the new ones set over the ghost candidates (a superset of
    // the patches with a live or ghost point); then the level lists
    go(k_pre_flags<R, CAP>, grid, unsigned(b.nm), TPB, s, b);
    go(k_flags_list<R, CAP>, grid, unsigned(b.nm), 64, s, b);
    go(k_patch_scan_b<R, CAP>, unsigned(jb - ja + 1), unsigned(b.nm), 1024, s, b);
}

template <class R, int CAP>
void launch_concat_batch(const MaskBatch<R, CAP>& b, unsigned grid, cudaStream_t s) {
    if (b.nm < 1 || b.nm > CAP) throw std::runtime_error("mask batch size");
    go(k_concat_b<R, CAP>, 1u, unsigned(b.nm), 1024, s, b);
    go(k_wl_build_b<R, CAP>, grid, unsigned(b.nm), TPB, s, b);
}

#define MASK_INST(R, CAP)                                                                                   \
    template void launch_mask_batch<R, CAP>(const MaskBatch<R, CAP>&, unsigned, cudaStream_t);            \
    template void launch_proposal_batch<R, CAP>(const MaskBatch<R, CAP>&, unsigned, int, cudaStream_t);   \
    template void launch_concat_batch<R, CAP>(const MaskBatch<R, CAP>&, unsigned, cudaStream_t);
MASK_INST(double, 1)
MASK_INST(float, 1)
MASK_INST(double, MASK_BATCH_MAX)
MASK_INST(float, MASK_BATCH_MAX)

}  // namespace sww
