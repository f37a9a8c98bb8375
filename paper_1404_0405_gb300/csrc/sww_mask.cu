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
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "sww_core.cuh"
#include "sww_kernels.h"
#include "sww_mask.h"

namespace sww {

namespace {

#include "sww_bodies.cuh"

constexpr int TPB = 256;

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

// all candidate flags of the levels of a patch span to zero
template <class R>
__global__ void k_clear_flags(const DevLevelT<R>* __restrict__ lvs, Span sp) {
    int j;
    int64_t P;
    if (!span_find(sp, gid(), j, P)) return;
    const DevLevelT<R>& L = lvs[j];
    L.zflag[P] = 0, L.sflag[P] = 0, L.cflag[P] = 0, L.lflag[P] = 0, L.gflag[P] = 0;
}

// significance over the items of the active patches above Jmin; the patch of each
// significant coefficient is recorded
template <class R>
__global__ void k_sig_list(const DevLevelT<R>* __restrict__ lvs, const int32_t* list, const int32_t* count, int P,
                           int jmin, const double* __restrict__ thr, int32_t* sig_any) {
    DevLevelT<R> none{};
    ITEMS(K_NODE | K_EDGE | K_CEDGE, lvs, none, list, count, P) {
        if (L.J == jmin) return;
        const DevLevelT<R>& C = lvs[L.J - 1];
        bool any;
        if (kind == K_NODE) {
            any = sig_node(L, id, thr[0]);
        } else if (kind == K_EDGE) {
            any = sig_edge(L, id, thr[1]);
        } else {
            const int32_t ce = L.f2c[el];
            if (ce < 0) return;
            any = sig_cedge(L, C, id * C.nelem + ce, thr[1]);
        }
        if (any) {
            sig_any[L.J] = 1;
            L.sflag[el < 0 ? L.npatch : el / (L.p * L.p)] = 1;
        }
    });
}

// seeds: every active patch, and the patches over an active patch holding a
// significant coefficient (one thread per list entry)
template <class R>
__global__ void k_seed(const DevLevelT<R>* __restrict__ lvs, const int32_t* list, const int32_t* count, int jb) {
    const int64_t t = gid();
    if (t >= *count) return;
    const int32_t ent = list[t];
    const int j = ent >> LVL_SHIFT;
    const int64_t P = ent & PATCH_MASK;
    const DevLevelT<R>& L = lvs[j];
    L.zflag[P] = 1;
    if (j < jb && L.sflag[P]) {
        const DevLevelT<R>& F = lvs[j + 1];
        for (int q = 0; q < 4; ++q) {
            const int32_t c = L.pchild[q * (L.npatch + 1) + P];
            if (c >= 0) F.zflag[c] = 1;
        }
    }
}

// one ring around the flagged patches of level j: out = in + neighbours of in.  The
// final pass writes the candidates and marks the patch under each candidate as a
// seed of level j-1.  `all`: every patch is a candidate.
template <class R>
__global__ void k_ring(DevLevelT<R> L, DevLevelT<R> C, int src, int final_pass, int push, int all) {
    const int64_t P = gid();
    if (P > L.npatch) return;
    const int64_t np1 = L.npatch + 1;
    const uint8_t* in = src == 0 ? L.zflag : L.gflag;
    uint8_t c = all ? 1 : in[P];
    for (int k = 0; k < NB && !c; ++k) {
        const int32_t Q = L.pnbr[k * np1 + P];
        if (Q < 0) break;
        c = in[Q];
    }
    if (final_pass) {
        L.cflag[P] = c;
        if (c && push && L.ppar[P] >= 0) C.zflag[L.ppar[P]] = 1;
    } else {
        L.gflag[P] = c;
    }
}

// ghost candidates: one ring around the patches with a live node; with two rings
// the first pass goes through cflag (no longer needed once the candidate lists are
// built).  Jmin (level ja of the span): every patch.
template <class R>
__global__ void k_gring(const DevLevelT<R>* __restrict__ lvs, Span sp, int pass, int rings) {
    int j;
    int64_t P;
    if (!span_find(sp, gid(), j, P)) return;
    const DevLevelT<R>& L = lvs[j];
    const int64_t np1 = L.npatch + 1;
    const uint8_t* in = pass == 0 ? L.lflag : L.cflag;
    uint8_t c = j == sp.ja ? 1 : in[P];
    for (int k = 0; k < NB && !c; ++k) {
        const int32_t Q = L.pnbr[k * np1 + P];
        if (Q < 0) break;
        c = in[Q];
    }
    (pass == 0 && rings == 2 ? L.cflag : L.gflag)[P] = c;
}

// compact flags of every level (one block per level) into level-tagged lists:
// which 1 candidates (cflag -> cand), 2 ghost candidates (gflag -> gcand)
template <class R>
__global__ void k_flag_scan(const DevLevelT<R>* __restrict__ lvs, int ja, int which) {
    const DevLevelT<R>& L = lvs[ja + int(blockIdx.x)];
    const uint8_t* flag = which == 1 ? L.cflag : L.gflag;
    int32_t* out = which == 1 ? L.cand : L.gcand;
    int32_t* nout = which == 1 ? L.ncand : L.ngcand;
    __shared__ int warp_tot[32];
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int32_t tag = int32_t(L.J) << LVL_SHIFT;
    for (int64_t start = 0; start <= L.npatch; start += blockDim.x) {
        const int64_t i = start + threadIdx.x;
        const int f = (i <= L.npatch) ? flag[i] : 0;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        const int pre = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) warp_tot[w] = __popc(bal);
        __syncthreads();
        int off = 0;
        for (int k = 0; k < w; ++k) off += warp_tot[k];
        if (f) out[base + off + pre] = tag | int32_t(i);
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int k = 0; k < nw; ++k) tot += warp_tot[k];
            base += tot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *nout = base;
}

// concatenation of the candidate lists of levels ja..jb
template <class R>
__global__ void k_cat(const DevLevelT<R>* __restrict__ lvs, int ja, int jb, int which, int32_t* all, int32_t* count) {
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int j = ja; j <= jb; ++j) {
        const DevLevelT<R>& L = lvs[j];
        const int32_t* src = which == 1 ? L.cand : L.gcand;
        const int n = which == 1 ? *L.ncand : *L.ngcand;
        for (int i = threadIdx.x; i < n; i += blockDim.x) all[base + i] = src[i];
        __syncthreads();
        if (threadIdx.x == 0) base += n;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = base;
}

template <class R>
__global__ void k_adjacent_list(const DevLevelT<R>* __restrict__ lvs, const int32_t* list, const int32_t* count, int P,
                                int jmin) {
    DevLevelT<R> none{};
    ITEMS(K_NODE, lvs, none, list, count, P) {
        if (L.J == jmin) return;
        adjacent_node(L, lvs[L.J - 1], L.J - 1 > jmin, id);
    });
}

template <class R>
__global__ void k_close_list(DevLevelT<R> F, DevLevelT<R> Fp, int has_finer, int P) {
    ITEMS(K_NODE, (const DevLevelT<R>*)nullptr, F, F.cand, F.ncand, P) { close_node(L, Fp, has_finer != 0, id); });
}

template <class R>
__global__ void k_live_list(const DevLevelT<R>* __restrict__ lvs, const int32_t* list, const int32_t* count, int P,
                            int jmin) {
    DevLevelT<R> none{};
    ITEMS(K_NODE, lvs, none, list, count, P) {
        if (live_node(L, id, L.J == jmin)) L.lflag[patch_of(L, id)] = 1;
    });
}

// the significance bytes of the previous mask, over its candidates (they stay
// readable until the next mask)
template <class R>
__global__ void k_clear_sig_list(const DevLevelT<R>* __restrict__ lvs, const int32_t* list, const int32_t* count, int P) {
    DevLevelT<R> none{};
    ITEMS(K_NODE, lvs, none, list, count, P) { L.sig[id] = 0; });
}

template <class R>
__global__ void k_live_edges_list(const DevLevelT<R>* __restrict__ lvs, const int32_t* list, const int32_t* count,
                                  int P) {
    DevLevelT<R> none{};
    ITEMS(K_EDGE, lvs, none, list, count, P) { live_edge(L, id); });
}

template <class R>
__global__ void k_dilate_list(const DevLevelT<R>* __restrict__ lvs, const int32_t* list, const int32_t* count, int P,
                              int jmin, int forward) {
    DevLevelT<R> none{};
    ITEMS(K_NODE, lvs, none, list, count, P) {
        if (L.J == jmin) return;
        dilate_node(L, id, forward != 0);
    });
}

template <class R>
__global__ void k_ghost_list(const DevLevelT<R>* __restrict__ lvs, const int32_t* list, const int32_t* count, int P,
                             int jmin, int in_band1) {
    DevLevelT<R> none{};
    ITEMS(K_NODE | K_EDGE, lvs, none, list, count, P) {
        if (L.J == jmin) return;
        const uint8_t* band = in_band1 ? L.band1 : L.band0;
        if (kind == K_NODE)
            ghost_node(L, id, band);
        else
            ghost_edge(L, id, band);
    });
}

template <class R>
__global__ void k_covered_list(const DevLevelT<R>* __restrict__ lvs, const int32_t* list, const int32_t* count, int P,
                               int jtop) {
    DevLevelT<R> none{};
    ITEMS(K_NODE, lvs, none, list, count, P) {
        if (L.J >= jtop) return;
        covered_node(L, lvs[L.J + 1], id);
    });
}

// before the new patch flags: the learned proposal's counts (misses, over-refined,
// proposed; levels above Jmin) and the old flags cleared, over the candidates (a
// superset of the old active patches and of the exact set)
template <class R>
__global__ void k_pre_flags(const DevLevelT<R>* __restrict__ lvs, const int32_t* list, const int32_t* count, int jmin,
                            unsigned long long* lstat) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t t = gid(); t < *count; t += stride) {
        const int32_t ent = list[t];
        const int j = ent >> LVL_SHIFT;
        const int64_t P = ent & PATCH_MASK;
        const DevLevelT<R>& L = lvs[j];
        if (P >= L.npatch) continue;
        if (lstat && j > jmin) {
            if (L.pexact[P] && !L.pflag[P]) atomicAdd(&lstat[0], 1ull);
            if (L.prop_prev[P] && !L.pexact[P]) atomicAdd(&lstat[1], 1ull);
            if (L.prop[P]) atomicAdd(&lstat[2], 1ull);
        }
        L.pflag[P] = 0;
    }
}

// patch flags over the ghost candidates (every patch with a live or ghost point is
// one), and the band bytes of their nodes cleared; a block per entry
template <class R>
__global__ void k_flags_list(const DevLevelT<R>* __restrict__ lvs, const int32_t* list, const int32_t* count) {
    for (int64_t t = blockIdx.x; t < *count; t += gridDim.x) {
        const int32_t ent = list[t];
        const int j = ent >> LVL_SHIFT;
        const int64_t P = ent & PATCH_MASK;
        const DevLevelT<R>& L = lvs[j];
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

}  // namespace

#define LAUNCH(kernel, grid, ...) (count_launch(1), kernel<<<(grid), TPB, 0, s>>>(__VA_ARGS__))

template <class R>
void launch_mask_lists(const MaskListArgs<R>& a, cudaStream_t s) {
    const int ja = a.ja, jb = a.jb;
    const int64_t npatches = a.patches.off[jb + 1 - ja];
    // seeds
    LAUNCH(k_clear_flags<R>, blocks_for(npatches, TPB), a.lvs, a.patches);
    LAUNCH(k_clear_sig_list<R>, a.grid, a.lvs, a.cand, a.cand_count, a.P);
    LAUNCH(k_sig_list<R>, a.grid, a.lvs, a.active, a.active_count, a.P, ja, a.thr, a.sig_any);
    LAUNCH(k_seed<R>, blocks_for(a.max_entries, TPB), a.lvs, a.active, a.active_count, jb);
    // candidates, from the top level down (Jmin and whole-lozenge levels: every patch)
    for (int j = jb; j >= ja; --j) {
        const DevLevelT<R>& L = a.host[j];
        const DevLevelT<R>& C = a.host[j > ja ? j - 1 : j];
        const int all = (j == ja || L.npatch <= 10) ? 1 : 0;
        const int push = j - 1 > ja ? 1 : 0;
        const unsigned g = blocks_for(L.npatch + 1, TPB);
        if (a.rings == 2 && !all) {
            LAUNCH(k_ring<R>, g, L, C, 0, 0, 0, 0);
            LAUNCH(k_ring<R>, g, L, C, 1, 1, push, 0);
        } else {
            LAUNCH(k_ring<R>, g, L, C, 0, 1, push, all);
        }
    }
    count_launch(2);
    k_flag_scan<R><<<unsigned(jb - ja + 1), 1024, 0, s>>>(a.lvs, ja, 1);
    k_cat<R><<<1, 1024, 0, s>>>(a.lvs, ja, jb, 1, a.cand, a.cand_count);
    // the set T, its closure from the top level down, live flags
    LAUNCH(k_adjacent_list<R>, a.grid, a.lvs, a.cand, a.cand_count, a.P, ja);
    for (int j = jb; j > ja; --j)
        LAUNCH(k_close_list<R>, a.grid_lv[j], a.host[j], a.host[j < jb ? j + 1 : j], j < jb ? 1 : 0, a.P);
    LAUNCH(k_live_list<R>, a.grid, a.lvs, a.cand, a.cand_count, a.P, ja);
    LAUNCH(k_live_edges_list<R>, a.grid, a.lvs, a.cand, a.cand_count, a.P);
    // ghost candidates (every patch of Jmin), ghost band, covered nodes
    LAUNCH(k_gring<R>, blocks_for(npatches, TPB), a.lvs, a.patches, 0, a.rings);
    if (a.rings == 2) LAUNCH(k_gring<R>, blocks_for(npatches, TPB), a.lvs, a.patches, 1, a.rings);
    count_launch(2);
    k_flag_scan<R><<<unsigned(jb - ja + 1), 1024, 0, s>>>(a.lvs, ja, 2);
    k_cat<R><<<1, 1024, 0, s>>>(a.lvs, ja, jb, 2, a.gcand, a.gcand_count);
    if (jb > ja) {
        for (int h = 0; h < a.hops; ++h)
            LAUNCH(k_dilate_list<R>, a.grid, a.lvs, a.gcand, a.gcand_count, a.P, ja, h % 2 == 0);
        LAUNCH(k_ghost_list<R>, a.grid, a.lvs, a.gcand, a.gcand_count, a.P, ja, a.hops % 2 == 1);
        LAUNCH(k_covered_list<R>, a.grid, a.lvs, a.cand, a.cand_count, a.P, jb);
    }
    // patch flags: the old ones cleared over the candidates (a superset of the old
    // active patches), the new ones set over the ghost candidates (a superset of
    // the patches with a live or ghost point)
    LAUNCH(k_pre_flags<R>, a.grid, a.lvs, a.cand, a.cand_count, ja, a.lstat);
    count_launch(1);
    k_flags_list<R><<<a.grid, 64, 0, s>>>(a.lvs, a.gcand, a.gcand_count);
}

template void launch_mask_lists<double>(const MaskListArgs<double>&, cudaStream_t);
template void launch_mask_lists<float>(const MaskListArgs<float>&, cudaStream_t);

}  // namespace sww
