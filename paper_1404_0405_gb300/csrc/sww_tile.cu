// Trend of an RK stage (Sec. 3.1) over the active patches of every member of an
// ensemble (one member: a handle stepping alone), structured where the patch is
// regular:
//
//   k_tile_trend  one block per active patch at a time (blocks grouped per
//                 member, striding over the member's all-level list): a regular
//                 patch runs tile_trend (F, q, div F, K, B, q F^perp from its tile in
//                 shared memory); an irregular one (a pentagon or a pole within
//                 reach, a level whose patch side differs, the viscous and
//                 advection forms) gets F and q from the tabulated bodies.
//   k_tile_irr    div F, K, B and q F^perp at the points of the irregular
//                 patches (the member's irregular list), from the F and q that
//                 k_tile_trend wrote for them and their neighbours.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "sww_core.cuh"
#include "sww_kernels.h"
#include "sww_stage.h"
#include "tile.h"

namespace sww {

namespace {

#include "sww_bodies.cuh"
#include "sww_tile.cuh"

constexpr int TILE_TPB = 256;
constexpr int MAXL = 12;
constexpr int MAXM = 128;

// the member's level records jmin..jmax into shared memory
template <class R>
__device__ __forceinline__ void stage_records(DevLevelT<R>* sl, const MemberRef<R>* mr, int jmin) {
    const int words = int((mr->jmax - jmin + 1) * sizeof(DevLevelT<R>) / sizeof(int));
    const int* src = reinterpret_cast<const int*>(mr->lvs + jmin);
    int* dst = reinterpret_cast<int*>(sl + jmin);
    for (int k = threadIdx.x; k < words; k += blockDim.x) dst[k] = src[k];
    __syncthreads();
}

// resident blocks per SM the tile kernel is built for: six for 8 x 8 tiles (40
// registers), four for 16 x 16 (their per-thread slot plan is larger)
template <int P>
constexpr int tile_min_blocks() { return P >= 16 ? 4 : 6; }

template <class R, int P>
__global__ void __launch_bounds__(TILE_TPB, tile_min_blocks<P>()) k_tile_trend(BatchArgs<R> a, int bpm) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ DevLevelT<R> sl[MAXL];
    const int m = blockIdx.x / bpm, b = blockIdx.x % bpm;
    const MemberRef<R>* mr = a.m + m;
    stage_records(sl, mr, a.jmin);
    const R H = R(a.H), g = R(a.g);
    TilePlan<P, TILE_TPB> plan;
    plan.init();
    TileCodes<P, TILE_TPB> cur, nxt;
    const int n = *mr->all_count;
    if (b < n) {
        const int32_t ent = mr->all_list[b];
        const DevLevelT<R>& L = sl[ent >> LVL_SHIFT];
        if (tile_regular(L, ent & PATCH_MASK)) cur.load(L, ent & PATCH_MASK, plan);
    }
    for (int e = b; e < n; e += bpm) {
        const int32_t ent = mr->all_list[e];
        const DevLevelT<R>& L = sl[ent >> LVL_SHIFT];
        const int64_t pat = ent & PATCH_MASK;
        // the next patch's halo ids, in flight while this one is worked on
        if (e + bpm < n) {
            const int32_t ent2 = mr->all_list[e + bpm];
            const DevLevelT<R>& L2 = sl[ent2 >> LVL_SHIFT];
            if (tile_regular(L2, ent2 & PATCH_MASK)) nxt.load(L2, ent2 & PATCH_MASK, plan);
        }
        if (tile_regular(L, pat)) {
            tile_trend<R, P, TILE_TPB>(L, pat, H, g, plan, cur, smem);
        } else {
            for (int it = threadIdx.x; it < 5 * a.P; it += blockDim.x) {
                auto body = [&](const DevLevelT<R>& LL, int kind, int64_t id, int64_t) {
                    if (kind == K_EDGE)
                        flux_at(LL, id, H);
                    else
                        pv_at(LL, id, H);
                };
                visit_item<K_EDGE | K_TRI>(L, pat, uint32_t(it), a.P, body);
            }
        }
        __syncthreads();   // the tile's shared memory is reused by the next patch
        cur = nxt;
    }
}

template <class R>
__global__ void __launch_bounds__(TILE_TPB) k_tile_irr(BatchArgs<R> a, int bpm) {
    __shared__ DevLevelT<R> sl[MAXL];
    const int m = blockIdx.x / bpm, b = blockIdx.x % bpm;
    const MemberRef<R>* mr = a.m + m;
    stage_records(sl, mr, a.jmin);
    const R g = R(a.g);
    const int lp = __ffs(a.P) - 1;
    const uint32_t n = uint32_t(*mr->irr_count) * (4u << lp);
    for (uint32_t it = uint32_t(b) * blockDim.x + threadIdx.x; it < n; it += uint32_t(bpm) * blockDim.x) {
        const uint32_t e = (it >> lp) / 4;
        const int32_t ent = mr->irr_list[e];
        const DevLevelT<R>& L = sl[ent >> LVL_SHIFT];
        auto body = [&](const DevLevelT<R>& LL, int kind, int64_t id, int64_t) {
            if (kind == K_NODE)
                node_at(LL, id, g);
            else
                coriolis_at(LL, id);
        };
        visit_item<K_NODE | K_EDGE>(L, int64_t(ent & PATCH_MASK), it - ((e * 4) << lp), a.P, body);
    }
}

template <class R, int P>
cudaError_t launch_trend_p(const BatchArgs<R>& a, int64_t entries, int64_t irr_entries, int nsm, int parts,
                           cudaStream_t s) {
    constexpr size_t smem = Tile<R, P>::BYTES;
    if (parts & 1) {
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_tile_trend<R, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
    }
    // blocks per member: one per active patch up to a full GPU over all members
    static int per_sm = 0;   // resident blocks per SM (the same on every GPU of a process here)
    if (per_sm == 0) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_tile_trend<R, P>, TILE_TPB, smem) != cudaSuccess)
            return cudaGetLastError();
        per_sm = std::max(n, 1);
    }
    const int cap = std::max(1, per_sm * nsm / a.nm);
    const int bpm = int(std::max<int64_t>(1, std::min<int64_t>((entries + a.nm - 1) / a.nm, cap)));
    count_launch(1);
    k_tile_trend<R, P><<<unsigned(a.nm * bpm), TILE_TPB, smem, s>>>(a, bpm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    }
    if (!(parts & 2)) return cudaSuccess;
    // the irregular patches: a bound on their items per member
    const int64_t items = (irr_entries + a.nm - 1) / a.nm * 4 * a.P;
    const int bpm2 = int(std::max<int64_t>(1, std::min<int64_t>((items + TILE_TPB - 1) / TILE_TPB,
                                                                   std::max(1, 8 * nsm / a.nm))));
    count_launch(1);
    k_tile_irr<R><<<unsigned(a.nm * bpm2), TILE_TPB, 0, s>>>(a, bpm2);
    return cudaGetLastError();
}

}  // namespace

template <class R>
cudaError_t launch_tile_trend(const BatchArgs<R>& a, int64_t entries, int64_t irr_entries, int nsm, int parts,
                              cudaStream_t s) {
    if (a.nm < 1 || a.nm > MAXM) return cudaErrorInvalidValue;
    switch (a.P) {
        case 64: return launch_trend_p<R, 8>(a, entries, irr_entries, nsm, parts, s);
        case 256: return launch_trend_p<R, 16>(a, entries, irr_entries, nsm, parts, s);
        default: return launch_trend_p<R, 4>(a, entries, irr_entries, nsm, parts, s);   // sides 1, 2: no regular tile
    }
}

template cudaError_t launch_tile_trend<double>(const BatchArgs<double>&, int64_t, int64_t, int, int, cudaStream_t);
template cudaError_t launch_tile_trend<float>(const BatchArgs<float>&, int64_t, int64_t, int, int, cudaStream_t);

}  // namespace sww
