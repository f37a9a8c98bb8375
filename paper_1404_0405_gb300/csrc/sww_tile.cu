// Trend of an RK stage (Sec. 3.1) over the active patches of every member of an
// ensemble (one member: a handle stepping alone), structured where the patch is
// regular:
//
//   k_tile_trend  one block per active patch at a time (blocks grouped per
//                 member, striding over the member's all-level list): a regular
//                 patch runs tile_trend (F, q, div F, K, B, q F^perp from its tile in
//                 shared memory, its geometry block brought in by a bulk copy one
//                 patch ahead); an irregular one (a pentagon or a pole within
//                 reach, a level whose patch side differs, the viscous and
//                 advection forms) gets F and q from the tabulated bodies.
//   k_tile_irr    div F, K, B and q F^perp at the points of the irregular
//                 patches (the member's irregular list), from the F and q that
//                 k_tile_trend wrote for them and their neighbours.
//   k_tile_geo    the geometry blocks of a level's regular patches (once per grid
//                 and precision).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "sww_core.cuh"
#include "sww_kernels.h"
#include "sww_stage.h"
#include "tile.h"

namespace sww {

namespace {

#include "bulk.cuh"
#include "sww_bodies.cuh"
#include "sww_tile.cuh"

constexpr int TILE_TPB = 256;
constexpr int MAXL = 12;
constexpr int MAXM = 128;
constexpr long long COPY_WAIT_CYCLES = 4000000000ll;   // ~2 s at 2 GHz: a bulk copy that has not landed

// the member's level records jmin..jmax into shared memory
template <class R>
__device__ __forceinline__ void stage_records(DevLevelT<R>* sl, const MemberRef<R>* mr, int jmin) {
    const int words = int((mr->jmax - jmin + 1) * sizeof(DevLevelT<R>) / sizeof(int));
    const int* src = reinterpret_cast<const int*>(mr->lvs + jmin);
    int* dst = reinterpret_cast<int*>(sl + jmin);
    for (int k = threadIdx.x; k < words; k += blockDim.x) dst[k] = src[k];
    __syncthreads();
}

// resident blocks per SM the tile kernel is built for: five for 8 x 8 tiles (48
// registers; measured 5 % faster than six blocks at 40 registers, which spilled
// the copy pipeline's state), four for 16 x 16 (their per-thread slot plan is
// larger)
template <int P>
constexpr int tile_min_blocks() { return P >= 16 ? 4 : 5; }

template <class R, int P>
__global__ void __launch_bounds__(TILE_TPB, tile_min_blocks<P>()) k_tile_trend(BatchArgs<R> a, int bpm) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ DevLevelT<R> sl[MAXL];
    const int m = blockIdx.x / bpm, b = blockIdx.x % bpm;
    const MemberRef<R>* mr = a.m + m;
    stage_records(sl, mr, a.jmin);
    const R H = R(a.H);
    const int area = a.P;
    tile_sweep<R, P, TILE_TPB>(sl, mr->all_list, *mr->all_count, b, bpm, H, R(a.g), smem, mr->err, COPY_WAIT_CYCLES,
                               [&](const DevLevelT<R>& L, int64_t pat) {
                                   for (int it = threadIdx.x; it < 5 * area; it += blockDim.x) {
                                       auto body = [&](const DevLevelT<R>& LL, int kind, int64_t id, int64_t) {
                                           if (kind == K_EDGE)
                                               flux_at(LL, id, H);
                                           else
                                               pv_at(LL, id, H);
                                       };
                                       visit_item<K_EDGE | K_TRI>(L, pat, uint32_t(it), area, body);
                                   }
                               });
}

// the geometry block of every regular patch of L (one block per patch)
template <class R, int P>
__global__ void __launch_bounds__(TILE_TPB) k_tile_geo(DevLevelT<R> L, R* out) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int64_t pat = blockIdx.x;
    if (pat >= L.npatch || L.tirr[pat]) return;
    tile_geo_build<R, P, TILE_TPB>(L, pat, out + pat * TileGeo<R, P>::WORDS, reinterpret_cast<R*>(smem));
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
    // the dynamic tile and the static level records together may pass the default
    // 48 KB: the dynamic size is always declared (once)
    static bool declared = false;
    if (!declared) {
        cudaError_t e0 = cudaFuncSetAttribute(k_tile_trend<R, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e0 != cudaSuccess) return e0;
        declared = true;
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
    // the irregular patches: a bound on their items per member, at most two waves
    // of 8 blocks per SM over all members
    const int64_t items = (irr_entries + a.nm - 1) / a.nm * 4 * a.P;
    const int bpm2 = int(std::max<int64_t>(1, std::min<int64_t>((items + TILE_TPB - 1) / TILE_TPB,
                                                                   std::max(1, 16 * nsm / a.nm))));
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
        case 16: return launch_trend_p<R, 4>(a, entries, irr_entries, nsm, parts, s);
        case 64: return launch_trend_p<R, 8>(a, entries, irr_entries, nsm, parts, s);
        case 256: return launch_trend_p<R, 16>(a, entries, irr_entries, nsm, parts, s);
        default: return cudaErrorInvalidValue;   // patch sides are 4, 8 or 16
    }
}

namespace {
template <class R, int P>
cudaError_t tile_geo_p(const DevLevelT<R>& L, R* out, cudaStream_t s) {
    constexpr size_t smem = sizeof(R) * 6 * TileGeo<R, P>::NN;   // the kites, for the inverse sums
    static_assert(smem <= 48 * 1024, "kite scratch");
    if (L.npatch < 1) return cudaSuccess;
    count_launch(1);
    k_tile_geo<R, P><<<unsigned(L.npatch), TILE_TPB, smem, s>>>(L, out);
    return cudaGetLastError();
}
}  // namespace

template <class R>
size_t tile_geo_words(int side) {
    switch (side) {
        case 4: return size_t(TileGeo<R, 4>::WORDS);
        case 8: return size_t(TileGeo<R, 8>::WORDS);
        case 16: return size_t(TileGeo<R, 16>::WORDS);
        default: return 0;
    }
}

template <class R>
cudaError_t build_tile_geo(const DevLevelT<R>& L, int side, R* out, cudaStream_t s) {
    switch (side) {
        case 4: return tile_geo_p<R, 4>(L, out, s);
        case 8: return tile_geo_p<R, 8>(L, out, s);
        case 16: return tile_geo_p<R, 16>(L, out, s);
        default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_tile_trend<double>(const BatchArgs<double>&, int64_t, int64_t, int, int, cudaStream_t);
template cudaError_t launch_tile_trend<float>(const BatchArgs<float>&, int64_t, int64_t, int, int, cudaStream_t);
template size_t tile_geo_words<double>(int);
template size_t tile_geo_words<float>(int);
template cudaError_t build_tile_geo<double>(const DevLevelT<double>&, int, double*, cudaStream_t);
template cudaError_t build_tile_geo<float>(const DevLevelT<float>&, int, float*, cudaStream_t);

}  // namespace sww
