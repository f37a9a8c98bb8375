// Persistent RK stage: one cooperative launch runs every phase of a trend
// evaluation and its stage update (Sec. 3.1), the phases separated by grid
// barriers instead of kernel boundaries:
//
//   ghosts of levels Jmin+1..top (coarse to fine, one phase per level)
//   -> the trend of every active patch: the structured tile of a regular patch
//      (F, q, div F, K, B, q F^perp), F and q from the tabulated bodies elsewhere
//   -> div, K, B and q F^perp at the points of the irregular patches
//   -> restriction of B, F, q F^perp and div, top-1 down to Jmin (two phases a level)
//   -> RK stage update of the live points (all levels)
//
// The level records are staged in shared memory once per block; the tile of the
// patch a block works on is staged in dynamic shared memory.  Loads of this
// translation unit bypass L1 (compiled with -dlcm=cg): values written by other
// blocks in one phase are read in the next.  Every barrier wait is bounded: after
// about two seconds a block sets the error flag and the kernel returns; so does
// the wait for a patch's geometry block (a bulk copy).
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

constexpr int STAGE_TPB = 512;
constexpr int MAXL = 12;
constexpr long long SPIN_CYCLES = 4000000000ll;   // ~2 s at 2 GHz
constexpr unsigned BAR_GROUPS = 16, BAR_STRIDE = 32;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier, two-level: a block arrives at one of GROUPS counters (each in
// its own 128-byte line), the last of a group at the root counter, and the last of
// all advances the generation word that the others wait on.  False when the wait
// timed out (after `spin` cycles, <= 0: SPIN_CYCLES) or a block has reported an
// error; a block that finds the error flag already set does not arrive, so no
// block passes a barrier once a wait has failed.  Block `skip` (fault injection,
// -1: none) leaves without arriving.
__device__ bool grid_sync(unsigned* bar, int* err, long long spin = 0, int skip = -1) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) ok = 1;
    if (threadIdx.x == 0 && (int(blockIdx.x) == skip || *reinterpret_cast<volatile int*>(err))) ok = 0;
    __syncthreads();
    if (!ok) return false;
    if (threadIdx.x == 0) {
        const long long limit = spin > 0 ? spin : SPIN_CYCLES;
        const unsigned groups = gridDim.x < BAR_GROUPS ? gridDim.x : BAR_GROUPS;
        const unsigned grp = blockIdx.x % groups;
        const unsigned in_grp = (gridDim.x - grp + groups - 1) / groups;
        unsigned* gen_p = bar;
        unsigned* grp_p = bar + BAR_STRIDE * (1 + grp);
        unsigned* root_p = bar + BAR_STRIDE * (1 + BAR_GROUPS);
        const unsigned gen = ld_acquire(gen_p);
        __threadfence();
        bool last = false;
        if (atomicAdd(grp_p, 1u) == in_grp - 1) {
            atomicExch(grp_p, 0u);
            if (atomicAdd(root_p, 1u) == groups - 1) {
                atomicExch(root_p, 0u);
                last = true;
            }
        }
        if (last) {
            __threadfence();
            atomicAdd(gen_p, 1u);
        } else {
            const long long t0 = clock64();
            while (ld_acquire(gen_p) == gen) {
                if (*reinterpret_cast<volatile int*>(err)) {
                    ok = 0;
                    break;
                }
                if (clock64() - t0 > limit) {
                    atomicExch(err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// barrier between phases: the grid barrier of the cooperative launch
template <class R>
__device__ __forceinline__ bool stage_sync(const StageArgs<R>& a) {
    return grid_sync(a.bar, a.err, a.spin, a.skip);
}

template <class R, int P>
__global__ void __launch_bounds__(STAGE_TPB) k_stage(StageArgs<R> a) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ DevLevelT<R> sl[MAXL];
    {
        const int words = int((a.jmax + 1) * sizeof(DevLevelT<R>) / sizeof(int));
        const int* src = reinterpret_cast<const int*>(a.lvs);
        int* dst = reinterpret_cast<int*>(sl);
        for (int k = threadIdx.x; k < words; k += blockDim.x) dst[k] = src[k];
        __syncthreads();
    }
    const DevLevelT<R>* lv = sl;
    const R H = R(a.H), g = R(a.g);
    // ghosts, coarse to fine
    for (int j = a.jmin + 1; j <= a.jtop; ++j) {
        const DevLevelT<R>& F = lv[j];
        const DevLevelT<R>& C = lv[j - 1];
        ITEMS(K_NODE | K_EDGE, (const DevLevelT<R>*)nullptr, F, F.patches, F.npatches, a.P) {
            if (kind == K_NODE)
                fill_node(L, C, id);
            else
                fill_edge(L, C, id);
        });
        if (!stage_sync(a)) return;
    }
    {
        // one active patch per block at a time
        const long long limit = a.spin > 0 ? a.spin : SPIN_CYCLES;
        const int area = a.P;
        const bool ok = tile_sweep<R, P, STAGE_TPB>(lv, a.all_list, *a.all_count, int(blockIdx.x), int(gridDim.x), H, g,
                                                    smem, a.err, limit, [&](const DevLevelT<R>& L, int64_t pat) {
                                                        for (int it = threadIdx.x; it < 5 * area; it += blockDim.x) {
                                                            auto body = [&](const DevLevelT<R>& LL, int kind, int64_t id,
                                                                            int64_t) {
                                                                if (kind == K_EDGE)
                                                                    flux_at(LL, id, H);
                                                                else
                                                                    pv_at(LL, id, H);
                                                            };
                                                            visit_item<K_EDGE | K_TRI>(L, pat, uint32_t(it), area, body);
                                                        }
                                                    });
        if (!ok) return;
    }
    if (!stage_sync(a)) return;
    ITEMS(K_NODE | K_EDGE, lv, lv[a.jmin], a.irr_list, a.irr_count, a.P) {
        if (kind == K_NODE)
            node_at(L, id, g);
        else
            coriolis_at(L, id);
    });
    if (!stage_sync(a)) return;
    // restriction, fine to coarse
    for (int j = a.jtop - 1; j >= a.jmin; --j) {
        const DevLevelT<R>& C = lv[j];
        const DevLevelT<R>& F = lv[j + 1];
        ITEMS(K_NODE | K_EDGE, (const DevLevelT<R>*)nullptr, C, C.patches, C.npatches, a.P) {
            restrict_item(L, F, kind, id);
        });
        if (!stage_sync(a)) return;
        ITEMS(K_NODE, (const DevLevelT<R>*)nullptr, C, C.patches, C.npatches, a.P) {
            if (restricted_div_node(L, id)) div_at(L, id);
        });
        if (!stage_sync(a)) return;
    }
    const R dt = R(a.dt ? *a.dt : 0.0);
    const RKStageR<R> sr(a.st);
    ITEMS(K_NODE | K_EDGE, lv, lv[a.jmin], a.all_list, a.all_count, a.P) {
        if (kind == K_NODE)
            update_node(L, id, sr, dt);
        else
            update_edge(L, id, sr, dt);
    });
}

template <class R, int P>
unsigned stage_grid_p(int nsm) {
    constexpr size_t smem = Tile<R, P>::BYTES;
    // the dynamic tile and the static level records together may pass the default
    // 48 KB: the dynamic size is always declared
    if (cudaFuncSetAttribute(k_stage<R, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stage<R, P>, STAGE_TPB, smem) != cudaSuccess) return 0;
    return unsigned(std::max(per_sm, 0) * nsm);
}

template <class R, int P>
cudaError_t launch_stage_p(const StageArgs<R>& a, unsigned grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(STAGE_TPB);
    cfg.dynamicSmemBytes = Tile<R, P>::BYTES;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launch(1);
    return cudaLaunchKernelEx(&cfg, k_stage<R, P>, a);
}

}  // namespace

// patch area -> tile side of the stage kernel (sides 1 and 2 have no regular tile)
template <class R>
unsigned stage_grid(int P, int nsm) {
    return P == 64 ? stage_grid_p<R, 8>(nsm) : P == 256 ? stage_grid_p<R, 16>(nsm) : stage_grid_p<R, 4>(nsm);
}

template <class R>
cudaError_t launch_stage(const StageArgs<R>& a, unsigned grid, cudaStream_t s) {
    if (a.jmax + 1 > MAXL) return cudaErrorInvalidValue;
    return a.P == 64 ? launch_stage_p<R, 8>(a, grid, s) : a.P == 256 ? launch_stage_p<R, 16>(a, grid, s)
                                                                    : launch_stage_p<R, 4>(a, grid, s);
}

template unsigned stage_grid<double>(int, int);
template unsigned stage_grid<float>(int, int);
template cudaError_t launch_stage<double>(const StageArgs<double>&, unsigned, cudaStream_t);
template cudaError_t launch_stage<float>(const StageArgs<float>&, unsigned, cudaStream_t);

}  // namespace sww
