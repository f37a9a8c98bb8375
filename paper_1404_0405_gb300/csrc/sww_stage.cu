// Persistent RK stage: one cooperative launch runs every phase of a trend
// evaluation and its stage update (Sec. 3.1), the phases separated by grid
// barriers instead of kernel boundaries:
//
//   ghosts of levels Jmin+1..top (coarse to fine, one phase per level)
//   -> q at triangles, F at edges (all levels)
//   -> div, K, B at nodes, q F^perp at edges (all levels)
//   -> restriction of B, F, q F^perp and div, top-1 down to Jmin (two phases a level)
//   -> RK stage update of the live points (all levels)
//
// The level records are staged in shared memory once per block.  Loads of this
// translation unit bypass L1 (compiled with -dlcm=cg): values written by other
// blocks in one phase are read in the next.  Every barrier wait is bounded: after
// about two seconds a block sets the error flag and the kernel returns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "sww_core.cuh"
#include "sww_kernels.h"
#include "sww_stage.h"

namespace sww {

namespace {

#include "sww_bodies.cuh"

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

// Barrier between phases: the grid barrier of a cooperative launch, or the
// hardware barrier of a thread-block cluster when the launch is one cluster (all
// its blocks are co-scheduled, and every thread runs every phase).
template <class R>
__device__ __forceinline__ bool stage_sync(const StageArgs<R>& a) {
    if (a.cluster) {
        asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
        asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
        return true;
    }
    return grid_sync(a.bar, a.err, a.spin, a.skip);
}

template <class R>
__global__ void __launch_bounds__(STAGE_TPB) k_stage(StageArgs<R> a) {
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
    ITEMS(K_EDGE | K_TRI, lv, lv[a.jmin], a.all_list, a.all_count, a.P) {
        if (kind == K_EDGE)
            flux_at(L, id, H);
        else
            pv_at(L, id, H);
    });
    if (!stage_sync(a)) return;
    ITEMS(K_NODE | K_EDGE, lv, lv[a.jmin], a.all_list, a.all_count, a.P) {
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
        ITEMS(K_NODE, (const DevLevelT<R>*)nullptr, C, C.patches, C.npatches, a.P) { div_at(L, id); });
        if (!stage_sync(a)) return;
    }
    const R dt = R(a.dt ? *a.dt : 0.0);
    ITEMS(K_NODE | K_EDGE, lv, lv[a.jmin], a.all_list, a.all_count, a.P) {
        if (kind == K_NODE)
            update_node(L, id, a.st, dt);
        else
            update_edge(L, id, a.st, dt);
    });
}

// ------------------------------------------------------------------ ensembles

constexpr int MAXM = 128;

// Items of one phase over the members of an ensemble.  mode < 0: each member's
// all-level list; else the level-j list of the members whose top level is at
// least j + mode (0 ghosts, -1 restriction).  body(L, kind, id, el, member).
template <int KINDS, class R, class Body>
__device__ __forceinline__ void batch_items(const BatchArgs<R>& a, int j, int mode, int64_t* pre, Body body) {
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        for (int m = 0; m < a.nm; ++m) {
            pre[m] = acc;
            const MemberRef<R>& M = a.m[m];
            if (mode < 0)
                acc += *M.all_count;
            else if (j <= M.jtop + mode)
                acc += *M.lvs[j].npatches;
        }
        pre[a.nm] = acc;
    }
    __syncthreads();
    constexpr int NS = slots_of<KINDS>();
    const int64_t S = int64_t(NS) * a.P;
    const int64_t n = pre[a.nm] * S;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t it = gid(); it < n; it += stride) {
        const int64_t e = it / S;
        int lo = 0, hi = a.nm - 1;   // last member whose first entry is <= e
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (pre[mid] <= e) lo = mid; else hi = mid - 1;
        }
        const MemberRef<R>& M = a.m[lo];
        const int32_t ent = mode < 0 ? M.all_list[e - pre[lo]] : M.lvs[j].patches[e - pre[lo]];
        const DevLevelT<R>& L = M.lvs[ent >> LVL_SHIFT];
        auto b = [&](const DevLevelT<R>& LL, int kind, int64_t id, int64_t el) { body(LL, kind, id, el, M); };
        visit_item<KINDS>(L, int64_t(ent & PATCH_MASK), uint32_t(it - e * S), a.P, b);
    }
    __syncthreads();
}

// One RK stage of every member of an ensemble, the phases of k_stage in order,
// each phase over all members (the levels of member m are a contiguous record
// array, so the coarser and finer records of L are (&L)[-1] and (&L)[1]).
template <class R>
__global__ void __launch_bounds__(STAGE_TPB) k_stage_batch(BatchArgs<R> a) {
    __shared__ int64_t pre[MAXM + 1];
    const R H = R(a.H), g = R(a.g);
    for (int j = a.jmin + 1; j <= a.jtop_max; ++j) {
        batch_items<K_NODE | K_EDGE>(a, j, 0, pre, [&](const DevLevelT<R>& L, int kind, int64_t id, int64_t, const MemberRef<R>&) {
            if (kind == K_NODE)
                fill_node(L, (&L)[-1], id);
            else
                fill_edge(L, (&L)[-1], id);
        });
        if (!grid_sync(a.bar, a.err)) return;
    }
    batch_items<K_EDGE | K_TRI>(a, 0, -1, pre, [&](const DevLevelT<R>& L, int kind, int64_t id, int64_t, const MemberRef<R>&) {
        if (kind == K_EDGE)
            flux_at(L, id, H);
        else
            pv_at(L, id, H);
    });
    if (!grid_sync(a.bar, a.err)) return;
    batch_items<K_NODE | K_EDGE>(a, 0, -1, pre, [&](const DevLevelT<R>& L, int kind, int64_t id, int64_t, const MemberRef<R>&) {
        if (kind == K_NODE)
            node_at(L, id, g);
        else
            coriolis_at(L, id);
    });
    if (!grid_sync(a.bar, a.err)) return;
    for (int j = a.jtop_max - 1; j >= a.jmin; --j) {
        batch_items<K_NODE | K_EDGE>(a, j, -1, pre, [&](const DevLevelT<R>& L, int kind, int64_t id, int64_t, const MemberRef<R>&) {
            restrict_item(L, (&L)[1], kind, id);
        });
        if (!grid_sync(a.bar, a.err)) return;
        batch_items<K_NODE>(a, j, -1, pre, [&](const DevLevelT<R>& L, int, int64_t id, int64_t, const MemberRef<R>&) {
            div_at(L, id);
        });
        if (!grid_sync(a.bar, a.err)) return;
    }
    batch_items<K_NODE | K_EDGE>(a, 0, -1, pre, [&](const DevLevelT<R>& L, int kind, int64_t id, int64_t, const MemberRef<R>& M) {
        const R dt = R(*M.dt);
        if (kind == K_NODE)
            update_node(L, id, a.st, dt);
        else
            update_edge(L, id, a.st, dt);
    });
}

}  // namespace

template <class R>
unsigned stage_grid(int nsm) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stage<R>, STAGE_TPB, 0) != cudaSuccess) return 0;
    return unsigned(std::max(per_sm, 0) * nsm);
}

template <class R>
cudaError_t launch_stage(const StageArgs<R>& a, unsigned grid, cudaStream_t s) {
    if (a.jmax + 1 > MAXL) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(STAGE_TPB);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launch(1);
    return cudaLaunchKernelEx(&cfg, k_stage<R>, a);
}

// One RK stage as a single thread-block cluster (up to 16 blocks): for members of an
// ensemble whose steps overlap on their own streams.
template <class R>
cudaError_t launch_stage_cluster(const StageArgs<R>& a, int blocks, cudaStream_t s) {
    if (a.jmax + 1 > MAXL || !a.cluster) return cudaErrorInvalidValue;
    if (blocks > 8) {
        cudaError_t e = cudaFuncSetAttribute(k_stage<R>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(STAGE_TPB);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = blocks;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launch(1);
    return cudaLaunchKernelEx(&cfg, k_stage<R>, a);
}

// largest cluster of stage blocks that can be resident (16, else 8, else 0)
template <class R>
int stage_cluster_size() {
    for (int c : {16, 8}) {
        if (c > 8 && cudaFuncSetAttribute(k_stage<R>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
            continue;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(c);
        cfg.blockDim = dim3(STAGE_TPB);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_stage<R>, &cfg) == cudaSuccess && n > 0) return c;
        cudaGetLastError();
    }
    return 0;
}

template <class R>
unsigned stage_batch_grid(int nsm) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stage_batch<R>, STAGE_TPB, 0) != cudaSuccess) return 0;
    return unsigned(std::max(per_sm, 0) * nsm);
}

template <class R>
cudaError_t launch_stage_batch(const BatchArgs<R>& a, unsigned grid, cudaStream_t s) {
    if (a.nm < 1 || a.nm > MAXM) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(STAGE_TPB);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launch(1);
    return cudaLaunchKernelEx(&cfg, k_stage_batch<R>, a);
}

template unsigned stage_grid<double>(int);
template unsigned stage_grid<float>(int);
template cudaError_t launch_stage<double>(const StageArgs<double>&, unsigned, cudaStream_t);
template cudaError_t launch_stage<float>(const StageArgs<float>&, unsigned, cudaStream_t);
template cudaError_t launch_stage_cluster<double>(const StageArgs<double>&, int, cudaStream_t);
template cudaError_t launch_stage_cluster<float>(const StageArgs<float>&, int, cudaStream_t);
template int stage_cluster_size<double>();
template int stage_cluster_size<float>();
template unsigned stage_batch_grid<double>(int);
template unsigned stage_batch_grid<float>(int);
template cudaError_t launch_stage_batch<double>(const BatchArgs<double>&, unsigned, cudaStream_t);
template cudaError_t launch_stage_batch<float>(const BatchArgs<float>&, unsigned, cudaStream_t);

}  // namespace sww
