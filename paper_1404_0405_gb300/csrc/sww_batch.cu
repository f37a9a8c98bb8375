// RK stage of every member of an ensemble as one regular launch per phase (the
// phases of one trend evaluation and its stage update, Sec. 3.1, in the order of
// the persistent stage): ghosts level by level, the structured trend and the
// irregular patches (sww_tile.cu), the restrictions level by level, the update.
// The kernel boundary is the barrier.
//
// Blocks come in groups, one group per member: a block copies the level records of
// its member that the phase touches into shared memory once, then strides over
// that member's items only (no search for the member of an item, and every field
// address from shared memory).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "sww_core.cuh"
#include "sww_kernels.h"
#include "sww_stage.h"

namespace sww {

namespace {

#include "sww_bodies.cuh"

constexpr int BATCH_TPB = 256;
constexpr int MAXL = 12;
constexpr int MAXM = 128;
enum {
    PH_FILL = 0, PH_RESTRICT, PH_DIV, PH_UPDATE, PH_SAVE, PH_DT, PH_DT_FINAL, PH_PARTIAL,
    PH_DETAILS, PH_THRESH, PH_INV_A, PH_INV_B, PH_INV_FILL, PH_OUT
};

struct MaxU64 {
    __device__ unsigned long long operator()(unsigned long long x, unsigned long long y) const { return x > y ? x : y; }
};
struct MinU64 {
    __device__ unsigned long long operator()(unsigned long long x, unsigned long long y) const { return x < y ? x : y; }
};

// block reduction of one word per thread (every thread returns the block's value)
template <class Op>
__device__ unsigned long long block_reduce_u64(unsigned long long v, Op op, unsigned long long* sh) {
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_down_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < nw; ++k) v = op(v, sh[k]);
        sh[0] = v;
    }
    __syncthreads();
    return sh[0];
}

// items of `n_entries` entries of `list` (levels from the staged records `sl`),
// block b of bpm blocks of the member
template <int KINDS, class R, class Body>
__device__ __forceinline__ void member_items(const DevLevelT<R>* sl, const int32_t* __restrict__ list,
                                             int64_t n_entries, int P, int b, int bpm, Body body) {
    constexpr uint32_t NS = slots_of<KINDS>();
    const int lp = __ffs(P) - 1;
    const uint32_t n = uint32_t(n_entries) * (NS << lp);
    const uint32_t stride = uint32_t(bpm) * blockDim.x;
    for (uint32_t it = uint32_t(b) * blockDim.x + threadIdx.x; it < n; it += stride) {
        const uint32_t e = (it >> lp) / NS;
        const int32_t ent = list[e];
        const DevLevelT<R>& L = sl[ent >> LVL_SHIFT];
        visit_item<KINDS>(L, int64_t(ent & PATCH_MASK), it - ((e * NS) << lp), P, body);
    }
}

// items of work lists k0 and k1 (k1 < 0: none) of level L, block b of the
// member's bpm blocks: body(0, id) for list k0, body(1, id) for list k1
template <class R, class Body>
__device__ __forceinline__ void member_wl(const DevLevelT<R>& L, int k0, int k1, int b, int bpm, Body body) {
    const int n0 = L.wl_n[k0], n1 = k1 >= 0 ? L.wl_n[k1] : 0;
    const int32_t* __restrict__ l0 = L.wl + wl_off(L, k0);
    const int32_t* __restrict__ l1 = k1 >= 0 ? L.wl + wl_off(L, k1) : l0;
    for (int i = b * int(blockDim.x) + int(threadIdx.x); i < n0 + n1; i += bpm * int(blockDim.x)) {
        if (i < n0)
            body(0, int64_t(l0[i]));
        else
            body(1, int64_t(l1[i - n0]));
    }
}

// Eight blocks per SM (32 registers, a few spilled): the phases are chains of
// dependent gathers, and more resident warps hide more of their latency (measured
// 15 % faster than the 44-register build at 62 % occupancy).
template <class R>
__global__ void __launch_bounds__(BATCH_TPB, 8) k_phase_batch(BatchArgs<R> a, int phase, int j, int bpm) {
    __shared__ DevLevelT<R> sl[MAXL];
    const int m = blockIdx.x / bpm, b = blockIdx.x % bpm;
    const MemberRef<R>* mr = a.m + m;
    const int jtop = mr->jtop;
    // one block per member
    if (phase == PH_DT_FINAL) {
        if (threadIdx.x == 0) {
            *mr->dt = cfl_step<R>(mr->lvs, mr->red, mr->cfl);
        }
        return;
    }
    if (phase == PH_THRESH) {   // relative thresholds on the live maxima (a prescribed velocity has none)
        if (threadIdx.x == 0) {
            mr->thr[0] = mr->eps_c * __longlong_as_double(static_cast<long long>(mr->red[2]));
            mr->thr[1] = mr->advect ? INFINITY : mr->eps_c * __longlong_as_double(static_cast<long long>(mr->red[3]));
        }
        return;
    }
    if (phase == PH_OUT) {
        BatchOut* o = reinterpret_cast<BatchOut*>(a.out) + m;
        const int t = threadIdx.x;
        if (t < 16) {
            const bool in = t >= a.jmin && t <= mr->jmax;
            o->counts[t] = in ? *mr->lvs[t].npatches : 0;
            o->live[t] = in ? mr->lvs[t].wl_n[WL_LIVE] : 0;
        }
        if (t == 0) {
            o->dt = *mr->dt;
            o->err = *mr->err;
        }
        return;
    }
    // level-serial phases skip the members that do not reach the level
    if (phase == PH_FILL && j > jtop) return;
    if ((phase == PH_RESTRICT || phase == PH_DIV || phase == PH_PARTIAL) && j > jtop - 1) return;
    const bool inv = phase == PH_INV_A || phase == PH_INV_B || phase == PH_INV_FILL;
    if (inv && j > mr->j1) return;
    // the member's records of the levels the phase reads (the inverse transform
    // reaches one level above the top)
    const bool serial = phase == PH_RESTRICT || phase == PH_DIV || phase == PH_PARTIAL;
    const int lo = (phase == PH_FILL || phase == PH_INV_A || phase == PH_INV_FILL) ? j - 1 : (serial || inv) ? j : a.jmin;
    const int hi = (phase == PH_RESTRICT || phase == PH_PARTIAL) ? j + 1 : (phase == PH_FILL || phase == PH_DIV || inv) ? j : jtop;
    {
        const int words = int((hi - lo + 1) * sizeof(DevLevelT<R>) / sizeof(int));
        const int* src = reinterpret_cast<const int*>(mr->lvs + lo);
        int* dst = reinterpret_cast<int*>(sl + lo);
        for (int k = threadIdx.x; k < words; k += blockDim.x) dst[k] = src[k];
    }
    __syncthreads();
    const R H = R(a.H), g = R(a.g);
    switch (phase) {
        case PH_FILL:
        case PH_INV_FILL:
            // ghost nodes and edges of level j from level j - 1
            member_wl(sl[j], WL_GN, WL_GE, b, bpm, [&](int k, int64_t id) {
                if (k == 0)
                    fill_node(sl[j], sl[j - 1], id);
                else
                    fill_edge(sl[j], sl[j - 1], id);
            });
            break;
        case PH_RESTRICT:
            // covered nodes and the edges with a covered end of level j
            member_wl(sl[j], WL_CN, WL_RE, b, bpm,
                      [&](int k, int64_t id) { restrict_item(sl[j], sl[j + 1], k == 0 ? K_NODE : K_EDGE, id); });
            break;
        case PH_DIV:
            member_wl(sl[j], WL_DN, -1, b, bpm, [&](int, int64_t id) { div_at(sl[j], id); });
            break;
        case PH_SAVE:
            // the RK base, and the time step: given (a.dt > 0) or its reduction words reset
            if (b == 0 && threadIdx.x == 0) {
                if (a.dt_given > 0) {
                    *mr->dt = a.dt_given;
                    mr->red[2] = 0ull;
                    mr->red[3] = 0ull;
                } else {
                    for (int w = 0; w < RED_WORDS; ++w) mr->red[w] = 0ull;
                }
            }
            member_items<K_NODE | K_EDGE>(sl, mr->all_list, *mr->all_count, a.P, b, bpm,
                                          [&](const DevLevelT<R>& L, int kind, int64_t id, int64_t) {
                                              if (kind == K_NODE) {
                                                  if (L.nflag[id] & LIVE) L.dh0[id] = L.dh[id];
                                              } else if (L.eflag[id] & LIVE) {
                                                  L.u0[id] = L.u[id];
                                              }
                                          });
            break;
        case PH_DT: {
            // largest omega^2 over live nodes (none with a prescribed velocity) and,
            // per level, largest |u| over live edges with u != 0 (NaN left out); the
            // step in PH_DT_FINAL (as k_dt and k_dt_final)
            __shared__ unsigned long long sh[BATCH_TPB / 32];
            __shared__ unsigned long long slev[RED_WORDS - RED_LEVEL];
            if (threadIdx.x < RED_WORDS - RED_LEVEL) slev[threadIdx.x] = 0ull;
            __syncthreads();
            unsigned long long wmax = 0;
            LevelMax um;
            member_items<K_NODE | K_EDGE>(sl, mr->all_list, *mr->all_count, a.P, b, bpm,
                                          [&](const DevLevelT<R>& L, int kind, int64_t id, int64_t) {
                                              if (kind == K_NODE) {
                                                  if (L.advect || !(L.nflag[id] & LIVE)) return;
                                                  wmax = max(wmax, dbits(omega2_at(L, id, a.H, a.g)));
                                              } else if (L.eflag[id] & LIVE) {
                                                  const unsigned long long k = abs_key(L.u[id]);
                                                  if (k && k <= inf_key<R>()) um.add(L.J, k, slev);
                                              }
                                          });
            um.flush(slev);
            wmax = block_reduce_u64(wmax, MaxU64(), sh);   // synchronises the block: slev is complete
            if (threadIdx.x == 0 && wmax) atomicMax(&mr->red[0], wmax);
            if (threadIdx.x < RED_WORDS - RED_LEVEL && slev[threadIdx.x])
                atomicMax(&mr->red[RED_LEVEL + threadIdx.x], slev[threadIdx.x]);
            break;
        }
        case PH_DETAILS: {
            // the wavelet coefficients (levels above Jmin) and, in the same pass, max |dh|
            // over live nodes and max |u| over live edges of every level (keys of the
            // field type, widened to FP64 once per block, as k_maxabs; the details only
            // read dh and u)
            __shared__ unsigned long long shm[BATCH_TPB / 32];
            unsigned long long hmax = 0, umax = 0;
            member_items<K_NODE | K_EDGE | K_CEDGE>(sl, mr->all_list, *mr->all_count, a.P, b, bpm,
                                                    [&](const DevLevelT<R>& L, int kind, int64_t id, int64_t el) {
                                                        if (kind == K_NODE) {
                                                            if (L.nflag[id] & LIVE) hmax = max(hmax, abs_key(L.dh[id]));
                                                        } else if (kind == K_EDGE) {
                                                            if (L.eflag[id] & LIVE) umax = max(umax, abs_key(L.u[id]));
                                                        }
                                                        if (L.J > a.jmin) details_item(L, (&L)[-1], kind, id, el);
                                                    });
            hmax = block_reduce_u64(hmax, MaxU64(), shm);
            umax = block_reduce_u64(umax, MaxU64(), shm);
            if (threadIdx.x == 0) {
                if (hmax) atomicMax(&mr->red[2], dbits(key_value<R>(hmax)));
                if (umax) atomicMax(&mr->red[3], dbits(key_value<R>(umax)));
            }
            break;
        }
        case PH_INV_A:
            member_items<K_NODE | K_EDGE>(sl, sl[j].patches, *sl[j].npatches, a.P, b, bpm,
                                          [&](const DevLevelT<R>& L, int kind, int64_t id, int64_t) {
                                              inverse_a_item(L, (&L)[-1], kind, id);
                                          });
            break;
        case PH_INV_B:
            member_items<K_NODE>(sl, sl[j].patches, *sl[j].npatches, a.P, b, bpm,
                                 [&](const DevLevelT<R>& L, int, int64_t id, int64_t) { inverse_b_item(L, id); });
            break;
        case PH_PARTIAL:
            // R_h at covered nodes of level j from level j + 1 (Eq. Rh)
            member_wl(sl[j], WL_CN, -1, b, bpm, [&](int, int64_t id) {
                                     const DevLevelT<R>& L = sl[j];
                                     if (!(L.nflag[id] & COVERED)) return;
                                     const DevLevelT<R>& F = (&L)[1];
                                     R v = F.dh[L.c2f[id]];
#pragma unroll
                                     for (int q = 0; q < 12; ++q) {
                                         const int32_t mm = L.mk_i[q * L.N + id];
                                         if (mm < 0 || !(F.nflag[mm] & LIVE)) continue;
                                         v += L.mk_w[q * L.N + id] * height_detail(F, mm);
                                     }
                                     L.dh[id] = v;
                                 });
            break;
        default: {
            const R dt = R(*mr->dt);
            const RKStageR<R> sr(a.st);
            member_items<K_NODE | K_EDGE>(sl, mr->all_list, *mr->all_count, a.P, b, bpm,
                                          [&](const DevLevelT<R>& L, int kind, int64_t id, int64_t) {
                                              if (kind == K_NODE)
                                                  update_node(L, id, sr, dt);
                                              else
                                                  update_edge(L, id, sr, dt);
                                          });
        }
    }
}

}  // namespace

template <class R>
cudaError_t launch_stage_batch_part(const BatchArgs<R>& a, const int64_t* level_entries, int64_t irr_entries, int nsm,
                                    int part, cudaStream_t s) {
    if (a.nm < 1 || a.nm > MAXM || a.jtop_max + 1 > MAXL) return cudaErrorInvalidValue;
    int64_t all = 0;
    for (int j = a.jmin; j <= a.jtop_max; ++j) all += level_entries[j];
    // blocks per member: enough for the member's share of the bound, at most two
    // waves of 8 blocks of 256 per SM over all members (measured a little faster
    // than one wave: the members' shares are uneven)
    const int cap = std::max(1, 16 * nsm / a.nm);
    auto bpm = [&](int64_t entries, int slots) {
        const int64_t per = (entries + a.nm - 1) / a.nm * a.P * slots;
        return int(std::max<int64_t>(1, std::min<int64_t>((per + BATCH_TPB - 1) / BATCH_TPB, cap)));
    };
    auto go = [&](int phase, int j, int k) {
        count_launch(1);
        k_phase_batch<R><<<unsigned(a.nm * k), BATCH_TPB, 0, s>>>(a, phase, j, k);
        return cudaGetLastError();
    };
    cudaError_t e = cudaSuccess;
    switch (part) {
        case 0:
            for (int j = a.jmin + 1; j <= a.jtop_max && e == cudaSuccess; ++j) e = go(PH_FILL, j, bpm(level_entries[j], 4));
            break;
        case 1:
        case 2:
            e = launch_tile_trend(a, all, irr_entries, nsm, part, s);
            break;
        case 3:
            for (int j = a.jtop_max - 1; j >= a.jmin && e == cudaSuccess; --j) {
                e = go(PH_RESTRICT, j, bpm(level_entries[j], 4));
                if (e == cudaSuccess) e = go(PH_DIV, j, bpm(level_entries[j], 1));
            }
            break;
        default:
            e = go(PH_UPDATE, 0, bpm(all, 4));
    }
    return e;
}

template <class R>
cudaError_t launch_stage_batch_phases(const BatchArgs<R>& a, const int64_t* level_entries, int64_t irr_entries, int nsm,
                                      cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    for (int part = 0; part < 5 && e == cudaSuccess; ++part)
        e = launch_stage_batch_part(a, level_entries, irr_entries, nsm, part, s);
    return e;
}

template <class R>
static int batch_bpm(const BatchArgs<R>& a, int64_t entries, int slots, int nsm) {
    const int cap = std::max(1, 16 * nsm / a.nm);   // two waves, as in launch_stage_batch_part
    const int64_t per = (entries + a.nm - 1) / a.nm * a.P * slots;
    return int(std::max<int64_t>(1, std::min<int64_t>((per + BATCH_TPB - 1) / BATCH_TPB, cap)));
}

template <class R>
static cudaError_t batch_go(const BatchArgs<R>& a, int phase, int j, int k, cudaStream_t s) {
    count_launch(1);
    k_phase_batch<R><<<unsigned(a.nm * k), BATCH_TPB, 0, s>>>(a, phase, j, k);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_batch_pre(const BatchArgs<R>& a, const int64_t* level_entries, int nsm, double dt, cudaStream_t s) {
    if (a.nm < 1 || a.nm > MAXM || a.jtop_max + 1 > MAXL) return cudaErrorInvalidValue;
    int64_t all = 0;
    for (int j = a.jmin; j <= a.jtop_max; ++j) all += level_entries[j];
    BatchArgs<R> b = a;
    b.dt_given = dt;
    cudaError_t e = batch_go(b, PH_SAVE, 0, batch_bpm(b, all, 4, nsm), s);
    if (e == cudaSuccess && !(dt > 0)) {
        e = batch_go(b, PH_DT, 0, batch_bpm(b, all, 4, nsm), s);
        if (e == cudaSuccess) e = batch_go(b, PH_DT_FINAL, 0, 1, s);
    }
    return e;
}

template <class R>
cudaError_t launch_batch_post(const BatchArgs<R>& a, const int64_t* level_entries, int nsm, cudaStream_t s) {
    if (a.nm < 1 || a.nm > MAXM || a.jtop_max + 1 > MAXL) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    for (int j = a.jtop_max - 1; j >= a.jmin && e == cudaSuccess; --j)
        e = batch_go(a, PH_PARTIAL, j, batch_bpm(a, level_entries[j], 1, nsm), s);
    for (int j = a.jmin + 1; j <= a.jtop_max && e == cudaSuccess; ++j)
        e = batch_go(a, PH_FILL, j, batch_bpm(a, level_entries[j], 4, nsm), s);
    return e;
}

template <class R>
cudaError_t launch_batch_adapt_pre(const BatchArgs<R>& a, const int64_t* level_entries, int nsm, cudaStream_t s) {
    if (a.nm < 1 || a.nm > MAXM || a.jtop_max + 1 > MAXL) return cudaErrorInvalidValue;
    int64_t all = 0;
    for (int j = a.jmin; j <= a.jtop_max; ++j) all += level_entries[j];
    cudaError_t e = batch_go(a, PH_DETAILS, 0, batch_bpm(a, all, 7, nsm), s);
    if (e == cudaSuccess) e = batch_go(a, PH_THRESH, 0, 1, s);
    return e;
}

template <class R>
cudaError_t launch_batch_adapt_post(const BatchArgs<R>& a, const int64_t* level_entries, int j1_max, int nsm,
                                    cudaStream_t s) {
    if (a.nm < 1 || a.nm > MAXM || j1_max + 1 > MAXL) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    for (int j = a.jmin + 1; j <= j1_max && e == cudaSuccess; ++j) {
        const int k = batch_bpm(a, level_entries[j], 4, nsm);
        e = batch_go(a, PH_INV_A, j, k, s);
        if (e == cudaSuccess) e = batch_go(a, PH_INV_B, j, batch_bpm(a, level_entries[j], 1, nsm), s);
        if (e == cudaSuccess) e = batch_go(a, PH_INV_FILL, j, k, s);
    }
    return e;
}

template <class R>
cudaError_t launch_batch_out(const BatchArgs<R>& a, cudaStream_t s) {
    if (a.nm < 1 || a.nm > MAXM) return cudaErrorInvalidValue;
    return batch_go(a, PH_OUT, 0, 1, s);
}

template cudaError_t launch_batch_adapt_pre<double>(const BatchArgs<double>&, const int64_t*, int, cudaStream_t);
template cudaError_t launch_batch_adapt_pre<float>(const BatchArgs<float>&, const int64_t*, int, cudaStream_t);
template cudaError_t launch_batch_adapt_post<double>(const BatchArgs<double>&, const int64_t*, int, int, cudaStream_t);
template cudaError_t launch_batch_adapt_post<float>(const BatchArgs<float>&, const int64_t*, int, int, cudaStream_t);
template cudaError_t launch_batch_out<double>(const BatchArgs<double>&, cudaStream_t);
template cudaError_t launch_batch_out<float>(const BatchArgs<float>&, cudaStream_t);
template cudaError_t launch_batch_pre<double>(const BatchArgs<double>&, const int64_t*, int, double, cudaStream_t);
template cudaError_t launch_batch_pre<float>(const BatchArgs<float>&, const int64_t*, int, double, cudaStream_t);
template cudaError_t launch_batch_post<double>(const BatchArgs<double>&, const int64_t*, int, cudaStream_t);
template cudaError_t launch_batch_post<float>(const BatchArgs<float>&, const int64_t*, int, cudaStream_t);
template cudaError_t launch_stage_batch_part<double>(const BatchArgs<double>&, const int64_t*, int64_t, int, int,
                                                     cudaStream_t);
template cudaError_t launch_stage_batch_part<float>(const BatchArgs<float>&, const int64_t*, int64_t, int, int,
                                                    cudaStream_t);
template cudaError_t launch_stage_batch_phases<double>(const BatchArgs<double>&, const int64_t*, int64_t, int,
                                                       cudaStream_t);
template cudaError_t launch_stage_batch_phases<float>(const BatchArgs<float>&, const int64_t*, int64_t, int,
                                                      cudaStream_t);

}  // namespace sww
