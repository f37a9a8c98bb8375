// CUDA kernels of the adaptive wavelet TRiSK step (sm_103a).  Every kernel that
// touches fields is a template on the working precision R: double (the FP64 form)
// or float (the FP32 form: fields, stencils and transforms in FP32; thresholds,
// time step and the mass/energy sums from FP64 arithmetic on the promoted values).
//
// FP64 work runs over active-patch work lists: a fixed grid (a multiple of the SM
// count) strides over the entries of a list, one thread per element of a p x p
// patch; an element is one node, its three edges and two triangles (Sec. 5.2).
// Lists are built on the device after each adaptation, per level and for all
// levels at once (kernels without a level dependency cover every level in one
// launch).  Byte-wide mask work of the adaptation runs densely over a level.
// Readings of silent or garbled passages are those stated in grid.cpp.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "sww_core.cuh"
#include "sww_kernels.h"

namespace sww {

std::atomic<int64_t> g_launches{0};
int64_t kernel_launches() { return g_launches.load(); }
void count_launch(int64_t n) { g_launches += n; }

namespace {

constexpr int TPB = 256;

#include "sww_bodies.cuh"

// ---------------------------------------------------------------------------- list kernels

template <class R>
__global__ void k_update(const DevLevelT<R>* __restrict__ lvs, const int32_t* list, const int32_t* count, int P,
                         RKStage st, const double* __restrict__ dtp) {
    DevLevelT<R> none{};
    R dt = R(dtp ? *dtp : 0.0);
    const RKStageR<R> sr(st);
    ITEMS(K_NODE | K_EDGE, lvs, none, list, count, P) {
        if (kind == K_NODE)
            update_node(L, id, sr, dt);
        else
            update_edge(L, id, sr, dt);
    });
}

template <class R>
__global__ void k_save_base(const DevLevelT<R>* __restrict__ lvs, const int32_t* list, const int32_t* count, int P) {
    DevLevelT<R> none{};
    ITEMS(K_NODE | K_EDGE, lvs, none, list, count, P) {
        if (kind == K_NODE) {
            if (L.nflag[id] & LIVE) L.dh0[id] = L.dh[id];
        } else if (L.eflag[id] & LIVE) {
            L.u0[id] = L.u[id];
        }
    });
}

// ghosts of level F from level C over F's work list
template <class R>
__global__ void k_fill(DevLevelT<R> F, DevLevelT<R> C, const int32_t* list, const int32_t* count, int P) {
    ITEMS(K_NODE | K_EDGE, (const DevLevelT<R>*)nullptr, F, list, count, P) {
        if (kind == K_NODE)
            fill_node(L, C, id);
        else
            fill_edge(L, C, id);
    });
}

// restriction from F = level j+1 to C = level j (Sec. 3.1)
template <class R>
__global__ void k_restrict(DevLevelT<R> C, DevLevelT<R> F, const int32_t* list, const int32_t* count, int P) {
    ITEMS(K_NODE | K_EDGE, (const DevLevelT<R>*)nullptr, C, list, count, P) { restrict_item(L, F, kind, id); });
}

template <class R>
__global__ void k_div(DevLevelT<R> C, const int32_t* list, const int32_t* count, int P) {
    ITEMS(K_NODE, (const DevLevelT<R>*)nullptr, C, list, count, P) {
        if (restricted_div_node(L, id)) div_at(L, id);
    });
}

// R_h at covered nodes of C from level F (Eq. Rh; coefficients of non-live points are zero)
template <class R>
__global__ void k_partial(DevLevelT<R> C, DevLevelT<R> F, const int32_t* list, const int32_t* count, int P) {
    ITEMS(K_NODE, (const DevLevelT<R>*)nullptr, C, list, count, P) {
        if (!(L.nflag[id] & COVERED)) return;
        R s = F.dh[L.c2f[id]];
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            int32_t m = L.mk_i[q * L.N + id];
            if (m < 0 || !(F.nflag[m] & LIVE)) continue;
            s += L.mk_w[q * L.N + id] * height_detail(F, m);
        }
        L.dh[id] = s;
    });
}

// wavelet coefficients at live points (body details_item)
template <class R>
__global__ void k_details(const DevLevelT<R>* __restrict__ lvs, const int32_t* list, const int32_t* count, int P,
                          int jmin) {
    DevLevelT<R> none{};
    ITEMS(K_NODE | K_EDGE | K_CEDGE, lvs, none, list, count, P) {
        if (L.J == jmin) return;
        details_item(L, lvs[L.J - 1], kind, id, el);
    });
}

// inverse transform of the retained coefficients onto the live points of F:
// (a) even nodes and all edges from level C, (b) odd nodes from the even ones
// (bodies inverse_a_item, inverse_b_item)
template <class R>
__global__ void k_inverse_a(DevLevelT<R> F, DevLevelT<R> C, const int32_t* list, const int32_t* count, int P) {
    ITEMS(K_NODE | K_EDGE, (const DevLevelT<R>*)nullptr, F, list, count, P) { inverse_a_item(L, C, kind, id); });
}

template <class R>
__global__ void k_inverse_b(DevLevelT<R> F, const int32_t* list, const int32_t* count, int P) {
    ITEMS(K_NODE, (const DevLevelT<R>*)nullptr, F, list, count, P) { inverse_b_item(L, id); });
}

// ---------------------------------------------------------------------------- reductions

// block-wide reduction; `idle` is the operation's identity (fills lanes without a warp)
template <typename T, typename Op>
__device__ T block_reduce(T v, Op op, T* sh, T idle) {
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_down_sync(0xffffffffu, v, o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    if (w == 0) {
        v = l < nw ? sh[l] : idle;
        for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_down_sync(0xffffffffu, v, o));
    }
    __syncthreads();
    return v;
}

struct MaxOp {
    __device__ unsigned long long operator()(unsigned long long a, unsigned long long b) const { return a > b ? a : b; }
};
struct MinOp {
    __device__ unsigned long long operator()(unsigned long long a, unsigned long long b) const { return a < b ? a : b; }
};
struct AddOp {
    __device__ unsigned long long operator()(unsigned long long a, unsigned long long b) const { return a + b; }
};

// max |dh| over live nodes, max |u| over live edges: compared as keys of the field
// type, widened to FP64 once per block (bit patterns of non-negative doubles)
template <class R>
__global__ void k_maxabs(const DevLevelT<R>* __restrict__ lvs, const int32_t* list, const int32_t* count, int S,
                         unsigned long long* red) {
    __shared__ unsigned long long sh[32];
    DevLevelT<R> none{};
    unsigned long long a = 0, b = 0;
    ITEMS(K_NODE | K_EDGE, lvs, none, list, count, S) {
        if (kind == K_NODE) {
            if (L.nflag[id] & LIVE) a = max(a, abs_key(L.dh[id]));
        } else if (L.eflag[id] & LIVE) {
            b = max(b, abs_key(L.u[id]));
        }
    });
    a = block_reduce(a, MaxOp(), sh, 0ull);
    if (threadIdx.x == 0 && a) atomicMax(&red[2], dbits(key_value<R>(a)));
    b = block_reduce(b, MaxOp(), sh, 0ull);
    if (threadIdx.x == 0 && b) atomicMax(&red[3], dbits(key_value<R>(b)));
}

// largest omega^2 = f^2 + g h (pi/dx)^2 over live nodes (none with a prescribed
// velocity, which carries no waves) and, per level, the largest |u| over live
// edges with u != 0 (NaN left out, as dx/|u| with u NaN takes no part); the step
// itself in k_dt_final
template <class R>
__global__ void k_dt(const DevLevelT<R>* __restrict__ lvs, const int32_t* list, const int32_t* count, int S, double H,
                     double g, unsigned long long* red) {
    __shared__ unsigned long long sh[32];
    __shared__ unsigned long long slev[RED_WORDS - RED_LEVEL];
    if (threadIdx.x < RED_WORDS - RED_LEVEL) slev[threadIdx.x] = 0ull;
    __syncthreads();
    DevLevelT<R> none{};
    unsigned long long a = 0;
    LevelMax um;
    ITEMS(K_NODE | K_EDGE, lvs, none, list, count, S) {
        if (kind == K_NODE) {
            if (L.advect || !(L.nflag[id] & LIVE)) return;
            a = max(a, dbits(omega2_at(L, id, H, g)));
        } else if (L.eflag[id] & LIVE) {
            const unsigned long long k = abs_key(L.u[id]);
            if (k && k <= inf_key<R>()) um.add(L.J, k, slev);
        }
    });
    um.flush(slev);
    a = block_reduce(a, MaxOp(), sh, 0ull);   // synchronises the block: slev is complete
    if (threadIdx.x == 0 && a) atomicMax(&red[0], a);
    if (threadIdx.x < RED_WORDS - RED_LEVEL && slev[threadIdx.x]) atomicMax(&red[RED_LEVEL + threadIdx.x], slev[threadIdx.x]);
}

template <class R>
__global__ void k_dt_final(const DevLevelT<R>* lvs, const unsigned long long* red, double cfl, double* dt) {
    if (threadIdx.x || blockIdx.x) return;
    *dt = cfl_step<R>(lvs, red, cfl);
}

// a prescribed velocity takes no part in the significance test (eps_u infinite
// unless given)
__global__ void k_thresholds(const unsigned long long* red, double eps, double eps_h, double eps_u, int advect,
                             double* thr) {
    if (threadIdx.x || blockIdx.x) return;
    thr[0] = eps_h > 0 ? eps_h : eps * __longlong_as_double(static_cast<long long>(red[2]));
    thr[1] = eps_u > 0 ? eps_u : advect ? INFINITY : eps * __longlong_as_double(static_cast<long long>(red[3]));
}

// Neumaier-compensated partial sums of mass and energy over level Jmin (dense)
__device__ __forceinline__ void neumaier(double& s, double& c, double x) {
    double t = s + x;
    c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
    s = t;
}

template <class R>
__global__ void k_sums(DevLevelT<R> L, double H, double g, double* part) {
    __shared__ double sh[2][TPB];
    int64_t v = gid();
    double m = 0, en = 0;
    if (v < L.N) {
        double h = H + double(L.dh[v]), A = L.A_i[v], ke = 0.0;
        for (int k = 0; k < L.deg[v]; ++k) {
            int64_t e = L.ring_e[k * L.N + v] >> 1;
            double ue = double(L.u[e]);
            ke += 0.25 * L.l_e[e] * L.d_e[e] * ue * ue;
        }
        m = A * h;
        en = g * h * (0.5 * g * h * A + ke);
    }
    sh[0][threadIdx.x] = m;
    sh[1][threadIdx.x] = en;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0, c0 = 0, s1 = 0, c1 = 0;
        for (int k = 0; k < blockDim.x; ++k) neumaier(s0, c0, sh[0][k]), neumaier(s1, c1, sh[1][k]);
        part[4 * blockIdx.x + 0] = s0;
        part[4 * blockIdx.x + 1] = c0;
        part[4 * blockIdx.x + 2] = s1;
        part[4 * blockIdx.x + 3] = c1;
    }
}

__global__ void k_sums_final(const double* part, int nblk, double* out) {
    if (threadIdx.x || blockIdx.x) return;
    double s0 = 0, c0 = 0, s1 = 0, c1 = 0;
    for (int b = 0; b < nblk; ++b) {
        neumaier(s0, c0, part[4 * b]);
        neumaier(s0, c0, part[4 * b + 1]);
        neumaier(s1, c1, part[4 * b + 2]);
        neumaier(s1, c1, part[4 * b + 3]);
    }
    out[0] = s0 + c0;
    out[1] = s1 + c1;
}

template <class R>
__global__ void k_count(DevLevelT<R> L, unsigned long long* cnt) {
    __shared__ unsigned long long sh[32];
    int64_t i = gid();
    unsigned long long a = 0, b = 0, c = 0;
    if (i < L.N) a = (L.nflag[i] & LIVE) ? 1 : 0, b = (L.nflag[i] & GHOST) ? 1 : 0;
    if (i < L.E) c = (L.eflag[i] & LIVE) ? 1 : 0;
    a = block_reduce(a, AddOp(), sh, 0ull);
    if (threadIdx.x == 0) atomicAdd(&cnt[0], a);
    b = block_reduce(b, AddOp(), sh, 0ull);
    if (threadIdx.x == 0) atomicAdd(&cnt[1], b);
    c = block_reduce(c, AddOp(), sh, 0ull);
    if (threadIdx.x == 0) atomicAdd(&cnt[2], c);
}

// ---------------------------------------------------------------------------- dense level kernels

// thread t of a multi-level dense launch -> (level, index within the level)
__device__ __forceinline__ bool locate(const Span& sp, int64_t t, int& j, int64_t& i) {
    for (j = sp.ja; j <= sp.jb; ++j)
        if (t < sp.off[j + 1 - sp.ja]) {
            i = t - sp.off[j - sp.ja];
            return true;
        }
    return false;
}

// Visit (level, index) of a multi-level dense launch.  The top level of a span may be
// a tail level (the level above the top live level): it gets a fixed number of
// threads that stride over it, and only when a point one level down was significant,
// since otherwise it cannot gain a point in this adaptation.
template <class Body>
__device__ __forceinline__ void dense_each(const Span& sp, int64_t t, const int32_t* __restrict__ sig_any, Body body) {
    int j;
    int64_t i;
    if (!locate(sp, t, j, i)) return;
    if (j != sp.tail_j) {
        body(j, i);
        return;
    }
    if (!sig_any[j - 1]) return;
    const int64_t stride = sp.off[j + 1 - sp.ja] - sp.off[j - sp.ja];
    for (; i < sp.tail_n; i += stride) body(j, i);
}

#define DENSE_EACH(sp, t, any) dense_each(sp, t, any, [&] __device__(int j, int64_t i)

// full restriction used at initialisation: R_h at every node, mean of halves at every edge
template <class R>
__global__ void k_restrict_full(DevLevelT<R> C, DevLevelT<R> F) {
    int64_t i = gid();
    if (i < C.N) {
        R s = F.dh[C.c2f[i]];
        for (int q = 0; q < 12; ++q) {
            int32_t m = C.mk_i[q * C.N + i];
            if (m >= 0) s += C.mk_w[q * C.N + i] * height_detail(F, m);
        }
        C.dh[i] = s;
    }
    if (i < C.E) C.u[i] = R(0.5) * (F.u[C.half[i]] + F.u[C.half[C.E + i]]);
}

// level F in full (Sec. 2.2): live points keep their values, every other point takes
// the inverse transform with zero coefficients of the full level below (cdh, cu;
// C gives the coarse half-edge table).  By the graded closure no live coefficient
// touches a non-live even node, which therefore takes the coarse value.  A
// prescribed velocity is kept as set.
template <class R>
__global__ void k_uniform(DevLevelT<R> F, DevLevelT<R> C, const R* __restrict__ cdh, const R* __restrict__ cu,
                          R* __restrict__ odh, R* __restrict__ ou) {
    const int64_t i = gid();
    if (i < F.N) {
        R v;
        if (F.nflag[i] & LIVE) {
            v = F.dh[i];
        } else if (F.f2c[i] >= 0) {
            v = cdh[F.f2c[i]];
        } else {
            v = R(0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int32_t p = F.par[q * F.N + i];
                v += F.ptw[q * F.N + i] * ((F.nflag[p] & LIVE) ? F.dh[p] : cdh[F.f2c[p]]);
            }
        }
        odh[i] = v;
    }
    if (i < F.E) {
        R v;
        if (F.advect || (F.eflag[i] & LIVE)) {
            v = F.u[i];
        } else {
            const R P = predict(F, cu, i);
            const int kind = F.fe_kind[i];
            if (kind == 2) {
                v = P;
            } else {
                const int64_t E = F.fe_ce[i];
                const int32_t other = C.half[(kind == 0 ? C.E : 0) + E];
                const R uc = cu[E];
                v = (F.eflag[other] & LIVE) ? R(2) * uc - F.u[other]
                                            : P + R(0.5) * (R(2) * uc - P - predict(F, cu, other));
            }
        }
        ou[i] = v;
    }
}

// the current live set becomes the support of the stored coefficients (WASLIVE),
// so that an inverse transform without adaptation uses every live coefficient
template <class R>
__global__ void k_mark_support(const DevLevelT<R>* __restrict__ lvs, const int32_t* list, const int32_t* count,
                               int P) {
    DevLevelT<R> none{};
    ITEMS(K_NODE | K_EDGE, lvs, none, list, count, P) {
        uint8_t* f = kind == K_NODE ? &L.nflag[id] : &L.eflag[id];
        *f = uint8_t((*f & ~WASLIVE) | ((*f & LIVE) ? WASLIVE : 0));
    });
}

// Dense multi-level mask kernels (bodies in sww_bodies.cuh).  sig_any[j] records
// whether level j holds a significant point.
template <class R>
__global__ void k_zero_sig(const DevLevelT<R>* __restrict__ lvs, Span sp, const int32_t* sig_any) {
    DENSE_EACH(sp, gid(), sig_any) { lvs[j].sig[i] = 0; });
}

template <class R>
__global__ void k_sig(const DevLevelT<R>* __restrict__ lvs, Span sp, const double* __restrict__ thr, int32_t* sig_any) {
    DENSE_EACH(sp, gid(), sig_any) {
        const DevLevelT<R>& F = lvs[j];
        const DevLevelT<R>& C = lvs[j - 1];
        bool any = false;
        const R eh = sig_thr<R>(thr[0]), eu = sig_thr<R>(thr[1]);
        if (i < F.N) any |= sig_node(F, i, eh);
        if (i < F.E) any |= sig_edge(F, i, eu);
        if (i < C.E) any |= sig_cedge(F, C, i, eu);
        if (any) sig_any[j] = 1;
    });
}

template <class R>
__global__ void k_adjacent(const DevLevelT<R>* __restrict__ lvs, Span sp, int jmin, const int32_t* sig_any) {
    DENSE_EACH(sp, gid(), sig_any) { adjacent_node(lvs[j], lvs[j - 1], j - 1 > jmin, i); });
}

// On a tail level the fixed grid strides over the level.
template <class R>
__global__ void k_close(DevLevelT<R> F, DevLevelT<R> Fp, int has_finer, const int32_t* sig_any, int tail) {
    if (tail && !sig_any[F.J - 1]) return;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t x = gid(); x < F.N; x += stride) close_node(F, Fp, has_finer != 0, x);
}

template <class R>
__global__ void k_live(const DevLevelT<R>* __restrict__ lvs, Span sp, int all_level, const int32_t* sig_any) {
    DENSE_EACH(sp, gid(), sig_any) { live_node(lvs[j], i, all_level == -2 || j == all_level); });
}

template <class R>
__global__ void k_live_edges(const DevLevelT<R>* __restrict__ lvs, Span sp, const int32_t* sig_any) {
    DENSE_EACH(sp, gid(), sig_any) { live_edge(lvs[j], i); });
}

template <class R>
__global__ void k_dilate(const DevLevelT<R>* __restrict__ lvs, Span sp, int forward, const int32_t* sig_any) {
    DENSE_EACH(sp, gid(), sig_any) { dilate_node(lvs[j], i, forward != 0); });
}

template <class R>
__global__ void k_ghost(const DevLevelT<R>* __restrict__ lvs, Span sp, int in_band1, const int32_t* sig_any) {
    DENSE_EACH(sp, gid(), sig_any) {
        const DevLevelT<R>& L = lvs[j];
        const uint8_t* band = in_band1 ? L.band1 : L.band0;
        if (i < L.N) ghost_node(L, i, band);
        if (i < L.E) ghost_edge(L, i, band);
    });
}

template <class R>
__global__ void k_covered(const DevLevelT<R>* __restrict__ lvs, Span sp) {
    int j;
    int64_t k;
    if (!locate(sp, gid(), j, k)) return;
    covered_node(lvs[j], lvs[j + 1], k);
}

// patches holding any live or ghost node or edge (one block per patch)
// With lstat, also counts per patch above Jmin: [0] the exact rules' set reaches a
// patch that was not active during the step (a late refinement), [1] a patch the
// previous proposal named holds none of the exact set, [2] the patches proposed.
template <class R>
__global__ void k_patch_flags(const DevLevelT<R>* __restrict__ lvs, Span sp, const int32_t* sig_any,
                              unsigned long long* lstat) {
    int j;
    int64_t pid;
    if (!locate(sp, int64_t(blockIdx.x), j, pid)) return;
    int64_t stride = 0;
    if (j == sp.tail_j) {
        if (!sig_any[j - 1]) return;
        stride = sp.off[j + 1 - sp.ja] - sp.off[j - sp.ja];
    }
    const DevLevelT<R>& L = lvs[j];
    const int64_t pp = L.p * L.p;
    const int64_t np = (j == sp.tail_j) ? sp.tail_n : pid + 1;
    for (; pid < np; pid += (stride ? stride : 1)) {
        int any = 0;
        for (int64_t l = threadIdx.x; l < pp; l += blockDim.x) {
            int64_t e = pid * pp + l;
            if ((L.nflag[e] | L.eflag[e] | L.eflag[L.nelem + e] | L.eflag[2 * L.nelem + e]) & AVAIL) any = 1;
        }
        any = __syncthreads_or(any);
        if (threadIdx.x == 0) {
            if (lstat && j > sp.ja) {
                if (L.pexact[pid] && !L.pflag[pid]) atomicAdd(&lstat[0], 1ull);
                if (L.prop_prev[pid] && !L.pexact[pid]) atomicAdd(&lstat[1], 1ull);
                if (L.prop[pid]) atomicAdd(&lstat[2], 1ull);
            }
            L.pflag[pid] = uint8_t(any);
        }
    }
}

// ascending level-tagged list of flagged patches, then the pole entry when a pole is
// live or ghost (one block; deterministic)
template <class R>
__global__ void k_patch_scan(const DevLevelT<R>* __restrict__ lvs, int ja, const int32_t* sig_any, int tail_j) {
    int j = ja + int(blockIdx.x);
    if (j == tail_j && !sig_any[j - 1]) return;
    patch_scan_level(lvs[j]);
}

template <class R>
__global__ void k_concat(const DevLevelT<R>* __restrict__ lvs, int jmin, int jmax, int32_t* all, int32_t* count,
                         int32_t* irr, int32_t* irr_count) {
    concat_lists(lvs, jmin, jmax, all, count, irr, irr_count);
}

// the point work lists of every level from the all-level list
template <class R>
__global__ void k_wl_build(const DevLevelT<R>* __restrict__ lvs, const int32_t* __restrict__ list,
                           const int32_t* __restrict__ count, int P) {
    DevLevelT<R> none{};
    ITEMS(K_NODE | K_EDGE, lvs, none, list, count, P) { wl_item(L, kind, id); });
}

}  // namespace

// ---------------------------------------------------------------------------- launchers

#define DENSE(kernel, n, ...) (g_launches++, kernel<<<blocks_for((n), TPB), TPB, 0, s>>>(__VA_ARGS__))
#define LIST(kernel, ...) (g_launches++, kernel<<<W.grid, TPB, 0, s>>>(__VA_ARGS__))

template <class R>
static int64_t span(const DevLevelT<R>& L) { return L.E > L.N ? L.E : L.N; }

template <class R>
void launch_update(const WorkT<R>& W, const RKStage& st, const double* dt, cudaStream_t s) {
    LIST(k_update<R>, W.lvs, W.list, W.count, W.S, st, dt);
}
template <class R>
void launch_save_base(const WorkT<R>& W, cudaStream_t s) {
    LIST(k_save_base<R>, W.lvs, W.list, W.count, W.S);
}
template <class R>
void launch_fill(const DevLevelT<R>& F, const DevLevelT<R>& C, const WorkT<R>& W, cudaStream_t s) {
    LIST(k_fill<R>, F, C, W.list, W.count, W.S);
}
template <class R>
void launch_restrict(const DevLevelT<R>& C, const DevLevelT<R>& F, const WorkT<R>& W, cudaStream_t s) {
    LIST(k_restrict<R>, C, F, W.list, W.count, W.S);
}
template <class R>
void launch_div(const DevLevelT<R>& C, const WorkT<R>& W, cudaStream_t s) {
    LIST(k_div<R>, C, W.list, W.count, W.S);
}
template <class R>
void launch_partial(const DevLevelT<R>& C, const DevLevelT<R>& F, const WorkT<R>& W, cudaStream_t s) {
    LIST(k_partial<R>, C, F, W.list, W.count, W.S);
}
template <class R>
void launch_details(const WorkT<R>& W, int jmin, cudaStream_t s) {
    LIST(k_details<R>, W.lvs, W.list, W.count, W.S, jmin);
}
template <class R>
void launch_inverse(const DevLevelT<R>& F, const DevLevelT<R>& C, const WorkT<R>& W, cudaStream_t s) {
    LIST(k_inverse_a<R>, F, C, W.list, W.count, W.S);
    LIST(k_inverse_b<R>, F, W.list, W.count, W.S);
}
template <class R>
void launch_maxabs(const WorkT<R>& W, unsigned long long* red, cudaStream_t s) {
    LIST(k_maxabs<R>, W.lvs, W.list, W.count, W.S, red);
}
template <class R>
void launch_dt(const WorkT<R>& W, double H, double g, unsigned long long* red, cudaStream_t s) {
    LIST(k_dt<R>, W.lvs, W.list, W.count, W.S, H, g, red);
}
template <class R>
void launch_dt_final(const DevLevelT<R>* lvs, const unsigned long long* red, double cfl, double* dt, cudaStream_t s) {
    g_launches++;
    k_dt_final<R><<<1, 32, 0, s>>>(lvs, red, cfl, dt);
}
void launch_thresholds(const unsigned long long* red, double eps, double eh, double eu, int advect, double* thr,
                       cudaStream_t s) {
    g_launches++;
    k_thresholds<<<1, 32, 0, s>>>(red, eps, eh, eu, advect, thr);
}

template <class R>
void launch_restrict_full(const DevLevelT<R>& C, const DevLevelT<R>& F, cudaStream_t s) {
    DENSE(k_restrict_full<R>, span(C), C, F);
}
template <class R>
void launch_uniform(const DevLevelT<R>& F, const DevLevelT<R>& C, const R* cdh, const R* cu, R* odh, R* ou,
                    cudaStream_t s) {
    DENSE(k_uniform<R>, span(F), F, C, cdh, cu, odh, ou);
}
template <class R>
void launch_mark_support(const WorkT<R>& W, cudaStream_t s) {
    LIST(k_mark_support<R>, W.lvs, W.list, W.count, W.S);
}
#define MULTI(kernel, sp, ...)                                                  \
    do {                                                                        \
        int64_t n_ = (sp).off[(sp).jb + 1 - (sp).ja];                           \
        if (n_ > 0) {                                                           \
            g_launches++;                                                       \
            kernel<<<blocks_for(n_, TPB), TPB, 0, s>>>(__VA_ARGS__);            \
        }                                                                       \
    } while (0)

template <class R>
void launch_mask(const MaskArgsT<R>& a, cudaStream_t s) {
    // a.sig_any is cleared by the caller (a proposal may already have marked levels)
    const int32_t* any = a.sig_any;
    // significance, adjacency in space and scale (levels ja+1..jb, independent)
    MULTI(k_zero_sig<R>, a.nodes_f, a.lvs, a.nodes_f, any);
    MULTI(k_sig<R>, a.edges_f, a.lvs, a.edges_f, a.thr, a.sig_any);
    MULTI(k_adjacent<R>, a.nodes_f, a.lvs, a.nodes_f, a.ja, any);
    // graded closure, from the top level down
    for (int j = a.jb; j > a.ja; --j) {
        const DevLevelT<R>& F = a.host[j];
        bool finer = j < a.jb;
        bool tail = j == a.nodes.tail_j;
        unsigned grid = tail ? a.tail_blocks : blocks_for(F.N, TPB);
        g_launches++;
        k_close<R><<<grid, TPB, 0, s>>>(F, finer ? a.host[j + 1] : F, finer, any, tail);
    }
    // live flags, ghost band, covered nodes, patch lists (levels ja..jb)
    MULTI(k_live<R>, a.nodes, a.lvs, a.nodes, a.ja, any);
    MULTI(k_live_edges<R>, a.edges, a.lvs, a.edges, any);
    for (int h = 0; h < a.hops; ++h) MULTI(k_dilate<R>, a.nodes_f, a.lvs, a.nodes_f, h % 2 == 0, any);
    MULTI(k_ghost<R>, a.edges_f, a.lvs, a.edges_f, a.hops % 2 == 1, any);
    if (a.jb > a.ja) MULTI(k_covered<R>, a.nodes_c, a.lvs, a.nodes_c);
    g_launches += 2;
    k_patch_flags<R><<<unsigned(a.patches.off[a.jb + 1 - a.ja]), 64, 0, s>>>(a.lvs, a.patches, any, a.lstat);
    k_patch_scan<R><<<unsigned(a.jb - a.ja + 1), 1024, 0, s>>>(a.lvs, a.ja, any, a.patches.tail_j);
}

template <class R>
void launch_live_all(const DevLevelT<R>* lvs, const Span& nodes, const Span& edges, cudaStream_t s) {
    MULTI(k_live<R>, nodes, lvs, nodes, -2, nullptr);
    MULTI(k_live_edges<R>, edges, lvs, edges, nullptr);
}

template <class R>
void launch_covered_all(const DevLevelT<R>* lvs, const Span& nodes_c, cudaStream_t s) {
    MULTI(k_covered<R>, nodes_c, lvs, nodes_c);
}

template <class R>
void launch_patches_all(const DevLevelT<R>* lvs, const Span& patches, cudaStream_t s) {
    g_launches += 2;
    k_patch_flags<R><<<unsigned(patches.off[patches.jb + 1 - patches.ja]), 64, 0, s>>>(lvs, patches, nullptr,
                                                                                         nullptr);
    k_patch_scan<R><<<unsigned(patches.jb - patches.ja + 1), 1024, 0, s>>>(lvs, patches.ja, nullptr, -1);
}

template <class R>
void launch_concat(const DevLevelT<R>* lvs, int jmin, int jmax, int32_t* all, int32_t* count, int32_t* irr,
                   int32_t* irr_count, int P, unsigned grid, cudaStream_t s) {
    g_launches += 2;
    k_concat<R><<<1, 1024, 0, s>>>(lvs, jmin, jmax, all, count, irr, irr_count);
    k_wl_build<R><<<grid, TPB, 0, s>>>(lvs, all, count, P);
}

template <class R>
int sums_blocks(const DevLevelT<R>& L) {
    return int(blocks_for(L.N, TPB));
}
template <class R>
void launch_sums(const DevLevelT<R>& L, double H, double g, double* part, double* out, cudaStream_t s) {
    int nb = sums_blocks(L);
    g_launches += 2;
    k_sums<R><<<nb, TPB, 0, s>>>(L, H, g, part);
    k_sums_final<<<1, 32, 0, s>>>(part, nb, out);
}
template <class R>
void launch_count(const DevLevelT<R>& L, unsigned long long* cnt, cudaStream_t s) {
    DENSE(k_count<R>, span(L), L, cnt);
}

// field conversion between the working precision and FP64
template <class A, class B>
__global__ void k_convert(const A* __restrict__ x, B* __restrict__ y, int64_t n) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = gid(); i < n; i += stride) y[i] = B(x[i]);
}
template <class A, class B>
void launch_convert(const A* x, B* y, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    g_launches++;
    k_convert<A, B><<<unsigned(std::min<int64_t>(blocks_for(n, TPB), 4096)), TPB, 0, s>>>(x, y, n);
}

#define SWW_INSTANTIATE(R)                                                                                   \
    template void launch_update<R>(const WorkT<R>&, const RKStage&, const double*, cudaStream_t);            \
    template void launch_save_base<R>(const WorkT<R>&, cudaStream_t);                                        \
    template void launch_fill<R>(const DevLevelT<R>&, const DevLevelT<R>&, const WorkT<R>&, cudaStream_t);   \
    template void launch_restrict<R>(const DevLevelT<R>&, const DevLevelT<R>&, const WorkT<R>&, cudaStream_t); \
    template void launch_div<R>(const DevLevelT<R>&, const WorkT<R>&, cudaStream_t);                          \
    template void launch_partial<R>(const DevLevelT<R>&, const DevLevelT<R>&, const WorkT<R>&, cudaStream_t); \
    template void launch_details<R>(const WorkT<R>&, int, cudaStream_t);                                     \
    template void launch_inverse<R>(const DevLevelT<R>&, const DevLevelT<R>&, const WorkT<R>&, cudaStream_t); \
    template void launch_maxabs<R>(const WorkT<R>&, unsigned long long*, cudaStream_t);                      \
    template void launch_dt<R>(const WorkT<R>&, double, double, unsigned long long*, cudaStream_t);          \
    template void launch_dt_final<R>(const DevLevelT<R>*, const unsigned long long*, double, double*, cudaStream_t); \
    template void launch_restrict_full<R>(const DevLevelT<R>&, const DevLevelT<R>&, cudaStream_t);           \
    template void launch_mask<R>(const MaskArgsT<R>&, cudaStream_t);                                         \
    template void launch_live_all<R>(const DevLevelT<R>*, const Span&, const Span&, cudaStream_t);           \
    template void launch_covered_all<R>(const DevLevelT<R>*, const Span&, cudaStream_t);                     \
    template void launch_uniform<R>(const DevLevelT<R>&, const DevLevelT<R>&, const R*, const R*, R*, R*,       \
                                    cudaStream_t);                                                           \
    template void launch_mark_support<R>(const WorkT<R>&, cudaStream_t);                                     \
    template void launch_patches_all<R>(const DevLevelT<R>*, const Span&, cudaStream_t);                     \
    template void launch_concat<R>(const DevLevelT<R>*, int, int, int32_t*, int32_t*, int32_t*, int32_t*, int,     \
                                   unsigned, cudaStream_t);         \
    template int sums_blocks<R>(const DevLevelT<R>&);                                                        \
    template void launch_sums<R>(const DevLevelT<R>&, double, double, double*, double*, cudaStream_t);       \
    template void launch_count<R>(const DevLevelT<R>&, unsigned long long*, cudaStream_t);

SWW_INSTANTIATE(double)
SWW_INSTANTIATE(float)
template void launch_convert<double, float>(const double*, float*, int64_t, cudaStream_t);
template void launch_convert<float, double>(const float*, double*, int64_t, cudaStream_t);

}  // namespace sww
