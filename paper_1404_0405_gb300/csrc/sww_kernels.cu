// CUDA kernels of the adaptive wavelet TRiSK step (sm_103a, FP64).
//
// Every kernel covers one level (or one pair of adjacent levels) with one thread
// per node / edge / triangle; threads of points that are neither live nor ghost
// leave at once after reading one flag byte.  Passages followed are cited at
// each kernel; the readings of silent or garbled passages are those stated in
// grid.cpp and listed with the design notes.
#include <atomic>
#include <cmath>

#include "sww_core.cuh"
#include "sww_kernels.h"

namespace sww {

namespace {

constexpr int TPB = 256;

__device__ __forceinline__ int64_t gid() { return int64_t(blockIdx.x) * blockDim.x + threadIdx.x; }
__device__ __forceinline__ double esign(int32_t code) { return (code & 1) ? -1.0 : 1.0; }

// neighbour across ring edge `code` of node v
__device__ __forceinline__ int32_t ring_nbr(const DevLevel& L, int32_t code) {
    int64_t e = code >> 1;
    return (code & 1) ? L.en[e] : L.en[L.E + e];
}

__device__ __forceinline__ double predict(const DevLevel& F, const double* __restrict__ uc, int64_t fe) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 12; ++k) s += F.vw[k * F.E + fe] * uc[F.vst[k * F.E + fe]];
    return s;
}

__device__ __forceinline__ double height_detail(const DevLevel& F, int64_t x) {
    double s = F.dh[x];
#pragma unroll
    for (int k = 0; k < 4; ++k) s -= F.ptw[k * F.N + x] * F.dh[F.par[k * F.N + x]];
    return s;
}

__device__ __forceinline__ unsigned long long dbits(double x) {
    return static_cast<unsigned long long>(__double_as_longlong(x));
}

// ---------------------------------------------------------------------------- trend (Sec. 3.1)

// potential vorticity q = (curl u + f)/h at triangles (dual cells)
__global__ void k_tri_q(DevLevel L, double H) {
    int64_t t = gid();
    if (t >= L.T) return;
    int32_t n0 = L.tn[t], n1 = L.tn[L.T + t], n2 = L.tn[2 * L.T + t];
    int32_t c0 = L.te[t], c1 = L.te[L.T + t], c2 = L.te[2 * L.T + t];
    if (!(L.nflag[n0] & AVAIL) || !(L.nflag[n1] & AVAIL) || !(L.nflag[n2] & AVAIL)) return;
    if (!(L.eflag[c0 >> 1] & AVAIL) || !(L.eflag[c1 >> 1] & AVAIL) || !(L.eflag[c2 >> 1] & AVAIL)) return;
    double circ = esign(c0) * L.u[c0 >> 1] * L.d_e[c0 >> 1] + esign(c1) * L.u[c1 >> 1] * L.d_e[c1 >> 1] +
                  esign(c2) * L.u[c2 >> 1] * L.d_e[c2 >> 1];
    double hv = L.kite[t] * (H + L.dh[n0]) + L.kite[L.T + t] * (H + L.dh[n1]) + L.kite[2 * L.T + t] * (H + L.dh[n2]);
    double Av = L.A_v[t];
    L.q[t] = (circ / Av + L.f_v[t]) / (hv / Av);
}

// thickness flux F = h_e u at edges
__global__ void k_edge_flux(DevLevel L, double H) {
    int64_t e = gid();
    if (e >= L.E) return;
    if (!(L.eflag[e] & AVAIL)) return;
    int32_t a = L.en[e], b = L.en[L.E + e];
    if (!(L.nflag[a] & AVAIL) || !(L.nflag[b] & AVAIL)) return;
    L.F[e] = 0.5 * ((H + L.dh[a]) + (H + L.dh[b])) * L.u[e];
}

// divergence, kinetic energy and Bernoulli function at nodes
__global__ void k_node(DevLevel L, double g) {
    int64_t v = gid();
    if (v >= L.N) return;
    if (!(L.nflag[v] & AVAIL)) return;
    int dg = L.deg[v];
    double div = 0.0, ke = 0.0;
    for (int k = 0; k < dg; ++k) {
        int32_t code = L.ring_e[k * L.N + v];
        int64_t e = code >> 1;
        if (!(L.eflag[e] & AVAIL)) return;
        div += esign(code) * L.F[e] * L.l_e[e];
        double ue = L.u[e];
        ke += 0.25 * L.l_e[e] * L.d_e[e] * ue * ue;
    }
    double A = L.A_i[v];
    L.c[v] = div / A;
    L.B[v] = g * L.dh[v] + ke / A;
}

// energy-conserving Coriolis tendency +q F.n_left at live edges (TRiSK)
__global__ void k_coriolis(DevLevel L) {
    int64_t e = gid();
    if (e >= L.E) return;
    if (!(L.eflag[e] & LIVE)) return;
    double qe = 0.5 * (L.q[L.et[e]] + L.q[L.et[L.E + e]]);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        int32_t e2 = L.cor_i[k * L.E + e];
        double w = L.cor_w[k * L.E + e];
        double q2 = 0.5 * (L.q[L.et[e2]] + L.q[L.et[L.E + e2]]);
        s += w * L.F[e2] * 0.5 * (qe + q2);
    }
    L.Q[e] = s;
}

// restriction from F = level j+1 to C = level j (Sec. 3.1): B by injection at covered
// nodes, flux by R_F on faces of covered nodes, Coriolis tendency by R_u where both
// ends are covered
__global__ void k_restrict(DevLevel C, DevLevel F) {
    int64_t i = gid();
    if (i < C.N && (C.nflag[i] & COVERED)) C.B[i] = F.B[C.c2f[i]];
    if (i >= C.E) return;
    bool ca = C.nflag[C.en[i]] & COVERED, cb = C.nflag[C.en[C.E + i]] & COVERED;
    if (ca || cb) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < 12; ++k) s += C.rf_fw[k * C.E + i] * F.F[C.rf_fi[k * C.E + i]];
#pragma unroll
        for (int k = 0; k < 11; ++k) s += C.rf_cw[k * C.E + i] * F.c[C.rf_ci[k * C.E + i]];
        C.F[i] = s / C.l_e[i];
    }
    if (ca && cb) C.Q[i] = 0.5 * (F.Q[C.half[i]] + F.Q[C.half[C.E + i]]);
}

__global__ void k_div(DevLevel L) {
    int64_t v = gid();
    if (v >= L.N) return;
    if (!(L.nflag[v] & AVAIL)) return;
    int dg = L.deg[v];
    double div = 0.0;
    for (int k = 0; k < dg; ++k) {
        int32_t code = L.ring_e[k * L.N + v];
        int64_t e = code >> 1;
        if (!(L.eflag[e] & AVAIL)) return;
        div += esign(code) * L.F[e] * L.l_e[e];
    }
    L.c[v] = div / L.A_i[v];
}

// trends at live points and one Runge-Kutta stage:
//   y <- a*y0 + b*y + (cdt*dt)*k + (ddt*dt)*acc,   acc <- al*acc + be*k
__global__ void k_update(DevLevel L, RKStage st, const double* __restrict__ dtp) {
    int64_t i = gid();
    double dt = dtp ? *dtp : 0.0;
    if (i < L.N && (L.nflag[i] & LIVE)) {
        double k = -L.c[i];
        L.dht[i] = k;
        if (st.apply) {
            // terms with a zero coefficient are skipped, so stale storage never enters
            double y = st.cdt * dt * k;
            if (st.a != 0.0) y += st.a * L.dh0[i];
            if (st.b != 0.0) y += st.b * L.dh[i];
            if (st.ddt != 0.0) y += st.ddt * dt * L.dha[i];
            if (st.al != 0.0 || st.be != 0.0) L.dha[i] = (st.al != 0.0 ? st.al * L.dha[i] : 0.0) + st.be * k;
            L.dh[i] = y;
        }
    }
    if (i < L.E && (L.eflag[i] & LIVE)) {
        double k = L.Q[i] - (L.B[L.en[L.E + i]] - L.B[L.en[i]]) / L.d_e[i];
        L.ut[i] = k;
        if (st.apply) {
            double y = st.cdt * dt * k;
            if (st.a != 0.0) y += st.a * L.u0[i];
            if (st.b != 0.0) y += st.b * L.u[i];
            if (st.ddt != 0.0) y += st.ddt * dt * L.ua[i];
            if (st.al != 0.0 || st.be != 0.0) L.ua[i] = (st.al != 0.0 ? st.al * L.ua[i] : 0.0) + st.be * k;
            L.u[i] = y;
        }
    }
}

__global__ void k_save_base(DevLevel L) {
    int64_t i = gid();
    if (i < L.N && (L.nflag[i] & LIVE)) L.dh0[i] = L.dh[i];
    if (i < L.E && (L.eflag[i] & LIVE)) L.u0[i] = L.u[i];
}

// ---------------------------------------------------------------------------- prolongation

// ghosts of level F from level C (inverse transform with zero coefficients, Eqs. 1-2)
__global__ void k_fill(DevLevel F, DevLevel C) {
    int64_t i = gid();
    if (i < F.N && (F.nflag[i] & GHOST)) {
        int32_t k = F.f2c[i];
        if (k >= 0) {
            F.dh[i] = C.dh[k];
        } else {
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                int32_t p = F.par[q * F.N + i];
                double v = (F.nflag[p] & LIVE) ? F.dh[p] : C.dh[F.f2c[p]];
                s += F.ptw[q * F.N + i] * v;
            }
            F.dh[i] = s;
        }
    }
    if (i < F.E && (F.eflag[i] & GHOST)) {
        int kind = F.fe_kind[i];
        double P = predict(F, C.u, i);
        if (kind == 2) {
            F.u[i] = P;
        } else {
            int64_t E = F.fe_ce[i];
            int32_t other = C.half[(kind == 0 ? C.E : 0) + E];
            double uc = C.u[E];
            if (F.eflag[other] & LIVE) {
                F.u[i] = 2.0 * uc - F.u[other];
            } else {
                double Po = predict(F, C.u, other);
                F.u[i] = P + 0.5 * (2.0 * uc - P - Po);
            }
        }
    }
}

// ---------------------------------------------------------------------------- partial transform

// R_h at covered nodes of C from level F (Eq. Rh; details of non-live points are zero)
__global__ void k_partial(DevLevel C, DevLevel F) {
    int64_t k = gid();
    if (k >= C.N || !(C.nflag[k] & COVERED)) return;
    double s = F.dh[C.c2f[k]];
    for (int q = 0; q < 12; ++q) {
        int32_t m = C.mk_i[q * C.N + k];
        if (m < 0 || !(F.nflag[m] & LIVE)) continue;
        s += C.mk_w[q * C.N + k] * height_detail(F, m);
    }
    C.dh[k] = s;
}

// full restriction used at initialisation: R_h at every node, mean of halves at every edge
__global__ void k_restrict_full(DevLevel C, DevLevel F) {
    int64_t i = gid();
    if (i < C.N) {
        double s = F.dh[C.c2f[i]];
        for (int q = 0; q < 12; ++q) {
            int32_t m = C.mk_i[q * C.N + i];
            if (m >= 0) s += C.mk_w[q * C.N + i] * height_detail(F, m);
        }
        C.dh[i] = s;
    }
    if (i < C.E) C.u[i] = 0.5 * (F.u[C.half[i]] + F.u[C.half[C.E + i]]);
}

// ---------------------------------------------------------------------------- adaptation (Sec. 2.3)

// wavelet coefficients at live points of level F
__global__ void k_details(DevLevel F, DevLevel C) {
    int64_t i = gid();
    if (i < F.N) F.hdet[i] = (F.f2c[i] < 0 && (F.nflag[i] & LIVE)) ? height_detail(F, i) : 0.0;
    if (i < F.E) F.ui[i] = (F.fe_kind[i] == 2 && (F.eflag[i] & LIVE)) ? F.u[i] - predict(F, C.u, i) : 0.0;
    if (i < C.E) {
        int32_t h0 = C.half[i], h1 = C.half[C.E + i];
        if ((F.eflag[h0] & LIVE) || (F.eflag[h1] & LIVE)) {
            double a = F.u[h0] - predict(F, C.u, h0);
            double b = F.u[h1] - predict(F, C.u, h1);
            F.ue[i] = 0.5 * (a - b);
        } else {
            F.ue[i] = 0.0;
        }
    }
}

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
    return v;
}

struct MaxOp {
    __device__ unsigned long long operator()(unsigned long long a, unsigned long long b) const { return a > b ? a : b; }
};
struct AddOp {
    __device__ unsigned long long operator()(unsigned long long a, unsigned long long b) const { return a + b; }
};
struct MinOp {
    __device__ unsigned long long operator()(unsigned long long a, unsigned long long b) const { return a < b ? a : b; }
};

// max |dh| over live nodes and max |u| over live edges (bit patterns of non-negative doubles)
__global__ void k_maxabs(DevLevel L, unsigned long long* red) {
    __shared__ unsigned long long sh[32];
    int64_t i = gid();
    unsigned long long a = 0, b = 0;
    if (i < L.N && (L.nflag[i] & LIVE)) a = dbits(fabs(L.dh[i]));
    if (i < L.E && (L.eflag[i] & LIVE)) b = dbits(fabs(L.u[i]));
    a = block_reduce(a, MaxOp(), sh, 0ull);
    if (threadIdx.x == 0 && a) atomicMax(&red[0], a);
    __syncthreads();
    b = block_reduce(b, MaxOp(), sh, 0ull);
    if (threadIdx.x == 0 && b) atomicMax(&red[1], b);
}

__global__ void k_thresholds(const unsigned long long* red, double eps, double eps_h, double eps_u, double* thr) {
    if (threadIdx.x || blockIdx.x) return;
    thr[0] = eps_h > 0 ? eps_h : eps * __longlong_as_double(static_cast<long long>(red[0]));
    thr[1] = eps_u > 0 ? eps_u : eps * __longlong_as_double(static_cast<long long>(red[1]));
}

// significance at level F: odd node with |h~| >= eps_h; both ends and midpoint of a
// coarse edge with |u~_E| >= eps_u; both ends of an interior edge with |u~| >= eps_u
__global__ void k_sig(DevLevel F, DevLevel C, const double* __restrict__ thr) {
    int64_t i = gid();
    double eh = thr[0], eu = thr[1];
    if (i < F.N && F.f2c[i] < 0 && (F.nflag[i] & LIVE) && fabs(F.hdet[i]) >= eh) F.sig[i] = 1;
    if (i < F.E && F.fe_kind[i] == 2 && (F.eflag[i] & LIVE) && fabs(F.ui[i]) >= eu) {
        F.sig[F.en[i]] = 1;
        F.sig[F.en[F.E + i]] = 1;
    }
    if (i < C.E) {
        int32_t h0 = C.half[i], h1 = C.half[C.E + i];
        if (((F.eflag[h0] & LIVE) || (F.eflag[h1] & LIVE)) && fabs(F.ue[i]) >= eu) {
            F.sig[C.c2f[C.en[i]]] = 1;
            F.sig[C.c2f[C.en[C.E + i]]] = 1;
            F.sig[C.mid[i]] = 1;
        }
    }
}

// T = S + same-level neighbours of S + children of the coarser significance set
__global__ void k_adjacent(DevLevel F, DevLevel C, int children) {
    int64_t x = gid();
    if (x >= F.N) return;
    int dg = F.deg[x];
    uint8_t t = F.sig[x];
    for (int k = 0; k < dg && !t; ++k) t = F.sig[ring_nbr(F, F.ring_e[k * F.N + x])];
    if (!t && children) {
        int32_t cx = F.f2c[x];
        if (cx >= 0 && C.sig[cx]) t = 1;
        for (int k = 0; k < dg && !t; ++k) {
            int32_t y = ring_nbr(F, F.ring_e[k * F.N + x]);
            int32_t cy = F.f2c[y];
            if (cy >= 0 && C.sig[cy]) t = 1;
        }
    }
    F.tmask[x] = t;
}

// graded closure at level F: coarse node of a live node of the finer level Fp, and the
// prediction parents of every live odd node (only ever sets bytes to 1)
__global__ void k_close(DevLevel F, DevLevel Fp, int has_finer) {
    int64_t x = gid();
    if (x >= F.N) return;
    uint8_t t = F.tmask[x];
    if (has_finer && Fp.tmask[F.c2f[x]]) t = 1;
    if (!t) return;
    F.tmask[x] = 1;
    if (F.f2c[x] < 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) F.tmask[F.par[q * F.N + x]] = 1;
    }
}

// live flags: all of Jmin, else the mask; an edge is live when an end node is
__global__ void k_live(DevLevel L, int all) {
    int64_t i = gid();
    if (i < L.N) {
        uint8_t lv = all ? 1 : L.tmask[i];
        L.nflag[i] = lv ? LIVE : 0;
        L.band0[i] = lv;
    }
}

__global__ void k_live_edges(DevLevel L) {
    int64_t e = gid();
    if (e >= L.E) return;
    L.eflag[e] = ((L.nflag[L.en[e]] | L.nflag[L.en[L.E + e]]) & LIVE) ? LIVE : 0;
}

__global__ void k_dilate(DevLevel L, const uint8_t* __restrict__ in, uint8_t* __restrict__ out) {
    int64_t x = gid();
    if (x >= L.N) return;
    uint8_t t = in[x];
    int dg = L.deg[x];
    for (int k = 0; k < dg && !t; ++k) t = in[ring_nbr(L, L.ring_e[k * L.N + x])];
    out[x] = t;
}

__global__ void k_ghost(DevLevel L, const uint8_t* __restrict__ band) {
    int64_t i = gid();
    if (i < L.N && !(L.nflag[i] & LIVE) && band[i]) L.nflag[i] |= GHOST;
    if (i < L.E && !(L.eflag[i] & LIVE) && band[L.en[i]] && band[L.en[L.E + i]]) L.eflag[i] |= GHOST;
}

// covered coarse nodes: the fine node at the same place and all of M_k live
__global__ void k_covered(DevLevel C, DevLevel F) {
    int64_t k = gid();
    if (k >= C.N) return;
    if (!(F.nflag[C.c2f[k]] & LIVE)) return;
    for (int q = 0; q < 12; ++q) {
        int32_t m = C.mk_i[q * C.N + k];
        if (m >= 0 && !(F.nflag[m] & LIVE)) return;
    }
    C.nflag[k] |= COVERED;
}

// patches holding any live or ghost node or edge (one block per patch)
__global__ void k_patch_flags(DevLevel L) {
    int64_t pid = blockIdx.x;
    int64_t pp = L.p * L.p;
    int any = 0;
    for (int64_t l = threadIdx.x; l < pp; l += blockDim.x) {
        int64_t e = pid * pp + l;
        if ((L.nflag[e] | L.eflag[e] | L.eflag[L.nelem + e] | L.eflag[2 * L.nelem + e]) & AVAIL) any = 1;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) L.pflag[pid] = uint8_t(any);
}

// ascending compacted list of flagged patches (one block; deterministic)
__global__ void k_patch_scan(DevLevel L) {
    __shared__ int warp_tot[32];
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t start = 0; start < L.npatch; start += blockDim.x) {
        int64_t i = start + threadIdx.x;
        int f = (i < L.npatch) ? L.pflag[i] : 0;
        unsigned bal = __ballot_sync(0xffffffffu, f);
        int pre = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) warp_tot[w] = __popc(bal);
        __syncthreads();
        int off = 0;
        for (int k = 0; k < w; ++k) off += warp_tot[k];
        if (f) L.patches[base + off + pre] = int32_t(i);
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int k = 0; k < nw; ++k) tot += warp_tot[k];
            base += tot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *L.npatches = base;
}

// inverse transform of the retained coefficients onto the live points of F:
// (a) even nodes and all edges from level C, (b) odd nodes from the even ones
__global__ void k_inverse_a(DevLevel F, DevLevel C) {
    int64_t i = gid();
    if (i < F.N && (F.nflag[i] & LIVE) && F.f2c[i] >= 0) {
        int32_t k = F.f2c[i];
        double s = C.dh[k];
        for (int q = 0; q < 12; ++q) {
            int32_t m = C.mk_i[q * C.N + k];
            if (m >= 0 && (F.nflag[m] & LIVE)) s -= C.mk_w[q * C.N + k] * F.hdet[m];
        }
        F.dh[i] = s;
    }
    if (i < F.E && (F.eflag[i] & LIVE)) {
        int kind = F.fe_kind[i];
        double P = predict(F, C.u, i);
        if (kind == 2) {
            F.u[i] = P + F.ui[i];
        } else {
            int64_t E = F.fe_ce[i];
            int32_t other = C.half[(kind == 0 ? C.E : 0) + E];
            double Po = predict(F, C.u, other);
            double delta = 0.5 * (2.0 * C.u[E] - P - Po);
            double d = F.ue[E];
            F.u[i] = P + delta + (kind == 0 ? d : -d);
        }
    }
}

__global__ void k_inverse_b(DevLevel F) {
    int64_t i = gid();
    if (i >= F.N || !(F.nflag[i] & LIVE) || F.f2c[i] >= 0) return;
    double s = F.hdet[i];
#pragma unroll
    for (int q = 0; q < 4; ++q) s += F.ptw[q * F.N + i] * F.dh[F.par[q * F.N + i]];
    F.dh[i] = s;
}

// ---------------------------------------------------------------------------- reductions (Sec. 3.1, 7.2)

// omega = sqrt(f^2 + g h (pi/dx)^2) at live nodes (max), dx/|u| at live edges (min)
__global__ void k_dt(DevLevel L, double H, double g, double dx, unsigned long long* red) {
    __shared__ unsigned long long sh[32];
    int64_t i = gid();
    unsigned long long a = 0, b = ~0ull;
    if (i < L.N && (L.nflag[i] & LIVE)) {
        double f = L.f_n[i], k = M_PI / dx;
        a = dbits(sqrt(f * f + g * (H + L.dh[i]) * k * k));
    }
    if (i < L.E && (L.eflag[i] & LIVE)) {
        double au = fabs(L.u[i]);
        if (au > 0) b = dbits(dx / au);
    }
    a = block_reduce(a, MaxOp(), sh, 0ull);
    if (threadIdx.x == 0 && a) atomicMax(&red[0], a);
    __syncthreads();
    b = block_reduce(b, MinOp(), sh, ~0ull);
    if (threadIdx.x == 0 && b != ~0ull) atomicMin(&red[1], b);
}

__global__ void k_dt_final(const unsigned long long* red, double cfl, double* dt) {
    if (threadIdx.x || blockIdx.x) return;
    double w = __longlong_as_double(static_cast<long long>(red[0]));
    double r = red[1] == ~0ull ? INFINITY : __longlong_as_double(static_cast<long long>(red[1]));
    *dt = cfl * fmin(1.0 / w, r);
}

// Neumaier-compensated partial sums of mass and energy over level Jmin
__device__ __forceinline__ void neumaier(double& s, double& c, double x) {
    double t = s + x;
    c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
    s = t;
}

__global__ void k_sums(DevLevel L, double H, double g, double* part) {
    __shared__ double sh[4][TPB];
    int64_t v = gid();
    double m = 0, en = 0;
    if (v < L.N) {
        double h = H + L.dh[v], A = L.A_i[v], ke = 0.0;
        for (int k = 0; k < L.deg[v]; ++k) {
            int64_t e = L.ring_e[k * L.N + v] >> 1;
            ke += 0.25 * L.l_e[e] * L.d_e[e] * L.u[e] * L.u[e];
        }
        m = A * h;
        en = g * h * (0.5 * g * h * A + ke);
    }
    sh[0][threadIdx.x] = m;
    sh[1][threadIdx.x] = 0;
    sh[2][threadIdx.x] = en;
    sh[3][threadIdx.x] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0, c0 = 0, s1 = 0, c1 = 0;
        for (int k = 0; k < blockDim.x; ++k) neumaier(s0, c0, sh[0][k]), neumaier(s1, c1, sh[2][k]);
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

__global__ void k_count(DevLevel L, unsigned long long* cnt) {
    __shared__ unsigned long long sh[32];
    int64_t i = gid();
    unsigned long long a = 0, b = 0, c = 0;
    if (i < L.N) a = (L.nflag[i] & LIVE) ? 1 : 0, b = (L.nflag[i] & GHOST) ? 1 : 0;
    if (i < L.E) c = (L.eflag[i] & LIVE) ? 1 : 0;
    AddOp add;
    a = block_reduce(a, add, sh, 0ull);
    if (threadIdx.x == 0) atomicAdd(&cnt[0], a);
    __syncthreads();
    b = block_reduce(b, add, sh, 0ull);
    if (threadIdx.x == 0) atomicAdd(&cnt[1], b);
    __syncthreads();
    c = block_reduce(c, add, sh, 0ull);
    if (threadIdx.x == 0) atomicAdd(&cnt[2], c);
}

int64_t span(const DevLevel& L) { return L.E > L.N ? L.E : L.N; }

}  // namespace

// ---------------------------------------------------------------------------- launchers

std::atomic<int64_t> g_launches{0};

int64_t kernel_launches() { return g_launches.load(); }
void count_launch(int64_t n) { g_launches += n; }

#define LAUNCH(kernel, n, ...) (g_launches++, kernel<<<blocks_for((n), TPB), TPB, 0, s>>>(__VA_ARGS__))

void launch_tri_q(const DevLevel& L, double H, cudaStream_t s) { LAUNCH(k_tri_q, L.T, L, H); }
void launch_edge_flux(const DevLevel& L, double H, cudaStream_t s) { LAUNCH(k_edge_flux, L.E, L, H); }
void launch_node(const DevLevel& L, double g, cudaStream_t s) { LAUNCH(k_node, L.N, L, g); }
void launch_coriolis(const DevLevel& L, cudaStream_t s) { LAUNCH(k_coriolis, L.E, L); }

void launch_restrict(const DevLevel& C, const DevLevel& F, cudaStream_t s) {
    LAUNCH(k_restrict, span(C), C, F);
    LAUNCH(k_div, C.N, C);
}

void launch_update(const DevLevel& L, const RKStage& st, const double* dt, cudaStream_t s) {
    LAUNCH(k_update, span(L), L, st, dt);
}

void launch_save_base(const DevLevel& L, cudaStream_t s) { LAUNCH(k_save_base, span(L), L); }

void launch_fill(const DevLevel& F, const DevLevel& C, cudaStream_t s) { LAUNCH(k_fill, span(F), F, C); }

void launch_partial(const DevLevel& C, const DevLevel& F, cudaStream_t s) { LAUNCH(k_partial, C.N, C, F); }

void launch_restrict_full(const DevLevel& C, const DevLevel& F, cudaStream_t s) {
    LAUNCH(k_restrict_full, span(C), C, F);
}

void launch_details(const DevLevel& F, const DevLevel& C, cudaStream_t s) {
    int64_t n = span(F) > C.E ? span(F) : C.E;
    LAUNCH(k_details, n, F, C);
}

void launch_maxabs(const DevLevel& L, unsigned long long* red, cudaStream_t s) { LAUNCH(k_maxabs, span(L), L, red); }

void launch_thresholds(const unsigned long long* red, double eps, double eh, double eu, double* thr, cudaStream_t s) {
    g_launches++;
    k_thresholds<<<1, 32, 0, s>>>(red, eps, eh, eu, thr);
}

void launch_sig(const DevLevel& F, const DevLevel& C, const double* thr, cudaStream_t s) {
    int64_t n = span(F) > C.E ? span(F) : C.E;
    LAUNCH(k_sig, n, F, C, thr);
}

void launch_adjacent(const DevLevel& F, const DevLevel& C, int children, cudaStream_t s) {
    LAUNCH(k_adjacent, F.N, F, C, children);
}

void launch_close(const DevLevel& F, const DevLevel& Fp, int has_finer, cudaStream_t s) {
    LAUNCH(k_close, F.N, F, Fp, has_finer);
}

void launch_live(const DevLevel& L, int all, cudaStream_t s) {
    LAUNCH(k_live, L.N, L, all);
    LAUNCH(k_live_edges, L.E, L);
}

void launch_ghost_band(const DevLevel& L, int hops, cudaStream_t s) {
    uint8_t* a = L.band0;
    uint8_t* b = L.band1;
    for (int h = 0; h < hops; ++h) {
        LAUNCH(k_dilate, L.N, L, a, b);
        uint8_t* t = a;
        a = b;
        b = t;
    }
    LAUNCH(k_ghost, span(L), L, a);
}

void launch_covered(const DevLevel& C, const DevLevel& F, cudaStream_t s) { LAUNCH(k_covered, C.N, C, F); }

void launch_patches(const DevLevel& L, cudaStream_t s) {
    int t = int(L.p * L.p < 256 ? L.p * L.p : 256);
    t = t < 32 ? 32 : t;
    g_launches += 2;
    k_patch_flags<<<unsigned(L.npatch), t, 0, s>>>(L);
    k_patch_scan<<<1, 1024, 0, s>>>(L);
}

void launch_inverse(const DevLevel& F, const DevLevel& C, cudaStream_t s) {
    LAUNCH(k_inverse_a, span(F), F, C);
    LAUNCH(k_inverse_b, F.N, F);
}

void launch_dt(const DevLevel& L, double H, double g, double dx, unsigned long long* red, cudaStream_t s) {
    LAUNCH(k_dt, span(L), L, H, g, dx, red);
}

void launch_dt_final(const unsigned long long* red, double cfl, double* dt, cudaStream_t s) {
    g_launches++;
    k_dt_final<<<1, 32, 0, s>>>(red, cfl, dt);
}

int sums_blocks(const DevLevel& L) { return int(blocks_for(L.N, TPB)); }

void launch_sums(const DevLevel& L, double H, double g, double* part, double* out, cudaStream_t s) {
    int nb = sums_blocks(L);
    g_launches += 2;
    k_sums<<<nb, TPB, 0, s>>>(L, H, g, part);
    k_sums_final<<<1, 32, 0, s>>>(part, nb, out);
}

void launch_count(const DevLevel& L, unsigned long long* cnt, cudaStream_t s) { LAUNCH(k_count, span(L), L, cnt); }

}  // namespace sww
