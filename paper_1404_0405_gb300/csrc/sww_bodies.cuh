// Device-side helpers shared by the kernel translation units: the work-list item
// loop and the per-item bodies of the trend, the RK stage and the prolongation.
// Included inside an anonymous namespace of each translation unit.
#pragma once

#include "f64conv.cuh"

__device__ __forceinline__ int64_t gid() { return int64_t(blockIdx.x) * blockDim.x + threadIdx.x; }
template <class R>
__device__ __forceinline__ R esign(int32_t code) { return (code & 1) ? R(-1) : R(1); }
// an FP64 geometry value entering arithmetic of the working precision (FP32: the
// integer-pipe rounding of f64conv.cuh)
template <class R>
__device__ __forceinline__ R to_r(double x);
template <>
__device__ __forceinline__ double to_r<double>(double x) { return x; }
template <>
__device__ __forceinline__ float to_r<float>(double x) { return f64_to_f32_rn(x); }
template <class R>
__device__ __forceinline__ R geo(const double* __restrict__ p, int64_t i) { return to_r<R>(p[i]); }


template <class R>
__device__ __forceinline__ R predict(const DevLevelT<R>& F, const R* __restrict__ uc, int64_t fe) {
    R s = R(0);
#pragma unroll
    for (int k = 0; k < 12; ++k) s += F.vw[k * F.E + fe] * uc[F.vst[k * F.E + fe]];
    return s;
}

template <class R>
__device__ __forceinline__ R height_detail(const DevLevelT<R>& F, int64_t x) {
    R s = F.dh[x];
#pragma unroll
    for (int k = 0; k < 4; ++k) s -= F.ptw[k * F.N + x] * F.dh[F.par[k * F.N + x]];
    return s;
}

__device__ __forceinline__ unsigned long long dbits(double x) {
    return static_cast<unsigned long long>(__double_as_longlong(x));
}

// the viscous form (nu != 0), tested on the bits of nu (either sign of zero is
// zero) on the integer pipe: the per-point bodies ask at every point
template <class Lv>
__device__ __forceinline__ bool viscous(const Lv& L) {
    return (dbits(L.nu) << 1) != 0;
}

// ---------------------------------------------------------------------------- CFL step and field maxima

// |x| as an unsigned key ordered like |x|: with the sign bit cleared, IEEE numbers
// order like their bit patterns, and NaN keys lie above the key of +infinity
__device__ __forceinline__ unsigned long long abs_key(float x) { return __float_as_uint(x) & 0x7fffffffu; }
__device__ __forceinline__ unsigned long long abs_key(double x) { return dbits(x) & 0x7fffffffffffffffull; }
template <class R>
__device__ __forceinline__ unsigned long long inf_key() {
    return sizeof(R) == 4 ? 0x7f800000ull : 0x7ff0000000000000ull;
}
// the magnitude a key stands for, as a double (exact: widening keeps the value)
template <class R>
__device__ __forceinline__ double key_value(unsigned long long k) {
    return sizeof(R) == 4 ? double(__uint_as_float(unsigned(k))) : __longlong_as_double(static_cast<long long>(k));
}

// squared CFL frequency f^2 + g h (pi/dx)^2 at node id, in FP64 with the products
// and sums rounded in the written order (no contraction).  The time step takes the
// square root of the maximum only: a correctly rounded square root is monotone, so
// that equals the maximum of the roots.
template <class R>
__device__ __forceinline__ double omega2_at(const DevLevelT<R>& L, int64_t id, double H, double g) {
    const double f = L.f_n[id];
    return __dadd_rn(__dmul_rn(f, f), __dmul_rn(__dmul_rn(g, __dadd_rn(H, double(L.dh[id]))), L.kx2));
}

// Running maximum of a key per level over one thread's items, flushed into the
// block's per-level words (shared memory) when the level changes: a thread meets
// its items in list order, which is level order, so it flushes a few times.
struct LevelMax {
    int j = -1;
    unsigned long long k = 0;
    __device__ __forceinline__ void flush(unsigned long long* sm) {
        if (k) atomicMax(sm + j, k);
    }
    __device__ __forceinline__ void add(int jj, unsigned long long key, unsigned long long* sm) {
        if (jj != j) {
            flush(sm);
            j = jj;
            k = 0;
        }
        k = key > k ? key : k;
    }
};

// Advective bound min over live edges of dx_j / |u| (Sec. 3.1's CFL condition):
// for one level, a correctly rounded dx_j / a falls as a grows, so the minimum is
// dx_j over the level's largest |u|; then the step cfl * min(1/omega, that bound).
template <class R>
__device__ __forceinline__ double cfl_step(const DevLevelT<R>* lvs, const unsigned long long* red, double cfl) {
    const double w = sqrt(__longlong_as_double(static_cast<long long>(red[0])));
    double r = INFINITY;
    for (int j = 0; j < RED_WORDS - RED_LEVEL; ++j) {
        const unsigned long long k = red[RED_LEVEL + j];
        if (k) r = fmin(r, lvs[j].dx / key_value<R>(k));
    }
    return cfl * fmin(1.0 / w, r);
}

// Item kinds of a work-list entry, in slot order.
constexpr int K_NODE = 1, K_EDGE = 2, K_TRI = 4, K_CEDGE = 8;

template <int KINDS>
__host__ __device__ constexpr int slots_of() {
    return ((KINDS & K_NODE) ? 1 : 0) + ((KINDS & K_EDGE) ? 3 : 0) + ((KINDS & K_TRI) ? 2 : 0) + ((KINDS & K_CEDGE) ? 3 : 0);
}

// Visit the items of the entries of a work list, one thread per item:
// body(L, kind, id, elem).  An entry covers slots x P threads (P = configured patch
// area): one slot of nodes, three of edges (orientation 0, 1, 2), two of triangles
// and three of the edges of the coarse element under an even element (id = the
// orientation), as KINDS selects.  A pole entry yields the two pole nodes with
// elem = -1.  Entries name their level in `lvs` (multi-level lists) or all belong
// to `one` when lvs is null.
// Item `local` (0 <= local < slots x P) of work-list entry patch `pat` of level L:
// body(L, kind, id, elem) when the slot holds an item (see for_items).
// P is a power of two (the patch side is), so slot and index are a shift and a mask.
template <int KINDS, class Lv, class Body>
__device__ __forceinline__ void visit_item(const Lv& L, int64_t pat, uint32_t local, int P, Body& body) {
    int slot = int(local >> (__ffs(P) - 1));
    const int64_t idx = int64_t(local & uint32_t(P - 1));
    if (pat == L.npatch) {
        if ((KINDS & K_NODE) && slot == 0 && idx < 2) body(L, K_NODE, L.nelem + idx, int64_t(-1));
        return;
    }
    const int64_t pp = L.p * L.p;
    if (idx >= pp) return;
    const int64_t el = pat * pp + idx;
    if (KINDS & K_NODE) {
        if (slot == 0) {
            body(L, K_NODE, el, el);
            return;
        }
        slot -= 1;
    }
    if (KINDS & K_EDGE) {
        if (slot < 3) {
            body(L, K_EDGE, slot * L.nelem + el, el);
            return;
        }
        slot -= 3;
    }
    if (KINDS & K_TRI) {
        if (slot < 2) {
            body(L, K_TRI, slot * L.nelem + el, el);
            return;
        }
        slot -= 2;
    }
    if (KINDS & K_CEDGE) body(L, K_CEDGE, int64_t(slot), el);
}

template <int KINDS, class Lv, class Body>
__device__ __forceinline__ void for_items(const Lv* __restrict__ lvs, const Lv& one,
                                          const int32_t* __restrict__ list, const int32_t* __restrict__ count, int P,
                                          Body body) {
    // 32-bit item numbers: a list holds fewer than 2^31 items up to level 11
    constexpr uint32_t NS = slots_of<KINDS>();
    const int lp = __ffs(P) - 1;
    const uint32_t n = uint32_t(*count) * (NS << lp);
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t it = blockIdx.x * blockDim.x + threadIdx.x; it < n; it += stride) {
        const uint32_t e = (it >> lp) / NS;
        const int32_t ent = list[e];
        const Lv& L = lvs ? lvs[ent >> LVL_SHIFT] : one;
        visit_item<KINDS>(L, int64_t(ent & PATCH_MASK), it - ((e * NS) << lp), P, body);
    }
}

// ---------------------------------------------------------------------------- trend bodies (Sec. 3.1)

// potential vorticity q = (curl u + f)/h at a triangle (dual cell)
template <class R>
__device__ __forceinline__ void pv_at(const DevLevelT<R>& L, int64_t t, R H) {
    if (L.advect) return;   // no velocity trend, no q
    int32_t n0 = L.tn[t], n1 = L.tn[L.T + t], n2 = L.tn[2 * L.T + t];
    int32_t c0 = L.te[t], c1 = L.te[L.T + t], c2 = L.te[2 * L.T + t];
    if (!(L.nflag[n0] & AVAIL) || !(L.nflag[n1] & AVAIL) || !(L.nflag[n2] & AVAIL)) return;
    if (!(L.eflag[c0 >> 1] & AVAIL) || !(L.eflag[c1 >> 1] & AVAIL) || !(L.eflag[c2 >> 1] & AVAIL)) return;
    R circ = esign<R>(c0) * L.u[c0 >> 1] * geo<R>(L.d_e, c0 >> 1) + esign<R>(c1) * L.u[c1 >> 1] * geo<R>(L.d_e, c1 >> 1) +
             esign<R>(c2) * L.u[c2 >> 1] * geo<R>(L.d_e, c2 >> 1);
    R hv = geo<R>(L.kite, t) * (H + L.dh[n0]) + geo<R>(L.kite, L.T + t) * (H + L.dh[n1]) +
           geo<R>(L.kite, 2 * L.T + t) * (H + L.dh[n2]);
    R Av = geo<R>(L.A_v, t);
    if (viscous(L)) L.zeta[t] = circ / Av;
    L.q[t] = (circ / Av + geo<R>(L.f_v, t)) / (hv / Av);
}

// thickness flux F = h_e u at an edge
template <class R>
__device__ __forceinline__ void flux_at(const DevLevelT<R>& L, int64_t e, R H) {
    if (!(L.eflag[e] & AVAIL)) return;
    int32_t a = L.en[e], b = L.en[L.E + e];
    if (!(L.nflag[a] & AVAIL) || !(L.nflag[b] & AVAIL)) return;
    L.F[e] = R(0.5) * ((H + L.dh[a]) + (H + L.dh[b])) * L.u[e];
    // viscous form: diffusive height flux -nu grad(dh) (joins F in the divergence)
    if (viscous(L)) L.Fd[e] = -R(L.nu) * (L.dh[b] - L.dh[a]) / geo<R>(L.d_e, e);
}

// divergence of the height flux (with the diffusive flux of the viscous form) at a node
template <class R>
__device__ __forceinline__ void div_at(const DevLevelT<R>& L, int64_t v) {
    if (!(L.nflag[v] & AVAIL)) return;
    const int dg = L.deg[v];
    R div = R(0);
    bool ok = true;   // every ring edge available (else nothing is written)
    const bool visc = viscous(L);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        if (k >= dg) break;
        const int32_t code = L.ring_e[k * L.N + v];
        const int64_t e = code >> 1;
        ok = ok && (L.eflag[e] & AVAIL);
        div += esign<R>(code) * (visc ? L.F[e] + L.Fd[e] : L.F[e]) * geo<R>(L.l_e, e);
    }
    if (!ok) return;
    L.c[v] = div / geo<R>(L.A_i, v);
}

// a node whose divergence the restricted fluxes change: available, with a covered
// node among itself and its neighbours (an edge is restricted when an end is
// covered).  The work list WL_DN holds exactly these nodes.
template <class R>
__device__ __forceinline__ bool restricted_div_node(const DevLevelT<R>& L, int64_t v) {
    const uint8_t f = L.nflag[v];
    if (!(f & AVAIL)) return false;
    if (f & COVERED) return true;
    // the neighbours' flags, their loads issued together (no early exit)
    const int dg = L.deg[v];
    uint8_t acc = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k)
        if (k < dg) acc |= L.nflag[L.ring_n[k * L.N + v]];
    return (acc & COVERED) != 0;
}

// divergence, kinetic energy and Bernoulli function at a node
template <class R>
__device__ __forceinline__ void node_at(const DevLevelT<R>& L, int64_t v, R g) {
    if (L.advect) return div_at(L, v);   // prescribed velocity: no Bernoulli function
    if (!(L.nflag[v] & AVAIL)) return;
    const int dg = L.deg[v];
    R div = R(0), ke = R(0), du = R(0);
    bool ok = true;   // every ring edge available (else nothing is written)
    const bool visc = viscous(L);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        if (k >= dg) break;
        const int32_t code = L.ring_e[k * L.N + v];
        const int64_t e = code >> 1;
        ok = ok && (L.eflag[e] & AVAIL);
        R ue = L.u[e];
        const R le = geo<R>(L.l_e, e);
        div += esign<R>(code) * (visc ? L.F[e] + L.Fd[e] : L.F[e]) * le;
        if (visc) du += esign<R>(code) * ue * le;
        ke += R(0.25) * le * geo<R>(L.d_e, e) * ue * ue;
    }
    if (!ok) return;
    R A = geo<R>(L.A_i, v);
    // viscous form: -nu div u joins B (so that -grad B gains +nu grad div u)
    if (visc) ke -= R(L.nu) * du;
    L.c[v] = div / A;
    L.B[v] = g * L.dh[v] + ke / A;
}

// energy-conserving Coriolis tendency +q F.n_left at a live edge (TRiSK)
template <class R>
__device__ __forceinline__ void coriolis_at(const DevLevelT<R>& L, int64_t e) {
    if (L.advect || !(L.eflag[e] & LIVE)) return;
    R qe = R(0.5) * (L.q[L.et[e]] + L.q[L.et[L.E + e]]);
    R s = R(0);
#pragma unroll
    for (int k = 0; k < 10; ++k) {
        int32_t e2 = L.cor_i[k * L.E + e];
        R w = geo<R>(L.cor_w, k * L.E + e);
        R q2 = R(0.5) * (L.q[L.et[e2]] + L.q[L.et[L.E + e2]]);
        s += w * L.F[e2] * R(0.5) * (qe + q2);
    }
    // viscous form: -nu grad^perp curl u, grad^perp zeta = (1/l_e) sum_{v at e} t_{e,v} zeta_v
    if (viscous(L)) {
        R gp = R(0);
        for (int side = 0; side < 2; ++side) {
            const int32_t t = L.et[side * L.E + e];
            for (int k = 0; k < 3; ++k) {
                const int32_t code = L.te[k * L.T + t];
                if ((code >> 1) == e) gp += esign<R>(code) * L.zeta[t];
            }
        }
        s -= R(L.nu) * gp / geo<R>(L.l_e, e);
    }
    L.Q[e] = s;
}

// trend and one Runge-Kutta stage at a live point (terms with a zero coefficient
// are skipped, so stale storage never enters):
//   y <- a*y0 + b*y + (cdt*dt)*k + (ddt*dt)*acc,   acc <- al*acc + be*k
// An RK stage in the working precision: the coefficients converted and their zero
// tests taken once per thread, not at every point (the FP64 pipe is narrow)
template <class R>
struct RKStageR {
    R a, b, cdt, ddt, al, be;
    bool apply, ha, hb, hddt, hacc, hal;
    __device__ explicit RKStageR(const RKStage& st)
        : a(R(st.a)), b(R(st.b)), cdt(R(st.cdt)), ddt(R(st.ddt)), al(R(st.al)), be(R(st.be)), apply(st.apply != 0),
          ha(st.a != 0.0), hb(st.b != 0.0), hddt(st.ddt != 0.0), hacc(st.al != 0.0 || st.be != 0.0), hal(st.al != 0.0) {}
};

template <class R>
__device__ __forceinline__ void rk_apply(const RKStageR<R>& st, R dt, R k, R* y, const R* y0, R* acc) {
    R v = st.cdt * dt * k;
    if (st.ha) v += st.a * *y0;
    if (st.hb) v += st.b * *y;
    if (st.hddt) v += st.ddt * dt * *acc;
    if (st.hacc) *acc = (st.hal ? st.al * *acc : R(0)) + st.be * k;
    *y = v;
}

template <class R>
__device__ __forceinline__ void update_node(const DevLevelT<R>& L, int64_t v, const RKStageR<R>& st, R dt) {
    if (!(L.nflag[v] & LIVE)) return;
    R k = -L.c[v];
    L.dht[v] = k;
    if (st.apply) rk_apply(st, dt, k, &L.dh[v], &L.dh0[v], &L.dha[v]);
}

template <class R>
__device__ __forceinline__ void update_edge(const DevLevelT<R>& L, int64_t e, const RKStageR<R>& st, R dt) {
    if (!(L.eflag[e] & LIVE)) return;
    if (L.advect) {   // prescribed velocity: zero trend, u untouched
        L.ut[e] = R(0);
        return;
    }
    R k = L.Q[e] - (L.B[L.en[L.E + e]] - L.B[L.en[e]]) / geo<R>(L.d_e, e);
    L.ut[e] = k;
    if (st.apply) rk_apply(st, dt, k, &L.u[e], &L.u0[e], &L.ua[e]);
}

// ---------------------------------------------------------------------------- prolongation (Eqs. 1-2)

// ghost node of level F from level C (inverse transform with zero coefficients)
template <class R>
__device__ __forceinline__ void fill_node(const DevLevelT<R>& F, const DevLevelT<R>& C, int64_t i) {
    if (!(F.nflag[i] & GHOST)) return;
    int32_t k = F.f2c[i];
    if (k >= 0) {
        F.dh[i] = C.dh[k];
        return;
    }
    R s = R(0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int32_t p = F.par[q * F.N + i];
        R v = (F.nflag[p] & LIVE) ? F.dh[p] : C.dh[F.f2c[p]];
        s += F.ptw[q * F.N + i] * v;
    }
    F.dh[i] = s;
}

template <class R>
__device__ __forceinline__ void fill_edge(const DevLevelT<R>& F, const DevLevelT<R>& C, int64_t i) {
    if (F.advect || !(F.eflag[i] & GHOST)) return;   // prescribed velocity is kept everywhere
    int kind = F.fe_kind[i];
    R P = predict(F, C.u, i);
    if (kind == 2) {
        F.u[i] = P;
        return;
    }
    int64_t E = F.fe_ce[i];
    int32_t other = C.half[(kind == 0 ? C.E : 0) + E];
    R uc = C.u[E];
    if (F.eflag[other] & LIVE) {
        F.u[i] = R(2) * uc - F.u[other];
    } else {
        R Po = predict(F, C.u, other);
        F.u[i] = P + R(0.5) * (R(2) * uc - P - Po);
    }
}


// ---------------------------------------------------------------------------- transforms (Eqs. 1-2)

// wavelet coefficients at a live point of F > Jmin from C = the level below
// (Eqs. 1-2; velocity transform of Sec. 4.1): h~ at odd nodes, u~ at interior fine
// edges, u~_E at the edges of the coarse element under each even fine element
template <class R>
__device__ __forceinline__ void details_item(const DevLevelT<R>& L, const DevLevelT<R>& C, int kind, int64_t id,
                                             int64_t el) {
    if (kind == K_NODE) {
        if (L.f2c[id] < 0 && (L.nflag[id] & LIVE)) L.hdet[id] = height_detail(L, id);
    } else if (kind == K_EDGE) {
        if (L.fe_kind[id] == 2 && (L.eflag[id] & LIVE)) L.ui[id] = L.u[id] - predict(L, C.u, id);
    } else {
        int32_t ce = L.f2c[el];
        if (ce < 0) return;
        int64_t E = id * C.nelem + ce;
        int32_t h0 = C.half[E], h1 = C.half[C.E + E];
        if ((L.eflag[h0] & LIVE) || (L.eflag[h1] & LIVE)) {
            R a = L.u[h0] - predict(L, C.u, h0);
            R b = L.u[h1] - predict(L, C.u, h1);
            L.ue[E] = R(0.5) * (a - b);
        }
    }
}

// inverse transform of the retained coefficients at a live point of F from C:
// (a) even nodes and edges; coefficients count only where the point was live
// before the adaptation (WASLIVE)
template <class R>
__device__ __forceinline__ void inverse_a_item(const DevLevelT<R>& L, const DevLevelT<R>& C, int kind, int64_t id) {
    if (kind == K_NODE) {
        if (!(L.nflag[id] & LIVE) || L.f2c[id] < 0) return;
        int32_t k = L.f2c[id];
        R s = C.dh[k];
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            int32_t m = C.mk_i[q * C.N + k];
            if (m >= 0 && (L.nflag[m] & LIVE) && (L.nflag[m] & WASLIVE)) s -= C.mk_w[q * C.N + k] * L.hdet[m];
        }
        L.dh[id] = s;
        return;
    }
    int64_t i = id;
    if (L.advect || !(L.eflag[i] & LIVE)) return;   // a prescribed velocity is kept as set
    int fk = L.fe_kind[i];
    R Pr = predict(L, C.u, i);
    if (fk == 2) {
        L.u[i] = Pr + ((L.eflag[i] & WASLIVE) ? L.ui[i] : R(0));
    } else {
        int64_t E = L.fe_ce[i];
        int32_t h0 = C.half[E], h1 = C.half[C.E + E];
        int32_t other = fk == 0 ? h1 : h0;
        R Po = predict(L, C.u, other);
        R delta = R(0.5) * (R(2) * C.u[E] - Pr - Po);
        R d = ((L.eflag[h0] | L.eflag[h1]) & WASLIVE) ? L.ue[E] : R(0);
        L.u[i] = Pr + delta + (fk == 0 ? d : -d);
    }
}

// (b) odd nodes from the even ones
template <class R>
__device__ __forceinline__ void inverse_b_item(const DevLevelT<R>& L, int64_t id) {
    if (!(L.nflag[id] & LIVE) || L.f2c[id] >= 0) return;
    R s = (L.nflag[id] & WASLIVE) ? L.hdet[id] : R(0);
#pragma unroll
    for (int q = 0; q < 4; ++q) s += L.ptw[q * L.N + id] * L.dh[L.par[q * L.N + id]];
    L.dh[id] = s;
}

#define ITEMS(KINDS, lvs, one, list, count, P) \
    for_items<KINDS>(lvs, one, list, count, P, [&](const auto& L, int kind, int64_t id, int64_t el)

// restriction from F = level j+1 to C = level j at one item of C (Sec. 3.1): B by
// injection at covered nodes, flux by R_F on faces of covered nodes, Coriolis
// tendency by R_u where both ends are covered
template <class R>
__device__ __forceinline__ void restrict_item(const DevLevelT<R>& L, const DevLevelT<R>& F, int kind, int64_t id) {
    if (kind == K_NODE) {
        if (!L.advect && (L.nflag[id] & COVERED)) L.B[id] = F.B[L.c2f[id]];
        return;
    }
    int64_t i = id;
    bool ca = L.nflag[L.en[i]] & COVERED, cb = L.nflag[L.en[L.E + i]] & COVERED;
    if (ca || cb) {
        // the restricted total height flux (mass flux plus the viscous form's
        // diffusive flux) goes to F; the coarse diffusive flux is then zero
        const bool visc = viscous(L);
        R s = R(0);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const int32_t f = L.rf_fi[k * L.E + i];
            s += L.rf_fw[k * L.E + i] * (visc ? F.F[f] + F.Fd[f] : F.F[f]);
        }
#pragma unroll
        for (int k = 0; k < 11; ++k) s += L.rf_cw[k * L.E + i] * F.c[L.rf_ci[k * L.E + i]];
        L.F[i] = s / geo<R>(L.l_e, i);
        if (visc) L.Fd[i] = R(0);
    }
    if (ca && cb && !L.advect) L.Q[i] = R(0.5) * (F.Q[L.half[i]] + F.Q[L.half[L.E + i]]);
}

// ---------------------------------------------------------------------------- mask items (Sec. 2.3)

// significance at level F (Sec. 2.3): odd node with |h~| >= eps_h; both ends of an
// interior edge with |u~| >= eps_u; both ends and the midpoint of a coarse edge with
// |u~_E| >= eps_u; only points live before the adaptation carry coefficients
// The significance threshold e (FP64) as a threshold of the field type: the least
// R value >= e, so that |x| >= e and |x| >= sig_thr<R>(e) agree for every x of type
// R (infinity and NaN included); the tests below then compare in R.
template <class R>
__device__ __forceinline__ R sig_thr(double e);
template <>
__device__ __forceinline__ double sig_thr<double>(double e) { return e; }
template <>
__device__ __forceinline__ float sig_thr<float>(double e) { return __double2float_ru(e); }

template <class R>
__device__ __forceinline__ bool sig_node(const DevLevelT<R>& F, int64_t i, R eh) {
    if (F.f2c[i] < 0 && (F.nflag[i] & LIVE) && fabs(F.hdet[i]) >= eh) {
        F.sig[i] = 1;
        return true;
    }
    return false;
}

template <class R>
__device__ __forceinline__ bool sig_edge(const DevLevelT<R>& F, int64_t i, R eu) {
    if (F.fe_kind[i] == 2 && (F.eflag[i] & LIVE) && fabs(F.ui[i]) >= eu) {
        F.sig[F.en[i]] = 1;
        F.sig[F.en[F.E + i]] = 1;
        return true;
    }
    return false;
}

template <class R>
__device__ __forceinline__ bool sig_cedge(const DevLevelT<R>& F, const DevLevelT<R>& C, int64_t i, R eu) {
    const int32_t h0 = C.half[i], h1 = C.half[C.E + i];
    if (((F.eflag[h0] & LIVE) || (F.eflag[h1] & LIVE)) && fabs(F.ue[i]) >= eu) {
        F.sig[C.c2f[C.en[i]]] = 1;
        F.sig[C.c2f[C.en[C.E + i]]] = 1;
        F.sig[C.mid[i]] = 1;
        return true;
    }
    return false;
}

// T = S + same-level neighbours of S + children of the coarser significance set; a
// patch the learned proposal names joins T as a whole (the exact rules' own set is
// recorded per patch for the proposal's statistics)
template <class R>
__device__ __forceinline__ void adjacent_node(const DevLevelT<R>& F, const DevLevelT<R>& C, bool children, int64_t x) {
    // significance bytes are 0 or 1; each group of loads is issued together
    uint8_t t = F.sig[x];
    if (!t) {
        const int dg = F.deg[x];
        int32_t y[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) y[k] = k < dg ? F.ring_n[k * F.N + x] : int32_t(x);
#pragma unroll
        for (int k = 0; k < 6; ++k) t |= F.sig[y[k]];
        if (!t && children) {
            int32_t cy[7];
            cy[6] = F.f2c[x];
#pragma unroll
            for (int k = 0; k < 6; ++k) cy[k] = F.f2c[y[k]];
#pragma unroll
            for (int k = 0; k < 7; ++k)
                if (cy[k] >= 0) t |= C.sig[cy[k]];
        }
    }
    const int64_t P = x < F.nelem ? x / (F.p * F.p) : F.npatch;
    if (t)
        F.pexact[P] = 1;
    else if (F.prop[P])
        t = 1;
    F.tmask[x] = t;
}

// graded closure at level F: coarse node of a live node of the finer level Fp, and
// the prediction parents of every live odd node (only ever sets bytes to 1)
template <class R>
__device__ __forceinline__ void close_node(const DevLevelT<R>& F, const DevLevelT<R>& Fp, bool has_finer, int64_t x) {
    uint8_t t = F.tmask[x];
    if (has_finer && Fp.tmask[F.c2f[x]]) t = 1;
    if (!t) return;
    F.tmask[x] = 1;
    if (F.f2c[x] < 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) F.tmask[F.par[q * F.N + x]] = 1;
    }
}

// live flag (every node when `all`, else the mask), remembering whether it was live
template <class R>
__device__ __forceinline__ uint8_t live_node(const DevLevelT<R>& L, int64_t i, bool all) {
    const uint8_t lv = all ? 1 : L.tmask[i];
    L.nflag[i] = uint8_t((lv ? LIVE : 0) | ((L.nflag[i] & LIVE) ? WASLIVE : 0));
    L.band0[i] = lv;
    return lv;
}

// an edge is live when an end node is
template <class R>
__device__ __forceinline__ void live_edge(const DevLevelT<R>& L, int64_t e) {
    const uint8_t was = (L.eflag[e] & LIVE) ? WASLIVE : 0;
    L.eflag[e] = uint8_t((((L.nflag[L.en[e]] | L.nflag[L.en[L.E + e]]) & LIVE) ? LIVE : 0) | was);
}

// one neighbour hop of the ghost band: band1 <- dilate(band0) when `forward`,
// band0 <- dilate(band1) otherwise
template <class R>
__device__ __forceinline__ void dilate_node(const DevLevelT<R>& L, int64_t x, bool forward) {
    const uint8_t* __restrict__ in = forward ? L.band0 : L.band1;
    uint8_t* __restrict__ out = forward ? L.band1 : L.band0;
    // band bytes are 0 or 1; the neighbours' loads are issued together
    uint8_t t = in[x];
    if (!t) {
        const int dg = L.deg[x];
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (k < dg) t |= in[L.ring_n[k * L.N + x]];
    }
    out[x] = t;
}

template <class R>
__device__ __forceinline__ void ghost_node(const DevLevelT<R>& L, int64_t i, const uint8_t* band) {
    if (!(L.nflag[i] & LIVE) && band[i]) L.nflag[i] |= GHOST;
}

template <class R>
__device__ __forceinline__ void ghost_edge(const DevLevelT<R>& L, int64_t e, const uint8_t* band) {
    if (!(L.eflag[e] & LIVE) && band[L.en[e]] && band[L.en[L.E + e]]) L.eflag[e] |= GHOST;
}

// covered coarse node: the fine node at the same place and all of M_k live
template <class R>
__device__ __forceinline__ void covered_node(const DevLevelT<R>& C, const DevLevelT<R>& F, int64_t k) {
    if (!(F.nflag[C.c2f[k]] & LIVE)) return;
    bool all = true;   // the loads issued together (no early exit)
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        const int32_t m = C.mk_i[q * C.N + k];
        if (m >= 0 && !(F.nflag[m] & LIVE)) all = false;
    }
    if (all) C.nflag[k] |= COVERED;
}

// ---------------------------------------------------------------------------- patch lists (Sec. 5.2)

// The indices of the nonzero bytes of flag[0..n) into out (tag | index), in
// ascending order, by one block: each thread takes 32 consecutive flags per pass
// (two 16-byte loads), the block forms an exclusive prefix of the counts, and each
// thread writes its entries.  flag must be 16-byte aligned.  Returns the count (in
// every thread).
__device__ int compact_flags(const uint8_t* __restrict__ flag, int64_t n, int32_t tag, int32_t* __restrict__ out) {
    __shared__ int wsum[32];
    __shared__ int total;
    if (threadIdx.x == 0) total = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int64_t start = 0; start < n; start += 32 * int64_t(blockDim.x)) {
        const int64_t i0 = start + 32 * int64_t(threadIdx.x);
        unsigned bits = 0u;
        if (i0 + 32 <= n) {
            const uint4 a = *reinterpret_cast<const uint4*>(flag + i0);
            const uint4 b = *reinterpret_cast<const uint4*>(flag + i0 + 16);
            const unsigned words[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
            for (int q = 0; q < 8; ++q)
#pragma unroll
                for (int k = 0; k < 4; ++k) bits |= (((words[q] >> (8 * k)) & 0xffu) ? 1u : 0u) << (4 * q + k);
        } else {
            for (int k = 0; k < 32 && i0 + k < n; ++k) bits |= (flag[i0 + k] ? 1u : 0u) << k;
        }
        const int cnt = __popc(bits);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        if (w == 0) {
            int v = lane < nw ? wsum[lane] : 0, iv = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, iv, o);
                if (lane >= o) iv += t;
            }
            if (lane < nw) wsum[lane] = iv - v;   // exclusive prefix over warps
        }
        __syncthreads();
        int pos = total + wsum[w] + incl - cnt;
        while (bits) {
            const int k = __ffs(bits) - 1;
            out[pos++] = tag | int32_t(i0 + k);
            bits &= bits - 1u;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) total += wsum[w] + incl;
        __syncthreads();
    }
    return total;
}

// The ascending list of level L's flagged patches (+ the pole entry when a pole is
// live or ghost), one block of any width (ballot and a warp-total prefix).
template <class R>
__device__ void patch_scan_level(const DevLevelT<R>& L) {
    const int32_t tag = int32_t(L.J) << LVL_SHIFT;
    const int n = compact_flags(L.pflag, L.npatch, tag, L.patches);
    if (threadIdx.x == 0) {
        int m = n;
        if ((L.nflag[L.nelem] | L.nflag[L.nelem + 1]) & AVAIL) L.patches[m++] = tag | int32_t(L.npatch);
        *L.npatches = m;
    }
}

// The all-level list of levels jmin..jmax from the levels' lists, and its entries
// whose tile is not regular (the irregular list, same order); one block.
template <class R>
__device__ void concat_lists(const DevLevelT<R>* __restrict__ lvs, int jmin, int jmax, int32_t* all, int32_t* count,
                             int32_t* irr, int32_t* irr_count) {
    __shared__ int base, ibase;
    __shared__ int warp_tot[32];
    if (threadIdx.x == 0) base = 0, ibase = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = jmin; j <= jmax; ++j) {
        const DevLevelT<R>& L = lvs[j];
        const int n = *L.npatches;
        const bool all_irr = viscous(L) || L.advect || L.thalo == nullptr;
        // all entries in level order; the entries whose tile is not regular (see
        // tile_regular) also into the irregular list, in the same order
        for (int start = 0; start < n; start += blockDim.x) {
            const int i = start + threadIdx.x;
            int32_t ent = 0;
            int f = 0;
            if (i < n) {
                ent = L.patches[i];
                all[base + i] = ent;
                const int64_t pat = ent & PATCH_MASK;
                f = (all_irr || pat >= L.npatch || L.tirr[pat]) ? 1 : 0;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, f);
            if (lane == 0) warp_tot[w] = __popc(bal);
            __syncthreads();
            int off = 0;
            for (int k = 0; k < w; ++k) off += warp_tot[k];
            if (f) irr[ibase + off + __popc(bal & ((1u << lane) - 1u))] = ent;
            __syncthreads();
            if (threadIdx.x == 0) {
                int tot = 0;
                for (int k = 0; k < nw; ++k) tot += warp_tot[k];
                ibase += tot;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) base += n;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = base, *irr_count = ibase;
    // the point work lists are rebuilt from these lists next (wl_build)
    for (int j = jmin + int(threadIdx.x); j <= jmax && threadIdx.x < 32; j += 32)
        if (lvs[j].wl_n)
            for (int k = 0; k < WL_WORDS; ++k) lvs[j].wl_n[k] = 0;
}

// offset of work list k of a level in wl
template <class R>
__device__ __forceinline__ int64_t wl_off(const DevLevelT<R>& L, int k) {
    return k == WL_GN ? 0 : k == WL_GE ? L.N : k == WL_CN ? L.N + L.E : k == WL_RE ? 2 * L.N + L.E : 2 * L.N + 2 * L.E;
}

// warp-aggregated append of v to work list k of L when pred (the lanes of the warp
// that reach the call take part).  All lanes of a warp belong to one level: the
// work-list build visits 4 x P items per list entry (node and edge slots), with
// P >= 16 (patch sides 4, 8, 16) a multiple of 32.
template <class R>
__device__ __forceinline__ void wl_push(const DevLevelT<R>& L, int k, bool pred, int32_t v) {
    const unsigned act = __activemask();
    const unsigned m = __ballot_sync(act, pred);
    if (!pred) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&L.wl_n[k], __popc(m));
    base = __shfl_sync(m, base, leader);
    L.wl[wl_off(L, k) + base + __popc(m & ((1u << lane) - 1u))] = v;
}

// The point work lists of one item of an active patch (node or edge, see
// visit_item): ghost points, covered nodes, edges with a covered end, and
// available nodes with a covered node among themselves and their neighbours (their
// divergence changes with the restricted fluxes); and the count of live nodes.
// The order of the lists is not fixed; every item's work is independent of it.
template <class R>
__device__ __forceinline__ void wl_item(const DevLevelT<R>& L, int kind, int64_t id) {
    if (kind == K_NODE) {
        const uint8_t f = L.nflag[id];
        {   // the level's live nodes (warp-aggregated)
            const unsigned act = __activemask();
            const unsigned m = __ballot_sync(act, (f & LIVE) != 0);
            if ((threadIdx.x & 31) == __ffs(act) - 1 && m) atomicAdd(&L.wl_n[WL_LIVE], __popc(m));
        }
        wl_push(L, WL_GN, (f & GHOST) != 0, int32_t(id));
        wl_push(L, WL_CN, (f & COVERED) != 0, int32_t(id));
        wl_push(L, WL_DN, restricted_div_node(L, id), int32_t(id));
    } else {
        const uint8_t f = L.eflag[id];
        wl_push(L, WL_GE, (f & GHOST) != 0, int32_t(id));
        const bool r = ((L.nflag[L.en[id]] | L.nflag[L.en[L.E + id]]) & COVERED) != 0;
        wl_push(L, WL_RE, r, int32_t(id));
    }
}

