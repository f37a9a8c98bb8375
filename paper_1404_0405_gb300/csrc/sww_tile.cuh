// Structured trend of one regular patch (Sec. 3.1 operators; Sec. 5.2 patches):
// the tile of tile.h staged in shared memory, neighbours at constant offsets,
// the energy-conserving Coriolis weights derived from the kite areas.
//
// Included inside an anonymous namespace after sww_bodies.cuh and bulk.cuh.  All
// threads of the block call tile_trend and tile_sweep together (they synchronise
// the block).
//
// Per tile: depth and velocity with their flags over the tile range (velocity
// signs turned to the local directions), copied asynchronously through the
// patch's halo table while the previous patch is worked on; and the patch's
// geometry block (TileGeo: edge lengths d_e and l_e, for
// each triangle its three kite areas, its area and its Coriolis parameter, the
// inverse kite sums of the nodes and the cell areas), the FP64 tables rounded
// once to the working precision exactly as the stencils round them, brought in
// whole by one bulk copy while the previous patch is worked on.  Then
//   F = h_e u at every available edge, q = (curl u + f)/h_v at every available
//   triangle (kite-weighted h_v);
//   div F, K and B = g dh + K at the patch's available nodes, and at its live
//   edges q F^perp = (1/d_e) sum over the ten edges e' of the two cells of
//   n_{e,i} n_{e',i} (1/2 - sum of the fractions passed counter-clockwise from e
//   to e') l_{e'} F_{e'} (q_e + q_{e'})/2, a node's kite fractions being its six
//   kites over their sum.
// The outputs are those of the tabulated bodies (flux_at, pv_at, node_at,
// coriolis_at): F at available edges, q at available triangles, c and B at
// available nodes, Q at live edges, for the patch's own points.
#pragma once
// (tile.h is included at file scope by the translation unit)

// Geometry block of one regular patch over the tile's slot ranges, in R: the FP64
// tables rounded once (geo<R>) to the values the stencils use.  Word offsets:
// d_e and l_e at edge slots, kite c of triangle slot (t, x) at (3 t + c) NN + x,
// the inverse kite sum at node slots of [0, P]^2, A_v and f_v at triangle slots,
// A_i of the patch's own nodes; padded to a multiple of 16 bytes (a bulk copy).
template <class R, int P>
struct TileGeo {
    static constexpr int W = P + 3, NN = W * W, PP = P * P;
    static constexpr int DE = 0, LE = DE + 3 * NN, KT = LE + 3 * NN, IS = KT + 6 * NN, AV = IS + NN, FV = AV + 2 * NN,
                         AI = FV + 2 * NN;
    static constexpr int WORDS = ((AI + PP) * int(sizeof(R)) + 15) / 16 * 16 / int(sizeof(R));
    static constexpr uint32_t BYTES = uint32_t(WORDS) * uint32_t(sizeof(R));
};

template <class R, int P>
struct Tile {
    static constexpr int W = P + 3;   // node positions per side, a = -1 .. P + 1
    static constexpr int NN = W * W;
    static constexpr tile::Shape S{P};
    static constexpr int HALO = S.halo();
    using G = TileGeo<R, P>;
    static constexpr size_t up16(size_t x) { return (x + 15) / 16 * 16; }
    // shared-memory layout (bytes): two geometry buffers and two buffers of staged
    // fields (patch i of a block's sweep uses buffers i mod 2), F and q, the
    // geometry buffers' mbarriers
    static constexpr size_t OFF_GEO = 0;   // R[2][G::WORDS]
    // staged fields: dh[NN], u[3 NN] (local direction), the flag words as copied
    // nfw[NN], efw[3 NN] (uint32), the flags nf[NN], ef[3 NN]
    static constexpr size_t STAGED = up16(sizeof(R) * 4 * NN + 4 * 4 * NN + 4 * NN);
    static constexpr size_t OFF_STG = OFF_GEO + 2 * size_t(G::BYTES);   // [2][STAGED]
    static constexpr size_t ST_DH = 0, ST_U = sizeof(R) * NN, ST_NFW = sizeof(R) * 4 * NN, ST_EFW = ST_NFW + 4 * NN,
                            ST_NF = ST_EFW + 4 * 3 * NN, ST_EF = ST_NF + NN;
    static constexpr size_t OFF_F = OFF_STG + 2 * STAGED;                 // R[3 NN]
    static constexpr size_t OFF_Q = OFF_F + sizeof(R) * 3 * NN;           // R[2 NN]
    static constexpr size_t OFF_BAR = up16(OFF_Q + sizeof(R) * 2 * NN);   // uint64[2]
    static constexpr size_t BYTES = OFF_BAR + 16;

    __device__ static int at(int a, int b) { return (a + 1) * W + (b + 1); }
};

// The slots of a tile one thread stages, for NT threads (slot i of thread t is
// node x = t + i NT, edge y = t + i NT, triangle z = t + i NT): own points as
// -(offset) - 1 (offset of the element in the patch, with o P^2 or t P^2 added for
// edges and triangles), halo points as their index in the patch's halo table,
// positions outside the block ranges as NONE.  The same for every tile.
template <int P, int NT>
struct TilePlan {
    static constexpr int W = P + 3, NN = W * W;
    static constexpr int SN = (NN + NT - 1) / NT, SE = (3 * NN + NT - 1) / NT, ST = (2 * NN + NT - 1) / NT;
    static constexpr int NONE = -(1 << 30);
    int n[SN], e[SE], t[ST];

    __device__ void init() {
        constexpr tile::Shape S{P};
        const int tid = threadIdx.x;
#pragma unroll
        for (int i = 0; i < SN; ++i) {
            const int x = tid + i * NT;
            int a = x / W - 1, b = x % W - 1;
            n[i] = x >= NN ? NONE : (a >= 0 && a < P && b >= 0 && b < P) ? -(a * P + b) - 1 : tile::slot(P, P + 1, a, b);
        }
#pragma unroll
        for (int i = 0; i < SE; ++i) {
            const int y = tid + i * NT, o = y / NN, x = y - o * NN;
            int a = x / W - 1, b = x % W - 1;
            e[i] = (y >= 3 * NN || a > S.eA(o) || b > S.eB(o)) ? NONE
                   : (a >= 0 && a < P && b >= 0 && b < P) ? -(o * P * P + a * P + b) - 1
                                                          : S.off_edge(o) + tile::slot(P, S.eB(o), a, b);
        }
#pragma unroll
        for (int i = 0; i < ST; ++i) {
            const int z = tid + i * NT, tt = z / NN, x = z - tt * NN;
            int a = x / W - 1, b = x % W - 1;
            t[i] = (z >= 2 * NN || a > P || b > P) ? NONE
                   : (a >= 0 && a < P && b >= 0 && b < P) ? -(tt * P * P + a * P + b) - 1
                                                          : S.off_tri(tt) + tile::slot(P, P, a, b);
        }
    }
};

// the structured path applies: a regular tile of a level with tiles, inviscid and
// with the velocity free (the viscous and advection forms take the tabulated path)
template <class R>
__device__ __forceinline__ bool tile_regular(const DevLevelT<R>& L, int64_t pat) {
    return pat < L.npatch && L.thalo != nullptr && L.tirr[pat] == 0 && !viscous(L) && !L.advect;
}

// position (a, b) of tile slot x = (a + 1) W + (b + 1)
template <int W>
__device__ __forceinline__ void tpos(int x, int& a, int& b) {
    a = x / W - 1;
    b = x % W - 1;
}

// Tile offsets, relative to node slot x, of the ring of a node: ring edge k (edge
// slot: 0..2 the node's own edges o = k, 3..5 the edges coming in from (a-1, b),
// (a-1, b-1), (a, b-1)) and ring triangle k (between ring edges k and k+1).
template <int W, int NN>
__device__ __forceinline__ constexpr int ring_edge_off(int k) {
    return k == 0 ? 0 : k == 1 ? NN : k == 2 ? 2 * NN : k == 3 ? -W : k == 4 ? NN - W - 1 : 2 * NN - 1;
}
template <int W, int NN>
__device__ __forceinline__ constexpr int ring_tri_off(int k) {
    return k == 0 ? 0 : k == 1 ? NN : k == 2 ? -W : k == 3 ? NN - W - 1 : k == 4 ? -W - 1 : NN - 1;
}

// Offset, in the kite array, of ring kite k of the node at slot 0: the node's
// vertex in ring triangle k (t0 (a,b) 0, t1 (a,b) 0, t0 (a-1,b) 1, t1 (a-1,b-1) 1,
// t0 (a-1,b-1) 2, t1 (a,b-1) 2) at (3 t + c) NN plus the triangle's slot offset.
template <int W, int NN>
__device__ __forceinline__ constexpr int kite_off(int k) {
    return ring_tri_off<W, NN>(k) - (k & 1) * NN + (3 * (k & 1) + (k >> 1)) * NN;
}

// q F^perp at the live edge of orientation O from node slot x: the two cells'
// contributions n_{e,i} sum_{m=1..5} n_{e',i} (1/2 - sum of the fractions passed) l_{e'}
// F_{e'} (q_e + q_{e'})/2, over d_e (edge e sits at ring position O of its origin and
// O + 3 of its end); a node's kite fractions are its kites times is (1 / their sum)
template <class R, int W, int NN, int O>
__device__ __forceinline__ R tile_coriolis(int x, const R* q, const R* F, const R* le, const R* de, const R* kt,
                                           const R* is) {
    constexpr int xe = O == 0 ? W : O == 1 ? W + 1 : 1;   // end node slot - origin node slot
    const int y = O * NN + x;
    const R qe = R(0.5) * (q[x + ring_tri_off<W, NN>(O)] + q[x + ring_tri_off<W, NN>((O + 5) % 6)]);
    const R inv_d = R(1) / de[y];
    R s = R(0);
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int xv = side == 0 ? x : x + xe;
        const int k = side == 0 ? O : O + 3;
        const R ne = side == 0 ? R(1) : R(-1);
        const R inv_s = is[xv];
        R csum = R(0);
#pragma unroll
        for (int m = 1; m < 6; ++m) {
            const int kk = (k + m) % 6, kp = (k + m + 5) % 6;
            csum += kt[kite_off<W, NN>(kp) + xv] * inv_s;
            const int y2 = xv + ring_edge_off<W, NN>(kk);
            const R n2 = kk < 3 ? R(1) : R(-1);
            const R q2 = R(0.5) * (q[xv + ring_tri_off<W, NN>(kk)] + q[xv + ring_tri_off<W, NN>((kk + 5) % 6)]);
            const R w = ne * n2 * (R(0.5) - csum) * le[y2] * inv_d;
            s += w * F[y2] * R(0.5) * (qe + q2);
        }
    }
    return s;
}

// The halo ids a thread's slots need for one tile (own slots: unused), loaded one
// tile ahead so that their latency overlaps the previous tile's work.
template <int P, int NT>
struct TileCodes {
    using PL = TilePlan<P, NT>;
    int32_t n[PL::SN], e[PL::SE], t[PL::ST];

    template <class Lv>
    __device__ void load(const Lv& L, int64_t pat, const PL& plan) {
        constexpr tile::Shape S{P};
        const int32_t* __restrict__ halo = L.thalo + pat * S.halo();
#pragma unroll
        for (int i = 0; i < PL::SN; ++i) n[i] = plan.n[i] >= 0 ? halo[plan.n[i]] : 0;
#pragma unroll
        for (int i = 0; i < PL::SE; ++i) e[i] = plan.e[i] >= 0 ? halo[plan.e[i]] : 0;
#pragma unroll
        for (int i = 0; i < PL::ST; ++i) t[i] = plan.t[i] >= 0 ? halo[plan.t[i]] : 0;
    }
};

// Edge e and its direction flip (halo) of edge slot code c, codes entry hc.
template <int P>
__device__ __forceinline__ int32_t slot_edge(int c, int32_t hc, int32_t nelem, int32_t base, bool& rev) {
    constexpr int PP = P * P;
    if (c < 0) {
        const int k = -c - 1, o = k / PP;
        rev = false;
        return o * nelem + base + (k - o * PP);
    }
    rev = hc & 1;
    return hc >> 1;
}

// The geometry block of regular patch `pat` of L into out (all threads of one
// block; kt: shared scratch of 6 NN values).  Each value is rounded from the FP64
// tables by geo<R>; the inverse kite sums are summed in the order tile_trend used
// to sum them.
template <class R, int P, int NT>
__device__ void tile_geo_build(const DevLevelT<R>& L, int64_t pat, R* __restrict__ out, R* kt) {
    using G = TileGeo<R, P>;
    using PL = TilePlan<P, NT>;
    constexpr int W = G::W, NN = G::NN, PP = G::PP;
    PL plan;
    plan.init();
    TileCodes<P, NT> codes;
    codes.load(L, pat, plan);
    const int32_t nelem = int32_t(L.nelem), ntri = int32_t(L.T), base = int32_t(pat) * PP;
    const int tid = threadIdx.x;
#pragma unroll
    for (int i = 0; i < PL::SE; ++i) {
        const int c = plan.e[i], y = tid + i * NT;
        if (c == PL::NONE) continue;
        bool rev;
        const int32_t e = slot_edge<P>(c, codes.e[i], nelem, base, rev);
        out[G::DE + y] = geo<R>(L.d_e, e);
        out[G::LE + y] = geo<R>(L.l_e, e);
    }
#pragma unroll
    for (int i = 0; i < PL::ST; ++i) {
        const int c = plan.t[i], z = tid + i * NT;
        if (c == PL::NONE) continue;
        int32_t tr;
        int sft;
        if (c < 0) {
            const int k = -c - 1, t = k / PP;
            tr = t * nelem + base + (k - t * PP);
            sft = 0;
        } else {
            tr = codes.t[i] >> 2;
            sft = codes.t[i] & 3;
        }
        const int t = z / NN, x = z - t * NN;
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            const int gc = cc + sft < 3 ? cc + sft : cc + sft - 3;
            const R k = geo<R>(L.kite, int64_t(gc) * ntri + tr);
            kt[(3 * t + cc) * NN + x] = k;
            out[G::KT + (3 * t + cc) * NN + x] = k;
        }
        out[G::AV + z] = geo<R>(L.A_v, tr);
        out[G::FV + z] = geo<R>(L.f_v, tr);
    }
    __syncthreads();
    for (int x = tid; x < NN; x += NT) {
        const int a = x / W - 1, b = x % W - 1;
        if (a < 0 || b < 0 || a > P || b > P) continue;
        // the node's six kites: t0 (a,b) vertex 0, t1 (a,b) 0, t0 (a-1,b) 1,
        // t1 (a-1,b-1) 1, t0 (a-1,b-1) 2, t1 (a,b-1) 2
        R s = R(0);
#pragma unroll
        for (int k = 0; k < 6; ++k) s += kt[kite_off<W, NN>(k) + x];
        out[G::IS + x] = R(1) / s;
    }
    for (int i = tid; i < PP; i += NT) out[G::AI + i] = geo<R>(L.A_i, base + i);
}

// Starts this thread's element copies of the fields of tile (L, pat) into staged
// buffer `stg`: dh and u at its slots, and for the flags the aligned 32-bit word
// holding each flag byte (the flag arrays are padded to a multiple of 16 bytes),
// with the byte's position in the word and the velocity's direction flip left in
// nf and ef for tile_trend to apply.
template <class R, int P, int NT>
__device__ __forceinline__ void tile_fetch(const DevLevelT<R>& L, int64_t pat, const TilePlan<P, NT>& plan,
                                           const TileCodes<P, NT>& codes, unsigned char* stg) {
    using T = Tile<R, P>;
    using PL = TilePlan<P, NT>;
    constexpr int PP = P * P;
    R* dh = reinterpret_cast<R*>(stg + T::ST_DH);
    R* u = reinterpret_cast<R*>(stg + T::ST_U);
    uint32_t* nfw = reinterpret_cast<uint32_t*>(stg + T::ST_NFW);
    uint32_t* efw = reinterpret_cast<uint32_t*>(stg + T::ST_EFW);
    uint8_t* nf = stg + T::ST_NF;
    uint8_t* ef = stg + T::ST_EF;
    const int32_t nelem = int32_t(L.nelem), base = int32_t(pat) * PP;
    const int tid = threadIdx.x;
#pragma unroll
    for (int i = 0; i < PL::SN; ++i) {
        const int c = plan.n[i];
        if (c == PL::NONE) continue;
        const int x = tid + i * NT;
        const int32_t v = c < 0 ? base + (-c - 1) : codes.n[i];
        async_copy<sizeof(R)>(dh + x, L.dh + v);
        async_copy<4>(nfw + x, L.nflag + (v & ~3));
        nf[x] = uint8_t(v & 3);
    }
#pragma unroll
    for (int i = 0; i < PL::SE; ++i) {
        const int c = plan.e[i], y = tid + i * NT;
        if (c == PL::NONE) continue;
        bool rev;
        const int32_t e = slot_edge<P>(c, codes.e[i], nelem, base, rev);
        async_copy<sizeof(R)>(u + y, L.u + e);
        async_copy<4>(efw + y, L.eflag + (e & ~3));
        ef[y] = uint8_t((e & 3) | (rev ? 4 : 0));
    }
    async_commit();
}

// The trend of one regular tile (all threads of the block): its fields fetched
// into staged-field buffer `k` (tile_fetch), its geometry block in `geo` (shared
// memory) once wait_geo() has returned true.  After the staging barrier the
// block's earlier tiles are done with every buffer but k's, and after_stage()
// runs (it may refill them).  False, for every thread, when wait_geo() failed for
// some thread (nothing is computed).
template <class R, int P, int NT, class WaitGeo, class AfterStage>
__device__ bool tile_trend(const DevLevelT<R>& L, int64_t pat, R H, R g, const TilePlan<P, NT>& plan,
                           unsigned char* smem, int k, const R* geo, WaitGeo wait_geo, AfterStage after_stage) {
    using T = Tile<R, P>;
    using G = TileGeo<R, P>;
    using PL = TilePlan<P, NT>;
    constexpr int W = T::W, NN = T::NN, PP = P * P;
    unsigned char* stg = smem + T::OFF_STG + k * T::STAGED;
    R* __restrict__ dh = reinterpret_cast<R*>(stg + T::ST_DH);
    R* __restrict__ u = reinterpret_cast<R*>(stg + T::ST_U);
    const uint32_t* __restrict__ nfw = reinterpret_cast<const uint32_t*>(stg + T::ST_NFW);
    const uint32_t* __restrict__ efw = reinterpret_cast<const uint32_t*>(stg + T::ST_EFW);
    uint8_t* __restrict__ nf = stg + T::ST_NF;
    uint8_t* __restrict__ ef = stg + T::ST_EF;
    R* __restrict__ F = reinterpret_cast<R*>(smem + T::OFF_F);
    R* __restrict__ q = reinterpret_cast<R*>(smem + T::OFF_Q);
    const R* __restrict__ de = geo + G::DE;
    const R* __restrict__ le = geo + G::LE;
    const R* __restrict__ kt = geo + G::KT;
    const R* __restrict__ is = geo + G::IS;
    const R* __restrict__ av = geo + G::AV;
    const R* __restrict__ fv = geo + G::FV;
    const R* __restrict__ ai = geo + G::AI;
    const int32_t nelem = int32_t(L.nelem);
    const int32_t base = int32_t(pat) * PP;
    const int tid = threadIdx.x;
    // --- the fields tile_fetch copied for this thread's slots: the flag bytes out of
    // their words (the byte's position was left in nf/ef), the velocity turned to the
    // local direction
    async_wait_all();
#pragma unroll
    for (int i = 0; i < PL::SN; ++i) {
        const int x = tid + i * NT;
        if (plan.n[i] == PL::NONE) continue;
        nf[x] = uint8_t(nfw[x] >> (8 * nf[x]));
    }
#pragma unroll
    for (int i = 0; i < PL::SE; ++i) {
        const int y = tid + i * NT;
        if (plan.e[i] == PL::NONE) {
            if (y < 3 * NN) ef[y] = 0;
            continue;
        }
        const uint8_t m = ef[y];
        ef[y] = uint8_t(efw[y] >> (8 * (m & 3)));
        if (m & 4) u[y] = -u[y];
    }
    if (!__syncthreads_and(wait_geo())) return false;
    after_stage();
    // --- F at edges, q at triangles
#pragma unroll
    for (int i = 0; i < PL::SE; ++i) {
        const int y = tid + i * NT;
        if (plan.e[i] == PL::NONE) continue;
        const int o = y / NN, x = y - o * NN;
        R f = R(0);
        if (ef[y] & AVAIL) {
            const int x2 = x + (o == 0 ? W : o == 1 ? W + 1 : 1);
            if ((nf[x] & AVAIL) && (nf[x2] & AVAIL)) {
                f = R(0.5) * ((H + dh[x]) + (H + dh[x2])) * u[y];
                if (plan.e[i] < 0) L.F[o * nelem + base + (-plan.e[i] - 1 - o * PP)] = f;
            }
        }
        F[y] = f;
    }
#pragma unroll
    for (int i = 0; i < PL::ST; ++i) {
        const int c = plan.t[i], z = tid + i * NT;
        if (c == PL::NONE) continue;
        const int t = z / NN, x = z - t * NN;
        // vertices and counter-clockwise sides: t0 (a,b),(a+1,b),(a+1,b+1) with sides
        // o0(a,b) +, o2(a+1,b) +, o1(a,b) -;  t1 (a,b),(a+1,b+1),(a,b+1) with sides
        // o1(a,b) +, o0(a,b+1) -, o2(a,b) -
        const int n1 = t == 0 ? x + W : x + W + 1, n2 = t == 0 ? x + W + 1 : x + 1;
        const int s0 = t == 0 ? x : NN + x, s1 = t == 0 ? 2 * NN + x + W : x + 1, s2 = t == 0 ? NN + x : 2 * NN + x;
        R qq = R(0);
        if ((nf[x] & AVAIL) && (nf[n1] & AVAIL) && (nf[n2] & AVAIL) && (ef[s0] & AVAIL) && (ef[s1] & AVAIL) &&
            (ef[s2] & AVAIL)) {
            const R circ = u[s0] * de[s0] + (t == 0 ? R(1) : R(-1)) * u[s1] * de[s1] + R(-1) * u[s2] * de[s2];
            const R hv = kt[(3 * t) * NN + x] * (H + dh[x]) + kt[(3 * t + 1) * NN + x] * (H + dh[n1]) +
                         kt[(3 * t + 2) * NN + x] * (H + dh[n2]);
            const R A = av[z];
            qq = (circ / A + fv[z]) / (hv / A);
            if (c < 0) L.q[t * nelem + base + (-c - 1 - t * PP)] = qq;
        }
        q[z] = qq;
    }
    __syncthreads();
    // --- the patch's own nodes (div F, K, B) and live edges (energy-conserving
    // q F^perp), in one pass of PP + 3 PP items (orientation uniform over a warp when
    // P * P is a multiple of 32)
    for (int w = tid; w < 4 * PP; w += NT) {
        if (w < PP) {
            const int i = w, x = T::at(i / P, i % P);
            if (!(nf[x] & AVAIL)) continue;
            bool okr = true;
            R div = R(0), ke = R(0);
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const int y = x + ring_edge_off<W, NN>(k);
                okr = okr && (ef[y] & AVAIL);
                const R n = k < 3 ? R(1) : R(-1);
                div += n * F[y] * le[y];
                ke += R(0.25) * le[y] * de[y] * u[y] * u[y];
            }
            if (!okr) continue;
            const int32_t v = base + i;
            const R A = ai[i];
            L.c[v] = div / A;
            L.B[v] = g * dh[x] + ke / A;
        } else {
            const int o = (w - PP) / PP, i = (w - PP) - o * PP, x = T::at(i / P, i % P);
            if (!(ef[o * NN + x] & LIVE)) continue;
            const R Q = o == 0 ? tile_coriolis<R, W, NN, 0>(x, q, F, le, de, kt, is)
                               : o == 1 ? tile_coriolis<R, W, NN, 1>(x, q, F, le, de, kt, is)
                                        : tile_coriolis<R, W, NN, 2>(x, q, F, le, de, kt, is);
            L.Q[o * nelem + base + i] = Q;
        }
    }
    return true;
}

// The trend of the active patches first, first + stride, ... (< n) of an
// all-level list, by one block: regular patches by tile_trend, other patches by
// other(L, pat).  Patch i of the sweep uses buffers i mod 2 (staged fields,
// geometry).  The next patch's fields (element copies, tile_fetch) and geometry
// block (a bulk copy) are started right after this patch's staging barrier, once
// every thread is done with the patch before, which used those buffers; the
// halo ids they need are loaded a patch earlier still.  So one barrier separates
// consecutive patches, and the copies run while this patch is worked on.  False,
// with *err set, when a bulk copy did not complete within `limit` cycles (the
// block then gives it one more bounded wait and leaves).
template <class R, int P, int NT, class Other>
__device__ bool tile_sweep(const DevLevelT<R>* lv, const int32_t* list, int n, int first, int stride, R H, R g,
                           unsigned char* smem, int* err, long long limit, Other other) {
    using T = Tile<R, P>;
    using G = TileGeo<R, P>;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + T::OFF_BAR);
    R* gbuf = reinterpret_cast<R*>(smem + T::OFF_GEO);
    if (threadIdx.x == 0) {
        mbar_init(bar);
        mbar_init(bar + 1);
        fence_barrier_init();
    }
    __syncthreads();
    TilePlan<P, NT> plan;
    plan.init();
    auto regular = [&](int e) -> bool {
        if (e >= n) return false;
        const int32_t ent = list[e];
        return tile_regular(lv[ent >> LVL_SHIFT], ent & PATCH_MASK);
    };
    auto codes_of = [&](int e, TileCodes<P, NT>& c) {
        const int32_t ent = list[e];
        c.load(lv[ent >> LVL_SHIFT], ent & PATCH_MASK, plan);
    };
    // list entry e (regular, halo ids c) into buffers k: its fields and, from
    // thread 0, its geometry block
    auto start = [&](int e, const TileCodes<P, NT>& c, int k) {
        const int32_t ent = list[e];
        const DevLevelT<R>& L = lv[ent >> LVL_SHIFT];
        const int64_t pat = ent & PATCH_MASK;
        tile_fetch<R, P, NT>(L, pat, plan, c, smem + T::OFF_STG + k * T::STAGED);
        if (threadIdx.x == 0) {
            fence_async_shared();   // the buffer's last readers are behind a block barrier
            bulk_load(gbuf + k * G::WORDS, L.tgeo + pat * G::WORDS, G::BYTES, bar + k);
        }
    };
    TileCodes<P, NT> c1, c2;   // halo ids of the next patch and of the one after
    bool reg = regular(first);
    bool reg1 = regular(first + stride);
    if (reg) {
        TileCodes<P, NT> c0;
        codes_of(first, c0);
        start(first, c0, 0);
    }
    if (reg1) codes_of(first + stride, c1);
    unsigned ph = 0;   // bit k: parity of buffer k's next phase
    int k = 0;
    for (int e = first; e < n; e += stride, k ^= 1) {
        const int32_t ent = list[e];
        const DevLevelT<R>& L = lv[ent >> LVL_SHIFT];
        const int64_t pat = ent & PATCH_MASK;
        const bool reg2 = regular(e + 2 * stride);
        if (reg2) codes_of(e + 2 * stride, c2);
        if (reg) {
            const uint32_t parity = (ph >> k) & 1u;
            ph ^= 1u << k;
            const bool done = tile_trend<R, P, NT>(
                L, pat, H, g, plan, smem, k, gbuf + k * G::WORDS, [&]() { return mbar_wait(bar + k, parity, limit); },
                [&]() {
                    if (reg1) start(e + stride, c1, k ^ 1);
                });
            if (!done) {
                // this patch's bulk copy did not land in time: report it, give it one
                // more bounded wait, and leave (nothing else was started)
                if (threadIdx.x == 0) atomicExch(err, 1);
                mbar_wait(bar + k, parity, limit);
                return false;
            }
        } else {
            // the tabulated path shares no buffer with the tiles; the next copies wait
            // for the block barrier that ends this patch
            other(L, pat);
            __syncthreads();
            if (reg1) start(e + stride, c1, k ^ 1);
        }
        c1 = c2;
        reg = reg1;
        reg1 = reg2;
    }
    return true;
}
