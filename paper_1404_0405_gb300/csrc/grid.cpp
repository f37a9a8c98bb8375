// Host construction of the nested icosahedral grid, its spherical geometry and
// the tables the CUDA kernels read (TRiSK reconstruction weights, lifting
// weights, velocity prediction weights, restricted-flux coefficients).
//
// Sec. 2.2 (nested grids by edge bisection and projection), Table 1, Sec. 3.1
// (staggered C-grid, TRiSK operators), Sec. 4.1 (spherical areas, arc lengths,
// hexagon intersection areas A_km, 12-edge velocity interpolation), Sec. 4.2-4.3
// (flux restriction), Sec. 5.2 (lozenges, elements, patches).  Readings taken
// where the text is silent are stated next to the code that applies them.
#include "grid.h"

#include "tile.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <stdexcept>
#include <string>

namespace sww {
namespace {

inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(V3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double len(V3 a) { return std::sqrt(dot(a, a)); }
inline V3 unit(V3 a) { return a * (1.0 / len(a)); }

// Great-circle angle; |a x b| taken as |a x (b - a)| to keep precision on short arcs.
inline double arc(V3 a, V3 b) { return std::atan2(len(cross(a, b - a)), dot(a, b)); }

// Signed spherical triangle area on the unit sphere, tan(E/2) = a.(b x c)/(1+a.b+b.c+c.a),
// with the triple product formed from differences (full precision for small triangles).
inline double tri_area(V3 a, V3 b, V3 c) {
    double num = dot(a, cross(b - a, c - a));
    double den = 1.0 + dot(a, b) + dot(b, c) + dot(c, a);
    return 2.0 * std::atan2(num, den);
}

// Point equidistant from a, b, c on the sphere, on the triangle's side.
inline V3 circumcentre(V3 a, V3 b, V3 c) {
    V3 nrm = unit(cross(b - a, c - a));
    if (dot(nrm, a + b + c) < 0) nrm = nrm * -1.0;
    return nrm;
}

inline void tangent_basis(V3 x, V3& e1, V3& e2) {
    V3 ref = std::fabs(x.x) < 0.8 ? V3{1, 0, 0} : V3{0, 1, 0};
    e1 = unit(cross(x, ref));
    e2 = cross(x, e1);                    // e1 x e2 = x: counter-clockwise seen from outside
}

// Area of the intersection of two convex spherical polygons (both counter-clockwise),
// by clipping `subj` against the great-circle half-spaces of `clipv`'s edges.
double intersection_area(const V3* subj, int ns, const V3* clipv, int nc) {
    V3 P[20], Q[20];
    int np = ns;
    for (int k = 0; k < ns; ++k) P[k] = subj[k];
    for (int h = 0; h < nc && np >= 3; ++h) {
        V3 a = clipv[h], b = clipv[(h + 1) % nc];
        V3 nrm = cross(a, b - a);
        int nq = 0;
        for (int k = 0; k < np; ++k) {
            V3 s = P[(k + np - 1) % np], e = P[k];
            double ds = dot(nrm, s - a), de = dot(nrm, e - a);
            bool si = ds >= 0.0, ei = de >= 0.0;
            if (si != ei) {
                double t = ds / (ds - de);
                Q[nq++] = unit(s * (1.0 - t) + e * t);
            }
            if (ei) Q[nq++] = e;
        }
        for (int k = 0; k < nq; ++k) P[k] = Q[k];
        np = nq;
    }
    if (np < 3) return 0.0;
    double area = 0.0;
    for (int k = 1; k + 1 < np; ++k) area += tri_area(P[0], P[k], P[k + 1]);
    return area;
}

// Solve the symmetric positive definite system G x = b (n <= 6) by Cholesky.
bool cholesky_solve(double G[6][6], double b[6], int n) {
    double L[6][6] = {};
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = G[i][j];
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            if (i == j) {
                if (!(s > 0)) return false;
                L[i][i] = std::sqrt(s);
            } else {
                L[i][j] = s / L[j][j];
            }
        }
    }
    double y[6];
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[i][k] * y[k];
        y[i] = s / L[i][i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < n; ++k) s -= L[k][i] * b[k];
        b[i] = s / L[i][i];
    }
    return true;
}

struct Lay {
    int64_t n, p, np, nelem;
    int64_t elem(int64_t d, int64_t i, int64_t j) const {
        return ((d * np + i / p) * np + j / p) * p * p + (i % p) * p + (j % p);
    }
    void coords(int64_t e, int64_t& d, int64_t& i, int64_t& j) const {
        int64_t pp = p * p, pid = e / pp, loc = e % pp;
        int64_t pj = pid % np, pi = (pid / np) % np;
        d = pid / (np * np);
        i = pi * p + loc / p;
        j = pj * p + loc % p;
    }
    // Node at lattice point (i, j), 0 <= i, j <= n, of lozenge d.  Lozenges 0..4
    // (north) have corners U_k, L_k, U_{k+1}, N at (0,0), (n,0), (n,n), (0,n);
    // lozenges 5..9 (south) have L_k, S, L_{k+1}, U_{k+1}.  Points on the far
    // sides belong to the neighbouring lozenge.
    int64_t node(int64_t d, int64_t i, int64_t j) const {
        if (i < n && j < n) return elem(d, i, j);
        bool north = d < 5;
        int64_t k = north ? d : d - 5, k1 = (k + 1) % 5;
        if (i == n && j == n) return north ? elem(k1, 0, 0) : elem(5 + k1, 0, 0);
        if (i == n) {
            if (north) return elem(5 + k, 0, j);
            if (j == 0) return nelem + 1;
            return elem(5 + k1, n - j, 0);
        }
        if (north) return i == 0 ? nelem : elem(k1, 0, n - i);
        return elem(k1, i, 0);
    }
};

const int DI[3] = {1, 1, 0}, DJ[3] = {0, 1, 1};

Lay layout_of(const HostLevel& L) { return Lay{L.n, L.p, L.np, L.nelem}; }

void init_level(HostLevel& L, int J, int patch) {
    L.J = J;
    L.n = int64_t(1) << J;
    L.p = std::min<int64_t>(patch, L.n);
    L.np = L.n / L.p;
    L.nelem = 10 * L.n * L.n;
    L.N = L.nelem + 2;
    L.E = 3 * L.nelem;
    L.T = 2 * L.nelem;
    L.npatch = 10 * L.np * L.np;
}

// ----------------------------------------------------------------------------- topology

void build_topology(HostLevel& L) {
    Lay Y = layout_of(L);
    const int64_t ne = L.nelem, N = L.N, E = L.E, T = L.T;
    for (int s = 0; s < 2; ++s) L.en[s].assign(E, -1), L.et[s].assign(E, -1);
    for (int c = 0; c < 3; ++c) L.tn[c].assign(T, -1), L.te[c].assign(T, -1);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < ne; ++e) {
        int64_t d, i, j;
        Y.coords(e, d, i, j);
        for (int o = 0; o < 3; ++o) {
            L.en[0][o * ne + e] = int32_t(e);
            L.en[1][o * ne + e] = int32_t(Y.node(d, i + DI[o], j + DJ[o]));
        }
        L.tn[0][e] = int32_t(e);
        L.tn[1][e] = int32_t(Y.node(d, i + 1, j));
        L.tn[2][e] = int32_t(Y.node(d, i + 1, j + 1));
        L.tn[0][ne + e] = int32_t(e);
        L.tn[1][ne + e] = int32_t(Y.node(d, i + 1, j + 1));
        L.tn[2][ne + e] = int32_t(Y.node(d, i, j + 1));
    }
    // incident edges of every node, then counter-clockwise order by angle
    std::vector<int32_t> cnt(N, 0), slot_e(6 * N, -1);
    for (int64_t e = 0; e < E; ++e) {
        for (int s = 0; s < 2; ++s) {
            int64_t v = L.en[s][e];
            if (cnt[v] >= 6) throw std::runtime_error("node degree above 6");
            slot_e[6 * v + cnt[v]++] = int32_t(2 * e + s);
        }
    }
    L.deg.assign(N, 0);
    for (int k = 0; k < 6; ++k) L.ring_e[k].assign(N, -1), L.ring_n[k].assign(N, -1), L.ring_t[k].assign(N, -1);
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < N; ++v) {
        int dg = cnt[v];
        if (dg != 5 && dg != 6) throw std::runtime_error("node degree not 5 or 6");
        V3 x = L.xyz[v], e1, e2;
        tangent_basis(x, e1, e2);
        double ang[6];
        int32_t code[6];
        for (int k = 0; k < dg; ++k) {
            code[k] = slot_e[6 * v + k];
            int64_t e = code[k] >> 1;
            int64_t other = L.en[(code[k] & 1) ? 0 : 1][e];
            V3 dv = L.xyz[other] - x;
            ang[k] = std::atan2(dot(dv, e2), dot(dv, e1));
        }
        for (int a = 1; a < dg; ++a)
            for (int b = a; b > 0 && ang[b] < ang[b - 1]; --b) std::swap(ang[b], ang[b - 1]), std::swap(code[b], code[b - 1]);
        L.deg[v] = uint8_t(dg);
        for (int k = 0; k < dg; ++k) {
            int64_t e = code[k] >> 1;
            L.ring_e[k][v] = code[k];
            L.ring_n[k][v] = L.en[(code[k] & 1) ? 0 : 1][e];
        }
    }
    auto edge_between = [&](int64_t a, int64_t b, int32_t& code) {
        for (int k = 0; k < L.deg[a]; ++k)
            if (L.ring_n[k][a] == b) {
                code = L.ring_e[k][a];      // bit 0 set: the edge points from b to a
                return;
            }
        throw std::runtime_error("missing edge");
    };
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < T; ++t) {
        for (int c = 0; c < 3; ++c) {
            int64_t a = L.tn[c][t], b = L.tn[(c + 1) % 3][t];
            int32_t code;
            edge_between(a, b, code);
            L.te[c][t] = code;                   // 2e + 1 when the edge runs b -> a
            L.et[(code & 1) ? 1 : 0][code >> 1] = int32_t(t);
        }
    }
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < N; ++v) {
        for (int k = 0; k < L.deg[v]; ++k) {
            int32_t code = L.ring_e[k][v];
            int64_t e = code >> 1;
            // triangle to the left of v -> ring_n[k]
            L.ring_t[k][v] = (code & 1) ? L.et[1][e] : L.et[0][e];
        }
    }
    for (int s = 0; s < 2; ++s)
        for (int64_t e = 0; e < E; ++e)
            if (L.et[s][e] < 0) throw std::runtime_error("edge without two triangles");
}

// ----------------------------------------------------------------------------- geometry

void build_geometry(HostLevel& L, double R, double omega) {
    const int64_t N = L.N, E = L.E, T = L.T;
    L.cc.resize(T);
    for (int c = 0; c < 3; ++c) L.kite[c].assign(T, 0);
    L.A_v.assign(T, 0);
    L.f_v.assign(T, 0);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < T; ++t) {
        V3 P[3] = {L.xyz[L.tn[0][t]], L.xyz[L.tn[1][t]], L.xyz[L.tn[2][t]]};
        V3 cc = circumcentre(P[0], P[1], P[2]);
        L.cc[t] = cc;
        double sum = 0;
        for (int c = 0; c < 3; ++c) {
            V3 a = P[c], nx = P[(c + 1) % 3], pv = P[(c + 2) % 3];
            double k = tri_area(a, unit(a + nx), cc) + tri_area(a, cc, unit(pv + a));
            L.kite[c][t] = k * R * R;
            sum += L.kite[c][t];
        }
        L.A_v[t] = sum;
        L.f_v[t] = 2.0 * omega * cc.z;
    }
    L.A_kite.assign(N, 0);
    L.f_n.assign(N, 0);
    for (int k = 0; k < 6; ++k) L.ring_R[k].assign(N, 0);
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < N; ++v) {
        double kk[6], s = 0;
        for (int k = 0; k < L.deg[v]; ++k) {
            int64_t t = L.ring_t[k][v];
            int c = L.tn[0][t] == v ? 0 : (L.tn[1][t] == v ? 1 : 2);
            kk[k] = L.kite[c][t];
            s += kk[k];
        }
        L.A_kite[v] = s;
        for (int k = 0; k < L.deg[v]; ++k) L.ring_R[k][v] = kk[k] / s;
        L.f_n[v] = 2.0 * omega * L.xyz[v].z;
    }
    L.A_i = L.A_kite;
    L.d_e.assign(E, 0);
    L.l_e.assign(E, 0);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; ++e) {
        L.d_e[e] = arc(L.xyz[L.en[0][e]], L.xyz[L.en[1][e]]) * R;
        L.l_e[e] = arc(L.cc[L.et[0][e]], L.cc[L.et[1][e]]) * R;
    }
    // TRiSK energy-conserving perpendicular flux (Ringler et al. 2010, Thuburn et al.
    // 2009): for cell i with ring edges e_1..e_D and kite fractions R_1..R_D, the flux
    // across the half edge from i to the midpoint of e_k is
    //   psi_k = sum_{k'!=k} (1/2 - sum_{m=k}^{k'-1} R_m) n_{k'} F_{k'} l_{k'},
    // and du_e/dt gets n_{e,i} psi_k / d_e from each of its two cells.
    for (int s = 0; s < COR; ++s) L.cor_i[s].assign(E, 0), L.cor_w[s].assign(E, 0);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; ++e) {
        int slot = 0;
        for (int side = 0; side < 2; ++side) {
            int64_t v = L.en[side][e];
            int dg = L.deg[v], k = -1;
            for (int r = 0; r < dg; ++r)
                if ((L.ring_e[r][v] >> 1) == e) k = r;
            double n_e = side == 0 ? 1.0 : -1.0;
            double csum = 0;
            for (int o = 1; o < dg; ++o) {
                int kk = (k + o) % dg;
                csum += L.ring_R[(k + o - 1) % dg][v];
                int32_t code = L.ring_e[kk][v];
                int64_t e2 = code >> 1;
                double n2 = (code & 1) ? -1.0 : 1.0;
                L.cor_i[slot][e] = int32_t(e2);
                L.cor_w[slot][e] = n_e * n2 * (0.5 - csum) * L.l_e[e2] / L.d_e[e];
                ++slot;
            }
        }
        for (; slot < COR; ++slot) L.cor_i[slot][e] = int32_t(e), L.cor_w[slot][e] = 0.0;
    }
}

// ----------------------------------------------------------------------------- tiles

// Halo tables of the structured trend kernel (tile.h).  For each patch the local
// lattice is laid out from its own elements by walking ring neighbours: a node at
// local position (a, b) whose ring slot k0 points along +a has its neighbour in
// direction m at ring slot (k0 + m) mod 6, and that neighbour's +a slot follows
// from where the walk came in.  A tile is regular when every node of its range
// has six neighbours and every walk agrees; otherwise (a pentagon or a pole in
// reach, a level whose patch side is not `patch`) it is marked irregular and the
// kernels take the tabulated path there.
void build_tiles(HostLevel& L, int patch) {
    L.tile_halo.clear();
    L.tile_irr.assign(L.npatch + 1, 1);
    const int p = int(L.p);
    if (!(patch == 4 || patch == 8 || patch == 16) || p != patch) return;
    const tile::Shape S{p};
    const int W = p + 3, HALO = S.halo();
    L.tile_halo.assign(size_t(L.npatch) * HALO, -1);
    Lay Y = layout_of(L);
    const int64_t np = L.np;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t P = 0; P < L.npatch; ++P) {
        const int64_t d = P / (np * np), pi = (P / np) % np, pj = P % np;
        std::vector<int64_t> gid(W * W, -1);
        std::vector<int> k0(W * W, -1), queue;
        auto at = [&](int a, int b) { return (a + 1) * W + (b + 1); };
        auto inside = [&](int a, int b) { return a >= -1 && a <= p + 1 && b >= -1 && b <= p + 1; };
        // seed: the patch's first element; its +a neighbour is lattice node (i + 1, j)
        const int64_t v0 = Y.elem(d, pi * p, pj * p), w0 = Y.node(d, pi * p + 1, pj * p);
        for (int k = 0; k < L.deg[v0]; ++k)
            if (L.ring_n[k][v0] == w0) k0[at(0, 0)] = k;
        gid[at(0, 0)] = v0;
        queue.push_back(at(0, 0));
        bool ok = k0[at(0, 0)] >= 0;
        for (size_t qi = 0; qi < queue.size() && ok; ++qi) {
            const int s = queue[qi], a = s / W - 1, b = s % W - 1;
            const int64_t v = gid[s];
            if (L.deg[v] != 6) {
                ok = false;
                break;
            }
            for (int m = 0; m < 6 && ok; ++m) {
                const int a2 = a + tile::da(m), b2 = b + tile::db(m);
                if (!inside(a2, b2)) continue;
                const int64_t w = L.ring_n[(k0[s] + m) % 6][v];
                if (L.deg[w] != 6) {
                    ok = false;
                    break;
                }
                int kv = -1;
                for (int k = 0; k < 6; ++k)
                    if (L.ring_n[k][w] == v) kv = k;
                const int kw = ((kv - (m + 3)) % 6 + 6) % 6;
                const int s2 = at(a2, b2);
                if (gid[s2] < 0) {
                    gid[s2] = w, k0[s2] = kw;
                    queue.push_back(s2);
                } else if (gid[s2] != w || k0[s2] != kw) {
                    ok = false;
                }
            }
        }
        if (!ok || int(queue.size()) != W * W) continue;
        // the interior is the patch's own elements, their edges and triangles
        for (int a = 0; a < p && ok; ++a)
            for (int b = 0; b < p && ok; ++b) {
                const int s = at(a, b);
                const int64_t el = Y.elem(d, pi * p + a, pj * p + b);
                if (gid[s] != el) ok = false;
                for (int o = 0; o < 3; ++o)
                    if (L.ring_e[(k0[s] + o) % 6][gid[s]] != int32_t(2 * (o * L.nelem + el))) ok = false;
                for (int t = 0; t < 2; ++t)
                    if (L.ring_t[(k0[s] + t) % 6][gid[s]] != int32_t(t * L.nelem + el)) ok = false;
            }
        if (!ok) throw std::runtime_error("tile: interior of a regular patch does not follow the layout");
        int32_t* H = L.tile_halo.data() + size_t(P) * HALO;
        for (int s = 0; s < S.nodes(); ++s) {
            int a, b;
            tile::pos(p, p + 1, s, a, b);
            H[s] = int32_t(gid[at(a, b)]);
        }
        for (int o = 0; o < 3; ++o)
            for (int s = 0; s < S.edges(o); ++s) {
                int a, b;
                tile::pos(p, S.eB(o), s, a, b);
                const int q = at(a, b), q2 = at(a + tile::da(o), b + tile::db(o));
                const int32_t code = L.ring_e[(k0[q] + o) % 6][gid[q]];
                const int64_t e = code >> 1;
                const int64_t other = L.en[(code & 1) ? 0 : 1][e];
                if (other != gid[q2]) throw std::runtime_error("tile: halo edge does not reach its end node");
                H[S.off_edge(o) + s] = code;
            }
        for (int t = 0; t < 2; ++t)
            for (int s = 0; s < S.tris(); ++s) {
                int a, b;
                tile::pos(p, p, s, a, b);
                const int q = at(a, b);
                const int64_t tri = L.ring_t[(k0[q] + t) % 6][gid[q]];
                // local vertices: t0 (a,b), (a+1,b), (a+1,b+1); t1 (a,b), (a+1,b+1), (a,b+1)
                const int64_t v0l = gid[q];
                int sft = -1;
                for (int c = 0; c < 3; ++c)
                    if (L.tn[c][tri] == v0l) sft = c;
                const int64_t v1l = gid[t == 0 ? at(a + 1, b) : at(a + 1, b + 1)];
                if (sft < 0 || L.tn[(1 + sft) % 3][tri] != v1l)
                    throw std::runtime_error("tile: halo triangle does not hold its nodes in order");
                H[S.off_tri(t) + s] = int32_t(4 * tri + sft);
            }
        L.tile_irr[P] = 0;
    }
}

// ----------------------------------------------------------------------------- inter-level

int64_t coarse_edge(const HostLevel& C, int64_t a, int64_t b) {
    for (int k = 0; k < C.deg[a]; ++k)
        if (C.ring_n[k][a] == b) return C.ring_e[k][a] >> 1;
    throw std::runtime_error("coarse edge not found");
}

int64_t third_node(const HostLevel& C, int64_t t, int64_t a, int64_t b) {
    for (int c = 0; c < 3; ++c) {
        int64_t v = C.tn[c][t];
        if (v != a && v != b) return v;
    }
    throw std::runtime_error("degenerate triangle");
}

// Links, parents and clipped overlap areas of the pair (C = level j-1, F = level j).
void link_levels(HostLevel& C, HostLevel& F, double R) {
    Lay Yc = layout_of(C), Yf = layout_of(F);
    const int64_t cne = C.nelem;
    C.c2f.assign(C.N, -1);
    C.mid.assign(C.E, -1);
    C.half[0].assign(C.E, -1);
    C.half[1].assign(C.E, -1);
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < cne; ++e) {
        int64_t d, i, j;
        Yc.coords(e, d, i, j);
        C.c2f[e] = int32_t(Yf.elem(d, 2 * i, 2 * j));
        for (int o = 0; o < 3; ++o) {
            int64_t m = Yf.elem(d, 2 * i + DI[o], 2 * j + DJ[o]);
            C.mid[o * cne + e] = int32_t(m);
            C.half[0][o * cne + e] = int32_t(o * F.nelem + Yf.elem(d, 2 * i, 2 * j));
            C.half[1][o * cne + e] = int32_t(o * F.nelem + m);
        }
    }
    C.c2f[cne] = int32_t(F.nelem);
    C.c2f[cne + 1] = int32_t(F.nelem + 1);
    for (int s = 0; s < 4; ++s) F.par[s].assign(F.N, -1), F.akm[s].assign(F.N, 0), F.ptw[s].assign(F.N, 0);
    // odd node m of the coarse edge e = (a -> b): parents a, b and the opposite vertices
    // of the left and right triangles (Sec. 4.3: two nearest and two second-nearest)
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t e = 0; e < C.E; ++e) {
        int64_t m = C.mid[e];
        int64_t a = C.en[0][e], b = C.en[1][e];
        int64_t c = third_node(C, C.et[0][e], a, b), d = third_node(C, C.et[1][e], a, b);
        int64_t pk[4] = {a, b, c, d};
        V3 hexm[6];
        if (F.deg[m] != 6) throw std::runtime_error("odd node is not a hexagon");
        for (int k = 0; k < 6; ++k) hexm[k] = F.cc[F.ring_t[k][m]];
        for (int s = 0; s < 4; ++s) {
            int64_t k = pk[s];
            V3 hexk[6];
            int dk = C.deg[k];
            for (int r = 0; r < dk; ++r) hexk[r] = C.cc[C.ring_t[r][k]];
            F.par[s][m] = C.c2f[k];
            F.akm[s][m] = intersection_area(hexm, 6, hexk, dk) * R * R;
        }
    }
}

// Tables of the pair (C, F) that need the final (normalised) areas.
void pair_tables(HostLevel& C, HostLevel& F, double R) {
    const int64_t cne = C.nelem;
    // fine-to-coarse node id (inverse of c2f) for parent lookups
    std::vector<int32_t> f2c(F.N, -1);
    for (int64_t k = 0; k < C.N; ++k) f2c[C.c2f[k]] = int32_t(k);
    auto overlap = [&](int64_t y_coarse, int64_t x_fine) -> double {
        int64_t fy = C.c2f[y_coarse];
        for (int s = 0; s < 4; ++s)
            if (F.par[s][x_fine] == fy) return F.akm[s][x_fine];
        throw std::runtime_error("overlap not in parent set");
    };
    // prediction weights s~_km = A_km / A_m
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < F.N; ++m) {
        if (F.par[0][m] < 0) continue;
        for (int s = 0; s < 4; ++s) F.ptw[s][m] = F.akm[s][m] / F.A_i[m];
    }
    // M_k with update weights s_km = A_km / A_k (Eq. 2)
    for (int s = 0; s < 12; ++s) C.mk_i[s].assign(C.N, -1), C.mk_w[s].assign(C.N, 0);
    {
        std::vector<int> cnt(C.N, 0);
        for (int64_t e = 0; e < C.E; ++e) {
            int64_t m = C.mid[e];
            for (int s = 0; s < 4; ++s) {
                int64_t k = f2c[F.par[s][m]];
                if (cnt[k] >= 12) throw std::runtime_error("M_k larger than 12");
                C.mk_i[cnt[k]][k] = int32_t(m);
                C.mk_w[cnt[k]][k] = F.akm[s][m] / C.A_i[k];
                ++cnt[k];
            }
        }
        for (int64_t k = 0; k < C.N; ++k)
            if (cnt[k] != 2 * C.deg[k]) throw std::runtime_error("M_k does not hold 2N nodes");
    }
    // velocity prediction (reading of Sec. 4.1): a fine edge touching or cutting off
    // coarse node a is predicted from the star of a (spokes + rim edges, 12 or 10) with
    // the minimum-norm weights reproducing every linear tangent field in the
    // orthographic plane at the fine edge midpoint (normal equations: one 6x6 solve).
    F.fe_kind.assign(F.E, -1);
    F.fe_ce.assign(F.E, -1);
    for (int s = 0; s < VST; ++s) F.vst[s].assign(F.E, 0), F.vw[s].assign(F.E, 0);
    std::vector<int64_t> centre(F.E, -1);
    for (int64_t e = 0; e < C.E; ++e) {
        for (int h = 0; h < 2; ++h) {
            int64_t fe = C.half[h][e];
            F.fe_kind[fe] = int8_t(h);
            F.fe_ce[fe] = int32_t(e);
            centre[fe] = C.en[h][e];
        }
    }
    for (int64_t t = 0; t < C.T; ++t) {
        for (int c = 0; c < 3; ++c) {
            int64_t m1 = C.mid[C.te[c][t] >> 1], m2 = C.mid[C.te[(c + 2) % 3][t] >> 1];
            int64_t fe = -1;
            for (int k = 0; k < 6; ++k)
                if (F.ring_n[k][m1] == m2) fe = F.ring_e[k][m1] >> 1;
            if (fe < 0) throw std::runtime_error("interior fine edge not found");
            F.fe_kind[fe] = 2;
            F.fe_ce[fe] = int32_t(3 * t + c);
            centre[fe] = C.tn[c][t];
        }
    }
    const double dx = nominal_spacing(C.J, 1.0);
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t fe = 0; fe < F.E; ++fe) {
        int64_t a = centre[fe];
        if (a < 0) throw std::runtime_error("fine edge without predictor");
        int dg = C.deg[a], ns = 2 * dg;
        int32_t st[VST];
        for (int k = 0; k < dg; ++k) {
            st[k] = C.ring_e[k][a] >> 1;
            int64_t t = C.ring_t[k][a];
            int32_t rim = -1;
            for (int c = 0; c < 3; ++c) {
                int64_t ed = C.te[c][t] >> 1;
                if (C.en[0][ed] != a && C.en[1][ed] != a) rim = int32_t(ed);
            }
            st[dg + k] = rim;
        }
        V3 x0 = F.xyz[F.en[0][fe]], x1 = F.xyz[F.en[1][fe]];
        V3 p = unit(x0 + x1), tf = unit(x1 - x0), e1, e2;
        tangent_basis(p, e1, e2);
        double M[6][VST];
        for (int s = 0; s < ns; ++s) {
            V3 ya = C.xyz[C.en[0][st[s]]], yb = C.xyz[C.en[1][st[s]]];
            V3 xm = unit(ya + yb), tm = unit(yb - ya);
            double xi = dot(xm, e1) / dx, eta = dot(xm, e2) / dx;
            double t1 = dot(tm, e1), t2 = dot(tm, e2);
            M[0][s] = t1;
            M[1][s] = t2;
            M[2][s] = xi * t1;
            M[3][s] = eta * t1;
            M[4][s] = xi * t2;
            M[5][s] = eta * t2;
        }
        double G[6][6], b[6] = {dot(tf, e1), dot(tf, e2), 0, 0, 0, 0};
        for (int r = 0; r < 6; ++r)
            for (int c = 0; c < 6; ++c) {
                double s = 0;
                for (int k = 0; k < ns; ++k) s += M[r][k] * M[c][k];
                G[r][c] = s;
            }
        if (!cholesky_solve(G, b, 6)) throw std::runtime_error("singular velocity stencil");
        for (int s = 0; s < VST; ++s) {
            double w = 0;
            if (s < ns)
                for (int r = 0; r < 6; ++r) w += M[r][s] * b[r];
            F.vst[s][fe] = s < ns ? st[s] : st[0];
            F.vw[s][fe] = w;
        }
    }
    // corner circulation x_T of each coarse triangle (reading of the x fluxes of
    // Sec. 4.2): flux through the segment from the coarse vertex V to the circumcentre
    // W of the central fine triangle, with the flux vector fitted to the three fine
    // faces meeting at W: x_T = sum_g gam_g F[cen_g].
    std::vector<int32_t> cen(3 * C.T);
    std::vector<double> gam(3 * C.T);
    Lay Yc = layout_of(C), Yf = layout_of(F);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < C.T; ++t) {
        int64_t o = t / cne, e = t % cne, d, i, j;
        Yc.coords(e, d, i, j);
        int64_t tc = o == 0 ? F.nelem + Yf.elem(d, 2 * i + 1, 2 * j) : Yf.elem(d, 2 * i, 2 * j + 1);
        int64_t mids[3] = {C.mid[C.te[0][t] >> 1], C.mid[C.te[1][t] >> 1], C.mid[C.te[2][t] >> 1]};
        for (int c = 0; c < 3; ++c) {
            int64_t v = F.tn[c][tc];
            if (v != mids[0] && v != mids[1] && v != mids[2]) throw std::runtime_error("central fine triangle mismatch");
        }
        V3 V = C.cc[t], W = F.cc[tc], e1, e2;
        tangent_basis(V, e1, e2);
        double t1[3], t2[3];
        for (int g = 0; g < 3; ++g) {
            int64_t fe = F.te[g][tc] >> 1;
            V3 tg = unit(F.xyz[F.en[1][fe]] - F.xyz[F.en[0][fe]]);
            t1[g] = dot(tg, e1);
            t2[g] = dot(tg, e2);
            cen[3 * t + g] = int32_t(fe);
        }
        V3 seg = cross(W - V, V) * R;
        double s1 = dot(seg, e1), s2 = dot(seg, e2);
        double a11 = 0, a12 = 0, a22 = 0;
        for (int g = 0; g < 3; ++g) a11 += t1[g] * t1[g], a12 += t1[g] * t2[g], a22 += t2[g] * t2[g];
        double det = a11 * a22 - a12 * a12;
        double y1 = (a22 * s1 - a12 * s2) / det, y2 = (a11 * s2 - a12 * s1) / det;
        for (int g = 0; g < 3; ++g) gam[3 * t + g] = t1[g] * y1 + t2[g] * y2;
    }
    // restricted flux R_F = R_F0 + R'_F through coarse face e = (k -> l), as linear
    // coefficients on fine fluxes (per unit length) and fine divergences
    for (int s = 0; s < RF_F; ++s) C.rf_fi[s].assign(C.E, 0), C.rf_fw[s].assign(C.E, 0);
    for (int s = 0; s < RF_C; ++s) C.rf_ci[s].assign(C.E, 0), C.rf_cw[s].assign(C.E, 0);
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t e = 0; e < C.E; ++e) {
        int64_t k = C.en[0][e], l = C.en[1][e];
        int64_t tp = C.et[0][e], tq = C.et[1][e];
        int64_t p = third_node(C, tp, k, l), q = third_node(C, tq, k, l);
        int64_t m = C.mid[e];
        int64_t m_kp = C.mid[coarse_edge(C, k, p)], m_lp = C.mid[coarse_edge(C, l, p)];
        int64_t m_kq = C.mid[coarse_edge(C, k, q)], m_lq = C.mid[coarse_edge(C, l, q)];
        auto opposite = [&](int64_t a, int64_t b, int64_t c) {
            int64_t ed = coarse_edge(C, a, b);
            int64_t t1 = C.et[0][ed], t2 = C.et[1][ed];
            int64_t t = third_node(C, t1, a, b) == c ? t2 : t1;
            return third_node(C, t, a, b);
        };
        int64_t pp1 = opposite(l, p, k), qq1 = opposite(l, q, k);
        int64_t pp2 = opposite(k, p, l), qq2 = opposite(k, q, l);
        // F1 = (F_in^k - F_in^l)/2 over the six faces of the fine hexagon m
        int64_t kside[3] = {C.c2f[k], m_kp, m_kq}, lside[3] = {C.c2f[l], m_lp, m_lq};
        int nf = 0, found = 0;
        for (int r = 0; r < 6; ++r) {
            int64_t x = F.ring_n[r][m];
            int32_t code = F.ring_e[r][m];
            int64_t fe = code >> 1;
            double s = (code & 1) ? -1.0 : 1.0;           // +1: m is the fine edge's origin
            double w = 0;
            for (int a = 0; a < 3; ++a) {
                if (x == kside[a]) w = -0.5 * s * F.l_e[fe], ++found;
                if (x == lside[a]) w = 0.5 * s * F.l_e[fe], ++found;
            }
            C.rf_fi[nf][e] = int32_t(fe);
            C.rf_fw[nf][e] = w;
            ++nf;
        }
        if (found != 6) throw std::runtime_error("fine hexagon ring does not match R_F stencil");
        for (int g = 0; g < 3; ++g) {
            C.rf_fi[nf][e] = cen[3 * tp + g];
            C.rf_fw[nf][e] = -gam[3 * tp + g];
            ++nf;
            C.rf_fi[nf][e] = cen[3 * tq + g];
            C.rf_fw[nf][e] = gam[3 * tq + g];
            ++nf;
        }
        // divergence terms
        int64_t nodes[RF_C] = {C.c2f[k], C.c2f[l], C.c2f[pp1], C.c2f[qq1], C.c2f[pp2], C.c2f[qq2], m, m_kp, m_kq, m_lp, m_lq};
        double w[RF_C] = {0};
        auto slot = [&](int64_t fine) {
            for (int s = 0; s < RF_C; ++s)
                if (nodes[s] == fine) return s;
            throw std::runtime_error("R_F node slot");
        };
        auto Am = [&](int64_t x) { return F.A_i[x]; };
        w[slot(m)] += 0.5 * (overlap(k, m) - overlap(l, m));
        w[slot(m_lp)] += 0.5 * overlap(k, m_lp);
        w[slot(m_kp)] -= 0.5 * overlap(l, m_kp);
        w[slot(m_lq)] += 0.5 * overlap(k, m_lq);
        w[slot(m_kq)] -= 0.5 * overlap(l, m_kq);
        auto kml = [&](int64_t a, int64_t x, int64_t b, double f) {
            double c = f * overlap(a, x) * overlap(b, x) / Am(x);
            w[slot(C.c2f[a])] += c;
            w[slot(C.c2f[b])] -= c;
        };
        kml(k, m, l, 1.0);
        kml(k, m_kp, l, 1.0);
        kml(k, m_kq, l, 1.0);
        kml(k, m_lp, l, 1.0);
        kml(k, m_lq, l, 1.0);
        kml(k, m_lp, pp1, 0.5);
        kml(k, m_lq, qq1, 0.5);
        kml(pp2, m_kp, l, 0.5);
        kml(qq2, m_kq, l, 0.5);
        for (int s = 0; s < RF_C; ++s) {
            C.rf_ci[s][e] = int32_t(nodes[s]);
            C.rf_cw[s][e] = w[s];
        }
    }
}

}  // namespace

double nominal_spacing(int j, double radius) {
    double N = 10.0 * std::pow(4.0, j) + 2.0;
    return std::sqrt(2.0 * 4.0 * M_PI * radius * radius / (std::sqrt(3.0) * N));
}

void build_hierarchy(Hierarchy& H, int jmin, int jmax, int patch, double R, double omega) {
    if (jmin < 1 || jmax < jmin || jmax > 11) throw std::runtime_error("levels must satisfy 1 <= jmin <= jmax <= 11");
    if (patch < 1 || (patch & (patch - 1))) throw std::runtime_error("patch must be a power of two");
    H.jmin = jmin, H.jmax = jmax, H.radius = R, H.omega = omega;
    H.lv.assign(jmax + 1, HostLevel());
    // level 0: icosahedron.  Lozenge k (north) has U_k at its origin, lozenge 5+k
    // (south) L_k; the upper ring U_k sits at latitude atan(1/2), longitude 72k deg,
    // the lower ring L_k at -atan(1/2), 72k + 36 deg.
    std::vector<V3> pos(12);
    double la = std::atan(0.5);
    for (int k = 0; k < 5; ++k) {
        double lo = 2.0 * M_PI * k / 5.0, lo2 = 2.0 * M_PI * (k + 0.5) / 5.0;
        pos[k] = {std::cos(la) * std::cos(lo), std::cos(la) * std::sin(lo), std::sin(la)};
        pos[5 + k] = {std::cos(la) * std::cos(lo2), std::cos(la) * std::sin(lo2), -std::sin(la)};
    }
    pos[10] = {0, 0, 1};
    pos[11] = {0, 0, -1};
    HostLevel prev;
    init_level(prev, 0, 1);
    prev.xyz = pos;
    for (int j = 1; j <= jmax; ++j) {
        HostLevel cur;
        init_level(cur, j, j >= jmin ? patch : 1);
        Lay Yc = layout_of(prev), Yf = layout_of(cur);
        cur.xyz.resize(cur.N);
#pragma omp parallel for schedule(static)
        for (int64_t e = 0; e < cur.nelem; ++e) {
            int64_t d, I, Jj;
            Yf.coords(e, d, I, Jj);
            int64_t i = I / 2, jj = Jj / 2, a = I & 1, b = Jj & 1;
            if (!a && !b)
                cur.xyz[e] = prev.xyz[Yc.elem(d, i, jj)];
            else
                cur.xyz[e] = unit(prev.xyz[Yc.node(d, i, jj)] + prev.xyz[Yc.node(d, i + a, jj + b)]);
        }
        cur.xyz[cur.nelem] = prev.xyz[prev.nelem];
        cur.xyz[cur.nelem + 1] = prev.xyz[prev.nelem + 1];
        if (j >= jmin) {
            build_topology(cur);
            build_geometry(cur, R, omega);
            build_tiles(cur, patch);
            H.lv[j] = std::move(cur);
            prev.xyz = H.lv[j].xyz;
            prev.J = j, prev.n = H.lv[j].n, prev.p = H.lv[j].p, prev.np = H.lv[j].np, prev.nelem = H.lv[j].nelem, prev.N = H.lv[j].N;
        } else {
            prev = std::move(cur);
        }
    }
    for (int j = jmin + 1; j <= jmax; ++j) link_levels(H.lv[j - 1], H.lv[j], R);
    // Reading (Sec. 4.1 area conditions): from Jmax down, the clipped overlaps of each
    // fine hexagon are scaled to add up to its area exactly, and a coarse hexagon's
    // area is the sum of its fine pieces, A_k^j = A_k^{j+1} + sum_m A_km; both
    // conditions then hold in stored numbers (and with them R_h o div = div o R_F).
    for (int j = jmax; j > jmin; --j) {
        HostLevel &C = H.lv[j - 1], &F = H.lv[j];
        std::vector<double> A(C.N);
        for (int64_t k = 0; k < C.N; ++k) A[k] = F.A_i[C.c2f[k]];
        for (int64_t e = 0; e < C.E; ++e) {
            int64_t m = C.mid[e];
            double s = F.akm[0][m] + F.akm[1][m] + F.akm[2][m] + F.akm[3][m];
            double scale = F.A_i[m] / s;
            for (int q = 0; q < 4; ++q) F.akm[q][m] *= scale;
        }
        // accumulate in a fixed order (by coarse edge) for reproducibility
        std::vector<int32_t> f2c(F.N, -1);
        for (int64_t k = 0; k < C.N; ++k) f2c[C.c2f[k]] = int32_t(k);
        for (int64_t e = 0; e < C.E; ++e) {
            int64_t m = C.mid[e];
            for (int q = 0; q < 4; ++q) A[f2c[F.par[q][m]]] += F.akm[q][m];
        }
        C.A_i = A;
    }
    for (int j = jmin + 1; j <= jmax; ++j) pair_tables(H.lv[j - 1], H.lv[j], R);
}

// Every id a device gather reads lies in its array: a first bad entry is named in
// *what.  (-1 marks the documented absent entries: ring slots past a pentagon's
// fifth, parents of even nodes, M_k past its last member.)
bool validate_tables(const Hierarchy& H, std::string* what) {
    auto bad = [&](const char* table, int j, int64_t i, int64_t v) {
        if (what) *what = std::string(table) + " of level " + std::to_string(j) + " at " + std::to_string(i) +
                          " holds " + std::to_string(v);
        return false;
    };
    auto in = [](int64_t v, int64_t n) { return v >= 0 && v < n; };
    for (int j = H.jmin; j <= H.jmax; ++j) {
        const HostLevel& L = H.lv[j];
        const int64_t N = L.N, E = L.E, T = L.T;
        for (int k = 0; k < 2; ++k)
            for (int64_t e = 0; e < E; ++e) {
                if (!in(L.en[k][e], N)) return bad("en", j, e, L.en[k][e]);
                if (!in(L.et[k][e], T)) return bad("et", j, e, L.et[k][e]);
            }
        for (int k = 0; k < 3; ++k)
            for (int64_t t = 0; t < T; ++t) {
                if (!in(L.tn[k][t], N)) return bad("tn", j, t, L.tn[k][t]);
                if (!in(L.te[k][t] >> 1, E)) return bad("te", j, t, L.te[k][t]);
            }
        for (int64_t i = 0; i < N; ++i) {
            const int dg = L.deg[i];
            if (dg != 5 && dg != 6) return bad("deg", j, i, dg);
            for (int k = 0; k < 6; ++k) {
                const bool used = k < dg;
                if (used ? !in(L.ring_e[k][i] >> 1, E) : L.ring_e[k][i] != -1) return bad("ring_e", j, i, L.ring_e[k][i]);
                if (used ? !in(L.ring_n[k][i], N) : L.ring_n[k][i] != -1) return bad("ring_n", j, i, L.ring_n[k][i]);
                if (used ? !in(L.ring_t[k][i], T) : L.ring_t[k][i] != -1) return bad("ring_t", j, i, L.ring_t[k][i]);
            }
        }
        for (int k = 0; k < COR; ++k)
            for (int64_t e = 0; e < E; ++e)
                if (!in(L.cor_i[k][e], E)) return bad("cor_i", j, e, L.cor_i[k][e]);
        if (int64_t(L.tile_irr.size()) != L.npatch + 1) return bad("tile_irr", j, 0, int64_t(L.tile_irr.size()));
        if (!L.tile_halo.empty()) {
            const tile::Shape S{int(L.p)};
            const int HALO = S.halo();
            if (int64_t(L.tile_halo.size()) != L.npatch * HALO) return bad("tile_halo", j, 0, int64_t(L.tile_halo.size()));
            for (int64_t P = 0; P < L.npatch; ++P) {
                if (L.tile_irr[P]) continue;
                const int32_t* H = L.tile_halo.data() + P * HALO;
                for (int s = 0; s < HALO; ++s) {
                    const int64_t v = H[s];
                    const bool ok = s < S.off_edge(0) ? in(v, N) : s < S.off_tri(0) ? in(v >> 1, E) : in(v >> 2, T) && (v & 3) < 3;
                    if (!ok) return bad("tile_halo", j, P * HALO + s, v);
                }
            }
        }
        if (j > H.jmin) {
            const HostLevel& C = H.lv[j - 1];
            for (int64_t i = 0; i < N; ++i) {
                const bool odd = L.par[0][i] >= 0;
                for (int k = 0; k < 4; ++k)
                    if (odd ? !in(L.par[k][i], N) : L.par[k][i] != -1) return bad("par", j, i, L.par[k][i]);
            }
            for (int64_t e = 0; e < E; ++e) {
                const int kind = L.fe_kind[e];
                if (kind < 0 || kind > 2) return bad("fe_kind", j, e, kind);
                // a half names its coarse edge, an interior edge 3 t + c (coarse triangle t)
                if (!in(L.fe_ce[e], kind == 2 ? 3 * C.T : C.E)) return bad("fe_ce", j, e, L.fe_ce[e]);
                for (int k = 0; k < VST; ++k)
                    if (!in(L.vst[k][e], C.E)) return bad("vst", j, e, L.vst[k][e]);
            }
        }
        if (j < H.jmax) {
            const HostLevel& F = H.lv[j + 1];
            for (int64_t i = 0; i < N; ++i) {
                if (!in(L.c2f[i], F.N)) return bad("c2f", j, i, L.c2f[i]);
                for (int k = 0; k < 12; ++k)
                    if (L.mk_i[k][i] != -1 && !in(L.mk_i[k][i], F.N)) return bad("mk_i", j, i, L.mk_i[k][i]);
            }
            for (int64_t e = 0; e < E; ++e) {
                if (!in(L.mid[e], F.N)) return bad("mid", j, e, L.mid[e]);
                for (int k = 0; k < 2; ++k)
                    if (!in(L.half[k][e], F.E)) return bad("half", j, e, L.half[k][e]);
                for (int k = 0; k < RF_F; ++k)
                    if (!in(L.rf_fi[k][e], F.E)) return bad("rf_fi", j, e, L.rf_fi[k][e]);
                for (int k = 0; k < RF_C; ++k)
                    if (!in(L.rf_ci[k][e], F.N)) return bad("rf_ci", j, e, L.rf_ci[k][e]);
            }
        }
    }
    return true;
}

}  // namespace sww
