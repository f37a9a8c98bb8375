// Host-side grid, geometry and operator tables of the icosahedral nested grid.
//
// Layout (Sec. 5.2: ten lozenges, elements of one node + three edges + two
// triangles, regular patches): level j has n = 2^j elements per lozenge side.
// Element (d, i, j) of lozenge d lives at
//     elem = ((d*np + i/p)*np + j/p)*p*p + (i%p)*p + (j%p)
// (patch-major, np = n/p patches per side), so every p x p patch is contiguous.
// It owns node elem, edges o*nelem + elem (o = 0: to (i+1, j), 1: to (i+1, j+1),
// 2: to (i, j+1); velocity positive along that direction) and triangles
// t*nelem + elem (t = 0: (i,j),(i+1,j),(i+1,j+1); 1: (i,j),(i+1,j+1),(i,j+1)).
// The two poles are nodes nelem (north) and nelem + 1 (south).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace sww {

struct V3 {
    double x, y, z;
};

constexpr int RF_F = 12;   // flux terms of one restricted coarse flux
constexpr int RF_C = 11;   // divergence terms of one restricted coarse flux
constexpr int VST = 12;    // coarse stencil of one predicted fine edge
constexpr int COR = 10;    // edges of the TRiSK perpendicular reconstruction

struct HostLevel {
    int J = 0;
    int64_t n = 0, p = 0, np = 0, nelem = 0, N = 0, E = 0, T = 0, npatch = 0;
    std::vector<V3> xyz;
    // topology
    std::vector<int32_t> en[2];       // edge -> origin, end node
    std::vector<int32_t> et[2];       // edge -> left, right triangle (of origin -> end)
    std::vector<int32_t> tn[3];       // triangle -> nodes, counter-clockwise
    std::vector<int32_t> te[3];       // triangle -> side edge, encoded 2*e + (edge against side)
    std::vector<uint8_t> deg;         // node degree (5 or 6)
    std::vector<int32_t> ring_e[6];   // node -> edges CCW, encoded 2*e + (edge points into node)
    std::vector<int32_t> ring_n[6];   // node -> neighbours CCW
    std::vector<int32_t> ring_t[6];   // node -> triangle between ring edges k and k+1
    // geometry (m, m^2)
    std::vector<V3> cc;               // triangle circumcentres (hexagon vertices)
    std::vector<double> kite[3];      // area of triangle t inside the hexagon of tn[c][t]
    std::vector<double> A_v, A_i, A_kite, d_e, l_e, f_v, f_n;
    std::vector<double> ring_R[6];    // kite fraction of ring triangle k in its node's hexagon
    // TRiSK perpendicular reconstruction: du_e/dt|cor = sum_k cor_w F[cor_i] (q_e + q_k)/2
    std::vector<int32_t> cor_i[COR];
    std::vector<double> cor_w[COR];
    // fine side of the pair (j-1, j), for j > jmin
    std::vector<int32_t> par[4];      // odd node -> prediction parents (fine ids of coarse nodes)
    std::vector<double> ptw[4];       // s~_km = A_km / A_m
    std::vector<double> akm[4];       // normalised overlap areas
    std::vector<int8_t> fe_kind;      // fine edge: 0/1 first/second half of a coarse edge, 2 interior
    std::vector<int32_t> fe_ce;       // coarse edge (halves) or coarse triangle (interior)
    std::vector<int32_t> vst[VST];    // coarse stencil (edge ids) of each fine edge
    std::vector<double> vw[VST];      // prediction weights
    // coarse side of the pair (j, j+1), for j < jmax (ids on level j+1 where noted)
    std::vector<int32_t> c2f;         // node -> fine node id at the same place
    std::vector<int32_t> mid;         // edge -> fine node at its midpoint
    std::vector<int32_t> half[2];     // edge -> fine half edges (same direction as the edge)
    std::vector<int32_t> mk_i[12];    // node -> odd fine nodes of M_k (-1 padded)
    std::vector<double> mk_w[12];     // s_km = A_km / A_k
    std::vector<int32_t> rf_fi[RF_F]; // restricted flux: fine edge ids
    std::vector<double> rf_fw[RF_F];  //                  weights on fine F (per unit length)
    std::vector<int32_t> rf_ci[RF_C]; //                  fine node ids
    std::vector<double> rf_cw[RF_C];  //                  weights on fine divergences
    // tiles of the structured trend kernel (tile.h), for patch sides 4, 8 and 16
    std::vector<int32_t> tile_halo;   // [npatch * halo]: halo ids of each patch (empty without tiles)
    std::vector<uint8_t> tile_irr;    // [npatch + 1]: 1 where the tile is not regular (the last: poles)
};

struct Hierarchy {
    int jmin = 0, jmax = 0;
    double radius = 0, omega = 0;
    std::vector<HostLevel> lv;        // index j (levels < jmin left empty)
};

// Build levels jmin..jmax with patch side `patch`.  Throws std::runtime_error on
// invalid arguments or inconsistent geometry.
void build_hierarchy(Hierarchy& H, int jmin, int jmax, int patch, double radius, double omega);

// Table 1 mean spacing sqrt(2 * 4 pi R^2 / (sqrt(3) N_j)).
double nominal_spacing(int j, double radius);

// Bounds of every index table the device gathers through (false and a message
// naming the first bad entry otherwise).
bool validate_tables(const Hierarchy& H, std::string* what);

}  // namespace sww
