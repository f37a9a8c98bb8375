// Tiles of the structured trend kernel (host table builder and device kernels).
//
// A tile is one p x p patch of elements (Sec. 5.2, Fig. 5) and the neighbourhood
// that the trend of its own points reads, in the local lattice coordinates (a, b)
// of the patch's lozenge: a along i, b along j, the patch's own elements at
// a, b in [0, p).  Away from the twelve pentagons the lattice continues across
// lozenge seams, so a tile is regular there and every neighbour is found at a
// constant offset:
//   nodes       (a, b), a and b in [-1, p+1]
//   edges o     from node (a, b) to (a + DI[o], b + DJ[o]) (o = 0: +a, 1: +a+b, 2: +b);
//               o = 0 on a in [-1, p], b in [-1, p+1]; o = 1 on a, b in [-1, p];
//               o = 2 on a in [-1, p+1], b in [-1, p]
//   triangles   t0 = (a,b), (a+1,b), (a+1,b+1) and t1 = (a,b), (a+1,b+1), (a,b+1),
//               a and b in [-1, p]
// The interior is the patch's own elements, whose ids follow from the layout.  The
// rest (the halo) is listed per patch in a table of HALO entries, block by block
// (nodes, edges o = 0, 1, 2, triangles t0, t1), each block row-major over its
// range without the interior.  Node entries are ids; edge entries 2 e + r with r =
// 1 when global edge e runs against the local direction; triangle entries 4 t + s
// with the triangle's local vertex c at its global position (c + s) mod 3.
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define SWW_HD __host__ __device__
#else
#define SWW_HD
#endif

namespace sww {
namespace tile {

// positions of a block: a in [-1, A], b in [-1, B], without the interior [0, p)^2
SWW_HD constexpr int count(int p, int A, int B) { return (B + 2) + p * (B - p + 2) + (A - p + 1) * (B + 2); }

// halo slot of position (a, b) in its block (-1 for the interior)
SWW_HD constexpr int slot(int p, int B, int a, int b) {
    return a < 0 ? b + 1
                 : a < p ? ((b >= 0 && b < p) ? -1 : (B + 2) + a * (B - p + 2) + (b < 0 ? 0 : b - p + 1))
                         : (B + 2) + p * (B - p + 2) + (a - p) * (B + 2) + (b + 1);
}

// position of halo slot s of a block
SWW_HD inline void pos(int p, int B, int s, int& a, int& b) {
    if (s < B + 2) {
        a = -1, b = s - 1;
        return;
    }
    s -= B + 2;
    const int hw = B - p + 2;
    if (s < p * hw) {
        a = s / hw;
        const int c = s % hw;
        b = c == 0 ? -1 : p - 1 + c;
        return;
    }
    s -= p * hw;
    a = p + s / (B + 2), b = s % (B + 2) - 1;
}

// block ranges (A, B) and offsets of a tile of side p
struct Shape {
    int p;
    SWW_HD constexpr int nA() const { return p + 1; }
    SWW_HD constexpr int nodes() const { return count(p, p + 1, p + 1); }
    // edges o: A = p + (o == 2), B = p + (o == 0)
    SWW_HD constexpr int eA(int o) const { return p + (o == 2 ? 1 : 0); }
    SWW_HD constexpr int eB(int o) const { return p + (o == 0 ? 1 : 0); }
    SWW_HD constexpr int edges(int o) const { return count(p, eA(o), eB(o)); }
    SWW_HD constexpr int tris() const { return count(p, p, p); }
    SWW_HD constexpr int off_edge(int o) const {
        return nodes() + (o > 0 ? edges(0) : 0) + (o > 1 ? edges(1) : 0);
    }
    SWW_HD constexpr int off_tri(int t) const { return off_edge(2) + edges(2) + (t > 0 ? tris() : 0); }
    SWW_HD constexpr int halo() const { return off_tri(1) + tris(); }
};

// lattice steps of the six ring directions m of a node, counter-clockwise from +a:
// (1,0), (1,1), (0,1), (-1,0), (-1,-1), (0,-1)
SWW_HD constexpr int da(int m) { return m < 2 ? 1 : (m == 2 || m == 5) ? 0 : -1; }
SWW_HD constexpr int db(int m) { return (m == 0 || m == 3) ? 0 : m < 3 ? 1 : -1; }

}  // namespace tile
}  // namespace sww
