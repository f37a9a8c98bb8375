"""Pins for the oracle's grid and geometry (Sec. 2.2, Table 1, Sec. 4.1).

Checked against things the oracle does not compute itself: the numbers of
Table 1, the sphere's area, scipy's independent spherical Voronoi tessellation
and convex hull, and the area conditions of Sec. 4.1."""
import math
import os

import numpy as np
import pytest
from scipy.spatial import ConvexHull, SphericalVoronoi

from oracle import grid

HERE = os.path.dirname(__file__)


def table1():
    rows = []
    for line in open(os.path.join(HERE, "golden", "table1.txt")):
        if line.startswith("#") or not line.strip():
            continue
        J, N, dof, dx, T = line.split()
        rows.append((int(J), int(N), int(dof), float(dx), int(T)))
    return rows


def test_table1_counts_built_levels():
    """N and d.o.f. (= nodes + edges) of the built grids match Table 1 exactly."""
    H = grid.Hierarchy(3, 6, radius=6.37122e6)
    by_j = {r[0]: r for r in table1()}
    for J in range(3, 7):
        L = H.levels[J]
        _, N, dof, dx, _ = by_j[J]
        assert L.N == N
        assert L.N + L.E == dof
        assert L.E == 30 * 4 ** J and L.T == 20 * 4 ** J
        # mean arc length of the built grid within 3% of the tabulated spacing
        assert abs(L.d_e.mean() / 1e3 / dx - 1) < 0.03


def test_table1_formulas_all_rows():
    """Every row: N = 10*4^J+2, dof = N + 30*4^J, dx within 0.2% of the
    mean-spacing formula (plus half a unit of the last printed digit)."""
    for J, N, dof, dx, T in table1():
        assert N == 10 * 4 ** J + 2
        assert dof == N + 30 * 4 ** J
        assert abs(grid.nominal_spacing(J, 6.37122e6) / 1e3 - dx) < 0.05 + 2e-3 * dx


def test_areas_tile_sphere(hier25):
    for J, L in hier25.levels.items():
        S = 4 * math.pi * L.radius ** 2
        assert abs(L.A_kite.sum() / S - 1) < 1e-13
        assert abs(L.A_v.sum() / S - 1) < 1e-13
        assert abs(L.A_i.sum() / S - 1) < 1e-13
        assert (L.kite > 0).all()


def test_nesting_and_topology(hier25):
    for J in range(3, 6):
        C, F = hier25.levels[J - 1], hier25.levels[J]
        assert np.array_equal(F.xyz[: C.N], C.xyz)             # even nodes keep their place
        a, b = C.edges[hier25.pedge[J], 0], C.edges[hier25.pedge[J], 1]
        mid = grid.normalize(C.xyz[a] + C.xyz[b])
        assert np.abs(F.xyz[hier25.odd[J]] - mid).max() < 1e-15
    L = hier25.levels[3]
    assert set(np.unique(L.deg)) == {5, 6} and (L.deg == 5).sum() == 12


def test_triangles_match_convex_hull():
    """The triangles are the convex hull facets of the nodes (Delaunay on the sphere)."""
    L = grid.Hierarchy(3, 3).levels[3]
    hull = ConvexHull(L.xyz)
    ours = {tuple(sorted(t)) for t in L.tri.tolist()}
    theirs = {tuple(sorted(t)) for t in hull.simplices.tolist()}
    assert ours == theirs


@pytest.mark.parametrize("J", [2, 3, 4])
def test_voronoi_cells_match_scipy(J):
    """Hexagon areas, vertices and face lengths agree with scipy's spherical
    Voronoi tessellation of the same nodes."""
    L = grid.Hierarchy(J, J).levels[J]
    sv = SphericalVoronoi(L.xyz, radius=1.0, center=np.zeros(3))
    sv.sort_vertices_of_regions()
    areas = sv.calculate_areas() * L.radius ** 2
    assert np.abs(areas / L.A_kite - 1).max() < 1e-10
    for i in range(0, L.N, max(1, L.N // 50)):
        verts = sv.vertices[sv.regions[i]]
        ours = L.hexagon(i)
        d = np.linalg.norm(verts[:, None, :] - ours[None, :, :], axis=2)
        assert d.min(axis=1).max() < 1e-12
    # face length = arc between the two vertices shared by adjacent regions
    regs = [set(r) for r in sv.regions]
    for e in range(0, L.E, max(1, L.E // 60)):
        a, b = L.edges[e]
        shared = sorted(regs[a] & regs[b])
        assert len(shared) == 2
        arc = grid.arc_length(sv.vertices[shared[0]], sv.vertices[shared[1]]) * L.radius
        assert abs(arc / L.l_e[e] - 1) < 1e-10


def test_overlap_area_conditions(hier25):
    """Sec. 4.1: the coarse hexagons cover every fine hexagon, and each coarse
    hexagon is tiled by its own fine hexagon plus the pieces A_km -- both checked
    with the clipped areas against independently computed kite areas."""
    for J in range(3, 6):
        C, F = hier25.levels[J - 1], hier25.levels[J]
        odd = hier25.odd[J]
        Akm = hier25.Akm_clip[J]
        # tolerance grows with 4^J: node positions are rounded off the sphere
        tol = 2e-14 * 4 ** (J - 2)
        assert np.abs(Akm.sum(axis=1) / F.A_kite[odd] - 1).max() < tol
        S = np.zeros(C.N)
        np.add.at(S, hier25.K[J].ravel(), Akm.ravel())
        assert np.abs((C.A_kite - S) / F.A_kite[: C.N] - 1).max() < tol
        # the two main parents hold most of each fine hexagon, the slivers little
        frac = hier25.Akm[J] / hier25.Am[J][:, None]
        assert frac[:, :2].min() > 0.4 and frac[:, 2:].max() < 0.1
        # stored (normalised) areas satisfy both conditions to rounding
        assert np.abs(hier25.Akm[J].sum(axis=1) / F.A_i[odd] - 1).max() < 1e-15 * 8
        S = F.A_i[: C.N].copy()
        np.add.at(S, hier25.K[J].ravel(), hier25.Akm[J].ravel())
        assert np.abs(S / C.A_i - 1).max() < 1e-15 * 8


def test_clip_matches_known_area():
    """Spherical polygon clipping against a case with a closed form: an octant
    triangle clipped by the hemisphere z >= 0 keeps its area; a lune quarter."""
    e = np.eye(3)
    P = np.array([[e[0], e[1], e[2]]])
    full = grid.polygon_area(P, np.array([3]))[0]
    assert abs(full - math.pi / 2) < 1e-14
    # clip by the half-space x >= y: the plane through z and (1,1,0) halves the octant
    n = np.cross(e[2], np.array([1.0, 1.0, 0.0]) / math.sqrt(2))
    n = -n                                          # keep x >= y
    Q, cnt = grid.clip_convex(P.copy(), np.array([3]), n[None, None, :], e[2][None, None, :])
    assert abs(grid.polygon_area(Q, cnt)[0] - math.pi / 4) < 1e-14
