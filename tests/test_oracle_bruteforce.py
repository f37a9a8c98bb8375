"""Brute-force pins of the oracle's TRiSK operators (Sec. 3.1) on the level-2 grid
(N = 162 nodes, E = 480 edges, T = 320 triangles).

Each operator is assembled here as a dense matrix from a geometry computed
independently of oracle/grid.py, then compared with the oracle's operator applied
to the unit vectors.  Only the node positions come from the oracle (they are
pinned by Table 1 and scipy's hull in test_oracle_grid); everything else is
rebuilt:

  * triangles and their counter-clockwise orientation: scipy ConvexHull;
  * hexagon vertices (triangle circumcentres) and each cell's counter-clockwise
    vertex order: scipy SphericalVoronoi;
  * kite areas A_{i,v}: the intersection of Voronoi cell i with Delaunay triangle
    v, clipped here by great circles, area by the angle excess (Girard's
    theorem) -- the oracle splits kites into two triangles and uses the
    tangent half-angle formula instead;
  * cell areas A_i = sum of the cell's kites (checked against scipy's own
    Voronoi areas), dual areas A_v = the triangle's angle excess;
  * lengths d_e (nodes) and l_e (circumcentres of the two triangles of e) as arcs.

The matrices (l_e, d_e, A per edge and cell; the weights of the Coriolis
reconstruction from the kite fractions in the Voronoi vertex order) are then
those of the operators' definitions:
  div     D[i, e] = n_{e,i} l_e / A_i
  grad    G[e, end] = 1/d_e, G[e, origin] = -1/d_e
  curl    C[v, e] = t_{e,v} d_e / A_v
  K       K[i, e] = l_e d_e / (4 A_i)   (on u_e^2)
  h_v     H[v, i] = A_{i,v} / A_v
  q F^perp: from cell i with faces e_1..e_D counter-clockwise and kite fractions
          R_m of the vertex between e_m and e_{m+1}, splitting each face's outflow
          evenly between its two kites and giving kite m the share R_m of the net
          outflow, the flux across the half face from i to the midpoint of e_k is
          sum_{k' != k} (1/2 - sum_{m=k}^{k'-1} R_m) phi_{k'} (phi = outward face
          fluxes n F l); its tangential component on e (left of origin -> end) is
          the origin cell's share minus the end cell's, divided by d_e, with the
          energy-conserving factor (q_e + q_e')/2 on each (e, e') term.

A plausible slip in the oracle -- equal thirds in place of the kite weights of
h_v, a dropped sign of a face, l_e and d_e exchanged, a kite fraction taken from
the wrong vertex -- changes one of these matrices by far more than the
bar, as the mutation checks at the end show.  The bar is 1e-13 relative for
lengths and 1e-12 for what depends on areas (the angle excess of a small polygon
keeps about 13 digits)."""
import numpy as np
import pytest
from scipy.spatial import ConvexHull, SphericalVoronoi, cKDTree

from oracle import grid, trisk

R = 6.371e6
OMEGA = 7.292e-5
TOL = 1e-13
# area-dependent quantities: the angle excess of a small polygon loses about three
# digits against its angles (sum of angles ~ (n - 2) pi, excess ~ 1e-2 sr here)
ATOL = 1e-12


def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def _arc(a, b):
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), np.sum(a * b, axis=-1))


def _excess(P):
    """Area of a convex spherical polygon P[n, 3] (unit sphere, any orientation) by
    Girard's theorem: the sum of its interior angles minus (n - 2) pi."""
    n = len(P)
    s = 0.0
    for k in range(n):
        a, b, c = P[k - 1], P[k], P[(k + 1) % n]
        ta = _unit(a - np.dot(a, b) * b)      # tangent at b towards a
        tc = _unit(c - np.dot(c, b) * b)      # tangent at b towards c
        s += np.arctan2(np.linalg.norm(np.cross(ta, tc)), np.dot(ta, tc))
    return s - (n - 2) * np.pi


def _clip(P, a, b, inside):
    """Part of the convex polygon P on the side of the great circle through a, b
    that holds the point `inside` (Sutherland-Hodgman on the sphere)."""
    nrm = np.cross(a, b)
    if np.dot(nrm, inside) < 0:
        nrm = -nrm
    out = []
    n = len(P)
    for k in range(n):
        s, e = P[k - 1], P[k]
        ds, de = np.dot(nrm, s), np.dot(nrm, e)
        if (ds >= 0) != (de >= 0):
            out.append(_unit(s + ds / (ds - de) * (e - s)))
        if de >= 0:
            out.append(e)
    return np.array(out)


class Brute:
    """The level-2 geometry and operator matrices, built from scipy's hull and
    Voronoi diagram over the oracle's node positions and the oracle's edge list
    (whose order and orientation index the matrices)."""

    def __init__(self, L):
        x = L.xyz
        N = len(x)
        hull = ConvexHull(x)
        tri = hull.simplices.copy()
        # counter-clockwise seen from outside
        flip = np.einsum("ij,ij->i", np.cross(x[tri[:, 1]] - x[tri[:, 0]], x[tri[:, 2]] - x[tri[:, 0]]),
                         x[tri].sum(axis=1)) < 0
        tri[flip] = tri[flip][:, ::-1]
        sv = SphericalVoronoi(x, radius=1.0)
        sv.sort_vertices_of_regions()
        # counter-clockwise seen from outside (scipy's sorted order may run either way)
        regions = []
        for i, reg in enumerate(sv.regions):
            reg = list(reg)
            P = sv.vertices[reg]
            turn = sum(np.dot(np.cross(P[k] - x[i], P[(k + 1) % len(P)] - x[i]), x[i]) for k in range(len(P)))
            regions.append(reg[::-1] if turn < 0 else reg)
        # circumcentre of each hull triangle: the Voronoi vertex nearest its centroid
        vt = cKDTree(sv.vertices)
        d, vid = vt.query(_unit(x[tri].mean(axis=1)))
        cc = sv.vertices[vid]
        # map the oracle's triangles to hull triangles by their node sets
        key = {tuple(sorted(t)): k for k, t in enumerate(tri)}
        self.t_of = np.array([key[tuple(sorted(t))] for t in L.tri])
        E = len(L.edges)
        self.N, self.E, self.T = N, E, len(tri)
        self.tri, self.cc = tri, cc
        # kites: Voronoi cell i clipped by the three sides of each triangle holding i
        kite = {}
        for t, (a, b, c) in enumerate(tri):
            for i in (a, b, c):
                P = sv.vertices[regions[i]]
                inside = _unit(x[a] + x[b] + x[c])
                for p, q in ((a, b), (b, c), (c, a)):
                    P = _clip(P, x[p], x[q], inside)
                kite[(i, t)] = _excess(P) * R * R
        self.kite = kite
        self.A_v = np.array([_excess(x[t]) * R * R for t in tri])
        self.A_i = np.zeros(N)
        for (i, t), k in kite.items():
            self.A_i[i] += k
        self.A_scipy = sv.calculate_areas() * R * R
        # edges: the oracle's list and orientation; their two triangles from the hull
        pair_tris = {}
        for t, (a, b, c) in enumerate(tri):
            for p, q in ((a, b), (b, c), (c, a)):
                pair_tris.setdefault((min(p, q), max(p, q)), []).append(t)
        self.edges = L.edges
        self.d_e = _arc(x[L.edges[:, 0]], x[L.edges[:, 1]]) * R
        self.l_e = np.empty(E)
        self.etris = np.empty((E, 2), dtype=np.int64)
        for e, (a, b) in enumerate(L.edges):
            t0, t1 = pair_tris[(min(a, b), max(a, b))]
            self.etris[e] = (t0, t1)
            self.l_e[e] = _arc(cc[t0], cc[t1]) * R
        self.eid = {(min(a, b), max(a, b)): e for e, (a, b) in enumerate(L.edges)}
        # each cell's faces in the Voronoi vertex order: the face between vertices
        # r_k and r_{k+1} is shared with the neighbour j whose triangle pair is
        # (t(r_k), t(r_{k+1})); kite fraction of vertex r_{k+1} sits between faces k and k+1
        vert_tri = {int(v): t for t, v in enumerate(vid)}
        self.faces, self.fracs = [], []
        for i in range(N):
            reg = regions[i]
            D = len(reg)
            faces, fr = [], []
            for k in range(D):
                ta, tb = vert_tri[reg[k]], vert_tri[reg[(k + 1) % D]]
                common = set(tri[ta]) & set(tri[tb])
                j = (common - {i}).pop()
                faces.append(self.eid[(min(i, j), max(i, j))])
            for k in range(D):
                fr.append(kite[(i, vert_tri[reg[(k + 1) % D]])] / self.A_i[i])
            self.faces.append(faces)
            self.fracs.append(fr)

    def n(self, e, i):
        return 1.0 if self.edges[e, 0] == i else -1.0

    def div(self):
        D = np.zeros((self.N, self.E))
        for e, (a, b) in enumerate(self.edges):
            D[a, e] += self.l_e[e] / self.A_i[a]
            D[b, e] -= self.l_e[e] / self.A_i[b]
        return D

    def grad(self):
        G = np.zeros((self.E, self.N))
        for e, (a, b) in enumerate(self.edges):
            G[e, b] += 1.0 / self.d_e[e]
            G[e, a] -= 1.0 / self.d_e[e]
        return G

    def curl(self):
        C = np.zeros((self.T, self.E))
        for t, (a, b, c) in enumerate(self.tri):
            for p, q in ((a, b), (b, c), (c, a)):
                e = self.eid[(min(p, q), max(p, q))]
                s = 1.0 if self.edges[e, 0] == p else -1.0
                C[t, e] += s * self.d_e[e] / self.A_v[t]
        return C

    def ke(self):
        K = np.zeros((self.N, self.E))
        for e, (a, b) in enumerate(self.edges):
            w = 0.25 * self.l_e[e] * self.d_e[e]
            K[a, e] += w / self.A_i[a]
            K[b, e] += w / self.A_i[b]
        return K

    def hv(self):
        H = np.zeros((self.T, self.N))
        for (i, t), k in self.kite.items():
            H[t, i] = k / self.A_v[t]
        return H

    def coriolis(self, F, q):
        """q F^perp at every edge, energy-conserving form, from the cells' faces."""
        qe = 0.5 * (q[self.etris[:, 0]] + q[self.etris[:, 1]])
        out = np.zeros(self.E)
        for i in range(self.N):
            faces, fr = self.faces[i], self.fracs[i]
            D = len(faces)
            for k in range(D):
                e = faces[k]
                psi, csum = 0.0, 0.0
                for o in range(1, D):
                    csum += fr[(k + o - 1) % D]
                    e2 = faces[(k + o) % D]
                    phi = self.n(e2, i) * F[e2] * self.l_e[e2]
                    psi += (0.5 - csum) * phi * 0.5 * (qe[e] + qe[e2])
                out[e] += self.n(e, i) * psi
        return out / self.d_e


@pytest.fixture(scope="module")
def pair():
    L = grid.Hierarchy(2, 2, radius=R, omega=OMEGA).levels[2]
    assert (L.N, L.E, L.T) == (162, 480, 320)
    return L, Brute(L)


def _apply(op, n):
    return np.stack([op(np.eye(n)[k]) for k in range(n)], axis=1)


def _close(A, B, tol=TOL):
    return np.abs(A - B).max() <= tol * np.abs(B).max()


def test_independent_geometry_is_consistent(pair):
    L, B = pair
    assert np.abs(B.A_i / B.A_scipy - 1).max() < 1e-12              # kites tile scipy's Voronoi cells
    assert abs(B.A_i.sum() / (4 * np.pi * R * R) - 1) < 1e-13          # angle excess: ~1e-16 rad per angle
    kv = np.zeros(B.T)
    for (i, t), k in B.kite.items():
        kv[t] += k
    assert np.abs(kv / B.A_v - 1).max() < 1e-13                     # kites tile the triangles


def test_geometry_matches_oracle(pair):
    L, B = pair
    assert np.abs(L.A_i / B.A_i - 1).max() < ATOL
    assert np.abs(L.A_v / B.A_v[B.t_of] - 1).max() < ATOL
    assert np.abs(L.d_e / B.d_e - 1).max() < TOL
    assert np.abs(L.l_e / B.l_e - 1).max() < TOL


def test_divergence_matrix(pair):
    L, B = pair
    assert _close(_apply(lambda F: trisk.divergence(L, F), L.E), B.div(), ATOL)


def test_gradient_matrix(pair):
    L, B = pair
    assert _close(_apply(lambda f: trisk.gradient(L, f), L.N), B.grad())


def test_curl_matrix(pair):
    L, B = pair
    C = B.curl()[B.t_of]
    assert _close(_apply(lambda u: trisk.vorticity(L, u), L.E), C, ATOL)


def test_kinetic_energy_matrix(pair):
    L, B = pair
    assert _close(_apply(lambda u: trisk.kinetic_energy(L, np.sqrt(np.abs(u))), L.E), B.ke(), ATOL)


def test_kite_weighted_depth_matrix(pair):
    """h_v = sum_i A_{i,v} h_i / A_v, as a matrix on the node depths (H = 0)."""
    L, B = pair
    H = B.hv()[B.t_of]
    assert _close(_apply(lambda h: trisk.depth_at_triangles(L, h, 0.0), L.N), H, ATOL)


def test_potential_vorticity(pair):
    L, B = pair
    rng = np.random.default_rng(7)
    dh, u = rng.standard_normal(L.N) * 50.0, rng.standard_normal(L.E) * 10.0
    H0 = 1.0e4
    f_v = 2.0 * OMEGA * B.cc[:, 2]
    q = (B.curl() @ u + f_v) / (B.hv() @ (H0 + dh))
    assert _close(trisk.potential_vorticity(L, dh, u, H0), q[B.t_of], ATOL)


def test_coriolis_reconstruction(pair):
    """q F^perp on random fluxes and potential vorticities, and its matrix at q = 1."""
    L, B = pair
    rng = np.random.default_rng(8)
    F = rng.standard_normal(L.E)
    q_ora = rng.standard_normal(L.T)
    q_hull = np.empty(L.T)
    q_hull[B.t_of] = q_ora
    assert _close(trisk.coriolis_tendency(L, F, q_ora), B.coriolis(F, q_hull), ATOL)
    W = _apply(lambda f: trisk.coriolis_tendency(L, f, np.ones(L.T)), L.E)
    Wb = _apply(lambda f: B.coriolis(f, np.ones(L.T)), L.E)
    assert _close(W, Wb, ATOL)


def test_mutations_are_caught(pair):
    """Plausible slips change the matrices far beyond the bar."""
    L, B = pair
    H = B.hv()[B.t_of]
    thirds = np.zeros_like(H)
    for v, t in enumerate(L.tri):
        thirds[v, t] = 1.0 / 3.0
    assert np.abs(thirds - H).max() > 1e-3 * np.abs(H).max()          # equal thirds for h_v
    D = B.div()
    swapped = D * (B.d_e / B.l_e)[None, :]
    assert np.abs(swapped - D).max() > 1e-3 * np.abs(D).max()         # d_e in place of l_e
    rng = np.random.default_rng(9)
    F = rng.standard_normal(L.E)
    ref = B.coriolis(F, np.ones(L.T))
    saved = [list(f) for f in B.fracs]
    try:
        for f in B.fracs:
            f.append(f.pop(0))                                          # fraction of the wrong vertex
        shifted = B.coriolis(F, np.ones(L.T))
    finally:
        B.fracs = saved
    assert np.abs(shifted - ref).max() > 1e-3 * np.abs(ref).max()
