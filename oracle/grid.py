"""Oracle: icosahedral nested grid and its spherical geometry.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows Sec. 2.2 (nested grids: icosahedron, edge bisection, projection onto
the sphere; Fig. 1), Table 1 (N = 10*4^J + 2 nodes), Sec. 3.1 (staggered C-grid:
height on the nodes of the triangular grid = centres of hexagons, normal
velocity at the midpoints of the triangle edges, oriented along the edges),
and Sec. 4.1 (areas are spherical polygons, lengths are arc lengths; hexagon
intersection areas A_km by clipping spherical polygons, great-circle
intersections).

Construction here is deliberately unlike a lozenge/patch layout: each level is
a flat list of triangles obtained by splitting every triangle of the coarser
level in four, with edge midpoints memoised in a dictionary.  Node ids are
nested: the nodes of level j keep their ids at level j+1 ("even" nodes) and the
new midpoint nodes ("odd" nodes, the set M(j)) are appended.

Reading (hexagon vertices): the hexagon (Voronoi cell) vertices are the
spherical circumcentres of the triangles, which TRiSK's orthogonality needs;
the barycentre of Sec. 4.1 is only the fan point used to split polygons.
Reading (areas): the hexagon area A_i is the sum of its kite areas and the dual
triangle area A_v is the sum of the three kites inside it, so that both kite
partitions hold exactly in stored numbers.
"""
from __future__ import annotations

import math
import numpy as np


# ----------------------------------------------------------------------------- spherical helpers

def normalize(v):
    v = np.asarray(v, dtype=np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        return v / np.linalg.norm(v, axis=-1, keepdims=True)


def arc_length(a, b):
    """Great-circle angle between unit vectors (radians)."""
    # |a x b| = |a x (b - a)|: the difference keeps full relative precision for short arcs
    return np.arctan2(np.linalg.norm(np.cross(a, b - a), axis=-1), np.sum(a * b, axis=-1))


def triangle_area(a, b, c):
    """Signed area of the spherical triangle (a, b, c) on the unit sphere
    (positive when counter-clockwise seen from outside), from
    tan(E/2) = a.(b x c) / (1 + a.b + b.c + c.a), with the triple product
    evaluated as a.((b - a) x (c - a)) to keep full relative precision for small
    triangles."""
    num = np.sum(a * np.cross(b - a, c - a), axis=-1)
    den = 1.0 + np.sum(a * b, axis=-1) + np.sum(b * c, axis=-1) + np.sum(c * a, axis=-1)
    return 2.0 * np.arctan2(num, den)


def circumcentre(a, b, c):
    """Spherical circumcentre of triangle (a, b, c): the unit normal of the plane
    through the three points, on the same side as the triangle."""
    n = np.cross(b - a, c - a)
    n = normalize(n)
    s = np.sign(np.sum(n * (a + b + c), axis=-1))
    return n * s[..., None]


def polygon_area(P, cnt):
    """Area of convex spherical polygons P[B, V, 3] with cnt[B] vertices (fan from vertex 0)."""
    B, V, _ = P.shape
    area = np.zeros(B)
    for k in range(1, V - 1):
        ok = (k + 1) < cnt
        if not np.any(ok):
            continue
        t = triangle_area(P[:, 0], P[:, k], P[:, k + 1])
        area += np.where(ok, t, 0.0)
    return area


def clip_convex(P, cnt, normals, anchors):
    """Sutherland-Hodgman clipping of convex spherical polygons P[B, V, 3] (cnt[B]
    vertices) by the great-circle half-spaces {x : n.(x - a) >= 0} for each
    normal n in normals[B, H, 3] and point a on the circle in anchors[B, H, 3]
    (n.a = 0, so this is n.x >= 0 evaluated without cancellation).  Returns the
    clipped polygons (as arrays, counts)."""
    B = P.shape[0]
    for h in range(normals.shape[1]):
        n = normals[:, h]
        V = P.shape[1]
        out = np.zeros((B, V + 1, 3))              # a half-space adds at most one vertex
        ocnt = np.zeros(B, dtype=np.int64)
        d = np.einsum("bvk,bk->bv", P - anchors[:, h][:, None, :], n)
        rows = np.arange(B)
        for k in range(V):
            valid = k < cnt
            kp = np.where(k == 0, cnt - 1, k - 1)
            kp = np.where(valid, kp, 0)
            s, e = P[rows, kp], P[:, k]
            ds, de = d[rows, kp], d[:, k]
            s_in, e_in = ds >= 0.0, de >= 0.0
            denom = ds - de
            denom = np.where(denom == 0.0, 1.0, denom)
            x = normalize((ds[:, None] * e - de[:, None] * s) / denom[:, None] + 0.0)
            # first emitted point: the intersection when the edge crosses the circle,
            # else the end point when it is inside
            cross = valid & (s_in != e_in)
            emit_e = valid & e_in
            p1 = np.where(cross[:, None], x, e)
            has1 = cross | emit_e
            slot = np.minimum(ocnt, V)
            out[rows, slot] = np.where(has1[:, None], p1, out[rows, slot])
            ocnt = ocnt + has1
            has2 = valid & (~s_in) & e_in          # crossing into the half-space: add e too
            slot = np.minimum(ocnt, V)
            out[rows, slot] = np.where(has2[:, None], e, out[rows, slot])
            ocnt = ocnt + has2
        P, cnt = out, ocnt
    return P, cnt


def _local_basis(x):
    """Tangent basis (e1, e2) at unit vectors x with e1 x e2 = x."""
    ref = np.where(np.abs(x[..., 2:3]) < 0.9, np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0]))
    e1 = normalize(np.cross(ref, x))
    e2 = np.cross(x, e1)
    return e1, e2


# ----------------------------------------------------------------------------- the icosahedron

def icosahedron():
    """Level 0 (Fig. 1): the 12 vertices of an icosahedron on the unit sphere --
    the two poles and two rings of five at latitude +-atan(1/2) -- and its 20
    triangular faces, counter-clockwise seen from outside."""
    lat = math.atan(0.5)
    pts = [(0.0, 0.0, 1.0)]
    for k in range(5):
        lo = 2 * math.pi * k / 5
        pts.append((math.cos(lat) * math.cos(lo), math.cos(lat) * math.sin(lo), math.sin(lat)))
    for k in range(5):
        lo = 2 * math.pi * (k + 0.5) / 5
        pts.append((math.cos(lat) * math.cos(lo), math.cos(lat) * math.sin(lo), -math.sin(lat)))
    pts.append((0.0, 0.0, -1.0))
    xyz = np.array(pts)
    N, S = 0, 11
    U = [1 + k for k in range(5)]
    L = [6 + k for k in range(5)]
    faces = []
    for k in range(5):
        k1 = (k + 1) % 5
        faces += [(N, U[k], U[k1]), (U[k], L[k], U[k1]), (U[k1], L[k], L[k1]), (S, L[k1], L[k])]
    faces = np.array(faces, dtype=np.int64)
    a, b, c = xyz[faces[:, 0]], xyz[faces[:, 1]], xyz[faces[:, 2]]
    flip = np.sum(np.cross(b - a, c - a) * (a + b + c), axis=1) < 0
    faces[flip] = faces[flip][:, [0, 2, 1]]
    return xyz, faces


def subdivide(xyz, tri):
    """One edge bisection (Sec. 2.2): every triangle (a, b, c) becomes four,
    with midpoints projected onto the sphere, m = (a + b)/|a + b|.  New node
    ids are appended in order of first appearance.  Returns the new positions,
    triangles and, for every new node, the coarse endpoints (a, b) of the edge
    it bisects."""
    mid = {}
    new_pts = []
    parents = []
    n0 = xyz.shape[0]

    def midpoint(a, b):
        key = (a, b) if a < b else (b, a)
        m = mid.get(key)
        if m is None:
            m = n0 + len(new_pts)
            mid[key] = m
            new_pts.append(key)
            parents.append(key)
        return m

    out = []
    for a, b, c in tri.tolist():
        ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
        out += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
    parents = np.array(parents, dtype=np.int64).reshape(-1, 2)
    new_xyz = normalize(xyz[parents[:, 0]] + xyz[parents[:, 1]])
    return np.concatenate([xyz, new_xyz]), np.array(out, dtype=np.int64), parents


# ----------------------------------------------------------------------------- one level

class Level:
    """Topology and geometry of one uniform level J (Sec. 3.1, Sec. 4.1).

    Arrays (N nodes, E edges, T triangles):
      xyz[N,3]             unit positions of the nodes (hexagon centres)
      tri[T,3]             triangle nodes, counter-clockwise from outside
      edges[E,2]           edge end nodes (origin, end); origin = smaller id;
                           the normal velocity u_e is positive from origin to end
      tri_edges[T,3], tri_esign[T,3]
                           edge of side k=(tri[t,k] -> tri[t,k+1]) and +1 when that
                           side runs along the edge direction (counter-clockwise
                           circulation sign t_{e,v})
      left[E], right[E]    triangle to the left / right of origin -> end
      deg[N]               5 (pentagon) or 6 (hexagon)
      nbr_edges[N,6], nbr_sign[N,6], nbr_nodes[N,6], nbr_tris[N,6]
                           counter-clockwise ring around each node: edge e_k to
                           neighbour nbr_nodes[k], with n_{e,i} = nbr_sign (+1 when
                           the node is the edge's origin, i.e. u points out of it),
                           and triangle v_k between e_k and e_{k+1}; padded with -1
      cc[T,3]              triangle circumcentres (hexagon vertices)
      kite[T,3]            area of triangle t inside the hexagon of tri[t,k]
      A_v[T], A_i[N]       dual triangle and hexagon areas (m^2)
      d_e[E], l_e[E]       node-to-node and circumcentre-to-circumcentre arc lengths (m)
      f_v[T]               Coriolis parameter 2 Omega sin(lat) at circumcentres
      kite_frac[N,6]       R_{i,v_k} = kite area of node i in v_k / (sum of its kites)
      A_kite[N]            sum of the kites of each node (= A_i at the finest level)
    """

    def __init__(self, J, xyz, tri, radius, omega):
        self.J = J
        self.radius = radius
        self.xyz = xyz
        self.tri = tri
        N, T = xyz.shape[0], tri.shape[0]
        self.N, self.T = N, T
        sides = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])       # (3T, 2): side k of all t
        lo, hi = np.minimum(sides[:, 0], sides[:, 1]), np.maximum(sides[:, 0], sides[:, 1])
        key = lo * N + hi
        ukey, inv = np.unique(key, return_inverse=True)
        self.E = ukey.size
        self.edges = np.stack([ukey // N, ukey % N], axis=1)
        sid = inv.reshape(3, T).T
        ssign = np.where(sides[:, 0] < sides[:, 1], 1, -1).reshape(3, T).T
        self.tri_edges, self.tri_esign = sid, ssign
        self.left = np.full(self.E, -1, dtype=np.int64)
        self.right = np.full(self.E, -1, dtype=np.int64)
        tt = np.repeat(np.arange(T)[:, None], 3, axis=1)
        self.left[sid[ssign > 0]] = tt[ssign > 0]
        self.right[sid[ssign < 0]] = tt[ssign < 0]
        assert (self.left >= 0).all() and (self.right >= 0).all()
        self._rings()
        self._geometry(omega)

    def _rings(self):
        N, E = self.N, self.E
        node = np.concatenate([self.edges[:, 0], self.edges[:, 1]])
        other = np.concatenate([self.edges[:, 1], self.edges[:, 0]])
        eid = np.concatenate([np.arange(E), np.arange(E)])
        sign = np.concatenate([np.ones(E, dtype=np.int64), -np.ones(E, dtype=np.int64)])
        x = self.xyz[node]
        e1, e2 = _local_basis(x)
        dvec = self.xyz[other] - x
        ang = np.arctan2(np.sum(dvec * e2, axis=1), np.sum(dvec * e1, axis=1))
        order = np.lexsort((ang, node))
        node, other, eid, sign = node[order], other[order], eid[order], sign[order]
        deg = np.bincount(node, minlength=N)
        assert set(np.unique(deg)) <= {5, 6}
        start = np.concatenate([[0], np.cumsum(deg)[:-1]])
        pos = np.arange(node.size) - start[node]
        self.deg = deg
        self.nbr_edges = np.full((N, 6), -1, dtype=np.int64)
        self.nbr_sign = np.zeros((N, 6), dtype=np.int64)
        self.nbr_nodes = np.full((N, 6), -1, dtype=np.int64)
        self.nbr_edges[node, pos] = eid
        self.nbr_sign[node, pos] = sign
        self.nbr_nodes[node, pos] = other
        # v_k: triangle to the left of the directed edge i -> nbr_k
        tris = np.where(sign > 0, self.left[eid], self.right[eid])
        self.nbr_tris = np.full((N, 6), -1, dtype=np.int64)
        self.nbr_tris[node, pos] = tris
        # consistency: v_k holds i, nbr_k and nbr_{k+1}
        for i in range(min(N, 64)):
            d = deg[i]
            for k in range(d):
                t = self.nbr_tris[i, k]
                assert {i, self.nbr_nodes[i, k], self.nbr_nodes[i, (k + 1) % d]} == set(self.tri[t].tolist())

    def _geometry(self, omega):
        R = self.radius
        x = self.xyz
        a, b, c = x[self.tri[:, 0]], x[self.tri[:, 1]], x[self.tri[:, 2]]
        self.cc = circumcentre(a, b, c)
        kite = np.zeros((self.T, 3))
        for k in range(3):
            p = x[self.tri[:, k]]
            nxt = x[self.tri[:, (k + 1) % 3]]
            prv = x[self.tri[:, (k + 2) % 3]]
            kite[:, k] = triangle_area(p, normalize(p + nxt), self.cc) + triangle_area(p, self.cc, normalize(prv + p))
        self.kite = kite * R * R
        self.A_v = self.kite.sum(axis=1)
        self.A_kite = np.zeros(self.N)
        np.add.at(self.A_kite, self.tri.ravel(), self.kite.ravel())
        self.A_i = self.A_kite.copy()
        self.d_e = arc_length(x[self.edges[:, 0]], x[self.edges[:, 1]]) * R
        self.l_e = arc_length(self.cc[self.left], self.cc[self.right]) * R
        self.f_v = 2.0 * omega * self.cc[:, 2]
        # kite fractions R_{i,v_k} in ring order
        kf = np.zeros((self.N, 6))
        for k in range(6):
            t = self.nbr_tris[:, k]
            ok = t >= 0
            tt = np.where(ok, t, 0)
            pos = np.argmax(self.tri[tt] == np.arange(self.N)[:, None], axis=1)
            kf[:, k] = np.where(ok, self.kite[tt, pos] / self.A_kite, 0.0)
        self.kite_frac = kf

    # convenience geometry for inputs and comparisons
    def edge_midpoints(self):
        return normalize(self.xyz[self.edges[:, 0]] + self.xyz[self.edges[:, 1]])

    def edge_tangents(self):
        """Unit tangent at the midpoint along origin -> end."""
        return normalize(self.xyz[self.edges[:, 1]] - self.xyz[self.edges[:, 0]])

    def hexagon(self, i):
        """Counter-clockwise hexagon (pentagon) vertices of node i."""
        return self.cc[self.nbr_tris[i, : self.deg[i]]]


def nominal_spacing(J, radius):
    """Mean node spacing of Table 1: sqrt(2 * 4 pi R^2 / (sqrt(3) N_J))."""
    N = 10 * 4 ** J + 2
    return math.sqrt(2.0 * 4.0 * math.pi * radius * radius / (math.sqrt(3.0) * N))


# ----------------------------------------------------------------------------- the hierarchy

class Hierarchy:
    """Levels Jmin..Jmax of the nested grid plus the inter-level structure.

    For each j in (Jmin, Jmax]:
      odd[j]       node ids of the odd nodes of level j (ids N_{j-1} .. N_j - 1)
      pedge[j]     coarse edge (level j-1) bisected by each odd node
      K[j][n,4]    K_m^{j-1}: the coarse nodes whose hexagons can overlap the fine
                   hexagon m -- the two ends a, b of the bisected coarse edge and the
                   opposite vertices c (left triangle), d (right triangle).  Reading:
                   this set is fixed by the topology (Sec. 4.3 names the two main and
                   the two second-nearest coarse neighbours of every m), so the same
                   points enter every stencil whatever the overlap areas are.
      Akm[j][n,4]  A_km^{j}: area of coarse hexagon k (level j-1) inside fine hexagon m,
                   normalised so that sum_k A_km = A_m (see below)
      Akm_clip[j]  the same areas as clipped, before normalisation
      Am[j][n]     A_m, the fine hexagon area of each odd node
      mid[j-1][E]  fine node at the midpoint of each coarse edge
      half[j-1][E,2]
                   fine edges (origin half, end half) of each coarse edge, both
                   oriented like the coarse edge via half_sign
    """

    def __init__(self, jmin, jmax, radius=6.371e6, omega=7.292e-5):
        assert 0 <= jmin <= jmax
        self.jmin, self.jmax, self.radius, self.omega = jmin, jmax, radius, omega
        xyz, tri = icosahedron()
        raw = {0: (xyz, tri, None)}
        for j in range(1, jmax + 1):
            xyz, tri, par = subdivide(xyz, tri)
            raw[j] = (xyz, tri, par)
        self.levels = {}
        for j in range(jmin, jmax + 1):
            self.levels[j] = Level(j, raw[j][0], raw[j][1], radius, omega)
        self.odd, self.pedge, self.K, self.Akm, self.Am, self.mid, self.half, self.half_sign = {}, {}, {}, {}, {}, {}, {}, {}
        self.Akm_clip = {}
        for j in range(jmin + 1, jmax + 1):
            self._link(j, raw[j][2])
        # Reading (Sec. 4.1 area conditions).  Going from Jmax down, the clipped
        # overlaps of every fine hexagon m are scaled so that they add up to the
        # fine hexagon area A_m exactly (first condition), and the area of a
        # coarse hexagon is the sum of the fine pieces that tile it,
        # A_k^j = A_k^{j+1} + sum_m A_km (second condition).  Both conditions then
        # hold in stored numbers, and with them R_h o div = div o R_F.  The
        # scaling changes the clipped areas by ~1e-11 relative at most (node
        # positions are rounded off the sphere by ~1 ulp, which moves each
        # circumcentre by ~ulp/dx).  The finest level keeps its kite sums.
        for j in range(jmax, jmin, -1):
            C, F = self.levels[j - 1], self.levels[j]
            Am = F.A_i[self.odd[j]]
            self.Akm_clip[j] = self.Akm[j]
            self.Akm[j] = self.Akm[j] * (Am / self.Akm[j].sum(axis=1))[:, None]
            self.Am[j] = Am
            A = F.A_i[: C.N].copy()
            np.add.at(A, self.K[j].ravel(), self.Akm[j].ravel())
            C.A_i = A

    def _link(self, j, par):
        C, F = self.levels[j - 1], self.levels[j]
        n0 = C.N
        odd = np.arange(n0, F.N)
        # coarse edge of each odd node
        key = C.edges[:, 0] * C.N + C.edges[:, 1]
        order = np.argsort(key)
        pkey = np.minimum(par[:, 0], par[:, 1]) * C.N + np.maximum(par[:, 0], par[:, 1])
        pe = order[np.searchsorted(key[order], pkey)]
        assert np.array_equal(key[pe], pkey)
        a, b = C.edges[pe, 0], C.edges[pe, 1]
        third = lambda t, p, q: C.tri[t].sum(axis=1) - p - q
        c = third(C.left[pe], a, b)
        d = third(C.right[pe], a, b)
        self.odd[j] = odd
        self.pedge[j] = pe
        self.K[j] = np.stack([a, b, c, d], axis=1)
        mid = np.empty(C.E, dtype=np.int64)
        mid[pe] = odd
        self.mid[j - 1] = mid
        # fine half edges of each coarse edge
        fkey = F.edges[:, 0] * F.N + F.edges[:, 1]
        forder = np.argsort(fkey)

        def fine_edge(p, q):
            k = np.minimum(p, q) * F.N + np.maximum(p, q)
            idx = forder[np.searchsorted(fkey[forder], k)]
            assert np.array_equal(fkey[idx], k)
            return idx, np.where(p < q, 1, -1)

        h0, s0 = fine_edge(C.edges[:, 0], mid)
        h1, s1 = fine_edge(mid, C.edges[:, 1])
        self.half[j - 1] = np.stack([h0, h1], axis=1)
        self.half_sign[j - 1] = np.stack([s0, s1], axis=1)
        # overlap areas A_km by clipping the fine hexagon m against coarse hexagon k
        Akm = np.zeros((odd.size, 4))
        P = F.cc[F.nbr_tris[odd]]                      # odd nodes are never pentagons
        assert (F.deg[odd] == 6).all()
        for col in range(4):
            k = self.K[j][:, col]
            hexk = C.cc[np.where(C.nbr_tris[k] >= 0, C.nbr_tris[k], C.nbr_tris[k][:, :1])]
            nxt = np.roll(hexk, -1, axis=1)
            pent = C.deg[k] == 5                       # repeat the first half-space for pentagons
            nxt[pent, 4] = hexk[pent, 0]
            normals = np.cross(hexk, nxt - hexk)
            anchors = hexk.copy()
            normals[pent, 5] = normals[pent, 0]
            anchors[pent, 5] = anchors[pent, 0]
            Q, cnt = clip_convex(P.copy(), np.full(odd.size, 6), normals, anchors)
            Akm[:, col] = polygon_area(Q, cnt) * self.radius ** 2
        self.Akm[j] = Akm
        self.Am[j] = Akm.sum(axis=1)
