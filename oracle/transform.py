"""Oracle: wavelet transforms between level j-1 (coarse) and level j (fine), and
the conservative flux restriction.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Height (Sec. 2.2 Eqs. 1-2, Sec. 4.1 Eq. Rh):
    predict  h~_m = h_m^j - sum_{k in K_m} s~_km h_k^j          s~_km = A_km / A_m
    update   h_k^{j-1} = h_k^j + sum_{m in M_k} s_km h~_m       s_km = A_km / A_k^{j-1}
    R_h      = update o predict.
  Even fine nodes carry the coarse node's id, so h_k^j is the fine value at k.

Velocity (Sec. 3.1, Sec. 4.1: non-separable vector transform, fine-edge velocity
interpolated from a symmetric 12-edge coarse stencil with weights of second-order
accuracy from 6x6 linear systems).  Readings:
  * restriction R_u: the coarse velocity is the mean of the two fine half edges
    (circulation preserving: the geodesic midpoint halves the coarse edge);
  * stencil: a fine edge touching or cutting off coarse node a is predicted from
    the 12 coarse edges of the star of a (6 spokes + 6 rim edges; 10 at a
    pentagon).  Each coarse edge has two half edges (predicted from the stars of
    its two ends) and each coarse triangle three interior fine edges;
  * weights: the minimum-norm weights that reproduce every linear tangent vector
    field (6 conditions) in the orthographic tangent plane at the fine-edge
    midpoint; the normal equations are one 6x6 solve per fine edge;
  * details: one per coarse edge, u~_E = ((u_h0 - P_h0) - (u_h1 - P_h1))/2 (the
    half-edge velocities along the coarse edge), and u~_f = u_f - P_f per
    interior fine edge.  The inverse keeps the coarse mean.

Flux restriction R_F = R_F0 + R'_F (Sec. 4.2, 4.3; Eqs. restr_flux, ho_flux, kml),
acting on integrated fluxes, for coarse edge E = (k -> l) with fine midpoint m,
left triangle (k, l, p), right triangle (l, k, q):
  R_F0 (reading; Fig. 3 is not in the text).  Within fine hexagon m a uniform
  divergence c_m splits m between its k side and its l side, which gives the flux
  through the part of the coarse face inside m as F_in^k + A_km c_m (Sec. 4.2),
  F_in^k the fine flux entering m through its three faces on the k side.  Taken
  antisymmetrically, F1 = (F_in^k - F_in^l)/2 + (A_km - A_lm) c_m / 2.  The
  sliver pieces at each coarse corner (fine hexagon of the midpoint opposite a
  coarse node reaching into that node's hexagon) are routed through the three
  coarse faces meeting at the corner with the minimum-norm circulation, which
  gives (s_k - s_l)/2 per corner with s_k = A_{k,m_lp} c_{m_lp},
  s_l = A_{l,m_kp} c_{m_kp}.  Then sum_{e at k} R_F0 = A_k^j c_k + sum_m A_km c_m.
  The x fluxes of Eq. (restr_flux) (reading): at each coarse corner the three
  fine hexagons of the edge midpoints meet at the circumcentre W of the central
  fine triangle, not at the coarse vertex V.  The fine-face construction above
  measures the flux up to W; the flux through the short segment V -> W,
  x_T = G.((W - V) x V) with G the flux vector fitted (least squares) to the
  three fine faces meeting at W, is taken off.  For each coarse triangle it is a
  circulation around the corner (-x_T on each coarse face oriented
  counter-clockwise around T), so, as Sec. 4.2 notes, the commutation holds
  whatever value it has; it makes R_F exact for uniform flows.
  R'_F: Eq. (ho_flux) is read as the corrective flux through the single coarse
  face k -> l_{2j} (the outer sum adds the faces of cell k), with
  (kml) = A_km A_lm / A_m (c_k - c_l), Eq. (kml).
Together sum_{e at k} R_F = A_k^{j-1} R_h(c)_k: Eq. (divRcommute).
"""
from __future__ import annotations

import numpy as np

from . import trisk
from .grid import _local_basis, normalize


# ----------------------------------------------------------------------------- height

def height_detail(Hy, j, hf):
    """h~_m for every odd node m of level j from the fine field hf (Eq. 1)."""
    K, Akm, Am = Hy.K[j], Hy.Akm[j], Hy.Am[j]
    odd = Hy.odd[j]
    st = Akm / Am[:, None]
    return hf[odd] - np.sum(st * hf[K], axis=1)


def height_update(Hy, j, hf, hdet):
    """Coarse scaling coefficients h^{j-1} from the fine even values and the details (Eq. 2)."""
    C = Hy.levels[j - 1]
    hc = hf[: C.N].copy()
    s = Hy.Akm[j] / C.A_i[Hy.K[j]]
    np.add.at(hc, Hy.K[j].ravel(), (s * hdet[:, None]).ravel())
    return hc


def restrict_height(Hy, j, hf):
    """R_h: level j -> level j-1 (Eq. Rh)."""
    return height_update(Hy, j, hf, height_detail(Hy, j, hf))


def inverse_height(Hy, j, hc, hdet):
    """Inverse lifting: undo the update, then undo the predict."""
    C, F = Hy.levels[j - 1], Hy.levels[j]
    s = Hy.Akm[j] / C.A_i[Hy.K[j]]
    even = hc.copy()
    np.subtract.at(even, Hy.K[j].ravel(), (s * hdet[:, None]).ravel())
    hf = np.empty(F.N)
    hf[: C.N] = even
    st = Hy.Akm[j] / Hy.Am[j][:, None]
    hf[Hy.odd[j]] = hdet + np.sum(st * even[Hy.K[j]], axis=1)
    return hf


# ----------------------------------------------------------------------------- velocity

class VelocityStencils:
    """Predicted fine edges of level j with their coarse stencils and weights.

      half_st[E,2,12], half_w[E,2,12]  stencil/weights of the two halves of each coarse edge
                                       (velocity along the coarse edge direction)
      int_edge[T,3]                    interior fine edge cutting off vertex tri[t,c]
      int_st[T,3,12], int_w[T,3,12]    its stencil/weights (velocity along the fine edge)
    Pentagon stars have 10 edges; the last two slots then carry weight 0.
    """

    def __init__(self, Hy, j):
        C, F = Hy.levels[j - 1], Hy.levels[j]
        self.j = j
        star = np.zeros((C.N, 12), dtype=np.int64)
        nst = 2 * C.deg
        for k in range(6):
            ok = k < C.deg
            spoke = np.where(ok, C.nbr_edges[:, k], C.nbr_edges[:, 0])
            t = np.where(ok, C.nbr_tris[:, k], C.nbr_tris[:, 0])
            te = C.tri_edges[t]
            tn = C.tri[t]
            # rim edge of triangle v_k: the side opposite the centre node
            opp = np.argmax(tn == np.arange(C.N)[:, None], axis=1)
            rim = te[np.arange(C.N), (opp + 1) % 3]
            star[:, k] = spoke
            star[:, 6 + k] = rim
        # compact pentagon stars into the first 10 slots
        pent = C.deg == 5
        star[pent, 5:10] = star[pent, 6:11]
        star[pent, 10:] = star[pent, :1]
        self.star, self.nst = star, nst
        cmid = C.edge_midpoints()
        ctan = C.edge_tangents()
        dx = np.mean(C.d_e) / C.radius
        fmid = F.edge_midpoints()
        ftan = F.edge_tangents()

        def weights(p, tf, centre):
            st = star[centre]
            n = nst[centre]
            w = solve_weights(p, tf, cmid[st], ctan[st], n, dx)
            return st, w

        # halves: along the coarse edge direction
        self.half = Hy.half[j - 1]
        self.half_sign = Hy.half_sign[j - 1]
        hs, hw = [], []
        for s in range(2):
            fe = self.half[:, s]
            centre = C.edges[:, s]
            st, w = weights(fmid[fe], ftan[fe] * self.half_sign[:, s][:, None], centre)
            hs.append(st)
            hw.append(w)
        self.half_st = np.stack(hs, axis=1)
        self.half_w = np.stack(hw, axis=1)
        # interior fine edges
        mid = Hy.mid[j - 1]
        fkey = F.edges[:, 0] * F.N + F.edges[:, 1]
        forder = np.argsort(fkey)

        def fine_edge(p, q):
            kk = np.minimum(p, q) * F.N + np.maximum(p, q)
            idx = forder[np.searchsorted(fkey[forder], kk)]
            assert np.array_equal(fkey[idx], kk)
            return idx

        te = C.tri_edges
        ie, ist, iw = [], [], []
        for c in range(3):
            # vertex tri[t,c]: its two sides are side c (c -> c+1) and side c-1 (c-1 -> c)
            m1 = mid[te[:, c]]
            m2 = mid[te[:, (c + 2) % 3]]
            fe = fine_edge(m1, m2)
            centre = C.tri[:, c]
            st, w = weights(fmid[fe], ftan[fe], centre)
            ie.append(fe)
            ist.append(st)
            iw.append(w)
        self.int_edge = np.stack(ie, axis=1)
        self.int_st = np.stack(ist, axis=1)
        self.int_w = np.stack(iw, axis=1)


def solve_weights(p, tf, xs, ts, n, dx):
    """Minimum-norm weights w (B, 12) with sum_i w_i V(x_i).t_i = V(p).t_f for every
    linear vector field V in the orthographic tangent plane at p (6 conditions);
    slots i >= n get weight 0."""
    e1, e2 = _local_basis(p)
    xi = np.einsum("bik,bk->bi", xs, e1) / dx
    eta = np.einsum("bik,bk->bi", xs, e2) / dx
    t1 = np.einsum("bik,bk->bi", ts, e1)
    t2 = np.einsum("bik,bk->bi", ts, e2)
    mask = np.arange(12)[None, :] < n[:, None]
    M = np.stack([t1, t2, xi * t1, eta * t1, xi * t2, eta * t2], axis=1) * mask[:, None, :]
    b = np.zeros((p.shape[0], 6))
    b[:, 0] = np.sum(tf * e1, axis=1)
    b[:, 1] = np.sum(tf * e2, axis=1)
    G = np.einsum("bri,bsi->brs", M, M)
    lam = np.linalg.solve(G, b[..., None])[..., 0]
    return np.einsum("bri,br->bi", M, lam)


def restrict_velocity(Hy, j, uf):
    """R_u: u_E^{j-1} = mean of the two fine half edges (along E)."""
    h, s = Hy.half[j - 1], Hy.half_sign[j - 1]
    return 0.5 * (s[:, 0] * uf[h[:, 0]] + s[:, 1] * uf[h[:, 1]])


def velocity_predict(VS, uc):
    ph = np.sum(VS.half_w * uc[VS.half_st], axis=2)        # (E, 2)
    pi = np.sum(VS.int_w * uc[VS.int_st], axis=2)          # (T, 3)
    return ph, pi


def velocity_detail(VS, uc, uf):
    """(u~ per coarse edge, u~ per interior fine edge) given coarse and fine velocities."""
    ph, pi = velocity_predict(VS, uc)
    a = VS.half_sign[:, 0] * uf[VS.half[:, 0]] - ph[:, 0]
    b = VS.half_sign[:, 1] * uf[VS.half[:, 1]] - ph[:, 1]
    return 0.5 * (a - b), uf[VS.int_edge] - pi


def inverse_velocity(VS, uc, udet_e, udet_i, n_fine_edges):
    ph, pi = velocity_predict(VS, uc)
    delta = 0.5 * (2.0 * uc - ph[:, 0] - ph[:, 1])
    uf = np.full(n_fine_edges, np.nan)
    uf[VS.half[:, 0]] = VS.half_sign[:, 0] * (ph[:, 0] + delta + udet_e)
    uf[VS.half[:, 1]] = VS.half_sign[:, 1] * (ph[:, 1] + delta - udet_e)
    uf[VS.int_edge] = pi + udet_i
    return uf


# ----------------------------------------------------------------------------- flux restriction

class FluxStencils:
    """Index plumbing of R_F for every coarse edge E = (k -> l) of level j-1."""

    def __init__(self, Hy, j):
        C, F = Hy.levels[j - 1], Hy.levels[j]
        E = C.E
        k, l = C.edges[:, 0], C.edges[:, 1]
        tp, tq = C.left, C.right
        third = lambda t, a, b: C.tri[t].sum(axis=1) - a - b
        p, q = third(tp, k, l), third(tq, k, l)
        ekey = C.edges[:, 0] * C.N + C.edges[:, 1]
        eorder = np.argsort(ekey)

        def cedge(a, b):
            kk = np.minimum(a, b) * C.N + np.maximum(a, b)
            idx = eorder[np.searchsorted(ekey[eorder], kk)]
            assert np.array_equal(ekey[idx], kk)
            return idx

        def opposite(a, b, c):
            """third vertex of the triangle across edge (a, b) from vertex c"""
            e = cedge(a, b)
            t1, t2 = C.left[e], C.right[e]
            t = np.where(third(t1, a, b) == c, t2, t1)
            return third(t, a, b)

        mid = Hy.mid[j - 1]
        self.tl, self.tr = tp, tq
        self._corner_geometry(Hy, j)
        self.k, self.l, self.p, self.q = k, l, p, q
        self.m = mid[np.arange(E)]
        self.m_kp, self.m_lp = mid[cedge(k, p)], mid[cedge(l, p)]
        self.m_kq, self.m_lq = mid[cedge(k, q)], mid[cedge(l, q)]
        self.pp1 = opposite(l, p, k)      # p' : across (l, p) from k
        self.qq1 = opposite(l, q, k)      # q' : across (l, q) from k
        self.pp2 = opposite(k, p, l)      # p'': across (k, p) from l
        self.qq2 = opposite(k, q, l)      # q'': across (k, q) from l
        # overlap lookup A_{y,x} for odd fine x and coarse y in K_x
        n0 = C.N
        self._K, self._A = Hy.K[j], Hy.Akm[j]
        self._n0 = n0
        self.Am = np.zeros(F.N)
        self.Am[Hy.odd[j]] = Hy.Am[j]
        # fine faces of m toward each neighbour
        self.ring_nodes = F.nbr_nodes[self.m]
        self.ring_edges = F.nbr_edges[self.m]
        self.ring_sign = F.nbr_sign[self.m]

    def _corner_geometry(self, Hy, j):
        """Per coarse triangle: the three fine edges of its central fine triangle,
        their unit tangents in the tangent plane at the coarse vertex V, and the
        rotated segment (W - V) x V (m) used by x_T."""
        C, F = Hy.levels[j - 1], Hy.levels[j]
        mid = Hy.mid[j - 1]
        te = C.tri_edges
        cm = mid[te]                                    # (T, 3) midpoint nodes of the sides
        fkey = F.edges[:, 0] * F.N + F.edges[:, 1]
        forder = np.argsort(fkey)

        def fine_edge(a, b):
            kk = np.minimum(a, b) * F.N + np.maximum(a, b)
            idx = forder[np.searchsorted(fkey[forder], kk)]
            assert np.array_equal(fkey[idx], kk)
            return idx

        self.cen_edges = np.stack([fine_edge(cm[:, c], cm[:, (c + 1) % 3]) for c in range(3)], axis=1)
        # central fine triangle = the one holding the three midpoints
        t = F.left[self.cen_edges[:, 0]]
        t = np.where(np.isin(F.tri[t], cm).all(axis=1), t, F.right[self.cen_edges[:, 0]])
        assert np.sort(F.tri[t], axis=1).tolist() == np.sort(cm, axis=1).tolist()
        V = C.cc
        W = F.cc[t]
        e1, e2 = _local_basis(V)
        ft = F.edge_tangents()[self.cen_edges]          # (T, 3, 3)
        self.cen_t1 = np.einsum("tck,tk->tc", ft, e1)
        self.cen_t2 = np.einsum("tck,tk->tc", ft, e2)
        seg = np.cross(W - V, V) * C.radius
        self.seg1 = np.sum(seg * e1, axis=1)
        self.seg2 = np.sum(seg * e2, axis=1)

    def corner_flux(self, Ff):
        """x_T for every coarse triangle from fine fluxes per unit length."""
        f = Ff[self.cen_edges]
        a11 = np.sum(self.cen_t1 ** 2, 1)
        a12 = np.sum(self.cen_t1 * self.cen_t2, 1)
        a22 = np.sum(self.cen_t2 ** 2, 1)
        b1 = np.sum(self.cen_t1 * f, 1)
        b2 = np.sum(self.cen_t2 * f, 1)
        det = a11 * a22 - a12 * a12
        g1 = (a22 * b1 - a12 * b2) / det
        g2 = (a11 * b2 - a12 * b1) / det
        return g1 * self.seg1 + g2 * self.seg2

    def overlap(self, y, x):
        r = x - self._n0
        col = np.argmax(self._K[r] == y[:, None], axis=1)
        assert (self._K[r][np.arange(r.size), col] == y).all()
        return self._A[r, col]

    def phi_into_m(self, Ff, lf, x):
        """Integrated fine flux from fine cell x into fine cell m."""
        hit = self.ring_nodes == x[:, None]
        assert (hit.sum(axis=1) == 1).all()
        col = np.argmax(hit, axis=1)
        r = np.arange(x.size)
        e = self.ring_edges[r, col]
        return -self.ring_sign[r, col] * Ff[e] * lf[e]


def restrict_flux(FS, Ff, lf, c):
    """Integrated coarse flux R_F(F) through every coarse face k -> l.

    Ff: fine flux per unit length, lf: fine face lengths, c: fine divergence."""
    k, l, m = FS.k, FS.l, FS.m
    A = FS.overlap
    F_in_k = FS.phi_into_m(Ff, lf, k) + FS.phi_into_m(Ff, lf, FS.m_kp) + FS.phi_into_m(Ff, lf, FS.m_kq)
    F_in_l = FS.phi_into_m(Ff, lf, l) + FS.phi_into_m(Ff, lf, FS.m_lp) + FS.phi_into_m(Ff, lf, FS.m_lq)
    F1 = 0.5 * (F_in_k - F_in_l) + 0.5 * (A(k, m) - A(l, m)) * c[m]
    corner = 0.5 * (A(k, FS.m_lp) * c[FS.m_lp] - A(l, FS.m_kp) * c[FS.m_kp]) \
        + 0.5 * (A(k, FS.m_lq) * c[FS.m_lq] - A(l, FS.m_kq) * c[FS.m_kq])

    def kml(a, x, b):
        return A(a, x) * A(b, x) / FS.Am[x] * (c[a] - c[b])

    corr = kml(k, m, l) + kml(k, FS.m_kp, l) + kml(k, FS.m_kq, l) + kml(k, FS.m_lp, l) + kml(k, FS.m_lq, l) \
        + 0.5 * kml(k, FS.m_lp, FS.pp1) + 0.5 * kml(k, FS.m_lq, FS.qq1) \
        + 0.5 * kml(FS.pp2, FS.m_kp, l) + 0.5 * kml(FS.qq2, FS.m_kq, l)
    xT = FS.corner_flux(Ff)
    return F1 + corner + corr - xT[FS.tl] + xT[FS.tr]
