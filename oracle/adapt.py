"""Oracle: the adapted grid -- significance mask, closure, ghost band, prolongation.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 2.3: keep every point whose wavelet coefficient is significant
(|coef| >= eps), all of Jmin, and the points adjacent to a significant one in
space (same level) and in scale (next finer level).  Sec. 3.1: also keep the
points the operators' stencils need, and make the height and velocity points
consistent; thresholds eps_h, eps_u follow from eps.

Readings, applied as a fixed sequence of set operations so that the mask is a
set, independent of any iteration order:
  1. significance at level j > Jmin: an odd node with |h~| >= eps_h; the two
     ends and the midpoint of a coarse edge with |u~_E| >= eps_u; the two ends
     of an interior fine edge with |u~_f| >= eps_u (an active edge activates
     both end nodes).  Only live points carry coefficients.
  2. adjacency: T^j = S^j + its same-level neighbours + the children of S^{j-1}
     (the fine node at the same place and its fine neighbours), capped at Jmax.
  3. graded closure, from Jmax down: every live odd node m brings its four
     prediction parents K_m (as fine even nodes) into level j, and every live
     even fine node brings its coarse node into level j-1.  A live fine point
     therefore always has its whole prediction stencil live one level down.
  4. Jmin is live everywhere; a live node activates its 5-6 edges (an edge is
     live when an end node is live).
  5. ghost band: nodes within 5 neighbour hops of a live node and edges between
     live-or-ghost nodes, not live themselves, are ghosts.  Ghost values are the
     inverse transform with zero wavelet coefficients (prolongation from level
     j-1), refreshed before each trend evaluation; they feed the stencils of live
     points and of the flux restriction, which reaches four hops.
Thresholds (reading): eps_h = eps * max|dh|, eps_u = eps * max|u| over live
points; a coefficient is significant when its modulus is >= the threshold.
"""
from __future__ import annotations

import numpy as np

GHOST_HOPS = 5


def dilate(L, S):
    """S plus every same-level neighbour of S (node sets as boolean arrays)."""
    out = S.copy()
    for k in range(6):
        nb = L.nbr_nodes[:, k]
        ok = nb >= 0
        out[nb[ok & S]] = True
    return out


def edges_touching(L, nodes):
    return nodes[L.edges[:, 0]] | nodes[L.edges[:, 1]]


def edges_within(L, nodes):
    return nodes[L.edges[:, 0]] & nodes[L.edges[:, 1]]


def significance(Hy, j, live_n, live_e, hdet, udet_e, udet_i, VS, eps_h, eps_u):
    """Step 1 at level j > Jmin.  hdet over odd nodes, udet_e over coarse edges,
    udet_i[T_coarse, 3] over interior fine edges (NaN where not computed)."""
    C, F = Hy.levels[j - 1], Hy.levels[j]
    S = np.zeros(F.N, dtype=bool)
    odd = Hy.odd[j]
    with np.errstate(invalid="ignore"):
        sh = live_n[odd] & (np.abs(hdet) >= eps_h)
        S[odd[sh]] = True
        se = np.abs(udet_e) >= eps_u
        S[C.edges[se, 0]] = True
        S[C.edges[se, 1]] = True
        S[Hy.mid[j - 1][se]] = True
        si = live_e[VS.int_edge] & (np.abs(udet_i) >= eps_u)
    fe = VS.int_edge[si]
    S[F.edges[fe, 0]] = True
    S[F.edges[fe, 1]] = True
    return S


def build_mask(Hy, sig, extra=None):
    """Steps 2-4.  sig[j] = significance set of level j (j > Jmin).  extra[j]
    (optional): nodes of level j added to T after step 2 (an external refinement
    proposal; the closure then treats them like any other point of T).  Returns
    live node and edge sets per level."""
    jmin, jmax = Hy.jmin, Hy.jmax
    T = {}
    for j in range(jmin + 1, jmax + 1):
        F = Hy.levels[j]
        t = dilate(F, sig[j])
        if j - 1 > jmin:
            ch = np.zeros(F.N, dtype=bool)
            ch[: Hy.levels[j - 1].N] = sig[j - 1]
            t |= dilate(F, ch)
        if extra is not None and j in extra:
            t |= extra[j]
        T[j] = t
    for j in range(jmax, jmin, -1):
        F = Hy.levels[j]
        oddlive = T[j][Hy.odd[j]]
        T[j][Hy.K[j][oddlive].ravel()] = True
        if j - 1 > jmin:
            T[j - 1] |= T[j][: Hy.levels[j - 1].N]
    live_n, live_e = {}, {}
    for j in range(jmin, jmax + 1):
        L = Hy.levels[j]
        live_n[j] = np.ones(L.N, dtype=bool) if j == jmin else T[j]
        live_e[j] = edges_touching(L, live_n[j])
    return live_n, live_e


def ghost_band(Hy, live_n, live_e):
    """Step 5."""
    ghost_n, ghost_e = {}, {}
    for j in range(Hy.jmin, Hy.jmax + 1):
        L = Hy.levels[j]
        if j == Hy.jmin:
            ghost_n[j] = np.zeros(L.N, dtype=bool)
            ghost_e[j] = np.zeros(L.E, dtype=bool)
            continue
        band = live_n[j]
        for _ in range(GHOST_HOPS):
            band = dilate(L, band)
        ghost_n[j] = band & ~live_n[j]
        ghost_e[j] = edges_within(L, band) & ~live_e[j]
    return ghost_n, ghost_e


def prolong_level(Hy, VS, j, dh, u, live_n, live_e, tgt_n, tgt_e):
    """Inverse transform with zero wavelet coefficients into the target points of
    level j from level j-1 (Eqs. 1-2 inverted with h~ = 0, u~ = 0).  Live values
    are kept; non-live even fine nodes take the coarse value (no live detail
    touches them, by the closure)."""
    C, F = Hy.levels[j - 1], Hy.levels[j]
    hc, hf = dh[j - 1], dh[j]
    nc = C.N
    even_t = tgt_n[:nc]
    hf[:nc][even_t] = hc[even_t]
    odd = Hy.odd[j]
    ot = tgt_n[odd]
    K = Hy.K[j][ot]
    st = Hy.Akm[j][ot] / Hy.Am[j][ot][:, None]
    vals = np.where(live_n[K], hf[K], hc[K])
    hf[odd[ot]] = np.sum(st * vals, axis=1)
    # velocity
    uc, uf = u[j - 1], u[j]
    ph, pi = np.sum(VS.half_w * uc[VS.half_st], axis=2), np.sum(VS.int_w * uc[VS.int_st], axis=2)
    h0, h1 = VS.half[:, 0], VS.half[:, 1]
    s0, s1 = VS.half_sign[:, 0], VS.half_sign[:, 1]
    l0, l1 = live_e[h0], live_e[h1]
    delta = 0.5 * (2.0 * uc - ph[:, 0] - ph[:, 1])
    t0 = tgt_e[h0] & ~l0
    t1 = tgt_e[h1] & ~l1
    a = t0 & ~l1
    uf[h0[a]] = s0[a] * (ph[a, 0] + delta[a])
    a = t0 & l1
    uf[h0[a]] = s0[a] * (2.0 * uc[a] - s1[a] * uf[h1[a]])
    b = t1 & ~l0
    uf[h1[b]] = s1[b] * (ph[b, 1] + delta[b])
    b = t1 & l0
    uf[h1[b]] = s1[b] * (2.0 * uc[b] - s0[b] * uf[h0[b]])
    it = tgt_e[VS.int_edge] & ~live_e[VS.int_edge]
    uf[VS.int_edge[it]] = pi[it]
