"""Oracle: TRiSK operators and the rotating shallow-water trend on one level.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sec. 3.1: the vector-invariant equations d(dh)/dt + div F = 0 (Eq. height),
du/dt + q F^perp + grad B = 0 (Eq. velo), q = (curl u + f)/h, F = h u,
h = H + dh, B = g dh + K, K = |u|^2/2, discretised with the TRiSK operators of
Ringler et al. (2010), energy-conserving variant for q F^perp.  Those operators
are written here from their published definitions:

  div at node i       (1/A_i) sum_e n_{e,i} F_e l_e           (n = +1 when u_e leaves i)
  grad at edge e      (B_end - B_origin) / d_e
  curl at triangle v  (1/A_v) sum_e t_{e,v} u_e d_e           (t = +1 counter-clockwise)
  K at node i         (1/A_i) sum_e (l_e d_e / 4) u_e^2
  h at triangle v     (1/A_v) sum_i A_{i,v} h_i                (kite-weighted)
  q F^perp at edge e  energy-conserving reconstruction from the normal fluxes of
                      the edges of the two cells sharing e (Thuburn et al. 2009
                      weights w = 1/2 - sum of the kite fractions R_{i,v} passed
                      going counter-clockwise from e to e')

Conventions: l_e is the hexagon face (circumcentre-to-circumcentre) length,
d_e the node-to-node length, u_e the velocity along origin -> end.

Reconstruction, derived here (cell i, edges e_1..e_D counter-clockwise, vertex
v_k between e_k and e_{k+1}, outward fluxes phi_k = n_{e_k,i} F_k l_k, kite
fractions R_k = R_{i,v_k}): splitting each face flux evenly between its two
kites and giving kite k the share R_k of the cell's net outflow, the flux
crossing the half-edge from i to the midpoint of e_k (counter-clockwise) is
    psi_k = sum_{k' != k} (1/2 - sum_{m=k}^{k'-1} R_m) phi_{k'},
with the weights antisymmetric in (k, k').  The tangential flux across the whole
edge e (left of origin -> end) is psi^(origin) - psi^(end), and the Coriolis
part of du_e/dt is +q F.n_left.  The energy-conserving form multiplies the
(e, e') term by (q_e + q_e')/2 with q_e the mean of the two triangles of e.

Missing values are NaN: an operator evaluated where its stencil is not
available yields NaN, so a missing stencil point can never pass silently.
"""
from __future__ import annotations

import numpy as np


def total_depth(dh, H):
    return H + dh


def thickness_flux(L, dh, u, H):
    """F_e = h_e u_e with h_e the mean depth of the two end nodes (per unit length)."""
    h = total_depth(dh, H)
    return 0.5 * (h[L.edges[:, 0]] + h[L.edges[:, 1]]) * u


def divergence(L, F):
    """(1/A_i) sum_e n_{e,i} F_e l_e at every node."""
    out = np.zeros(L.N)
    for k in range(6):
        e = L.nbr_edges[:, k]
        ok = e >= 0
        ee = np.where(ok, e, 0)
        out += np.where(ok, L.nbr_sign[:, k] * F[ee] * L.l_e[ee], 0.0)
    return out / L.A_i


def outflux(L, F):
    """Net integrated outflow sum_e n_{e,i} F_e l_e of every cell (m^3/s)."""
    return divergence(L, F) * L.A_i


def gradient(L, B):
    return (B[L.edges[:, 1]] - B[L.edges[:, 0]]) / L.d_e


def kinetic_energy(L, u):
    out = np.zeros(L.N)
    for k in range(6):
        e = L.nbr_edges[:, k]
        ok = e >= 0
        ee = np.where(ok, e, 0)
        out += np.where(ok, 0.25 * L.l_e[ee] * L.d_e[ee] * u[ee] ** 2, 0.0)
    return out / L.A_i


def vorticity(L, u):
    """zeta_v = (1/A_v) sum t_{e,v} u_e d_e at every triangle."""
    e = L.tri_edges
    return np.sum(L.tri_esign * u[e] * L.d_e[e], axis=1) / L.A_v


def depth_at_triangles(L, dh, H):
    h = total_depth(dh, H)
    return np.sum(L.kite * h[L.tri], axis=1) / L.A_v


def potential_vorticity(L, dh, u, H):
    return (vorticity(L, u) + L.f_v) / depth_at_triangles(L, dh, H)


def coriolis_tendency(L, F, q):
    """Coriolis part of du_e/dt, +q F.n_left, energy-conserving TRiSK form."""
    qe = 0.5 * (q[L.left] + q[L.right])
    acc = np.zeros(L.E)
    N = L.N
    deg = L.deg
    for k in range(6):
        ek = L.nbr_edges[:, k]
        has_k = ek >= 0
        ekk = np.where(has_k, ek, 0)
        psi = np.zeros(N)
        csum = np.zeros(N)        # sum_{m=k}^{k'-1} R_m
        for o in range(1, 6):
            kk = (k + o) % deg
            kp = (k + o - 1) % deg
            ok = has_k & (o < deg)
            csum = csum + np.where(ok, L.kite_frac[np.arange(N), kp], 0.0)
            e2 = L.nbr_edges[np.arange(N), kk]
            e2 = np.where(ok, e2, 0)
            phi = L.nbr_sign[np.arange(N), kk] * F[e2] * L.l_e[e2]
            w = 0.5 - csum
            psi += np.where(ok, w * phi * 0.5 * (qe[ekk] + qe[e2]), 0.0)
        # n_{e,i} psi / d_e: + for the origin cell, - for the end cell
        contrib = np.where(has_k, L.nbr_sign[:, k] * psi, 0.0)
        np.add.at(acc, ekk[has_k], contrib[has_k])
    return acc / L.d_e


def bernoulli(L, dh, u, g):
    return g * dh + kinetic_energy(L, u)


def perp_gradient(L, z):
    """grad^perp of a dual-cell field at every edge: (1/l_e) sum_{v at e} t_{e,v} z_v,
    the adjoint of the vorticity (sum_e l_e d_e u_e (grad^perp z)_e = sum_v A_v z_v zeta_v)."""
    out = np.zeros(L.E)
    for k in range(3):
        np.add.at(out, L.tri_edges[:, k], L.tri_esign[:, k] * z)
    return out / L.l_e


def laplacian(L, a):
    """div grad of a node field (Sec. 3.1, viscous form)."""
    return divergence(L, gradient(L, a))


def vector_laplacian(L, u):
    """grad div u - grad^perp curl u at every edge (Sec. 3.1, viscous form)."""
    return gradient(L, divergence(L, u)) - perp_gradient(L, vorticity(L, u))


def trend(L, dh, u, H, g, nu=0.0):
    """Uniform-level trend (d dh/dt, du/dt) of Eqs. (height), (velo); with nu > 0 the
    viscous form: nu div grad(dh) on the height, nu (grad div u - grad^perp curl u) on
    the velocity (the Bernoulli gradient stays grad B; B already holds K)."""
    F = thickness_flux(L, dh, u, H)
    q = potential_vorticity(L, dh, u, H)
    B = bernoulli(L, dh, u, g)
    a = -divergence(L, F)
    b = coriolis_tendency(L, F, q) - gradient(L, B)
    if nu:
        a = a + nu * laplacian(L, dh)
        b = b + nu * vector_laplacian(L, u)
    return a, b
