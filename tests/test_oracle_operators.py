"""Pins for the oracle's TRiSK operators (Sec. 3.1) and transforms (Sec. 2.2, 4).

Each check is something the mathematics fixes independently of the code: the
discrete mimetic identities of TRiSK, the Thuburn (steady geostrophic mode)
condition, energy neutrality of the Coriolis term, invertibility and mass
conservation of the lifting scheme, reproduction of constants and linear
fields, second-order decay of the wavelet coefficients of a smooth field, and
the commutation R_h o div = div o R_F of Eq. (divRcommute)."""
import math

import numpy as np
import pytest

import workloads
from oracle import grid, transform, trisk


@pytest.fixture(scope="module")
def L3():
    return grid.Hierarchy(3, 3).levels[3]


def test_div_of_rotational_flow_is_zero(L3):
    rng = np.random.default_rng(0)
    psi = rng.standard_normal(L3.T)
    u = -(psi[L3.left] - psi[L3.right]) / L3.l_e
    div = trisk.divergence(L3, u)
    assert np.abs(div * L3.A_i).max() < 1e-12 * np.abs(u * L3.l_e).max()


def test_curl_of_gradient_is_zero(L3):
    rng = np.random.default_rng(1)
    phi = rng.standard_normal(L3.N)
    z = trisk.vorticity(L3, trisk.gradient(L3, phi))
    assert np.abs(z * L3.A_v).max() < 1e-12


def test_coriolis_is_energy_neutral(L3):
    rng = np.random.default_rng(2)
    F = rng.standard_normal(L3.E)
    q = rng.standard_normal(L3.T)
    cor = trisk.coriolis_tendency(L3, F, q)
    work = L3.d_e * L3.l_e * F * cor
    assert abs(work.sum()) < 1e-13 * np.abs(work).sum()


def test_thuburn_condition(L3):
    """Uniform q: the net flux of the reconstructed perpendicular flux out of a
    dual triangle equals the kite-weighted sum of the cell divergences."""
    rng = np.random.default_rng(3)
    F = rng.standard_normal(L3.E)
    cor = trisk.coriolis_tendency(L3, F, np.ones(L3.T))
    e = L3.tri_edges
    out_of_triangle = -np.sum(L3.tri_esign * cor[e] * L3.d_e[e], axis=1)
    kf = L3.kite / L3.A_kite[L3.tri]
    rhs = np.sum(kf * trisk.outflux(L3, F)[L3.tri], axis=1)
    assert np.abs(out_of_triangle - rhs).max() < 1e-13 * np.abs(rhs).max()


def test_perp_reconstruction_sign_and_size():
    """For a smooth solid-body flow the reconstruction approaches F.n_left in the
    rms sense (its maximum error on plain bisection grids does not vanish: the
    known inconsistency of the scheme near the icosahedron's edges)."""
    rms = []
    for J in (3, 4, 5):
        L = grid.Hierarchy(J, J).levels[J]
        m, t = L.edge_midpoints(), L.edge_tangents()
        east = np.stack([-m[:, 1], m[:, 0], 0 * m[:, 0]], 1)
        u = np.sum(east * t, 1)
        exact = np.sum(east * np.cross(m, t), 1)
        err = trisk.coriolis_tendency(L, u, np.ones(L.T)) - exact
        rms.append(np.sqrt(np.mean(err ** 2)))
    assert rms[0] < 0.05 and rms[1] < rms[0] and rms[2] < rms[1]


def test_kinetic_energy_sum(L3):
    """sum_i A_i K_i = sum_e (l_e d_e / 2) u_e^2."""
    u = np.random.default_rng(4).standard_normal(L3.E)
    K = trisk.kinetic_energy(L3, u)
    assert abs((L3.A_i * K).sum() / (0.5 * L3.l_e * L3.d_e * u ** 2).sum() - 1) < 1e-14


def test_resting_state_has_zero_trend(L3):
    dh = np.zeros(L3.N)
    u = np.zeros(L3.E)
    a, b = trisk.trend(L3, dh, u, 1.0e4, 9.80616)
    assert np.abs(a).max() == 0.0 and np.abs(b).max() == 0.0


def test_tc2_imbalance_order():
    """Williamson TC2 (Sec. 6.2) is an exact steady state: the zonal mass flux has
    zero divergence and the Coriolis force balances the Bernoulli gradient.  The
    trend of the sampled state is the discrete imbalance, so its decay with
    resolution is the operators' order of accuracy on this grid.

    On the plain bisection grid (no Heikes-Randall or Xu optimisation, Sec. 3.2)
    the divergence part converges at first order in the rms (the depth trend
    falls by about 2.2-2.4 per level, J3..6), while the velocity imbalance falls
    by only about 1.4 per level in the rms and not at all in the maximum: the
    known inconsistency of TRiSK's Coriolis and kinetic-energy operators on
    unoptimised icosahedral grids.  The paper's second-order statement is for its
    optimised grids.  A sign or weight slip in div, grad, K or q F^perp breaks
    these rates (the imbalance then stays O(1) of the terms)."""
    g = 9.80616
    rms_h, rms_u, max_u = [], [], []
    for J in (3, 4, 5, 6):
        L = grid.Hierarchy(J, J).levels[J]
        W = workloads.Workload("tc2", mean_depth=2.94e4 / g)
        dh, u = W.fields(L.xyz, L.edge_midpoints(), L.edge_tangents())
        a, b = trisk.trend(L, dh, u, 2.94e4 / g, g)
        rms_h.append(math.sqrt(np.mean(a ** 2)))
        rms_u.append(math.sqrt(np.mean(b ** 2)))
        max_u.append(np.abs(b).max())
    rate_h = [rms_h[k] / rms_h[k + 1] for k in range(3)]
    rate_u = [rms_u[k] / rms_u[k + 1] for k in range(3)]
    print("TC2 depth-trend rms ratios", rate_h, "velocity-trend rms ratios", rate_u)
    assert all(1.9 < r < 2.8 for r in rate_h), rate_h          # first order
    assert all(1.25 < r < 1.6 for r in rate_u), rate_u         # about half order in the rms
    # the imbalance is a small fraction of the balanced terms (f u ~ 3e-3 m/s^2)
    assert max(max_u) < 0.15 * 7.292e-5 * 2 * (2 * math.pi * 6.371e6 / (12 * 86400))


# ----------------------------------------------------------------------------- transforms

@pytest.mark.parametrize("j", [3, 4, 5])
def test_height_lifting_inverts_and_conserves(hier25, j):
    C, F = hier25.levels[j - 1], hier25.levels[j]
    rng = np.random.default_rng(j)
    hf = rng.standard_normal(F.N) + 3.0
    d = transform.height_detail(hier25, j, hf)
    hc = transform.height_update(hier25, j, hf, d)
    assert np.abs(transform.inverse_height(hier25, j, hc, d) - hf).max() < 1e-14
    assert abs(C.A_i @ hc / (F.A_i @ hf) - 1) < 1e-15 * 8
    assert np.abs(transform.height_detail(hier25, j, np.full(F.N, 7.0))).max() < 1e-14


def test_height_details_decay_second_order(hier25):
    W = workloads.Workload("harmonic", seed=2)
    mx = []
    for j in (3, 4, 5):
        F = hier25.levels[j]
        dh, _ = W.fields(F.xyz, F.edge_midpoints(), F.edge_tangents())
        mx.append(np.abs(transform.height_detail(hier25, j, dh)).max())
    assert 3.0 < mx[0] / mx[1] < 5.0 and 3.0 < mx[1] / mx[2] < 5.0


@pytest.mark.parametrize("j", [3, 4, 5])
def test_velocity_transform_inverts(hier25, j):
    F = hier25.levels[j]
    VS = transform.VelocityStencils(hier25, j)
    uf = np.random.default_rng(j).standard_normal(F.E)
    uc = transform.restrict_velocity(hier25, j, uf)
    de, di = transform.velocity_detail(VS, uc, uf)
    assert np.abs(transform.inverse_velocity(VS, uc, de, di, F.E) - uf).max() < 1e-14


def test_velocity_weights_reproduce_linear_fields(hier25):
    """Constructing a linear tangent field in each fine edge's orthographic plane,
    the weighted coarse values give the fine value exactly."""
    j = 4
    C, F = hier25.levels[j - 1], hier25.levels[j]
    VS = transform.VelocityStencils(hier25, j)
    rng = np.random.default_rng(5)
    fe = VS.int_edge[:, 0]
    p = F.edge_midpoints()[fe]
    tf = F.edge_tangents()[fe]
    e1, e2 = grid._local_basis(p)
    st = VS.int_st[:, 0]
    xs, ts = C.edge_midpoints()[st], C.edge_tangents()[st]
    A = rng.standard_normal((p.shape[0], 2, 3))    # V(x) = a0 + A1 (x.e1, x.e2)

    def field(x, t):
        xi = np.stack([np.einsum("bik,bk->bi", x, e1), np.einsum("bik,bk->bi", x, e2)], -1)
        v = A[:, None, :, 0] + A[:, None, :, 1] * xi[..., :1] + A[:, None, :, 2] * xi[..., 1:]
        tt = np.stack([np.einsum("bik,bk->bi", t, e1), np.einsum("bik,bk->bi", t, e2)], -1)
        return np.sum(v * tt, -1)

    vals = field(xs, ts)
    target = field(p[:, None, :] * 0.0, tf[:, None, :])[:, 0]
    pred = np.sum(VS.int_w[:, 0] * vals, axis=1)
    assert np.abs(pred - target).max() < 1e-12


def test_velocity_details_decay(hier25):
    W = workloads.Workload("harmonic", seed=3)
    me, mi = [], []
    for j in (3, 4, 5):
        F = hier25.levels[j]
        _, u = W.fields(F.xyz, F.edge_midpoints(), F.edge_tangents())
        VS = transform.VelocityStencils(hier25, j)
        de, di = transform.velocity_detail(VS, transform.restrict_velocity(hier25, j, u), u)
        me.append(np.abs(de).max())
        mi.append(np.abs(di).max())
    assert me[0] / me[1] > 3.0 and me[1] / me[2] > 3.0
    assert mi[0] / mi[1] > 3.0 and mi[1] / mi[2] > 3.0


@pytest.mark.parametrize("j", [3, 4, 5])
def test_flux_restriction_commutes(hier25, j):
    """Eq. (divRcommute): R_h(div_j F) = div_{j-1}(R_F F) for random fluxes."""
    C, F = hier25.levels[j - 1], hier25.levels[j]
    Ff = np.random.default_rng(10 + j).standard_normal(F.E)
    c = trisk.divergence(F, Ff)
    FS = transform.FluxStencils(hier25, j)
    Fc = transform.restrict_flux(FS, Ff, F.l_e, c)
    lhs = transform.restrict_height(hier25, j, c)
    rhs = trisk.divergence(C, Fc / C.l_e)
    assert np.abs(lhs - rhs).max() < 1e-14 * np.abs(lhs).max()


def test_flux_restriction_of_uniform_flow_is_consistent(hier25):
    """A smooth flow's restricted flux approximates the coarse-level flux
    (the restriction is a consistent average, not only a conservative one)."""
    j = 5
    C, F = hier25.levels[j - 1], hier25.levels[j]
    W = workloads.Workload("harmonic", seed=4)
    _, uf = W.fields(F.xyz, F.edge_midpoints(), F.edge_tangents())
    _, uc = W.fields(C.xyz, C.edge_midpoints(), C.edge_tangents())
    FS = transform.FluxStencils(hier25, j)
    Fc = transform.restrict_flux(FS, uf, F.l_e, trisk.divergence(F, uf)) / C.l_e
    assert np.sqrt(np.mean((Fc - uc) ** 2)) < 0.05 * np.sqrt(np.mean(uc ** 2))


def test_flux_restriction_converges(hier25):
    """The restricted flux of a smooth flow approaches the coarse flux as the
    levels refine: the rms error falls by more than 2.5 per level (measured 3.1;
    Sec. 4.2 builds the x fluxes to second order, ratio 4 on equilateral
    triangles, and Sec. 3.2 notes the bisection grid's distortion lowers the
    order).  The x fluxes cancel in the divergence, so commutation alone does not
    see them; dropping them, halving them or turning their sign leaves an error
    of 13-50 % that does not fall with the level."""
    W = workloads.Workload("harmonic", seed=4)
    errs = []
    for j in (3, 4, 5):
        C, F = hier25.levels[j - 1], hier25.levels[j]
        _, uf = W.fields(F.xyz, F.edge_midpoints(), F.edge_tangents())
        _, uc = W.fields(C.xyz, C.edge_midpoints(), C.edge_tangents())
        FS = transform.FluxStencils(hier25, j)
        Fc = transform.restrict_flux(FS, uf, F.l_e, trisk.divergence(F, uf)) / C.l_e
        errs.append(np.sqrt(np.mean((Fc - uc) ** 2)) / np.sqrt(np.mean(uc ** 2)))
    assert errs[0] / errs[1] > 2.5 and errs[1] / errs[2] > 2.5, errs


# ----------------------------------------------------------------------------- viscous form (Sec. 3.1)

def test_scalar_laplacian_identities(L3):
    """div grad: conserves mass and is the negative of the discrete gradient energy,
    sum_i A_i a_i (div grad a)_i = -sum_e l_e d_e (grad a)_e^2 (summation by parts)."""
    rng = np.random.default_rng(21)
    a = rng.normal(0, 1, L3.N)
    lap = trisk.laplacian(L3, a)
    assert abs(np.sum(L3.A_i * lap)) < 1e-10 * np.sum(L3.A_i * np.abs(lap))
    gr = trisk.gradient(L3, a)
    lhs = np.sum(L3.A_i * a * lap)
    rhs = -np.sum(L3.l_e * L3.d_e * gr ** 2)
    assert rhs < 0 and abs(lhs / rhs - 1) < 1e-12


def test_vector_laplacian_energy_identity(L3):
    """sum_e l_e d_e u_e (grad div u - grad^perp curl u)_e = -sum_i A_i D_i^2
    - sum_v A_v zeta_v^2: both parts dissipate, with the signs of the paper's form."""
    rng = np.random.default_rng(22)
    u = rng.normal(0, 1, L3.E)
    lap = trisk.vector_laplacian(L3, u)
    D = trisk.divergence(L3, u)
    z = trisk.vorticity(L3, u)
    lhs = np.sum(L3.l_e * L3.d_e * u * lap)
    rhs = -np.sum(L3.A_i * D ** 2) - np.sum(L3.A_v * z ** 2)
    assert abs(lhs / rhs - 1) < 1e-12


def _y2(xyz):
    """A degree-2 real spherical harmonic (xy), eigenfunction of the sphere's
    Laplacian with eigenvalue -l(l+1)/R^2 = -6/R^2."""
    return xyz[:, 0] * xyz[:, 1]


@pytest.mark.parametrize("kind", ["scalar", "gradient"])
def test_laplacians_of_a_spherical_harmonic_converge(kind):
    """The discrete Laplacians of a degree-2 harmonic (scalar, and its gradient
    field) approach -6/R^2 times it as the grid is refined."""
    errs = []
    for J in (3, 4, 5):
        L = grid.Hierarchy(J, J).levels[J]
        R = L.radius
        if kind == "scalar":
            y = _y2(L.xyz)
            got, want = trisk.laplacian(L, y), -6.0 / R ** 2 * y
        else:
            u = trisk.gradient(L, _y2(L.xyz))
            got, want = trisk.vector_laplacian(L, u), -6.0 / R ** 2 * u
        errs.append(np.sqrt(np.mean((got - want) ** 2)) / np.sqrt(np.mean(want ** 2)))
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 0.05


def test_viscous_trend_adds_the_laplacians(L3):
    rng = np.random.default_rng(23)
    dh = rng.normal(0, 50, L3.N)
    u = rng.normal(0, 5, L3.E)
    a0, b0 = trisk.trend(L3, dh, u, 1e4, 9.80616)
    a1, b1 = trisk.trend(L3, dh, u, 1e4, 9.80616, nu=1e5)
    assert np.allclose(a1 - a0, 1e5 * trisk.laplacian(L3, dh), rtol=1e-9, atol=1e-18)
    assert np.allclose(b1 - b0, 1e5 * trisk.vector_laplacian(L3, u), rtol=1e-9, atol=1e-18)


def test_rotational_laplacian_rayleigh_quotient():
    """The curl-curl part on the dual cells does not converge pointwise on grids
    refined by bisection (the paper notes the Laplacian's non-convergence on such
    grids, Sec. 3.2); its weak form does: for the rotated gradient of a degree-2
    harmonic, <u, Lap u> / <u, u> (l d weights) stays within 5 % of -6/R^2 and the
    field is divergence-free to rounding."""
    for J in (3, 4, 5):
        L = grid.Hierarchy(J, J).levels[J]
        R = L.radius
        cc = L.cc / np.linalg.norm(L.cc, axis=1)[:, None]
        u = trisk.perp_gradient(L, _y2(cc))
        lap = trisk.vector_laplacian(L, u)
        w = L.l_e * L.d_e
        ratio = np.sum(w * u * lap) / np.sum(w * u * u) / (-6.0 / R ** 2)
        assert 0.95 < ratio < 1.05
        assert np.abs(trisk.divergence(L, u)).max() * R < 1e-12 * np.abs(u).max() * 1e3
