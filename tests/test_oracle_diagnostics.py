"""Pins for the oracle's mass and energy diagnostics (Sec. 6, Eq. for E and c).

Closed forms the code does not compute itself: the mass of a resting layer of
depth H is H times the sphere's area; the energy of a resting layer (u = 0) is
g^2/2 times the area-weighted variance of h about its mean (the c^4 term removes
exactly the mean part); a uniform layer at rest has zero energy; and with a flow
the energy grows by g sum_i A_i h_i K_i with K_i = (1/A_i) sum_e 1/4 l_e d_e u_e^2."""
import math

import numpy as np
import pytest

from oracle import grid, model


@pytest.fixture(scope="module")
def hy():
    return grid.Hierarchy(2, 3)


def _model(hy, dh, u):
    M = model.Model(hy, eps=1e-2, rk="rk4", cfl=0.8)
    M.set_uniform(dh, u)
    return M


def test_mass_of_resting_layer(hy):
    L = hy.levels[3]
    M = _model(hy, np.zeros(L.N), np.zeros(L.E))
    area = 4.0 * math.pi * L.radius ** 2
    assert abs(M.mass() / (M.H * area) - 1) < 1e-14


def test_energy_of_uniform_rest_is_zero(hy):
    L = hy.levels[3]
    M = _model(hy, np.zeros(L.N), np.zeros(L.E))
    scale = 0.5 * (M.g * M.H) ** 2 * 4.0 * math.pi * L.radius ** 2
    assert abs(M.energy()) < 1e-13 * scale


def test_energy_of_perturbed_rest_is_variance(hy):
    rng = np.random.default_rng(5)
    L = hy.levels[3]
    M = _model(hy, rng.normal(0.0, 50.0, L.N), np.zeros(L.E))
    Lm = hy.levels[2]
    h = M.H + M.dh[2]
    hbar = np.sum(Lm.A_i * h) / np.sum(Lm.A_i)
    want = 0.5 * M.g ** 2 * np.sum(Lm.A_i * (h - hbar) ** 2)
    assert abs(M.energy() / want - 1) < 1e-6


def test_energy_kinetic_part(hy):
    rng = np.random.default_rng(6)
    L = hy.levels[3]
    dh = rng.normal(0.0, 50.0, L.N)
    u = rng.normal(0.0, 10.0, L.E)
    M = _model(hy, dh, u)
    R = _model(hy, dh, np.zeros(L.E))
    Lm = hy.levels[2]
    uc = M.u[2]
    en = Lm.edges
    K = np.zeros(Lm.N)
    for e in range(Lm.E):
        w = 0.25 * Lm.l_e[e] * Lm.d_e[e] * uc[e] ** 2
        K[en[e, 0]] += w
        K[en[e, 1]] += w
    K /= Lm.A_i
    want = M.g * np.sum(Lm.A_i * (M.H + M.dh[2]) * K)
    assert abs((M.energy() - R.energy()) / want - 1) < 1e-9
