"""The seeded inputs follow their stated definitions (the generators hold no
method arithmetic; these checks keep them honest):

* turbulence: the energy per degree follows (l/32)^2 below degree 32 and
  (l/32)^-3 above, the rms velocity is 20 m/s, the depth is in geostrophic
  balance with the stream function;
* the shared sampling gives the same values as direct evaluation.
"""
import math

import numpy as np

import workloads


def test_turbulence_spectrum_and_amplitude():
    W = workloads.Workload("turbulence", seed=3)
    S = W._psi
    E = np.array([l * (l + 1) * (np.sum(S.a[l] ** 2) + np.sum(S.b[l, 1:] ** 2)) for l in range(S.lmax + 1)])
    shape = np.array([0.0] + [(l / 32.0) ** 2 if l < 32 else (l / 32.0) ** -3.0 for l in range(1, S.lmax + 1)])
    ok = shape > 0
    ratio = E[ok] / shape[ok]
    assert np.allclose(ratio, ratio[0], rtol=1e-12)
    # rms of the velocity over the sphere from random points and directions
    rng = np.random.default_rng(0)
    x = rng.standard_normal((40000, 3))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    t = np.cross(x, rng.standard_normal((40000, 3)))
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    rms_component = math.sqrt(np.mean(W.velocity(x, t) ** 2))
    assert abs(rms_component * math.sqrt(2.0) / 20.0 - 1) < 0.05
    # geostrophic depth: g (h - H) = f0 psi
    assert np.allclose(W.depth(x) - 1.0e4, W.f0 * S(x) / W.g, rtol=1e-12, atol=1e-9)


def test_sampling_matches_direct_evaluation():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3000, 3))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    m = rng.standard_normal((5000, 3))
    m /= np.linalg.norm(m, axis=1, keepdims=True)
    t = np.cross(m, rng.standard_normal((5000, 3)))
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    S = workloads.Sampling(x, m, t)
    for kind in ("jet", "tc2", "harmonic", "tc1_smooth", "turbulence"):
        W = workloads.Workload(kind, seed=2)
        a, b = W.fields(x, m, t), W.fields_on(S)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), kind
