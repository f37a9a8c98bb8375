"""Pins for the oracle's perceptron (learned refinement proposal).

* BF16 rounding against an independent definition: scale to 8 significant bits
  and round half to even with numpy's rint;
* the chain-rule gradient against central finite differences of the loss;
* closed forms: logit 0 gives loss log 2 for either label; a zero network's
  gradient of b2 is the mean of (p - y) weighted by the class weight; Adam's
  bias-corrected step under a constant gradient;
* the mask with an external proposal: extra nodes join T before the closure, as
  a literal set construction."""
import math

import numpy as np
import pytest

from oracle import adapt, grid, mlp


def _bf16_ref(x):
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    nz = x != 0
    e = np.floor(np.log2(np.abs(x[nz])))
    out[nz] = np.rint(x[nz] * 2.0 ** (7 - e)) * 2.0 ** (e - 7)
    return out


def test_bf16_rounding():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 1, 5000), rng.normal(0, 1e-3, 1000), rng.normal(0, 1e4, 1000)])
    x = x.astype(np.float32).astype(np.float64)
    assert np.array_equal(mlp.bf16(x), _bf16_ref(x))
    # ties: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 -> even (1); 1 + 3*2^-8 -> 1 + 2^-6
    assert mlp.bf16([1 + 2.0 ** -8])[0] == 1.0
    assert mlp.bf16([1 + 3 * 2.0 ** -8])[0] == 1 + 2.0 ** -6


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    X = rng.normal(0, 1, (40, mlp.F))
    y = (rng.random(40) < 0.3).astype(float)
    W1 = rng.normal(0, 0.5, (mlp.F, mlp.H))
    b1 = rng.normal(0, 0.1, mlp.H)
    w2 = rng.normal(0, 0.5, mlp.H)
    b2 = 0.2
    pos_w = 3.0
    L, dW1, db1, dw2, db2 = mlp.loss_grad(X, y, W1, b1, w2, b2, pos_w)
    assert abs(L - mlp.loss(X, y, W1, b1, w2, b2, pos_w)) < 1e-14
    h = 1e-6
    num = []
    theta = mlp.flat(W1, b1, w2, b2)
    for k in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        def L_of(t):
            return mlp.loss(X, y, t[:mlp.F * mlp.H].reshape(mlp.F, mlp.H), t[mlp.F * mlp.H:mlp.F * mlp.H + mlp.H],
                            t[mlp.F * mlp.H + mlp.H:-1], t[-1], pos_w)
        num.append((L_of(tp) - L_of(tm)) / (2 * h))
    ana = mlp.flat(dW1, db1, dw2, db2)
    assert np.max(np.abs(np.array(num) - ana)) < 1e-7


def test_closed_forms():
    X = np.ones((4, mlp.F))
    z = np.zeros((mlp.F, mlp.H))
    b = np.zeros(mlp.H)
    for y in (0.0, 1.0):
        assert abs(mlp.loss(X, [y] * 4, z, b, b, 0.0, 1.0) - math.log(2)) < 1e-15
    y = np.array([1.0, 0.0, 0.0, 1.0])
    L, _, _, _, db2 = mlp.loss_grad(X, y, z, b, b, 0.0, 2.0)
    assert abs(db2 - np.mean(2.0 * y * (0.5 - 1) + (1 - y) * 0.5)) < 1e-15


def test_adam_steps_of_a_constant_gradient():
    """Adam (Kingma & Ba) with its bias corrections: under a constant gradient the
    corrected moments are the gradient and its square at every step, so each
    update is lr g / (|g| + eps), the first one included."""
    rng = np.random.default_rng(2)
    g = rng.standard_normal(50)
    p = rng.standard_normal(50)
    m, v = np.zeros(50), np.zeros(50)
    lr = 1e-3
    for t in range(1, 6):
        q, m, v = mlp.adam(p, g, m, v, t, lr)
        assert np.allclose(p - q, lr * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
        p = q


def test_mask_with_external_proposal():
    Hy = grid.Hierarchy(2, 4)
    rng = np.random.default_rng(3)
    sig = {j: rng.random(Hy.levels[j].N) < 0.01 for j in range(3, 5)}
    extra = {j: rng.random(Hy.levels[j].N) < 0.02 for j in range(3, 5)}
    ln0, _ = adapt.build_mask(Hy, sig)
    ln1, _ = adapt.build_mask(Hy, sig, extra)
    # the plain mask with the extra nodes as significant-without-neighbours points:
    # T gains exactly them before the closure
    nbr_free = {}
    for j in range(3, 5):
        t = adapt.dilate(Hy.levels[j], sig[j])
        if j - 1 > 2:
            ch = np.zeros(Hy.levels[j].N, dtype=bool)
            ch[: Hy.levels[j - 1].N] = sig[j - 1]
            t |= adapt.dilate(Hy.levels[j], ch)
        nbr_free[j] = t | extra[j]
    for j in range(4, 2, -1):
        odd = Hy.odd[j]
        nbr_free[j][Hy.K[j][nbr_free[j][odd]].ravel()] = True
        if j - 1 > 2:
            nbr_free[j - 1] |= nbr_free[j][: Hy.levels[j - 1].N]
    for j in range(3, 5):
        assert np.array_equal(ln1[j], nbr_free[j])
        assert np.all(ln1[j] >= ln0[j])
        assert np.all(ln1[j][extra[j]])
