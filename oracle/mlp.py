"""Oracle: the two-layer perceptron of the learned refinement proposal, in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The proposal is an extension of the method (the paper's criterion is the
threshold rule of Sec. 2.3); this module states what the library's perceptron
computes, so that its GPU forward pass and gradient can be checked:

    z = b1 + x W1,  a = max(z, 0),  logit = b2 + a . w2,  p = 1 / (1 + exp(-logit))
    loss = mean_i [ pos_w y_i (-log p_i) + (1 - y_i) (-log(1 - p_i)) ]

with W1 [F][H] and w2 [H] rounded to BF16 (round to nearest, ties to even, on the
FP32 master values) and the biases kept in FP32.  The gradient is taken with
respect to the weights as used (BF16-rounded), which is what the library passes
straight through to the FP32 masters.
"""
from __future__ import annotations

import numpy as np

F, H = 8, 32
NPARAM = F * H + H + H + 1


def bf16(x):
    """Round FP32 values to BF16 (the upper 16 bits of the FP32 pattern, round to
    nearest with ties to even); returned as float64."""
    b = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params, round_bf16=True):
    """(W1 [F][H], b1 [H], w2 [H], b2) from the flat FP32 parameter vector."""
    p = np.asarray(params, dtype=np.float32)
    W1 = p[: F * H].reshape(F, H)
    b1 = p[F * H: F * H + H].astype(np.float64)
    w2 = p[F * H + H: F * H + 2 * H]
    b2 = float(p[F * H + 2 * H])
    if round_bf16:
        return bf16(W1), b1, bf16(w2), b2
    return W1.astype(np.float64), b1, w2.astype(np.float64), b2


def forward(X, W1, b1, w2, b2):
    X = np.asarray(X, dtype=np.float64)
    z = b1[None, :] + X @ W1
    a = np.maximum(z, 0.0)
    logit = b2 + a @ w2
    return z, a, logit


def softplus(t):
    return np.where(t > 0, t + np.log1p(np.exp(-np.abs(t))), np.log1p(np.exp(np.minimum(t, 0.0))))


def loss(X, y, W1, b1, w2, b2, pos_w):
    _, _, logit = forward(X, W1, b1, w2, b2)
    y = np.asarray(y, dtype=np.float64)
    sp = softplus(logit)
    return float(np.mean(pos_w * y * (sp - logit) + (1.0 - y) * sp))


def loss_grad(X, y, W1, b1, w2, b2, pos_w):
    """Mean loss and its gradient (dW1, db1, dw2, db2) by the chain rule."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = X.shape[0]
    z, a, logit = forward(X, W1, b1, w2, b2)
    p = 1.0 / (1.0 + np.exp(-logit))
    g = (pos_w * y * (p - 1.0) + (1.0 - y) * p) / n          # d loss / d logit
    dz = (g[:, None] * w2[None, :]) * (z > 0)
    sp = softplus(logit)
    L = float(np.mean(pos_w * y * (sp - logit) + (1.0 - y) * sp))
    return L, X.T @ dz, dz.sum(axis=0), a.T @ g, float(g.sum())


def flat(dW1, db1, dw2, db2):
    return np.concatenate([dW1.ravel(), db1, dw2, [db2]])


def predict(X, params):
    W1, b1, w2, b2 = unpack(params)
    _, _, logit = forward(X, W1, b1, w2, b2)
    return 1.0 / (1.0 + np.exp(-logit))


def adam(params, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba), in FP64 on copies."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
