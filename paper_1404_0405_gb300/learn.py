"""Training and evaluation of the learned refinement proposal.

Argument marshalling and loop control only: features, labels, the perceptron's
loss gradient, the Adam update and the proposal itself all run in the library's
kernels (``sww_set_learned``, ``sww_get_patch_data``, ``sww_mlp_loss_grad``,
``sww_mlp_adam``, ``sww_mlp_predict``).

Training data come from the method itself: the features of every patch above
Jmin at one adaptation, labelled by whether the exact rules' set T of the *next*
adaptation reaches the patch.  The trained network then proposes, before each
mask, the patches the next step will need; the exact rules still run and add
every patch it missed.
"""
from __future__ import annotations

import math

import numpy as np

from . import (MLP_FEATURES, MLP_HIDDEN, MLP_PARAMS, MLP_WORK, P_EXACT, P_FEATURES, mlp_adam, mlp_loss_grad,
               mlp_predict)


def _mask_levels(model):
    """Levels above Jmin that the next mask covers: those holding active patches
    and the one above them."""
    act = model.stats()["active_patches"]
    top = max([j for j in range(model.jmin, model.jmax + 1) if act.get(j, 0) > 0], default=model.jmin)
    return list(range(model.jmin + 1, min(top + 1, model.jmax) + 1))


def collect(model, steps, dt=-1.0):
    """Advance `steps` adaptive steps with features on; return (X [n, F] float32,
    y [n] float32): features of each patch of the levels the mask of adaptation k
    covered, and whether the exact set of adaptation k+1 reached it."""
    model.set_learned(1)
    model.adapt()                      # features of the current state
    Xs, ys = [], []
    for _ in range(steps):
        levels = _mask_levels(model)
        feats = {j: model.patch_data(j, P_FEATURES) for j in levels}
        model.step(dt, 1, adapt=True)
        for j in levels:
            Xs.append(np.ascontiguousarray(feats[j].T))
            ys.append(model.patch_data(j, P_EXACT).astype(np.float32))
    model.set_learned(0)
    return np.concatenate(Xs).astype(np.float32), np.concatenate(ys).astype(np.float32)


def init_params(prior, seed=0):
    """He-initialised first layer, small output layer, output bias at the prior's logit."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0.0, math.sqrt(2.0 / MLP_FEATURES), (MLP_FEATURES, MLP_HIDDEN))
    b1 = np.zeros(MLP_HIDDEN)
    w2 = rng.normal(0.0, math.sqrt(1.0 / MLP_HIDDEN), MLP_HIDDEN)
    p = min(max(prior, 1e-4), 1 - 1e-4)
    b2 = math.log(p / (1 - p))
    return np.concatenate([W1.ravel(), b1, w2, [b2]]).astype(np.float32)


def train(X, y, epochs=300, lr=1e-2, pos_weight=None, seed=0):
    """Full-batch Adam on the GPU.  Returns (params float32 [MLP_PARAMS], losses)."""
    import torch
    dev = torch.device("cuda")
    prior = float(np.mean(y)) if len(y) else 0.5
    if pos_weight is None:
        pos_weight = (1.0 - prior) / max(prior, 1e-6)
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(dev)
    yd = torch.from_numpy(np.ascontiguousarray(y, dtype=np.float32)).to(dev)
    params = torch.from_numpy(init_params(prior, seed)).to(dev)
    m = torch.zeros(MLP_PARAMS, device=dev)
    v = torch.zeros(MLP_PARAMS, device=dev)
    work = torch.empty(MLP_WORK, device=dev)
    out = torch.empty(MLP_PARAMS + 1, device=dev)
    losses = torch.empty(epochs, device=dev)
    for t in range(1, epochs + 1):
        mlp_loss_grad(Xd, yd, params, pos_weight, work, out)
        losses[t - 1] = out[MLP_PARAMS]
        mlp_adam(params, out, m, v, t, lr)
    return params.cpu().numpy(), losses.cpu().numpy()


def predict(X, params):
    import torch
    dev = torch.device("cuda")
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(dev)
    pd = torch.from_numpy(np.ascontiguousarray(params, dtype=np.float32)).to(dev)
    out = torch.empty(Xd.shape[0], device=dev)
    mlp_predict(Xd, pd, out)
    return out.cpu().numpy()


def late_refinements(model, steps, params=None, tau=0.5, dt=-1.0):
    """Advance `steps` adaptive steps with the proposal (params) or without it
    (params None) and return the library's counts: misses (patches the exact set
    reached that were not active during the step), over-refined and proposed
    patches, and the mean number of live nodes."""
    if params is None:
        model.set_learned(1)
    else:
        model.set_learned(2, params, tau)
    model.learn_stats(reset=True)
    live = 0.0
    for _ in range(steps):
        model.step(dt, 1, adapt=True)
        live += sum(model.stats()["live_nodes"].values())
    out = model.learn_stats(reset=True)
    out["live"] = live / max(steps, 1)
    model.set_learned(0)
    return out
