"""The learned refinement proposal on the GPU: the perceptron's loss, gradient,
Adam step and prediction against the FP64 oracle (oracle/mlp.py); the mask with a
proposal bit-exact against the oracle's mask with the same extra nodes; the
features against their definition recomputed from the library's own coefficient
arrays; and what a trained network gains over the plain criterion."""
import numpy as np
import pytest

from oracle import mlp
from test_gpu_parity import Pair

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch, torch.device("cuda")


def _problem(n=3000, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.gamma(1.0, 1.0, (n, mlp.F)).astype(np.float32)
    y = (rng.random(n) < 1 / (1 + np.exp(-(X[:, 0] - X[:, 4])))).astype(np.float32)
    params = (rng.normal(0, 0.4, mlp.NPARAM)).astype(np.float32)
    return X, y, params


def test_loss_and_gradient_match_oracle():
    import paper_1404_0405_gb300 as sww
    torch, dev = _torch()
    X, y, params = _problem()
    out = torch.empty(sww.MLP_PARAMS + 1, device=dev)
    work = torch.empty(sww.MLP_WORK, device=dev)
    sww.mlp_loss_grad(torch.from_numpy(X).to(dev), torch.from_numpy(y).to(dev), torch.from_numpy(params).to(dev),
                      2.5, work, out)
    got = out.cpu().numpy().astype(np.float64)
    W1, b1, w2, b2 = mlp.unpack(params)
    L, dW1, db1, dw2, db2 = mlp.loss_grad(X, y, W1, b1, w2, b2, 2.5)
    want = mlp.flat(dW1, db1, dw2, db2)
    assert abs(got[-1] / L - 1) < 1e-5
    assert np.max(np.abs(got[:-1] - want)) < 1e-5 * max(np.max(np.abs(want)), 1e-3)


def test_adam_and_predict_match_oracle():
    import paper_1404_0405_gb300 as sww
    torch, dev = _torch()
    X, y, params = _problem(500, 1)
    rng = np.random.default_rng(2)
    g = rng.normal(0, 1, mlp.NPARAM).astype(np.float32)
    m0 = rng.normal(0, 0.1, mlp.NPARAM).astype(np.float32)
    v0 = rng.random(mlp.NPARAM).astype(np.float32)
    p, m, v = (torch.from_numpy(a.copy()).to(dev) for a in (params, m0, v0))
    sww.mlp_adam(p, torch.from_numpy(g).to(dev), m, v, 3, 1e-2)
    want_p, want_m, want_v = mlp.adam(params.astype(np.float64), g.astype(np.float64), m0.astype(np.float64),
                                      v0.astype(np.float64), 3, 1e-2)
    assert np.max(np.abs(p.cpu().numpy() - want_p)) < 1e-6
    assert np.max(np.abs(m.cpu().numpy() - want_m)) < 1e-6
    out = torch.empty(X.shape[0], device=dev)
    sww.mlp_predict(torch.from_numpy(X).to(dev), torch.from_numpy(params).to(dev), out)
    assert np.max(np.abs(out.cpu().numpy() - mlp.predict(X, params))) < 1e-5


def _patch_nodes(lib, level, flags):
    """Library node ids of the proposed patches of a level (poles: last flag)."""
    N, E, T, npatch = lib.sizes(level)
    nelem = E // 3
    pp = nelem // npatch
    sel = np.zeros(N, dtype=bool)
    idx = np.flatnonzero(flags[:npatch])
    for P in idx:
        sel[P * pp:(P + 1) * pp] = True
    if flags[npatch]:
        sel[nelem:nelem + 2] = True
    return sel


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_proposal_mask_bit_exact(precision):
    P = Pair(2, 4, kind="jet", seed=4, precision=precision)
    P.adapt()
    rng = np.random.default_rng(7)
    act = P.lib.stats()["active_patches"]
    extra, sent = {}, {}
    for j in range(3, 5):
        if act[j] == 0:
            continue
        np1 = P.lib.sizes(j)[3] + 1
        flags = (rng.random(np1) < 0.15).astype(np.uint8)
        P.lib.propose(j, flags)
        sent[j] = flags
        extra[j] = P.maps[j].nodes_to_ora(_patch_nodes(P.lib, j, flags).astype(np.uint8)) > 0
    P.ora.adapt(extra=extra)
    P.lib.adapt()
    P.check_masks()
    if precision == "fp64":
        P.check_fields()
    for j in sent:
        assert np.array_equal(P.lib.patch_data(j, P.sww.P_PROPOSAL), sent[j])


def test_features_match_definition():
    """Features are computed between the coefficients and the mask of an
    adaptation, from the live set before that mask."""
    import paper_1404_0405_gb300 as sww
    P = Pair(2, 4, kind="jet", seed=2)
    lib = P.lib
    lib.set_learned(1)
    lib.adapt()
    pre = {j: lib.get(j, sww.NODE_FLAGS) for j in range(2, 5)}
    lib.adapt()
    st = lib.stats()
    eh = st["eps_h"]
    jmin, jmax = 2, 4
    for j in range(3, 5):
        N, E, T, npatch = lib.sizes(j)
        nelem = E // 3
        pp = nelem // npatch
        live_n = (pre[j] & 1) > 0
        hd = lib.get(j, sww.HDET)
        feats = lib.patch_data(j, sww.P_FEATURES)
        # even nodes carry no height coefficient (0 in the library's array)
        mh = np.array([np.max(np.abs(hd[Pp * pp:(Pp + 1) * pp][live_n[Pp * pp:(Pp + 1) * pp]]), initial=0.0)
                       for Pp in range(npatch)])
        assert np.allclose(feats[0, :npatch], np.log2(1 + mh / eh), rtol=1e-6, atol=1e-6)
        frac = np.array([live_n[Pp * pp:(Pp + 1) * pp].mean() for Pp in range(npatch)])
        assert np.allclose(feats[6, :npatch], frac, atol=1e-7)
        assert np.allclose(feats[7, :npatch], (j - jmin) / (jmax - jmin))
        # neighbour maxima: every patch's value is at least each neighbour's own feature
        # (the patch graph is symmetric), and a patch whose neighbours are all zero has 0
        assert np.all(feats[4] >= 0) and np.all(feats[5] >= 0)
    lib.set_learned(0)


def test_trained_proposal_against_plain_criterion():
    """Train on masks the method produces (three seeds), then run a held-out seed
    with and without the proposal.  The exact rules keep the last word, so the grid
    with the proposal contains the plain one (never fewer live points), and its
    late refinements (patches the exact set reaches that were not active during
    the step) are no more than the plain criterion's.  The counts are printed."""
    import paper_1404_0405_gb300 as sww
    from paper_1404_0405_gb300 import learn
    from lib_mapping import lib_edge_geometry
    import workloads

    def model(seed):
        m = sww.Model(3, 6, patch=4, eps=1e-2)
        xyz, en = m.grid(6)
        mid, tan = lib_edge_geometry(xyz, en)
        dh, u = workloads.Workload("jet", seed=seed).fields(xyz, mid, tan)
        m.set_state(dh, u)
        m.adapt()
        return m

    Xs, ys = [], []
    for seed in (20, 21, 22):
        X, y = learn.collect(model(seed), 15)
        Xs.append(X)
        ys.append(y)
    X, y = np.concatenate(Xs), np.concatenate(ys)
    params, losses = learn.train(X, y, epochs=300)
    assert losses[-1] < 0.5 * losses[0]
    p = learn.predict(X, params)
    recall = np.sum((p > 0.5) & (y > 0)) / max(1, y.sum())
    assert recall > 0.9
    plain = learn.late_refinements(model(99), 15)
    learned = learn.late_refinements(model(99), 15, params, 0.5)
    print(f"held-out: plain {plain}  learned {learned}  train recall {recall:.3f}")
    assert learned["misses"] <= plain["misses"]
    assert learned["live"] >= plain["live"]
