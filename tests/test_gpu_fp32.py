"""FP32 form against the FP64 oracle: fields, stencils and transforms in FP32
(weights rounded once from the FP64 tables); thresholds, time step and the
mass/energy sums from FP64 arithmetic on the FP32 values.

Stated errors (ℓ∞ relative to the field's ℓ∞, Jmin=2..Jmax=4 jet):
  * initial restriction of the FP64 input: <= FP32_INIT (a few FP32 ulps);
  * after adaptation and three RK4 steps: <= FP32_STEP per field;
  * mass: relative drift <= FP32_MASS over the steps (the FP64 form: 1e-14).
Integer work stays exact: a mask built from identical coefficients is
bit-identical, and the patch lists follow the flags."""
import numpy as np
import pytest

from test_gpu_parity import Pair, rel_err

pytestmark = pytest.mark.gpu

FP32_INIT = 2e-6
FP32_STEP = 2e-5
FP32_MASS = 1e-7


def _errors(P, which="state"):
    out = {}
    for j in range(P.jmin, P.jmax + 1):
        M = P.maps[j]
        a = M.nodes_to_ora(P.lib.get(j, P.sww.DH))
        b = M.edges_to_ora(P.lib.get(j, P.sww.U))
        mn = P.ora.live_n[j] | P.ora.ghost_n[j]
        me = P.ora.live_e[j] | P.ora.ghost_e[j]
        out[f"dh{j}"] = rel_err(a[mn], P.ora.dh[j][mn]) if mn.any() else 0.0
        out[f"u{j}"] = rel_err(b[me], P.ora.u[j][me]) if me.any() else 0.0
    return out


def test_fp32_initial_restriction():
    P = Pair(2, 4, precision="fp32")
    err = _errors(P)
    assert max(err.values()) < FP32_INIT, err
    P.check_masks()


def test_fp32_mask_from_identical_coefficients():
    """Coefficients exactly representable in FP32 on both sides: bit-identical mask."""
    P = Pair(2, 4, kind="jet", seed=5, precision="fp32")
    hdet, ue, ui = P.ora.details()
    r32 = lambda d: {j: np.asarray(np.asarray(v, dtype=np.float32), dtype=np.float64) for j, v in d.items()}
    hdet, ue, ui = r32(hdet), r32(ue), r32(ui)
    lib_h, lib_e, lib_i = {}, {}, {}
    for j in range(3, 5):
        Mf, Mc = P.maps[j], P.maps[j - 1]
        VS = P.ora.VS[j]
        full_h = np.zeros(P.Hy.levels[j].N)
        full_h[P.Hy.odd[j]] = np.nan_to_num(hdet[j])
        lib_h[j] = Mf.nodes_to_lib(full_h)
        lib_e[j] = np.nan_to_num(ue[j])[Mc.edge]
        full_i = np.zeros(P.Hy.levels[j].E)
        full_i[VS.int_edge.ravel()] = np.nan_to_num(ui[j]).ravel()
        lib_i[j] = Mf.edges_to_lib(full_i)
    eh, eu = 4.0, 0.3
    sig = P.ora.significance(hdet, ue, ui, eh, eu)
    from oracle import adapt
    live_n, live_e = adapt.build_mask(P.Hy, sig)
    P.ora.apply_mask(live_n, live_e, hdet, ue, ui)
    P.lib.mask_from_coeffs(lib_h, lib_e, lib_i, eh, eu)
    for j in range(3, 5):
        s = P.maps[j].nodes_to_ora(P.lib.get(j, P.sww.SIG))
        assert np.array_equal(s > 0, sig[j])
    P.check_masks()
    err = _errors(P)
    assert max(err.values()) < FP32_INIT, err


def test_fp32_adaptive_steps():
    P = Pair(2, 4, precision="fp32")
    P.adapt()
    P.check_masks()
    m0 = P.ora.mass()
    for _ in range(3):
        dt = P.ora.dt_cfl()
        P.ora.step(dt)
        P.lib.step(dt, 1, adapt=True)
        P.check_masks()
    err = _errors(P)
    print("FP32 errors after 3 RK4 steps:", {k: f"{v:.2e}" for k, v in err.items()})
    assert max(err.values()) < FP32_STEP, err
    st = P.lib.stats()
    assert abs(st["mass"] / m0 - 1) < FP32_MASS
    assert abs(st["energy"] / P.ora.energy() - 1) < 1e-5
