"""Parity at the benchmark's kernel configuration: an ensemble of members on a
shared grid stepped through the batched phases (persistent = "phased", the
benchmark's chosen form), patch side 8, against one FP64 oracle per member.

At Jmin=2..Jmax=6 the finest level holds 640 patches of 8 x 8 of which only a
part is active, so the mask's one-ring candidate lists (patch side >= 8) prune,
as at the benchmark's size; levels 2 and 3 are whole-lozenge patches.

Bar (as in test_gpu_parity and test_gpu_fp32): masks bit-exact; FP64 fields
within 1e-12 of the field's maximum and the CFL time step within 1e-12; FP32
fields within the stated FP32 bound after the three steps, taken with a given
time step common to the members and the oracles."""
import numpy as np
import pytest

from test_gpu_fp32 import FP32_STEP, _errors
from test_gpu_parity import Pair

pytestmark = pytest.mark.gpu

SEEDS = (0, 1, 2)


def _ensemble(precision):
    import paper_1404_0405_gb300 as sww
    sww.build()
    base = sww.Model(2, 6, patch=8)
    pairs = [Pair(2, 6, seed=s, patch=8, precision=precision, persistent="phased", share=base) for s in SEEDS]
    return sww, pairs


def test_phased_ensemble_fp64_matches_oracle():
    sww, pairs = _ensemble("fp64")
    for P in pairs:
        P.adapt()
        P.check_masks()
        assert P.lib.stats()["active_patches"][6] < P.lib.sizes(6)[3]   # level 6 is pruned
    m0 = [P.lib.stats()["mass"] for P in pairs]
    for _ in range(3):
        dts = [P.ora.dt_cfl() for P in pairs]
        for P, dt in zip(pairs, dts):
            P.ora.step(dt)
        sww.step_ensemble([P.lib for P in pairs], -1.0, 1, True)
        for P, dt in zip(pairs, dts):
            assert abs(P.lib.stats()["dt"] / dt - 1) < 1e-12
            P.check_masks()
            P.check_fields()
    for P, m in zip(pairs, m0):
        assert abs(P.lib.stats()["mass"] / m - 1) < 1e-14


def test_phased_ensemble_fp32_matches_oracle():
    sww, pairs = _ensemble("fp32")
    for P in pairs:
        P.adapt()
        P.check_masks()
    for _ in range(3):
        dt = min(P.ora.dt_cfl() for P in pairs)
        for P in pairs:
            P.ora.step(dt)
        sww.step_ensemble([P.lib for P in pairs], dt, 1, True)
        for P in pairs:
            P.check_masks()
    worst = {}
    for P in pairs:
        err = _errors(P)
        worst = {k: max(worst.get(k, 0.0), v) for k, v in err.items()}
        assert max(err.values()) < FP32_STEP, err
    print("FP32 phased ensemble, worst member error per field after 3 RK4 steps:",
          {k: f"{v:.2e}" for k, v in worst.items()})
