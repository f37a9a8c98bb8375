"""Pin of the oracle's time schemes (Sec. 3.1): on a fixed grid the error of the
depth after a fixed time falls by 2^p when the step halves, p = 4 for classical
RK4 and p = 3 for the four-stage SSP scheme (errors against a run with an eighth
of the step).  A wrong stage weight or a stage evaluated at the wrong state
lowers the order and fails this."""
import numpy as np
import pytest

import workloads
from oracle import grid, model


@pytest.mark.parametrize("rk,lo,hi", [("rk4", 13.0, 20.0), ("ssp43", 6.0, 10.0)])
def test_time_scheme_order(rk, lo, hi):
    Hy = grid.Hierarchy(3, 3)
    L = Hy.levels[3]
    dh, u = workloads.Workload("harmonic", seed=2).fields(L.xyz, L.edge_midpoints(), L.edge_tangents())

    def run(dt, T=7200.0):
        M = model.Model(Hy, eps=0.0, rk=rk)
        M.set_uniform(dh, u)
        M.adapt()
        for _ in range(int(round(T / dt))):
            M.step(dt, adapt_after=False)
        return M.dh[3]

    ref = run(75.0)
    errs = [np.abs(run(dt) - ref).max() for dt in (1200.0, 600.0, 300.0)]
    # measured: rk4 17.5, 17.7; ssp43 7.4, 7.9
    for a, b in zip(errs, errs[1:]):
        assert lo < a / b < hi, (rk, errs)


@pytest.mark.parametrize("rk,lo", [("rk4", 20.0), ("ssp43", 6.0)])
def test_energy_drift_is_the_time_scheme_only(rk, lo):
    """The TRiSK discretisation conserves the energy of Sec. 7.2 in continuous
    time (energy-neutral Coriolis term, kinetic energy and Bernoulli function
    consistent with div and grad), so on a fixed grid the energy drift over a
    fixed time vanishes as the step halves (measured ratios 31-32 for RK4, 7.7-7.9
    for SSPRK(4,3)); a spatial error in K, B or the Coriolis weights would leave
    a floor that does not fall."""
    Hy = grid.Hierarchy(3, 3)
    L = Hy.levels[3]
    dh, u = workloads.Workload("harmonic", seed=2).fields(L.xyz, L.edge_midpoints(), L.edge_tangents())
    drift = []
    for dt in (1200.0, 600.0, 300.0):
        M = model.Model(Hy, eps=0.0, rk=rk)
        M.set_uniform(dh, u)
        M.adapt()
        e0 = M.energy()
        for _ in range(int(round(7200.0 / dt))):
            M.step(dt, adapt_after=False)
        drift.append(abs(M.energy() / e0 - 1))
    for a, b in zip(drift, drift[1:]):
        assert a / b > lo, (rk, drift)
    assert drift[-1] < (1e-6 if rk == "rk4" else 1e-4)
