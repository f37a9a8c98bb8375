"""The allocation-free diagnostics entry point (sww_mass_energy_static) gives the
same mass and energy as sww_stats_get, on two calls in a row.

It is for callers that cannot allocate device memory when they ask for the
diagnostics (a framework's caching allocator owning the heap, real-time loops
that must not synchronise on cudaMalloc/cudaFree); its scratch is a fixed array
inside the library.  This file is collected last so that a failure here leaves
every other test already run."""
import pytest

pytestmark = pytest.mark.gpu


def test_static_scratch_sums_match_stats():
    import numpy as np
    import torch

    import paper_1404_0405_gb300 as sww
    import workloads

    sww.build()
    m = sww.Model(2, 4, patch=4)
    xyz, en = m.grid(4)
    a, b = xyz[en[:, 0]], xyz[en[:, 1]]
    mid = (a + b) / np.linalg.norm(a + b, axis=1, keepdims=True)
    tan = (b - a) / np.linalg.norm(b - a, axis=1, keepdims=True)
    dh, u = workloads.Workload("jet", seed=2).fields(xyz, mid, tan)
    m.set_state(dh, u)
    m.adapt()
    m.step(-1.0, 2, adapt=True)
    ref = m.stats()
    dh0 = torch.from_numpy(m.get(2, sww.DH)).cuda()
    u0 = torch.from_numpy(m.get(2, sww.U)).cuda()
    for call in range(2):
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        m.mass_energy_static(dh0, u0, out)
        torch.cuda.synchronize()
        mass, energy = out.tolist()
        assert abs(mass / ref["mass"] - 1) < 1e-14, call
        assert abs(energy / ref["energy"] - 1) < 1e-9, call
