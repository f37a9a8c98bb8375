"""The allocation-free diagnostics entry point (sww_mass_energy_static) gives the
same mass and energy as sww_stats_get, on two calls in a row.

It is for callers that cannot allocate device memory when they ask for the
diagnostics (a framework's caching allocator owning the heap, real-time loops
that must not synchronise on cudaMalloc/cudaFree); its scratch is a fixed array
inside the library.  This file is collected last so that a failure here leaves
every other test already run."""
import pytest

pytestmark = pytest.mark.gpu


def _stepped(precision):
    import numpy as np

    import paper_1404_0405_gb300 as sww
    import workloads

    sww.build()
    m = sww.Model(2, 4, patch=4, precision=precision)
    xyz, en = m.grid(4)
    a, b = xyz[en[:, 0]], xyz[en[:, 1]]
    mid = (a + b) / np.linalg.norm(a + b, axis=1, keepdims=True)
    tan = (b - a) / np.linalg.norm(b - a, axis=1, keepdims=True)
    dh, u = workloads.Workload("jet", seed=2).fields(xyz, mid, tan)
    m.set_state(dh, u)
    m.adapt()
    m.step(-1.0, 2, adapt=True)
    return m


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_scratch_sums_match_stats(precision):
    """Both calls reduce the same FP64 values (an FP32 state promoted exactly) with
    the same compensated tree and the same final roundings, so the results are
    equal bit for bit, call after call."""
    import torch

    import paper_1404_0405_gb300 as sww

    m = _stepped(precision)
    ref = m.stats()
    dh0 = torch.from_numpy(m.get(2, sww.DH)).cuda()
    u0 = torch.from_numpy(m.get(2, sww.U)).cuda()
    for call in range(2):
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        m.mass_energy_static(dh0, u0, out)
        torch.cuda.synchronize()
        mass, energy = out.tolist()
        assert mass == ref["mass"], (call, mass, ref["mass"])
        assert energy == ref["energy"], (call, energy, ref["energy"])


def test_static_scratch_refuses_bad_arguments():
    """Tensors of the wrong kind are refused in the binding (the C call cannot
    see lengths), host pointers in the library; nothing is launched."""
    import numpy as np
    import torch

    import paper_1404_0405_gb300 as sww

    m = _stepped("fp64")
    N, E, _, _ = m.sizes(2)
    dh = torch.zeros(N, dtype=torch.float64, device="cuda")
    u = torch.zeros(E, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for bad in (dict(dh=dh[:-1]), dict(u=u.float()), dict(out=out.cpu()), dict(dh=np.zeros(N)),
                dict(u=torch.zeros(2 * E, dtype=torch.float64, device="cuda")[::2])):
        args = dict(dh=dh, u=u, out=out)
        args.update(bad)
        with pytest.raises(sww.SwwError) as ei:
            m.mass_energy_static(args["dh"], args["u"], args["out"])
        assert ei.value.code == sww.E_ARG
    host = np.zeros(N)
    rc = sww.load().sww_mass_energy_static(m._h, host.ctypes.data, u.data_ptr(), out.data_ptr())
    assert rc == sww.E_ARG
    rc = sww.load().sww_mass_energy_static(m._h, None, u.data_ptr(), out.data_ptr())
    assert rc == sww.E_ARG


def test_static_scratch_refuses_large_jmin():
    """A Jmin level above 1,048,576 nodes (Jmin = 9: 2,621,442) does not fit the
    static scratch and is refused with SWW_E_ARG before any launch."""
    import torch

    import paper_1404_0405_gb300 as sww

    sww.build()
    m = sww.Model(9, 9, patch=8)
    N, E, _, _ = m.sizes(9)
    dh = torch.zeros(N, dtype=torch.float64, device="cuda")
    u = torch.zeros(E, dtype=torch.float64, device="cuda")
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    with pytest.raises(sww.SwwError) as ei:
        m.mass_energy_static(dh, u, out)
    assert ei.value.code == sww.E_ARG and "1,048,576" in str(ei.value)
    assert out.tolist() == [-1.0, -1.0]
