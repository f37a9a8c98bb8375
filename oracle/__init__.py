"""Plain FP64 CPU oracle of the conservative adaptive wavelet TRiSK method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import anything here.  The CUDA library
shares no code with this package, and this package imports nothing from the
library.

Aechtner, Kevlahan & Dubos, "A conservative adaptive wavelet method for the
shallow water equations on the sphere" (arXiv:1404.0405).  Modules:

* ``grid``      -- icosahedral nested grid and spherical geometry (Sec. 2.2, Table 1,
                   Sec. 4.1)
* ``trisk``     -- TRiSK operators and the shallow-water trend (Sec. 3.1)
* ``transform`` -- height lifting (Eqs. 1, 2, Rh), velocity transform, flux
                   restriction R_F = R_F0 + R'_F (Sec. 4.2, 4.3)
* ``adapt``     -- significance mask with neighbour/scale/closure rules (Sec. 2.3, 3.1)
* ``model``     -- adaptive RK step driver (Sec. 3.1), with the viscous form,
                   the prescribed-velocity mode of the advection test (Sec. 7.1)
                   and the full-level reconstruction
* ``mlp``       -- the learned proposal's perceptron: BF16 rounding, forward,
                   loss and gradient (an extension of Sec. 2.3)

Every function states the passage it follows.  Where the paper is silent,
garbled or ambiguous the reading taken is stated in the docstring.

Parity unpinned: the basic flux restriction R_F0 against the paper's own formula,
which rests on a figure absent from the text.  R_F0 is pinned only by the
commutation identity R_h(div F) = div(R_F F) and by the convergence of a smooth
flow's restricted flux to the coarse flux as the levels refine.
"""
