"""GB300 adaptive wavelet TRiSK shallow-water library (arXiv:1404.0405), Python binding.

A thin ctypes layer over the C ABI in ``include/sww.h``: argument marshalling
only.  Every step of the method runs in the CUDA kernels of ``libsww.so``; there
is no CPU fallback, and the calls raise if the library or a GPU is missing.
Device pointers may be passed as torch CUDA tensors; the default stream is
torch's current stream when torch has CUDA.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .buildlib import LIB, build

__all__ = ["Model", "SwwError", "step_ensemble", "mlp_loss_grad", "mlp_adam", "mlp_predict", "load", "lib_path", "DH", "U", "DH_T", "U_T", "NODE_FLAGS", "EDGE_FLAGS",
           "HDET", "UDET_E", "UDET_I", "SIG", "LIVE", "GHOST", "COVERED"]

DH, U, DH_T, U_T, NODE_FLAGS, EDGE_FLAGS, HDET, UDET_E, UDET_I, SIG = range(10)
LIVE, GHOST, COVERED = 1, 2, 4
MLP_FEATURES, MLP_HIDDEN = 8, 32
MLP_PARAMS = MLP_FEATURES * MLP_HIDDEN + 2 * MLP_HIDDEN + 1
MLP_WORK = 256 * (MLP_PARAMS + 1)
P_FEATURES, P_EXACT, P_PROPOSAL, P_ACTIVE = range(4)
RK4, SSP43 = 0, 1
# bytes a batched ensemble step copies back to the host per member: its time step,
# error flag, and the active patch and live node counts of levels 0..15
BATCH_OUT_BYTES = 144

EXPORTS = ["sww_create", "sww_destroy", "sww_level_sizes", "sww_get_grid", "sww_set_state", "sww_adapt",
           "sww_mask_from_coeffs", "sww_rhs", "sww_step", "sww_get_level", "sww_set_level", "sww_get_patches",
           "sww_stats_get", "sww_last_error", "sww_profile", "sww_profile_read", "sww_mass_energy_static",
           "sww_create_shared", "sww_step_ensemble", "sww_set_learned", "sww_propose", "sww_get_patch_data",
           "sww_learn_stats", "sww_mlp_loss_grad", "sww_mlp_adam", "sww_mlp_predict", "sww_forward", "sww_inverse",
           "sww_get_coeffs", "sww_set_coeffs", "sww_get_state", "sww_save", "sww_load", "sww_set_state_level",
           "sww_get_mask", "sww_barrier_fault", "sww_live_nodes"]
KERNEL_CLASSES = ["trend", "irregular", "node", "reserved", "restrict", "update", "fill", "partial", "coeff", "mask",
                  "inverse", "dt", "stage"]


class SwwError(RuntimeError):
    """A failed call; ``code`` is the library's negative status (SWW_E_*)."""

    def __init__(self, msg, code=0):
        super().__init__(msg)
        self.code = code


E_ARG, E_CUDA, E_POOL, E_TIMEOUT, E_STATE, E_NUMERIC = -1, -2, -3, -4, -5, -6


class Config(ctypes.Structure):
    _fields_ = [("jmin", ctypes.c_int), ("jmax", ctypes.c_int), ("radius", ctypes.c_double),
                ("omega", ctypes.c_double), ("g", ctypes.c_double), ("H", ctypes.c_double),
                ("patch", ctypes.c_int), ("rk", ctypes.c_int), ("cfl", ctypes.c_double), ("eps", ctypes.c_double),
                ("blocks_per_sm", ctypes.c_int), ("precision", ctypes.c_int), ("persistent", ctypes.c_int),
                ("mask", ctypes.c_int), ("nu", ctypes.c_double), ("advect", ctypes.c_int), ("regime", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("dt", ctypes.c_double), ("mass", ctypes.c_double),
                ("energy", ctypes.c_double), ("eps_h", ctypes.c_double), ("eps_u", ctypes.c_double),
                ("steps", ctypes.c_int64), ("live_nodes", ctypes.c_int64 * 16), ("ghost_nodes", ctypes.c_int64 * 16),
                ("live_edges", ctypes.c_int64 * 16), ("active_patches", ctypes.c_int64 * 16),
                ("kernel_launches", ctypes.c_int64)]


_lib = None


def lib_path() -> str:
    return LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libsww.so (building it in-tree first when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        if not build_if_missing:
            raise SwwError(f"{LIB} is missing; run paper_1404_0405_gb300.buildlib")
        build()
    lib = ctypes.CDLL(LIB)
    P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_int64)
    sig = {
        "sww_create": [ctypes.POINTER(Config), P, ctypes.POINTER(P)],
        "sww_destroy": [P],
        "sww_level_sizes": [P, I, I64, I64, I64, I64],
        "sww_get_grid": [P, I, P, P],
        "sww_set_state": [P, P, P, I],
        "sww_adapt": [P, D, D],
        "sww_mask_from_coeffs": [P, P, P, P, D, D],
        "sww_rhs": [P],
        "sww_step": [P, D, I, I],
        "sww_get_level": [P, I, I, P],
        "sww_set_level": [P, I, P, P],
        "sww_get_patches": [P, I, P, ctypes.POINTER(ctypes.c_int32)],
        "sww_live_nodes": [P, ctypes.POINTER(ctypes.c_int64)],
        "sww_stats_get": [P, ctypes.POINTER(Stats)],
        "sww_last_error": [ctypes.c_char_p, ctypes.c_size_t],
        "sww_profile": [P, ctypes.c_uint32],
        "sww_profile_read": [P, ctypes.POINTER(ctypes.c_double), I64],
        "sww_mass_energy_static": [P, P, P, P],
        "sww_create_shared": [ctypes.POINTER(Config), P, P, ctypes.POINTER(P)],
        "sww_step_ensemble": [ctypes.POINTER(P), I, D, I, I],
        "sww_set_learned": [P, I, P, ctypes.c_float],
        "sww_propose": [P, I, P],
        "sww_get_patch_data": [P, I, I, P],
        "sww_learn_stats": [P, I64, I],
        "sww_mlp_loss_grad": [P, P, ctypes.c_int64, P, ctypes.c_float, P, P, P],
        "sww_mlp_adam": [P, P, P, P, I, ctypes.c_float, P],
        "sww_mlp_predict": [P, ctypes.c_int64, P, P, P],
        "sww_forward": [P],
        "sww_inverse": [P],
        "sww_get_coeffs": [P, I, P, P, P],
        "sww_set_coeffs": [P, I, P, P, P],
        "sww_get_state": [P, I, P, P],
        "sww_save": [P, ctypes.c_char_p],
        "sww_load": [P, ctypes.c_char_p],
        "sww_set_state_level": [P, I, P, P, I],
        "sww_get_mask": [P, I, P, P],
        "sww_barrier_fault": [P, ctypes.c_longlong, I],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc):
    if rc != 0:
        buf = ctypes.create_string_buffer(1024)
        _lib.sww_last_error(buf, 1024)
        raise SwwError(f"sww error {rc}: {buf.value.decode(errors='replace')}", rc)


def _ptr(a):
    """(pointer, is_device) of a numpy array or a torch tensor."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(ctypes.c_void_p), 0
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda)
    raise TypeError(type(a))


def _default_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(None)


def step_ensemble(models, dt=-1.0, nsteps=1, adapt=True):
    """nsteps steps of every member; the members' steps overlap on the GPU
    (sww_step_ensemble)."""
    hs = (ctypes.c_void_p * len(models))(*[m._h.value for m in models])
    _check(load().sww_step_ensemble(hs, len(models), float(dt), int(nsteps), int(bool(adapt))))


def mlp_loss_grad(X, y, params, pos_weight, work, out, stream=None):
    """Device tensors: X[n, 8], y[n], params[MLP_PARAMS], work[MLP_WORK], out[MLP_PARAMS + 1]
    (gradient, then the mean loss) -- sww_mlp_loss_grad."""
    st = stream if stream is not None else _default_stream()
    _check(load().sww_mlp_loss_grad(_ptr(X)[0], _ptr(y)[0], X.shape[0], _ptr(params)[0], float(pos_weight),
                                    _ptr(work)[0], _ptr(out)[0], st))


def mlp_adam(params, grad, m, v, t, lr, stream=None):
    st = stream if stream is not None else _default_stream()
    _check(load().sww_mlp_adam(_ptr(params)[0], _ptr(grad)[0], _ptr(m)[0], _ptr(v)[0], int(t), float(lr), st))


def mlp_predict(X, params, out, stream=None):
    st = stream if stream is not None else _default_stream()
    _check(load().sww_mlp_predict(_ptr(X)[0], X.shape[0], _ptr(params)[0], _ptr(out)[0], st))


class Model:
    """One adapted grid Jmin..Jmax and its state on the GPU (sww_create)."""

    def __init__(self, jmin, jmax, radius=6.371e6, omega=7.292e-5, g=9.80616, H=1.0e4, patch=8, rk="rk4",
                 cfl=0.8, eps=1e-2, stream=None, share=None, blocks_per_sm=0, precision="fp64", persistent=True,
                 mask="lists", nu=0.0, advect=False, regime=0):
        """share: another Model whose grid and tables this one reuses (sww_create_shared).
        persistent: True/"auto", "phased" (ensemble steps as one launch per
        phase over all members) or False/"never" (see sww_config.persistent).  advect: prescribed velocity
        (see sww_config.advect).  regime: 1 scales the thresholds by eps^{3/2}
        (see sww_config.regime)."""
        lib = load()
        self.jmin, self.jmax = jmin, jmax
        self.cfg = Config(jmin, jmax, radius, omega, g, H, patch, RK4 if rk == "rk4" else SSP43, cfl, eps,
                          blocks_per_sm, {"fp64": 0, "fp32": 1}[precision],
                          {True: 0, "auto": 0, "phased": 3, False: -1, "never": -1}[persistent],
                          {"lists": 0, "dense": 1}[mask], float(nu), int(bool(advect)), int(regime))
        h = ctypes.c_void_p()
        st = stream if stream is not None else _default_stream()
        if share is None:
            _check(lib.sww_create(ctypes.byref(self.cfg), st, ctypes.byref(h)))
        else:
            _check(lib.sww_create_shared(ctypes.byref(self.cfg), st, share._h, ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().sww_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ grid
    def sizes(self, level):
        out = [ctypes.c_int64() for _ in range(4)]
        _check(load().sww_level_sizes(self._h, level, *[ctypes.byref(o) for o in out]))
        return tuple(o.value for o in out)

    def grid(self, level):
        """(node_xyz[N,3] unit vectors, edge_nodes[E,2] origin/end)."""
        N, E, _, _ = self.sizes(level)
        xyz = np.empty((N, 3))
        en = np.empty((E, 2), dtype=np.int32)
        _check(load().sww_get_grid(self._h, level, _ptr(xyz)[0], _ptr(en)[0]))
        return xyz, en

    # ------------------------------------------------------------------ state
    def set_state(self, dh, u, level=None):
        """Fields on the full level Jmax, or on `level` (levels above it start
        empty); numpy host arrays or torch CUDA tensors, float64."""
        if isinstance(dh, np.ndarray):
            dh = np.ascontiguousarray(dh, dtype=np.float64)
            u = np.ascontiguousarray(u, dtype=np.float64)
        pd, dev = _ptr(dh)
        pu, _ = _ptr(u)
        if level is None:
            _check(load().sww_set_state(self._h, pd, pu, dev))
        else:
            _check(load().sww_set_state_level(self._h, int(level), pd, pu, dev))

    def adapt(self, eps_h=-1.0, eps_u=-1.0):
        _check(load().sww_adapt(self._h, eps_h, eps_u))

    def mask_from_coeffs(self, hdet, udet_e, udet_i, eps_h, eps_u):
        """hdet/udet_e/udet_i: dicts level -> array (level Jmin+1..Jmax)."""
        cat = lambda d: np.ascontiguousarray(np.concatenate([d[j] for j in range(self.jmin + 1, self.jmax + 1)]),
                                             dtype=np.float64)
        a, b, c = cat(hdet), cat(udet_e), cat(udet_i)
        _check(load().sww_mask_from_coeffs(self._h, _ptr(a)[0], _ptr(b)[0], _ptr(c)[0], eps_h, eps_u))

    def rhs(self):
        _check(load().sww_rhs(self._h))

    def step(self, dt=-1.0, nsteps=1, adapt=True):
        _check(load().sww_step(self._h, float(dt), int(nsteps), int(bool(adapt))))

    def get(self, level, what):
        N, E, _, _ = self.sizes(level)
        if what in (DH, DH_T, HDET):
            out = np.empty(N)
        elif what in (U, U_T, UDET_I):
            out = np.empty(E)
        elif what == UDET_E:
            out = np.empty(self.sizes(level - 1)[1])
        elif what in (NODE_FLAGS, SIG):
            out = np.empty(N, dtype=np.uint8)
        elif what == EDGE_FLAGS:
            out = np.empty(E, dtype=np.uint8)
        else:
            raise ValueError(what)
        _check(load().sww_get_level(self._h, level, what, _ptr(out)[0]))
        return out

    def mask(self, level):
        """(node flags [N_j], edge flags [E_j]) of level j: bit 0 live, 1 ghost, 2 covered."""
        N, E, _, _ = self.sizes(level)
        nodes, edges = np.empty(N, dtype=np.uint8), np.empty(E, dtype=np.uint8)
        _check(load().sww_get_mask(self._h, level, nodes.ctypes.data_as(ctypes.c_void_p),
                                   edges.ctypes.data_as(ctypes.c_void_p)))
        return nodes, edges

    def forward(self):
        _check(load().sww_forward(self._h))

    def inverse(self):
        _check(load().sww_inverse(self._h))

    def coeffs(self, level):
        """(hdet[N_j], udet_e[E_{j-1}], udet_i[E_j]) of level j > Jmin."""
        N, E, _, _ = self.sizes(level)
        Ec = self.sizes(level - 1)[1]
        out = (np.empty(N), np.empty(Ec), np.empty(E))
        _check(load().sww_get_coeffs(self._h, level, *[o.ctypes.data_as(ctypes.c_void_p) for o in out]))
        return out

    def set_coeffs(self, level, hdet=None, udet_e=None, udet_i=None):
        args = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in (hdet, udet_e, udet_i)]
        _check(load().sww_set_coeffs(self._h, level, *[None if a is None else a.ctypes.data_as(ctypes.c_void_p)
                                                         for a in args]))

    def get_state(self, level):
        """(dh[N_j], u[E_j]) on the full level j (zero coefficients away from live points)."""
        N, E, _, _ = self.sizes(level)
        dh, u = np.empty(N), np.empty(E)
        _check(load().sww_get_state(self._h, level, dh.ctypes.data_as(ctypes.c_void_p),
                                    u.ctypes.data_as(ctypes.c_void_p)))
        return dh, u

    def save(self, path):
        _check(load().sww_save(self._h, os.fsencode(path)))

    def load(self, path):
        _check(load().sww_load(self._h, os.fsencode(path)))

    def set_level(self, level, dh=None, u=None):
        a = None if dh is None else np.ascontiguousarray(dh, dtype=np.float64)
        b = None if u is None else np.ascontiguousarray(u, dtype=np.float64)
        _check(load().sww_set_level(self._h, level, None if a is None else _ptr(a)[0], None if b is None else _ptr(b)[0]))

    def live_nodes(self):
        """Live nodes over every level as of the last set_state, adapt or step
        (sww_live_nodes: no device work)."""
        n = ctypes.c_int64()
        _check(load().sww_live_nodes(self._h, ctypes.byref(n)))
        return n.value

    def patches(self, level):
        n = self.sizes(level)[3]
        out = np.empty(n, dtype=np.int32)
        cnt = ctypes.c_int32()
        _check(load().sww_get_patches(self._h, level, _ptr(out)[0], ctypes.byref(cnt)))
        return out[: cnt.value].copy()

    def profile(self, classes=()):
        """Start recording CUDA-event durations for the named kernel classes."""
        mask = 0
        for c in classes:
            mask |= 1 << KERNEL_CLASSES.index(c)
        _check(load().sww_profile(self._h, mask))

    def profile_read(self):
        """{class: (total ms, launches)} since profile() / the last read."""
        ms = (ctypes.c_double * len(KERNEL_CLASSES))()
        n = (ctypes.c_int64 * len(KERNEL_CLASSES))()
        _check(load().sww_profile_read(self._h, ms, n))
        return {c: (ms[i], n[i]) for i, c in enumerate(KERNEL_CLASSES)}

    def mass_energy_static(self, dh, u, out):
        """Mass and energy of level Jmin into out[2] without any device allocation
        (dh[N_Jmin], u[E_Jmin], out[2]: contiguous torch CUDA float64 tensors;
        asynchronous on the caller's stream).  The C call cannot see array lengths,
        so the tensors are checked here before it."""
        N, E, _, _ = self.sizes(self.jmin)
        for name, t, n in (("dh", dh, N), ("u", u, E), ("out", out, 2)):
            ok = (hasattr(t, "is_cuda") and t.is_cuda and str(t.dtype) == "torch.float64" and t.is_contiguous()
                  and t.numel() == n)
            if not ok:
                raise SwwError(f"mass_energy_static: {name} must be a contiguous CUDA float64 tensor of {n} values",
                               E_ARG)
        _check(load().sww_mass_energy_static(self._h, _ptr(dh)[0], _ptr(u)[0], _ptr(out)[0]))

    def barrier_fault(self, spin_cycles=0, skip_block=-1):
        """Fault injection for tests of the persistent stage's bounded barrier
        (sww_barrier_fault): waits give up after spin_cycles clock cycles (0: the
        default) and block skip_block leaves without arriving (-1: none)."""
        _check(load().sww_barrier_fault(self._h, int(spin_cycles), int(skip_block)))

    # ------------------------------------------------------------------ learned proposal
    def set_learned(self, mode, params=None, tau=0.5):
        """mode 0 off, 1 features only, 2 features and proposal (params: MLP_PARAMS floats)."""
        buf = None
        if params is not None:
            buf = np.ascontiguousarray(np.asarray(params, dtype=np.float32).ravel())
            assert buf.size == MLP_PARAMS
        _check(load().sww_set_learned(self._h, int(mode), None if buf is None else _ptr(buf)[0], float(tau)))

    def propose(self, level, flags):
        f = np.ascontiguousarray(np.asarray(flags, dtype=np.uint8))
        assert f.size == self.sizes(level)[3] + 1
        _check(load().sww_propose(self._h, level, _ptr(f)[0]))

    def patch_data(self, level, what):
        np1 = self.sizes(level)[3] + 1
        if what == P_FEATURES:
            out = np.empty((MLP_FEATURES, np1), dtype=np.float32)
        elif what in (P_EXACT, P_PROPOSAL):
            out = np.empty(np1, dtype=np.uint8)
        elif what == P_ACTIVE:
            out = np.empty(np1 - 1, dtype=np.uint8)
        else:
            raise ValueError(what)
        _check(load().sww_get_patch_data(self._h, level, what, _ptr(out)[0]))
        return out

    def learn_stats(self, reset=False):
        out = (ctypes.c_int64 * 3)()
        _check(load().sww_learn_stats(self._h, out, int(bool(reset))))
        return {"misses": out[0], "over": out[1], "proposed": out[2]}

    def stats(self):
        st = Stats()
        _check(load().sww_stats_get(self._h, ctypes.byref(st)))
        lv = range(self.jmin, self.jmax + 1)
        return {"t": st.t, "dt": st.dt, "mass": st.mass, "energy": st.energy, "eps_h": st.eps_h, "eps_u": st.eps_u,
                "steps": st.steps, "live_nodes": {j: st.live_nodes[j] for j in lv},
                "ghost_nodes": {j: st.ghost_nodes[j] for j in lv}, "live_edges": {j: st.live_edges[j] for j in lv},
                "active_patches": {j: st.active_patches[j] for j in lv}, "kernel_launches": st.kernel_launches}
