"""Thin ctypes binding of libqlbm.so (include/qlbm.h), with the same entry-point names.

Argument marshalling only: every step of the solver runs in the CUDA library.
PyTorch, when present, supplies the device allocator (its caching allocator)
and the stream.  There is no fallback: if the library has not been built this
module raises on first use.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqlbm.so")

QL_OK, QL_EINVAL, QL_ENOMEM, QL_ECUDA, QL_ENONPHYSICAL, QL_ETIMEOUT, QL_EUNSUPPORTED = range(7)
QL_FP64, QL_FP32 = 0, 1
QL_SUMS_DFP32, QL_SUMS_FP64 = 0, 1
QL_LAUNCH_AUTO, QL_LAUNCH_STAGES, QL_LAUNCH_RUN = 0, 1, 2
QL_BC_PERIODIC, QL_BC_FIXED = 0, 1
QL_INIT_SOUND, QL_INIT_RIEMANN, QL_INIT_SHOCK, QL_INIT_FIELDS = 0, 1, 2, 3
QL_PR_CONST, QL_PR_DENSE = 0, 1
QL_CHI_SET, QL_CHI_RET_FM = 0, 1
QL_FM_MAX_HALFWIDTH = 256
SUPPORTED_Q = (8, 16, 20, 24, 32, 40)  # tiled kernels; other even Q <= 200 run the generic FP64 path
MAX_Q = 200
SUPPORTED_BATCH_Q = (8, 16, 24, 32)
EXPORTED = ("ql_create", "ql_step", "ql_sync", "ql_moments", "ql_totals", "ql_get_state", "ql_set_state",
            "ql_load_fields", "ql_rhs", "ql_state_device", "ql_info", "ql_velocity_set", "ql_eta_of_denseness",
            "ql_sound_speed2", "ql_rankine_hugoniot", "ql_riemann_exact", "ql_destroy", "ql_last_error",
            "ql_batch_create", "ql_batch_tune", "ql_batch_run", "ql_batch_sync", "ql_batch_moments",
            "ql_batch_get_state", "ql_batch_info", "ql_batch_destroy", "ql_batch_last_error", "ql_step_noalloc",
            "ql_batch_set_shape",
            "ql_batch_fields", "ql_batch_project", "ql_sound_modes", "ql_closure_create", "ql_closure_forward", "ql_closure_gradients",
            "ql_closure_train_step", "ql_closure_train_steps", "ql_closure_params", "ql_closure_destroy",
            "ql_closure_last_error", "ql_step_count", "ql_save", "ql_checkpoint_read_info", "ql_load",
            "ql_launch_info")


class QLError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"qlbm status {status}: {msg}")
        self.status = status


class ql_velset(C.Structure):
    _fields_ = [("Q", C.c_int32), ("kind", C.c_int32)]


class ql_grid(C.Structure):
    _fields_ = [("nx", C.c_int64), ("length", C.c_double), ("dt", C.c_double)]


class ql_bc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad_", C.c_int32)]


_DP = C.POINTER(C.c_double)


class ql_init(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad_", C.c_int32), ("prm", C.c_double * 8),
                ("rho", _DP), ("u", _DP), ("T", _DP), ("ghost", _DP)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class ql_opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("pr_mode", C.c_int32), ("enskog", C.c_int32), ("device", C.c_int32),
                ("chi_mode", C.c_int32), ("fault", C.c_int32), ("sums", C.c_int32), ("launch", C.c_int32),
                ("pr_const", C.c_double), ("rho_ref", C.c_double), ("stream", C.c_void_p),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p)]


class ql_instance(C.Structure):
    _fields_ = [("vs", ql_velset), ("grid", ql_grid), ("denseness", C.c_double), ("kn", C.c_double),
                ("bc", ql_bc), ("init", ql_init), ("pr_mode", C.c_int32), ("enskog", C.c_int32),
                ("pr_const", C.c_double), ("rho_ref", C.c_double), ("chi_mode", C.c_int32), ("pad_", C.c_int32)]


class ql_checkpoint_info(C.Structure):
    _fields_ = [("Q", C.c_int32), ("bc_kind", C.c_int32), ("precision", C.c_int32), ("pr_mode", C.c_int32),
                ("enskog", C.c_int32), ("chi_mode", C.c_int32), ("nx", C.c_int64), ("steps", C.c_int64),
                ("length", C.c_double), ("dt", C.c_double), ("denseness", C.c_double), ("kn", C.c_double),
                ("pr_const", C.c_double), ("rho_ref", C.c_double), ("ghost", C.c_double * 18)]


class ql_closure_desc(C.Structure):
    _fields_ = [("in_channels", C.c_int32), ("out_channels", C.c_int32), ("width", C.c_int32),
                ("layers", C.c_int32), ("ksize", C.c_int32), ("positions", C.c_int32), ("max_batch", C.c_int32),
                ("pad_", C.c_int32), ("seed", C.c_uint64), ("in_shift", C.c_float * 8), ("in_scale", C.c_float * 8),
                ("out_scale", C.c_float * 8)]


_lib = None


def lib():
    """Loads libqlbm.so; raises if it is missing (build it with paper_2211_16933_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing; run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        V = C.c_void_p
        L.ql_create.argtypes = [C.POINTER(ql_velset), C.POINTER(ql_grid), C.c_double, C.c_double, C.POINTER(ql_bc),
                                C.POINTER(ql_init), C.POINTER(ql_opts), C.POINTER(V)]
        L.ql_step.argtypes = [V, C.c_int64]
        L.ql_sync.argtypes = [V]
        L.ql_moments.argtypes = [V] + [_DP] * 7
        L.ql_totals.argtypes = [V, _DP]
        L.ql_get_state.argtypes = [V, _DP, _DP]
        L.ql_set_state.argtypes = [V, _DP, _DP]
        L.ql_load_fields.argtypes = [V, _DP, _DP, _DP]
        L.ql_rhs.argtypes = [V, _DP, _DP]
        L.ql_state_device.argtypes = [V, C.POINTER(V), C.POINTER(C.c_int64)]
        L.ql_info.argtypes = [V, _DP]
        L.ql_launch_info.argtypes = [V, C.POINTER(C.c_int64)]
        L.ql_destroy.argtypes = [V]
        L.ql_last_error.argtypes = [V]
        L.ql_last_error.restype = C.c_char_p
        L.ql_velocity_set.argtypes = [C.c_int32, _DP, _DP]
        L.ql_eta_of_denseness.argtypes = [C.c_double, _DP]
        L.ql_sound_speed2.argtypes = [C.c_double] * 4
        L.ql_sound_speed2.restype = C.c_double
        L.ql_rankine_hugoniot.argtypes = [C.c_double] * 5 + [_DP]
        L.ql_riemann_exact.argtypes = [C.c_double, C.c_double, _DP, _DP, _DP, C.c_int64, _DP, _DP, _DP, _DP]
        L.ql_batch_create.argtypes = [C.POINTER(ql_instance), C.c_int64, C.POINTER(ql_opts), C.POINTER(V)]
        L.ql_batch_tune.argtypes = [V, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        L.ql_batch_set_shape.argtypes = [V, C.c_int32, C.c_int32]
        L.ql_batch_run.argtypes = [V, C.c_int64]
        L.ql_batch_sync.argtypes = [V, C.POINTER(C.c_uint32)]
        L.ql_batch_moments.argtypes = [V, C.c_int64] + [_DP] * 7
        L.ql_batch_get_state.argtypes = [V, C.c_int64, _DP, _DP]
        L.ql_batch_info.argtypes = [V, _DP]
        L.ql_batch_destroy.argtypes = [V]
        L.ql_batch_last_error.argtypes = [V]
        L.ql_batch_last_error.restype = C.c_char_p
        L.ql_step_noalloc.argtypes = [C.POINTER(ql_velset), C.POINTER(ql_grid), C.c_double, C.c_double,
                                      C.POINTER(ql_bc), C.POINTER(ql_opts), V, C.c_int64, C.c_int64]
        L.ql_batch_fields.argtypes = [V, C.c_int32, V]
        L.ql_batch_project.argtypes = [V, C.c_int32, V]
        L.ql_sound_modes.argtypes = [C.c_double] * 4 + [C.c_int32] + [C.c_double] * 4 + [_DP]
        F = C.POINTER(C.c_float)
        L.ql_closure_create.argtypes = [C.POINTER(ql_closure_desc), C.POINTER(ql_opts), C.POINTER(V)]
        L.ql_closure_forward.argtypes = [V, V, V, C.c_int64, V]
        L.ql_closure_gradients.argtypes = [V, V, V, V, C.c_int64, F, F]
        L.ql_closure_train_step.argtypes = [V, V, V, V, C.c_int64, C.c_float, F]
        L.ql_closure_train_steps.argtypes = [V, V, V, V, C.c_int64, V, C.c_int64, C.c_int64,
                                             C.POINTER(C.c_float), V]
        L.ql_closure_params.argtypes = [V, F, F, C.POINTER(C.c_int64)]
        L.ql_closure_destroy.argtypes = [V]
        L.ql_closure_last_error.argtypes = [V]
        L.ql_closure_last_error.restype = C.c_char_p
        L.ql_step_count.argtypes = [V, C.POINTER(C.c_int64)]
        L.ql_save.argtypes = [V, C.c_char_p]
        L.ql_checkpoint_read_info.argtypes = [C.c_char_p, C.POINTER(ql_checkpoint_info)]
        L.ql_load.argtypes = [C.c_char_p, C.POINTER(ql_opts), C.POINTER(V)]
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


def _check(st, ctx=None):
    if st != QL_OK:
        msg = lib().ql_last_error(ctx)
        raise QLError(st, msg.decode() if msg else "")


# ---------------------------------------------------------------- host-only helpers
_VELSET_CACHE = {}


def ql_velocity_set(Q: int):
    """Nodes and weights of the Q-point set (computed by the library once per Q, about a millisecond at
    Q = 32; copies are returned)."""
    if Q not in _VELSET_CACHE:
        p, w = np.zeros(Q), np.zeros(Q)
        _check(lib().ql_velocity_set(Q, _ptr(p), _ptr(w)))
        _VELSET_CACHE[Q] = (p, w)
    p, w = _VELSET_CACHE[Q]
    return p.copy(), w.copy()


def ql_eta_of_denseness(El: float) -> float:
    out = C.c_double()
    _check(lib().ql_eta_of_denseness(El, C.byref(out)))
    return out.value


def ql_sound_speed2(eta0, rho_ref, rho, T) -> float:
    return lib().ql_sound_speed2(eta0, rho_ref, rho, T)


def ql_rankine_hugoniot(eta0, rho_ref, rho1, T1, mach):
    out = np.zeros(4)
    _check(lib().ql_rankine_hugoniot(eta0, rho_ref, rho1, T1, mach, _ptr(out)))
    return tuple(out)


def ql_riemann_exact(eta0, rho_ref, left, right, xi=()):
    """Inviscid shock tube of the dense gas (host): left and right states (rho, T) at rest.  Returns the waves
    {P_c, u_c, rho1, T1, rho2, T2, xi_head, xi_tail, xi_shock} as a dict and rho, u, T at the given xi."""
    xi = np.ascontiguousarray(xi, dtype=np.float64).ravel()
    n = xi.size
    waves, rho, u, T = np.zeros(9), np.zeros(max(n, 1)), np.zeros(max(n, 1)), np.zeros(max(n, 1))
    lv = np.ascontiguousarray(left, dtype=np.float64)
    rv = np.ascontiguousarray(right, dtype=np.float64)
    if lv.size != 2 or rv.size != 2:
        raise ValueError("left and right are (rho, T) pairs")
    _check(lib().ql_riemann_exact(eta0, rho_ref, _ptr(lv), _ptr(rv), _ptr(waves), n, _ptr(xi) if n else None,
                                  _ptr(rho), _ptr(u), _ptr(T)))
    keys = ("P_c", "u_c", "rho1", "T1", "rho2", "T2", "xi_head", "xi_tail", "xi_shock")
    return dict(zip(keys, waves.tolist())), rho[:n], u[:n], T[:n]


# ---------------------------------------------------------------- context entry points
def ql_create(vs, grid, denseness, kn, bc, init, opts):
    ctx = C.c_void_p()
    _check(lib().ql_create(C.byref(vs), C.byref(grid), denseness, kn, C.byref(bc), C.byref(init), C.byref(opts),
                           C.byref(ctx)))
    return ctx


def ql_step(ctx, nsteps: int):
    _check(lib().ql_step(ctx, nsteps), ctx)


def ql_sync(ctx):
    _check(lib().ql_sync(ctx), ctx)


def ql_moments(ctx, rho=None, u=None, T=None, P=None, q=None, Pxx=None, totals=None):
    _check(lib().ql_moments(ctx, *[_ptr(a) for a in (rho, u, T, P, q, Pxx, totals)]), ctx)


def ql_totals(ctx, totals):
    _check(lib().ql_totals(ctx, _ptr(totals)), ctx)


def ql_get_state(ctx, phi, theta):
    _check(lib().ql_get_state(ctx, _ptr(phi), _ptr(theta)), ctx)


def ql_set_state(ctx, phi, theta):
    _check(lib().ql_set_state(ctx, _ptr(phi), _ptr(theta)), ctx)


def ql_load_fields(ctx, rho, u, T):
    _check(lib().ql_load_fields(ctx, _ptr(rho), _ptr(u), _ptr(T)), ctx)


def ql_rhs(ctx, Lphi, Ltheta):
    _check(lib().ql_rhs(ctx, _ptr(Lphi), _ptr(Ltheta)), ctx)


def ql_state_device(ctx):
    p, s = C.c_void_p(), C.c_int64()
    _check(lib().ql_state_device(ctx, C.byref(p), C.byref(s)), ctx)
    return p.value, s.value


def ql_info(ctx, Q):
    out = np.zeros(6 + 2 * Q)
    _check(lib().ql_info(ctx, _ptr(out)), ctx)
    return out


def ql_launch_info(ctx):
    """Steps one launch of the whole-run kernel covers, 0 if the solver launches per stage."""
    n = C.c_int64(0)
    _check(lib().ql_launch_info(ctx, C.byref(n)), ctx)
    return n.value


def ql_destroy(ctx):
    _check(lib().ql_destroy(ctx))


def ql_step_count(ctx) -> int:
    n = C.c_int64()
    _check(lib().ql_step_count(ctx, C.byref(n)), ctx)
    return n.value


def ql_save(ctx, path):
    _check(lib().ql_save(ctx, os.fsencode(path)), ctx)


def ql_checkpoint_read_info(path) -> ql_checkpoint_info:
    info = ql_checkpoint_info()
    _check(lib().ql_checkpoint_read_info(os.fsencode(path), C.byref(info)))
    return info


def ql_load(path, opts):
    ctx = C.c_void_p()
    _check(lib().ql_load(os.fsencode(path), C.byref(opts) if opts is not None else None, C.byref(ctx)))
    return ctx


def ql_step_noalloc(vs, grid, denseness, kn, bc, opts, psi, row_stride, nsteps):
    """Steps a caller-owned device state (pointer psi) without any allocation."""
    _check(lib().ql_step_noalloc(C.byref(vs), C.byref(grid), denseness, kn, C.byref(bc), C.byref(opts),
                                 C.c_void_p(psi), row_stride, nsteps))


# ---------------------------------------------------------------- batched form
def _bcheck(st, b=None):
    if st != QL_OK:
        msg = lib().ql_batch_last_error(b)
        raise QLError(st, msg.decode() if msg else "")


def ql_batch_create(insts, opts):
    arr = (ql_instance * len(insts))(*insts)
    b = C.c_void_p()
    _bcheck(lib().ql_batch_create(arr, len(insts), C.byref(opts), C.byref(b)))
    return b


def ql_batch_tune(b, trial_launches=3):
    w, c = C.c_int32(), C.c_int32()
    _bcheck(lib().ql_batch_tune(b, trial_launches, C.byref(w), C.byref(c)), b)
    return w.value, c.value


def ql_batch_set_shape(b, warps, ctas_per_sm):
    _bcheck(lib().ql_batch_set_shape(b, warps, ctas_per_sm), b)


def ql_batch_run(b, nsteps):
    _bcheck(lib().ql_batch_run(b, nsteps), b)


def ql_batch_sync(b, n):
    flags = (C.c_uint32 * n)()
    st = lib().ql_batch_sync(b, flags)
    return st, np.array(flags[:], dtype=np.uint32)


def ql_batch_moments(b, i, rho=None, u=None, T=None, P=None, q=None, Pxx=None, totals=None):
    _bcheck(lib().ql_batch_moments(b, i, *[_ptr(a) for a in (rho, u, T, P, q, Pxx, totals)]), b)


def ql_batch_get_state(b, i, phi, theta):
    _bcheck(lib().ql_batch_get_state(b, i, _ptr(phi), _ptr(theta)), b)


def ql_batch_info(b):
    out = np.zeros(6)
    _bcheck(lib().ql_batch_info(b, _ptr(out)), b)
    return out


def ql_batch_destroy(b):
    _bcheck(lib().ql_batch_destroy(b))


def ql_batch_fields(b, ncoarse, out_ptr):
    _bcheck(lib().ql_batch_fields(b, ncoarse, C.c_void_p(out_ptr)), b)


def ql_batch_project(b, mode, out_ptr):
    _bcheck(lib().ql_batch_project(b, mode, C.c_void_p(out_ptr)), b)


def ql_sound_modes(denseness, kn, length, rho, T, k, rho_ref=1.0, pr_mode=QL_PR_DENSE, pr_const=2.0 / 3.0):
    """(c_s, alpha_a, alpha_a without bulk viscosity, alpha_t, gamma) of a sound wave, Eqs. sw_cs / sw_coeff."""
    out = np.zeros(5)
    _check(lib().ql_sound_modes(denseness, kn, length, rho_ref, pr_mode, pr_const, rho, T, k, _ptr(out)))
    return out


def make_instance(Q, nx, length, dt, denseness, kn, *, bc=QL_BC_PERIODIC, init_kind=QL_INIT_SOUND, prm=(),
                  pr_mode=QL_PR_DENSE, pr_const=2.0 / 3.0, enskog=1, rho_ref=1.0, keep=None, rho=None, u=None, T=None,
                  ghost=None, chi_mode=QL_CHI_SET):
    """One ql_instance; `keep` (a list) holds the numpy arrays its pointers refer to."""
    I = ql_instance()
    I.vs = ql_velset(Q, 0)
    I.grid = ql_grid(nx, length, dt)
    I.denseness, I.kn = denseness, kn
    I.bc = ql_bc(bc, 0)
    I.init.kind = init_kind
    for j, v in enumerate(prm):
        I.init.prm[j] = v
    for name, arr in (("rho", rho), ("u", u), ("T", T), ("ghost", ghost)):
        if arr is not None:
            a = np.ascontiguousarray(arr, dtype=np.float64)
            if keep is not None:
                keep.append(a)
            setattr(I.init, name, _ptr(a))
    I.pr_mode, I.enskog, I.pr_const, I.rho_ref = pr_mode, enskog, pr_const, rho_ref
    I.chi_mode = chi_mode
    return I


class Batch:
    """A batch of instances on one device; stream from PyTorch when available."""

    def __init__(self, instances, precision=QL_FP32, device=0, use_torch=True, sums=QL_SUMS_DFP32):
        o = ql_opts()
        o.precision, o.device, o.sums = precision, device, sums
        self.n = len(instances)
        self.Qs = [I.vs.Q for I in instances]
        self.nxs = [I.grid.nx for I in instances]
        if use_torch:
            import torch
            if torch.cuda.is_available():
                torch.cuda.set_device(device)
                self._stream = torch.cuda.Stream(device)
                o.stream = C.c_void_p(self._stream.cuda_stream)
        self.b = ql_batch_create(instances, o)

    def tune(self, trial_launches=3):
        return ql_batch_tune(self.b, trial_launches)

    def set_shape(self, warps, ctas_per_sm):
        """warps per CTA (8 or 4); ctas_per_sm 0: one CTA per work item, else a persistent grid."""
        ql_batch_set_shape(self.b, warps, ctas_per_sm)

    def run(self, nsteps):
        ql_batch_run(self.b, nsteps)

    def sync(self):
        st, flags = ql_batch_sync(self.b, self.n)
        if st != QL_OK:
            _bcheck(st, self.b)
        return flags

    def moments(self, i):
        nx = self.nxs[i]
        out = {k: np.zeros(nx) for k in ("rho", "u", "T", "P", "q", "Pxx")}
        tot = np.zeros(3)
        ql_batch_moments(self.b, i, out["rho"], out["u"], out["T"], out["P"], out["q"], out["Pxx"], tot)
        out["totals"] = tot
        return out

    def state(self, i):
        nx, Q = self.nxs[i], self.Qs[i]
        a, c = np.zeros(nx * Q), np.zeros(nx * Q)
        ql_batch_get_state(self.b, i, a, c)
        return a.reshape(nx, Q), c.reshape(nx, Q)

    def info(self):
        return ql_batch_info(self.b)

    def fields(self, ncoarse, out):
        """out: a device tensor of n * 5 * ncoarse float64 (its data pointer is passed)."""
        ql_batch_fields(self.b, ncoarse, out.data_ptr())

    def project(self, mode, out):
        """Density mode amplitudes of all instances into a device tensor of n float64."""
        ql_batch_project(self.b, mode, out.data_ptr())

    def close(self):
        if getattr(self, "b", None) is not None:
            ql_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- learned closure
def _ccheck(st, c=None):
    if st != QL_OK:
        msg = lib().ql_closure_last_error(c)
        raise QLError(st, msg.decode() if msg else "")


class Closure:
    """The learned coarse-grid closure network; device tensors are passed by data pointer."""

    def __init__(self, in_channels, out_channels, positions, max_batch, seed=0, in_shift=None, in_scale=None,
                 out_scale=None, layers=5, width=64, device=0):
        import torch
        d = ql_closure_desc()
        d.in_channels, d.out_channels, d.width, d.layers, d.ksize = in_channels, out_channels, width, layers, 5
        d.positions, d.max_batch, d.seed = positions, max_batch, seed
        for i in range(8):
            d.in_shift[i] = float(in_shift[i]) if in_shift is not None and i < len(in_shift) else 0.0
            d.in_scale[i] = float(in_scale[i]) if in_scale is not None and i < len(in_scale) else 1.0
            d.out_scale[i] = float(out_scale[i]) if out_scale is not None and i < len(out_scale) else 1.0
        o = ql_opts()
        o.device = device
        self._stream = torch.cuda.current_stream(device)
        o.stream = C.c_void_p(self._stream.cuda_stream)
        self.c = C.c_void_p()
        _ccheck(lib().ql_closure_create(C.byref(d), C.byref(o), C.byref(self.c)))
        self.in_channels, self.out_channels, self.positions = in_channels, out_channels, positions

    def forward(self, x, periodic, y):
        _ccheck(lib().ql_closure_forward(self.c, C.c_void_p(x.data_ptr()), C.c_void_p(periodic.data_ptr()),
                                         x.shape[0], C.c_void_p(y.data_ptr())), self.c)

    def gradients(self, x, y, periodic):
        n = self.nparams()
        g = np.zeros(n, dtype=np.float32)
        loss = C.c_float()
        _ccheck(lib().ql_closure_gradients(self.c, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                           C.c_void_p(periodic.data_ptr()), x.shape[0], C.byref(loss),
                                           g.ctypes.data_as(C.POINTER(C.c_float))), self.c)
        return loss.value, g

    def train_step(self, x, y, periodic, lr, want_loss=False):
        loss = C.c_float()
        _ccheck(lib().ql_closure_train_step(self.c, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                            C.c_void_p(periodic.data_ptr()), x.shape[0], lr,
                                            C.byref(loss) if want_loss else None), self.c)
        return loss.value if want_loss else None

    def train_steps(self, x, y, periodic, perm, lr, losses=None):
        """len(lr) Adam steps on batches gathered on the device: step s takes the samples
        perm[s B:(s + 1) B] of the device tensors x, y, periodic (B = len(perm) // len(lr)); losses (device
        float32 tensor of len(lr), optional) receives each step's loss.  Synchronises once."""
        lr = np.ascontiguousarray(lr, dtype=np.float32)
        nsteps = len(lr)
        if nsteps == 0:
            return
        if perm.numel() % nsteps != 0:
            raise ValueError("perm must hold the same number of samples for every step")
        B = perm.numel() // nsteps
        _ccheck(lib().ql_closure_train_steps(self.c, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                             C.c_void_p(periodic.data_ptr()), x.shape[0],
                                             C.c_void_p(perm.data_ptr()), nsteps, B,
                                             lr.ctypes.data_as(C.POINTER(C.c_float)),
                                             C.c_void_p(losses.data_ptr()) if losses is not None else None),
                self.c)

    def nparams(self):
        n = C.c_int64()
        _ccheck(lib().ql_closure_params(self.c, None, None, C.byref(n)), self.c)
        return n.value

    def get_params(self):
        p = np.zeros(self.nparams(), dtype=np.float32)
        _ccheck(lib().ql_closure_params(self.c, p.ctypes.data_as(C.POINTER(C.c_float)), None, None), self.c)
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _ccheck(lib().ql_closure_params(self.c, None, p.ctypes.data_as(C.POINTER(C.c_float)), None), self.c)

    def close(self):
        if getattr(self, "c", None) is not None and self.c:
            lib().ql_closure_destroy(self.c)
            self.c = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- convenience object
class Solver:
    """One solver context.  Device memory comes from PyTorch's caching allocator and
    work goes on PyTorch's current stream when torch is importable with CUDA."""

    def __init__(self, Q, nx, length, dt, denseness, kn, *, bc=QL_BC_PERIODIC, init_kind=QL_INIT_SOUND,
                 prm=(1.0, 1.0, 1e-3), rho=None, u=None, T=None, ghost=None, precision=QL_FP64,
                 pr_mode=QL_PR_DENSE, pr_const=2.0 / 3.0, enskog=1, rho_ref=1.0, device=0, use_torch=True,
                 chi_mode=None, fault=0, sums=QL_SUMS_DFP32, launch=QL_LAUNCH_AUTO):
        """fault = 1 is for failure-detection tests (ql_opts.fault): the stage kernels give up waiting for
        copies that are never issued and the next synchronising call raises QLError(QL_ECUDA).  sums
        (FP32 only): QL_SUMS_DFP32 or QL_SUMS_FP64, the arithmetic of the per-cell conserved sums.
        launch (ql_opts.launch): QL_LAUNCH_AUTO, QL_LAUNCH_STAGES (one launch per stage) or QL_LAUNCH_RUN (one
        launch per step call where the solver supports it)."""
        self.Q, self.nx, self.precision = Q, nx, precision
        vs = ql_velset(Q, 0)
        grid = ql_grid(nx, length, dt)
        b = ql_bc(bc, 0)
        ini = ql_init()
        ini.kind = init_kind
        for j, v in enumerate(prm):
            ini.prm[j] = v
        self._keep = []
        for name, arr in (("rho", rho), ("u", u), ("T", T), ("ghost", ghost)):
            if arr is not None:
                a = np.ascontiguousarray(arr, dtype=np.float64)
                self._keep.append(a)
                setattr(ini, name, _ptr(a))
        o = ql_opts()
        o.precision, o.pr_mode, o.enskog, o.device = precision, pr_mode, enskog, device
        o.pr_const, o.rho_ref = pr_const, rho_ref
        o.chi_mode = QL_CHI_SET if chi_mode is None else chi_mode
        o.fault = fault
        o.sums = sums
        o.launch = launch
        self._attach_torch(o, device, use_torch)
        self.ctx = ql_create(vs, grid, denseness, kn, b, ini, o)
        self._read_info()

    def _attach_torch(self, o, device, use_torch):
        """Work on PyTorch's current stream and device memory from its caching allocator, when available."""
        self._torch_blocks = {}
        if use_torch:
            import torch
            if torch.cuda.is_available():
                torch.cuda.set_device(device)
                stream = torch.cuda.current_stream(device)
                o.stream = C.c_void_p(stream.cuda_stream)
                self._stream = stream

                def _alloc(nbytes, user):
                    ptr = torch.cuda.caching_allocator_alloc(int(nbytes), device, stream)
                    self._torch_blocks[ptr] = nbytes
                    return ptr

                def _free(ptr, user):
                    if ptr in self._torch_blocks:
                        del self._torch_blocks[ptr]
                        torch.cuda.caching_allocator_delete(ptr)

                self._alloc_cb, self._free_cb = ALLOC_FN(_alloc), FREE_FN(_free)
                o.alloc, o.free = self._alloc_cb, self._free_cb

    def _read_info(self):
        Q = self.Q
        info = ql_info(self.ctx, Q)
        self.eta0, self.chi0, self.sigma, self.dx, self.dt, self.pmax = info[:6]
        self.p, self.w = info[6:6 + Q], info[6 + Q:]

    @classmethod
    def load(cls, path, *, device=0, use_torch=True):
        """A solver resumed from a restart file written by save(): the stored parameters, state and step count."""
        info = ql_checkpoint_read_info(path)
        self = cls.__new__(cls)
        self.Q, self.nx, self.precision = info.Q, info.nx, info.precision
        self._keep = []
        o = ql_opts()
        o.device = device
        self._attach_torch(o, device, use_torch)
        self.ctx = ql_load(path, o)
        self._read_info()
        return self

    def save(self, path):
        """Writes a restart file (parameters, step count and state)."""
        ql_save(self.ctx, path)

    def step_count(self):
        return ql_step_count(self.ctx)

    def step(self, n=1):
        ql_step(self.ctx, n)

    def steps_per_launch(self):
        """Steps one launch covers on the whole-run path, 0 when each stage is a launch (ql_launch_info)."""
        return ql_launch_info(self.ctx)

    def sync(self):
        ql_sync(self.ctx)

    def moments(self):
        out = {k: np.zeros(self.nx) for k in ("rho", "u", "T", "P", "q", "Pxx")}
        tot = np.zeros(3)
        ql_moments(self.ctx, out["rho"], out["u"], out["T"], out["P"], out["q"], out["Pxx"], tot)
        out["totals"] = tot
        return out

    def totals(self):
        t = np.zeros(3)
        ql_totals(self.ctx, t)
        return t

    def state(self):
        phi, th = np.zeros(self.nx * self.Q), np.zeros(self.nx * self.Q)
        ql_get_state(self.ctx, phi, th)
        return phi.reshape(self.nx, self.Q), th.reshape(self.nx, self.Q)

    def set_state(self, phi, theta):
        ql_set_state(self.ctx, np.ascontiguousarray(phi, dtype=np.float64).ravel(),
                     np.ascontiguousarray(theta, dtype=np.float64).ravel())

    def load_fields(self, rho, u, T):
        f = [np.ascontiguousarray(a, dtype=np.float64) for a in (rho, u, T)]
        ql_load_fields(self.ctx, *f)

    def rhs(self):
        a, b = np.zeros(self.nx * self.Q), np.zeros(self.nx * self.Q)
        ql_rhs(self.ctx, a, b)
        return a.reshape(self.nx, self.Q), b.reshape(self.nx, self.Q)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            ql_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
