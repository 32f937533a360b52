"""FP64 CPU oracle of the finite-difference Enskog-Shakhov lattice Boltzmann model.

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()`` and
by the cpu_baseline / ``--impl reference`` legs of ``bench.py``.  The product
library never imports it.  The arithmetic lives in ``fdlb_oracle.c`` (plain C,
double precision); this module compiles it with gcc and marshals numpy arrays.

Parity status of each function is given in the header of ``fdlb_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdlb_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

QMAX = 200
NG = 3


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, no FMA contraction)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


class Model(C.Structure):
    _fields_ = [
        ("Q", C.c_int), ("nx", C.c_int), ("bc", C.c_int), ("pr_mode", C.c_int),
        ("enskog", C.c_int), ("chi_mode", C.c_int),
        ("L", C.c_double), ("dx", C.c_double), ("dt", C.c_double),
        ("denseness", C.c_double), ("kn", C.c_double), ("pr_const", C.c_double),
        ("rho_ref", C.c_double),
        ("eta0", C.c_double), ("chi0", C.c_double), ("sigma", C.c_double),
        ("p", C.c_double * QMAX), ("w", C.c_double * QMAX),
        ("ghost_left", (C.c_double * 3) * NG), ("ghost_right", (C.c_double * 3) * NG),
    ]


_D = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        # ORACLE_LIB names a deliberately mutated build; only the mutation test sets it
        path = os.environ.get("ORACLE_LIB") or build()
        L = C.CDLL(path)
        for name in ("oq_chi_set", "oq_cs_compressibility", "oq_denseness", "oq_eta_from_denseness",
                     "oq_prandtl_dense"):
            getattr(L, name).restype = C.c_double
            getattr(L, name).argtypes = [C.c_double]
        L.oq_hermite.restype = C.c_double
        L.oq_hermite.argtypes = [C.c_int, C.c_double]
        L.oq_quadrature.argtypes = [C.c_int, _D, _D]
        L.oq_equilibrium.argtypes = [C.c_int, _D, _D, C.c_double, C.c_double, C.c_double, _D]
        L.oq_moments.argtypes = [C.c_int, _D, _D, _D, _D]
        L.oq_mu_ratio.restype = C.c_double
        L.oq_mu_ratio.argtypes = [C.c_double] * 3
        L.oq_lambda_over_lambdaref.restype = C.c_double
        L.oq_lambda_over_lambdaref.argtypes = [C.c_double] * 3
        L.oq_tau.restype = C.c_double
        L.oq_tau.argtypes = [C.POINTER(Model), C.c_double, C.c_double]
        L.oq_prandtl.restype = C.c_double
        L.oq_prandtl.argtypes = [C.POINTER(Model), C.c_double]
        L.oq_shakhov.argtypes = [C.c_int, _D, _D] + [C.c_double] * 5 + [_D, _D]
        L.oq_j1.argtypes = [C.c_int, _D, _D] + [C.c_double] * 8 + [_D, _D]
        L.oq_weno5_weights.argtypes = [C.c_double] * 3 + [_D]
        L.oq_weno5_face.restype = C.c_double
        L.oq_weno5_face.argtypes = [_D]
        L.oq_cd6.restype = C.c_double
        L.oq_cd6.argtypes = [_D, C.c_double]
        L.oq_model_init.argtypes = [C.POINTER(Model)]
        L.oq_fm_weight.restype = C.c_double
        L.oq_fm_weight.argtypes = [C.c_int, C.c_double, C.c_double]
        L.oq_fm_halfwidth.restype = C.c_int
        L.oq_fm_halfwidth.argtypes = [C.c_double, C.c_double]
        L.oq_fm_average.argtypes = [C.POINTER(Model), _D, _D]
        L.oq_sound_modes.argtypes = [C.POINTER(Model), C.c_double, C.c_double, C.c_double, _D]
        L.oq_rhs.argtypes = [C.POINTER(Model), _D, _D, _D, _D]
        L.oq_rk3_step.argtypes = [C.POINTER(Model), _D, _D]
        L.oq_run.argtypes = [C.POINTER(Model), _D, _D, C.c_long]
        L.oq_equilibrium_state.argtypes = [C.POINTER(Model), _D, _D, _D, _D, _D]
        L.oq_fields.argtypes = [C.POINTER(Model)] + [_D] * 8
        L.oq_totals.argtypes = [C.POINTER(Model), _D, _D, _D]
        L.oq_sound_speed2.restype = C.c_double
        L.oq_sound_speed2.argtypes = [C.c_double] * 4
        L.oq_rankine_hugoniot.argtypes = [C.c_double] * 5 + [_D]
        L.oq_init_fields.argtypes = [C.POINTER(Model), C.c_int, _D, C.c_long, C.c_long, _D, _D, _D]
        assert L.oq_model_sizeof() == C.sizeof(Model), "oracle struct layout mismatch"
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# ---------------------------------------------------------------- scalars
def chi_set(eta: float) -> float:
    return lib().oq_chi_set(eta)


def cs_compressibility(eta: float) -> float:
    return lib().oq_cs_compressibility(eta)


def denseness(eta: float) -> float:
    return lib().oq_denseness(eta)


def eta_from_denseness(El: float) -> float:
    return lib().oq_eta_from_denseness(El)


def prandtl_dense(Y: float) -> float:
    return lib().oq_prandtl_dense(Y)


def mu_over_muref(bn: float, chi: float, T: float) -> float:
    return lib().oq_mu_ratio(bn, chi, T)


def lambda_over_lambdaref(bn: float, chi: float, T: float) -> float:
    return lib().oq_lambda_over_lambdaref(bn, chi, T)


def hermite(l: int, p: float) -> float:
    return lib().oq_hermite(l, p)


def sound_speed2(eta0: float, rho_ref: float, rho: float, T: float) -> float:
    return lib().oq_sound_speed2(eta0, rho_ref, rho, T)


def rankine_hugoniot(eta0: float, rho_ref: float, rho1: float, T1: float, mach: float):
    """Standing-shock states: returns (u1, rho2, u2, T2)."""
    out = np.zeros(4)
    st = lib().oq_rankine_hugoniot(eta0, rho_ref, rho1, T1, mach, _p(out))
    if st:
        raise ValueError(f"oq_rankine_hugoniot failed ({st})")
    return tuple(out)


# ---------------------------------------------------------------- velocity space
def quadrature(Q: int):
    p = np.zeros(Q)
    w = np.zeros(Q)
    st = lib().oq_quadrature(Q, _p(p), _p(w))
    if st:
        raise ValueError(f"oq_quadrature({Q}) failed ({st})")
    return p, w


def equilibrium(p, w, n, u, T) -> np.ndarray:
    p, w = _f64(p), _f64(w)
    out = np.zeros(len(p))
    lib().oq_equilibrium(len(p), _p(p), _p(w), n, u, T, _p(out))
    return out


def moments(p, phi, theta):
    """(n, u, T, Pi, q) of one cell."""
    p, phi, theta = _f64(p), _f64(phi), _f64(theta)
    out = np.zeros(5)
    lib().oq_moments(len(p), _p(p), _p(phi), _p(theta), _p(out))
    return tuple(out)


def shakhov(p, w, n, u, T, q, Pr):
    p, w = _f64(p), _f64(w)
    a, b = np.zeros(len(p)), np.zeros(len(p))
    lib().oq_shakhov(len(p), _p(p), _p(w), n, u, T, q, Pr, _p(a), _p(b))
    return a, b


def j1(p, w, n, u, T, Y, dlnchi, dlnrho, du, dlnT):
    p, w = _f64(p), _f64(w)
    a, b = np.zeros(len(p)), np.zeros(len(p))
    lib().oq_j1(len(p), _p(p), _p(w), n, u, T, Y, dlnchi, dlnrho, du, dlnT, _p(a), _p(b))
    return a, b


def weno5_weights(b1, b2, b3):
    out = np.zeros(3)
    lib().oq_weno5_weights(b1, b2, b3, _p(out))
    return out


def weno5_face(f) -> float:
    f = _f64(f)
    assert f.shape == (5,)
    return lib().oq_weno5_face(_p(f))


def cd6(q, dx) -> float:
    q = _f64(q)
    assert q.shape == (7,)
    return lib().oq_cd6(_p(q), dx)


# ---------------------------------------------------------------- whole model
INIT_SOUND, INIT_RIEMANN, INIT_SHOCK = 0, 1, 2
BC_PERIODIC, BC_FIXED = 0, 1
CHI_SET, CHI_RET_FM = 0, 1


def make_model(Q, nx, L, dt, denseness, kn, pr_mode=1, pr_const=2.0 / 3.0, rho_ref=1.0,
               bc=BC_PERIODIC, enskog=1, chi_mode=CHI_SET) -> Model:
    m = Model()
    m.Q, m.nx, m.bc, m.pr_mode, m.enskog, m.chi_mode = Q, nx, bc, pr_mode, enskog, chi_mode
    m.L, m.dt, m.denseness, m.kn, m.pr_const, m.rho_ref = L, dt, denseness, kn, pr_const, rho_ref
    st = lib().oq_model_init(C.byref(m))
    if st:
        raise ValueError(f"oq_model_init failed ({st})")
    return m


def fm_weight(d: int, dx: float, sigma: float) -> float:
    """Weight of the cell at offset d in the Fischer-Methfessel density average (Eq. chi_ret)."""
    return lib().oq_fm_weight(d, dx, sigma)


def fm_halfwidth(dx: float, sigma: float) -> int:
    return lib().oq_fm_halfwidth(dx, sigma)


def fm_average(m: Model, n_ext):
    """Fischer-Methfessel averages of the densities of the extended cells -3 .. nx+2."""
    n_ext = _f64(n_ext)
    assert n_ext.shape == (m.nx + 6,)
    out = np.zeros_like(n_ext)
    lib().oq_fm_average(C.byref(m), _p(n_ext), _p(out))
    return out


def sound_modes(m: Model, rho: float, T: float, k: float):
    """(c_s, alpha_a, alpha_a without bulk viscosity, alpha_t, gamma) of a sound wave of wave number k."""
    out = np.zeros(5)
    lib().oq_sound_modes(C.byref(m), rho, T, k, _p(out))
    return out


def velocity_set(m: Model):
    return np.array(m.p[:m.Q]), np.array(m.w[:m.Q])


def tau(m: Model, n, T) -> float:
    return lib().oq_tau(C.byref(m), n, T)


def prandtl(m: Model, n) -> float:
    return lib().oq_prandtl(C.byref(m), n)


def init_fields(m: Model, kind: int, prm, i0: int = 0, count: int | None = None):
    """Initial (rho, u, T) at global cells i0 .. i0+count-1 (ghost indices allowed)."""
    count = m.nx if count is None else count
    prm = _f64(prm)
    r, u, T = np.zeros(count), np.zeros(count), np.zeros(count)
    st = lib().oq_init_fields(C.byref(m), kind, _p(prm), i0, count, _p(r), _p(u), _p(T))
    if st:
        raise ValueError(f"oq_init_fields failed ({st})")
    return r, u, T


def set_ghosts(m: Model, left, right):
    """left/right: 3 (rho, u, T) triples each; left[g] is cell g-3, right[g] is cell nx+g."""
    for g in range(NG):
        for c in range(3):
            m.ghost_left[g][c] = float(left[g][c])
            m.ghost_right[g][c] = float(right[g][c])


def set_ghosts_from_init(m: Model, kind: int, prm):
    """Fixed ghost cells holding the initial state's far field (kind 1 and 2)."""
    rl, ul, Tl = init_fields(m, kind, prm, -NG, NG)
    rr, ur, Tr = init_fields(m, kind, prm, m.nx, NG)
    set_ghosts(m, np.stack([rl, ul, Tl], 1), np.stack([rr, ur, Tr], 1))


def equilibrium_state(m: Model, rho, u, T):
    rho, u, T = _f64(rho), _f64(u), _f64(T)
    phi = np.zeros(m.nx * m.Q)
    th = np.zeros(m.nx * m.Q)
    lib().oq_equilibrium_state(C.byref(m), _p(rho), _p(u), _p(T), _p(phi), _p(th))
    return phi.reshape(m.nx, m.Q), th.reshape(m.nx, m.Q)


def rhs(m: Model, phi, theta):
    phi, theta = _f64(phi), _f64(theta)
    a, b = np.zeros_like(phi), np.zeros_like(theta)
    st = lib().oq_rhs(C.byref(m), _p(phi), _p(theta), _p(a), _p(b))
    if st:
        raise FloatingPointError(f"oq_rhs: non-physical state ({st})")
    return a, b


def run(m: Model, phi, theta, nsteps: int):
    """Returns new (phi, theta) after nsteps RK3 steps; inputs are not modified."""
    phi, theta = _f64(phi).copy(), _f64(theta).copy()
    st = lib().oq_run(C.byref(m), _p(phi), _p(theta), nsteps)
    if st:
        raise FloatingPointError(f"oq_run: non-physical state ({st})")
    return phi, theta


def fields(m: Model, phi, theta):
    """dict of rho, u, T, P, q, Pxx per cell."""
    phi, theta = _f64(phi), _f64(theta)
    out = {k: np.zeros(m.nx) for k in ("rho", "u", "T", "P", "q", "Pxx")}
    lib().oq_fields(C.byref(m), _p(phi), _p(theta), *[_p(out[k]) for k in ("rho", "u", "T", "P", "q", "Pxx")])
    return out


def totals(m: Model, phi, theta):
    phi, theta = _f64(phi), _f64(theta)
    out = np.zeros(3)
    lib().oq_totals(C.byref(m), _p(phi), _p(theta), _p(out))
    return out
