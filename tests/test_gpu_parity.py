"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances, L-infinity, fields normalised by reference scales (rho_ref = T_ref = 1,
u by sqrt(T_ref), P by rho_ref T_ref (1 + b rho chi)_ref, q by rho_ref T_ref^(3/2)):
  FP64 mode  1e-10 for rho, u, T, P, q and for every psi_k relative to the
             largest |psi_k| of that velocity.
  FP32 mode  1e-5 for the fields after short runs (<= 10 steps) of states whose
             temperatures stay in [0.5, 1.8]; psi within 2e-5 of the largest
             |psi| of its component (phi or theta).  The state is stored in FP32,
             so errors grow with the number of steps (about 1e-8 per step on the
             sound wave: 4e-5 after 2000 steps), and they scale with the
             conditioning kappa = sum_k |g_k| of the Hermite equilibrium, which
             is 1 for T <= 1.8 but 114 at the T = 2.08 downstream state of the
             Mach-2 shock with Q = 32 (tolerance 4e-4 there).
"""
import functools

import numpy as np
import pytest

import oracle as O
from paper_2211_16933_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-5}          # fields, by precision (QL_FP64 = 0, QL_FP32 = 1)
TOL_PSI = {0: 1e-10, 1: 2e-5}


def _setup(q, w, precision, dt=None, fields=None, ghost=None, enskog=1, chi_mode=0):
    """Oracle model + initial state and a GPU solver for the same workload dict."""
    Q, nx, L = w["Q"], w["nx"], w["length"]
    p, _ = O.quadrature(Q)
    dt = dt or inputs.cfl_dt(L / nx, abs(p).max())
    bc = O.BC_PERIODIC if w["bc"] == "periodic" else O.BC_FIXED
    prm = 1 if w["pr_mode"] == "dense" else 0
    m = O.make_model(Q, nx, L, dt, w["denseness"], w["kn"], pr_mode=prm, pr_const=w["pr_const"], bc=bc,
                     enskog=enskog, chi_mode=chi_mode)
    kind = {"sound": O.INIT_SOUND, "riemann": O.INIT_RIEMANN, "shock": O.INIT_SHOCK, "fields": 3}[w["init"]]
    kw = {}
    if kind == 3:
        r, u, T = fields
        kw = dict(rho=r, u=u, T=T)
        if bc == O.BC_FIXED:
            O.set_ghosts(m, ghost[:3], ghost[3:])
            kw["ghost"] = np.asarray(ghost, dtype=float).ravel()
    else:
        r, u, T = O.init_fields(m, kind, w["prm"])
        if bc == O.BC_FIXED:
            O.set_ghosts_from_init(m, kind, w["prm"])
    ph, th = O.equilibrium_state(m, r, u, T)
    s = q.Solver(Q, nx, L, dt, w["denseness"], w["kn"], bc=bc, init_kind=kind, prm=w["prm"] if kind != 3 else (),
                 precision=precision, pr_mode=prm, pr_const=w["pr_const"], enskog=enskog, chi_mode=chi_mode, **kw)
    return m, ph, th, s


def _field_errors(m, ph, th, s):
    f_or = O.fields(m, ph, th)
    f_gp = s.moments()
    Y0 = 4 * m.eta0 * O.chi_set(m.eta0)
    scale = dict(rho=1.0, u=1.0, T=1.0, P=1.0 + Y0, q=1.0)
    return {k: float(np.abs(f_gp[k] - f_or[k]).max() / scale[k]) for k in scale}


def _psi_error(ph, th, s, precision):
    """FP64: per velocity row; FP32: relative to the largest |psi| of the component."""
    gp, gt = s.state()
    e = 0.0
    for a, b in ((gp, ph), (gt, th)):
        if precision == 0:
            scale = np.abs(b).max(axis=0)
            e = max(e, float((np.abs(a - b).max(axis=0) / scale).max()))
        else:
            e = max(e, float(np.abs(a - b).max() / np.abs(b).max()))
    return e


def _check(m, ph, th, s, precision, tol=None, tol_psi=None):
    errs = _field_errors(m, ph, th, s)
    assert max(errs.values()) <= (tol or TOL[precision]), errs
    e = _psi_error(ph, th, s, precision)
    assert e <= (tol_psi or TOL_PSI[precision]), e
    return errs, e


def _smooth_workload(Q, nx, bc="periodic"):
    return dict(Q=Q, nx=nx, length=1.0, denseness=1.1, kn=0.02, bc=bc, init="fields", prm=(),
                pr_mode="dense", pr_const=2.0 / 3.0)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("Q", [8, 16, 20, 24, 32, 40])
def test_rhs_matches_oracle(gpu, Q, precision):
    """L[psi] of Eq. (cast) on an off-equilibrium periodic state spanning 3 tiles + a ragged tail."""
    nx = 3 * 248 + 17
    w = _smooth_workload(Q, nx)
    f = inputs.smooth_periodic_fields(nx, seed=Q)
    m, ph, th, s = _setup(gpu, w, precision, fields=f)
    noise = inputs.state_noise(ph.shape, seed=Q + 1, scale=1e-2)
    ph = ph * noise
    s.set_state(ph, th)
    if precision == 1:  # the FP32 solver holds the rounded state
        ph, th = (a.astype(np.float32).astype(np.float64) for a in s.state())
    Lp_o, Lt_o = O.rhs(m, ph, th)
    Lp_g, Lt_g = s.rhs()
    for a, b in ((Lp_g, Lp_o), (Lt_g, Lt_o)):
        if precision == 0:
            scale = np.abs(b).max(axis=0) + 1e-300
            assert float((np.abs(a - b).max(axis=0) / scale).max()) <= 1e-11
        else:
            # FP32: the flux difference p (h+ - h-)/dx amplifies the FP32 rounding of the face values
            assert float(np.abs(a - b).max() / np.abs(b).max()) <= 2e-4


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("Q", [8, 16, 20, 24, 32, 40])
@pytest.mark.parametrize("bc", ["periodic", "fixed"])
def test_steps_match_oracle(gpu, Q, precision, bc):
    nx = 3 * 248 + 17
    w = _smooth_workload(Q, nx, bc)
    f = inputs.smooth_periodic_fields(nx, seed=7 * Q)
    ghost = None
    if bc == "fixed":
        ghost = [(f[0][0], f[1][0], f[2][0])] * 3 + [(f[0][-1], f[1][-1], f[2][-1])] * 3
    m, ph, th, s = _setup(gpu, w, precision, fields=f, ghost=ghost)
    ph, th = O.run(m, ph, th, 6)
    s.step(6)
    _check(m, ph, th, s, precision)


@functools.lru_cache(maxsize=None)
def _sound_wave_oracle():
    w = inputs.sound_wave()
    m, ph, th, _ = _setup_oracle_only(w)
    return w, m, O.run(m, ph, th, w["steps"])


def _setup_oracle_only(w):
    Q, nx, L = w["Q"], w["nx"], w["length"]
    p, _ = O.quadrature(Q)
    dt = inputs.cfl_dt(L / nx, abs(p).max())
    m = O.make_model(Q, nx, L, dt, w["denseness"], w["kn"], pr_mode=0, pr_const=w["pr_const"])
    r, u, T = O.init_fields(m, O.INIT_SOUND, w["prm"])
    ph, th = O.equilibrium_state(m, r, u, T)
    return m, ph, th, dt


@pytest.mark.parametrize("precision", [0, 1])
def test_sound_wave_2000_steps(gpu, precision):
    """Periodic sound wave, Nx = 256, Q = 16, E_l = 0.1, Kn = 0.1, Pr = 2/3, A = 1e-3, 2000 steps."""
    w, m, (ph, th) = _sound_wave_oracle()
    s = gpu.Solver(w["Q"], w["nx"], w["length"], m.dt, w["denseness"], w["kn"], bc=gpu.QL_BC_PERIODIC,
                   init_kind=gpu.QL_INIT_SOUND, prm=w["prm"], precision=precision, pr_mode=gpu.QL_PR_CONST,
                   pr_const=w["pr_const"])
    s.step(w["steps"])
    errs, e = _check(m, ph, th, s, precision, tol=1e-10 if precision == 0 else 4e-5,
                     tol_psi=1e-10 if precision == 0 else 1e-4)
    # the perturbation itself is resolved: errors are small relative to its amplitude 1e-3
    assert errs["rho"] / 1e-3 <= (1e-7 if precision == 0 else 4e-2)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("mach,El", [(2.0, 0.1), (1.4, 0.05), (1.4, 0.2)])
def test_normal_shock_steps(gpu, precision, mach, El):
    """Standing shock, Nx = 4096, Q = 32, fixed Rankine-Hugoniot ghosts: a few steps against the oracle."""
    w = inputs.normal_shock(mach, El)
    m, ph, th, s = _setup(gpu, w, precision)
    n = 3 if (mach, El) == (2.0, 0.1) else 1
    ph, th = O.run(m, ph, th, n)
    s.step(n)
    # kappa = sum_k |g_k| is 114 at the Mach-2 downstream state (T = 2.08, Q = 32)
    tol = None if precision == 0 or mach < 1.5 else 4e-4
    _check(m, ph, th, s, precision, tol=tol)


@pytest.mark.parametrize("nx", [8, 31, 248, 249, 496])
@pytest.mark.parametrize("bc", ["periodic", "fixed"])
def test_edge_sizes(gpu, nx, bc):
    """Minimum size, sizes below/at/above one tile, fixed and periodic ends."""
    w = _smooth_workload(16, nx, bc)
    f = inputs.smooth_periodic_fields(nx, seed=nx)
    ghost = [(1.0, 0.0, 1.0)] * 3 + [(1.0, 0.0, 1.0)] * 3 if bc == "fixed" else None
    m, ph, th, s = _setup(gpu, w, 0, fields=f, ghost=ghost)
    ph, th = O.run(m, ph, th, 4)
    s.step(4)
    _check(m, ph, th, s, 0)


def test_uniform_state_is_stationary(gpu):
    nx = 300
    f = [np.full(nx, 1.3), np.full(nx, 0.4), np.full(nx, 0.8)]
    w = _smooth_workload(24, nx, "fixed")
    m, ph, th, s = _setup(gpu, w, 0, fields=f, ghost=[(1.3, 0.4, 0.8)] * 6)
    s.step(10)
    gp, gt = s.state()
    np.testing.assert_allclose(gp, ph, rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(gt, th, rtol=1e-12, atol=1e-16)


@pytest.mark.parametrize("precision", [0, 1])
def test_mass_conservation_periodic(gpu, precision):
    nx = 777
    w = _smooth_workload(16, nx)
    f = inputs.smooth_periodic_fields(nx, seed=3)
    m, ph, th, s = _setup(gpu, w, precision, fields=f)
    t0 = s.totals()
    s.step(100)
    t1 = s.totals()
    assert abs(t1[0] - t0[0]) <= (1e-13 if precision == 0 else 2e-6)
    to = O.totals(m, ph, th)
    assert abs(t0[0] - to[0]) <= (1e-14 if precision == 0 else 1e-6)


def test_nonphysical_state_is_reported(gpu):
    """A cell with negative density sets the device error word; the next sync reports it."""
    nx = 64
    w = _smooth_workload(16, nx)
    m, ph, th, s = _setup(gpu, w, 0, fields=inputs.smooth_periodic_fields(nx, 1))
    ph = ph.copy()
    ph[10] *= -1.0
    s.set_state(ph, th)
    s.step(1)
    with pytest.raises(gpu.QLError) as e:
        s.sync()
    assert e.value.status == gpu.QL_ENONPHYSICAL


def test_state_roundtrip(gpu):
    nx = 260
    w = _smooth_workload(32, nx)
    m, ph, th, s = _setup(gpu, w, 0, fields=inputs.smooth_periodic_fields(nx, 9))
    a = ph * inputs.state_noise(ph.shape, 4)
    s.set_state(a, th)
    b, c = s.state()
    np.testing.assert_array_equal(b, a)
    np.testing.assert_array_equal(c, th)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("bc", ["periodic", "fixed"])
def test_ret_fm_rhs_and_steps_match_oracle(gpu, precision, bc):
    """chi_RET-FM (Eq. chi_ret): sigma / dx = 3.7, so the ball reaches 4 cells on each side; 3 tiles and
    a ragged tail; the RHS of an off-equilibrium state, then 6 steps (each stage feeds the averaged
    density of its output to the next)."""
    nx = 3 * 248 + 17
    w = _smooth_workload(16, nx, bc)
    w["kn"] = 3.7 / (nx * w["denseness"])  # sigma = E_l Kn L
    f = inputs.smooth_periodic_fields(nx, seed=77)
    ghost = None
    if bc == "fixed":
        ghost = [(f[0][0], f[1][0], f[2][0])] * 3 + [(f[0][-1] * 0.9, f[1][-1], f[2][-1])] * 3
    m, ph, th, s = _setup(gpu, w, precision, fields=f, ghost=ghost, chi_mode=1)
    assert O.fm_halfwidth(m.dx, m.sigma) == 4
    noise = inputs.state_noise(ph.shape, seed=78, scale=1e-2)
    ph = ph * noise
    s.set_state(ph, th)
    if precision == 1:
        ph, th = (a.astype(np.float32).astype(np.float64) for a in s.state())
    Lp_o, Lt_o = O.rhs(m, ph, th)
    Lp_g, Lt_g = s.rhs()
    for a, b in ((Lp_g, Lp_o), (Lt_g, Lt_o)):
        if precision == 0:
            scale = np.abs(b).max(axis=0) + 1e-300
            assert float((np.abs(a - b).max(axis=0) / scale).max()) <= 1e-11
        else:
            assert float(np.abs(a - b).max() / np.abs(b).max()) <= 2e-4
    ph, th = O.run(m, ph, th, 6)
    s.step(6)
    _check(m, ph, th, s, precision)


def test_ret_fm_differs_from_set(gpu):
    """The averaged density changes the result: the chi_RET-FM and chi_SET right-hand sides of the same
    state differ far beyond the FP64 tolerance, and the chi_RET-FM one matches its oracle."""
    nx = 300
    w = _smooth_workload(16, nx)
    w["kn"] = 3.7 / (nx * w["denseness"])
    f = inputs.smooth_periodic_fields(nx, seed=5, amp=(0.2, 0.1, 0.05))
    m, ph, th, s_ret = _setup(gpu, w, 0, fields=f, chi_mode=1)
    _, _, _, s_set = _setup(gpu, w, 0, fields=f, chi_mode=0)
    Lr, _ = s_ret.rhs()
    Ls, _ = s_set.rhs()
    assert np.abs(Lr - Ls).max() > 1e-6 * np.abs(Ls).max()
    Lo, _ = O.rhs(m, ph, th)
    assert np.abs(Lr - Lo).max() <= 1e-11 * np.abs(Lo).max()


@pytest.mark.parametrize("Q,bc,reach", [(48, "fixed", 4), (200, "periodic", 2)])
def test_large_q_ret_fm_matches_oracle(gpu, Q, bc, reach):
    """chi_RET-FM on the generic FP64 path (the paper's sigma = 1 shock runs use it with Q = 200): each stage
    averages the densities of its own input over the ball; the right-hand side and 3 steps against the oracle,
    a ball reaching `reach` cells on each side, and the chi_SET right-hand side of the same state differs."""
    nx = 40
    w = _smooth_workload(Q, nx, bc)
    w["kn"] = (reach - 0.3) / (nx * w["denseness"])  # sigma = E_l Kn L
    f = inputs.smooth_periodic_fields(nx, seed=Q + 5, amp=(0.2, 0.2, 0.1))
    ghost = None
    if bc == "fixed":
        ghost = [(f[0][0], f[1][0], f[2][0])] * 3 + [(f[0][-1] * 0.9, f[1][-1], f[2][-1])] * 3
    m, ph, th, s = _setup(gpu, w, 0, fields=f, ghost=ghost, chi_mode=1)
    assert O.fm_halfwidth(m.dx, m.sigma) == reach
    noise = inputs.state_noise(ph.shape, seed=Q + 6, scale=1e-2)
    ph = ph * noise
    s.set_state(ph, th)
    Lp_o, Lt_o = O.rhs(m, ph, th)
    Lp_g, Lt_g = s.rhs()
    for a, b in ((Lp_g, Lp_o), (Lt_g, Lt_o)):
        assert float(np.abs(a - b).max() / np.abs(b).max()) <= 1e-11
    _, _, _, s_set = _setup(gpu, w, 0, fields=f, ghost=ghost, chi_mode=0)
    s_set.set_state(ph, th)
    Ls, _ = s_set.rhs()
    assert np.abs(Lp_g - Ls).max() > 1e-6 * np.abs(Ls).max()
    ph, th = O.run(m, ph, th, 3)
    s.step(3)
    errs = _field_errors(m, ph, th, s)
    assert max(errs.values()) <= 1e-10, errs
    gp, gt = s.state()
    for a, b in ((gp, ph), (gt, th)):
        assert float(np.abs(a - b).max() / np.abs(b).max()) <= 1e-11


@pytest.mark.parametrize("Q", [16, 32])
def test_fp32_totals_kernel_matches_field_totals(gpu, Q):
    """The FP32 totals-only kernel (double-FP32 sums and reductions) gives the domain totals of the field
    kernel (FP64 per cell) to 1e-12, on several blocks and a ragged tail, and reports a negative density."""
    nx = 5 * 256 + 77
    w = _smooth_workload(Q, nx)
    m, ph, th, s = _setup(gpu, w, 1, fields=inputs.smooth_periodic_fields(nx, seed=Q, amp=(0.2, 0.3, 0.1)))
    s.step(3)
    t_only = s.totals()
    t_fields = s.moments()["totals"]
    np.testing.assert_allclose(t_only, t_fields, rtol=1e-12, atol=1e-14)
    ph2, th2 = s.state()
    ph2[nx // 2] *= -1.0
    s.set_state(ph2, th2)
    with pytest.raises(gpu.QLError) as e:
        s.totals()
    assert e.value.status == gpu.QL_ENONPHYSICAL


@pytest.mark.parametrize("Q,bc", [(48, "periodic"), (64, "fixed"), (100, "periodic"), (200, "periodic")])
def test_large_q_generic_path_matches_oracle(gpu, Q, bc):
    """Velocity sets without tiled kernels (the paper's near-ballistic runs use Q = 200) run on the generic
    FP64 path: its right-hand side and 3 steps against the oracle.  Errors are taken relative to the largest
    |psi| of each component: the outermost nodes carry weights below 1e-100, where both sides round
    differently in the Hermite sum."""
    nx = 40
    w = _smooth_workload(Q, nx, bc)
    w["kn"] = 0.05
    f = inputs.smooth_periodic_fields(nx, seed=Q)
    ghost = None
    if bc == "fixed":
        ghost = [(f[0][0], f[1][0], f[2][0])] * 3 + [(f[0][-1], f[1][-1], f[2][-1])] * 3
    m, ph, th, s = _setup(gpu, w, 0, fields=f, ghost=ghost)
    noise = inputs.state_noise(ph.shape, seed=Q + 1, scale=1e-2)
    ph = ph * noise
    s.set_state(ph, th)
    Lp_o, Lt_o = O.rhs(m, ph, th)
    Lp_g, Lt_g = s.rhs()
    for a, b in ((Lp_g, Lp_o), (Lt_g, Lt_o)):
        assert float(np.abs(a - b).max() / np.abs(b).max()) <= 1e-11
    ph, th = O.run(m, ph, th, 3)
    s.step(3)
    errs = _field_errors(m, ph, th, s)
    assert max(errs.values()) <= 1e-10, errs
    gp, gt = s.state()
    for a, b in ((gp, ph), (gt, th)):
        assert float(np.abs(a - b).max() / np.abs(b).max()) <= 1e-11
