"""Each term of the stage kernel's right-hand side against the oracle's separately pinned pieces (moments,
Shakhov targets, tau and Pr; J1 with its CD6 gradients; WENO-5 advection), through ql_rhs:

  - a spatially uniform off-equilibrium state has no advection and no gradients: L is the relaxation alone;
  - L with the Enskog term minus L without it is J1 alone;
  - L minus the oracle's relaxation and J1 is the advection alone.

Several tiles and a ragged tail (N_x = 600), Q = 16 and 32, FP64 to 1e-11 and FP32 to 2e-5 of the largest |L|."""
import numpy as np
import pytest

import oracle as O
from paper_2211_16933_gb300 import inputs
from rhs_terms import rhs_terms

pytestmark = pytest.mark.gpu

NX, EL, KN = 600, 0.4, 0.05


def _pair(q, Q, precision, enskog, ph, th):
    p, _ = O.quadrature(Q)
    dt = inputs.cfl_dt(1.0 / NX, float(np.abs(p).max()))
    m = O.make_model(Q, NX, 1.0, dt, EL, KN, bc=O.BC_PERIODIC, enskog=enskog)
    r, u, T = O.fields(m, ph, th)["rho"], O.fields(m, ph, th)["u"], O.fields(m, ph, th)["T"]
    s = q.Solver(Q, NX, 1.0, dt, EL, KN, bc=q.QL_BC_PERIODIC, init_kind=q.QL_INIT_FIELDS, rho=r, u=u, T=T,
                 precision=precision, pr_mode=q.QL_PR_DENSE, enskog=enskog)
    s.set_state(ph, th)
    return m, s


def _state(Q, uniform):
    p, _ = O.quadrature(Q)
    m = O.make_model(Q, NX, 1.0, 1e-3, EL, KN, bc=O.BC_PERIODIC)
    r, u, T = inputs.smooth_periodic_fields(NX, seed=Q, amp=(0.1, 0.2, 0.1))
    if uniform:
        r, u, T = np.full(NX, r[0]), np.full(NX, u[0]), np.full(NX, T[0])
    ph, th = O.equilibrium_state(m, r, u, T)
    noise_p = inputs.state_noise((1 if uniform else NX, Q), seed=Q + 1, scale=2e-2)
    noise_t = inputs.state_noise((1 if uniform else NX, Q), seed=Q + 2, scale=2e-2)
    return ph * noise_p, th * noise_t


def _tol(precision):
    return 1e-11 if precision == 0 else 2e-5


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("Q", [16, 32])
def test_relaxation_term_alone(gpu, Q, precision):
    ph, th = _state(Q, uniform=True)
    m, s = _pair(gpu, Q, precision, 1, ph, th)
    Lp, Lt = s.rhs()
    relax, j1, adv = rhs_terms(m, ph, th)
    for c, L in enumerate((Lp, Lt)):
        scale = np.abs(relax[c]).max()
        # identical cells: J1 and the advection vanish (to rounding in the oracle's own pieces)
        assert np.abs(j1[c]).max() <= 1e-13 * scale and np.abs(adv[c]).max() <= 1e-13 * scale
        assert np.abs(L - relax[c]).max() <= _tol(precision) * scale


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("Q", [16, 32])
def test_enskog_and_advection_terms_alone(gpu, Q, precision):
    ph, th = _state(Q, uniform=False)
    m1, s1 = _pair(gpu, Q, precision, 1, ph, th)
    _, s0 = _pair(gpu, Q, precision, 0, ph, th)
    L1 = s1.rhs()
    L0 = s0.rhs()
    relax, j1, adv = rhs_terms(m1, ph, th)
    for c in range(2):
        scale = np.abs(L1[c]).max()
        assert np.abs(j1[c]).max() > 1e-3 * scale and np.abs(adv[c]).max() > 1e-3 * scale
        # J1: the difference of the two right-hand sides
        assert np.abs((L1[c] - L0[c]) - j1[c]).max() <= _tol(precision) * scale
        # advection: what remains after the oracle's relaxation and J1
        assert np.abs((relax[c] + j1[c] - L1[c]) - adv[c]).max() <= _tol(precision) * scale
