"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks one oracle function against something other than itself:
values printed in the paper (tests/golden/), closed forms, invariants, library
routines, or the paper's 3D formulas reduced by numerical integration.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _frac(s):
    return float(Fraction(s))


# ----------------------------------------------------------------- Sec. II.A-B
def test_denseness_matches_printed_values():
    """Printed (eta, E_l) pairs of Sec. IV reproduce from Eq. (chi) and E_l = 3/sqrt2 b n chi."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "denseness_eta.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 5
    for eta, El, dec in rows:
        got = O.denseness(float(eta))
        assert round(got, int(dec)) == pytest.approx(float(El), abs=0.6 * 10 ** -int(dec)), (eta, got, El)
        assert O.eta_from_denseness(float(El)) == pytest.approx(float(eta), rel=2e-4)


def test_chi_matches_carnahan_starling_eos():
    """Eq. (chi): chi = (P^hs/(n k T) - 1)/(n b) with n b = 4 eta, against the CS EOS form."""
    for eta in np.linspace(0.0, 0.5, 26):
        assert 1.0 + 4.0 * eta * O.chi_set(eta) == pytest.approx(O.cs_compressibility(eta), rel=1e-14)
    assert O.chi_set(0.0) == 1.0
    for El in (1e-3, 0.1, 0.5, 2.0):
        assert O.denseness(O.eta_from_denseness(El)) == pytest.approx(El, rel=1e-13)


def test_dense_prandtl_equals_viscosity_over_conductivity():
    """Pr of Sec. II.B equals c_P mu / lambda built from Eqs. (viscosity), (conductivity)
    with mu_ref / lambda_ref = (5/16)/(75/64) and c_P = 5/2."""
    for eta in (1e-6, 0.01, 0.1, 0.25, 0.4):
        chi = O.chi_set(eta)
        bn = 4 * eta
        Y = bn * chi
        mu_rel = O.mu_over_muref(bn, chi, 1.3)
        lam_rel = O.lambda_over_lambdaref(bn, chi, 1.3)
        pr = 2.5 * (5.0 / 16.0) * mu_rel / ((75.0 / 64.0) * lam_rel)
        assert O.prandtl_dense(Y) == pytest.approx(pr, rel=1e-13)
    assert O.prandtl_dense(0.0) == pytest.approx(2.0 / 3.0, rel=1e-15)


def test_tau_dilute_limit_is_hard_sphere_bgk():
    """E_l -> 0: tau -> mu_HS/(n T) = 5 sqrt(2 pi)/16 * l0 / (rho_hat sqrt T), the first
    Chapman-Enskog approximation for hard spheres with l0 = 1/(sqrt2 pi sigma^2 n0)."""
    m = O.make_model(16, 32, 2.0, 1e-3, 1e-9, 0.05)
    l0 = 0.05 * 2.0
    for rho, T in ((1.0, 1.0), (0.5, 2.0), (3.0, 0.7)):
        ref = 5.0 * math.sqrt(2 * math.pi) / 16.0 * l0 / (rho * math.sqrt(T))
        assert O.tau(m, rho, T) == pytest.approx(ref, rel=1e-7)


def test_tau_scales_with_sigma_at_fixed_eta():
    """Eq. (tau_sigma): tau = sigma g[eta]; at fixed E_l, sigma = E_l Kn L, so tau is linear in Kn."""
    a = O.make_model(16, 32, 1.0, 1e-3, 1.1, 0.01)
    b = O.make_model(16, 32, 1.0, 1e-3, 1.1, 0.03)
    for rho, T in ((1.0, 1.0), (1.4, 1.8)):
        assert O.tau(b, rho, T) == pytest.approx(3.0 * O.tau(a, rho, T), rel=1e-13)


# ----------------------------------------------------------------- Sec. II.D quadrature
@pytest.mark.parametrize("Q", [7, 8, 16, 24, 32, 48, 101, 150, 200])
def test_quadrature_matches_gauss_hermite_library(Q):
    """Up to Q = 100 the weights follow the printed formula; beyond it the normalised identity (READING c2b)."""
    p, w = O.quadrature(Q)
    x, wl = np.polynomial.hermite_e.hermegauss(Q)
    wl = wl / math.sqrt(2 * math.pi)
    np.testing.assert_allclose(p, x, rtol=0, atol=1e-12 * max(1.0, abs(x).max()))
    # weights of the outermost nodes fall below 1e-300 for large Q; compare where they are representable
    sel = wl > 1e-280
    np.testing.assert_allclose(w[sel], wl[sel], rtol=1e-11, atol=0)
    assert w.sum() == pytest.approx(1.0, abs=1e-13)


@pytest.mark.parametrize("Q", [8, 16, 24, 32])
def test_quadrature_moments_and_hermite_orthogonality(Q):
    """sum w_k p_k^j = (j-1)!! for even j <= 2Q-1, 0 for odd j; He orthogonality with norm l!."""
    p, w = O.quadrature(Q)
    assert w.sum() == pytest.approx(1.0, abs=1e-14)
    for j in range(0, 2 * Q):
        exact = 0.0 if j % 2 else float(np.prod(np.arange(j - 1, 0, -2, dtype=float)))
        got = float(np.sum(w * p ** j))
        scale = float(np.sum(w * np.abs(p) ** j))
        assert got == pytest.approx(exact, rel=1e-11, abs=1e-13 * scale), j
    for l in range(Q):
        for l2 in range(Q):
            if l + l2 > 2 * Q - 1:
                continue
            got = sum(w[k] * O.hermite(l, p[k]) * O.hermite(l2, p[k]) for k in range(Q))
            exact = math.factorial(l) if l == l2 else 0.0
            assert got == pytest.approx(exact, rel=1e-10, abs=1e-10 * math.factorial(max(l, l2)))
    # He_l against the library
    for l in range(12):
        c = np.zeros(l + 1)
        c[l] = 1
        for x in (-3.3, 0.0, 0.7, 5.1):
            assert O.hermite(l, x) == pytest.approx(np.polynomial.hermite_e.hermeval(x, c), rel=1e-13, abs=1e-13)


# ----------------------------------------------------------------- Eq. (feq)
def _gauss_raw_moment(j, u, T):
    return sum(math.comb(j, 2 * i) * u ** (j - 2 * i) * T ** i * float(np.prod(np.arange(2 * i - 1, 0, -2, dtype=float)))
               for i in range(j // 2 + 1))


@pytest.mark.parametrize("Q", [8, 16, 32])
def test_equilibrium_moments_exact_up_to_order_Q_minus_1(Q):
    """Discrete moments of n g_k equal the Maxwellian's raw moments for j <= N = Q-1 (READING c1),
    and the order-Q moment is not reproduced for u != 0, T != 1."""
    p, w = O.quadrature(Q)
    n, u, T = 1.3, 0.4, 1.25
    f = O.equilibrium(p, w, n, u, T)
    for j in range(Q):
        exact = n * _gauss_raw_moment(j, u, T)
        assert float(np.sum(f * p ** j)) == pytest.approx(exact, rel=1e-10, abs=1e-12 * max(1, abs(exact))), j
    f2 = O.equilibrium(p, w, n, 1.2, 1.8)
    jq = float(np.sum(f2 * p ** Q))
    assert abs(jq / (n * _gauss_raw_moment(Q, 1.2, 1.8)) - 1) > 1e-6
    # rest state of unit temperature: g_k = w_k
    np.testing.assert_allclose(O.equilibrium(p, w, 1.0, 0.0, 1.0), w, rtol=1e-15)


@pytest.mark.parametrize("Q", [16, 64, 200])
def test_moments_of_equilibrium_state(Q):
    """Moments of (phi, theta) = (n g_k, 2 T n g_k) return (n, u, T, Pi = n T, q = 0), also for the large
    velocity sets of the near-ballistic runs."""
    p, w = O.quadrature(Q)
    for n, u, T in ((1.0, 0.0, 1.0), (0.7, -0.3, 1.6), (2.0, 1.1, 0.8)):
        f = O.equilibrium(p, w, n, u, T)
        mo = O.moments(p, f, 2 * T * f)
        np.testing.assert_allclose(mo[:4], (n, u, T, n * T), rtol=1e-11, atol=1e-14)
        assert abs(mo[4]) < 1e-11


# ----------------------------------------------------------------- Sec. II.B-C collision terms
def _perp_nodes(T, npts=12):
    """Nodes and weights for expectations over xi_y, xi_z ~ N(0, T)."""
    x, wl = np.polynomial.hermite_e.hermegauss(npts)
    wl = wl / math.sqrt(2 * math.pi)
    Y, Z = np.meshgrid(x * math.sqrt(T), x * math.sqrt(T), indexing="ij")
    W = np.outer(wl, wl)
    return Y.ravel(), Z.ravel(), W.ravel()


def test_reduced_shakhov_equals_integrated_3d_shakhov():
    """phi_S/f_MB and theta_S/f_MB of Sec. II.C equal the 3D Shakhov factor of Sec. II.B
    integrated over p_y, p_z (weights 1 and p_y^2 + p_z^2) by product Gauss-Hermite."""
    Q = 16
    p, w = O.quadrature(Q)
    n, u, T, q, Pr = 1.2, 0.3, 1.4, 0.05, 0.55
    phiS, thS = O.shakhov(p, w, n, u, T, q, Pr)
    f = O.equilibrium(p, w, n, u, T)
    yy, zz, W = _perp_nodes(T)
    Pi = n * T
    for k in range(Q):
        xi = p[k] - u
        xi2 = xi ** 2 + yy ** 2 + zz ** 2
        fac = 1.0 + (1 - Pr) / (Pi * T) * (xi2 / (5 * T) - 1.0) * xi * q
        assert phiS[k] / f[k] == pytest.approx(np.sum(W * fac), rel=1e-12)
        assert thS[k] / f[k] == pytest.approx(np.sum(W * (yy ** 2 + zz ** 2) * fac), rel=1e-12)


def test_shakhov_collision_invariants_and_heat_flux():
    """sum phi_S = n, momentum and energy of the Shakhov target equal those of the state,
    and its heat flux is (1 - Pr) q (Q >= 7)."""
    Q = 16
    p, w = O.quadrature(Q)
    rng = np.random.default_rng(3)
    f0 = O.equilibrium(p, w, 1.1, 0.2, 1.3)
    phi = f0 * (1 + 0.2 * rng.standard_normal(Q) * np.exp(-0.1 * p ** 2))
    th = 2 * 1.3 * f0 * (1 + 0.2 * rng.standard_normal(Q) * np.exp(-0.1 * p ** 2))
    n, u, T, Pi, q = O.moments(p, phi, th)
    for Pr in (2.0 / 3.0, 0.4, 1.0):
        phiS, thS = O.shakhov(p, w, n, u, T, q, Pr)
        nS, uS, TS, PiS, qS = O.moments(p, phiS, thS)
        assert nS == pytest.approx(n, rel=1e-13)
        assert uS == pytest.approx(u, rel=1e-12)
        assert TS == pytest.approx(T, rel=1e-12)
        assert qS == pytest.approx((1 - Pr) * q, rel=1e-10, abs=1e-14)


def test_reduced_j1_equals_integrated_3d_j1():
    """J1^phi, J1^theta of Eq. (j1_expanded), with b rho chi on both lines (READING c4), equal
    the 3D J1(f_MB, f_MB) of Sec. II.B with 1D gradients, integrated over p_y, p_z."""
    Q = 16
    p, w = O.quadrature(Q)
    n, u, T, Y = 0.9, -0.2, 1.7, 0.37
    dlnchi, dlnrho, du, dlnT = 0.21, -0.8, 0.33, 0.57
    jp, jt = O.j1(p, w, n, u, T, Y, dlnchi, dlnrho, du, dlnT)
    f = O.equilibrium(p, w, n, u, T)
    yy, zz, W = _perp_nodes(T)
    for k in range(Q):
        xix = p[k] - u
        xi2 = xix ** 2 + yy ** 2 + zz ** 2
        z2 = xi2 / (2 * T)
        zx2 = xix ** 2 / (2 * T)
        brace = (xix * (2 * dlnrho + dlnchi + dlnT + 0.6 * (z2 - 2.5) * dlnT)
                 + 0.4 * (2 * zx2 * du + (z2 - 2.5) * du))
        j3 = -Y * brace
        assert jp[k] / f[k] == pytest.approx(np.sum(W * j3), rel=1e-11, abs=1e-13)
        assert jt[k] / f[k] == pytest.approx(np.sum(W * (yy ** 2 + zz ** 2) * j3), rel=1e-11, abs=1e-13)


def test_j1_moments_are_collisional_transfer():
    """Mass moment of J1 is 0, momentum moment is -d_x(P_c), energy moment is -d_x(P_c u),
    with P_c = b rho chi n T and d_x ln P_c = d ln chi + 2 d ln rho + d ln T (Y fixed at the cell)."""
    Q = 16
    p, w = O.quadrature(Q)
    n, u, T, Y = 1.3, 0.45, 1.2, 0.61
    g = dict(dlnchi=0.1, dlnrho=-0.35, du=0.27, dlnT=0.44)
    jp, jt = O.j1(p, w, n, u, T, Y, g["dlnchi"], g["dlnrho"], g["du"], g["dlnT"])
    Pc = Y * n * T
    dPc = Pc * (g["dlnchi"] + 2 * g["dlnrho"] + g["dlnT"])
    assert abs(jp.sum()) < 1e-13
    assert float(np.sum(p * jp)) == pytest.approx(-dPc, rel=1e-12)
    energy = 0.5 * float(np.sum(p ** 2 * jp + jt))
    assert energy == pytest.approx(-(dPc * u + Pc * g["du"]), rel=1e-12)


# ----------------------------------------------------------------- App. A numerics
def test_weno_zero_indicator_table():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "weno_zero_table.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 7
    for r in rows:
        z = [int(v) for v in r[:3]]
        want = [_frac(v) for v in r[3:]]
        b = [0.0 if zi else 0.37 * (i + 1) for i, zi in enumerate(z)]
        np.testing.assert_allclose(O.weno5_weights(*b), want, rtol=0, atol=1e-16)


def test_weno_weights_limits_of_general_formula():
    """Each table row is the limit of delta_q/beta_q^2 normalized as the zero betas shrink."""
    delta = [_frac(v) for v in open(os.path.join(GOLDEN, "weno_ideal_weights.txt")).read().split("\n")[1].split()]
    assert delta == pytest.approx([0.1, 0.6, 0.3])
    for z in ((0, 1, 1), (1, 0, 1), (1, 1, 0), (1, 0, 0)):
        b = [1e-60 if zi else 0.5 for zi in z]
        lim = O.weno5_weights(*[0.0 if zi else 0.5 for zi in z])
        np.testing.assert_allclose(O.weno5_weights(*b), lim, atol=1e-12)
    b = (0.2, 0.5, 0.9)
    t = np.array(delta) / np.array(b) ** 2
    np.testing.assert_allclose(O.weno5_weights(*b), t / t.sum(), rtol=1e-15)


def test_weno_is_scale_invariant_down_to_the_smallest_weights():
    """The weights depend on the ratios of the indicators only and the face value is homogeneous of degree one
    in f: both hold at the magnitudes of the outer nodes of Q = 200 (psi ~ 1e-165, indicators ~ 1e-330 would
    underflow if squared; READING c23), where the quotient form gives inf / inf."""
    for b in ((0.2, 0.5, 0.9), (1.0, 1e-30, 3.0), (2.0, 1.0, 1e-100)):
        ref = O.weno5_weights(*b)
        for c in (1e-200, 1e-150, 1e150, 1e200):  # every scaled indicator stays a normal double
            got = O.weno5_weights(*(c * x for x in b))
            np.testing.assert_allclose(got, ref, rtol=1e-14, atol=1e-300)
    f = np.array([0.3, -0.1, 0.7, 1.2, 0.4])
    ref = O.weno5_face(f)
    for c in (2.0 ** -540, 1e-160, 1e-100):
        assert O.weno5_face(c * f) == pytest.approx(c * ref, rel=1e-13)


def _weno_derivative(f, dx):
    """(face_{i+1/2} - face_{i-1/2})/dx on a periodic array, positive advection."""
    N = len(f)
    face = np.array([O.weno5_face(f[[(i + r) % N for r in range(-2, 3)]]) for i in range(N)])
    return (face - np.roll(face, 1)) / dx


def test_weno_exact_for_quadratics_and_fifth_order():
    N = 40
    x = np.arange(N) * 0.1
    for f, d in ((2.0 + 0.5 * x, 0.5 + 0 * x), (1.0 - 0.3 * x + 0.07 * x ** 2, -0.3 + 0.14 * x)):
        dx = 0.1
        got = np.array([(O.weno5_face(f[i - 2:i + 3]) - O.weno5_face(f[i - 3:i + 2])) / dx for i in range(3, N - 2)])
        np.testing.assert_allclose(got, d[3:N - 2], rtol=0, atol=1e-12)
    errs = []
    for N in (16, 32, 64):
        dx = 1.0 / N
        x = np.arange(-3, N + 3) * dx
        f = np.exp(x)
        got = np.array([(O.weno5_face(f[i + 1:i + 6]) - O.weno5_face(f[i:i + 5])) / dx for i in range(N)])
        errs.append(np.abs(got - np.exp(x[3:N + 3])).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders.min() > 4.6, orders


def test_cd6_exact_for_degree_six():
    dx, x0 = 0.13, 0.4
    xs = x0 + dx * np.arange(-3, 4)
    for d in range(7):
        assert O.cd6(xs ** d, dx) == pytest.approx(d * x0 ** (d - 1) if d else 0.0, abs=1e-11)
    assert abs(O.cd6(xs ** 7, dx) - 7 * x0 ** 6) > 1e-8


def _butcher_stability(z):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "rk3_butcher.txt")) if l.strip() and l[0] != "#"]
    A = np.zeros((3, 3))
    b = None
    s = 0
    for r in rows:
        if r[0] == "c":
            if "|" in r:
                vals = [_frac(v) for v in r[r.index("|") + 1:]]
                A[s, :len(vals)] = vals
            s += 1
        else:
            b = np.array([_frac(v) for v in r[1:]])
    return 1.0 + z * b @ np.linalg.solve(np.eye(3) - z * A, np.ones(3))


def test_rk3_matches_butcher_tableau_on_linear_relaxation():
    """A uniform non-equilibrium state with Pr = 1 relaxes linearly to a fixed f_MB: one step of
    Eq. (rk3) multiplies psi - f_MB by the tableau's stability polynomial R(-dt/tau)."""
    Q, nx = 16, 4
    for ratio in (0.3, 1.0, 2.2):
        m0 = O.make_model(Q, nx, 1.0, 1.0, 0.1, 0.02, pr_mode=0, pr_const=1.0)
        p, w = O.velocity_set(m0)
        f0 = O.equilibrium(p, w, 1.0, 0.0, 1.0)
        bump = 0.05 * np.sin(p) * f0
        phi1 = f0 + bump
        th1 = 2 * f0 * (1 + 0.03 * np.cos(p))
        n, u, T, _, _ = O.moments(p, phi1, th1)
        tau = O.tau(m0, n, T)
        m = O.make_model(Q, nx, 1.0, ratio * tau, 0.1, 0.02, pr_mode=0, pr_const=1.0)
        phi = np.tile(phi1, (nx, 1))
        th = np.tile(th1, (nx, 1))
        ph2, th2 = O.run(m, phi, th, 1)
        feq = O.equilibrium(p, w, n, u, T)
        R = _butcher_stability(-ratio)
        np.testing.assert_allclose(ph2[0] - feq, R * (phi1 - feq), rtol=1e-9, atol=1e-15)
        np.testing.assert_allclose(th2[0] - 2 * T * feq, R * (th1 - 2 * T * feq), rtol=1e-9, atol=1e-15)


def test_advection_term_is_fifth_order_upwind_derivative():
    """With collisions switched off (Kn huge, J1 off), L[psi_k] -> -p_k d_x psi_k."""
    Q = 8
    errs = []
    for nx in (32, 64):
        m = O.make_model(Q, nx, 1.0, 1e-3, 0.1, 1e14, enskog=0)
        p, w = O.velocity_set(m)
        x = (np.arange(nx) + 0.5) / nx
        f0 = O.equilibrium(p, w, 1.0, 0.0, 1.0)
        ph = f0[None, :] * (1 + 0.1 * np.sin(2 * np.pi * x[:, None] + np.arange(Q)[None, :]))
        th = 2 * ph * (1 + 0.05 * np.cos(2 * np.pi * x[:, None]))
        Lp, Lt = O.rhs(m, ph, th)
        dph = f0[None, :] * 0.1 * 2 * np.pi * np.cos(2 * np.pi * x[:, None] + np.arange(Q)[None, :])
        errs.append(np.abs(Lp + p[None, :] * dph).max())
    assert errs[1] < errs[0] / 20, errs


# ----------------------------------------------------------------- whole-model invariants
def _random_periodic_state(m, seed):
    rng = np.random.default_rng(seed)
    x = (np.arange(m.nx) + 0.5) / m.nx * m.L
    rho = 1.0 + 0.05 * np.sin(2 * np.pi * x / m.L + rng.uniform(0, 6))
    u = 0.1 * np.cos(2 * np.pi * x / m.L + rng.uniform(0, 6))
    T = 1.0 + 0.04 * np.sin(4 * np.pi * x / m.L + rng.uniform(0, 6))
    ph, th = O.equilibrium_state(m, rho, u, T)
    ph = ph * (1 + 0.01 * rng.standard_normal(ph.shape) * np.exp(-0.2 * O.velocity_set(m)[0] ** 2))
    return ph, th


@pytest.mark.parametrize("bc", [O.BC_PERIODIC, O.BC_FIXED])
def test_uniform_equilibrium_is_a_fixed_point(bc):
    """A uniform equilibrium is stationary with J1 on, for periodic cells and for fixed ghost
    cells holding the same state (READING c10)."""
    m = O.make_model(16, 12, 1.0, 2e-3, 1.1, 0.05, bc=bc)
    state = (1.2, 0.3, 0.9)
    O.set_ghosts(m, [state] * 3, [state] * 3)
    ph, th = O.equilibrium_state(m, np.full(12, state[0]), np.full(12, state[1]), np.full(12, state[2]))
    ph2, th2 = O.run(m, ph, th, 5)
    np.testing.assert_allclose(ph2, ph, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(th2, th, rtol=1e-12, atol=1e-15)


def test_conservation_periodic():
    """J1 off: mass, momentum, energy conserved to rounding (flux form + Shakhov invariants).
    J1 on: mass still conserved to rounding (zero mass moment of J1)."""
    for enskog in (0, 1):
        m = O.make_model(16, 48, 1.0, 1e-3, 1.1, 0.05, enskog=enskog)
        ph, th = _random_periodic_state(m, 11)
        t0 = O.totals(m, ph, th)
        ph2, th2 = O.run(m, ph, th, 10)
        t1 = O.totals(m, ph2, th2)
        assert abs(t1[0] - t0[0]) < 1e-13
        if enskog == 0:
            assert abs(t1[1] - t0[1]) < 1e-13
            assert abs(t1[2] - t0[2]) < 1e-13


def test_mirror_symmetry_of_rhs():
    """x -> L - x with p_k -> -p_k maps the RHS onto itself mirrored (upwind mirror of READING c8)."""
    m = O.make_model(16, 40, 1.0, 1e-3, 1.1, 0.05)
    ph, th = _random_periodic_state(m, 5)
    Lp, Lt = O.rhs(m, ph, th)
    phr, thr = ph[::-1, ::-1].copy(), th[::-1, ::-1].copy()
    Lpr, Ltr = O.rhs(m, phr, thr)
    np.testing.assert_allclose(Lpr, Lp[::-1, ::-1], rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(Ltr, Lt[::-1, ::-1], rtol=1e-9, atol=1e-13)


def test_sound_wave_initial_pressure_is_uniform_and_eos():
    m = O.make_model(16, 64, 1.0, 1e-3, 1.1, 0.1, pr_mode=0)
    r, u, T = O.init_fields(m, O.INIT_SOUND, [1.0, 1.0, 1e-3])
    ph, th = O.equilibrium_state(m, r, u, T)
    f = O.fields(m, ph, th)
    Z = np.array([O.cs_compressibility(m.eta0 * ri) for ri in f["rho"]])
    np.testing.assert_allclose(f["P"], f["rho"] * f["T"] * Z, rtol=1e-13)
    assert np.ptp(f["P"]) < 1e-13
    assert np.ptp(f["rho"]) == pytest.approx(2e-3, rel=1e-2)


def test_sound_speed_formulas_agree():
    """The c_s^2 of Sec. IV.B (oracle) equals Eq. (sw_cs), d_rho P + P/(rho^2 c_V) d_T P with c_V = 3/2,
    the derivatives of P = rho T Z_CS(eta0 rho) taken by central differences."""
    for El in (1e-8, 0.48, 1.1, 4.4):
        eta0 = O.eta_from_denseness(El)
        rho, T = 1.0, 1.0

        def P(r, t):
            return r * t * O.cs_compressibility(eta0 * r)
        h = 1e-5
        dPr = (P(rho + h, T) - P(rho - h, T)) / (2 * h)
        dPT = (P(rho, T + h) - P(rho, T - h)) / (2 * h)
        cs2 = dPr + P(rho, T) / (rho ** 2 * 1.5) * dPT
        assert O.sound_speed2(eta0, 1.0, rho, T) == pytest.approx(cs2, rel=1e-8)
    assert O.sound_speed2(0.0, 1.0, 1.0, 1.0) == pytest.approx(5.0 / 3.0, rel=1e-15)


def test_rankine_hugoniot_dilute_and_dense():
    # dilute: textbook gamma = 5/3 normal-shock jumps
    for M in (1.4, 2.0, 3.0):
        g = 5.0 / 3.0
        u1, r2, u2, T2 = O.rankine_hugoniot(1e-12, 1.0, 1.0, 1.0, M)
        r_ratio = (g + 1) * M ** 2 / ((g - 1) * M ** 2 + 2)
        p_ratio = 1 + 2 * g / (g + 1) * (M ** 2 - 1)
        assert r2 == pytest.approx(r_ratio, rel=1e-9)
        assert T2 == pytest.approx(p_ratio / r_ratio, rel=1e-9)
        assert u1 == pytest.approx(M * math.sqrt(g), rel=1e-9)
    assert O.rankine_hugoniot(1e-12, 1.0, 1.0, 1.0, 2.0)[3] == pytest.approx(2.078125, rel=1e-9)
    # dense: the jump conditions hold with the dense EOS
    for El in (0.05, 0.1, 0.2, 1.1):
        eta0 = O.eta_from_denseness(El)
        for M in (1.4, 2.0, 3.0):
            u1, r2, u2, T2 = O.rankine_hugoniot(eta0, 1.0, 1.0, 1.0, M)
            P1 = 1.0 * O.cs_compressibility(eta0)
            P2 = r2 * T2 * O.cs_compressibility(eta0 * r2)
            assert u1 == r2 * u2 or abs(u1 - r2 * u2) < 1e-13
            assert u1 ** 2 + P1 == pytest.approx(r2 * u2 ** 2 + P2, rel=1e-13)
            E1 = (1.5 + 0.5 * u1 ** 2 + P1) * u1
            E2 = (1.5 * r2 * T2 + 0.5 * r2 * u2 ** 2 + P2) * u2
            assert E1 == pytest.approx(E2, rel=1e-12)
            assert r2 > 1.0 and T2 > 1.0


@pytest.mark.slow
def test_sound_speed_of_dense_gas_from_a_run():
    """A small-amplitude sound wave of the full model propagates at the dense-gas c_s of
    Eq. (sw_cs) (closed form above), which the simplified Enskog term J1 must produce;
    with J1 switched off it propagates at the ideal-gas value sqrt(5/3)."""
    from scipy.optimize import curve_fit
    El, nx, Q, kn = 1.1057637, 48, 16, 2e-3
    for enskog in (1, 0):
        p, _ = O.quadrature(Q)
        dt = 0.35 * (1.0 / nx) / p.max()
        m = O.make_model(Q, nx, 1.0, dt, El, kn, pr_mode=1, enskog=enskog)
        r, u, T = O.init_fields(m, O.INIT_SOUND, [1.0, 1.0, 1e-4])
        ph, th = O.equilibrium_state(m, r, u, T)
        x = (np.arange(nx) + 0.5) / nx
        ts, amps = [], []
        every, nsamp = 8, 110
        for s in range(nsamp):
            f = O.fields(m, ph, th)
            ts.append(s * every * dt)
            amps.append(2.0 / nx * np.sum(f["rho"] * np.cos(2 * np.pi * x)))
            ph, th = O.run(m, ph, th, every)
        ts, amps = np.array(ts), np.array(amps) / 1e-4
        cs_exact = math.sqrt(O.sound_speed2(m.eta0, 1.0, 1.0, 1.0)) if enskog else math.sqrt(5.0 / 3.0)
        k = 2 * np.pi

        def model(t, a, at, b, aa, c, om):
            return a * np.exp(-at * t) + np.exp(-aa * t) * (b * np.cos(om * t) + c * np.sin(om * t))
        popt, _ = curve_fit(model, ts, amps, p0=[0.3, 0.1, 0.7, 0.1, 0.0, k * cs_exact], maxfev=20000)
        assert popt[5] / k == pytest.approx(cs_exact, rel=1e-3), (enskog, popt[5] / k, cs_exact)


# ---------------------------------------------------------------------------
# chi_RET-FM (Eq. chi_ret): the Fischer-Methfessel density average


def _ball_fraction_below(t, sigma):
    """Fraction of a ball of radius sigma lying at x < t: the spherical cap of height h = sigma + t has
    volume pi h^2 (3 sigma - h) / 3 (textbook cap formula)."""
    h = min(max(sigma + t, 0.0), 2 * sigma)
    return math.pi * h * h * (3 * sigma - h) / 3.0 / (4.0 / 3.0 * math.pi * sigma ** 3)


@pytest.mark.parametrize("ratio", [0.3, 0.5, 1.0, 2.0, 2.6, 7.3])
def test_fm_weights_are_ball_volume_fractions(ratio):
    """K_d is the fraction of the ball's volume inside cell d: differences of spherical-cap volumes."""
    dx, sigma = 0.37, 0.37 * ratio
    W = O.fm_halfwidth(dx, sigma)
    assert (W - 0.5) * dx < sigma <= (W + 0.5) * dx or (W == 0 and sigma <= 0.5 * dx)
    tot = 0.0
    for d in range(-W - 2, W + 3):
        ref = _ball_fraction_below((d + 0.5) * dx, sigma) - _ball_fraction_below((d - 0.5) * dx, sigma)
        k = O.fm_weight(d, dx, sigma)
        assert k == pytest.approx(ref, abs=1e-14)
        if abs(d) > W:
            assert k == 0.0
        tot += k
    assert tot == pytest.approx(1.0, abs=1e-14)


def test_fm_average_of_a_fourier_mode_and_reduction_to_the_local_density():
    """Periodic: the average of c + A sin(k x) is c + A sin(k x) sum_d K_d cos(k d dx) (symmetric
    kernel); for sigma <= dx/2 the ball stays inside the cell and nbar = n."""
    nx, L = 40, 1.0
    for kn, expect_identity in ((0.05, False), (0.005, True)):
        m = O.make_model(16, nx, L, 1e-3, 1.1, kn, bc=O.BC_PERIODIC)
        dx, sigma = L / nx, 1.1 * kn * L
        W = O.fm_halfwidth(dx, sigma)
        x = (np.arange(-3, nx + 3) + 0.5) * dx
        k = 2 * np.pi * 3 / L
        n = 1.0 + 0.2 * np.sin(k * x)
        nbar = O.fm_average(m, n)
        gain = sum(O.fm_weight(d, dx, sigma) * math.cos(k * d * dx) for d in range(-W, W + 1))
        np.testing.assert_allclose(nbar, 1.0 + 0.2 * gain * np.sin(k * x), rtol=0, atol=1e-14)
        if expect_identity:
            assert W == 0 and gain == pytest.approx(1.0, abs=1e-15)
        else:
            assert W >= 2 and gain < 0.99


def test_fm_average_fixed_boundaries_continue_the_ghost_density():
    """Fixed ghosts: beyond the ghost cells the density is that of the outermost ghost cell, so a
    state uniform near each end averages to that end's density."""
    nx = 30
    m = O.make_model(16, nx, 1.0, 1e-3, 1.1, 0.1, bc=O.BC_FIXED)
    dx, sigma = 1.0 / nx, 1.1 * 0.1
    W = O.fm_halfwidth(dx, sigma)
    assert W == 3
    n = np.where(np.arange(-3, nx + 3) < nx // 2, 1.0, 0.25)
    nbar = O.fm_average(m, n)
    i = np.arange(-3, nx + 3)
    far = np.abs(i + 0.5 - nx // 2) > W + 0.5
    np.testing.assert_allclose(nbar[far], n[far], rtol=0, atol=1e-15)
    # next to the jump the average mixes both states with the cap weights
    j = nx // 2 + 3  # cell nx//2 (first of the right state) in the extended array
    ref = sum(O.fm_weight(d, dx, sigma) * (1.0 if d < 0 else 0.25) for d in range(-W, W + 1))
    assert nbar[j] == pytest.approx(ref, abs=1e-15)


def test_ret_fm_uniform_equilibrium_is_a_fixed_point():
    for bc in (O.BC_PERIODIC, O.BC_FIXED):
        m = O.make_model(16, 12, 1.0, 2e-3, 1.1, 0.1, bc=bc, chi_mode=O.CHI_RET_FM)
        state = (1.2, 0.3, 0.9)
        O.set_ghosts(m, [state] * 3, [state] * 3)
        ph, th = O.equilibrium_state(m, np.full(12, state[0]), np.full(12, state[1]), np.full(12, state[2]))
        Lp, Lt = O.rhs(m, ph, th)
        assert np.abs(Lp).max() < 1e-12 and np.abs(Lt).max() < 1e-12


def test_ret_fm_collision_terms_from_pinned_parts():
    """RHS(RET-FM) - RHS(SET) is the difference of the collision terms alone (the advection is the
    same); rebuild it cell by cell from the pinned pieces with chi = chi_SET(nbar) in b rho chi, tau,
    Pr and J1, and d ln chi the 6th-order difference of ln chi(nbar)."""
    nx, L, El, kn = 36, 1.0, 1.1, 0.08
    mr = O.make_model(16, nx, L, 1e-3, El, kn, chi_mode=O.CHI_RET_FM)
    ms = O.make_model(16, nx, L, 1e-3, El, kn, chi_mode=O.CHI_SET)
    ph, th = _random_periodic_state(ms, 21)
    Lr_p, Lr_t = O.rhs(mr, ph, th)
    Ls_p, Ls_t = O.rhs(ms, ph, th)
    p, w = O.velocity_set(ms)
    dx, sigma, eta0 = L / nx, El * kn * L, ms.eta0
    ext = np.arange(-3, nx + 3) % nx
    mom = np.array([O.moments(p, ph[i], th[i]) for i in range(nx)])
    n_ext = mom[ext, 0]
    nbar = O.fm_average(mr, n_ext)
    lnchi_ret = np.log([O.chi_set(eta0 * v) for v in nbar])
    lnn, uu, lnT = np.log(mom[ext, 0]), mom[ext, 1], np.log(mom[ext, 2])
    b = 2 * math.pi * sigma ** 3 / 3
    mu_ref = 5.0 / (16.0 * sigma * sigma) * math.sqrt(1 / math.pi)

    def coll(i, chi, dlnchi):
        n, u, T, q = mom[i, 0], mom[i, 1], mom[i, 2], mom[i, 4]
        eta = eta0 * n
        Y = 4 * eta * chi
        tau = mu_ref * O.mu_over_muref(4 * eta, chi, T) / ((4 * eta / b) * T)
        Pr = O.prandtl_dense(Y)
        j = i + 3
        dlnrho, du, dlnT = (O.cd6(a[j - 3:j + 4], dx) for a in (lnn, uu, lnT))
        phS, thS = O.shakhov(p, w, n, u, T, q, Pr)
        jp, jt = O.j1(p, w, n, u, T, Y, dlnchi, dlnrho, du, dlnT)
        return -(ph[i] - phS) / tau + jp, -(th[i] - thS) / tau + jt

    worst = 0.0
    for i in range(nx):
        j = i + 3
        eta = eta0 * mom[i, 0]
        dlnrho = O.cd6(lnn[j - 3:j + 4], dx)
        cs_p, cs_t = coll(i, O.chi_set(eta), eta * (3 / (1 - eta) - 1 / (2 - eta)) * dlnrho)
        cr_p, cr_t = coll(i, math.exp(lnchi_ret[j]), O.cd6(lnchi_ret[j - 3:j + 4], dx))
        scale = np.abs(Ls_p[i]).max()
        np.testing.assert_allclose(Lr_p[i] - Ls_p[i], cr_p - cs_p, rtol=0, atol=1e-10 * scale)
        np.testing.assert_allclose(Lr_t[i] - Ls_t[i], cr_t - cs_t, rtol=0, atol=1e-10 * np.abs(Ls_t[i]).max())
        worst = max(worst, np.abs(cr_p - cs_p).max() / scale)
    assert worst > 1e-4  # the two closures do differ on this state


def test_ret_fm_conserves_mass_and_is_mirror_symmetric():
    m = O.make_model(16, 40, 1.0, 1e-3, 1.1, 0.06, chi_mode=O.CHI_RET_FM)
    ph, th = _random_periodic_state(m, 8)
    t0 = O.totals(m, ph, th)
    ph2, th2 = O.run(m, ph, th, 10)
    assert abs(O.totals(m, ph2, th2)[0] - t0[0]) < 1e-13
    Lp, Lt = O.rhs(m, ph, th)
    Lpr, Ltr = O.rhs(m, ph[::-1, ::-1].copy(), th[::-1, ::-1].copy())
    np.testing.assert_allclose(Lpr, Lp[::-1, ::-1], rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(Ltr, Lt[::-1, ::-1], rtol=1e-9, atol=1e-13)


# ---------------------------------------------------------------------------
# Sound-wave modes (Eqs. sw_cs, sw_coeff)


@pytest.mark.parametrize("El", [0.01, 0.4825, 1.917, 6.3])
def test_sound_modes_are_the_small_k_roots_of_the_linear_hydrodynamic_equations(El):
    """The closed forms for c_s, alpha_a and alpha_t agree with the roots of the secular cubic of the
    linearised mass, momentum and energy equations with the same coefficients (perturbations exp(ikx - alpha t))
    to O((k l)^2); the roots are found by numpy's polynomial solver."""
    m = O.make_model(16, 64, 1.0, 1e-3, El, 1e-3)
    rho, T, k = 1.0, 1.0, 2 * math.pi
    cs, aa, aa0, at, gamma = O.sound_modes(m, rho, T, k)
    # coefficients of the linear equations, from the same model pieces
    eta = m.eta0 * rho
    chi = O.chi_set(eta)
    Y = 4 * eta * chi
    dchi = (5 - 2 * eta) / (2 * (1 - eta) ** 4)
    Z, dZ = 1 + Y, 4 * chi + 4 * eta * dchi
    Prho, PT = T * (Z + eta * dZ), rho * Z
    mu = O.tau(m, rho, T) * rho * T
    lam = 2.5 * mu / O.prandtl(m, rho)
    muv = mu * 16 / (5 * math.pi) * Y * Y / (1 + 0.8 * Y + 0.16 * (1 + 12 / math.pi) * Y * Y)
    D, cV = 4 * mu / 3 + muv, 1.5
    a, c = rho, rho * cV
    coeffs = [-a * c, k * k * (a * lam + c * D), -(k ** 4 * D * lam + k * k * T * PT ** 2 + k * k * rho * Prho * c),
              k ** 4 * rho * Prho * lam]
    roots = np.roots(coeffs)
    real = roots[np.abs(roots.imag) < 1e-12 * np.abs(roots).max()].real
    cplx = roots[roots.imag > 0][0]
    kl = k * mu / (rho * cs)  # k times a viscous length
    assert abs(cplx.imag - k * cs) <= 2 * kl ** 2 * k * cs
    assert abs(cplx.real - aa) <= 2 * kl ** 2 * aa
    assert abs(real[0] - at) <= 2 * kl ** 2 * at
    # the thermodynamic identity c_s^2 = gamma (dP/drho)_T with c_P - c_V = T PT^2 / (rho^2 Prho)
    assert gamma * cV - cV == pytest.approx(T * PT ** 2 / (rho ** 2 * Prho), rel=1e-12)
    assert aa >= aa0 and (aa - aa0) / aa < (0.5 if El > 1 else 0.05)


def test_hermite_equilibrium_conditioning_bounded_only_below_twice_the_reference_temperature():
    """READINGS c17, c24: the weighted L2 norm of the Maxwellian against the Gauss-Hermite weight is finite only for
    T < 2, so the conditioning kappa = sum_k |g_k| / n of the discrete equilibrium stays near 1 for every Q below
    it and grows without bound with Q above it (the Mach 2.0 downstream state u = 1.19, T = 2.08; T = 2.5 at rest)."""
    def kappa(Q, u, T):
        p, w = O.quadrature(Q)
        return float(np.abs(O.equilibrium(p, w, 1.0, u, T)).sum())

    for u, T in ((0.0, 1.5), (1.19, 1.8), (2.64, 1.0)):
        assert max(kappa(Q, u, T) for Q in (16, 32, 48, 64)) < 2.0, (u, T)
    for u, T in ((1.19, 2.08), (0.0, 2.5)):
        k = [kappa(Q, u, T) for Q in (16, 32, 48, 64)]
        assert all(b > 3.0 * a for a, b in zip(k[1:], k[2:])) and k[-1] > 1e3, (u, T, k)


def test_rhs_is_the_sum_of_its_pinned_terms():
    """The oracle's right-hand side equals relaxation + J1 - advection rebuilt cell by cell from the separately
    pinned moments, Shakhov targets, J1, CD6 and WENO-5 faces (periodic, off-equilibrium state)."""
    from rhs_terms import rhs_terms
    from paper_2211_16933_gb300 import inputs
    nx, Q = 24, 16
    p, _ = O.quadrature(Q)
    m = O.make_model(Q, nx, 1.0, 1e-3, 0.4, 0.05, bc=O.BC_PERIODIC)
    r, u, T = inputs.smooth_periodic_fields(nx, seed=3, amp=(0.1, 0.2, 0.1))
    ph, th = O.equilibrium_state(m, r, u, T)
    ph = ph * inputs.state_noise(ph.shape, seed=4, scale=2e-2)
    th = th * inputs.state_noise(th.shape, seed=5, scale=2e-2)
    Lp, Lt = O.rhs(m, ph, th)
    relax, j1, adv = rhs_terms(m, ph, th)
    for c, L in enumerate((Lp, Lt)):
        np.testing.assert_allclose(relax[c] + j1[c] - adv[c], L, rtol=0, atol=1e-12 * np.abs(L).max())
    assert np.abs(j1[0]).max() > 1e-3 * np.abs(Lp).max()  # every term matters here
    assert np.abs(adv[0]).max() > 1e-3 * np.abs(Lp).max()
