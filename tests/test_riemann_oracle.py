"""Pins of the dense-gas shock-tube reference (oracle/riemann.py): the dilute limit against the textbook
ideal-gas solution, the Rankine-Hugoniot relations, and isentropy of the rarefaction in the
Carnahan-Starling entropy."""
import numpy as np
import pytest

import oracle as O
from oracle import riemann as R


def test_dilute_limit_is_the_ideal_gas_solution():
    st = R.ShockTube(R.DenseGas(1e-9), 1.0, 1.0, 0.125, 1.0)
    P, u, rho1, rho2, S = R.ideal_gas_sod(1.0, 1.0, 0.125, 0.125)
    np.testing.assert_allclose([st.Pc, st.uc, st.rho1, st.rho2, st.xi_s], [P, u, rho1, rho2, S], rtol=1e-7)


@pytest.mark.parametrize("El", [0.4825, 1.917])
def test_dense_shock_satisfies_rankine_hugoniot(El):
    g = R.DenseGas(O.eta_from_denseness(El))
    st = R.ShockTube(g, 1.0, 1.0, 0.125, 1.0)
    eR, T2 = 1.5 * 0.125 * 1.0, g.temperature(st.rho2, st.Pc)
    e2 = 1.5 * st.rho2 * T2
    scale = st.PL * st.xi_s
    assert abs(st.rho2 * (st.uc - st.xi_s) + st.xi_s * 0.125) < 1e-12
    assert abs(st.rho2 * st.uc * (st.uc - st.xi_s) + st.Pc - st.PR) < 1e-12 * scale
    assert abs((e2 + 0.5 * st.rho2 * st.uc ** 2) * (st.uc - st.xi_s) + st.uc * st.Pc + eR * st.xi_s) < 1e-12 * scale
    # the dense gas differs from the ideal one
    P, u, *_ = R.ideal_gas_sod(1.0, st.PL, 0.125, st.PR)
    assert abs(st.uc - u) > 1e-3


@pytest.mark.parametrize("El", [0.4825, 1.917])
def test_rarefaction_is_isentropic_for_the_carnahan_starling_gas(El):
    """Along dP = c_s^2 d rho with the sound speed of Sec. IV.B, the hard-sphere entropy
    (3/2) ln T - ln rho - eta (4 - 3 eta) / (1 - eta)^2 stays constant; the ideal-gas entropy does not."""
    g = R.DenseGas(O.eta_from_denseness(El))
    st = R.ShockTube(g, 1.0, 1.0, 0.125, 1.0)
    T = g.temperature(st.rho_t, st.P_t)
    eta = g.eta(st.rho_t)
    s = 1.5 * np.log(T) - np.log(st.rho_t) - eta * (4 - 3 * eta) / (1 - eta) ** 2
    assert s.max() - s.min() < 1e-8
    s_ideal = 1.5 * np.log(T) - np.log(st.rho_t)
    assert s_ideal.max() - s_ideal.min() > 1e-3


def test_profile_is_continuous_through_the_fan_and_piecewise_constant_elsewhere():
    g = R.DenseGas(O.eta_from_denseness(0.4825))
    st = R.ShockTube(g, 1.0, 1.0, 0.125, 1.0)
    eps = 1e-9
    r, u, T = st.sample([st.xi_head - eps, st.xi_head + eps, st.xi_tail - eps, st.xi_tail + eps])
    np.testing.assert_allclose(r, [1.0, 1.0, st.rho1, st.rho1], rtol=1e-6)
    np.testing.assert_allclose(u, [0.0, 0.0, st.uc, st.uc], atol=1e-6)
    r, u, T = st.sample([st.uc - eps, st.uc + eps, st.xi_s - eps, st.xi_s + eps])
    np.testing.assert_allclose(r, [st.rho1, st.rho2, st.rho2, 0.125], rtol=1e-12)
    # pressure continuous across the contact
    assert g.pressure(r[0], T[0]) == pytest.approx(g.pressure(r[1], T[1]), rel=1e-12)
