"""Inviscid limit of the dense-gas shock tube: the exact Riemann solution of the
Euler equations with the Carnahan-Starling equation of state (Sec. IV.B,
"Inviscid limit", Eqs. euler, euler_xi, sod_sol, rankine_hugoniot).

TEST INFRASTRUCTURE ONLY: used by tests/ as an analytic reference for the
solver's shock-tube runs at small Knudsen number.  Plain numpy, FP64.

Units as in Sec. II.A (m = k_B = 1, rho = n).  Gas: P = rho T Z(eta),
Z = 1 + 4 eta chi_SET(eta), eta = eta0 rho / rho_ref; internal energy density
e = (3/2) rho T (hard spheres carry no potential energy).

Wave pattern for a left state at higher pressure: a left-facing rarefaction
(along which P and rho follow dP = c_s^2 d rho and u + int c_s / rho d rho is
constant, Eq. sod_sol), a contact at u = u_c, and a right-facing shock
(Eq. rankine_hugoniot).  READING c20: the energy relation of Eq.
(rankine_hugoniot) is printed with +e_R xi_s on the right-hand side; energy
conservation across a shock moving into gas at rest gives -e_R xi_s, which is
used.  The star pressure P_c is found by bisection so that both sides give the
same u_c.

Pinned by tests/test_riemann_oracle.py: the dilute limit against the textbook
ideal-gas (gamma = 5/3) solution, the Rankine-Hugoniot residuals, and the
constancy along the rarefaction of the Carnahan-Starling entropy
s = (3/2) ln T - ln rho - eta (4 - 3 eta) / (1 - eta)^2.
"""
from __future__ import annotations

import math

import numpy as np


def chi_set(eta):
    return 0.5 * (2.0 - eta) / (1.0 - eta) ** 3


def z_factor(eta):
    return 1.0 + 4.0 * eta * chi_set(eta)


class DenseGas:
    def __init__(self, eta0: float, rho_ref: float = 1.0):
        self.eta0, self.rho_ref = eta0, rho_ref

    def eta(self, rho):
        return self.eta0 * rho / self.rho_ref

    def pressure(self, rho, T):
        return rho * T * z_factor(self.eta(rho))

    def temperature(self, rho, P):
        return P / (rho * z_factor(self.eta(rho)))

    def sound_speed2(self, rho, P):
        """c_s^2(rho, P) = P/rho + 2P(1 + b rho chi)/(3 rho) + b P (chi + rho d_rho chi)/(1 + b rho chi),
        b rho = 4 eta, d chi / d eta = (5 - 2 eta) / (2 (1 - eta)^4) (Sec. IV.B)."""
        eta = self.eta(rho)
        chi = chi_set(eta)
        Y = 4.0 * eta * chi
        b = 4.0 * self.eta0 / self.rho_ref
        dchi_drho = (self.eta0 / self.rho_ref) * (5.0 - 2.0 * eta) / (2.0 * (1.0 - eta) ** 4)
        return P / rho + 2.0 * P * (1.0 + Y) / (3.0 * rho) + b * P * (chi + rho * dchi_drho) / (1.0 + Y)


def _rarefaction_table(gas: DenseGas, rhoL: float, PL: float, uL: float, rho_min: float, n: int = 4000):
    """RK4 in rho from rho_L down to rho_min of dP/drho = c_s^2 and du/drho = -c_s/rho; returns arrays
    (rho, P, u) ordered by decreasing rho."""
    rho = np.linspace(rhoL, rho_min, n + 1)
    P = np.empty(n + 1)
    u = np.empty(n + 1)
    P[0], u[0] = PL, uL

    def f(r, p):
        c2 = gas.sound_speed2(r, p)
        return c2, -math.sqrt(c2) / r

    for i in range(n):
        h = rho[i + 1] - rho[i]
        r, p, v = rho[i], P[i], u[i]
        k1p, k1u = f(r, p)
        k2p, k2u = f(r + h / 2, p + h / 2 * k1p)
        k3p, k3u = f(r + h / 2, p + h / 2 * k2p)
        k4p, k4u = f(r + h, p + h * k3p)
        P[i + 1] = p + h / 6 * (k1p + 2 * k2p + 2 * k3p + k4p)
        u[i + 1] = v + h / 6 * (k1u + 2 * k2u + 2 * k3u + k4u)
    return rho, P, u


def _shock_from_pc(gas: DenseGas, rhoR: float, PR: float, Pc: float):
    """Shock into gas at rest (rho_R, P_R) with post-shock pressure Pc > PR: (rho2, u_c, xi_s).
    Hugoniot: (3/2)(T2 - T_R) = (Pc + PR)/2 (1/rho_R - 1/rho2), with T2 = T(rho2, Pc); bisection in rho2."""
    TR = gas.temperature(rhoR, PR)

    def hug(r2):
        return 1.5 * (gas.temperature(r2, Pc) - TR) - 0.5 * (Pc + PR) * (1.0 / rhoR - 1.0 / r2)

    lo, hi = rhoR * (1 + 1e-12), 0.49 * gas.rho_ref / gas.eta0 if gas.eta0 > 0 else rhoR * 1e3
    hi = min(hi, rhoR * 1e3)
    flo, fhi = hug(lo), hug(hi)
    if flo * fhi > 0:
        raise ValueError("no shock density bracket")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        fm = hug(mid)
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
    rho2 = 0.5 * (lo + hi)
    xi_s = math.sqrt((Pc - PR) / (rhoR * (1.0 - rhoR / rho2)))
    u_c = xi_s * (1.0 - rhoR / rho2)
    return rho2, u_c, xi_s


class ShockTube:
    """Exact solution for left state (rho_L, T_L, u_L = 0) and right state (rho_R, T_R, u_R = 0)."""

    def __init__(self, gas: DenseGas, rhoL: float, TL: float, rhoR: float, TR: float):
        self.gas = gas
        self.rhoL, self.rhoR = rhoL, rhoR
        self.PL, self.PR = gas.pressure(rhoL, TL), gas.pressure(rhoR, TR)
        assert self.PL > self.PR
        self.rho_t, self.P_t, self.u_t = _rarefaction_table(gas, rhoL, self.PL, 0.0, rhoR * 0.2)

        def u_rar(Pc):
            # rarefaction state at pressure Pc (P decreases monotonically along the table)
            j = np.searchsorted(-self.P_t, -Pc)
            j = min(max(j, 1), len(self.P_t) - 1)
            t = (Pc - self.P_t[j - 1]) / (self.P_t[j] - self.P_t[j - 1])
            return (self.rho_t[j - 1] + t * (self.rho_t[j] - self.rho_t[j - 1]),
                    self.u_t[j - 1] + t * (self.u_t[j] - self.u_t[j - 1]))

        lo, hi = self.PR * (1 + 1e-9), self.PL * (1 - 1e-9)
        for _ in range(200):
            Pc = 0.5 * (lo + hi)
            _, ur = u_rar(Pc)
            _, us, _ = _shock_from_pc(gas, rhoR, self.PR, Pc)
            if ur > us:
                lo = Pc
            else:
                hi = Pc
        self.Pc = 0.5 * (lo + hi)
        self.rho1, self.uc = u_rar(self.Pc)
        self.rho2, _, self.xi_s = _shock_from_pc(gas, rhoR, self.PR, self.Pc)
        self.xi_head = -math.sqrt(gas.sound_speed2(rhoL, self.PL))
        self.xi_tail = self.uc - math.sqrt(gas.sound_speed2(self.rho1, self.Pc))
        # characteristic speed u - c_s along the table, for the fan interior
        self.lam_t = self.u_t - np.sqrt(gas.sound_speed2(self.rho_t, self.P_t))

    def sample(self, xi):
        """(rho, u, T) at similarity coordinate xi = (x - x0) / t (array)."""
        xi = np.asarray(xi, dtype=float)
        rho = np.empty_like(xi)
        u = np.empty_like(xi)
        P = np.empty_like(xi)
        g = self.gas
        for n_, x in np.ndenumerate(xi):
            if x <= self.xi_head:
                r, v, p = self.rhoL, 0.0, self.PL
            elif x < self.xi_tail:
                # lam_t = u - c_s increases from xi_head as rho decreases from rho_L
                j = np.searchsorted(self.lam_t, x)
                j = min(max(j, 1), len(self.lam_t) - 1)
                t = (x - self.lam_t[j - 1]) / (self.lam_t[j] - self.lam_t[j - 1])
                r = self.rho_t[j - 1] + t * (self.rho_t[j] - self.rho_t[j - 1])
                v = self.u_t[j - 1] + t * (self.u_t[j] - self.u_t[j - 1])
                p = self.P_t[j - 1] + t * (self.P_t[j] - self.P_t[j - 1])
            elif x < self.uc:
                r, v, p = self.rho1, self.uc, self.Pc
            elif x < self.xi_s:
                r, v, p = self.rho2, self.uc, self.Pc
            else:
                r, v, p = self.rhoR, 0.0, self.PR
            rho[n_], u[n_], P[n_] = r, v, p
        return rho, u, g.temperature(rho, P)


def ideal_gas_sod(rhoL, PL, rhoR, PR, gamma=5.0 / 3.0):
    """Textbook exact solution of the ideal-gas shock tube (both states at rest): star pressure from
    the shock/rarefaction velocity functions of Toro, Ch. 4; returns (P*, u*, rho1, rho2, shock speed)."""
    cL, cR = math.sqrt(gamma * PL / rhoL), math.sqrt(gamma * PR / rhoR)
    AR, BR = 2.0 / ((gamma + 1) * rhoR), (gamma - 1) / (gamma + 1) * PR

    def fL(P):
        return 2 * cL / (gamma - 1) * ((P / PL) ** ((gamma - 1) / (2 * gamma)) - 1)

    def fR(P):
        return (P - PR) * math.sqrt(AR / (P + BR))

    lo, hi = PR, PL
    for _ in range(200):
        P = 0.5 * (lo + hi)
        if fL(P) + fR(P) < 0:
            lo = P
        else:
            hi = P
    P = 0.5 * (lo + hi)
    u = 0.5 * (fR(P) - fL(P))
    rho1 = rhoL * (P / PL) ** (1 / gamma)
    g1 = (gamma - 1) / (gamma + 1)
    rho2 = rhoR * (P / PR + g1) / (g1 * P / PR + 1)
    S = cR * math.sqrt((gamma + 1) / (2 * gamma) * P / PR + (gamma - 1) / (2 * gamma))
    return P, u, rho1, rho2, S
