"""Sound-wave dispersion study (Sec. IV.A): a sweep of the reduced density,
the amplitude of the density mode followed in time, and a Levenberg-Marquardt
fit of the sound speed and the two damping rates, against the linear-theory
values of ql_sound_modes.

All instances run together as one batch (every step in the library's
kernels); ql_batch_project writes the density-mode amplitude of every instance
into a device array at each sample time.  Only the fit runs on the host.
"""
from __future__ import annotations

import math

import numpy as np

from . import inputs
from . import qlbm as q


def sweep_specs(denseness_values, nx=128, Q=16, kn=0.005, amp=1e-3, length=1.0):
    """One periodic sound wave per E_l: rho = 1 + amp cos(2 pi x / L), u = 0, T = 1 (an isothermal
    perturbation, the initial state for which Eq. sw_solution holds); dense Prandtl number; Kn small
    enough for hydrodynamic damping (k l ~ 2 pi Kn)."""
    return [dict(denseness=float(El), nx=nx, Q=Q, kn=kn, amp=amp, length=length) for El in denseness_values]


def run(specs, t_end, samples, precision=q.QL_FP64):
    """Runs every spec to t_end and records the density-mode amplitude at `samples` + 1 equally spaced
    times (the same time step for all, set by the fastest velocity set).  Returns (times, amplitudes[S+1][n],
    updates)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    pmax = max(float(np.abs(q.ql_velocity_set(s["Q"])[0]).max()) for s in specs)
    dx = min(s["length"] / s["nx"] for s in specs)
    dt0 = inputs.cfl_dt(dx, pmax)
    per = max(1, int(math.ceil(t_end / samples / dt0)))
    dt = t_end / samples / per
    keep, insts = [], []
    for s in specs:
        x = (np.arange(s["nx"]) + 0.5) * s["length"] / s["nx"]
        rho = 1.0 + s["amp"] * np.cos(2.0 * math.pi * x / s["length"])
        insts.append(q.make_instance(s["Q"], s["nx"], s["length"], dt, s["denseness"], s["kn"], bc=q.QL_BC_PERIODIC,
                                     init_kind=q.QL_INIT_FIELDS, rho=rho, u=np.zeros(s["nx"]), T=np.ones(s["nx"]),
                                     keep=keep))
    b = q.Batch(insts, precision=precision)
    out = torch.zeros(samples + 1, len(specs), dtype=torch.float64, device=dev)
    b._stream.wait_stream(torch.cuda.current_stream())
    b.project(1, out[0])
    for j in range(1, samples + 1):
        b.run(per)
        b.project(1, out[j])
    b.sync()
    amps = out.cpu().numpy()
    updates = sum(s["nx"] * s["Q"] for s in specs) * per * samples
    b.close()
    return np.arange(samples + 1) * per * dt, amps, updates


def model(t, d0, gamma, k, cs, aa, at):
    """Eq. (sw_solution), the density mode of an isothermal start (delta T = 0, u = 0: the initial state whose
    acoustic share is 1/gamma): d0 [(1 - 1/gamma) exp(-alpha_t t) + (1/gamma) exp(-alpha_a t) cos(k c_s t)]."""
    return d0 * ((1.0 - 1.0 / gamma) * np.exp(-at * t) + np.exp(-aa * t) * np.cos(k * cs * t) / gamma)


def fit(t, y, gamma, k, guess):
    """Levenberg-Marquardt fit of (c_s, alpha_a, alpha_t) with d0 = y(0) and gamma fixed."""
    from scipy.optimize import least_squares
    d0 = y[0]

    def res(p):
        return (model(t, d0, gamma, k, *p) - y) / abs(d0)

    r = least_squares(res, np.asarray(guess, dtype=float), method="lm", xtol=1e-14, ftol=1e-14, gtol=1e-14)
    return r.x, float(np.sqrt(np.mean(r.fun ** 2)))


def study(denseness_values, t_end=5.0, samples=500, **kw):
    """Runs the sweep and fits every instance; returns a list of dicts with the fitted and the linear-theory
    values (alpha_a with and without bulk viscosity)."""
    specs = sweep_specs(denseness_values, **kw)
    t, amps, updates = run(specs, t_end, samples)
    rows = []
    for i, s in enumerate(specs):
        k = 2.0 * math.pi / s["length"]
        cs, aa, aa0, at, gamma = q.ql_sound_modes(s["denseness"], s["kn"], s["length"], 1.0, 1.0, k)
        (fcs, faa, fat), rms = fit(t, amps[:, i], gamma, k, (cs, aa0, at))
        rows.append(dict(denseness=s["denseness"], eta0=q.ql_eta_of_denseness(s["denseness"]), gamma=gamma,
                         cs=cs, alpha_a=aa, alpha_a_no_bulk=aa0, alpha_t=at,
                         fit_cs=float(fcs), fit_alpha_a=float(faa), fit_alpha_t=float(fat), fit_rms=rms))
    return rows, updates
