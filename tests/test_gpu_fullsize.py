"""Parity at the benchmark's full size: Sod tube, Nx = 2^22, Q = 32, FP32 and FP64,
in the launch configuration the benchmark times.

The oracle cannot run 2^22 cells, so sampled cells are checked one by one: after
s steps a cell depends only on cells within 9 s of it (3 per Runge-Kutta stage),
so the oracle runs a window of the same grid around each sampled cell, with
fixed ghost cells holding the initial state at the window's edges.
"""
import numpy as np
import pytest

import oracle as O
from paper_2211_16933_gb300 import inputs

pytestmark = pytest.mark.gpu
STEPS = 2
HALF = 9 * STEPS + 6


def _window_oracle(w, dt, c, steps):
    """Oracle fields and psi at global cell c after `steps` steps, from a window run."""
    nx, L, Q = w["nx"], w["length"], w["Q"]
    dx = L / nx
    a, b = max(0, c - HALF), min(nx, c + HALF + 1)
    nw = b - a
    gm = O.make_model(Q, nx, L, dt, w["denseness"], w["kn"], pr_mode=1, bc=O.BC_FIXED)
    r, u, T = O.init_fields(gm, O.INIT_RIEMANN, w["prm"], a, nw)
    gl = O.init_fields(gm, O.INIT_RIEMANN, w["prm"], a - 3, 3)
    gr = O.init_fields(gm, O.INIT_RIEMANN, w["prm"], b, 3)
    # same dx, same mean free path l0 = Kn L, same denseness
    m = O.make_model(Q, nw, nw * dx, dt, w["denseness"], w["kn"] * L / (nw * dx), pr_mode=1, bc=O.BC_FIXED)
    O.set_ghosts(m, np.stack(gl, 1), np.stack(gr, 1))
    ph, th = O.equilibrium_state(m, r, u, T)
    ph, th = O.run(m, ph, th, steps)
    f = O.fields(m, ph, th)
    j = c - a
    return {k: v[j] for k, v in f.items()}, ph[j], th[j]


@pytest.mark.parametrize("precision", [1, 0])
def test_sod_full_size_sampled(gpu, precision):
    w = inputs.sod_tube()
    nx, Q = w["nx"], w["Q"]
    p, _ = O.quadrature(Q)
    dt = inputs.cfl_dt(w["length"] / nx, abs(p).max())
    s = gpu.Solver(Q, nx, w["length"], dt, w["denseness"], w["kn"], bc=gpu.QL_BC_FIXED,
                   init_kind=gpu.QL_INIT_RIEMANN, prm=w["prm"], precision=precision, pr_mode=gpu.QL_PR_DENSE)
    s.step(STEPS)
    f = s.moments()
    gphi, gth = s.state()
    rng = np.random.default_rng(5)
    cells = [0, 1, 2, 3, 7, nx // 2 - 4, nx // 2 - 1, nx // 2, nx // 2 + 1, nx // 2 + 3, nx - 4, nx - 1]
    cells += [int(v) for v in rng.integers(0, nx, 4)]
    tol = 1e-10 if precision == 0 else 1e-5
    tol_psi = 1e-10 if precision == 0 else 2e-5
    Y0 = 4 * O.eta_from_denseness(w["denseness"]) * O.chi_set(O.eta_from_denseness(w["denseness"]))
    for c in cells:
        fo, po, to = _window_oracle(w, dt, c, STEPS)
        for k, sc in (("rho", 1.0), ("u", 1.0), ("T", 1.0), ("P", 1 + Y0), ("q", 1.0)):
            assert abs(f[k][c] - fo[k]) / sc <= tol, (c, k, f[k][c], fo[k])
        for a, b in ((gphi[c], po), (gth[c], to)):
            assert float(np.abs(a - b).max() / np.abs(b).max()) <= tol_psi, c
    # the membrane has started to move: the sampled cells see a non-trivial state
    assert abs(f["u"][nx // 2]) > 1e-6
    s.close()
