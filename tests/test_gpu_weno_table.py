"""WENO-5 faces where indicators vanish (App. A.2, Table weno_x), through ql_rhs against the oracle.

The state is the equilibrium of piecewise-constant fields whose plateaus are 1 to 6 cells long, so that the
faces of every row meet one, two and three vanishing smoothness indicators (the rows of Table weno_x) next to
faces with none.  The state is rounded to FP32 first, so that both precisions and the oracle start from the
same numbers and a plateau is exactly flat.  The FP32 kernel evaluates the weights with reciprocals of the
rescaled indicators (each raised by 2^-50), FP64 in the product form; both must give the right-hand side the
oracle gives with the table: FP64 to 1e-11 and FP32 to 2e-5 of the largest |L| (the tolerances of the other
right-hand-side tests).  N_x = 600 (several tiles, a ragged tail), periodic, Q = 16 and 32."""
import numpy as np
import pytest

import oracle as O
from paper_2211_16933_gb300 import inputs
from rhs_terms import rhs_terms

pytestmark = pytest.mark.gpu

NX, EL, KN = 600, 0.2, 0.05


def _plateau_fields(seed):
    rng = np.random.default_rng(seed)
    r, u, T = np.empty(NX), np.empty(NX), np.empty(NX)
    i = 0
    while i < NX:
        n = int(rng.integers(1, 7))
        r[i:i + n] = rng.uniform(0.8, 1.2)
        u[i:i + n] = rng.uniform(-0.2, 0.2)
        T[i:i + n] = rng.uniform(0.85, 1.15)
        i += n
    return r, u, T


def _zero_patterns(f):
    """Per face of a periodic row, how many of the three upwind stencils (positive velocity) are flat."""
    counts = np.zeros(4, dtype=int)
    for i in range(NX):
        s = [f[(i - 2 + r) % NX] for r in range(5)]
        z = int(s[0] == s[1] == s[2]) + int(s[1] == s[2] == s[3]) + int(s[2] == s[3] == s[4])
        counts[z] += 1
    return counts


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("Q", [16, 32])
def test_rhs_on_plateaus_matches_the_table(gpu, Q, precision):
    q = gpu
    p, _ = O.quadrature(Q)
    dt = inputs.cfl_dt(1.0 / NX, float(np.abs(p).max()))
    m = O.make_model(Q, NX, 1.0, dt, EL, KN, bc=O.BC_PERIODIC)
    r, u, T = _plateau_fields(seed=100 + Q)
    ph, th = O.equilibrium_state(m, r, u, T)
    ph = ph.astype(np.float32).astype(np.float64)
    th = th.astype(np.float32).astype(np.float64)
    # every row of Table weno_x occurs
    c = _zero_patterns(ph[:, Q // 2])
    assert c[0] > 0 and c[1] > 0 and c[2] > 0 and c[3] > 0, c
    s = q.Solver(Q, NX, 1.0, dt, EL, KN, bc=q.QL_BC_PERIODIC, init_kind=q.QL_INIT_FIELDS, rho=r, u=u, T=T,
                 precision=precision, pr_mode=q.QL_PR_DENSE)
    s.set_state(ph, th)
    L = s.rhs()
    relax, j1, adv = rhs_terms(m, ph, th)
    tol = 1e-11 if precision == 0 else 2e-5
    for k in range(2):
        ref = relax[k] + j1[k] - adv[k]  # L = relaxation + J1 - advection (Eq. cast)
        scale = np.abs(ref).max()
        assert np.abs(adv[k]).max() > 0.1 * scale
        assert np.abs(L[k] - ref).max() <= tol * scale
    s.close()
