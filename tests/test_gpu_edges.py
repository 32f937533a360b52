"""Edge cases of the CUDA path against the oracle: domains smaller than a tile and than the ghost width times
two, sizes at and around the 248-cell tile boundary, the pure Shakhov model (J1 off), zero-step calls, and a
batch of one instance of the smallest size."""
import numpy as np
import pytest

import oracle as O
from paper_2211_16933_gb300 import inputs

pytestmark = pytest.mark.gpu


def _run_pair(q, Q, nx, bc, precision, steps, enskog=1, seed=3):
    L = 1.0
    p, _ = O.quadrature(Q)
    dt = inputs.cfl_dt(L / nx, abs(p).max())
    bco = O.BC_PERIODIC if bc == "periodic" else O.BC_FIXED
    m = O.make_model(Q, nx, L, dt, 1.1, 0.02, pr_mode=1, bc=bco, enskog=enskog)
    f = inputs.smooth_periodic_fields(nx, seed=seed)
    kw = dict(rho=f[0], u=f[1], T=f[2])
    if bc == "fixed":
        ghost = [(f[0][0], f[1][0], f[2][0])] * 3 + [(f[0][-1], f[1][-1], f[2][-1])] * 3
        O.set_ghosts(m, ghost[:3], ghost[3:])
        kw["ghost"] = np.asarray(ghost, dtype=float).ravel()
    ph, th = O.equilibrium_state(m, *f)
    s = q.Solver(Q, nx, L, dt, 1.1, 0.02, bc=q.QL_BC_PERIODIC if bc == "periodic" else q.QL_BC_FIXED,
                 init_kind=q.QL_INIT_FIELDS, prm=(), precision=precision, pr_mode=q.QL_PR_DENSE, enskog=enskog, **kw)
    ph, th = O.run(m, ph, th, steps)
    s.step(steps)
    f_or, f_gp = O.fields(m, ph, th), s.moments()
    s.close()
    return max(float(np.abs(f_gp[k] - f_or[k]).max()) for k in ("rho", "u", "T", "q"))


@pytest.mark.parametrize("nx", [8, 9, 13, 247, 248, 249, 496, 497])
@pytest.mark.parametrize("bc", ["periodic", "fixed"])
def test_sizes_around_the_tile_and_ghost_widths(gpu, nx, bc):
    assert _run_pair(gpu, 16, nx, bc, 0, 4) <= 1e-10


@pytest.mark.parametrize("precision", [0, 1])
def test_pure_shakhov_model_without_j1(gpu, precision):
    assert _run_pair(gpu, 32, 3 * 248 + 5, "periodic", precision, 5, enskog=0) <= (1e-10 if precision == 0 else 1e-5)


def test_zero_steps_change_nothing(gpu):
    q = gpu
    s = q.Solver(16, 64, 1.0, 1e-3, 0.1, 0.1, bc=q.QL_BC_PERIODIC, init_kind=q.QL_INIT_SOUND, prm=(1.0, 1.0, 1e-3),
                 precision=q.QL_FP64)
    a = s.state()
    s.step(0)
    b = s.state()
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_of_one_smallest_instance_matches_the_single_solver(gpu, precision):
    q = gpu
    keep = []
    p, _ = q.ql_velocity_set(16)
    dt = inputs.cfl_dt(1.0 / 8, float(np.abs(p).max()))
    I = q.make_instance(16, 8, 1.0, dt, 0.1, 0.1, bc=q.QL_BC_PERIODIC, init_kind=q.QL_INIT_SOUND,
                        prm=(1.0, 1.0, 1e-3), keep=keep)
    b = q.Batch([I], precision=precision)
    b.run(0)
    b.run(7)
    b.sync()
    a = b.state(0)
    b.close()
    s = q.Solver(16, 8, 1.0, dt, 0.1, 0.1, bc=q.QL_BC_PERIODIC, init_kind=q.QL_INIT_SOUND, prm=(1.0, 1.0, 1e-3),
                 precision=precision, pr_mode=q.QL_PR_DENSE)
    s.step(7)
    r = s.state()
    s.close()
    np.testing.assert_array_equal(a[0], r[0])
    np.testing.assert_array_equal(a[1], r[1])
