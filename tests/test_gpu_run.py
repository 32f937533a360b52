"""Whole runs of steps as one launch (ql_opts.launch = QL_LAUNCH_RUN; QL_LAUNCH_AUTO, the default, picks it for
FP32 chi_SET solvers of the tiled velocity sets on domains of one to eight times as many tiles as the GPU holds
CTAs): each (stage, tile) work item starts once the previous stage of its tile and of the tiles it reads has
completed.  The state must be bit for bit that of one launch per Runge-Kutta stage (QL_LAUNCH_STAGES), for any
split of the steps into calls: fixed and periodic ends, one to several hundred tiles (more than the GPU holds at
once), ragged last tiles, a periodic domain whose last tile holds fewer cells than the halo (tiles 0 and N - 2
then exchange ghost images), both per-cell sum modes, and runs much longer than the domain is wide in tiles
(most work items then wait for their neighbours)."""
import numpy as np
import pytest

from paper_2211_16933_gb300 import inputs

pytestmark = pytest.mark.gpu


def _solver(q, Q, nx, periodic, launch, sums=0):
    p, _ = q.ql_velocity_set(Q)
    dt = inputs.cfl_dt(1.0 / nx, float(np.abs(p).max()))
    if periodic:
        w = inputs.sound_wave(nx=nx, Q=Q)
        return q.Solver(Q, nx, w["length"], dt, w["denseness"], w["kn"], bc=q.QL_BC_PERIODIC,
                        init_kind=q.QL_INIT_SOUND, prm=(1.0, 1.0, 0.05), precision=q.QL_FP32,
                        pr_mode=q.QL_PR_CONST, pr_const=w["pr_const"], launch=launch, sums=sums)
    w = inputs.sod_tube(nx=nx, Q=Q)
    return q.Solver(Q, nx, w["length"], dt, w["denseness"], w["kn"], bc=q.QL_BC_FIXED, init_kind=q.QL_INIT_RIEMANN,
                    prm=w["prm"], precision=q.QL_FP32, pr_mode=q.QL_PR_DENSE, launch=launch, sums=sums)


def _same(a, b):
    for x, y in zip(a.state(), b.state()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("Q,nx,periodic,sums", [
    (32, 700, False, 0),            # 3 tiles, ragged last tile
    (32, 3 * 248 + 2, True, 0),     # last tile of 2 cells: tiles 0 and N - 2 share ghost images
    (16, 248, True, 0),             # one tile, its own neighbour on both sides
    (8, 2 * 248, True, 0),          # two tiles
    (24, 4096, False, 1),           # FP64 per-cell sums
    (40, 5000, True, 0),            # two CTAs per SM
    (20, 2 * 248 + 3, False, 0),    # fixed ends, last tile shorter than the halo
])
def test_run_launch_matches_stage_launches(gpu, Q, nx, periodic, sums):
    q = gpu
    a = _solver(q, Q, nx, periodic, q.QL_LAUNCH_STAGES, sums)
    b = _solver(q, Q, nx, periodic, q.QL_LAUNCH_RUN, sums)
    for _ in range(7):
        a.step(1)
    b.step(7)  # odd: the buffers end swapped
    _same(a, b)
    a.step(4)
    for _ in range(4):
        b.step(1)
    _same(a, b)
    a.step(40)
    b.step(40)  # 120 stages of a domain a few tiles wide: most work items wait for their neighbours
    _same(a, b)
    a.sync()
    b.sync()  # the error word is clean: no wait gave up
    assert a.step_count() == b.step_count() == 51
    a.close()
    b.close()


def test_run_launch_wider_than_the_gpu(gpu):
    """1058 tiles per stage, more than the GPU holds at once, 12 steps in one call and in single calls."""
    q = gpu
    nx = 1 << 18
    a = _solver(q, 32, nx, False, q.QL_LAUNCH_STAGES)
    b = _solver(q, 32, nx, False, q.QL_LAUNCH_RUN)
    c = _solver(q, 32, nx, False, q.QL_LAUNCH_RUN)
    a.step(12)
    b.step(12)
    for _ in range(12):
        c.step(1)
    _same(a, b)
    _same(a, c)
    b.sync()
    c.sync()
    for s in (a, b, c):
        s.close()


def test_auto_launch_picks_by_domain_size(gpu):
    """QL_LAUNCH_AUTO: the whole-run launch for 2^17 cells (529 tiles, 1.2 times the 456 CTAs the GPU holds),
    per-stage launches for 8192 cells (fewer tiles than CTA slots) and for 2^22 cells (37 waves); the same
    state either way."""
    q = gpu
    nx = 1 << 17
    a = _solver(q, 32, nx, False, q.QL_LAUNCH_STAGES)
    b = _solver(q, 32, nx, False, q.QL_LAUNCH_AUTO)
    assert a.steps_per_launch() == 0 and b.steps_per_launch() > 0
    a.step(5)
    b.step(5)
    _same(a, b)
    b.sync()
    a.close()
    b.close()
    for n in (8192, 1 << 22):
        s = _solver(q, 32, n, False, q.QL_LAUNCH_AUTO)
        assert s.steps_per_launch() == 0, n
        s.close()
