"""The solver's buffer rotation: on the tiled path a step leaves psi^(n+1) in the buffer that held psi^(1) and
the two buffers swap roles, and several steps in one call replay one recorded step graph per buffer order.
Any sequence of calls must therefore give the state of the same number of single steps, bit for bit: single
steps against multi-step calls of odd and even length, interleaved with state reads and a state reload, on the
tiled path (FP32 and FP64, fixed and periodic ends, Q = 16 and 32) and on the generic large-Q path (FP64,
Q = 48, which keeps its state in place)."""
import numpy as np
import pytest

from paper_2211_16933_gb300 import inputs

pytestmark = pytest.mark.gpu


def _solver(q, Q, precision, periodic):
    nx = 700
    p, _ = q.ql_velocity_set(Q)
    dt = inputs.cfl_dt(1.0 / nx, float(np.abs(p).max()))
    if periodic:
        w = inputs.sound_wave(nx=nx, Q=Q)
        return q.Solver(Q, nx, w["length"], dt, w["denseness"], w["kn"], bc=q.QL_BC_PERIODIC,
                        init_kind=q.QL_INIT_SOUND, prm=w["prm"], precision=precision, pr_mode=q.QL_PR_CONST,
                        pr_const=w["pr_const"])
    w = inputs.sod_tube(nx=nx, Q=Q)
    return q.Solver(Q, nx, w["length"], dt, w["denseness"], w["kn"], bc=q.QL_BC_FIXED, init_kind=q.QL_INIT_RIEMANN,
                    prm=w["prm"], precision=precision, pr_mode=q.QL_PR_DENSE)


def _same(a, b):
    for x, y in zip(a.state(), b.state()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("Q,precision,periodic", [(32, 1, False), (32, 1, True), (16, 0, False), (32, 0, True),
                                                  (48, 0, False)])
def test_any_split_of_steps_gives_the_same_state(gpu, Q, precision, periodic):
    q = gpu
    a, b = _solver(q, Q, precision, periodic), _solver(q, Q, precision, periodic)
    for _ in range(5):
        a.step(1)
    b.step(5)  # odd: the buffers end swapped
    _same(a, b)
    a.step(1)
    a.step(1)
    b.step(2)  # even, from the swapped order: the other recorded step
    _same(a, b)
    b.step(3)
    for _ in range(3):
        a.step(1)
    _same(a, b)
    # a reloaded state goes to the buffer that holds the state now
    ph, th = a.state()
    b.set_state(ph, th)
    a.step(2)
    b.step(1)
    b.step(1)
    _same(a, b)
    assert a.step_count() == b.step_count() == 12
    a.close()
    b.close()
