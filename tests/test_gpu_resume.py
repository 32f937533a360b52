"""Checkpoint and resume through the C ABI: a run stopped after N steps, its state read back (ql_get_state),
loaded into a new solver of the same parameters (ql_set_state) and continued for M steps gives bitwise the state
of an uninterrupted run of N + M steps, in both precisions and with both boundary kinds.  The state is the whole
restart record: the scheme has no time-dependent forcing, and the fixed ghosts come from the parameters."""
import numpy as np
import pytest

from paper_2211_16933_gb300 import inputs

pytestmark = pytest.mark.gpu


def _make(q, w, precision):
    p, _ = q.ql_velocity_set(w["Q"])
    dt = inputs.cfl_dt(w["length"] / w["nx"], float(np.abs(p).max()))
    bc = q.QL_BC_PERIODIC if w["bc"] == "periodic" else q.QL_BC_FIXED
    kind = {"sound": q.QL_INIT_SOUND, "riemann": q.QL_INIT_RIEMANN, "shock": q.QL_INIT_SHOCK}[w["init"]]
    pr = q.QL_PR_DENSE if w["pr_mode"] == "dense" else q.QL_PR_CONST
    return q.Solver(w["Q"], w["nx"], w["length"], dt, w["denseness"], w["kn"], bc=bc, init_kind=kind, prm=w["prm"],
                    precision=precision, pr_mode=pr, pr_const=w["pr_const"])


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("case", ["sod", "sound"])
def test_resume_is_bitwise(gpu, precision, case):
    q = gpu
    if case == "sod":
        w = inputs.sod_tube(nx=3001, Q=32)
    else:
        w = dict(inputs.sound_wave())
    N, M = 7, 5
    a = _make(q, w, precision)
    a.step(N + M)
    b = _make(q, w, precision)
    b.step(N)
    phi, theta = b.state()
    c = _make(q, w, precision)
    c.step(3)  # any other state: it is overwritten
    c.set_state(phi, theta)
    c.step(M)
    pa, ta = a.state()
    pc, tc = c.state()
    np.testing.assert_array_equal(pc, pa)
    np.testing.assert_array_equal(tc, ta)
    ma, mc = a.moments(), c.moments()
    for f in ("rho", "u", "T", "P", "q", "Pxx"):
        np.testing.assert_array_equal(mc[f], ma[f])


@pytest.mark.parametrize("precision,Q,chi", [(0, 16, 0), (1, 32, 0), (1, 16, 1), (0, 48, 1)])
def test_replayed_steps_equal_single_steps(gpu, precision, Q, chi):
    """ql_step of several steps replays one recorded step: bitwise the state of as many single-step calls,
    on the tiled kernels (FP64, FP32, chi_RET-FM) and the generic large-Q path (chi_RET-FM), fixed ends."""
    q = gpu
    nx, L, El = 611, 1.0, 0.4825
    p, _ = q.ql_velocity_set(Q)
    dt = inputs.cfl_dt(L / nx, float(np.abs(p).max()))
    kn = 3.7 / (nx * El)  # the chi_RET-FM ball reaches 4 cells

    def make():
        return q.Solver(Q, nx, L, dt, El, kn, bc=q.QL_BC_FIXED, init_kind=q.QL_INIT_RIEMANN,
                        prm=(1.0, 0.0, 1.0, 0.125, 0.0, 1.0), precision=precision, chi_mode=chi)
    a, b = make(), make()
    a.step(7)
    for _ in range(7):
        b.step(1)
    pa, ta = a.state()
    pb, tb = b.state()
    np.testing.assert_array_equal(pa, pb)
    np.testing.assert_array_equal(ta, tb)
    a.step(2)  # the recorded step is reused
    b.step(1)
    b.step(1)
    np.testing.assert_array_equal(a.state()[0], b.state()[0])


@pytest.mark.parametrize("precision,Q,chi,bc", [(0, 32, 0, "fixed"), (1, 16, 1, "fixed"), (0, 48, 1, "periodic")])
def test_resume_from_restart_file_is_bitwise(gpu, tmp_path, precision, Q, chi, bc):
    """ql_save after N steps, ql_load into a new context, M more steps: bitwise the state and moments of an
    uninterrupted N + M step run, with the step count carried over; tiled FP64 and FP32 (chi_RET-FM) with
    fixed ends and the generic path (chi_RET-FM) with periodic ones, a constant Prandtl number."""
    q = gpu
    nx, L, El = 611, 1.0, 0.4825
    p, _ = q.ql_velocity_set(Q)
    dt = inputs.cfl_dt(L / nx, float(np.abs(p).max()))
    kn = 3.7 / (nx * El)
    if bc == "fixed":
        kw = dict(bc=q.QL_BC_FIXED, init_kind=q.QL_INIT_RIEMANN, prm=(1.0, 0.0, 1.0, 0.125, 0.0, 1.0))
    else:
        kw = dict(bc=q.QL_BC_PERIODIC, init_kind=q.QL_INIT_SOUND, prm=(1.0, 1.0, 1e-2))

    def make():
        return q.Solver(Q, nx, L, dt, El, kn, precision=precision, chi_mode=chi, pr_mode=q.QL_PR_CONST,
                        pr_const=0.7, **kw)
    N, M = 6, 5
    a = make()
    a.step(N + M)
    b = make()
    b.step(N)
    path = tmp_path / "run.qlbm"
    b.save(path)
    info = q.ql_checkpoint_read_info(path)
    assert (info.Q, info.nx, info.steps, info.precision, info.chi_mode) == (Q, nx, N, precision, chi)
    c = q.Solver.load(path)
    assert c.step_count() == N
    assert (c.dt, c.sigma, c.eta0) == (a.dt, a.sigma, a.eta0)
    c.step(M)
    assert c.step_count() == a.step_count() == N + M
    pa, ta = a.state()
    pc, tc = c.state()
    np.testing.assert_array_equal(pc, pa)
    np.testing.assert_array_equal(tc, ta)
    ma, mc = a.moments(), c.moments()
    for f in ("rho", "u", "T", "P", "q", "Pxx"):
        np.testing.assert_array_equal(mc[f], ma[f])
