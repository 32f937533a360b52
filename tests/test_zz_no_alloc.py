"""ql_step_noalloc: stepping a caller-owned state with no device allocation.

Some callers cannot call cudaMalloc (a memory budget reserved by another
framework, or a latency-critical loop where an allocation could synchronise the
device).  This entry point keeps its two stage buffers in a fixed scratch array
of the library.  It launches the same stage kernels as ql_step on the same state
layout with the same launch shape, so its results must equal those of ql_step
bit for bit, on two calls in a row (the scratch keeps the previous call's
contents), and a call must leave the device's free memory unchanged.
"""
import numpy as np
import pytest

from paper_2211_16933_gb300 import inputs

pytestmark = pytest.mark.gpu


def _case(q, precision, kind):
    if kind == "sound":
        w = inputs.sound_wave(nx=300, Q=16)
        bc, init = q.QL_BC_PERIODIC, q.QL_INIT_SOUND
    else:
        w = inputs.normal_shock(1.4, 0.1, nx=520, Q=32)
        bc, init = q.QL_BC_FIXED, q.QL_INIT_SHOCK
    p, _ = q.ql_velocity_set(w["Q"])
    dt = inputs.cfl_dt(w["length"] / w["nx"], abs(p).max())
    pr = q.QL_PR_CONST if w["pr_mode"] == "const" else q.QL_PR_DENSE
    mk = lambda: q.Solver(w["Q"], w["nx"], w["length"], dt, w["denseness"], w["kn"], bc=bc, init_kind=init,
                          prm=w["prm"], precision=precision, pr_mode=pr, pr_const=w["pr_const"])
    return w, dt, bc, pr, mk


def _opts(q, w, precision, pr):
    import torch
    o = q.ql_opts()
    o.precision, o.pr_mode, o.enskog, o.device = precision, pr, 1, 0
    o.pr_const, o.rho_ref = w["pr_const"], 1.0
    o.stream = torch.cuda.current_stream().cuda_stream
    return o


@pytest.mark.parametrize("precision,kind", [(0, "sound"), (1, "sound"), (0, "shock"), (1, "shock")])
def test_noalloc_matches_ql_step_on_two_calls(gpu, precision, kind):
    q = gpu
    w, dt, bc, pr, mk = _case(q, precision, kind)
    ref, own = mk(), mk()
    psi, stride = q.ql_state_device(own.ctx)
    vs, grid, b = q.ql_velset(w["Q"], 0), q.ql_grid(w["nx"], w["length"], dt), q.ql_bc(bc, 0)
    o = _opts(q, w, precision, pr)
    for _ in range(2):
        q.ql_step_noalloc(vs, grid, w["denseness"], w["kn"], b, o, psi, stride, 3)
        ref.step(3)
        a, c = own.state(), ref.state()
        for x, y in zip(a, c):
            assert np.array_equal(x, y)
    ref.close()
    own.close()


def test_noalloc_call_leaves_device_memory_unchanged(gpu):
    """After a first call (which may load kernels and looks up the scratch address), a further call takes no
    device memory: the free memory the driver reports is the same before and after it."""
    import torch
    q = gpu
    w, dt, bc, pr, mk = _case(q, 1, "shock")
    own = mk()
    psi, stride = q.ql_state_device(own.ctx)
    vs, grid, b = q.ql_velset(w["Q"], 0), q.ql_grid(w["nx"], w["length"], dt), q.ql_bc(bc, 0)
    o = _opts(q, w, 1, pr)
    q.ql_step_noalloc(vs, grid, w["denseness"], w["kn"], b, o, psi, stride, 2)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    q.ql_step_noalloc(vs, grid, w["denseness"], w["kn"], b, o, psi, stride, 2)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    own.close()


def test_noalloc_rejects_states_beyond_the_scratch(gpu):
    q = gpu
    nx = 1 << 20  # FP64, Q = 32: two stage buffers of about 0.5 GiB each
    vs, grid, b = q.ql_velset(32, 0), q.ql_grid(nx, 1.0, 1e-8), q.ql_bc(q.QL_BC_FIXED, 0)
    o = q.ql_opts()
    o.precision, o.pr_mode, o.enskog, o.rho_ref = 0, q.QL_PR_DENSE, 1, 1.0
    with pytest.raises(q.QLError) as e:
        q.ql_step_noalloc(vs, grid, 0.1, 0.05, b, o, 1 << 12, nx + 512, 1)
    assert e.value.status == q.QL_EINVAL
    assert "scratch" in str(e.value)
