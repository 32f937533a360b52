"""Failure detection without a GPU fault: the tile-staging wait of the stage kernel is bounded.  With
ql_opts.fault = 1 the kernel arms its barrier for copies it never issues (nothing is in flight, nothing can fault),
every CTA's wait runs out, the kernel sets its error bit and returns, and the next synchronising call reports
QL_ECUDA.  The context stays usable: a normal solver in the same process runs on and matches a fresh one."""
import time

import numpy as np
import pytest

from paper_2211_16933_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 1])
def test_stalled_staging_wait_gives_up_and_reports(gpu, precision):
    q = gpu
    w = inputs.sound_wave(nx=200, Q=16)  # one tile: one CTA waits
    p, _ = q.ql_velocity_set(16)
    dt = inputs.cfl_dt(w["length"] / w["nx"], float(np.abs(p).max()))
    kw = dict(bc=q.QL_BC_PERIODIC, init_kind=q.QL_INIT_SOUND, prm=w["prm"], precision=precision,
              pr_mode=q.QL_PR_CONST, pr_const=w["pr_const"])
    ref = q.Solver(16, w["nx"], w["length"], dt, w["denseness"], w["kn"], **kw)
    m0 = ref.moments()
    s = q.Solver(16, w["nx"], w["length"], dt, w["denseness"], w["kn"], fault=1, **kw)
    t0 = time.perf_counter()
    s.step(1)
    with pytest.raises(q.QLError) as e:
        s.totals()
    elapsed = time.perf_counter() - t0
    assert e.value.status == q.QL_ECUDA and "gave up" in str(e.value)
    assert elapsed < 20.0, elapsed  # six bounded waits (two per stage kernel) of about 0.25 s
    s.close() if hasattr(s, "close") else None
    # the GPU context is intact: a normal solver steps and agrees with a fresh one
    ref.step(4)
    again = q.Solver(16, w["nx"], w["length"], dt, w["denseness"], w["kn"], **kw)
    np.testing.assert_array_equal(again.moments()["rho"], m0["rho"])
    again.step(4)
    np.testing.assert_array_equal(again.moments()["rho"], ref.moments()["rho"])
