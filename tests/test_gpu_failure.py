"""Failure detection of the step kernel without a GPU fault: every shared-memory wait of the
step is bounded, and a wait that gives up records LBM_ERR_TIMEOUT in the context's device error
word.  lbm_inject_timeout makes the first wait of every warp give up at once (its row copy is
then waited for with the normal bound, so no bulk copy outlives its block); the test checks that
the error is reported, and that re-initialising the state clears it and the same context then
steps exactly like a fresh one."""
import numpy as np
import pytest

from paper_1909_04166_gb300 import lbm
from paper_1909_04166_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_timeout_is_reported_and_cleared_by_reinitialisation(precision):
    case = W.random_drop(96, 70, seed=21, wall_y=True, rho_ratio=100.0, gravity=1e-6)
    with lbm.Simulation(case, precision=precision) as a, \
            lbm.Simulation(case, precision=precision) as fresh:
        a.init_case().step(5)
        lbm.lbm_check(a.ctx)
        lbm.lbm_inject_timeout(a.ctx, True)
        a.step(3)
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_check(a.ctx)
        assert e.value.status == lbm.LBM_ERR_TIMEOUT
        with pytest.raises(lbm.LbmError) as e:      # every synchronising read reports it
            a.fields()
        assert e.value.status == lbm.LBM_ERR_TIMEOUT
        lbm.lbm_inject_timeout(a.ctx, False)
        a.init_case().step(37)                       # graph replays and a single launch
        lbm.lbm_check(a.ctx)
        fresh.init_case().step(37)
        ga, fa = a.populations()
        gb, fb = fresh.populations()
    assert np.array_equal(ga, gb) and np.array_equal(fa, fb)


def test_inject_timeout_rejects_bad_values():
    case = W.random_drop(40, 30, seed=2)
    with lbm.Simulation(case, precision="fp32") as s:
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_inject_timeout(s.ctx, 2)
        assert e.value.status == lbm.LBM_ERR_ARG
