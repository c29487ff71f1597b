"""Failure detection of the step kernel without a GPU fault: every shared-memory wait of the
step is bounded, and a wait that gives up records LBM_ERR_TIMEOUT in the context's device error
word.  lbm_inject_timeout makes the first wait of every warp give up at once (its row copy is
then waited for with the normal bound, so no bulk copy outlives its block); the test checks that
the error is reported, and that re-initialising the state clears it and the same context then
steps exactly like a fresh one.  The multi-step kernel's waits for its neighbouring warps are
bounded the same way and tested with their own hook."""
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


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_neighbour_wait_timeout_is_reported_and_cleared(precision):
    """The multi-step kernel's waits for neighbouring warps between steps are bounded: with the
    hook that makes them unreachable, a run reports LBM_ERR_TIMEOUT (after the first step every
    warp waits out its bound and returns, no copy in flight); re-initialising clears it and the
    context then steps like a fresh one."""
    case = W.random_drop(130, 90, seed=23, wall_x=True, rho_ratio=100.0, gravity=1e-6)
    with lbm.Simulation(case, precision=precision) as a, \
            lbm.Simulation(case, precision=precision) as fresh:
        lbm.lbm_set_persistent(a.ctx, True)
        lbm.lbm_set_persistent(fresh.ctx, True)
        a.init_case().step(4)
        assert lbm.lbm_get_step_path(a.ctx) == lbm.LBM_PATH_MULTI
        lbm.lbm_inject_timeout(a.ctx, 2)
        assert lbm.lbm_get_step_path(a.ctx) == lbm.LBM_PATH_MULTI
        a.step(5)
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_check(a.ctx)
        assert e.value.status == lbm.LBM_ERR_TIMEOUT
        lbm.lbm_inject_timeout(a.ctx, 0)
        a.init_case().step(23)
        lbm.lbm_check(a.ctx)
        fresh.init_case().step(23)
        ga, fa = a.populations()
        gb, fb = fresh.populations()
    assert np.array_equal(ga, gb) and np.array_equal(fa, fb)


def test_inject_timeout_rejects_bad_values():
    case = W.random_drop(40, 30, seed=2)
    with lbm.Simulation(case, precision="fp32") as s:
        for bad in (3, -1):
            with pytest.raises(lbm.LbmError) as e:
                lbm.lbm_inject_timeout(s.ctx, bad)
            assert e.value.status == lbm.LBM_ERR_ARG
