"""The bounds-checked step kernel (lbm_set_checked), standing in for a device memory checker:
on ragged and tiny grids with every kind of side, in every storage precision, the checked
kernel finds no global load, store or bulk copy outside the state buffers, and its results are
bitwise those of the plain kernel."""
import numpy as np
import pytest

from paper_1909_04166_gb300 import lbm
from paper_1909_04166_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# (nx, ny, (left, right), (bottom, top)) with 0 periodic, 1 no-slip, 2 free-slip
SHAPES = [
    (1, 1, (0, 0), (0, 0)),
    (1, 9, (2, 2), (1, 2)),
    (5, 1, (1, 1), (0, 0)),
    (2, 3, (1, 2), (2, 1)),
    (31, 7, (0, 0), (1, 1)),
    (33, 17, (2, 1), (0, 0)),
    (63, 5, (1, 1), (2, 2)),
    (64, 40, (0, 0), (1, 2)),
    (65, 9, (2, 2), (1, 1)),
    (97, 33, (1, 2), (2, 1)),
    (130, 12, (0, 0), (0, 0)),
]


def run(case, precision, checked, nsteps, seg=0, block=0):
    with lbm.Simulation(case, precision=precision) as sim:
        sim.init_case()
        if seg or block:
            lbm.lbm_set_launch(sim.ctx, seg, block)
        lbm.lbm_set_checked(sim.ctx, checked)
        sim.step(nsteps)
        status = lbm.lib().lbm_check(sim.ctx)
        state, _ = sim.save_state()
    return status, state


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("nx,ny,bx,by", SHAPES)
def test_checked_kernel_finds_no_stray_access(nx, ny, bx, by, precision):
    case = W.random_drop(nx, ny, seed=nx * 37 + ny, wall_x=bx[0], wall_x_hi=bx[1],
                         wall_y=by[0], wall_y_hi=by[1], rho_ratio=50.0, gravity=1e-6,
                         marangoni=-2e-5)
    s_plain, plain = run(case, precision, False, 7)
    s_checked, checked = run(case, precision, True, 7)
    assert s_plain == lbm.LBM_OK
    assert s_checked == lbm.LBM_OK, lbm.lbm_strerror(s_checked)
    assert np.array_equal(plain, checked)


@pytest.mark.parametrize("seg,block", [(1, 32), (3, 64), (5, 256), (64, 128)])
def test_checked_kernel_under_other_launch_shapes(seg, block):
    case = W.random_drop(70, 37, seed=3, wall_x=2, wall_x_hi=1, wall_y=1, wall_y_hi=2,
                         rho_ratio=100.0)
    for precision in ("fp32", "fp16"):
        s_plain, plain = run(case, precision, False, 9, seg, block)
        s_checked, checked = run(case, precision, True, 9, seg, block)
        assert s_plain == lbm.LBM_OK and s_checked == lbm.LBM_OK
        assert np.array_equal(plain, checked)


def test_checked_mode_is_refused_for_step_variants():
    case = W.random_drop(16, 16, seed=1, collision=1)
    with lbm.Simulation(case, precision="fp32") as sim:
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_set_checked(sim.ctx, True)
        assert e.value.status == lbm.LBM_ERR_UNSUPPORTED


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_checker_reports_accesses_outside_its_declared_bounds(precision):
    """Self-test of the checker (mode 2): the declared bounds leave out the last row of both
    buffers (allocated memory, so nothing stray is touched); the steps' loads, copies and stores
    of that row are refused and reported as LBM_ERR_INDEX by every later synchronising call of
    that context, while the device stays usable for others."""
    case = W.random_drop(45, 20, seed=9, wall_y=1, rho_ratio=10.0)
    with lbm.Simulation(case, precision=precision) as sim:
        sim.init_case()
        lbm.lbm_set_checked(sim.ctx, 2)
        sim.step(3)
        assert lbm.lib().lbm_check(sim.ctx) == lbm.LBM_ERR_INDEX
        with pytest.raises(lbm.LbmError) as e:
            sim.fields()
        assert e.value.status == lbm.LBM_ERR_INDEX
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_set_checked(sim.ctx, 3)
        assert e.value.status == lbm.LBM_ERR_ARG
    with lbm.Simulation(case, precision=precision) as other:
        other.init_case().step(3)
        assert lbm.lib().lbm_check(other.ctx) == lbm.LBM_OK
