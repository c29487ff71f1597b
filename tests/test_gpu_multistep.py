"""The multi-step kernel (lbm_step's optional form for runs of two or more steps,
lbm_set_persistent) against one launch per step: the same state, bit for bit.

Both forms run the same per-warp march; the multi-step kernel only replaces the end of every
launch (all warps finished) by waits of each warp for its eight neighbouring warps, and reads
the halo columns through L2 instead of the read-only cache.  So any difference would be a
synchronisation error: a warp reading rows a neighbour had not finished writing, or overwriting
rows a neighbour was still reading.  The cases cover ragged and tiny grids, every side kind,
the four storage precisions, both collision models, both sigma laws, the imposed flow across
its reversal, launch shapes with many short segments (many neighbours per warp), and the
benchmark's drop impact, with runs of odd and even lengths.
"""
import numpy as np
import pytest

from paper_1909_04166_gb300 import lbm
from paper_1909_04166_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RUNS = (2, 7, 1, 12, 3)

SHAPES = [
    (16, 16, 0, 0),
    (17, 9, 1, 1),
    (33, 5, 0, 1),
    (70, 37, 1, 0),
    (1, 1, 0, 0),
    (1, 7, 0, 1),
    (5, 1, 1, 0),
    (96, 64, 0, 1),
    (130, 203, 0, 2),
    (257, 140, 2, 0),
]


def run(case, precision, path, runs=RUNS, launch=None):
    with lbm.Simulation(case, precision=precision) as sim:
        sim.init_case()
        if launch:
            lbm.lbm_set_launch(sim.ctx, *launch)
        lbm.lbm_set_persistent(sim.ctx, path == "multi")
        lbm.lbm_set_graphs(sim.ctx, path == "graphs")
        want = {"multi": lbm.LBM_PATH_MULTI, "graphs": lbm.LBM_PATH_GRAPHS,
                "single": lbm.LBM_PATH_SINGLE}[path]
        assert lbm.lbm_get_step_path(sim.ctx) == want
        for n in runs:
            sim.step(n)
        lbm.lbm_check(sim.ctx)
        assert lbm.lbm_steps_done(sim.ctx) == sum(runs)
        raw, steps = sim.save_state()
    return raw


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("nx,ny,bx,by", SHAPES)
def test_multistep_matches_single_launches(nx, ny, bx, by, precision):
    case = W.random_drop(nx, ny, seed=nx * 7 + ny, wall_x=bx, wall_y=by, rho_ratio=100.0,
                         gravity=1e-6, marangoni=-2e-5)
    assert np.array_equal(run(case, precision, "multi"), run(case, precision, "single"))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("collision,sigma_model", [(1, 0), (0, 1), (1, 1)])
def test_multistep_step_variants(precision, collision, sigma_model):
    case = W.random_drop(75, 66, seed=5, wall_y=1, rho_ratio=10.0, gravity=1e-6,
                         collision=collision, sigma_model=sigma_model, beta=0.4, psi0=0.2,
                         gradpsi_x=1e-3)
    assert np.array_equal(run(case, precision, "multi"), run(case, precision, "single"))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_multistep_imposed_flow_across_the_reversal(precision):
    case = W.shear_circle(L0=64, u0=0.03)
    case.update(reverse_step=20)
    runs = (15, 11, 2, 13)     # the second run is split at the reversal
    assert np.array_equal(run(case, precision, "multi", runs),
                          run(case, precision, "single", runs))


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
@pytest.mark.parametrize("launch", [(1, 32), (2, 64), (3, 128), (5, 256)])
def test_multistep_with_short_segments(precision, launch):
    """Segments of one to five rows: every warp waits for eight distinct neighbours, and the
    rows a warp reads are written by up to three segments."""
    case = W.random_drop(200, 90, seed=31, wall_y=1, rho_ratio=100.0, gravity=1e-6)
    with lbm.Simulation(case, precision=precision) as sim:
        lbm.lbm_set_launch(sim.ctx, *launch)
        lbm.lbm_set_persistent(sim.ctx, True)
        assert lbm.lbm_get_step_path(sim.ctx) == lbm.LBM_PATH_MULTI
    assert np.array_equal(run(case, precision, "multi", launch=launch),
                          run(case, precision, "single", launch=launch))


def test_launch_shape_beyond_residency_falls_back_to_graphs():
    """One-row segments on a grid whose warps cannot all be resident: the multi-step kernel is
    not used (it needs every warp resident), runs go to the graphs, with the same results."""
    case = W.random_drop(512, 600, seed=3, wall_y=1, rho_ratio=100.0)
    with lbm.Simulation(case, precision="fp32") as sim:
        lbm.lbm_set_persistent(sim.ctx, True)
        assert lbm.lbm_get_step_path(sim.ctx) == lbm.LBM_PATH_MULTI
        lbm.lbm_set_launch(sim.ctx, 1, 128)
        assert lbm.lbm_get_step_path(sim.ctx) == lbm.LBM_PATH_GRAPHS
    a = run(case, "fp32", "graphs", runs=(6, 3), launch=(1, 128))
    b = run(case, "fp32", "single", runs=(6, 3))
    assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", ["fp32", "fp16"])
def test_multistep_at_the_benchmark_size(precision):
    case = W.impact()
    runs = (20, 7)
    assert np.array_equal(run(case, precision, "multi", runs),
                          run(case, precision, "graphs", runs))


def test_default_paths():
    """FP32 storage takes the multi-step kernel by default where one wave of warps of segments
    at least 3 rows tall covers the grid; grids of shorter segments or several waves, and the
    other storage modes, take graph replays; 1 forces the multi-step kernel where it fits."""
    with lbm.Simulation(W.random_drop(96, 64, seed=2), precision="fp32") as sim:
        assert lbm.lbm_get_step_path(sim.ctx) == lbm.LBM_PATH_GRAPHS
        lbm.lbm_set_persistent(sim.ctx, 1)
        assert lbm.lbm_get_step_path(sim.ctx) == lbm.LBM_PATH_MULTI
        lbm.lbm_set_persistent(sim.ctx, 2)
        assert lbm.lbm_get_step_path(sim.ctx) == lbm.LBM_PATH_GRAPHS
        with pytest.raises(lbm.LbmError):
            lbm.lbm_set_persistent(sim.ctx, 3)
    for case, prec, path in ((W.impact(), "fp32", lbm.LBM_PATH_MULTI),
                             (W.rt(), "fp32", lbm.LBM_PATH_MULTI),
                             (W.marangoni(), "fp32", lbm.LBM_PATH_GRAPHS),
                             (W.random_drop(96, 64, seed=2), "fp32", lbm.LBM_PATH_GRAPHS),
                             (W.impact(ny=4096), "fp32", lbm.LBM_PATH_GRAPHS),
                             (W.impact(), "fp16", lbm.LBM_PATH_GRAPHS),
                             (W.impact(), "bf16", lbm.LBM_PATH_GRAPHS),
                             (W.random_drop(96, 64, seed=2), "fp64", lbm.LBM_PATH_GRAPHS)):
        with lbm.Simulation(case, precision=prec) as sim:
            assert lbm.lbm_get_step_path(sim.ctx) == path, (case["ny"], prec)
