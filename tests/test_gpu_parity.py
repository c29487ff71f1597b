"""Element-wise parity of the CUDA library (through the C ABI) with the FP64 oracle.

Tolerances: relative L2 <= 1e-12 for the FP64 mode (any number of steps tested here), and for
FP32 storage/compute <= 2e-5 after the stated number of steps.  Populations are compared
plane by plane; fields (phi, p, u, rho) through lbm_get_fields.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_04166_gb300 import lbm
from paper_1909_04166_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def oracle_run(case, nsteps):
    oc = O.OracleCase.from_dict(case.params)
    fl = case["fields"]
    g, f = O.init(oc, fl["phi"], fl["p"], fl["ux"], fl["uy"])
    if nsteps:
        g, f = O.run(oc, g, f, nsteps)
    return oc, g, f


SHAPES = [
    (16, 16, False, False),
    (17, 9, True, True),
    (33, 5, False, True),
    (70, 37, True, False),
    (1, 1, False, False),
    (1, 7, False, True),
    (5, 1, True, False),
    (96, 64, False, True),
]


@pytest.mark.parametrize("nx,ny,wx,wy", SHAPES)
def test_init_matches_oracle(nx, ny, wx, wy):
    case = W.random_drop(nx, ny, seed=nx * 131 + ny, wall_x=wx, wall_y=wy)
    _, g_ref, f_ref = oracle_run(case, 0)
    with lbm.Simulation(case, precision="fp64") as sim:
        g, f = sim.init_case().populations()
    assert rel_l2(g, g_ref) <= 1e-13
    assert rel_l2(f, f_ref) <= 1e-13


@pytest.mark.parametrize("nx,ny,wx,wy", SHAPES)
@pytest.mark.parametrize("nsteps", [1, 40])
def test_fp64_step_parity(nx, ny, wx, wy, nsteps):
    case = W.random_drop(nx, ny, seed=nx * 7 + ny, wall_x=wx, wall_y=wy, rho_ratio=100.0,
                         gravity=1e-6, marangoni=-2e-5)
    oc, g_ref, f_ref = oracle_run(case, nsteps)
    with lbm.Simulation(case, precision="fp64") as sim:
        sim.init_case().step(nsteps)
        g, f = sim.populations()
        fl = sim.fields()
    assert rel_l2(g, g_ref) <= 1e-12
    assert rel_l2(f, f_ref) <= 1e-12
    ref = O.fields(oc, g_ref, f_ref)
    for k in ("phi", "p", "ux", "uy", "rho"):
        assert rel_l2(fl[k], ref[k]) <= 1e-12, k


# full 64-column strips without x walls take the paired stores of the fast path: one strip that
# wraps onto itself, and two strips whose edge lanes store into each other
FULL_STRIPS = [(64, 40, False, False), (128, 24, False, True)]


@pytest.mark.parametrize("nx,ny,wx,wy", SHAPES[:4] + SHAPES[7:] + FULL_STRIPS)
def test_fp32_parity_200_steps(nx, ny, wx, wy):
    case = W.random_drop(nx, ny, seed=nx + 3 * ny, wall_x=wx, wall_y=wy, rho_ratio=100.0,
                         gravity=1e-6, marangoni=-2e-5)
    oc, g_ref, f_ref = oracle_run(case, 200)
    with lbm.Simulation(case, precision="fp32") as sim:
        sim.init_case().step(200)
        g, f = sim.populations()
        fl = sim.fields()
    ref = O.fields(oc, g_ref, f_ref)
    assert rel_l2(f, f_ref) <= 2e-5
    assert rel_l2(g, g_ref) <= 2e-5
    for k in ("phi", "p", "ux", "uy"):
        assert rel_l2(fl[k], ref[k]) <= 2e-5, k


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16"])
def test_launch_shape_does_not_change_results(prec):
    """Segments of different heights (and both marching directions) and block sizes give
    identical bits, for one column per lane (FP64) and the paired forms (FP32, 16-bit)."""
    case = W.random_drop(75, 61, seed=4, wall_y=True, rho_ratio=100.0)
    outs = []
    for seg, block in ((0, 0), (1, 32), (3, 64), (7, 256), (61, 128)):
        with lbm.Simulation(case, precision=prec) as sim:
            sim.init_case()
            lbm.lbm_set_launch(sim.ctx, seg, block)
            sim.step(9)
            outs.append(sim.populations())
    for g, f in outs[1:]:
        assert np.array_equal(g, outs[0][0]) and np.array_equal(f, outs[0][1])


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
def test_graph_replays_match_single_launches(precision):
    """Runs of every length give the same state, bit for bit, as one launch per step: as graph
    replays (the default: graphs of 32, 16, 8, 4 and 2 chained launches, a last odd step alone)
    and as multi-step launches."""
    case = W.random_drop(64, 48, seed=12, wall_y=True, rho_ratio=100.0)
    outs = []
    for persistent, graphs, path in ((False, False, lbm.LBM_PATH_SINGLE),
                                     (False, True, lbm.LBM_PATH_GRAPHS),
                                     (True, True, lbm.LBM_PATH_MULTI)):
        with lbm.Simulation(case, precision=precision) as sim:
            sim.init_case()
            lbm.lbm_set_persistent(sim.ctx, persistent)
            lbm.lbm_set_graphs(sim.ctx, graphs)
            assert lbm.lbm_get_step_path(sim.ctx) == path
            for n in (70, 33, 20, 3, 2, 1, 17, 31):
                sim.step(n)
            assert lbm.lbm_steps_done(sim.ctx) == 177
            outs.append(sim.populations())
    for g, f in outs[1:]:
        assert np.array_equal(outs[0][0], g) and np.array_equal(outs[0][1], f)


@pytest.mark.parametrize("persistent", [False, True])
def test_zero_steps_change_nothing(persistent):
    """lbm_step(ctx, 0) is a no-op (state bytes and step counter), before and after other
    runs, on every launch path."""
    case = W.random_drop(37, 29, seed=4, wall_x=True, rho_ratio=100.0)
    with lbm.Simulation(case, precision="fp32") as sim:
        sim.init_case()
        lbm.lbm_set_persistent(sim.ctx, persistent)
        a, ta = sim.save_state()
        sim.step(0)
        b, tb = sim.save_state()
        assert ta == tb == 0 and np.array_equal(a, b)
        sim.step(5)
        a, ta = sim.save_state()
        sim.step(0)
        b, tb = sim.save_state()
        assert ta == tb == 5 and np.array_equal(a, b)


def test_checkpoint_restart_is_exact():
    case = W.random_drop(48, 40, seed=8, wall_x=True, rho_ratio=50.0)
    for prec in ("fp64", "fp32"):
        with lbm.Simulation(case, precision=prec) as a:
            a.init_case().step(10)
            g, f = a.populations()
            a.step(15)
            ga, fa = a.populations()
        with lbm.Simulation(case, precision=prec) as b:
            b.set_populations(g, f).step(15)
            gb, fb = b.populations()
        assert np.array_equal(ga, gb) and np.array_equal(fa, fb)


def test_diagnostics_match_oracle_fields():
    """lbm_diagnostics reduces the fields of the GPU state; the oracle's fields of the same
    state (populations copied out exactly) give the reference sums."""
    case = W.laplace(n=48, radius=12.0, width=5.0, rho_ratio=1000.0, sigma=1e-3)
    oc = O.OracleCase.from_dict(case.params)
    y, x = np.mgrid[0:48, 0:48].astype(float)
    r = np.hypot(x - 24, y - 24)
    for prec in ("fp64", "fp32"):
        with lbm.Simulation(case, precision=prec) as sim:
            sim.init_case().step(300)
            d = sim.diagnostics(24.0, 24.0, 2.0, 22.0)
            g, f = sim.populations()
        ref = O.fields(oc, g, f)
        tol = 1e-12 if prec == "fp64" else 2e-6
        assert d["nonfinite"] == 0
        assert d["sum_phi"] == pytest.approx(ref["phi"].sum(), rel=1e-13 if prec == "fp64" else 1e-7)
        assert d["sum_p"] == pytest.approx(ref["p"].sum(), rel=tol, abs=1e-16)
        assert d["max_speed"] == pytest.approx(np.hypot(ref["ux"], ref["uy"]).max(), rel=tol)
        dp = ref["p"][r < 2.0].mean() - ref["p"][r > 22.0].mean()
        assert d["dp_laplace"] == pytest.approx(dp, rel=tol)


def test_phi_mass_conserved_fp64_and_fp32():
    case = W.random_drop(130, 70, seed=2, wall_x=True, wall_y=True, rho_ratio=100.0)
    for prec, tol in (("fp64", 1e-13), ("fp32", 2e-6)):
        with lbm.Simulation(case, precision=prec) as sim:
            sim.init_case()
            m0 = sim.diagnostics()["sum_phi"]
            sim.step(500)
            m1 = sim.diagnostics()["sum_phi"]
        assert abs(m1 - m0) <= tol * abs(m0), prec


def test_errors_are_returned_not_raised_on_device():
    case = W.random_drop(16, 16, seed=1)
    p = lbm.make_params(case, "fp32")
    p.rho_b = -1.0
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(p)
    assert e.value.status == lbm.LBM_ERR_PARAM
    p = lbm.make_params(case, "fp32")
    p.nx = 0
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(p)
    assert e.value.status == lbm.LBM_ERR_ARG
    p = lbm.make_params(case, "fp32")
    p.precision = 9
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(p)
    assert e.value.status == lbm.LBM_ERR_UNSUPPORTED
    with lbm.Simulation(case) as sim:
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_step(sim.ctx, 1)      # not initialised
        assert e.value.status == lbm.LBM_ERR_STATE
        sim.init_case()
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_step(sim.ctx, -1)
        assert e.value.status == lbm.LBM_ERR_ARG
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_set_launch(sim.ctx, 0, 48)
        assert e.value.status == lbm.LBM_ERR_ARG
        sim.step(1)


def test_nonfinite_fields_are_reported():
    case = W.random_drop(20, 20, seed=1)
    fl = dict(case["fields"])
    phi = fl["phi"].copy()
    phi[5, 7] = np.nan
    with lbm.Simulation(case, precision="fp32") as sim:
        sim.init(phi, fl["p"], fl["ux"], fl["uy"])
        d = lbm.lbm_diagnostics(sim.ctx)
        assert d["nonfinite"] >= 1
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_diagnostics(sim.ctx, allow_nonfinite=False)
        assert e.value.status == lbm.LBM_ERR_NONFINITE


def test_caller_supplied_device_buffer():
    torch = pytest.importorskip("torch")
    case = W.random_drop(40, 24, seed=6, wall_y=True)
    p = lbm.make_params(case, "fp32", stream=torch.cuda.current_stream().cuda_stream)
    nbytes = lbm.lbm_state_bytes(p)
    buf = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    ctx = lbm.lbm_create_with_buffer(p, buf.data_ptr(), nbytes)
    try:
        fl = case["fields"]
        dev = [torch.tensor(fl[k], dtype=torch.float64, device="cuda") for k in
               ("phi", "p", "ux", "uy")]
        lbm.lbm_init_fields_device(ctx, *(t.data_ptr() for t in dev))
        lbm.lbm_step(ctx, 12)
        g = np.empty((9, 24, 40))
        f = np.empty((9, 24, 40))
        lbm.lbm_get_populations(ctx, g, f)
    finally:
        lbm.lbm_destroy(ctx)
    with lbm.Simulation(case, precision="fp32") as sim:
        g2, f2 = sim.init_case().step(12).populations()
    assert np.array_equal(g, g2) and np.array_equal(f, f2)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_create_with_buffer(p, buf.data_ptr(), nbytes - 1)
