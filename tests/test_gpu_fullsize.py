"""Parity at the benchmark's full size and launch configuration (2048 x 1024 drop impact at
density ratio 1000, default launch of lbm_step as bench.py times it).

* one step from a GPU state, GPU vs the FP64 oracle stepping the same state (element-wise);
* FP32 after 1000 steps against the FP64 oracle run from the same initial fields (the north-star
  gate: relative L2 <= 2e-5) and against the GPU FP64 mode;
* Rayleigh-Taylor 256 x 1024 (walls, gravity) FP32 after 1000 steps against the oracle.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_04166_gb300 import lbm
from paper_1909_04166_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def impact_case():
    return W.impact()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-7)])
def test_one_step_at_full_size(impact_case, prec, tol):
    oc = O.OracleCase.from_dict(impact_case.params)
    with lbm.Simulation(impact_case, precision=prec) as sim:
        sim.init_case().step(20)
        g0, f0 = sim.populations()          # exact (FP32 values are representable in FP64)
        sim.step(1)
        g1, f1 = sim.populations()
    g_ref, f_ref = O.step(oc, g0, f0)
    assert rel_l2(g1, g_ref) <= tol
    assert rel_l2(f1, f_ref) <= tol
    # sampled nodes, element by element (interface, film, wall rows, periodic seam)
    for (x, y) in [(1024, 120), (1024, 20), (0, 0), (2047, 1023), (900, 200), (1100, 5)]:
        for a in range(9):
            assert abs(g1[a, y, x] - g_ref[a, y, x]) <= 1e-5 * np.abs(g_ref).max()
            assert abs(f1[a, y, x] - f_ref[a, y, x]) <= 1e-5


def test_fp32_after_1000_steps_matches_fp64_oracle(impact_case):
    oc = O.OracleCase.from_dict(impact_case.params)
    fl = impact_case["fields"]
    g, f = O.init(oc, fl["phi"], fl["p"], fl["ux"], fl["uy"])
    g, f = O.run(oc, g, f, 1000)
    ref = O.fields(oc, g, f)
    with lbm.Simulation(impact_case, precision="fp32") as sim:
        got = sim.init_case().step(1000).fields()
        g32, f32 = sim.populations()
    assert rel_l2(f32, f) <= 2e-5
    assert rel_l2(g32, g) <= 2e-5
    for k in ("phi", "p", "ux", "uy"):
        assert rel_l2(got[k], ref[k]) <= 2e-5, k


def test_fp32_matches_fp64_mode_after_1000_steps(impact_case):
    out = {}
    for prec in ("fp64", "fp32"):
        with lbm.Simulation(impact_case, precision=prec) as sim:
            out[prec] = sim.init_case().step(1000).fields()
    for k in ("phi", "p", "ux", "uy"):
        assert rel_l2(out["fp32"][k], out["fp64"][k]) <= 2e-5, k


def test_rayleigh_taylor_fp32_1000_steps():
    case = W.rt()
    oc = O.OracleCase.from_dict(case.params)
    fl = case["fields"]
    g, f = O.init(oc, fl["phi"], fl["p"], fl["ux"], fl["uy"])
    g, f = O.run(oc, g, f, 1000)
    ref = O.fields(oc, g, f)
    with lbm.Simulation(case, precision="fp32") as sim:
        got = sim.init_case().step(1000).fields()
    for k in ("phi", "p", "ux", "uy"):
        assert rel_l2(got[k], ref[k]) <= 2e-5, k
