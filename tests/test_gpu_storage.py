"""16-bit storage modes (LBM_FP32_FP16, LBM_FP32_BF16): populations stored as scaled deviations
from w_a * ref in half / bfloat16, collided in float.

What is pinned: the codec round trip is exact (a state read out and written back is stored
bit for bit as before); one step from a representable state differs from the FP64 step of the
same state only by the storage rounding of the result; over 1000 steps the fields stay within
the stated bounds of the FP64 oracle (bounds measured on this path and recorded in the
design notes; 16-bit storage is far less accurate than FP32 storage for slow flows, because
the stored values carry the pressure level while the momentum is much smaller)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_04166_gb300 import lbm
from paper_1909_04166_gb300 import workloads as W

pytestmark = pytest.mark.gpu
FORMATS = ["fp16", "bf16"]


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("prec", FORMATS)
def test_codec_round_trip_is_exact(prec):
    case = W.random_drop(70, 45, seed=3, wall_y=True, rho_ratio=10.0)
    with lbm.Simulation(case, precision=prec) as s:
        s.init_case().step(30)
        g, f = s.populations()
        s.set_populations(g, f)
        g2, f2 = s.populations()
        assert np.array_equal(g, g2) and np.array_equal(f, f2)
        s.step(7)
        g3, f3 = s.populations()
    with lbm.Simulation(case, precision=prec) as t:
        t.set_populations(g, f).step(7)
        g4, f4 = t.populations()
    assert np.array_equal(g3, g4) and np.array_equal(f3, f4)


@pytest.mark.parametrize("prec,tol_g,tol_f", [("fp16", 5e-4, 2e-4), ("bf16", 4e-3, 1e-3)])
def test_one_step_differs_by_storage_rounding_only(prec, tol_g, tol_f):
    case = W.marangoni()
    with lbm.Simulation(case, precision=prec) as s:
        s.init_case().step(50)
        g, f = s.populations()
        g1, f1 = s.step(1).populations()
    with lbm.Simulation(case, precision="fp64") as t:
        gr, fr = t.set_populations(g, f).step(1).populations()
    assert rel_l2(g1, gr) <= tol_g
    assert rel_l2(f1, fr) <= tol_f


BOUNDS = {  # 1000 steps of the Marangoni drop (density ratio 10) against the FP64 oracle
    "fp16": {"phi": 5e-3, "p": 2.5e-2, "ux": 0.25, "uy": 0.25, "mass": 5e-5},
    "bf16": {"phi": 1.5e-2, "p": 2.5e-2, "ux": 0.4, "uy": 0.4, "mass": 2e-4},
}


@pytest.mark.parametrize("prec", FORMATS)
def test_1000_steps_within_stated_bounds(prec):
    case = W.marangoni()
    oc = O.OracleCase.from_dict(case.params)
    fl = case["fields"]
    g0, f0 = O.init(oc, fl["phi"], fl["p"], fl["ux"], fl["uy"])
    ref = O.fields(oc, *O.run(oc, g0, f0, 1000))
    with lbm.Simulation(case, precision=prec) as s:
        s.init_case()
        m0 = s.diagnostics()["sum_phi"]
        got = s.step(1000).fields()
        m1 = s.diagnostics()["sum_phi"]
    for k in ("phi", "p", "ux", "uy"):
        assert rel_l2(got[k], ref[k]) <= BOUNDS[prec][k], k
    assert abs(m1 - m0) <= BOUNDS[prec]["mass"] * m0


def test_fp16_impact_at_density_ratio_1000():
    case = W.impact()
    with lbm.Simulation(case, precision="fp64") as a, lbm.Simulation(case, precision="fp16") as b:
        ref = a.init_case().step(1000).fields()
        got = b.init_case().step(1000).fields()
    for k, bound in (("phi", 1e-2), ("p", 3e-2), ("ux", 0.25), ("uy", 0.25)):
        assert np.isfinite(got[k]).all()
        assert rel_l2(got[k], ref[k]) <= bound, k
