"""Element-wise parity of the CUDA library with the FP64 oracle on seeded random combinations of
everything a case can choose: grid size (ragged, down to one node wide), the kind of each of the
four sides (periodic pair, no-slip, free-slip, mixed), density and viscosity ratios, gravity,
the Marangoni gradient, the collision model (cascaded or single relaxation time, Secs. 4, 5,
7), the surface-tension law (linear in T, or the Langmuir isotherm of Sec. 6.7) and the storage
precision.  Each case runs 12 steps; bounds as for the other parity tests: relative L2
<= 1e-12 in FP64, <= 2e-5 in FP32, and for the 16-bit storage modes the measured bounds below.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_04166_gb300 import lbm
from paper_1909_04166_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NSTEPS = 12
TOL = {"fp64": 1e-12, "fp32": 2e-5}
SIDES = [(0, 0), (1, 1), (2, 2), (1, 2), (2, 1)]       # (low side, high side) of one axis


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def random_case(seed):
    rng = np.random.default_rng(7000 + seed)
    nx = int(rng.choice([1, 2, 5, 31, 32, 33, 63, 64, 65, 97]))
    ny = int(rng.integers(3, 41))
    bx, by = SIDES[rng.integers(len(SIDES))], SIDES[rng.integers(len(SIDES))]
    ratio = float(10 ** rng.uniform(0.0, 3.0))
    extra = dict(wall_x_hi=bx[1], wall_y_hi=by[1], collision=int(rng.integers(2)))
    if rng.random() < 0.4:   # Langmuir isotherm; psi stays well below 1 on the grid
        extra.update(sigma_model=1, beta=float(rng.uniform(0.1, 1.0)),
                     psi0=float(rng.uniform(0.0, 0.4)),
                     gradpsi_x=float(rng.uniform(-1e-3, 1e-3)),
                     gradpsi_y=float(rng.uniform(-1e-3, 1e-3)))
    return W.random_drop(nx, ny, seed=seed, wall_x=bx[0], wall_y=by[0], rho_ratio=ratio,
                         width=5.0 if ratio > 100 else 4.0,
                         gravity=float(rng.uniform(0.0, 2e-6)),
                         marangoni=float(rng.uniform(-3e-5, 3e-5)),
                         nu_a=float(rng.uniform(0.02, 0.2)), nu_b=float(rng.uniform(0.02, 0.2)),
                         **extra)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("seed", range(16))
def test_random_case_parity(seed, precision):
    case = random_case(seed)
    oc = O.OracleCase.from_dict(case.params)
    fl = case["fields"]
    g_ref, f_ref = O.init(oc, fl["phi"], fl["p"], fl["ux"], fl["uy"])
    g_ref, f_ref = O.run(oc, g_ref, f_ref, NSTEPS)
    ref = O.fields(oc, g_ref, f_ref)
    with lbm.Simulation(case, precision=precision) as sim:
        sim.init_case().step(NSTEPS)
        g, f = sim.populations()
        out = sim.fields()
    tol = TOL[precision]
    assert rel_l2(g, g_ref) <= tol, case["name"]
    assert rel_l2(f, f_ref) <= tol, case["name"]
    for k in ("phi", "p", "ux", "uy"):
        assert rel_l2(out[k], ref[k]) <= tol, (case["name"], k)


# 16-bit storage (the cascaded coupled step with the linear sigma(T), the forms it offers):
# bounds about three times the largest error measured over these 16 cases after 12 steps
# before the rest population's rounding compensation (which lowered the errors on the drop
# workloads; these cases pass with it under the same bounds) (FP16: g
# 5.1e-4, f 2.5e-5, phi 2.3e-5, p 6.2e-4, u 3.0e-3; BF16: g 3.4e-3, f 2.3e-4, phi 1.6e-4, p
# 4.5e-3, u 1.4e-2).
BOUNDS16 = {
    "fp16": {"g": 1.5e-3, "f": 1e-4, "phi": 1e-4, "p": 2e-3, "ux": 1e-2, "uy": 1e-2},
    "bf16": {"g": 1e-2, "f": 7e-4, "phi": 5e-4, "p": 1.5e-2, "ux": 5e-2, "uy": 5e-2},
}


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
@pytest.mark.parametrize("seed", range(16))
def test_random_case_16bit_storage(seed, precision):
    case = random_case(seed)
    case.update(collision=0, sigma_model=0)
    oc = O.OracleCase.from_dict(case.params)
    fl = case["fields"]
    g_ref, f_ref = O.init(oc, fl["phi"], fl["p"], fl["ux"], fl["uy"])
    g_ref, f_ref = O.run(oc, g_ref, f_ref, NSTEPS)
    ref = O.fields(oc, g_ref, f_ref)
    with lbm.Simulation(case, precision=precision) as sim:
        sim.init_case().step(NSTEPS)
        g, f = sim.populations()
        out = sim.fields()
    b = BOUNDS16[precision]
    assert rel_l2(g, g_ref) <= b["g"], case["name"]
    assert rel_l2(f, f_ref) <= b["f"], case["name"]
    for k in ("phi", "p", "ux", "uy"):
        assert rel_l2(out[k], ref[k]) <= b[k], (case["name"], k)
