"""Element-wise parity of the CUDA library with the FP64 oracle for the further forms: free-slip
walls (Secs. 6.4-6.6), the single-relaxation-time operators (Sec. 7), the Langmuir isotherm
(Sec. 6.7) and the interface lattice alone in the imposed reversing shear flow (Sec. 6.1).

Tolerances as for the coupled cascaded step: relative L2 <= 1e-12 in FP64 mode, <= 2e-5 in FP32
after the stated steps.  In the imposed-flow mode only the interface populations are state.
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


def gpu_run(case, precision, nsteps, path="graphs"):
    """path: how runs of two or more steps are issued (one launch per step, graph replays, the
    default, or the multi-step kernel)."""
    with lbm.Simulation(case, precision=precision) as sim:
        sim.init_case()
        lbm.lbm_set_persistent(sim.ctx, path == "multi")
        lbm.lbm_set_graphs(sim.ctx, path != "single")
        sim.step(nsteps)
        g, f = sim.populations()
        fl = sim.fields()
    return g, f, fl


# boundary kinds (left/right, bottom/top): 0 periodic, 1 no-slip, 2 free-slip
FREESLIP = [
    (45, 37, (0, 0), (1, 2)),    # no-slip bottom, free-slip top (drop impact, Sec. 6.6)
    (70, 33, (0, 0), (2, 2)),    # free-slip top and bottom (falling drop, Sec. 6.4)
    (33, 70, (2, 2), (1, 1)),    # free-slip sides, no-slip ends (rising bubble, Sec. 6.5)
    (40, 29, (2, 1), (1, 2)),    # mixed corners
    (64, 64, (2, 2), (2, 2)),    # free-slip all round
    (1, 9, (2, 2), (1, 2)),      # one column between free-slip sides
]


def _fs_case(nx, ny, bx, by, **kw):
    return W.random_drop(nx, ny, seed=nx * 11 + ny, wall_x=bx[0], wall_x_hi=bx[1],
                         wall_y=by[0], wall_y_hi=by[1], rho_ratio=100.0, gravity=1e-6,
                         marangoni=-2e-5, **kw)


@pytest.mark.parametrize("nx,ny,bx,by", FREESLIP)
@pytest.mark.parametrize("nsteps", [1, 40])
def test_freeslip_fp64_parity(nx, ny, bx, by, nsteps):
    case = _fs_case(nx, ny, bx, by)
    oc, g_ref, f_ref = oracle_run(case, nsteps)
    g, f, fl = gpu_run(case, "fp64", nsteps)
    assert rel_l2(g, g_ref) <= 1e-12
    assert rel_l2(f, f_ref) <= 1e-12
    ref = O.fields(oc, g_ref, f_ref)
    for k in ("phi", "p", "ux", "uy"):
        assert rel_l2(fl[k], ref[k]) <= 1e-12, k


@pytest.mark.parametrize("nx,ny,bx,by", FREESLIP[:5])
def test_freeslip_fp32_parity_200_steps(nx, ny, bx, by):
    case = _fs_case(nx, ny, bx, by)
    oc, g_ref, f_ref = oracle_run(case, 200)
    g, f, fl = gpu_run(case, "fp32", 200)
    assert rel_l2(f, f_ref) <= 2e-5
    assert rel_l2(g, g_ref) <= 2e-5


SRT_SHAPES = [(16, 16, 0, 0), (45, 37, 1, 1), (70, 33, 0, 1), (33, 70, 2, 1), (1, 7, 0, 1)]


@pytest.mark.parametrize("nx,ny,wx,wy", SRT_SHAPES)
@pytest.mark.parametrize("nsteps", [1, 40])
def test_srt_fp64_parity(nx, ny, wx, wy, nsteps):
    case = W.random_drop(nx, ny, seed=nx + 5 * ny, wall_x=wx, wall_y=wy, rho_ratio=10.0,
                         gravity=1e-6, marangoni=-2e-5, collision=1)
    oc, g_ref, f_ref = oracle_run(case, nsteps)
    g, f, fl = gpu_run(case, "fp64", nsteps)
    assert rel_l2(g, g_ref) <= 1e-12
    assert rel_l2(f, f_ref) <= 1e-12
    ref = O.fields(oc, g_ref, f_ref)
    for k in ("phi", "p", "ux", "uy"):
        assert rel_l2(fl[k], ref[k]) <= 1e-12, k


@pytest.mark.parametrize("nx,ny,wx,wy", SRT_SHAPES[:4])
def test_srt_fp32_parity_200_steps(nx, ny, wx, wy):
    case = W.random_drop(nx, ny, seed=nx + 5 * ny, wall_x=wx, wall_y=wy, rho_ratio=10.0,
                         gravity=1e-6, marangoni=-2e-5, collision=1)
    _, g_ref, f_ref = oracle_run(case, 200)
    g, f, _ = gpu_run(case, "fp32", 200)
    assert rel_l2(f, f_ref) <= 2e-5
    assert rel_l2(g, g_ref) <= 2e-5


LANGMUIR = [
    (40, 64, 0, 1, dict(beta=0.5, psi0=0.05, gradpsi_x=0.0, gradpsi_y=2e-3)),
    (70, 37, 1, 0, dict(beta=0.8, psi0=0.3, gradpsi_x=-3e-3, gradpsi_y=1e-3)),
    (33, 33, 2, 2, dict(beta=0.25, psi0=0.6, gradpsi_x=1e-3, gradpsi_y=-2e-3)),
]


@pytest.mark.parametrize("nx,ny,wx,wy,lang", LANGMUIR)
@pytest.mark.parametrize("collision", [0, 1])
def test_langmuir_fp64_parity(nx, ny, wx, wy, lang, collision):
    case = W.random_drop(nx, ny, seed=nx * 3 + ny, wall_x=wx, wall_y=wy, rho_ratio=10.0,
                         sigma=2e-3, sigma_model=1, collision=collision, **lang)
    oc, g_ref, f_ref = oracle_run(case, 40)
    g, f, fl = gpu_run(case, "fp64", 40)
    assert rel_l2(g, g_ref) <= 1e-12
    assert rel_l2(f, f_ref) <= 1e-12
    ref = O.fields(oc, g_ref, f_ref)
    for k in ("phi", "p", "ux", "uy"):
        assert rel_l2(fl[k], ref[k]) <= 1e-12, k


@pytest.mark.parametrize("nx,ny,wx,wy,lang", LANGMUIR[:2])
def test_langmuir_fp32_parity_200_steps(nx, ny, wx, wy, lang):
    case = W.random_drop(nx, ny, seed=nx * 3 + ny, wall_x=wx, wall_y=wy, rho_ratio=10.0,
                         sigma=2e-3, sigma_model=1, **lang)
    _, g_ref, f_ref = oracle_run(case, 200)
    g, f, _ = gpu_run(case, "fp32", 200)
    assert rel_l2(f, f_ref) <= 2e-5
    assert rel_l2(g, g_ref) <= 2e-5


def _shear(L0, u0, reverse_step, collision=0, nx=None):
    case = W.shear_circle(L0=L0, u0=u0)
    case.update(reverse_step=reverse_step, collision=collision)
    if nx is not None:   # a non-square, ragged box
        case.update(nx=nx)
        y, x = np.mgrid[0:L0, 0:nx].astype(float)
        case["fields"] = dict(phi=W.tanh_profile(0.2 * L0 - np.hypot(x - nx / 2, y - 0.3 * L0),
                                                 3.0),
                              p=np.zeros((L0, nx)), ux=np.zeros((L0, nx)), uy=np.zeros((L0, nx)))
    return case


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
@pytest.mark.parametrize("path", ["single", "graphs", "multi"])
@pytest.mark.parametrize("collision", [0, 1])
def test_shear_flow_parity_across_the_reversal(precision, tol, path, collision):
    """100 steps with the reversal at step 40: one launch per step, graph chunks of 32 on both
    sides of it, or one multi-step launch on each side; f and the reported fields against the
    oracle."""
    case = _shear(48, 0.03, 40, collision)
    oc, _, f_ref = oracle_run(case, 100)
    _, f, fl = gpu_run(case, precision, 100, path=path)
    assert rel_l2(f, f_ref) <= tol
    oc.t = 100
    ref = O.fields(oc, np.zeros_like(f_ref), f_ref)
    assert rel_l2(fl["phi"], ref["phi"]) <= tol
    for k in ("ux", "uy"):
        assert rel_l2(fl[k], ref[k]) <= max(tol, 1e-7 if precision == "fp32" else 0), k
    assert np.all(fl["p"] == 0.0)


def test_shear_flow_ragged_box_parity():
    case = _shear(40, 0.02, 25, nx=71)
    _, _, f_ref = oracle_run(case, 60)
    _, f, _ = gpu_run(case, "fp64", 60)
    assert rel_l2(f, f_ref) <= 1e-12


def test_shear_flow_returns_the_circle_at_full_size():
    """Sec. 6.1 at the paper's resolution: L0 = 200, W = 3, Pe = 60, U_0 = 0.02, reversed at
    T_f = 10000, back at 2 T_f = 20000 steps (FP32).  The phase mass is conserved."""
    case = W.shear_circle(L0=200, u0=0.02)
    tf = case["meta"]["t_f"]
    phi0 = case["fields"]["phi"]
    with lbm.Simulation(case, precision="fp32") as sim:
        sim.init_case()
        m0 = sim.diagnostics()["sum_phi"]
        sim.step(tf)
        phi_mid = sim.fields()["phi"]
        sim.step(tf)
        phi_end = sim.fields()["phi"]
        m1 = sim.diagnostics()["sum_phi"]

    def area_mismatch(a, b):
        return np.sum((a > 0.5) != (b > 0.5)) / np.sum(b > 0.5)

    # bounds from the oracle's resolution trend (L0 = 64: 0.039 / 0.134, L0 = 128: 0.012 /
    # 0.071); measured here 0.069 for the relative L2
    assert area_mismatch(phi_mid, phi0) > 1.0
    assert area_mismatch(phi_end, phi0) < 0.02
    assert rel_l2(phi_end, phi0) < 0.08
    assert abs(m1 - m0) <= 1e-5 * m0
