"""Pins of the FP64 oracle for the paper's further boundary, collision and surface-tension forms
(CPU only): free-slip walls (Secs. 6.4-6.6), the single-relaxation-time operators of the
stability comparison (Sec. 7), the Langmuir isotherm of the surfactant Marangoni case (Sec. 6.7)
and the interface lattice in the imposed reversing shear flow (Sec. 6.1).

Each test checks the oracle against something other than itself: mirror images of runs that use
only no-slip or periodic boundaries, population-space BGK relaxation towards the (separately
pinned) equilibria, reductions to already pinned cases, the Laplace law and the Marangoni
traction of a flat interface, and the shape return of the reversed shear flow.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_04166_gb300 import workloads as W

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
MIRROR_Y = [0, 1, 4, 3, 2, 8, 7, 6, 5]   # population index under y -> -y
MIRROR_X = [0, 3, 2, 1, 4, 6, 5, 8, 7]   # under x -> -x
RNG = np.random.default_rng(90416)


def _state(case):
    oc = O.OracleCase.from_dict(case.params)
    fl = case["fields"]
    g, f = O.init(oc, fl["phi"], fl["p"], fl["ux"], fl["uy"])
    return oc, g, f


def _case(nx, ny, fields, **kw):
    c = W.random_drop(nx, ny, seed=0, rho_ratio=10.0, sigma=1e-3, mobility=0.05, width=4.0)
    c.update(kw)
    c["fields"] = fields
    return c


def _mirror_fields_y(nx, H, rng):
    """Fields on a 2H-row grid, mirror-symmetric about y = H - 1/2 (u_y odd), with a drop cut
    by the mirror line and a random velocity field."""
    y, x = np.mgrid[0:2 * H, 0:nx].astype(float)
    phi = W.tanh_profile(0.35 * H - np.hypot(x - nx / 2 + 0.3, y - (H - 0.5)), 4.0)
    ux = 1e-3 * rng.standard_normal((H, nx))
    uy = 1e-3 * rng.standard_normal((H, nx))
    p = 1e-4 * rng.standard_normal((H, nx))
    ux = np.concatenate([ux, ux[::-1]])
    uy = np.concatenate([uy, -uy[::-1]])
    p = np.concatenate([p, p[::-1]])
    return dict(phi=phi, p=p, ux=ux, uy=uy)


def _half(fields, rows=None, cols=None):
    return {k: np.ascontiguousarray(v[rows or slice(None), cols or slice(None)])
            for k, v in fields.items()}


# ---------------------------------------------------------------------------------------------
# Free-slip walls (R14)
# ---------------------------------------------------------------------------------------------

def test_freeslip_top_is_mirror_plane_of_noslip_channel():
    """A channel with a no-slip bottom and a free-slip top evolves exactly as the lower half of
    the channel twice as high with no-slip walls on both ends, started mirror-symmetric: the
    free-slip wall is its symmetry line."""
    nx, H, steps = 12, 10, 30
    full = _mirror_fields_y(nx, H, np.random.default_rng(1))
    kw = dict(gx=1e-5, gy=0.0, rho_ref=0.2, dsigma_dT=-2e-5, gradT_x=0.01, gradT_y=0.0)
    oa, ga, fa = _state(_case(nx, 2 * H, full, wall_x=0, wall_y=1, **kw))
    ob, gb, fb = _state(_case(nx, H, _half(full, rows=slice(0, H)), wall_x=0, wall_y=1,
                              wall_y_hi=2, **kw))
    ga, fa = O.run(oa, ga, fa, steps)
    gb, fb = O.run(ob, gb, fb, steps)
    # the doubled run stays symmetric, and its lower half is the free-slip run
    assert np.allclose(fa[MIRROR_Y][:, ::-1], fa, rtol=0, atol=1e-13)
    assert np.allclose(fb, fa[:, :H], rtol=0, atol=1e-13)
    assert np.allclose(gb, ga[:, :H], rtol=0, atol=1e-14)


def test_freeslip_both_ends_is_periodic_mirror():
    """Free-slip walls at both ends: the lower half of a periodic box twice as high whose
    initial state is mirror-symmetric about y = H - 1/2 (and, through the period, y = -1/2)."""
    nx, H, steps = 9, 8, 30
    full = _mirror_fields_y(nx, H, np.random.default_rng(2))
    kw = dict(gx=-2e-5, gy=0.0, rho_ref=0.5)
    oa, ga, fa = _state(_case(nx, 2 * H, full, wall_x=0, wall_y=0, **kw))
    ob, gb, fb = _state(_case(nx, H, _half(full, rows=slice(0, H)), wall_x=0, wall_y=2, **kw))
    ga, fa = O.run(oa, ga, fa, steps)
    gb, fb = O.run(ob, gb, fb, steps)
    assert np.allclose(fb, fa[:, :H], rtol=0, atol=1e-13)
    assert np.allclose(gb, ga[:, :H], rtol=0, atol=1e-14)


def test_freeslip_left_side_is_mirror_plane():
    """x version with mixed sides: a free-slip left side and a no-slip right side (the rising
    bubble's sides, Sec. 6.5) against the right half of a box twice as wide with no-slip sides,
    mirror-symmetric about x = Wd - 1/2, under vertical gravity and no-slip ends."""
    Wd, ny, steps = 9, 14, 30
    rng = np.random.default_rng(3)
    y, x = np.mgrid[0:ny, 0:2 * Wd].astype(float)
    phi = W.tanh_profile(np.hypot(x - (Wd - 0.5), y - ny / 2) - 3.0, 4.0)
    ux = 1e-3 * rng.standard_normal((ny, Wd))
    uy = 1e-3 * rng.standard_normal((ny, Wd))
    p = 1e-4 * rng.standard_normal((ny, Wd))
    full = dict(phi=phi, p=np.concatenate([p[:, ::-1], p], axis=1),
                ux=np.concatenate([-ux[:, ::-1], ux], axis=1),
                uy=np.concatenate([uy[:, ::-1], uy], axis=1))
    kw = dict(gx=0.0, gy=-3e-5, rho_ref=1.0)
    oa, ga, fa = _state(_case(2 * Wd, ny, full, wall_x=1, wall_y=1, **kw))
    ob, gb, fb = _state(_case(Wd, ny, _half(full, cols=slice(Wd, 2 * Wd)), wall_x=2,
                              wall_x_hi=1, wall_y=1, **kw))
    ga, fa = O.run(oa, ga, fa, steps)
    gb, fb = O.run(ob, gb, fb, steps)
    assert np.allclose(fa[MIRROR_X][:, :, ::-1], fa, rtol=0, atol=1e-13)
    assert np.allclose(fb, fa[:, :, Wd:], rtol=0, atol=1e-13)
    assert np.allclose(gb, ga[:, :, Wd:], rtol=0, atol=1e-14)


def test_freeslip_walls_keep_uniform_tangential_flow():
    """Specular reflection keeps the tangential momentum: a uniform single-phase flow along
    free-slip walls stays uniform (with no-slip walls the same flow is slowed at the walls)."""
    nx, ny, U = 6, 10, 0.05
    fields = dict(phi=np.ones((ny, nx)), p=np.zeros((ny, nx)), ux=np.full((ny, nx), U),
                  uy=np.zeros((ny, nx)))
    for kind, stays in ((2, True), (1, False)):
        oc, g, f = _state(_case(nx, ny, dict(fields), wall_x=0, wall_y=kind))
        g, f = O.run(oc, g, f, 50)
        fl = O.fields(oc, g, f)
        dev = max(np.abs(fl["ux"] - U).max(), np.abs(fl["uy"]).max(), np.abs(fl["p"]).max())
        assert (dev < 1e-14) == stays, (kind, dev)


def test_freeslip_conserves_phase_mass():
    oc, g, f = _state(W.random_drop(17, 13, seed=4, wall_x=2, wall_y=1, wall_y_hi=2,
                                    rho_ratio=10.0, gravity=1e-6))
    m0 = f.sum()
    g, f = O.run(oc, g, f, 150)
    assert np.isfinite(g).all() and abs(f.sum() - m0) <= 1e-13 * m0


# ---------------------------------------------------------------------------------------------
# Single relaxation time (R15)
# ---------------------------------------------------------------------------------------------

def _basis_K():
    ex, ey = EX.astype(float), EY.astype(float)
    one = np.ones(9)
    return np.stack([one, ex, ey, 3 * (ex ** 2 + ey ** 2) - 4, ex ** 2 - ey ** 2, ex * ey,
                     -3 * ex ** 2 * ey + 2 * ey, -3 * ex * ey ** 2 + 2 * ex,
                     9 * ex ** 2 * ey ** 2 - 6 * (ex ** 2 + ey ** 2) + 4], axis=1)


@pytest.mark.parametrize("trial", range(8))
def test_srt_fluid_collision_is_bgk_without_forces(trial):
    """With all rates equal to omega and no forces, the fluid operator of Sec. 4 is BGK in
    population space towards g^eq(p, u, rho) (pinned against the transformed Maxwellian)."""
    rho = RNG.uniform(0.001, 1.0)
    p = RNG.uniform(-1e-3, 1e-3)
    ux, uy = RNG.uniform(-0.1, 0.1, 2)
    geq = O.geq(p, ux, uy, rho)
    g = geq + _basis_K()[:, 3:] @ RNG.uniform(-1e-3, 1e-3, 6)   # no zeroth / first moment
    w = RNG.uniform(0.2, 1.95)
    out, _ = O.fluid_collide(g, p, ux, uy, rho, 0.0, 0.0, 0.0, 0.0, np.full(9, w))
    assert np.allclose(out, g + w * (geq - g), rtol=0, atol=1e-15)


@pytest.mark.parametrize("trial", range(8))
def test_srt_ace_collision_is_bgk(trial):
    """With all rates equal to omega^phi the interface operator of Sec. 5 is BGK towards
    f^eq(phi, u, M_phi theta n) (pinned against the continuous moments)."""
    f = RNG.uniform(0.0, 0.2, 9)
    ux, uy = RNG.uniform(-0.2, 0.2, 2)
    jx, jy = RNG.uniform(-0.01, 0.01, 2)
    w = RNG.uniform(0.2, 1.95)
    out, _ = O.ace_collide(f, ux, uy, jx, jy, np.full(9, w))
    feq = O.feq(f.sum(), ux, uy, jx, jy)
    assert np.allclose(out, f + w * (feq - f), rtol=0, atol=1e-15)


def test_srt_equals_cascaded_when_every_rate_is_one():
    """nu = 1/6 and M_phi = 1/6 make every rate 1 in both models: the step is then the same
    computation; with another viscosity the two models differ."""
    base = W.random_drop(14, 11, seed=6, wall_y=1, rho_ratio=1.0, gravity=1e-6,
                         marangoni=-2e-5, mobility=1.0 / 6.0, nu_a=1.0 / 6.0, nu_b=1.0 / 6.0)
    runs = {}
    for col in (0, 1):
        case = W.random_drop(14, 11, seed=6, wall_y=1, rho_ratio=1.0, gravity=1e-6,
                             marangoni=-2e-5, mobility=1.0 / 6.0, nu_a=1.0 / 6.0,
                             nu_b=1.0 / 6.0, collision=col)
        oc, g, f = _state(case)
        runs[col] = O.run(oc, g, f, 20)
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    assert base["mu_a"] == pytest.approx(1.0 / 6.0)
    other = {}
    for col in (0, 1):
        oc, g, f = _state(W.random_drop(14, 11, seed=6, wall_y=1, rho_ratio=1.0, nu_a=0.02,
                                        nu_b=0.02, collision=col))
        other[col] = O.run(oc, g, f, 20)
    assert not np.allclose(other[0][0], other[1][0], rtol=0, atol=1e-9)


def test_srt_conserves_phase_mass():
    oc, g, f = _state(W.random_drop(15, 12, seed=8, wall_x=1, rho_ratio=10.0, collision=1))
    m0 = f.sum()
    g, f = O.run(oc, g, f, 100)
    assert np.isfinite(g).all() and abs(f.sum() - m0) <= 1e-13 * m0


# ---------------------------------------------------------------------------------------------
# Langmuir isotherm (R16)
# ---------------------------------------------------------------------------------------------

def test_langmuir_without_elasticity_is_constant_sigma():
    """beta = 0: sigma = sigma0 everywhere, the same step as the constant-sigma case."""
    runs = []
    for model in (0, 1):
        case = W.random_drop(16, 13, seed=9, wall_y=1, rho_ratio=10.0, marangoni=0.0,
                             sigma_model=model, beta=0.0, psi0=0.2, gradpsi_x=3e-3,
                             gradpsi_y=-1e-3)
        oc, g, f = _state(case)
        runs.append(O.run(oc, g, f, 15))
    assert np.allclose(runs[0][0], runs[1][0], rtol=0, atol=1e-17)
    assert np.allclose(runs[0][1], runs[1][1], rtol=0, atol=1e-15)


@pytest.mark.parametrize("psi0,beta", [(0.3, 0.4), (0.6, 0.25)])
def test_langmuir_uniform_psi_scales_laplace_pressure(psi0, beta):
    """With a uniform psi the drop feels sigma(psi0) = sigma0 [1 + beta ln(1 - psi0)] (Sec. 6.7
    Eq. Langmuirisotherm): the step equals the constant-sigma step with that sigma, and the
    Laplace pressure (linear in sigma) is that of the clean interface times 1 + beta ln(1-psi0)."""
    factor = 1.0 + beta * math.log(1.0 - psi0)
    dps = []
    for kw in (dict(sigma0=1e-3, sigma_model=1, beta=beta, psi0=psi0),
               dict(sigma0=1e-3 * factor, sigma_model=0),
               dict(sigma0=1e-3, sigma_model=0)):
        case = W.laplace(n=48, radius=12.0, width=4.0, rho_ratio=10.0, sigma=1e-3)
        case.update(kw)
        oc, g, f = _state(case)
        g, f = O.run(oc, g, f, 300)
        fl = O.fields(oc, g, f)
        y, x = np.mgrid[0:48, 0:48].astype(float)
        r = np.hypot(x - 24, y - 24)
        dps.append(fl["p"][r < 4].mean() - fl["p"][r > 20].mean())
    assert dps[0] == pytest.approx(dps[1], rel=1e-9)
    assert dps[0] / dps[2] == pytest.approx(factor, rel=0.01)


@pytest.mark.parametrize("width,tol", [(4.0, 0.07), (8.0, 0.02)])
def test_langmuir_marangoni_traction_of_flat_interface(width, tol):
    """Across a flat interface the tangential force integrates to d sigma/dx of the isotherm in
    the imposed psi(x) (Sec. 6.7 Eqs. surfacetensiongeometricsurfactantsxcomp, Langmuirisotherm);
    the derivative is taken by a central difference of sigma(psi(x))."""
    case = W.flat(nx=8, ny=64, width=width, mobility=0.05, rho_ratio=1.0, sigma=1e-3)
    case.update(sigma_model=1, beta=0.6, psi0=0.2, gradpsi_x=0.02, gradpsi_y=0.0)
    oc, g, f = _state(case)
    xn = 3
    col = [O.node_info(oc, g, f, xn, j) for j in range(case["ny"] // 2)]
    fsx = sum(c["Fsx"] for c in col)
    fsy = sum(c["Fsy"] for c in col)

    def sigma(x):
        return 1e-3 * (1.0 + 0.6 * math.log(1.0 - (0.2 + 0.02 * x)))

    h = 1e-4
    dsig_dx = (sigma(xn + h) - sigma(xn - h)) / (2 * h)
    assert fsx == pytest.approx(dsig_dx, rel=tol)
    assert abs(fsy) < 1e-9 * abs(dsig_dx)


# ---------------------------------------------------------------------------------------------
# Imposed shear flow (R17)
# ---------------------------------------------------------------------------------------------

def test_shear_flow_returns_circle_after_reversal():
    """Sec. 6.1: the circle is stretched by the shear and, with the field reversed at T_f,
    comes back to its initial shape at 2 T_f; the fluid populations are carried unchanged."""
    case = W.shear_circle(L0=64, u0=0.05)
    tf = case["meta"]["t_f"]
    oc, g0, f0 = _state(case)
    g1, f1 = O.run(oc, g0, f0, tf)
    oc.t = tf
    g2, f2 = O.run(oc, g1, f1, tf)
    phi0, phi1, phi2 = f0.sum(0), f1.sum(0), f2.sum(0)

    def rel(a, b):
        return np.linalg.norm(a - b) / np.linalg.norm(b)

    def area_mismatch(a, b):    # area of the symmetric difference of the phi > 1/2 regions
        return np.sum((a > 0.5) != (b > 0.5)) / np.sum(b > 0.5)

    assert area_mismatch(phi1, phi0) > 1.0    # stretched far from the circle at T_f
    assert area_mismatch(phi2, phi0) < 0.05   # back to it at 2 T_f (0.012 at L0 = 128)
    assert rel(phi2, phi0) < 0.15             # (0.071 at L0 = 128)
    assert abs(phi2.sum() - phi0.sum()) <= 1e-12 * phi0.sum()
    assert np.array_equal(g2, g0)


def test_shear_flow_velocity_reverses_at_the_reversal_step():
    """The velocity the step uses (reported by the fields) flips sign at reverse_step and is
    divergence-free, tangential to the box boundary in its normal component."""
    case = W.shear_circle(L0=32, u0=0.01)
    oc, g, f = _state(case)
    oc.t = case["reverse_step"] - 1
    a = O.fields(oc, g, f)
    oc.t = case["reverse_step"]
    b = O.fields(oc, g, f)
    assert np.array_equal(a["ux"], -b["ux"]) and np.array_equal(a["uy"], -b["uy"])
    assert np.abs(a["ux"][:, 0]).max() < 1e-15 and np.abs(a["uy"][0, :]).max() < 1e-15
    assert np.abs(a["ux"]).max() == pytest.approx(0.01 * math.pi, rel=1e-2)
    assert np.all(a["p"] == 0.0)


def test_shear_flow_step_is_interface_lattice_only():
    """Only f changes, and with u0 = 0 it changes exactly as the interface lattice of the
    coupled step does for a fluid at rest (a flat slab, equal densities, no surface tension:
    the coupled fluid stays at u = 0)."""
    case = W.shear_circle(L0=32, u0=0.0, reverse=False)
    case.update(mobility=0.02)
    y = np.mgrid[0:32, 0:32][0].astype(float)
    case["fields"]["phi"] = W.tanh_profile(np.minimum(y - 8, 24 - y), 3.0)
    oc, g, f = _state(case)
    g1, f1 = O.run(oc, g, f, 100)
    assert np.array_equal(g1, g)
    coupled = W.Case(case)
    coupled.update(flow=0, sigma0=0.0)
    occ, gc, fc = _state(coupled)
    gc, fc = O.run(occ, gc, fc, 100)
    assert np.abs(O.fields(occ, gc, fc)["ux"]).max() == 0.0
    assert np.array_equal(fc, f1)
    assert np.abs(f1.sum(0) - f.sum(0)).max() > 1e-6     # the slab profile did evolve
