"""Physics pins of the FP64 oracle (CPU): closed-form or textbook results the whole step must
reproduce.  Laplace law for a static drop (Sec. 6.2), the tanh equilibrium interface profile
(Sec. 2 Eq. hyperbolictangentprofile), layered two-phase Poiseuille flow (viscosity
interpolation, Eq. fluidviscosity, body force, walls), diffusion at the mobility M_phi (Sec. 5),
the integrated Marangoni traction of a flat interface (Sec. 6.7), Galilean translation of a
drop and the linear modes of a pressure wave in a uniform stream (the two parts of the net
gradient pressure force F_p, Sec. 3), and the symmetry of the whole step under the diagonal
reflection x <-> y (the D2Q9 lattice and the moment bases of Secs. 3 and 5).
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_1909_04166_gb300 import workloads as W


def discrete_surface_factor(width, offset=0.0):
    """Sum over nodes of (central-difference d phi/d zeta)^2 across a sampled tanh profile,
    divided by its continuum value 2/(3W): the discrete surface-energy factor that multiplies
    sigma in kappa-tilde = (3/2) sigma W on the lattice."""
    z = np.arange(-80, 81) + offset
    phi = W.tanh_profile(z, width)
    d = 0.5 * (phi[2:] - phi[:-2])
    return float(np.sum(d * d) / (2.0 / (3.0 * width)))


def run_case(case, nsteps):
    oc = O.OracleCase.from_dict(case.params)
    fl = case["fields"]
    g, f = O.init(oc, fl["phi"], fl["p"], fl["ux"], fl["uy"])
    g, f = O.run(oc, g, f, nsteps)
    return oc, g, f, O.fields(oc, g, f)


def laplace_dp(case, fields):
    n = case["nx"]
    y, x = np.mgrid[0:n, 0:n].astype(float)
    r = np.hypot(x - n / 2, y - n / 2)
    R, Wd = case["meta"]["radius"], case["width"]
    return fields["p"][r < R - 2 * Wd].mean() - fields["p"][r > R + 2 * Wd].mean()


@pytest.mark.parametrize("ratio,width", [(1000.0, 5.0), (10.0, 4.0)])
def test_laplace_law(ratio, width):
    sigma = 1e-3
    case = W.laplace(n=64, radius=16.0, width=width, rho_ratio=ratio, sigma=sigma)
    oc, g, f, fl = run_case(case, 3000)
    assert np.isfinite(fl["p"]).all()
    dp = laplace_dp(case, fl)
    r_eff = np.sqrt(fl["phi"].sum() / np.pi)
    expect = sigma * discrete_surface_factor(width) / r_eff
    assert dp == pytest.approx(expect, rel=0.015)
    # spurious currents stay small next to the capillary velocity sigma / mu
    assert np.hypot(fl["ux"], fl["uy"]).max() < 0.1 * sigma / case["mu_a"]


def test_laplace_pressure_is_linear_in_sigma():
    dps = []
    for sigma in (5e-4, 1e-3, 2e-3):
        case = W.laplace(n=48, radius=12.0, width=5.0, rho_ratio=100.0, sigma=sigma)
        _, _, _, fl = run_case(case, 2000)
        dps.append(laplace_dp(case, fl))
    assert dps[1] / dps[0] == pytest.approx(2.0, rel=0.01)
    assert dps[2] / dps[1] == pytest.approx(2.0, rel=0.01)


def test_flat_interface_keeps_tanh_profile():
    """The tanh profile is the interface's equilibrium up to the second-order lattice error:
    the steady deviation falls like 1/W^2 and the slab stays at rest."""
    errs = []
    for width in (4.0, 8.0):
        case = W.flat(nx=4, ny=int(16 * width), width=width, mobility=0.05, rho_ratio=10.0)
        _, _, _, fl = run_case(case, 2000)
        errs.append(np.abs(fl["phi"] - case["fields"]["phi"]).max())
        assert errs[-1] < 0.11 / width ** 2
        assert np.hypot(fl["ux"], fl["uy"]).max() < 1e-7
    assert 3.0 < errs[0] / errs[1] < 5.0


def _layered_reference(case):
    """Steady u(y) of d/dy (mu(y) du/dy) = -F between walls at y = -1/2 and ny - 1/2, with
    mu(y) = mu_B + phi(y) (mu_A - mu_B) and phi the tanh profile of the initial interface."""
    ny = case["ny"]
    F = case["gx"] * case["rho_a"]
    yi = (ny - 1) / 2.0
    mu = lambda s: case["mu_b"] + W.tanh_profile(yi - s, case["width"]) * (case["mu_a"]
                                                                            - case["mu_b"])
    a, b = -0.5, ny - 0.5
    i1 = integrate.quad(lambda s: 1.0 / mu(s), a, b, limit=200)[0]
    i2 = integrate.quad(lambda s: s / mu(s), a, b, limit=200)[0]
    y0 = i2 / i1
    return np.array([-F * integrate.quad(lambda s: (s - y0) / mu(s), a, yy, limit=200)[0]
                     for yy in range(ny)])


@pytest.mark.parametrize("mu_b", [0.1, 0.025])
def test_layered_poiseuille(mu_b):
    case = W.layered(nx=4, ny=32, mu_a=0.1, mu_b=mu_b, force=1e-6, width=4.0)
    _, _, _, fl = run_case(case, 30000)
    u = fl["ux"].mean(axis=1)
    ref = _layered_reference(case)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 0.01
    assert np.abs(fl["uy"]).max() < 1e-3 * np.abs(ref).max()


def test_phase_field_diffuses_at_the_mobility():
    """With equal densities, no surface tension and a very wide interface (theta -> 0) the
    interface lattice solves d phi/dt = M_phi lap phi: a Gaussian's variance grows by 2 M_phi t
    per axis."""
    n, s0, M, t = 64, 4.0, 0.05, 200
    case = W.flat(nx=n, ny=n, width=1e9, mobility=M, rho_ratio=1.0, sigma=0.0)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    bump = 0.1 * np.exp(-((x - n / 2) ** 2 + (y - n / 2) ** 2) / (2 * s0 * s0))
    case["fields"]["phi"] = 0.5 + bump
    _, _, _, fl = run_case(case, t)
    d = fl["phi"] - 0.5
    var_x = np.sum(d * (x - n / 2) ** 2) / np.sum(d)
    assert (var_x - s0 * s0) / (2 * t) == pytest.approx(M, rel=0.01)


@pytest.mark.parametrize("width,tol", [(4.0, 0.07), (8.0, 0.02)])
def test_marangoni_traction_of_flat_interface(width, tol):
    """Across a flat interface the tangential surface force integrates to the surface gradient
    of sigma (Sec. 6.7 Eq. surfacetensiongeometricsurfactantsxcomp); the normal one to zero."""
    case = W.flat(nx=8, ny=64, width=width, mobility=0.05, rho_ratio=1.0, sigma=1e-3)
    case.update(dsigma_dT=-2e-6, gradT_x=0.01)
    oc = O.OracleCase.from_dict(case.params)
    fl = case["fields"]
    g, f = O.init(oc, fl["phi"], fl["p"], fl["ux"], fl["uy"])
    col = [O.node_info(oc, g, f, 3, j) for j in range(case["ny"] // 2)]   # lower interface
    fsx = sum(c["Fsx"] for c in col)
    fsy = sum(c["Fsy"] for c in col)
    dsig_dx = case["dsigma_dT"] * case["gradT_x"]
    assert fsx == pytest.approx(dsig_dx, rel=tol)
    assert abs(fsy) < 1e-9 * abs(dsig_dx)


def _periodic_centroid(phi):
    ny, nx = phi.shape
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    out = []
    for coord, L in ((x, nx), (y, ny)):
        th = 2 * np.pi * coord / L
        a = np.arctan2((phi * np.sin(th)).sum(), (phi * np.cos(th)).sum())
        out.append((a % (2 * np.pi)) * L / (2 * np.pi))
    return np.array(out)


@pytest.mark.parametrize("ratio", [10.0, 100.0])
def test_drop_translates_with_a_uniform_flow(ratio):
    """Galilean invariance: a drop in a uniform stream U (periodic box, no gravity, weak sigma)
    is carried along at U and the stream stays uniform.  With a density contrast the
    c_s^2 (rho_A - rho_B) grad phi part of F_p (Sec. 3 Eq. netgradientpressureforce, reading R7)
    is what keeps the momentum of the heavy and light phases consistent with the pressure
    evolution: without it the drop lags at half the speed (ratio 10) or the run diverges
    (ratio 100)."""
    n, steps, U = 48, 400, np.array([0.02, 0.01])
    y, x = np.mgrid[0:n, 0:n].astype(float)
    oc = O.OracleCase(nx=n, ny=n, rho_a=1.0, rho_b=1.0 / ratio, mu_a=0.1, mu_b=0.1 / ratio,
                      sigma0=1e-4, mobility=0.02, width=4.0)
    phi0 = W.tanh_profile(n / 4.8 - np.hypot(x - n / 2, y - n / 2), 4.0)
    g, f = O.init(oc, phi0, np.zeros((n, n)), np.full((n, n), U[0]), np.full((n, n), U[1]))
    g, f = O.run(oc, g, f, steps)
    fl = O.fields(oc, g, f)
    assert np.isfinite(fl["p"]).all()
    shift = _periodic_centroid(fl["phi"]) - _periodic_centroid(phi0)
    assert np.allclose(shift, U * steps, rtol=0.02)
    du = np.hypot(fl["ux"] - U[0], fl["uy"] - U[1]).max()
    assert du < (0.15 if ratio < 50 else 0.75) * np.hypot(*U)


@pytest.mark.parametrize("U", [0.05, 0.1])
def test_pressure_wave_in_a_uniform_stream_follows_the_linear_modes(U):
    """Uniform density, uniform stream U along x, a small standing pressure wave p' = eps cos kx.
    The zeroth and first moments of the modified Boltzmann equation (Sec. 3: p = sum g,
    sum g e = rho c_s^2 u, Gamma^p_00 = F_p . u with F_p = -grad psi) give, linearised,
    d_t p' + U d_x p' = -rho c_s^2 d_x u' and d_t u' + 2 U d_x u' = -d_x p' / rho (the momentum
    flux rho u u is conservative with rho fixed by phi).  So the modes are
    omega = k (3U/2 +- sqrt(c_s^2 + U^2/4)), with amplitudes set by u'(0) = 0.  The -grad p*
    part of F_p is what advects p (reading R7): the complex amplitude of the k-mode of p
    follows the two modes in phase to 0.05 rad; with that part dropped or of the other sign the
    phase is off by 0.2 - 0.45 rad at t = 100."""
    nx, ny, eps = 64, 2, 1e-5
    oc = O.OracleCase(nx=nx, ny=ny, rho_a=1.0, rho_b=1.0, mu_a=0.01, mu_b=0.01, sigma0=0.0,
                      mobility=0.02, width=4.0)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    k = 2 * np.pi / nx
    g, f = O.init(oc, np.ones((ny, nx)), eps * np.cos(k * x), np.full((ny, nx), U),
                  np.zeros((ny, nx)))
    s = np.sqrt(1.0 / 3.0 + U * U / 4)
    w_plus, w_minus = k * (1.5 * U + s), k * (1.5 * U - s)
    # p'(0) = eps, u'(0) = 0: A+ (U/2 + s) + A- (U/2 - s) = 0, A+ + A- = 1
    a_minus = (0.5 * U + s) / (2 * s)
    a_plus = 1.0 - a_minus
    t = 0
    for t_check in (50, 100):
        g, f = O.run(oc, g, f, t_check - t)
        t = t_check
        a = (O.fields(oc, g, f)["p"] * np.exp(-1j * k * x)).mean() * 2 / eps
        pred = a_plus * np.exp(-1j * w_plus * t) + a_minus * np.exp(-1j * w_minus * t)
        assert abs(np.angle(a / pred)) < 0.05, (t, np.angle(a / pred))
        assert 0.85 < abs(a) / abs(pred) <= 1.0   # viscous and bulk damping only


@pytest.mark.parametrize("rho_ref", [0.0, 0.25])
def test_uniform_body_force_accelerates_at_the_closed_form(rho_ref):
    """One phase in a periodic box under F = (rho - rho_ref) g (Sec. 3): nothing varies in
    space, so every node's momentum grows by F per step and the corrected velocity of Sec. 4
    Eq. hydrodynamicfields, (sum g-bar e + c_s^2 F / 2) / (rho c_s^2), is (n + 1/2) F / rho
    after n steps, with the pressure uniform; a uniform stream with no force stays as it is."""
    n, nx, ny, g = 60, 12, 10, 2e-5
    oc = O.OracleCase(nx=nx, ny=ny, rho_a=1.0, rho_b=0.1, mu_a=0.05, mu_b=0.005,
                      sigma0=1e-3, gx=0.3 * g, gy=-g, rho_ref=rho_ref)
    ones, zeros = np.ones((ny, nx)), np.zeros((ny, nx))
    g0, f0 = O.init(oc, ones, zeros, zeros, zeros)
    fl = O.fields(oc, *O.run(oc, g0, f0, n))
    F = (1.0 - rho_ref) * np.array([0.3 * g, -g])
    assert np.allclose(fl["ux"], (n + 0.5) * F[0], rtol=1e-12, atol=0)
    assert np.allclose(fl["uy"], (n + 0.5) * F[1], rtol=1e-12, atol=0)
    assert np.ptp(fl["p"]) <= 1e-15 and np.abs(fl["phi"] - 1.0).max() <= 1e-14
    oc2 = O.OracleCase(nx=nx, ny=ny, rho_a=1.0, rho_b=0.1, mu_a=0.05, mu_b=0.005)
    g1, f1 = O.init(oc2, ones, zeros, np.full((ny, nx), 0.07), np.full((ny, nx), -0.02))
    g2, f2 = O.run(oc2, g1, f1, n)
    assert np.allclose(g2, g1, rtol=0, atol=1e-16) and np.allclose(f2, f1, rtol=0, atol=1e-16)


DIAGONAL = [0, 2, 1, 4, 3, 5, 8, 7, 6]   # population index under the reflection x <-> y


def _reflected(case):
    """The same problem seen across the diagonal: every x quantity becomes the y one."""
    d = dict(case.params)
    for a, b in (("nx", "ny"), ("wall_x", "wall_y"), ("wall_x_hi", "wall_y_hi"),
                 ("gradT_x", "gradT_y"), ("gx", "gy"), ("gradpsi_x", "gradpsi_y")):
        d[a], d[b] = case.get(b), case.get(a)
    d = {k: v for k, v in d.items() if v is not None}
    fl = case["fields"]
    return d, (fl["phi"].T, fl["p"].T, fl["uy"].T, fl["ux"].T)


@pytest.mark.parametrize("extra", [
    dict(wall_x=1, wall_x_hi=2, wall_y=0, gravity=1e-6, marangoni=-2e-5, rho_ratio=100.0),
    dict(wall_x=2, wall_y=1, wall_y_hi=2, gravity=2e-6, rho_ratio=10.0, collision=1),
    dict(wall_x=0, wall_y=1, rho_ratio=30.0, sigma_model=1, beta=0.5, psi0=0.2,
         gradpsi_x=8e-4, gradpsi_y=-3e-4),
])
def test_step_is_equivariant_under_the_diagonal_reflection(extra):
    """The D2Q9 lattice, its isotropic stencils and the moment bases of Secs. 3 and 5 are
    symmetric under the reflection x <-> y (directions 1 <-> 2, 3 <-> 4, 6 <-> 8; the
    relaxation rates of each pair of swapped moments are equal), so stepping the reflected
    problem must give the reflected populations up to rounding.  A term with a wrong index or
    sign in only one of the two axes breaks this."""
    kw = dict(extra)
    gravity, marangoni, ratio = kw.pop("gravity", 0.0), kw.pop("marangoni", 0.0), kw.pop("rho_ratio")
    wx, wy = kw.pop("wall_x"), kw.pop("wall_y")
    case = W.random_drop(23, 37, seed=11, wall_x=wx, wall_y=wy, rho_ratio=ratio, gravity=gravity,
                         marangoni=marangoni, **kw)
    case["gx"] = 0.4 * case["gy"]                  # a force along both axes
    _, g, f, _ = run_case(case, 20)
    d, fields = _reflected(case)
    oc = O.OracleCase.from_dict(d)
    gr, fr = O.run(oc, *O.init(oc, *fields), 20)
    g_back = gr[DIAGONAL].transpose(0, 2, 1)
    f_back = fr[DIAGONAL].transpose(0, 2, 1)
    assert np.linalg.norm(g_back - g) <= 1e-12 * np.linalg.norm(g)
    assert np.linalg.norm(f_back - f) <= 1e-12 * np.linalg.norm(f)
    assert np.linalg.norm(g - g[:, :, ::-1]) > 1e-3 * np.linalg.norm(g)   # not trivially symmetric


# ---------------------------------------------------------------------------------------------
# Reading R6: the regularised interface normal n = grad phi / (|grad phi| + eps), eps = 1e-6.
# Sec. 2 defines n = grad phi / |grad phi| and leaves it undefined where grad phi vanishes.  Two
# pins bracket eps: inside a bulk phase the conservative Allen-Cahn equation has no interface to
# sharpen (theta = 4 phi (1 - phi)/W ~ 0) and reduces to the diffusion equation
# d phi/dt = M_phi lap phi, which must hold for rounding-sized departures of phi from 0 or 1
# (rejects eps below ~4e-7: the sharpening flux M theta n then acts on the noise at a fixed
# magnitude and amplifies it); and the flat tanh profile of Sec. 2 must stay the interface's
# equilibrium (rejects eps above ~1e-4: |n| < 1 in the profile's tails shifts the balance).
# ---------------------------------------------------------------------------------------------
def bulk_mode_decay(phi0, nsteps=500, n=32, amp=1e-10):
    """Amplitude ratio after nsteps of a sine mode of phi (wavelength n) riding on a uniform
    bulk value phi0, and the largest departure from a pure sine relative to amp."""
    x = np.arange(n)
    mode = np.sin(2.0 * np.pi * x / n)
    phi = np.tile(phi0 + amp * mode, (4, 1))
    oc = O.OracleCase(nx=n, ny=4, rho_a=1.0, rho_b=0.001, mu_a=0.1, mu_b=1e-4, sigma0=1e-3,
                      mobility=0.02, width=4.0)
    g, f = O.run(oc, *O.init(oc, phi, 0.0, 0.0, 0.0), nsteps)
    row = O.fields(oc, g, f)["phi"][0]
    d = row - row.mean()
    a = 2.0 * float(np.dot(d, mode)) / n
    return a / amp, float(np.abs(d - a * mode).max()) / amp


@pytest.mark.parametrize("phi0", [1.0 - 5e-8, 5e-8])
def test_bulk_phase_noise_diffuses_at_the_mobility(phi0):
    """R6 pin (lower side): a 1e-10 sine mode in a bulk phase 5e-8 away from phi_A or phi_B
    decays like the diffusion equation's exp(-M_phi k^2 t) (3 %, the lattice and the residual
    theta / eps = 0.05 of the regularisation) and stays a sine mode."""
    nsteps, n, M = 500, 32, 0.02
    ratio, resid = bulk_mode_decay(phi0, nsteps, n)
    k = 2.0 * np.pi / n
    assert ratio == pytest.approx(np.exp(-M * k * k * nsteps), rel=0.03)
    assert resid < 1e-3


def test_normal_regularisation_pins_reject_other_eps():
    """The two R6 pins fail for an eps far from 1e-6: with 1e-9 or the cut-off 1e-24 the bulk
    mode grows instead of decaying; with 1e-3 the flat interface leaves its tanh profile."""
    default = O.normal_eps()
    assert default == 1e-6
    try:
        for eps in (1e-24, 1e-9):
            O.set_normal_eps(eps)
            ratio, _ = bulk_mode_decay(1.0 - 5e-8)
            assert abs(ratio) > 5.0, eps
        O.set_normal_eps(1e-3)
        width = 8.0
        case = W.flat(nx=4, ny=int(16 * width), width=width, mobility=0.05, rho_ratio=10.0)
        _, _, _, fl = run_case(case, 2000)
        assert np.abs(fl["phi"] - case["fields"]["phi"]).max() > 0.11 / width ** 2
    finally:
        O.set_normal_eps(default)
