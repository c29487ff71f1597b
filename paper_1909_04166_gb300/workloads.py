"""Seeded synthetic inputs for the paper's benchmark setups.

This module builds initial nodal fields (phi, p, ux, uy) and the physical parameters of each
case.  It holds none of the method's arithmetic (no equilibria, moments, collisions or
stencils): both the CUDA library and the FP64 oracle take their inputs from here and derive
everything else on their own.

Cases (sizes and parameters from the paper's problem statements, Secs. 6.2-6.7, scaled to the
workloads named in the package documentation):

* ``laplace``   static drop in a periodic box (Sec. 6.2).
* ``rt``        Rayleigh-Taylor instability, periodic in x, walls in y (Sec. 6.3).
* ``marangoni`` thermocapillary drop migration, sigma linear in a prescribed T (Sec. 6.7).
* ``impact``    drop impact on a thin film at density ratio 1000 (Sec. 6.6).
* ``layered``   two-layer Poiseuille channel (a closed-form check, not a paper figure).
* ``flat``      flat interface at rest (tanh-profile check).
* ``random_drop`` a drop with a seeded random velocity perturbation (parity cases).
* ``shear_circle`` circular interface in the imposed reversing shear flow (Sec. 6.1).
* ``falling_drop`` drop falling under gravity between free-slip walls (Sec. 6.4).
* ``rising_bubble`` bubble rising between free-slip sides and no-slip ends (Sec. 6.5).
* ``young_drop`` neutrally buoyant drop in an imposed surfactant gradient, Langmuir isotherm
  (Young's problem, Sec. 6.7).
* ``oscillating_cylinder`` elliptic liquid cylinder oscillating under capillarity (Sec. 7).

Coordinates: node (i, j) sits at x = i, y = j; arrays are ``(ny, nx)``.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["Case", "laplace", "rt", "marangoni", "impact", "layered", "flat", "random_drop",
           "shear_circle", "falling_drop", "rising_bubble", "young_drop", "oscillating_cylinder",
           "ensemble", "tanh_profile"]


class Case(dict):
    """Physical parameters (keys of the problem statement) plus initial fields.

    Keys: nx, ny, wall_x, wall_y, rho_a, rho_b, mu_a, mu_b, sigma0, dsigma_dT, T0, gradT_x,
    gradT_y, mobility, width, gx, gy, rho_ref, collision, sigma_model, beta, psi0, gradpsi_x,
    gradpsi_y, flow, reverse_step, u0, optionally wall_x_hi / wall_y_hi; and ``fields`` =
    dict(phi, p, ux, uy).  Boundary kinds: 0 (or False) periodic, 1 (or True) no-slip, 2
    free-slip; wall_x / wall_y set both sides of an axis, wall_x_hi / wall_y_hi the right / top
    side when it differs.  collision: 0 cascaded, 1 single relaxation time.  sigma_model: 0
    sigma linear in T, 1 Langmuir isotherm in psi = psi0 + gradpsi . x.  flow: 0 coupled
    lattices, 1 interface lattice alone in the imposed shear flow (amplitude u0, reversed from
    time level reverse_step on).
    """

    @property
    def params(self) -> dict:
        return {k: v for k, v in self.items() if k not in ("fields", "name", "meta")}

    @property
    def nodes(self) -> int:
        return int(self["nx"]) * int(self["ny"])


def _base(nx, ny, **kw) -> Case:
    c = Case(nx=int(nx), ny=int(ny), wall_x=False, wall_y=False, rho_a=1.0, rho_b=1.0,
             mu_a=0.1, mu_b=0.1, sigma0=0.0, dsigma_dT=0.0, T0=0.0, gradT_x=0.0, gradT_y=0.0,
             mobility=0.02, width=4.0, gx=0.0, gy=0.0, rho_ref=0.0, collision=0, sigma_model=0,
             beta=0.0, psi0=0.0, gradpsi_x=0.0, gradpsi_y=0.0, flow=0, reverse_step=0, u0=0.0)
    c.update(kw)
    return c


def tanh_profile(zeta, width):
    """The equilibrium phase-field profile across an interface (Sec. 2), phi_A = 1, phi_B = 0:
    phi = 1/2 + 1/2 tanh(2 zeta / W), zeta the signed distance into phase A."""
    return 0.5 + 0.5 * np.tanh(2.0 * np.asarray(zeta, dtype=np.float64) / width)


def _grid(nx, ny):
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    return x, y


def laplace(n=64, radius=16.0, width=5.0, rho_ratio=1000.0, nu=0.1, sigma=1e-3,
            mobility=0.02) -> Case:
    """Static drop of phase A (rho = 1) of radius R centred in an n x n periodic box."""
    rho_b = 1.0 / rho_ratio
    c = _base(n, n, rho_a=1.0, rho_b=rho_b, mu_a=nu, mu_b=nu * rho_b, sigma0=sigma,
              mobility=mobility, width=width)
    x, y = _grid(n, n)
    r = np.hypot(x - n / 2, y - n / 2)
    phi = tanh_profile(radius - r, width)
    c["fields"] = dict(phi=phi, p=np.zeros_like(phi), ux=np.zeros_like(phi),
                       uy=np.zeros_like(phi))
    c["name"] = f"laplace_{n}x{n}_R{radius:g}_W{width:g}_ratio{rho_ratio:g}"
    c["meta"] = dict(radius=radius, centre=(n / 2, n / 2))
    return c


def rt(nx=256, ny=1024, atwood=0.5, reynolds=3000.0, width=5.0, sigma=5e-5, mobility=0.1,
       amp_frac=0.1, uc=0.04) -> Case:
    """Heavy (phi = 1) over light fluid, interface y = ny/2 + amp nx cos(2 pi x / nx);
    gravity from U_c = sqrt(nx g) and nu = U_c nx / Re in both phases."""
    rho_a = 1.0
    rho_b = rho_a * (1.0 - atwood) / (1.0 + atwood)
    g = uc * uc / nx
    nu = uc * nx / reynolds
    c = _base(nx, ny, wall_y=True, rho_a=rho_a, rho_b=rho_b, mu_a=nu * rho_a, mu_b=nu * rho_b,
              sigma0=sigma, mobility=mobility, width=width, gx=0.0, gy=-g,
              rho_ref=0.5 * (rho_a + rho_b))
    x, y = _grid(nx, ny)
    yi = ny / 2 + amp_frac * nx * np.cos(2 * np.pi * x / nx)
    phi = tanh_profile(y - yi, width)
    c["fields"] = dict(phi=phi, p=np.zeros_like(phi), ux=np.zeros_like(phi),
                       uy=np.zeros_like(phi))
    c["name"] = f"rt_{nx}x{ny}"
    return c


def marangoni(nx=512, ny=256, radius=32.0, rho_ratio=10.0, nu_a=0.05, sigma0=1e-3,
              dsigma_dT=-2e-6, gradT=0.01, width=4.0, mobility=0.02) -> Case:
    """Drop in a channel (periodic x, walls y) under sigma(T) = sigma0 + dsigma/dT (T - T0),
    T = T0 + gradT x; equal dynamic viscosities (viscosity ratio 1)."""
    rho_b = 1.0 / rho_ratio
    mu = nu_a * 1.0
    c = _base(nx, ny, wall_y=True, rho_a=1.0, rho_b=rho_b, mu_a=mu, mu_b=mu, sigma0=sigma0,
              dsigma_dT=dsigma_dT, T0=0.0, gradT_x=gradT, mobility=mobility, width=width)
    x, y = _grid(nx, ny)
    r = np.hypot(x - nx / 2, y - ny / 2)
    phi = tanh_profile(radius - r, width)
    c["fields"] = dict(phi=phi, p=np.zeros_like(phi), ux=np.zeros_like(phi),
                       uy=np.zeros_like(phi))
    c["name"] = f"marangoni_{nx}x{ny}"
    return c


def impact(nx=2048, ny=1024, diameter=200.0, film_frac=0.1, gap=0.0, velocity=0.05,
           reynolds=100.0, weber=8000.0, rho_ratio=1000.0, mu_ratio=10.0, width=5.0,
           mobility=0.1) -> Case:
    """Drop of diameter D moving down at speed U, initially touching a film of thickness
    film_frac D on the bottom wall (periodic x, walls y): mu_A = rho_A U D / Re,
    sigma = rho_A U^2 D / We, mu_B = mu_A / mu_ratio.

    The defaults take the paper's own drop-impact parameters (Sec. 6.6: density ratio 1000,
    viscosity ratio 10, We = 8000, U = 0.05, W = 5, and the higher of its two Reynolds numbers,
    Re = 2 rho_A U R / mu_A = 100, the case that forms an ejecta sheet) on a 2048 x 1024 grid
    with D = 200 and a film of 0.1 D.  The paper gives no mobility for this case: M_phi = 0.1
    runs stably (0.05 - 0.2 do; 0.02 diverges within 1000 steps at Re = 100).  Re >= 150
    diverges within 500 steps for every mobility in 0.02 - 0.5 and width 5 - 8."""
    rho_a, rho_b = 1.0, 1.0 / rho_ratio
    mu_a = rho_a * velocity * diameter / reynolds
    sigma = rho_a * velocity ** 2 * diameter / weber
    c = _base(nx, ny, wall_y=True, rho_a=rho_a, rho_b=rho_b, mu_a=mu_a, mu_b=mu_a / mu_ratio,
              sigma0=sigma, mobility=mobility, width=width)
    x, y = _grid(nx, ny)
    h = film_frac * diameter
    R = diameter / 2
    yc = h + R + gap
    phi_film = tanh_profile(h - y, width)
    phi_drop = tanh_profile(R - np.hypot(x - nx / 2, y - yc), width)
    phi = np.maximum(phi_film, phi_drop)
    c["fields"] = dict(phi=phi, p=np.zeros_like(phi), ux=np.zeros_like(phi),
                       uy=-velocity * phi_drop)
    c["name"] = f"impact_{nx}x{ny}_Re{reynolds:g}"
    return c


def layered(nx=4, ny=32, mu_a=0.1, mu_b=0.05, rho=1.0, force=1e-6, width=4.0,
            mobility=0.02) -> Case:
    """Channel with walls in y, phase A in the lower half, phase B above, equal densities,
    driven by a uniform body force F = rho g along x (rho_ref = 0)."""
    c = _base(nx, ny, wall_y=True, rho_a=rho, rho_b=rho, mu_a=mu_a, mu_b=mu_b, sigma0=0.0,
              mobility=mobility, width=width, gx=force / rho, gy=0.0, rho_ref=0.0)
    x, y = _grid(nx, ny)
    phi = tanh_profile((ny - 1) / 2.0 - y, width)
    c["fields"] = dict(phi=phi, p=np.zeros_like(phi), ux=np.zeros_like(phi),
                       uy=np.zeros_like(phi))
    c["name"] = f"layered_{nx}x{ny}"
    return c


def flat(nx=4, ny=64, width=4.0, mobility=0.02, rho_ratio=1.0, sigma=1e-3) -> Case:
    """Periodic slab of phase A between y = ny/4 and 3 ny/4, at rest."""
    rho_b = 1.0 / rho_ratio
    c = _base(nx, ny, rho_a=1.0, rho_b=rho_b, mu_a=0.1, mu_b=0.1 * rho_b, sigma0=sigma,
              mobility=mobility, width=width)
    x, y = _grid(nx, ny)
    d = np.minimum(y - ny / 4, 3 * ny / 4 - y)
    phi = tanh_profile(d, width)
    c["fields"] = dict(phi=phi, p=np.zeros_like(phi), ux=np.zeros_like(phi),
                       uy=np.zeros_like(phi))
    c["name"] = f"flat_{nx}x{ny}"
    return c


def random_drop(nx, ny, seed=0, wall_x=False, wall_y=False, rho_ratio=10.0, sigma=1e-3,
                width=4.0, mobility=0.05, amp=1e-3, gravity=0.0, marangoni=0.0,
                nu_a=0.1, nu_b=0.1, **extra) -> Case:
    """A drop at a seeded position with a seeded random velocity field and pressure noise; used
    for element-wise parity on grids of any (ragged) shape and boundary combination.  ``extra``
    sets further case keys (wall_x_hi, collision, sigma_model, beta, psi0, gradpsi_x, ...)."""
    rng = np.random.default_rng(seed)
    rho_b = 1.0 / rho_ratio
    c = _base(nx, ny, wall_x=int(wall_x), wall_y=int(wall_y), rho_a=1.0, rho_b=rho_b,
              mu_a=nu_a, mu_b=nu_b * rho_b, sigma0=sigma, dsigma_dT=marangoni, T0=0.0,
              gradT_x=0.01, gradT_y=0.005, mobility=mobility, width=width, gx=0.0,
              gy=-gravity, rho_ref=0.5 * (1.0 + rho_b))
    c.update(extra)
    x, y = _grid(nx, ny)
    R = max(1.5, 0.3 * min(nx, ny))
    xc = nx * rng.uniform(0.35, 0.65)
    yc = ny * rng.uniform(0.35, 0.65)
    phi = tanh_profile(R - np.hypot(x - xc, y - yc), width)
    c["fields"] = dict(phi=phi,
                       p=amp * 0.1 * rng.standard_normal((ny, nx)),
                       ux=amp * rng.standard_normal((ny, nx)),
                       uy=amp * rng.standard_normal((ny, nx)))
    c["name"] = f"random_drop_{nx}x{ny}_s{seed}"
    return c


def shear_circle(L0=200, u0=0.02, peclet=60.0, width=3.0, radius_frac=0.2, yc_frac=0.3,
                 reverse=True) -> Case:
    """Sec. 6.1: a circle of radius L0/5 centred at (L0/2, 3 L0/10) in a periodic L0 x L0 box,
    advected by the imposed single-vortex shear of amplitude U_0, reversed at T_f = L0 / U_0 so
    that it should return to its start at 2 T_f; W = 3 and M_phi = U_0 W / Pe with Pe = 60."""
    tf = int(round(L0 / u0)) if u0 else 0
    c = _base(L0, L0, mobility=u0 * width / peclet, width=width, flow=1, u0=u0,
              reverse_step=tf if reverse else 0)
    x, y = _grid(L0, L0)
    R = radius_frac * L0
    phi = tanh_profile(R - np.hypot(x - L0 / 2, y - yc_frac * L0), width)
    c["fields"] = dict(phi=phi, p=np.zeros_like(phi), ux=np.zeros_like(phi),
                       uy=np.zeros_like(phi))
    c["name"] = f"shear_circle_{L0}"
    c["meta"] = dict(t_f=tf)
    return c


def falling_drop(nx=151, ny=451, diameter=30.0, centre=(75.0, 300.0), rho_ratio=5.0, eotvos=43.0,
                 ohnesorge=0.3, sigma=1e-3, width=4.0, mobility=0.02) -> Case:
    """Sec. 6.4: drop of phase A falling under F_ext = -(rho - rho_B) g j, free-slip walls at
    top and bottom, periodic sides; Eo = g (rho_A - rho_B) D^2 / sigma, Oh = mu_A /
    sqrt(rho_A D sigma), nu_A = nu_B.  sigma (not given in the paper) sets the scale."""
    rho_a, rho_b = 1.0, 1.0 / rho_ratio
    mu_a = ohnesorge * math.sqrt(rho_a * diameter * sigma)
    nu = mu_a / rho_a
    g = eotvos * sigma / ((rho_a - rho_b) * diameter ** 2)
    c = _base(nx, ny, wall_y=2, rho_a=rho_a, rho_b=rho_b, mu_a=mu_a, mu_b=nu * rho_b,
              sigma0=sigma, mobility=mobility, width=width, gy=-g, rho_ref=rho_b)
    x, y = _grid(nx, ny)
    phi = tanh_profile(diameter / 2 - np.hypot(x - centre[0], y - centre[1]), width)
    c["fields"] = dict(phi=phi, p=np.zeros_like(phi), ux=np.zeros_like(phi),
                       uy=np.zeros_like(phi))
    c["name"] = f"falling_drop_{nx}x{ny}"
    return c


def rising_bubble(nx=161, ny=481, diameter=64.0, centre=(80.0, 120.0), rho_ratio=10.0,
                  mu_ratio=10.0, reynolds=35.0, eotvos=10.0, ug=0.02, width=4.0,
                  mobility=0.02) -> Case:
    """Sec. 6.5: bubble of phase B in liquid A, F_ext = -(rho - rho_A) g j, free-slip sides
    and no-slip top and bottom; U_g = sqrt(g D), Re = rho_A U_g D / mu_A, Eo = rho_A U_g^2 D /
    sigma.  U_g (not given) sets the lattice velocity scale."""
    rho_a, rho_b = 1.0, 1.0 / rho_ratio
    g = ug * ug / diameter
    mu_a = rho_a * ug * diameter / reynolds
    sigma = rho_a * ug * ug * diameter / eotvos
    c = _base(nx, ny, wall_x=2, wall_y=1, rho_a=rho_a, rho_b=rho_b, mu_a=mu_a,
              mu_b=mu_a / mu_ratio, sigma0=sigma, mobility=mobility, width=width, gy=-g,
              rho_ref=rho_a)
    x, y = _grid(nx, ny)
    phi = tanh_profile(np.hypot(x - centre[0], y - centre[1]) - diameter / 2, width)
    c["fields"] = dict(phi=phi, p=np.zeros_like(phi), ux=np.zeros_like(phi),
                       uy=np.zeros_like(phi))
    c["name"] = f"rising_bubble_{nx}x{ny}"
    return c


def young_drop(nx=51, ny=201, diameter=30.0, yc=45.0, nu=0.05, grad_psi=9.95e-5,
               sigma0_beta=0.0244, beta=5.0, psi0=0.0, width=4.0, mobility=0.02) -> Case:
    """Sec. 6.7, Young's problem recast for a surfactant: a neutrally buoyant drop (density and
    viscosity ratio 1) near the bottom of a channel (periodic x, no-slip y) in the imposed
    psi = psi0 + G y with the Langmuir isotherm sigma = sigma0 [1 + beta ln(1 - psi)].  The
    paper gives sigma0 beta and G; beta (hence sigma0) and psi0 are not given.  beta = 5 keeps
    sigma0 small (1e-3 .. 5e-3): with beta = 1/2 (sigma0 up to 0.05) the capillary part's
    discretisation noise swamps the slow migration."""
    sigma0 = sigma0_beta / beta
    c = _base(nx, ny, wall_y=1, rho_a=1.0, rho_b=1.0, mu_a=nu, mu_b=nu, sigma0=sigma0,
              mobility=mobility, width=width, sigma_model=1, beta=beta, psi0=psi0,
              gradpsi_x=0.0, gradpsi_y=grad_psi)
    x, y = _grid(nx, ny)
    phi = tanh_profile(diameter / 2 - np.hypot(x - nx // 2, y - yc), width)
    c["fields"] = dict(phi=phi, p=np.zeros_like(phi), ux=np.zeros_like(phi),
                       uy=np.zeros_like(phi))
    c["name"] = f"young_{nx}x{ny}"
    c["meta"] = dict(diameter=diameter, sigma_gamma=-sigma0_beta, grad_psi=grad_psi)
    return c


def oscillating_cylinder(n=200, a=25.0, b=15.0, kappa=0.01, rho_ratio=100.0, nu=0.01,
                         width=5.0, mobility=0.02, collision=0) -> Case:
    """Sec. 7: elliptic liquid cylinder (semi-axes a, b) of phase A in a periodic n x n box,
    released at rest; kappa-tilde = 3/2 sigma W given, nu_A = nu_B."""
    rho_b = 1.0 / rho_ratio
    sigma = kappa / (1.5 * width)
    c = _base(n, n, rho_a=1.0, rho_b=rho_b, mu_a=nu, mu_b=nu * rho_b, sigma0=sigma,
              mobility=mobility, width=width, collision=collision)
    x, y = _grid(n, n)
    dx, dy = x - n / 2, y - n / 2
    r = (np.hypot(dx / a, dy / b) - 1.0) * min(a, b)
    phi = tanh_profile(-r, width)
    c["fields"] = dict(phi=phi, p=np.zeros_like(phi), ux=np.zeros_like(phi),
                       uy=np.zeros_like(phi))
    c["name"] = f"cylinder_{n}_ratio{rho_ratio:g}_nu{nu:g}"
    return c


def ensemble(ncases=512, seed0=1000, side_min=32, side_max=256, nu=0.1, mobility=0.02,
             width=5.0) -> list:
    """Independent static and oscillating drops of uneven sizes: case i draws its grid, radius,
    density ratio (log-uniform 10..1000), sigma (log-uniform 1e-4..1e-2) and a 1 % random
    velocity perturbation from seed seed0 + i; even cases are circles, odd ones 5:3 ellipses.
    W = 5: with W = 4 the density-ratio-1000 cases diverge."""
    cases = []
    for i in range(ncases):
        rng = np.random.default_rng(seed0 + i)
        nx = int(rng.integers(side_min, side_max + 1))
        ny = int(rng.integers(side_min, side_max + 1))
        R = float(rng.uniform(0.2, 0.35)) * min(nx, ny)
        ratio = float(math.exp(rng.uniform(math.log(10.0), math.log(1000.0))))
        sigma = float(math.exp(rng.uniform(math.log(1e-4), math.log(1e-2))))
        rho_b = 1.0 / ratio
        c = _base(nx, ny, rho_a=1.0, rho_b=rho_b, mu_a=nu, mu_b=nu * rho_b, sigma0=sigma,
                  mobility=mobility, width=width)
        x, y = _grid(nx, ny)
        dx, dy = x - nx / 2, y - ny / 2
        if i % 2 == 0:
            r = np.hypot(dx, dy) - R
        else:   # ellipse with axes ratio 5:3 and the area of the circle of radius R
            a, b = R * math.sqrt(5 / 3), R * math.sqrt(3 / 5)
            r = (np.hypot(dx / a, dy / b) - 1.0) * min(a, b)
        phi = tanh_profile(-r, width)
        ucap = math.sqrt(sigma / (1.0 * R))
        amp = 0.01 * ucap
        c["fields"] = dict(phi=phi, p=np.zeros_like(phi),
                           ux=amp * rng.standard_normal((ny, nx)),
                           uy=amp * rng.standard_normal((ny, nx)))
        c["name"] = f"ensemble_{i}"
        cases.append(c)
    return cases
