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

Coordinates: node (i, j) sits at x = i, y = j; arrays are ``(ny, nx)``.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["Case", "laplace", "rt", "marangoni", "impact", "layered", "flat", "random_drop",
           "ensemble", "tanh_profile"]


class Case(dict):
    """Physical parameters (keys of the problem statement) plus initial fields.

    Keys: nx, ny, wall_x, wall_y, rho_a, rho_b, mu_a, mu_b, sigma0, dsigma_dT, T0, gradT_x,
    gradT_y, mobility, width, gx, gy, rho_ref; and ``fields`` = dict(phi, p, ux, uy).
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
             mobility=0.02, width=4.0, gx=0.0, gy=0.0, rho_ref=0.0)
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
           reynolds=20.0, weber=8000.0, rho_ratio=1000.0, mu_ratio=10.0, width=5.0,
           mobility=0.02) -> Case:
    """Drop of diameter D moving down at speed U, initially touching a film of thickness
    film_frac D on the bottom wall (periodic x, walls y): mu_A = rho_A U D / Re,
    sigma = rho_A U^2 D / We, mu_B = mu_A / mu_ratio.

    The defaults take the paper's own drop-impact parameters (Sec. 6.6: density ratio 1000,
    viscosity ratio 10, We = 8000, U = 0.05, Re = 2 rho_A U R / mu_A = 20, W = 5) on a
    2048 x 1024 grid with D = 200 and a film of 0.1 D.  At Re >= 100 with this thin film the
    run diverges within a few hundred steps (air squeezed out at |u| > 0.3)."""
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
                nu_a=0.1, nu_b=0.1) -> Case:
    """A drop at a seeded position with a seeded random velocity field and pressure noise; used
    for element-wise parity on grids of any (ragged) shape and boundary combination."""
    rng = np.random.default_rng(seed)
    rho_b = 1.0 / rho_ratio
    c = _base(nx, ny, wall_x=bool(wall_x), wall_y=bool(wall_y), rho_a=1.0, rho_b=rho_b,
              mu_a=nu_a, mu_b=nu_b * rho_b, sigma0=sigma, dsigma_dT=marangoni, T0=0.0,
              gradT_x=0.01, gradT_y=0.005, mobility=mobility, width=width, gx=0.0,
              gy=-gravity, rho_ref=0.5 * (1.0 + rho_b))
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
