"""Element-wise parity of the CUDA library with the FP64 oracle in the degenerate states of the
method and on the setups of the force-coupling pins.

* One phase only: grad phi = 0, so the interface normal is the regularised zero vector,
  theta = 4 phi (1 - phi) / W = 0, there is no surface force, and rho, mu are the pure-phase
  values (Sec. 2).  Phase B (phi = 0) carries no phase flux, so the fluid lattice alone
  evolves: a pressure wave in a uniform stream (the setup of the linear-mode pin of the
  -grad p* part of F_p, Sec. 3), and the same between no-slip or free-slip walls under gravity.
  Phase A (phi = 1) is tested where the flow stays divergence-free (a uniform stream is an
  exact fixed point; uniform acceleration by a body force has the closed form
  u(n) = (n + 1/2) F_ext / rho of the half-force-corrected velocity, Sec. 4 Eq.
  hydrodynamicfields): wherever compression pushes phi above 1, theta changes sign and the
  sharpening flux amplifies rounding differences (1e-15 grows to 1e-8 in 100 steps in the
  oracle itself), so element-wise parity there means nothing.
* A drop carried by a uniform stream (the setup of the Galilean-translation pin of the
  c_s^2 (rho_A - rho_B) grad phi part of F_p).
* A flat interface at rest with p = 0 and no forces: the flow stays at rest to rounding.

Tolerances as for the other parity tests: relative L2 <= 1e-12 in FP64, <= 2e-5 in FP32,
measured against the array's own norm or, where the exact array is zero up to rounding, an
absolute floor stated with the test.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_04166_gb300 import lbm
from paper_1909_04166_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}


def err(a, b, floor=0.0):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), floor * np.sqrt(b.size), 1e-300)


def compare(case, nsteps, precision, floors=None):
    """Run oracle and library from the same fields; compare populations and fields."""
    floors = floors or {}
    oc = O.OracleCase.from_dict(case.params)
    fl = case["fields"]
    g_ref, f_ref = O.init(oc, fl["phi"], fl["p"], fl["ux"], fl["uy"])
    g_ref, f_ref = O.run(oc, g_ref, f_ref, nsteps)
    ref = O.fields(oc, g_ref, f_ref)
    with lbm.Simulation(case, precision=precision) as sim:
        sim.init_case().step(nsteps)
        g, f = sim.populations()
        out = sim.fields()
    tol = TOL[precision]
    assert err(g, g_ref, floors.get("g", 0.0)) <= tol
    assert err(f, f_ref, floors.get("f", 0.0)) <= tol
    for k in ("phi", "p", "ux", "uy"):
        assert err(out[k], ref[k], floors.get(k, 0.0)) <= tol, k
    return out, ref


def single_phase(phase, nx=64, ny=6, U=0.1, wave=1e-5, ratio=1000.0):
    """phi = phase everywhere, a uniform stream (U, -0.3 U) and a pressure wave of amplitude
    `wave` along x; densities 1 and 1/ratio."""
    rho_b = 1.0 / ratio
    c = W._base(nx, ny, rho_a=1.0, rho_b=rho_b, mu_a=0.01, mu_b=0.01 * rho_b, sigma0=1e-3,
                mobility=0.02, width=4.0)
    _, x = np.mgrid[0:ny, 0:nx].astype(float)
    c["fields"] = dict(phi=np.full((ny, nx), float(phase)),
                       p=wave * np.cos(2 * np.pi * x / nx),
                       ux=np.full((ny, nx), U), uy=np.full((ny, nx), -0.3 * U))
    return c


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_phase_b_pressure_wave_in_a_stream_parity(precision):
    out, _ = compare(single_phase(0), 120, precision)
    assert np.all(out["phi"] == 0.0)          # no phase appears from nothing


@pytest.mark.parametrize("wall_y", [1, 2])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_phase_b_between_walls_under_gravity_parity(wall_y, precision):
    """No-slip (1) or free-slip (2) bottom and top, gravity along -y, a pressure wave along x:
    the hydrostatic adjustment runs through F_ext and both wall schemes with no interface."""
    case = single_phase(0, nx=40, ny=24, U=0.0)
    case.update(wall_y=wall_y, gy=-1e-3, rho_ref=0.0)
    out, _ = compare(case, 80, precision)
    assert np.all(out["phi"] == 0.0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_phase_a_uniform_stream_is_a_fixed_point(precision):
    """phi = 1, p = 0, uniform u: the equilibria are uniform, streaming moves equal values and
    every source term is zero, so the state does not change.  Floor for p, which is zero
    exactly; populations and u are compared with their own norms."""
    case = single_phase(1, wave=0.0)
    out, _ = compare(case, 50, precision, floors={"p": 1e-3})
    tol = 4e-15 if precision == "fp64" else 5e-7
    assert np.abs(out["phi"] - 1.0).max() <= tol
    assert np.abs(out["ux"] - 0.1).max() <= tol and np.abs(out["uy"] + 0.03).max() <= tol
    assert np.abs(out["p"]).max() <= tol


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_phase_a_uniform_acceleration(precision):
    """phi = 1 in a periodic box under a body force F = (rho - rho_ref) g: the corrected
    velocity after n steps is (n + 1/2) F / rho at every node (momentum n F from the sources,
    plus half a step's force in Eq. hydrodynamicfields) and the pressure stays uniform."""
    case = single_phase(1, nx=40, ny=24, U=0.0, wave=0.0)
    case.update(gy=-1e-5, rho_ref=0.25)
    n = 80
    out, _ = compare(case, n, precision, floors={"p": 1e-3, "ux": 1e-3})
    F_over_rho = (1.0 - 0.25) * -1e-5 / 1.0
    rel = 1e-13 if precision == "fp64" else 1e-5
    assert np.allclose(out["uy"], (n + 0.5) * F_over_rho, rtol=rel, atol=0)
    assert np.abs(out["ux"]).max() <= (1e-18 if precision == "fp64" else 1e-9)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("ratio", [10.0, 100.0])
def test_drop_in_uniform_stream_parity(ratio, precision):
    n = 48
    c = W._base(n, n, rho_a=1.0, rho_b=1.0 / ratio, mu_a=0.1, mu_b=0.1 / ratio, sigma0=1e-4,
                mobility=0.02, width=4.0)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    phi = W.tanh_profile(n / 4.8 - np.hypot(x - n / 2, y - n / 2), 4.0)
    c["fields"] = dict(phi=phi, p=np.zeros((n, n)), ux=np.full((n, n), 0.02),
                       uy=np.full((n, n), 0.01))
    compare(c, 150, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_flat_interface_at_rest_stays_at_rest(precision):
    """A flat interface at rest with p = 0, no gravity and no surface tension.  The fluid
    populations and the velocity are zero up to rounding (floor 1e-3 of the interface
    populations' scale); phi relaxes slightly (the tanh profile is the interface's equilibrium
    only up to lattice error), in the library as in the oracle."""
    case = W.flat(nx=8, ny=48, width=4.0, mobility=0.02, rho_ratio=100.0, sigma=0.0)
    out, _ = compare(case, 50, precision, floors={"g": 1e-3, "p": 1e-3, "ux": 1e-3,
                                                  "uy": 1e-3})
    tol = 1e-15 if precision == "fp64" else 1e-8
    assert np.abs(out["ux"]).max() <= tol and np.abs(out["uy"]).max() <= tol
