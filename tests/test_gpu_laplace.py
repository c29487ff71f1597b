"""The static-drop Laplace test of Sec. 6.2 on the GPU in FP64, at the configured size and
horizon: 64 x 64 periodic, drop radius 16 centred, density ratio 1000, kinematic viscosity 0.1 in
both phases, sigma = 1e-3, M_phi = 0.02, no gravity, u = 0, 2000 steps.  The interface width is
W = 5, the paper's own width for its ratio-1000 cases: with W = 4 this 64 x 64 case diverges
after about 450 steps in the FP64 oracle itself (the interface equilibrium undershoots phi < 0
along the diagonals, and the density jump across one node exceeds what the finite-difference
c_s^2 grad rho term of F_p balances).

Conditioning.  The pressure-based scheme is weakly compressible, and at density ratio 1000 the
drop's core is compressed so that phi departs from 1 by up to ~5e-4.  Where phi sits slightly
below 1 with small gradients, the sharpening flux M_phi theta n of the interface lattice is
anti-diffusive (theta exceeds the regularisation of n), so grid-scale differences grow: in the
FP64 oracle itself a 2^-52 relative change of the initial populations reaches 1e-13 after about
30 steps and saturates near 1e-7 (phi) / 1e-5 (g-bar) after a few hundred.  The library's FP64
arithmetic (fused multiply-adds, another evaluation order) differs from the oracle's by a few
ulps per step, so element-wise agreement is gated at 1e-12 or twenty times the oracle's own
one-ulp spread at the same step, whichever is larger (the spread is measured in the test).

* After 20 steps (the spread is far below 1e-12 for phi and f) and after 2000 steps, the
  library's FP64 state and fields match the oracle's under that rule.
* After 2000 steps the pressure jump dp (mean p inside r < R - 2W minus mean p outside
  r > R + 2W, from the library's FP64 diagnostics) matches sigma / R_eff times the discrete
  surface factor of the sampled tanh profile within 1.5 % (as the oracle's own Laplace pin), and
  the phase mass sum(phi) is conserved to rounding.
"""
import numpy as np
import pytest

import _conditioning as C
from paper_1909_04166_gb300 import lbm
from paper_1909_04166_gb300 import workloads as W
from test_oracle_physics import discrete_surface_factor

pytestmark = pytest.mark.gpu

SIGMA, RADIUS, WIDTH = 1e-3, 16.0, 5.0
CHECKS = (20, 2000)


@pytest.fixture(scope="module")
def laplace_runs():
    case = W.laplace(n=64, radius=RADIUS, width=WIDTH, rho_ratio=1000.0, sigma=SIGMA)
    orc = C.ulp_spread(case, CHECKS)
    got, t = {}, 0
    with lbm.Simulation(case, precision="fp64") as sim:
        sim.init_case()
        d0 = sim.diagnostics()
        for c in CHECKS:
            sim.step(c - t)
            t = c
            g, f = sim.populations()
            got[c] = dict(sim.fields(), g=g, f=f)
        d1 = sim.diagnostics(32.0, 32.0, RADIUS - 2 * WIDTH, RADIUS + 2 * WIDTH)
    return dict(case=case, ref=orc["ref"], spread=orc["spread"], got=got, d0=d0, d1=d1)


@pytest.mark.parametrize("nsteps", CHECKS)
def test_fp64_state_matches_the_oracle(laplace_runs, nsteps):
    r = laplace_runs
    ref, got, spread = r["ref"][nsteps], r["got"][nsteps], r["spread"][nsteps]
    for k in ("g", "f") + C.FIELDS:
        tol = max(1e-12, 20.0 * spread[k])
        assert C.rel_l2(got[k], ref[k]) <= tol, (k, C.rel_l2(got[k], ref[k]), spread[k])
    if nsteps == CHECKS[0]:   # before the growth sets in: the strict gate, element by element
        for k in ("f", "phi"):
            assert spread[k] < 1e-14
            assert np.abs(got[k] - ref[k]).max() <= 1e-12 * np.abs(ref[k]).max(), k


def test_pressure_jump_follows_the_laplace_law(laplace_runs):
    r = laplace_runs
    r_eff = np.sqrt(r["d1"]["sum_phi"] / np.pi)
    expect = SIGMA * discrete_surface_factor(WIDTH) / r_eff
    assert r["d1"]["dp_laplace"] == pytest.approx(expect, rel=0.015)
    # the device diagnostic is the oracle's definition evaluated on the library's fields
    n = r["case"]["nx"]
    y, x = np.mgrid[0:n, 0:n].astype(float)
    rr = np.hypot(x - n / 2, y - n / 2)
    p = r["got"][CHECKS[-1]]["p"]
    dp_host = p[rr < RADIUS - 2 * WIDTH].mean() - p[rr > RADIUS + 2 * WIDTH].mean()
    assert r["d1"]["dp_laplace"] == pytest.approx(dp_host, rel=1e-12)
    # and the oracle's own jump agrees with the library's to the conditioning of p
    p_ref = r["ref"][CHECKS[-1]]["p"]
    dp_ref = p_ref[rr < RADIUS - 2 * WIDTH].mean() - p_ref[rr > RADIUS + 2 * WIDTH].mean()
    assert dp_host == pytest.approx(dp_ref, rel=1e-4)


def test_phase_mass_is_conserved(laplace_runs):
    r = laplace_runs
    m0, m1 = r["d0"]["sum_phi"], r["d1"]["sum_phi"]
    assert abs(m1 - m0) <= 1e-13 * m0
    assert m1 == pytest.approx(r["ref"][CHECKS[-1]]["phi"].sum(), rel=1e-13)
