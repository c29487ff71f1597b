"""Parity at the benchmark's full size and over long horizons.

* One step at the bench workload (2048 x 1024 drop impact, density ratio 1000, default launch as
  bench.py times it): GPU vs the FP64 oracle stepping the same state, element by element.
* 100 and 1000 steps on the Marangoni drop (512 x 256, density ratio 10), Rayleigh-Taylor
  (256 x 1024, Atwood 0.5) and the impact, against the FP64 oracle.  The step map amplifies
  perturbations (tests/_conditioning.py): a 2^-52 change of the oracle's initial state grows to
  3e-5 within 100 steps on Rayleigh-Taylor and saturates near 1.5e-3 by 1000, so a fixed
  element-wise tolerance cannot hold there for any implementation that rounds differently.  The
  gates are therefore set by what rounding alone does in the oracle, measured in the test:
    - FP32: the FP64 oracle with its populations rounded to float32 after every step (FP32
      storage, FP64 arithmetic) and, where it is larger, its one-ulp spread.  The FP32 step also
      rounds its arithmetic: every population passes through about ten roundings at its own
      scale per step (zeroth-moment sums, the interface collision's moments and their inverse,
      the fluid source terms) against one for storage.  On the well-conditioned Marangoni drop
      the FP32 deviation is 5 - 13 times the storage-alone deviation; evaluating the interface
      collision in double about halves it, the fluid collision or the forces in double change it
      by under 15 % (measured with variants of the kernel that evaluate one part in double, not
      part of the library).  The gate is max(2e-5, 16 x that reference).
    - FP64: 1e-12, or twenty times the oracle's one-ulp spread where that is larger (the
      library's fused multiply-adds and evaluation order differ from the oracle's by a few ulps
      per step).
* Strict FP32 gate on a well-conditioned case: phi and p within 2e-5 after 1000 steps.
"""
import numpy as np
import pytest

import _conditioning as C
from oracle import oracle as O
from paper_1909_04166_gb300 import lbm
from paper_1909_04166_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CHECKS = (100, 1000)
FP32_FACTOR = 16.0
FP64_FACTOR = 20.0


def rel_l2(a, b):
    return C.rel_l2(a, b)


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
    # every node, element by element, against the scale of each lattice
    assert np.abs(g1 - g_ref).max() <= (1e-13 if prec == "fp64" else 1e-6) * np.abs(g_ref).max()
    assert np.abs(f1 - f_ref).max() <= (1e-13 if prec == "fp64" else 1e-6) * np.abs(f_ref).max()


_REFS = {}


def references(name):
    """The oracle's plain FP64 fields at CHECKS, the float32-storage deviation and (except for
    the impact, where it costs another minute of host time and the storage deviation is of the
    same size) the one-ulp spread; computed once per case."""
    if name not in _REFS:
        case = C.CASES[name]()
        if name == "impact":
            ref = C.oracle_series(case, CHECKS, "fp64")
            ulp = None
        else:
            u = C.ulp_spread(case, CHECKS, seeds=(0,))
            ref, ulp = u["ref"], u["spread"]
        stor = C.deviations(C.oracle_series(case, CHECKS, "float_storage"), ref)
        _REFS[name] = (case, ref, stor, ulp)
    return _REFS[name]


@pytest.mark.parametrize("name", ["marangoni", "rt", "impact"])
def test_fp32_horizon_within_rounding_conditioning(name):
    case, ref, stor, ulp = references(name)
    got = C.deviations(C.gpu_series(case, "fp32", CHECKS), ref)
    for c in CHECKS:
        for k in C.FIELDS:
            floor = max(stor[c][k], ulp[c][k] if ulp else 0.0)
            assert got[c][k] <= max(2e-5, FP32_FACTOR * floor), (c, k, got[c][k], floor)


@pytest.mark.parametrize("name", ["marangoni", "rt"])
def test_fp64_horizon_within_ulp_spread(name):
    case, ref, _, ulp = references(name)
    got = C.deviations(C.gpu_series(case, "fp64", CHECKS), ref)
    for c in CHECKS:
        for k in C.FIELDS:
            assert got[c][k] <= max(1e-12, FP64_FACTOR * ulp[c][k]), (c, k, got[c][k], ulp[c][k])


def test_fp32_strict_gate_on_a_well_conditioned_case():
    """Marangoni drop (density ratio 10): phi and p of the FP32 path within 2e-5 relative L2 of
    the FP64 oracle after 1000 steps."""
    _, ref, _, _ = references("marangoni")
    got = C.gpu_series(C.CASES["marangoni"](), "fp32", (1000,))
    for k in ("phi", "p"):
        assert rel_l2(got[1000][k], ref[1000][k]) <= 2e-5, k
