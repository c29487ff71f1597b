"""How far an FP32 run can stay from the FP64 one on a given workload: the FP32 path's deviation
from FP64 over a horizon, set beside what FP32 *storage* rounding alone does.

Test infrastructure (used by tests/test_gpu_fullsize.py and tests/test_gpu_laplace.py).  The
step map of the method amplifies perturbations (where phi leaves [0, 1], theta = 4 phi (1 - phi)
/ W changes sign and the sharpening flux acts on small gradients; the impact flow itself is
sensitive), so the deviation of an FP32 run from the FP64 one after N steps is set by the
workload's conditioning, not only by the kernel.  The references here are:

* ``float_storage``: the FP64 oracle with its state rounded to float32 on entry and after every
  step (``oracle.run_float_storage``): every operation in FP64, only the storage rounding of an
  FP32 implementation.  No FP32 implementation can avoid that rounding, so its deviation from
  the FP64 run is a floor for any FP32 path that stores FP32 populations;
* ``rounded_start``: the FP64 oracle from the float32-rounded initial state, rounded once only:
  how the map amplifies a single storage rounding.

Run as a script to print, per checkpoint, the four deviations side by side (one GPU and the host
cores):

    python tests/_conditioning.py [impact rt marangoni]
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle as O                       # noqa: E402
from paper_1909_04166_gb300 import lbm                # noqa: E402
from paper_1909_04166_gb300 import workloads as W     # noqa: E402

FIELDS = ("phi", "p", "ux", "uy")
CHECKPOINTS = (100, 250, 500, 1000)
CASES = {"impact": W.impact, "rt": W.rt, "marangoni": W.marangoni}


def rel_l2(a, b) -> float:
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def oracle_series(case, checkpoints=CHECKPOINTS, mode="fp64") -> dict:
    """Oracle fields at each checkpoint.  mode: "fp64" (plain), "float_storage" (state rounded
    to float32 after every step) or "rounded_start" (initial state rounded to float32 once)."""
    oc = O.OracleCase.from_dict(case.params)
    fl = case["fields"]
    g, f = O.init(oc, fl["phi"], fl["p"], fl["ux"], fl["uy"])
    if mode == "rounded_start":
        g = g.astype(np.float32).astype(np.float64)
        f = f.astype(np.float32).astype(np.float64)
    out, t = {}, 0
    for c in checkpoints:
        if mode == "float_storage":
            g, f = O.run_float_storage(oc, g, f, c - t)
        else:
            g, f = O.run(oc, g, f, c - t)
        t = c
        out[c] = O.fields(oc, g, f)
    return out


def ulp_spread(case, checkpoints, seeds=(0, 1, 2)) -> dict:
    """The oracle's own response to a one-ulp change of its initial state: for each checkpoint,
    the largest relative L2 deviation (fields and populations g, f) over runs whose initial
    populations carry i.i.d. relative noise of 2^-52 (seeded), from the plain run."""
    oc = O.OracleCase.from_dict(case.params)
    fl = case["fields"]
    g0, f0 = O.init(oc, fl["phi"], fl["p"], fl["ux"], fl["uy"])

    def series(g, f):
        out, t = {}, 0
        for c in checkpoints:
            g, f = O.run(oc, g, f, c - t)
            t = c
            out[c] = dict(O.fields(oc, g, f), g=g, f=f)
        return out

    ref = series(g0, f0)
    worst = {c: dict.fromkeys(FIELDS + ("g", "f"), 0.0) for c in checkpoints}
    for s in seeds:
        rng = np.random.default_rng(s)
        run = series(g0 * (1 + 2.0 ** -52 * rng.standard_normal(g0.shape)),
                     f0 * (1 + 2.0 ** -52 * rng.standard_normal(f0.shape)))
        for c in checkpoints:
            for k in worst[c]:
                worst[c][k] = max(worst[c][k], rel_l2(run[c][k], ref[c][k]))
    return {"ref": ref, "spread": worst}


def gpu_series(case, precision, checkpoints=CHECKPOINTS) -> dict:
    """Library fields at each checkpoint (the default launch, graph replays as lbm_step issues
    them)."""
    out, t = {}, 0
    with lbm.Simulation(case, precision=precision) as sim:
        sim.init_case()
        for c in checkpoints:
            sim.step(c - t)
            t = c
            out[c] = sim.fields()
    return out


def deviations(series: dict, ref: dict) -> dict:
    """{checkpoint: {field: relative L2 against ref}}."""
    return {c: {k: rel_l2(series[c][k], ref[c][k]) for k in FIELDS} for c in ref}


def table(name: str, checkpoints=CHECKPOINTS) -> list[str]:
    case = CASES[name]()
    t0 = time.perf_counter()
    ref = oracle_series(case, checkpoints, "fp64")
    stor = deviations(oracle_series(case, checkpoints, "float_storage"), ref)
    once = deviations(oracle_series(case, checkpoints, "rounded_start"), ref)
    gpu = deviations(gpu_series(case, "fp32", checkpoints), ref)
    g64 = deviations(gpu_series(case, "fp64", checkpoints), ref)
    lines = [f"## {case['name']} ({case['nx']} x {case['ny']}; oracle on "
             f"{O.num_threads()} threads, {time.perf_counter() - t0:.0f} s)",
             "| steps | field | FP32 library | FP32 storage alone | one rounding at t = 0 | "
             "FP64 library |", "|---|---|---|---|---|---|"]
    for c in checkpoints:
        for k in FIELDS:
            lines.append(f"| {c} | {k} | {gpu[c][k]:.2e} | {stor[c][k]:.2e} | "
                         f"{once[c][k]:.2e} | {g64[c][k]:.2e} |")
    return lines


if __name__ == "__main__":
    names = sys.argv[1:] or list(CASES)
    for n in names:
        print("\n".join(table(n)), flush=True)
        print(flush=True)
