"""The paper's experiments (Secs. 6.1 and 6.3 - 7), run on the GPU through the C ABI.  (The
Laplace law of Sec. 6.2 is checked on the FP64 oracle in the tests.)

* ``e1``  circular interface in the imposed reversing shear flow (Sec. 6.1): shape error when it
  returns at 2 T_f, and the phase-mass drift.
* ``e3``  Rayleigh-Taylor instability (Sec. 6.3, Atwood 0.5, Re = 3000, 256 x 1024): positions
  of the bubble front and the spike tip against time.
* ``e4``  drop falling under gravity (Sec. 6.4, density ratio 5, Eo = 43): the drop's extent
  (width and height of phi > 1/2) and centroid at the paper's three Ohnesorge numbers; the
  paper finds less deformation at larger Oh and a bag with side tails at Oh = 0.3.
* ``e5``  bubble rising at density ratio 1000 and viscosity ratio 100 (Sec. 6.5, Re = 35): the
  bubble's extent and centroid at Eo = 10, 50, 125; the paper finds a flattened cap at low Eo
  and an elongating skirt with tails as Eo grows.
* ``e6``  drop impact on a thin film at density ratio 1000 (Sec. 6.6): the outcome at the
  paper's two Reynolds numbers, deposition at Re = 20 and an ejecta sheet at Re = 100, read
  off the height that liquid (phi > 1/2) reaches above the film outside the drop's footprint.
* ``e7``  Young's problem recast for a surfactant (Sec. 6.7): migration velocity of a neutrally
  buoyant drop in the imposed psi = psi0 + G y with the Langmuir isotherm, against the creeping-
  flow terminal velocity V = -sigma_Gamma G D / (6 mu_B + 9 mu_A), sigma_Gamma = -sigma0 beta,
  for the paper's three sensitivities sigma0 beta.
* ``e8``  numerical stability of the two collision models (Sec. 7): the smallest kinematic
  viscosity nu_A = nu_B at which the oscillating elliptic cylinder (kappa-tilde = 0.01) still runs
  stably, for the cascaded and the single-relaxation-time operators at density ratios 500, 600,
  800 and 900, on a grid of quarter decades in nu.

``python -m paper_1909_04166_gb300.experiments [e1|e3|e4|e5|e6|e7|e8|all]`` prints one JSON
line each.
"""
from __future__ import annotations

import json
import math
import sys
import time

import numpy as np

from . import lbm
from . import workloads as W


def _area_mismatch(a, b):
    return float(np.sum((a > 0.5) != (b > 0.5)) / np.sum(b > 0.5))


def e1(L0=200, u0=0.02, precision="fp32") -> dict:
    case = W.shear_circle(L0=L0, u0=u0)
    tf = case["meta"]["t_f"]
    phi0 = case["fields"]["phi"]
    t0 = time.perf_counter()
    with lbm.Simulation(case, precision=precision) as sim:
        sim.init_case()
        m0 = sim.diagnostics()["sum_phi"]
        sim.step(tf)
        mid = sim.fields()["phi"]
        sim.step(tf)
        end = sim.fields()["phi"]
        m1 = sim.diagnostics()["sum_phi"]
    return {"experiment": "e1 reversing shear (Sec. 6.1)", "L0": L0, "u0": u0, "T_f": tf,
            "precision": precision, "area_mismatch_at_Tf": round(_area_mismatch(mid, phi0), 4),
            "area_mismatch_at_2Tf": round(_area_mismatch(end, phi0), 5),
            "rel_l2_phi_at_2Tf": round(float(np.linalg.norm(end - phi0) /
                                             np.linalg.norm(phi0)), 5),
            "phase_mass_drift": float(abs(m1 - m0) / m0),
            "wall_s": round(time.perf_counter() - t0, 2)}


def e7(sens=(0.0048, 0.0146, 0.0244), steps=100000, sample=1000, precision="fp32",
       widths=(51,)) -> dict:
    """One row per sensitivity and box width (the paper's box is 51 wide; wider boxes show how
    much of the gap to the unbounded 3-D value is the periodic confinement)."""
    out = {"experiment": "e7 Young's problem, Langmuir isotherm (Sec. 6.7)", "steps": steps,
           "precision": precision, "cases": []}
    for nx, sb in [(w, s) for w in widths for s in sens]:
        case = W.young_drop(nx=nx, sigma0_beta=sb)
        meta = case["meta"]
        mu_a, mu_b = case["mu_a"], case["mu_b"]
        v_theory = -meta["sigma_gamma"] * meta["grad_psi"] * meta["diameter"] / (6 * mu_b
                                                                                 + 9 * mu_a)
        vs, ys = [], []
        with lbm.Simulation(case, precision=precision) as sim:
            sim.init_case()
            for k in range(steps // sample):
                sim.step(sample)
                fl = sim.fields()
                ph = np.clip(fl["phi"], 0.0, 1.0)
                vs.append(float((ph * fl["uy"]).sum() / ph.sum()))
                y = np.arange(case["ny"], dtype=float)[:, None]
                ys.append(float((ph * y).sum() / ph.sum()))
        tail = vs[len(vs) // 2:]
        out["cases"].append({
            "nx": nx, "sigma0_beta": sb, "v_theory": v_theory,
            "v_mean_second_half": float(np.mean(tail)),
            "ratio": float(np.mean(tail) / v_theory),
            "centroid_start_end": [round(ys[0], 3), round(ys[-1], 3)],
            "v_centroid_second_half": float((ys[-1] - ys[len(ys) // 2]) /
                                            (sample * (len(ys) - 1 - len(ys) // 2))),
        })
    return out


def _extent(phi):
    """Width and height of the region phi > 1/2, and its phi-weighted centroid height."""
    inside = phi > 0.5
    if not inside.any():
        return {"width": 0, "height": 0, "yc": float("nan")}
    rows, cols = np.nonzero(inside)
    y = np.arange(phi.shape[0], dtype=float)[:, None]
    return {"width": int(cols.max() - cols.min() + 1), "height": int(rows.max() - rows.min() + 1),
            "yc": round(float((phi * y).sum() / phi.sum()), 2)}


def _shape_history(case, steps, sample, precision, of_phase_b=False):
    rows = []
    with lbm.Simulation(case, precision=precision) as sim:
        sim.init_case()
        for k in range(steps // sample):
            sim.step(sample)
            phi = sim.fields()["phi"]
            rows.append({"t": (k + 1) * sample, **_extent(1.0 - phi if of_phase_b else phi)})
    return rows


def e3(steps=20000, sample=1600, precision="fp32") -> dict:
    """Heavy fluid over light, interface ny/2 + 0.1 nx cos(2 pi x / nx): the light fluid rises
    as a bubble at x = 0 and the heavy one falls as a spike at x = nx/2.  Positions relative to
    the initial mean interface in units of nx, time t* = t sqrt(g / nx) (6400 steps)."""
    case = W.rt()
    nx, ny = case["nx"], case["ny"]
    rows = []
    with lbm.Simulation(case, precision=precision) as sim:
        sim.init_case()
        for k in range(steps // sample):
            sim.step(sample)
            phi = sim.fields()["phi"]
            light_at_0 = np.nonzero(phi[:, 0] < 0.5)[0]
            heavy_at_mid = np.nonzero(phi[:, nx // 2] > 0.5)[0]
            t = (k + 1) * sample
            rows.append({"t": t, "t_star": round(t / 6400.0, 3),
                         "bubble": round((light_at_0.max() - ny / 2) / nx, 3),
                         "spike": round((heavy_at_mid.min() - ny / 2) / nx, 3)})
    return {"experiment": "e3 Rayleigh-Taylor instability (Sec. 6.3)", "steps": steps,
            "precision": precision, "history": rows}


def e4(ohnesorge=(0.3, 0.7, 1.0), steps=8000, sample=2000, precision="fp32") -> dict:
    """151 x 451, D = 30 at (75, 300), free-slip top and bottom, periodic sides, sigma = 1e-3
    (sets the scale; the time unit sqrt(D/g) is 709 steps)."""
    out = {"experiment": "e4 falling drop (Sec. 6.4)", "steps": steps, "precision": precision,
           "time_unit_steps": 709, "cases": []}
    for oh in ohnesorge:
        out["cases"].append({"Oh": oh, "history": _shape_history(W.falling_drop(ohnesorge=oh),
                                                                 steps, sample, precision)})
    return out


def e5(eotvos=(10.0, 50.0, 125.0), steps=9600, sample=1600, precision="fp32") -> dict:
    """161 x 481, D = 64, density ratio 1000, viscosity ratio 100, Re = 35, W = 5, U_g = 0.02
    (the time unit D / U_g is 3200 steps, so 9600 steps are t* = 3)."""
    out = {"experiment": "e5 rising bubble (Sec. 6.5)", "steps": steps, "precision": precision,
           "time_unit_steps": 3200, "cases": []}
    for eo in eotvos:
        case = W.rising_bubble(rho_ratio=1000.0, mu_ratio=100.0, eotvos=eo, width=5.0)
        out["cases"].append({"Eo": eo, "history": _shape_history(case, steps, sample, precision,
                                                                 of_phase_b=True)})
    return out


def _impact_shape(phi, film, xc, R):
    """Height above the film reached by liquid outside |x - xc| <= R (the ejecta), and the
    half-width of the liquid above the film (the spreading lamella)."""
    liquid = phi > 0.5
    ny, nx = phi.shape
    x = np.arange(nx)
    rows = np.arange(ny)[:, None]
    top = np.where(liquid, rows, -1).max(axis=0)              # highest liquid node per column
    outside = np.abs(x - xc) > R
    ejecta = float(max(top[outside].max() - film, 0.0))
    above = liquid[int(film) + 3]
    half_width = float(np.abs(x[above] - xc).max()) if above.any() else 0.0
    return ejecta, half_width


def e6(reynolds=(20.0, 100.0), steps=16000, sample=2000, precision="fp32") -> dict:
    """2048 x 1024 impact (D = 200, film 0.1 D, We = 8000, viscosity ratio 10, W = 5,
    M_phi = 0.1); the time unit is 2R/U = 4000 steps."""
    out = {"experiment": "e6 drop impact on a thin film (Sec. 6.6)", "steps": steps,
           "precision": precision, "time_unit_steps": 4000, "cases": []}
    for re_ in reynolds:
        case = W.impact(reynolds=re_)
        film, R, xc = 0.1 * 200.0, 100.0, case["nx"] / 2
        rows = []
        with lbm.Simulation(case, precision=precision) as sim:
            sim.init_case()
            for k in range(steps // sample):
                sim.step(sample)
                fl = sim.fields()
                ej, hw = _impact_shape(fl["phi"], film, xc, R)
                rows.append({"t": (k + 1) * sample, "ejecta_height": ej, "lamella_half_width": hw,
                             "max_speed": float(np.nanmax(np.hypot(fl["ux"], fl["uy"])))})
        out["cases"].append({"Re": re_, "history": rows,
                             "max_ejecta_height": max(r["ejecta_height"] for r in rows)})
    return out


def _stable(case, precision, steps, check, umax):
    """Run `steps` steps; unstable at the first checkpoint with a non-finite node or a speed
    above umax (the flow has left the low-Mach range the scheme is built for)."""
    with lbm.Simulation(case, precision=precision) as sim:
        sim.init_case()
        done, peak = 0, 0.0
        while done < steps:
            n = min(check, steps - done)
            sim.step(n)
            done += n
            d = sim.diagnostics()
            if d["nonfinite"] or not math.isfinite(d["max_speed"]) or d["max_speed"] > umax:
                return False, done, peak
            peak = max(peak, d["max_speed"])
    return True, done, peak


def _stable_batch(cases, precision, steps, check, umax):
    """_stable for many cases of one collision model advanced together in one batch (each case
    evolves bitwise as in its own context); returns (stable, steps run, peak speed) per case."""
    n = len(cases)
    ok, done, peak = [True] * n, [steps] * n, [0.0] * n
    with lbm.Batch(cases, precision=precision, layout=lbm.LBM_BATCH_AS_GIVEN) as b:
        b.init_all()
        t = 0
        while t < steps:
            k = min(check, steps - t)
            b.step(k)
            t += k
            for i, c in enumerate(cases):
                if not ok[i]:
                    continue
                shape = (int(c["ny"]), int(c["nx"]))
                p, ux, uy = np.empty(shape), np.empty(shape), np.empty(shape)
                lbm.lbm_batch_get_fields(b.b, i, None, p, ux, uy, None)
                speed = float(np.hypot(ux, uy).max())
                if not (np.isfinite(p).all() and math.isfinite(speed)) or speed > umax:
                    ok[i], done[i] = False, t
                else:
                    peak[i] = max(peak[i], speed)
    return list(zip(ok, done, peak))


def e8(ratios=(500.0, 600.0, 800.0, 900.0), steps=50000, check=2000, umax=0.1, nu_max=0.1,
       nu_min=1e-8, per_decade=4, precision="fp32") -> dict:
    """A run counts as stable when every checkpoint (each `check` steps, `steps` in all: about
    eight capillary oscillation periods) has finite fields and a largest speed <= umax.  Every
    viscosity of the grid runs (one batch per collision model holds all ratios and viscosities);
    per ratio and model the result gives the stability of each viscosity, the smallest stable
    viscosity above the first unstable one (the search of the paper, from large to small nu) and
    the smallest stable one anywhere on the grid."""
    nus = [nu_max * 10 ** (-k / per_decade)
           for k in range(int(round(per_decade * math.log10(nu_max / nu_min))) + 1)]
    out = {"experiment": "e8 minimum stable viscosity, oscillating cylinder (Sec. 7)",
           "steps": steps, "check_every": check, "max_speed_bound": umax, "kappa_tilde": 0.01,
           "precision": precision, "nu_grid": [float(f"{v:.4g}") for v in nus], "rows": []}
    t0 = time.perf_counter()
    runs = {}
    for model, col in (("cascaded", 0), ("srt", 1)):
        cases = [W.oscillating_cylinder(rho_ratio=ratio, nu=nu, collision=col)
                 for ratio in ratios for nu in nus]
        res = _stable_batch(cases, precision, steps, check, umax)
        for j, r in enumerate(res):
            runs[(model, ratios[j // len(nus)], j % len(nus))] = r
    for ratio in ratios:
        row = {"density_ratio": ratio}
        for model in ("cascaded", "srt"):
            res = [runs[(model, ratio, k)] for k in range(len(nus))]
            smallest, failed_at = None, None
            for nu, (ok, done, _) in zip(nus, res):     # decreasing nu
                if not ok:
                    failed_at = {"nu": float(f"{nu:.4g}"), "step": done}
                    break
                smallest = nu
            stable = [nu for nu, r in zip(nus, res) if r[0]]
            row[f"nu_min_{model}"] = None if smallest is None else float(f"{smallest:.4g}")
            row[f"first_unstable_{model}"] = failed_at
            row[f"nu_min_anywhere_{model}"] = float(f"{min(stable):.4g}") if stable else None
            row[f"stable_{model}"] = "".join("s" if r[0] else "u" for r in res)
        if row["nu_min_cascaded"] and row["nu_min_srt"]:
            row["srt_over_cascaded"] = row["nu_min_srt"] / row["nu_min_cascaded"]
        out["rows"].append(row)
    out["wall_s"] = round(time.perf_counter() - t0, 1)
    return out


def main(argv=None):
    which = (argv or sys.argv[1:] or ["all"])[0]
    for name, fn in (("e1", e1), ("e3", e3), ("e4", e4), ("e5", e5), ("e6", e6), ("e7", e7),
                     ("e8", e8)):
        if which in (name, "all"):
            print(json.dumps(fn()), flush=True)


if __name__ == "__main__":
    main()
