"""The paper's experimental findings, reproduced by the CUDA library (FP32) as regression checks.

Each test runs one of paper_1909_04166_gb300.experiments and asserts the qualitative outcome
the paper reports (Secs. 6.3 - 7); the numbers they print are recorded in the design notes.
The reversing shear flow (Sec. 6.1) is checked in test_gpu_next.py, the Laplace law (Sec. 6.2)
on the oracle.
"""
import pytest

from paper_1909_04166_gb300 import experiments as E
from paper_1909_04166_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_rayleigh_taylor_spike_outruns_the_bubble():
    """Sec. 6.3, Atwood 0.5: the light fluid rises as a bubble and the heavy one falls as a
    spike, both steadily; at Atwood 0.5 the spike is the faster of the two."""
    h = E.e3(steps=19200, sample=3200)["history"]
    bubble = [r["bubble"] for r in h]
    spike = [r["spike"] for r in h]
    assert all(b2 > b1 for b1, b2 in zip(bubble, bubble[1:]))
    assert all(s2 < s1 for s1, s2 in zip(spike, spike[1:]))
    assert -spike[-1] > 1.3 * bubble[-1] > 0.6


def test_falling_drop_deforms_less_at_larger_ohnesorge():
    """Sec. 6.4: at Oh = 0.3 the drop becomes a bag with side tails; at Oh = 0.7 and 1.0 it
    flattens, the less the larger Oh."""
    cases = E.e4(steps=8000, sample=8000)["cases"]
    end = {c["Oh"]: c["history"][-1] for c in cases}
    assert end[0.3]["width"] > end[0.7]["width"] > end[1.0]["width"]
    assert end[0.3]["height"] > 3 * end[0.7]["height"]          # the trailing tails
    assert end[0.7]["height"] < 30 and end[1.0]["height"] < 30    # flattened (D = 30)


def test_rising_bubble_grows_a_skirt_with_eotvos():
    """Sec. 6.5, density ratio 1000: at Eo = 10 the bubble flattens into a cap; as Eo grows its
    rear stretches into a skirt with tails, so its height grows with Eo."""
    cases = E.e5(steps=9600, sample=9600)["cases"]
    h = {c["Eo"]: c["history"][-1] for c in cases}
    assert h[10.0]["height"] < 50 < h[50.0]["height"] < h[125.0]["height"]
    for c in h.values():
        assert c["yc"] > 170.0                                      # it rose (from y = 120)


def test_drop_impact_deposits_at_re20_and_splashes_at_re100():
    """Sec. 6.6, density ratio 1000: at Re = 20 the drop merges with the film and the flow
    dies out; at Re = 100 an ejecta sheet keeps rising."""
    cases = {c["Re"]: c["history"] for c in E.e6(steps=16000, sample=4000)["cases"]}
    low, high = cases[20.0], cases[100.0]
    assert low[-1]["max_speed"] < 0.05 * 0.05 and low[-1]["ejecta_height"] < 80
    ej = [r["ejecta_height"] for r in high]
    assert all(b > a for a, b in zip(ej, ej[1:])) and ej[-1] > 250
    assert high[-1]["max_speed"] > 0.5 * 0.05


def test_cascaded_operator_runs_where_single_relaxation_time_fails():
    """Sec. 7, oscillating cylinder at density ratio 900: the cascaded operators run stably at
    a viscosity the single-relaxation-time ones cannot reach (the paper's factor is above 55)."""
    ok_cascaded, _, _ = E._stable(W.oscillating_cylinder(rho_ratio=900.0, nu=3e-4, collision=0),
                                  "fp32", 20000, 2000, 0.1)
    ok_srt, _, _ = E._stable(W.oscillating_cylinder(rho_ratio=900.0, nu=1e-2, collision=1),
                             "fp32", 20000, 2000, 0.1)
    assert ok_cascaded and not ok_srt


def test_batched_stability_check_agrees_with_single_runs():
    """The E8 sweep advances all its viscosities in one batch; each case must reach the same
    verdict, at the same checkpoint, as when it runs alone."""
    cases = [W.oscillating_cylinder(rho_ratio=900.0, nu=nu, collision=1) for nu in (1e-2, 5e-2)]
    batched = E._stable_batch(cases, "fp32", 6000, 2000, 0.1)
    for c, (ok, done, peak) in zip(cases, batched):
        ok1, done1, peak1 = E._stable(c, "fp32", 6000, 2000, 0.1)
        assert (ok, done) == (ok1, done1)
        assert abs(peak - peak1) <= 1e-12 * max(peak1, 1e-300)
    assert not batched[0][0]          # SRT at nu = 0.01 fails (Sec. 7)
