"""Batched stepping (lbm_batch_*): one launch per step over many independent cases.

Each case must evolve as in its own context: bitwise when stored as given (the batched kernel
runs the per-node arithmetic of the single-grid step), to rounding when stored transposed (the
reflected problem evaluates its sums in the reflected order); match the FP64 oracle, with its
fields and populations returned in its own orientation; and survive the autotuner bit for bit
(within one kernel the launch shape does not change any result)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_04166_gb300 import lbm
from paper_1909_04166_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def mixed_cases():
    return [
        W.random_drop(40, 33, seed=1, wall_y=True, rho_ratio=100.0, gravity=1e-6),
        W.random_drop(97, 64, seed=2, wall_x=True, rho_ratio=10.0, marangoni=-2e-5),
        W.random_drop(17, 120, seed=3, rho_ratio=1000.0, width=5.0),
        W.random_drop(1, 9, seed=4, wall_y=True),
        W.random_drop(64, 64, seed=5, wall_x=True, wall_y=True, rho_ratio=50.0),
        W.random_drop(129, 31, seed=6, rho_ratio=300.0, width=5.0),
    ]


# cases stored transposed under the fewest-columns layout: strips of 64 columns with FP32
# arithmetic, 32 in FP64
TRANSPOSED = {"fp32": [1, 2, 3], "fp16": [1, 2, 3], "fp64": [1, 2, 3, 5]}


# Bound on a transposed case against its own context after 37 steps: rounding level in FP32 /
# FP64; in FP16 storage a last-bit difference before encoding flips a 16-bit rounding, so the
# two runs differ by up to about the FP16 unit roundoff 2^-11 = 4.9e-4 (2.7e-4 measured)
@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp64", 1e-14), ("fp16", 1e-3)])
def test_batch_cases_match_their_own_contexts(prec, tol):
    cases = mixed_cases()
    got = {}
    for layout in (lbm.LBM_BATCH_AS_GIVEN, lbm.LBM_BATCH_FEWEST_COLUMNS):
        with lbm.Batch(cases, precision=prec, layout=layout) as b:
            tr = [i for i in range(len(cases)) if b.transposed(i)]
            assert tr == ([] if layout == lbm.LBM_BATCH_AS_GIVEN else TRANSPOSED[prec])
            b.init_all().step(37)
            got[layout] = [(b.populations(i), b.fields(i)) for i in range(len(cases))]
    for i, c in enumerate(cases):
        with lbm.Simulation(c, precision=prec) as s:
            s.init_case().step(37)
            g, f = s.populations()
            fl = s.fields()
        (g0, f0), fl0 = got[lbm.LBM_BATCH_AS_GIVEN][i]
        assert np.array_equal(g0, g) and np.array_equal(f0, f), i
        (g1, f1), fl1 = got[lbm.LBM_BATCH_FEWEST_COLUMNS][i]
        assert np.linalg.norm(g1 - g) <= tol * np.linalg.norm(g), i
        assert np.linalg.norm(f1 - f) <= tol * np.linalg.norm(f), i
        for k in ("phi", "p", "ux", "uy", "rho"):
            assert np.linalg.norm(fl1[k] - fl[k]) <= 10 * tol * np.linalg.norm(fl[k]) + 1e-300, (i, k)


def test_batch_layout_argument_is_checked():
    p = [lbm.make_params(c, "fp32") for c in mixed_cases()[:2]]
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_batch_create_ex(p, 2)
    assert e.value.status == lbm.LBM_ERR_ARG
    with lbm.Batch(mixed_cases()[:2]) as b:
        with pytest.raises(lbm.LbmError) as e:
            b.transposed(2)
        assert e.value.status == lbm.LBM_ERR_ARG


def test_batch_matches_oracle_fp64():
    """Cases 1 and 2 are stored transposed, the others as given."""
    cases = mixed_cases()[:3] + W.ensemble(ncases=4)[1:3]
    with lbm.Batch(cases, precision="fp64") as b:
        assert b.transposed(1) and b.transposed(2) and not b.transposed(0)
        b.init_all().step(6)
        for i, c in enumerate(cases):
            oc = O.OracleCase.from_dict(c.params)
            fl = c["fields"]
            g0, f0 = O.init(oc, fl["phi"], fl["p"], fl["ux"], fl["uy"])
            g_ref, f_ref = O.run(oc, g0, f0, 6)
            g, f = b.populations(i)
            # relative 1e-12, with an absolute floor of 1e-15 per element: where p and u are
            # tiny the populations are ~1e-9 while intermediate terms such as c^6 rho and
            # psi c^4 (~0.04) cancel, so rounding differences of two correct evaluation
            # orders sit at ~1e-17 absolute
            floor = 1e-15 * np.sqrt(g.size)
            assert np.linalg.norm(g - g_ref) <= 1e-12 * np.linalg.norm(g_ref) + floor, i
            assert np.linalg.norm(f - f_ref) <= 1e-12 * np.linalg.norm(f_ref) + floor, i


def test_autotuner_restores_state_and_keeps_results():
    cases = mixed_cases()
    with lbm.Batch(cases, precision="fp32") as b:
        b.init_all().step(5)
        before = [b.populations(i) for i in range(len(cases))]
        seg, block = lbm.lbm_batch_tune(b.b, 3)
        assert seg >= 1 and block in (64, 128)
        assert lbm.lbm_batch_get_launch(b.b) == (seg, block)
        after = [b.populations(i) for i in range(len(cases))]
        for (g0, f0), (g1, f1) in zip(before, after):
            assert np.array_equal(g0, g1) and np.array_equal(f0, f1)
        b.step(11)
        tuned = [b.populations(i) for i in range(len(cases))]
    with lbm.Batch(cases, precision="fp32") as b:
        b.init_all().step(16)
        ref = [b.populations(i) for i in range(len(cases))]
    for (g0, f0), (g1, f1) in zip(tuned, ref):
        assert np.array_equal(g0, g1) and np.array_equal(f0, f1)


def test_ensemble_of_512_cases_stays_finite_and_conserves_phi():
    cases = W.ensemble()
    with lbm.Batch(cases, precision="fp32") as b:
        b.init_all()
        m0 = np.array([b.fields(i)["phi"].sum() for i in range(len(cases))])
        b.step(500)
        m1 = []
        for i in range(len(cases)):
            fl = b.fields(i)
            assert np.isfinite(fl["p"]).all() and np.isfinite(fl["ux"]).all(), i
            m1.append(fl["phi"].sum())
    assert np.all(np.abs(np.array(m1) - m0) <= 1e-5 * m0)


def test_batch_rejects_mixed_precision():
    cases = mixed_cases()[:2]
    p = [lbm.make_params(cases[0], "fp32"), lbm.make_params(cases[1], "fp64")]
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_batch_create(p)
    assert e.value.status == lbm.LBM_ERR_ARG


def variant_cases(collision, sigma_model):
    extra = dict(collision=collision, sigma_model=sigma_model)
    if sigma_model == 1:
        extra.update(beta=0.5, psi0=0.2, gradpsi_x=6e-4, gradpsi_y=-2e-4)
    return [
        W.random_drop(40, 33, seed=11, wall_y=True, rho_ratio=20.0, gravity=1e-6, **extra),
        W.random_drop(97, 64, seed=12, wall_x=True, rho_ratio=10.0, marangoni=-2e-5, **extra),
        W.random_drop(17, 70, seed=13, wall_x=2, wall_y=1, rho_ratio=50.0, **extra),
        W.random_drop(65, 9, seed=14, rho_ratio=5.0, **extra),
    ]


@pytest.mark.parametrize("collision,sigma_model", [(1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp64", 1e-13)])
def test_batch_of_step_variants_matches_their_own_contexts(collision, sigma_model, prec, tol):
    """Batches of single-relaxation-time cases (Sec. 7) and of Langmuir-isotherm cases (Sec.
    6.7): bitwise as their own contexts when stored as given, to rounding when transposed."""
    cases = variant_cases(collision, sigma_model)
    got = {}
    for layout in (lbm.LBM_BATCH_AS_GIVEN, lbm.LBM_BATCH_FEWEST_COLUMNS):
        with lbm.Batch(cases, precision=prec, layout=layout) as b:
            if layout == lbm.LBM_BATCH_FEWEST_COLUMNS:
                assert b.transposed(1) and b.transposed(2) and not b.transposed(0)
            b.init_all().step(40)
            lbm.lbm_batch_check(b.b)
            got[layout] = [b.populations(i) for i in range(len(cases))]
    for i, c in enumerate(cases):
        with lbm.Simulation(c, precision=prec) as s:
            g, f = s.init_case().step(40).populations()
        g0, f0 = got[lbm.LBM_BATCH_AS_GIVEN][i]
        assert np.array_equal(g0, g) and np.array_equal(f0, f), i
        g1, f1 = got[lbm.LBM_BATCH_FEWEST_COLUMNS][i]
        assert np.linalg.norm(g1 - g) <= tol * np.linalg.norm(g), i
        assert np.linalg.norm(f1 - f) <= tol * np.linalg.norm(f), i


def test_batch_of_step_variants_matches_oracle_fp64():
    cases = variant_cases(1, 1)[:3]
    with lbm.Batch(cases, precision="fp64") as b:
        b.init_all().step(5)
        for i, c in enumerate(cases):
            oc = O.OracleCase.from_dict(c.params)
            fl = c["fields"]
            g_ref, f_ref = O.run(oc, *O.init(oc, fl["phi"], fl["p"], fl["ux"], fl["uy"]), 5)
            g, f = b.populations(i)
            assert np.linalg.norm(g - g_ref) <= 1e-12 * np.linalg.norm(g_ref), i
            assert np.linalg.norm(f - f_ref) <= 1e-12 * np.linalg.norm(f_ref), i


def test_batch_refuses_mixed_variants_and_the_imposed_flow():
    a, b = variant_cases(0, 0)[:2]
    b = dict(b)
    b["collision"] = 1
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_batch_create([lbm.make_params(a, "fp32"), lbm.make_params(b, "fp32")])
    assert e.value.status == lbm.LBM_ERR_ARG
    shear = W.shear_circle(L0=64)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_batch_create([lbm.make_params(shear, "fp32")])
    assert e.value.status == lbm.LBM_ERR_UNSUPPORTED
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_batch_create([lbm.make_params(b, "fp16")])
    assert e.value.status == lbm.LBM_ERR_UNSUPPORTED


def test_transposed_case_fields_with_some_outputs_omitted():
    """Any output pointer of lbm_batch_get_fields may be NULL, transposed or not."""
    cases = mixed_cases()[1:3]
    with lbm.Batch(cases) as b:
        assert b.transposed(0) and b.transposed(1)
        b.init_all().step(3)
        for i, c in enumerate(cases):
            full = b.fields(i)
            shape = (int(c["ny"]), int(c["nx"]))
            p, uy = np.empty(shape), np.empty(shape)
            lbm.lbm_batch_get_fields(b.b, i, None, p, None, uy, None)
            assert np.array_equal(p, full["p"]) and np.array_equal(uy, full["uy"])


def _batch_states(cases, prec, persistent, runs, layout=lbm.LBM_BATCH_FEWEST_COLUMNS,
                  seg_rows=0):
    with lbm.Batch(cases, precision=prec, layout=layout) as b:
        if seg_rows:
            lbm.lbm_batch_set_launch(b.b, seg_rows, 0)
        lbm.lbm_batch_set_persistent(b.b, persistent)
        assert lbm.lbm_batch_get_step_path(b.b) == (lbm.LBM_PATH_MULTI if persistent
                                                    else lbm.LBM_PATH_GRAPHS)
        b.init_all()
        for n in runs:
            b.step(n)
        lbm.lbm_batch_check(b.b)
        return [b.populations(i) for i in range(len(cases))]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp16", "bf16"])
@pytest.mark.parametrize("layout", [lbm.LBM_BATCH_AS_GIVEN, lbm.LBM_BATCH_FEWEST_COLUMNS])
def test_batch_multistep_matches_graph_replays(prec, layout):
    """The batched multi-step kernel (one cooperative launch per run, each task waiting only for
    the tasks of its own case within reach) gives every case the same state, bit for bit, as one
    launch per step; runs of odd and even lengths."""
    cases = mixed_cases()
    runs = (7, 2, 1, 12)
    a = _batch_states(cases, prec, 1, runs, layout)
    b = _batch_states(cases, prec, 0, runs, layout)
    for i in range(len(cases)):
        assert np.array_equal(a[i][0], b[i][0]) and np.array_equal(a[i][1], b[i][1]), i


@pytest.mark.parametrize("seg_rows", [1, 2, 5, 64])
def test_batch_multistep_with_any_task_height(seg_rows):
    """Tasks of one row (every task waits for two segments either side), two, five, and whole
    cases; FP32."""
    cases = mixed_cases()
    a = _batch_states(cases, "fp32", 1, (9, 4), seg_rows=seg_rows)
    b = _batch_states(cases, "fp32", 0, (9, 4), seg_rows=seg_rows)
    for i in range(len(cases)):
        assert np.array_equal(a[i][0], b[i][0]) and np.array_equal(a[i][1], b[i][1]), i


@pytest.mark.parametrize("collision,sigma_model", [(1, 0), (0, 1)])
def test_batch_multistep_step_variants(collision, sigma_model):
    cases = [W.random_drop(nx, ny, seed=nx + ny, wall_y=1, rho_ratio=10.0, gravity=1e-6,
                           collision=collision, sigma_model=sigma_model, beta=0.4, psi0=0.2,
                           gradpsi_x=1e-3) for nx, ny in ((40, 33), (97, 64), (65, 20))]
    a = _batch_states(cases, "fp32", 1, (6, 3))
    b = _batch_states(cases, "fp32", 0, (6, 3))
    for i in range(len(cases)):
        assert np.array_equal(a[i][0], b[i][0]) and np.array_equal(a[i][1], b[i][1]), i


def test_batch_persistent_rejects_bad_values():
    with lbm.Batch(mixed_cases()[:2]) as b:
        for bad in (2, -1):
            with pytest.raises(lbm.LbmError) as e:
                lbm.lbm_batch_set_persistent(b.b, bad)
            assert e.value.status == lbm.LBM_ERR_ARG
