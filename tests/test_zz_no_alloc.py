"""The allocation-free diagnostics entry point (lbm_diagnostics_noalloc) against the context
diagnostics (lbm_diagnostics), through the C ABI, on two calls in a row.

lbm_diagnostics_noalloc exists for callers that cannot allocate device memory at the moment they
need the diagnostics, e.g. inside CUDA-graph capture or in loops whose buffers are all sized up
front; it reduces caller-owned device fields using a fixed device array in the library."""
import numpy as np
import pytest

from paper_1909_04166_gb300 import lbm
from paper_1909_04166_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_diagnostics_match_context_diagnostics_twice():
    torch = pytest.importorskip("torch")
    n = 96
    case = W.laplace(n=n, radius=24.0, width=5.0, rho_ratio=1000.0, sigma=1e-3)
    stream = torch.cuda.current_stream().cuda_stream
    with lbm.Simulation(case, precision="fp32", stream=stream) as sim:
        sim.init_case().step(40)
        for call in range(2):
            ref = sim.diagnostics(n / 2, n / 2, 10.0, 40.0)
            fl = sim.fields()
            dev = [torch.tensor(fl[k], dtype=torch.float64, device="cuda")
                   for k in ("phi", "p", "ux", "uy")]
            out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
            lbm.lbm_diagnostics_noalloc(*(t.data_ptr() for t in dev), n, n, lbm.LBM_PERIODIC,
                                        lbm.LBM_PERIODIC, n / 2, n / 2, 10.0, 40.0,
                                        out.data_ptr(), stream)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            nonfinite = int(out.view(torch.int64)[4].item())
            assert nonfinite == ref["nonfinite"] == 0
            assert got[0] == pytest.approx(ref["sum_phi"], rel=1e-12)
            assert got[1] == pytest.approx(ref["sum_p"], rel=1e-10, abs=1e-16)
            assert got[2] == pytest.approx(ref["max_speed"], rel=1e-12)
            assert got[3] == pytest.approx(ref["dp_laplace"], rel=1e-10)
            assert np.isfinite(got[:4]).all()
            sim.step(25)


def test_noalloc_rejects_grids_beyond_its_fixed_array():
    torch = pytest.importorskip("torch")
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_diagnostics_noalloc(buf.data_ptr(), buf.data_ptr(), buf.data_ptr(),
                                    buf.data_ptr(), 4096, 4096, 0, 0, 0.0, 0.0, -1.0, 0.0,
                                    buf.data_ptr())
    assert e.value.status == lbm.LBM_ERR_ARG
