"""The C-ABI library builds, loads and exports every function include/cmlbm.h declares (CPU)."""
import ctypes
import os
import re

import pytest

from paper_1909_04166_gb300 import build, lbm

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "cmlbm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for core in ("lbm_create", "lbm_init_fields", "lbm_step", "lbm_get_fields", "lbm_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol():
    L = ctypes.CDLL(build.build())
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert sorted(declared_functions()) == sorted(lbm.EXPORTS)


def test_host_only_calls_work_without_a_device():
    assert lbm.lbm_strerror(lbm.LBM_ERR_PARAM) == "invalid physical parameter"
    assert lbm.lbm_strerror(12345) == "unknown status"
    from paper_1909_04166_gb300 import workloads as W
    p = lbm.make_params(W.laplace(n=40), "fp32")
    # two buffers of ceil(40/32) = 2 strips x 40 rows x 18 x 32 floats
    assert lbm.lbm_state_bytes(p) == 2 * 2 * 40 * 18 * 32 * 4
    p64 = lbm.make_params(W.laplace(n=40), "fp64")
    assert lbm.lbm_state_bytes(p64) == 2 * lbm.lbm_state_bytes(p)
    bad = lbm.make_params(W.laplace(n=40), "fp32")
    bad.width = 0.0
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_state_bytes(bad)
    assert e.value.status == lbm.LBM_ERR_PARAM


def test_create_reports_cuda_error_without_a_device():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    from paper_1909_04166_gb300 import workloads as W
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(lbm.make_params(W.laplace(n=16), "fp32"))
    assert e.value.status == lbm.LBM_ERR_CUDA
    lbm.lbm_destroy(None)
