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
    # 16-bit: two FP32 zeroth-moment planes and 18 planes of 16-bit deviations per tile
    p16 = lbm.make_params(W.laplace(n=40), "fp16")
    assert lbm.lbm_state_bytes(p16) == 2 * 2 * 40 * (2 * 32 * 4 + 18 * 32 * 2)
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


def test_binding_struct_matches_header_layout(tmp_path):
    """sizeof and every field offset of lbm_params / lbm_diag as the C compiler lays them out
    from include/cmlbm.h equal the ctypes structures of the binding."""
    structs = {"lbm_params": lbm.lbm_params, "lbm_diag": lbm.lbm_diag}
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"',
             "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-std=c11", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for line in filter(None, out):
        name, field, value = line.split()
        cls = structs[name]
        expect = ctypes.sizeof(cls) if field == "sizeof" else getattr(cls, field).offset
        assert int(value) == expect, (name, field)
        seen += 1
    assert seen == sum(len(c._fields_) + 1 for c in structs.values())


def test_new_forms_are_validated_without_a_device():
    """Boundary pairs, collision / sigma / flow enums, the Langmuir domain psi < 1 and the
    16-bit storage limits are checked before any device work (lbm_state_bytes validates)."""
    from paper_1909_04166_gb300 import workloads as W

    def status(precision="fp32", **kw):
        case = W.random_drop(40, 30, seed=0)
        case.update(kw)
        try:
            lbm.lbm_state_bytes(lbm.make_params(case, precision))
            return lbm.LBM_OK
        except lbm.LbmError as e:
            return e.status

    assert status(wall_y=1, wall_y_hi=2) == lbm.LBM_OK
    assert status(wall_x=2) == lbm.LBM_OK
    assert status(wall_y=0, wall_y_hi=2) == lbm.LBM_ERR_ARG      # periodic must pair
    assert status(wall_x=3) == lbm.LBM_ERR_ARG
    assert status(collision=1) == lbm.LBM_OK
    assert status(collision=2) == lbm.LBM_ERR_ARG
    assert status(sigma_model=1, beta=0.5, psi0=0.2, gradpsi_x=0.01) == lbm.LBM_OK
    # psi reaches 0.2 + 0.03 * 39 > 1 at the right edge: ln(1 - psi) undefined
    assert status(sigma_model=1, beta=0.5, psi0=0.2, gradpsi_x=0.03) == lbm.LBM_ERR_PARAM
    assert status(flow=1, u0=0.02, reverse_step=100) == lbm.LBM_OK
    assert status(flow=5) == lbm.LBM_ERR_ARG
    assert status("fp16", collision=1) == lbm.LBM_ERR_UNSUPPORTED
    assert status("bf16", flow=1, u0=0.01) == lbm.LBM_ERR_UNSUPPORTED
    assert status("fp16", wall_y=2) == lbm.LBM_OK


def test_batch_rejects_mixed_step_forms_without_a_device():
    """The cases of a batch share the collision model and the sigma law (else LBM_ERR_ARG); the
    imposed flow is not batched (LBM_ERR_UNSUPPORTED); the checks come before any device
    work."""
    from paper_1909_04166_gb300 import workloads as W
    base = lbm.make_params(W.random_drop(40, 30, seed=1), "fp32")
    for bad, code in ((dict(collision=1), lbm.LBM_ERR_ARG),
                      (dict(sigma_model=1, beta=0.5), lbm.LBM_ERR_ARG),
                      (dict(flow=1, u0=0.01), lbm.LBM_ERR_UNSUPPORTED)):
        c = W.random_drop(40, 30, seed=2)
        c.update(bad)
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_batch_create([base, lbm.make_params(c, "fp32")])
        assert e.value.status == code, bad


def test_batch_layout_is_checked_without_a_device():
    """lbm_batch_create_ex takes LBM_BATCH_AS_GIVEN or LBM_BATCH_FEWEST_COLUMNS only, checked
    before any device work; lbm_batch_case_transposed refuses a NULL batch."""
    import ctypes
    from paper_1909_04166_gb300 import workloads as W
    p = [lbm.make_params(W.random_drop(40, 30, seed=1), "fp32")]
    for layout in (-1, 2):
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_batch_create_ex(p, layout)
        assert e.value.status == lbm.LBM_ERR_ARG
    assert lbm.lib().lbm_batch_case_transposed(ctypes.c_void_p(), 0) == lbm.LBM_ERR_ARG


def test_grid_extents_are_validated_without_a_device():
    """1 .. 65536 nodes along each axis (include/cmlbm.h); 0, negative and 65537 are refused
    before any device work, and the state size of the largest extents is computed in 64 bits."""
    from paper_1909_04166_gb300 import workloads as W

    def state_bytes(nx, ny, precision="fp32"):
        case = W.random_drop(8, 8, seed=0)
        case.update(nx=nx, ny=ny)
        return lbm.lbm_state_bytes(lbm.make_params(case, precision))

    for nx, ny in ((0, 8), (8, 0), (-1, 8), (8, -5), (65537, 8), (8, 65537)):
        with pytest.raises(lbm.LbmError) as e:
            state_bytes(nx, ny)
        assert e.value.status == lbm.LBM_ERR_ARG, (nx, ny)
    # two buffers of ny rows x ceil(nx / 32) tiles (2304 B per FP32 tile, 1408 B 16-bit,
    # 4608 B FP64)
    assert state_bytes(1, 1) == 2 * 2304
    assert state_bytes(65536, 65536) == 2 * 65536 * 2048 * 2304
    assert state_bytes(65536, 65536, "fp16") == 2 * 65536 * 2048 * 1408
    assert state_bytes(65536, 65536, "fp64") == 2 * 65536 * 2048 * 4608
    assert state_bytes(33, 1, "bf16") == 2 * 2 * 1408
