"""Thin ctypes binding of the C ABI in ``include/cmlbm.h`` (argument marshalling only).

Every function keeps the C name and returns what the C call returns through its out-arguments;
a non-zero status raises ``LbmError``.  All computation runs in ``libcmlbm.so``; if the library
is missing or cannot be loaded this module raises on first use - there is no fallback.

Host arrays are numpy float64, nodal fields ``(ny, nx)``, populations ``(9, ny, nx)``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

LBM_OK = 0
LBM_ERR_ARG = -1
LBM_ERR_PARAM = -2
LBM_ERR_CUDA = -3
LBM_ERR_NOMEM = -4
LBM_ERR_STATE = -5
LBM_ERR_NONFINITE = -6
LBM_ERR_UNSUPPORTED = -7
LBM_ERR_TIMEOUT = -8
LBM_ERR_INDEX = -9

LBM_FP64 = 0
LBM_FP32 = 1
LBM_FP32_FP16 = 2
LBM_FP32_BF16 = 3
PRECISIONS = {"fp64": LBM_FP64, "fp32": LBM_FP32, "fp16": LBM_FP32_FP16, "bf16": LBM_FP32_BF16}

LBM_PERIODIC = 0
LBM_WALL = 1
LBM_FREESLIP = 2
LBM_CASCADED = 0
LBM_SRT = 1
LBM_SIGMA_LINEAR_T = 0
LBM_SIGMA_LANGMUIR = 1
LBM_FLOW_COUPLED = 0
LBM_FLOW_SHEAR = 1
LBM_BATCH_AS_GIVEN = 0
LBM_BATCH_FEWEST_COLUMNS = 1

EXPORTS = [
    "lbm_state_bytes", "lbm_create", "lbm_create_with_buffer", "lbm_init_fields",
    "lbm_init_fields_device", "lbm_step", "lbm_get_fields", "lbm_get_populations",
    "lbm_set_populations", "lbm_save_state", "lbm_load_state", "lbm_state_device",
    "lbm_diagnostics", "lbm_set_launch",
    "lbm_get_launch", "lbm_steps_done", "lbm_destroy", "lbm_strerror", "lbm_last_cuda_error",
    "lbm_check", "lbm_set_graphs", "lbm_set_persistent", "lbm_get_step_path",
    "lbm_set_checked", "lbm_diagnostics_noalloc",
    "lbm_inject_timeout",
    "lbm_batch_create", "lbm_batch_init_fields", "lbm_batch_step", "lbm_batch_get_fields",
    "lbm_batch_get_populations", "lbm_batch_set_launch", "lbm_batch_get_launch",
    "lbm_batch_tune", "lbm_batch_nodes", "lbm_batch_check", "lbm_batch_destroy",
    "lbm_batch_create_ex", "lbm_batch_case_transposed", "lbm_batch_set_persistent",
    "lbm_batch_get_step_path",
]


class LbmError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {lbm_strerror(status)} ({status})")


class lbm_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32),
        ("rho_a", ctypes.c_double), ("rho_b", ctypes.c_double),
        ("mu_a", ctypes.c_double), ("mu_b", ctypes.c_double),
        ("sigma0", ctypes.c_double), ("dsigma_dT", ctypes.c_double),
        ("T0", ctypes.c_double), ("gradT_x", ctypes.c_double), ("gradT_y", ctypes.c_double),
        ("mobility", ctypes.c_double), ("width", ctypes.c_double),
        ("gx", ctypes.c_double), ("gy", ctypes.c_double), ("rho_ref", ctypes.c_double),
        ("precision", ctypes.c_int32), ("device", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("store_scale_g", ctypes.c_double), ("store_scale_f", ctypes.c_double),
        ("bc_x_hi", ctypes.c_int32), ("bc_y_hi", ctypes.c_int32),
        ("collision", ctypes.c_int32), ("sigma_model", ctypes.c_int32),
        ("beta", ctypes.c_double), ("psi0", ctypes.c_double),
        ("gradpsi_x", ctypes.c_double), ("gradpsi_y", ctypes.c_double),
        ("flow", ctypes.c_int32), ("reverse_step", ctypes.c_int32),
        ("u0", ctypes.c_double),
    ]


class lbm_diag(ctypes.Structure):
    _fields_ = [("sum_phi", ctypes.c_double), ("sum_p", ctypes.c_double),
                ("max_speed", ctypes.c_double), ("dp_laplace", ctypes.c_double),
                ("nonfinite", ctypes.c_int64)]


_lib = None


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libcmlbm.so (building it with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: build it with "
                           "paper_1909_04166_gb300.build.build()")
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, dp, i32, i64 = ctypes.c_void_p, P(ctypes.c_double), ctypes.c_int32, ctypes.c_int64
    pp = P(lbm_params)
    L.lbm_state_bytes.argtypes = [pp, P(ctypes.c_size_t)]
    L.lbm_create.argtypes = [pp, P(vp)]
    L.lbm_create_with_buffer.argtypes = [pp, vp, ctypes.c_size_t, P(vp)]
    L.lbm_init_fields.argtypes = [vp, dp, dp, dp, dp]
    L.lbm_init_fields_device.argtypes = [vp, vp, vp, vp, vp]
    L.lbm_step.argtypes = [vp, i32]
    L.lbm_get_fields.argtypes = [vp, dp, dp, dp, dp, dp]
    L.lbm_get_populations.argtypes = [vp, dp, dp]
    L.lbm_set_populations.argtypes = [vp, dp, dp]
    L.lbm_save_state.argtypes = [vp, vp, ctypes.c_size_t, P(i64)]
    L.lbm_load_state.argtypes = [vp, vp, ctypes.c_size_t, i64]
    L.lbm_state_device.argtypes = [vp, P(vp), P(i32), P(i64)]
    L.lbm_diagnostics.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, P(lbm_diag)]
    L.lbm_set_launch.argtypes = [vp, i32, i32]
    L.lbm_get_launch.argtypes = [vp, P(i32), P(i32)]
    L.lbm_steps_done.argtypes = [vp]
    L.lbm_steps_done.restype = i64
    L.lbm_destroy.argtypes = [vp]
    L.lbm_destroy.restype = None
    L.lbm_strerror.argtypes = [ctypes.c_int]
    L.lbm_strerror.restype = ctypes.c_char_p
    L.lbm_last_cuda_error.argtypes = [vp]
    L.lbm_check.argtypes = [vp]
    L.lbm_set_graphs.argtypes = [vp, i32]
    L.lbm_set_persistent.argtypes = [vp, i32]
    L.lbm_get_step_path.argtypes = [vp, P(i32)]
    L.lbm_set_checked.argtypes = [vp, i32]
    L.lbm_inject_timeout.argtypes = [vp, i32]
    dd = ctypes.c_double
    L.lbm_diagnostics_noalloc.argtypes = [vp, vp, vp, vp, i32, i32, i32, i32, dd, dd, dd, dd,
                                          vp, vp]
    L.lbm_batch_create.argtypes = [P(lbm_params), i32, P(vp)]
    L.lbm_batch_create_ex.argtypes = [P(lbm_params), i32, i32, P(vp)]
    L.lbm_batch_case_transposed.argtypes = [vp, i32]
    L.lbm_batch_init_fields.argtypes = [vp, i32, dp, dp, dp, dp]
    L.lbm_batch_step.argtypes = [vp, i32]
    L.lbm_batch_get_fields.argtypes = [vp, i32, dp, dp, dp, dp, dp]
    L.lbm_batch_get_populations.argtypes = [vp, i32, dp, dp]
    L.lbm_batch_set_launch.argtypes = [vp, i32, i32]
    L.lbm_batch_get_launch.argtypes = [vp, P(i32), P(i32)]
    L.lbm_batch_set_persistent.argtypes = [vp, i32]
    L.lbm_batch_get_step_path.argtypes = [vp, P(i32)]
    L.lbm_batch_tune.argtypes = [vp, i32, P(i32), P(i32)]
    L.lbm_batch_nodes.argtypes = [vp]
    L.lbm_batch_nodes.restype = i64
    L.lbm_batch_check.argtypes = [vp]
    L.lbm_batch_destroy.argtypes = [vp]
    L.lbm_batch_destroy.restype = None
    _lib = L
    return L


def _check(status: int, what: str) -> None:
    if status != LBM_OK:
        raise LbmError(status, what)


def _dptr(a):
    if a is None:
        return None
    assert isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_params(case: dict, precision="fp32", device=0, stream=0) -> lbm_params:
    """lbm_params from a case dictionary (keys of ``workloads.Case``; boundary kinds 0 / False
    periodic, 1 / True no-slip, 2 free-slip; wall_x_hi / wall_y_hi for a differing right / top
    side)."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    hi_x, hi_y = case.get("wall_x_hi"), case.get("wall_y_hi")
    return lbm_params(
        int(case["nx"]), int(case["ny"]),
        int(case.get("wall_x", 0)), int(case.get("wall_y", 0)),
        float(case["rho_a"]), float(case["rho_b"]), float(case["mu_a"]), float(case["mu_b"]),
        float(case.get("sigma0", 0.0)), float(case.get("dsigma_dT", 0.0)),
        float(case.get("T0", 0.0)), float(case.get("gradT_x", 0.0)),
        float(case.get("gradT_y", 0.0)), float(case["mobility"]), float(case["width"]),
        float(case.get("gx", 0.0)), float(case.get("gy", 0.0)), float(case.get("rho_ref", 0.0)),
        prec, int(device), ctypes.c_void_p(int(stream)),
        float(case.get("store_scale_g", 0.0)), float(case.get("store_scale_f", 0.0)),
        0 if hi_x is None else int(hi_x), 0 if hi_y is None else int(hi_y),
        int(case.get("collision", 0)), int(case.get("sigma_model", 0)),
        float(case.get("beta", 0.0)), float(case.get("psi0", 0.0)),
        float(case.get("gradpsi_x", 0.0)), float(case.get("gradpsi_y", 0.0)),
        int(case.get("flow", 0)), int(case.get("reverse_step", 0)), float(case.get("u0", 0.0)))


# ---- ABI wrappers (same names as the C entry points) ------------------------------------------

def lbm_strerror(status: int) -> str:
    return lib().lbm_strerror(int(status)).decode()


def lbm_state_bytes(params: lbm_params) -> int:
    n = ctypes.c_size_t(0)
    _check(lib().lbm_state_bytes(ctypes.byref(params), ctypes.byref(n)), "lbm_state_bytes")
    return int(n.value)


def lbm_create(params: lbm_params) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    _check(lib().lbm_create(ctypes.byref(params), ctypes.byref(ctx)), "lbm_create")
    return ctx


def lbm_create_with_buffer(params: lbm_params, device_ptr: int, nbytes: int):
    ctx = ctypes.c_void_p()
    _check(lib().lbm_create_with_buffer(ctypes.byref(params), ctypes.c_void_p(int(device_ptr)),
                                        ctypes.c_size_t(int(nbytes)), ctypes.byref(ctx)),
           "lbm_create_with_buffer")
    return ctx


def lbm_init_fields(ctx, phi, p, ux, uy) -> None:
    _check(lib().lbm_init_fields(ctx, _dptr(phi), _dptr(p), _dptr(ux), _dptr(uy)),
           "lbm_init_fields")


def lbm_init_fields_device(ctx, phi_ptr: int, p_ptr: int, ux_ptr: int, uy_ptr: int) -> None:
    v = ctypes.c_void_p
    _check(lib().lbm_init_fields_device(ctx, v(phi_ptr), v(p_ptr), v(ux_ptr), v(uy_ptr)),
           "lbm_init_fields_device")


def lbm_step(ctx, nsteps: int) -> None:
    _check(lib().lbm_step(ctx, int(nsteps)), "lbm_step")


def lbm_get_fields(ctx, phi=None, p=None, ux=None, uy=None, rho=None) -> None:
    _check(lib().lbm_get_fields(ctx, _dptr(phi), _dptr(p), _dptr(ux), _dptr(uy), _dptr(rho)),
           "lbm_get_fields")


def lbm_get_populations(ctx, g, f) -> None:
    _check(lib().lbm_get_populations(ctx, _dptr(g), _dptr(f)), "lbm_get_populations")


def lbm_set_populations(ctx, g, f) -> None:
    _check(lib().lbm_set_populations(ctx, _dptr(g), _dptr(f)), "lbm_set_populations")


def lbm_save_state(ctx, nbytes: int):
    """Exact checkpoint: (bytes of the current state buffer, step counter)."""
    buf = np.empty(int(nbytes), dtype=np.uint8)
    steps = ctypes.c_int64()
    _check(lib().lbm_save_state(ctx, buf.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(buf.size),
                                ctypes.byref(steps)), "lbm_save_state")
    return buf, int(steps.value)


def lbm_load_state(ctx, buf: np.ndarray, steps: int) -> None:
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(lib().lbm_load_state(ctx, buf.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(buf.size),
                                ctypes.c_int64(int(steps))), "lbm_load_state")


def lbm_state_device(ctx):
    ptr, nstrips, elems = ctypes.c_void_p(), ctypes.c_int32(), ctypes.c_int64()
    _check(lib().lbm_state_device(ctx, ctypes.byref(ptr), ctypes.byref(nstrips),
                                  ctypes.byref(elems)), "lbm_state_device")
    return int(ptr.value or 0), int(nstrips.value), int(elems.value)


def lbm_diagnostics_noalloc(phi_ptr: int, p_ptr: int, ux_ptr: int, uy_ptr: int, nx: int,
                            ny: int, bc_x: int, bc_y: int, xc: float, yc: float, r_in: float,
                            r_out: float, out_ptr: int, stream: int = 0) -> None:
    """Allocation-free diagnostics of device nodal fields into a device lbm_diag (see the C
    header); asynchronous on `stream`."""
    v = ctypes.c_void_p
    _check(lib().lbm_diagnostics_noalloc(v(phi_ptr), v(p_ptr), v(ux_ptr), v(uy_ptr), int(nx),
                                         int(ny), int(bc_x), int(bc_y), float(xc), float(yc),
                                         float(r_in), float(r_out), v(out_ptr), v(int(stream))),
           "lbm_diagnostics_noalloc")


def lbm_set_graphs(ctx, enable: bool) -> None:
    _check(lib().lbm_set_graphs(ctx, int(bool(enable))), "lbm_set_graphs")


def lbm_set_persistent(ctx, enable) -> None:
    """True / 1: the multi-step kernel wherever it fits; False / 0: never; 2: automatic."""
    _check(lib().lbm_set_persistent(ctx, int(enable)), "lbm_set_persistent")


LBM_PATH_SINGLE, LBM_PATH_GRAPHS, LBM_PATH_MULTI = 0, 1, 2


def lbm_get_step_path(ctx) -> int:
    v = ctypes.c_int32()
    _check(lib().lbm_get_step_path(ctx, ctypes.byref(v)), "lbm_get_step_path")
    return int(v.value)


def lbm_set_checked(ctx, enable) -> None:
    """enable: 0 / False plain kernel, 1 / True checked kernel, 2 the checker's self-test."""
    _check(lib().lbm_set_checked(ctx, int(enable)), "lbm_set_checked")


def lbm_check(ctx) -> None:
    _check(lib().lbm_check(ctx), "lbm_check")


def lbm_inject_timeout(ctx, enable) -> None:
    """Test hook of the failure path: 1, the first bounded wait of every warp of a step gives
    up at once; 2, the multi-step kernel's waits for neighbouring warps never succeed (both
    report LBM_ERR_TIMEOUT; nothing faults or hangs)."""
    _check(lib().lbm_inject_timeout(ctx, int(enable)), "lbm_inject_timeout")


def lbm_diagnostics(ctx, xc=0.0, yc=0.0, r_in=-1.0, r_out=0.0, allow_nonfinite=True) -> dict:
    d = lbm_diag()
    s = lib().lbm_diagnostics(ctx, float(xc), float(yc), float(r_in), float(r_out),
                              ctypes.byref(d))
    if s != LBM_OK and not (allow_nonfinite and s == LBM_ERR_NONFINITE):
        _check(s, "lbm_diagnostics")
    return {k: getattr(d, k) for k, _ in lbm_diag._fields_}


def lbm_set_launch(ctx, seg_rows: int = 0, block_threads: int = 0) -> None:
    _check(lib().lbm_set_launch(ctx, int(seg_rows), int(block_threads)), "lbm_set_launch")


def lbm_get_launch(ctx):
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().lbm_get_launch(ctx, ctypes.byref(a), ctypes.byref(b)), "lbm_get_launch")
    return int(a.value), int(b.value)


def lbm_steps_done(ctx) -> int:
    return int(lib().lbm_steps_done(ctx))


def lbm_destroy(ctx) -> None:
    if ctx is not None and ctx.value:
        lib().lbm_destroy(ctx)
        ctx.value = None


def lbm_last_cuda_error(ctx) -> int:
    return int(lib().lbm_last_cuda_error(ctx))


def lbm_batch_create(params_list) -> ctypes.c_void_p:
    arr = (lbm_params * len(params_list))(*params_list)
    b = ctypes.c_void_p()
    _check(lib().lbm_batch_create(arr, len(params_list), ctypes.byref(b)), "lbm_batch_create")
    return b


def lbm_batch_create_ex(params_list, layout: int) -> ctypes.c_void_p:
    arr = (lbm_params * len(params_list))(*params_list)
    b = ctypes.c_void_p()
    _check(lib().lbm_batch_create_ex(arr, len(params_list), int(layout), ctypes.byref(b)),
           "lbm_batch_create_ex")
    return b


def lbm_batch_case_transposed(b, c: int) -> bool:
    s = int(lib().lbm_batch_case_transposed(b, int(c)))
    _check(min(s, 0), "lbm_batch_case_transposed")
    return bool(s)


def lbm_batch_init_fields(b, c, phi, p, ux, uy) -> None:
    _check(lib().lbm_batch_init_fields(b, int(c), _dptr(phi), _dptr(p), _dptr(ux), _dptr(uy)),
           "lbm_batch_init_fields")


def lbm_batch_step(b, nsteps: int) -> None:
    _check(lib().lbm_batch_step(b, int(nsteps)), "lbm_batch_step")


def lbm_batch_get_fields(b, c, phi=None, p=None, ux=None, uy=None, rho=None) -> None:
    _check(lib().lbm_batch_get_fields(b, int(c), _dptr(phi), _dptr(p), _dptr(ux), _dptr(uy),
                                      _dptr(rho)), "lbm_batch_get_fields")


def lbm_batch_get_populations(b, c, g, f) -> None:
    _check(lib().lbm_batch_get_populations(b, int(c), _dptr(g), _dptr(f)),
           "lbm_batch_get_populations")


def lbm_batch_set_launch(b, seg_rows: int = 0, block_threads: int = 0) -> None:
    _check(lib().lbm_batch_set_launch(b, int(seg_rows), int(block_threads)),
           "lbm_batch_set_launch")


def lbm_batch_get_launch(b):
    a, c = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().lbm_batch_get_launch(b, ctypes.byref(a), ctypes.byref(c)), "lbm_batch_get_launch")
    return int(a.value), int(c.value)


def lbm_batch_set_persistent(b, enable) -> None:
    _check(lib().lbm_batch_set_persistent(b, int(enable)), "lbm_batch_set_persistent")


def lbm_batch_get_step_path(b) -> int:
    v = ctypes.c_int32()
    _check(lib().lbm_batch_get_step_path(b, ctypes.byref(v)), "lbm_batch_get_step_path")
    return int(v.value)


def lbm_batch_tune(b, trial_steps: int = 8):
    a, c = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().lbm_batch_tune(b, int(trial_steps), ctypes.byref(a), ctypes.byref(c)),
           "lbm_batch_tune")
    return int(a.value), int(c.value)


def lbm_batch_nodes(b) -> int:
    return int(lib().lbm_batch_nodes(b))


def lbm_batch_check(b) -> None:
    _check(lib().lbm_batch_check(b), "lbm_batch_check")


def lbm_batch_destroy(b) -> None:
    if b is not None and b.value:
        lib().lbm_batch_destroy(b)
        b.value = None


# ---- convenience ------------------------------------------------------------------------------

class Batch:
    """Owns one batch of independent cases (dictionaries from ``workloads``)."""

    def __init__(self, cases, precision="fp32", device=0, stream=0,
                 layout=LBM_BATCH_FEWEST_COLUMNS):
        self.cases = list(cases)
        self.params = [make_params(c, precision, device, stream) for c in self.cases]
        self.b = lbm_batch_create_ex(self.params, layout)

    def transposed(self, i) -> bool:
        return lbm_batch_case_transposed(self.b, i)

    def init_case(self, i, fields=None):
        c = self.cases[i]
        f = fields or c["fields"]
        shape = (int(c["ny"]), int(c["nx"]))
        arrs = [np.ascontiguousarray(np.broadcast_to(np.asarray(f[k], np.float64), shape))
                for k in ("phi", "p", "ux", "uy")]
        lbm_batch_init_fields(self.b, i, *arrs)
        return self

    def init_all(self):
        for i in range(len(self.cases)):
            self.init_case(i)
        return self

    def step(self, n=1):
        lbm_batch_step(self.b, n)
        return self

    def fields(self, i) -> dict:
        c = self.cases[i]
        shape = (int(c["ny"]), int(c["nx"]))
        out = {k: np.empty(shape) for k in ("phi", "p", "ux", "uy", "rho")}
        lbm_batch_get_fields(self.b, i, out["phi"], out["p"], out["ux"], out["uy"], out["rho"])
        return out

    def populations(self, i):
        c = self.cases[i]
        g = np.empty((9, int(c["ny"]), int(c["nx"])))
        f = np.empty_like(g)
        lbm_batch_get_populations(self.b, i, g, f)
        return g, f

    def close(self):
        lbm_batch_destroy(self.b)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Simulation:
    """Owns one context; a case dictionary from ``workloads`` gives its parameters."""

    def __init__(self, case: dict, precision="fp32", device=0, stream=0):
        self.case = case
        self.nx, self.ny = int(case["nx"]), int(case["ny"])
        self.params = make_params(case, precision, device, stream)
        self.ctx = lbm_create(self.params)

    def init(self, phi, p, ux, uy):
        shape = (self.ny, self.nx)
        arrs = [np.ascontiguousarray(np.broadcast_to(np.asarray(a, np.float64), shape))
                for a in (phi, p, ux, uy)]
        lbm_init_fields(self.ctx, *arrs)
        return self

    def init_case(self):
        f = self.case["fields"]
        return self.init(f["phi"], f["p"], f["ux"], f["uy"])

    def step(self, n=1):
        lbm_step(self.ctx, n)
        return self

    def fields(self) -> dict:
        shape = (self.ny, self.nx)
        out = {k: np.empty(shape) for k in ("phi", "p", "ux", "uy", "rho")}
        lbm_get_fields(self.ctx, out["phi"], out["p"], out["ux"], out["uy"], out["rho"])
        return out

    def populations(self):
        g = np.empty((9, self.ny, self.nx))
        f = np.empty((9, self.ny, self.nx))
        lbm_get_populations(self.ctx, g, f)
        return g, f

    def set_populations(self, g, f):
        lbm_set_populations(self.ctx, np.ascontiguousarray(g, np.float64),
                            np.ascontiguousarray(f, np.float64))
        return self

    def save_state(self):
        """Exact checkpoint (raw state bytes, step counter)."""
        return lbm_save_state(self.ctx, lbm_state_bytes(self.params) // 2)

    def load_state(self, checkpoint):
        lbm_load_state(self.ctx, *checkpoint)
        return self

    def diagnostics(self, xc=0.0, yc=0.0, r_in=-1.0, r_out=0.0) -> dict:
        return lbm_diagnostics(self.ctx, xc, yc, r_in, r_out)

    def close(self):
        lbm_destroy(self.ctx)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
