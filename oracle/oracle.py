"""ctypes binding of the FP64 C oracle (``cmlbm_oracle.c``).

Test infrastructure only: the tests, the smoke check and the benchmark's CPU-baseline leg load
it.  Arrays are numpy float64; a population field is ``(9, ny, nx)`` (plane alpha, row y,
column x), a nodal field ``(ny, nx)``.  Velocity ordering and moment conventions are those of
Sec. 4 of the paper (D2Q9, e_x = (0,1,0,-1,0,1,-1,-1,1), e_y = (0,0,1,0,-1,1,1,-1,-1)).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cmlbm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libcmlbm_oracle.so")

__all__ = [
    "OracleCase", "build", "lib", "init", "step", "run", "step_rows", "fields", "node_info",
    "stencils", "fluid_collide", "fluid_source", "ace_collide", "geq", "feq", "num_threads",
    "run_float_storage", "normal_eps", "set_normal_eps",
]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FP contraction, OpenMP over rows)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-shared", "-fPIC", "-o",
            _LIB_PATH + ".tmp", _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)   # no OpenMP on this host: single-threaded oracle
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


class _Case(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("bc_x0", ctypes.c_int), ("bc_x1", ctypes.c_int),
        ("bc_y0", ctypes.c_int), ("bc_y1", ctypes.c_int),
        ("rho_a", ctypes.c_double), ("rho_b", ctypes.c_double),
        ("mu_a", ctypes.c_double), ("mu_b", ctypes.c_double),
        ("sigma0", ctypes.c_double), ("dsigma_dT", ctypes.c_double),
        ("T0", ctypes.c_double), ("gradT_x", ctypes.c_double), ("gradT_y", ctypes.c_double),
        ("mobility", ctypes.c_double), ("width", ctypes.c_double),
        ("gx", ctypes.c_double), ("gy", ctypes.c_double), ("rho_ref", ctypes.c_double),
        ("collision", ctypes.c_int), ("sigma_model", ctypes.c_int),
        ("beta", ctypes.c_double), ("psi0", ctypes.c_double),
        ("gradpsi_x", ctypes.c_double), ("gradpsi_y", ctypes.c_double),
        ("flow", ctypes.c_int), ("reverse_step", ctypes.c_int),
        ("u0", ctypes.c_double), ("t", ctypes.c_int),
    ]


# boundary kinds of one side (wall_x / wall_y and their *_hi overrides)
PERIODIC, NOSLIP, FREESLIP = 0, 1, 2


def side_kinds(lo, hi):
    """(low side, high side) kinds of one axis: ``lo`` is 0 / False (periodic), 1 / True
    (no-slip) or 2 (free-slip) and applies to both sides unless ``hi`` (None = same) is given."""
    lo = int(lo)
    hi = lo if hi is None or int(hi) == 0 else int(hi)
    if lo not in (0, 1, 2) or hi not in (0, 1, 2) or (lo == 0) != (hi == 0):
        raise ValueError(f"invalid boundary pair ({lo}, {hi})")
    return lo, hi


class _Node(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "phi", "rho", "mu", "omega_nu", "pstar", "p", "ux", "uy",
        "dphix", "dphiy", "lap", "hxx", "hyy", "hxy", "dpx", "dpy",
        "nx", "ny", "theta", "Fsx", "Fsy", "Ftx", "Fty", "Fpx", "Fpy")]


@dataclass
class OracleCase:
    """Physical parameters of one case (the paper's statement of the problem).

    wall_x / wall_y: boundary kind of the left+right / bottom+top sides (0 or False periodic,
    1 or True no-slip, 2 free-slip); wall_x_hi / wall_y_hi override the right / top side.
    collision: 0 cascaded, 1 single relaxation time.  sigma_model: 0 sigma linear in T, 1
    Langmuir isotherm in the imposed psi.  flow: 0 coupled lattices, 1 interface lattice alone in
    the imposed reversing shear flow (amplitude u0, reversed for time levels >= reverse_step);
    t: time level of the state that step / run start from."""
    nx: int
    ny: int
    wall_x: int = 0
    wall_y: int = 0
    rho_a: float = 1.0
    rho_b: float = 1.0
    mu_a: float = 0.1
    mu_b: float = 0.1
    sigma0: float = 0.0
    dsigma_dT: float = 0.0
    T0: float = 0.0
    gradT_x: float = 0.0
    gradT_y: float = 0.0
    mobility: float = 0.02
    width: float = 4.0
    gx: float = 0.0
    gy: float = 0.0
    rho_ref: float = 0.0
    wall_x_hi: Optional[int] = None
    wall_y_hi: Optional[int] = None
    collision: int = 0
    sigma_model: int = 0
    beta: float = 0.0
    psi0: float = 0.0
    gradpsi_x: float = 0.0
    gradpsi_y: float = 0.0
    flow: int = 0
    reverse_step: int = 0
    u0: float = 0.0
    t: int = 0

    def c(self) -> _Case:
        bx0, bx1 = side_kinds(self.wall_x, self.wall_x_hi)
        by0, by1 = side_kinds(self.wall_y, self.wall_y_hi)
        return _Case(int(self.nx), int(self.ny), bx0, bx1, by0, by1,
                     self.rho_a, self.rho_b, self.mu_a, self.mu_b, self.sigma0, self.dsigma_dT,
                     self.T0, self.gradT_x, self.gradT_y, self.mobility, self.width,
                     self.gx, self.gy, self.rho_ref, int(self.collision), int(self.sigma_model),
                     self.beta, self.psi0, self.gradpsi_x, self.gradpsi_y, int(self.flow),
                     int(self.reverse_step), self.u0, int(self.t))

    @classmethod
    def from_dict(cls, d: dict) -> "OracleCase":
        keys = cls.__dataclass_fields__.keys()
        return cls(**{k: v for k, v in d.items() if k in keys})


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        d = ctypes.c_double
        dp = P(d)
        cp = P(_Case)
        _lib.orc_init.argtypes = [cp, dp, dp, dp, dp, dp, dp]
        _lib.orc_step.argtypes = [cp, dp, dp, dp, dp]
        _lib.orc_step_rows.argtypes = [cp, dp, dp, dp, dp, ctypes.c_int, ctypes.c_int]
        _lib.orc_run.argtypes = [cp, dp, dp, dp, dp, ctypes.c_int]
        _lib.orc_run_float_storage.argtypes = [cp, dp, dp, dp, dp, ctypes.c_int]
        _lib.orc_set_normal_eps.argtypes = [d]
        _lib.orc_set_normal_eps.restype = None
        _lib.orc_get_normal_eps.restype = d
        _lib.orc_fields.argtypes = [cp, dp, dp, dp, dp, dp, dp, dp]
        _lib.orc_node_info.argtypes = [cp, dp, dp, ctypes.c_int, ctypes.c_int, P(_Node)]
        _lib.orc_stencils.argtypes = [cp, dp, dp, dp, dp, dp, dp, dp]
        _lib.orc_fluid_collide.argtypes = [dp, d, d, d, d, d, d, d, d, dp, dp, dp]
        _lib.orc_fluid_source.argtypes = [d, d, d, d, d, d, dp, dp, dp, dp]
        _lib.orc_ace_collide.argtypes = [dp, d, d, d, d, dp, dp, dp]
        _lib.orc_geq.argtypes = [d, d, d, d, dp]
        _lib.orc_feq.argtypes = [d, d, d, d, d, dp]
        _lib.orc_num_threads.restype = ctypes.c_int
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def init(case: OracleCase, phi, p, ux, uy):
    """Equilibrium populations (g-bar, f) from nodal fields, each ``(ny, nx)``."""
    shape = (case.ny, case.nx)
    phi, p, ux, uy = (_f64(np.broadcast_to(a, shape)) for a in (phi, p, ux, uy))
    g = np.empty((9,) + shape)
    f = np.empty((9,) + shape)
    lib().orc_init(case.c(), _ptr(phi), _ptr(p), _ptr(ux), _ptr(uy), _ptr(g), _ptr(f))
    return g, f


def step(case: OracleCase, g, f):
    """One time step; returns the new (g-bar, f)."""
    g, f = _f64(g), _f64(f)
    gn, fn = np.empty_like(g), np.empty_like(f)
    lib().orc_step(case.c(), _ptr(g), _ptr(f), _ptr(gn), _ptr(fn))
    return gn, fn


def step_rows(case: OracleCase, g, f, gn, fn, y0: int, y1: int) -> None:
    """Rows [y0, y1) of one time step written into gn, fn (bounded timing sample)."""
    lib().orc_step_rows(case.c(), _ptr(g), _ptr(f), _ptr(gn), _ptr(fn), int(y0), int(y1))


def run(case: OracleCase, g, f, nsteps: int):
    """nsteps time steps; returns the new (g-bar, f)."""
    g, f = _f64(g).copy(), _f64(f).copy()
    gt, ft = np.empty_like(g), np.empty_like(f)
    lib().orc_run(case.c(), _ptr(g), _ptr(f), _ptr(gt), _ptr(ft), int(nsteps))
    return g, f


def run_float_storage(case: OracleCase, g, f, nsteps: int):
    """As run, with the state rounded to float32 on entry and after every step (FP32 storage
    with FP64 arithmetic); returns the new (g-bar, f)."""
    g, f = _f64(g).copy(), _f64(f).copy()
    gt, ft = np.empty_like(g), np.empty_like(f)
    lib().orc_run_float_storage(case.c(), _ptr(g), _ptr(f), _ptr(gt), _ptr(ft), int(nsteps))
    return g, f


def normal_eps() -> float:
    """The regularisation eps of the interface normal n = grad phi / (|grad phi| + eps)."""
    return float(lib().orc_get_normal_eps())


def set_normal_eps(eps: float) -> None:
    """Set eps (tests of reading R6 only: they restore the default afterwards)."""
    lib().orc_set_normal_eps(float(eps))


def fields(case: OracleCase, g, f) -> dict:
    """phi, corrected p, ux, uy, rho of a state, each ``(ny, nx)``."""
    g, f = _f64(g), _f64(f)
    shape = (case.ny, case.nx)
    out = {k: np.empty(shape) for k in ("phi", "p", "ux", "uy", "rho")}
    lib().orc_fields(case.c(), _ptr(g), _ptr(f), *(_ptr(out[k]) for k in
                                                   ("phi", "p", "ux", "uy", "rho")))
    return out


def node_info(case: OracleCase, g, f, x: int, y: int) -> dict:
    g, f = _f64(g), _f64(f)
    n = _Node()
    lib().orc_node_info(case.c(), _ptr(g), _ptr(f), int(x), int(y), ctypes.byref(n))
    return {k: getattr(n, k) for k, _ in _Node._fields_}


def stencils(case: OracleCase, a) -> dict:
    """Isotropic gradient, Laplacian and Hessian of a nodal field under the case's boundaries."""
    a = _f64(a)
    out = {k: np.empty_like(a) for k in ("gx", "gy", "lap", "hxx", "hyy", "hxy")}
    lib().orc_stencils(case.c(), _ptr(a), *(_ptr(out[k]) for k in
                                            ("gx", "gy", "lap", "hxx", "hyy", "hxy")))
    return out


def fluid_source(Ftx, Fty, Fpx, Fpy, ux, uy, omega):
    omega = _f64(omega)
    sig, mh, dg = np.empty(9), np.empty(9), np.empty(9)
    lib().orc_fluid_source(Ftx, Fty, Fpx, Fpy, ux, uy, _ptr(omega), _ptr(sig), _ptr(mh),
                           _ptr(dg))
    return sig, mh, dg


def fluid_collide(gbar, p, ux, uy, rho, Ftx, Fty, Fpx, Fpy, omega):
    """Post-collision g-bar-tilde (incl. delta g^s) and h-hat at one node."""
    gbar, omega = _f64(gbar), _f64(omega)
    out, h = np.empty(9), np.empty(9)
    lib().orc_fluid_collide(_ptr(gbar), p, ux, uy, rho, Ftx, Fty, Fpx, Fpy, _ptr(omega),
                            _ptr(out), _ptr(h))
    return out, h


def ace_collide(f, ux, uy, jx, jy, omega):
    """Post-collision f-tilde and g-hat at one node; (jx, jy) = M_phi theta n."""
    f, omega = _f64(f), _f64(omega)
    out, gh = np.empty(9), np.empty(9)
    lib().orc_ace_collide(_ptr(f), ux, uy, jx, jy, _ptr(omega), _ptr(out), _ptr(gh))
    return out, gh


def geq(p, ux, uy, rho):
    out = np.empty(9)
    lib().orc_geq(p, ux, uy, rho, _ptr(out))
    return out


def feq(phi, ux, uy, jx=0.0, jy=0.0):
    out = np.empty(9)
    lib().orc_feq(phi, ux, uy, jx, jy, _ptr(out))
    return out
