"""TEST INFRASTRUCTURE: ctypes loader for the plain-C FP64 oracle (iga_oracle.c).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may use
this package.  It compiles iga_oracle.c with the host C compiler on first use
(or via ``build()``) into ``oracle/_build/`` and shares no code with the CUDA
path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "iga_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAP_KINDS = {"identity": 0, "affine": 1, "sinprod": 2}
KAPPA_KINDS = {"const": 0, "sin2d": 1, "expsin3d": 2, "poly": 3, "bspline3": 4}


class OrcProblem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32),
        ("p", ctypes.c_int32),
        ("n_el", ctypes.c_int32 * 3),
        ("map_kind", ctypes.c_int32),
        ("kappa_kind", ctypes.c_int32),
        ("kappa_deg", ctypes.c_int32),
        ("map_amp", ctypes.c_double),
        ("affine", ctypes.c_double * 12),
        ("kappa_a", ctypes.c_double),
        ("kappa_b", ctypes.c_double),
        ("kappa_poly", ctypes.c_double * 64),
        ("kappa_nctrl", ctypes.c_int32 * 3),
        ("kappa_ctrl", ctypes.POINTER(ctypes.c_double)),
    ]


def build(force: bool = False) -> str:
    """Compile iga_oracle.c into oracle/_build/liboracle.so (host compiler)."""
    with _lock:
        if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
            return _SO
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True, capture_output=True)
        os.replace(tmp, _SO)
        return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.POINTER(OrcProblem)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_gauss_legendre.argtypes = [ctypes.c_int, dp, dp]
        L.orc_open_uniform_knots.argtypes = [ctypes.c_int, ctypes.c_int, dp]
        L.orc_bspline_all.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_double, dp, dp]
        L.orc_map.argtypes = [P, dp, dp, dp]
        L.orc_kappa.argtypes = [P, dp]
        L.orc_kappa.restype = ctypes.c_double
        L.orc_coefficient.argtypes = [P, dp, dp]
        L.orc_num_dofs.argtypes = [P]
        L.orc_num_dofs.restype = ctypes.c_int64
        L.orc_num_slots.argtypes = [P]
        L.orc_exact_rows.argtypes = [P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), dp]
        L.orc_mass_rows.argtypes = [P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), dp]
        L.orc_elementwise_dense.argtypes = [P, dp]
        L.orc_manufactured_load.argtypes = [P, ctypes.c_int, dp, dp]
        L.orc_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_problem(prob) -> OrcProblem:
    """Convert a neutral problem description (see iga_workloads.Problem) to the C struct."""
    s = OrcProblem()
    s.dim = prob.dim
    s.p = prob.p
    for d in range(3):
        s.n_el[d] = prob.n_el[d] if d < prob.dim else 1
    s.map_kind = MAP_KINDS[prob.map_kind]
    s.map_amp = float(prob.map_amp)
    aff = list(prob.affine) if prob.affine is not None else [1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0]
    for k in range(12):
        s.affine[k] = float(aff[k])
    s.kappa_kind = KAPPA_KINDS[prob.kappa_kind]
    s.kappa_a = float(prob.kappa_a)
    s.kappa_b = float(prob.kappa_b)
    s.kappa_deg = int(prob.kappa_deg)
    coef = list(prob.kappa_poly) if prob.kappa_poly is not None else []
    for k in range(64):
        s.kappa_poly[k] = float(coef[k]) if k < len(coef) else 0.0
    if prob.kappa_kind == "bspline3":
        nc = list(prob.kappa_nctrl) + [1] * (3 - len(prob.kappa_nctrl))
        for d in range(3):
            s.kappa_nctrl[d] = int(nc[d])
        ctrl = np.ascontiguousarray(np.asarray(prob.kappa_ctrl, dtype=np.float64))
        assert ctrl.size == int(np.prod(nc[: prob.dim]))
        s._ctrl_keepalive = ctrl                  # the struct only holds a pointer
        s.kappa_ctrl = _dptr(ctrl)
    return s


def num_threads() -> int:
    return int(lib().orc_num_threads())
