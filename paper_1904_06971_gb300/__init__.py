"""Python binding of libiga: GPU exact / surrogate IGA stiffness assembly and stencil SpMV.

Thin ctypes marshalling over the C ABI in ``include/iga.h``; every step of the
computation runs in the CUDA kernels of ``csrc/``.  PyTorch supplies device
memory and streams.  There is no CPU fallback: if the in-tree ``libiga.so``
cannot be built or loaded, every call raises.

Problems are described by any object with the attributes ``dim, p, n_el,
map_kind ('identity'|'affine'|'sinprod'), map_amp, affine, kappa_kind
('const'|'sin2d'|'expsin3d'|'poly'), kappa_a, kappa_b, kappa_deg,
kappa_poly``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading
from typing import Optional

import numpy as np

from . import _build

__all__ = ["IgaError", "Matrix", "assemble_exact", "assemble_surrogate", "assemble_mass", "assemble_mass_surrogate",
           "surrogate_plan", "manufactured_load",
           "kappa_gradient", "stiffness_apply", "assemble_batch", "batch_info", "batch_set_modes", "batch_mode", "batch_release",
           "batch_status", "batch_selftest_timeout", "load", "launch_count",
           "profile_enable", "profile_read", "kernel_names", "set_arithmetic", "get_arithmetic",
           "F64", "F32", "ARITH"]

F64, F32 = 0, 1
ARITH = {"fp64": 0, "df64": 1, "fp32": 2, "bf16x3": 3, "df64_tc": 4}
_MAP = {"identity": 0, "affine": 1, "sinprod": 2}
_KAPPA = {"const": 0, "sin2d": 1, "expsin3d": 2, "poly": 3, "bspline3": 4}
_lock = threading.Lock()
_lib = None


class IgaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libiga error {code}: {msg}")
        self.code = code


class Patch(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("n_el", ctypes.c_int32 * 3)]


class Map(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("amp", ctypes.c_double), ("affine", ctypes.c_double * 12)]


class Kappa(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("deg", ctypes.c_int32), ("a", ctypes.c_double),
                ("b", ctypes.c_double), ("poly", ctypes.c_double * 64), ("nctrl", ctypes.c_int32 * 3),
                ("ctrl", ctypes.c_void_p)]


class BatchItem(ctypes.Structure):
    _fields_ = [("patch", Patch), ("p", ctypes.c_int32), ("map", Map), ("kappa", Kappa), ("M", ctypes.c_int32),
                ("q", ctypes.c_int32), ("domains", ctypes.c_int32)]


def load():
    """Build (if stale) and load the in-tree libiga.so."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        so = _build.build()
        if not os.path.exists(so):
            raise ImportError(f"libiga.so missing at {so}")
        L = ctypes.CDLL(so)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        H = ctypes.c_void_p
        L.iga_assemble_exact.argtypes = [ctypes.POINTER(Patch), ctypes.c_int, ctypes.POINTER(Map),
                                         ctypes.POINTER(Kappa), ctypes.c_int, vp, ctypes.POINTER(H)]
        L.iga_assemble_surrogate.argtypes = [ctypes.POINTER(Patch), ctypes.c_int, ctypes.POINTER(Map),
                                             ctypes.POINTER(Kappa), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             vp, ctypes.POINTER(H)]
        L.iga_assemble_surrogate_domains.argtypes = [ctypes.POINTER(Patch), ctypes.c_int, ctypes.POINTER(Map),
                                                     ctypes.POINTER(Kappa), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                     ctypes.c_int, vp, ctypes.POINTER(H)]
        L.iga_assemble_mass.argtypes = [ctypes.POINTER(Patch), ctypes.c_int, ctypes.POINTER(Map), ctypes.c_int, vp,
                                        ctypes.POINTER(H)]
        L.iga_assemble_mass_surrogate.argtypes = [ctypes.POINTER(Patch), ctypes.c_int, ctypes.POINTER(Map),
                                                  ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(H)]
        P32 = ctypes.POINTER(i32)
        L.iga_surrogate_plan.argtypes = [ctypes.POINTER(Patch), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, P32, P32, P32, P32, P32, P32, ctypes.POINTER(ctypes.c_int)]
        L.iga_kappa_gradient.argtypes = [ctypes.POINTER(Patch), ctypes.c_int, ctypes.POINTER(Map),
                                         ctypes.POINTER(Kappa), ctypes.c_int, ctypes.c_int, vp, vp, vp, vp]
        L.iga_assemble_batch.argtypes = [ctypes.c_int, ctypes.POINTER(BatchItem), ctypes.c_int, vp,
                                         ctypes.POINTER(H)]
        L.iga_batch_info.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_float)]
        L.iga_batch_release.argtypes = []
        L.iga_batch_set_modes.argtypes = [ctypes.c_int, ctypes.c_int]
        L.iga_batch_mode.argtypes = [ctypes.POINTER(ctypes.c_int)] * 3
        L.iga_batch_status.argtypes = [vp]
        L.iga_batch_selftest_timeout.argtypes = [ctypes.c_longlong, vp]
        L.iga_assemble_exact_noalloc.argtypes = [ctypes.POINTER(Patch), ctypes.c_int, ctypes.POINTER(Map),
                                                 ctypes.POINTER(Kappa), ctypes.c_int, vp, vp]
        L.iga_manufactured_load.argtypes = [ctypes.POINTER(Patch), ctypes.c_int, ctypes.POINTER(Map),
                                            ctypes.POINTER(Kappa), ctypes.c_int, vp, vp, vp]
        L.iga_apply.argtypes = [H, vp, vp, vp]
        L.iga_cg.argtypes = [H, vp, vp, ctypes.c_double, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(ctypes.c_double)]
        L.iga_apply_host.argtypes = [H, vp, vp, vp]
        L.iga_matrix_info.argtypes = [H, ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i64),
                                      ctypes.POINTER(i32)]
        L.iga_matrix_values.argtypes = [H, ctypes.POINTER(vp)]
        L.iga_matrix_copy_values.argtypes = [H, vp, ctypes.c_int, vp]
        L.iga_matrix_destroy.argtypes = [H]
        L.iga_launch_count.restype = i64
        L.iga_profile_enable.argtypes = [ctypes.c_int]
        L.iga_profile_read.argtypes = [ctypes.c_int, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double)]
        L.iga_kernel_name.restype = ctypes.c_char_p
        L.iga_kernel_name.argtypes = [ctypes.c_int]
        L.iga_last_error.restype = ctypes.c_char_p
        _lib = L
        return L


def _check(rc: int):
    if rc != 0:
        raise IgaError(rc, load().iga_last_error().decode())


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _structs(prob, ctrl=None):
    pt = Patch()
    pt.dim = int(prob.dim)
    for d in range(3):
        pt.n_el[d] = int(prob.n_el[d]) if d < prob.dim else 1
    mp = Map()
    mp.kind = _MAP[prob.map_kind]
    mp.amp = float(getattr(prob, "map_amp", 0.0))
    aff = getattr(prob, "affine", None) or (1, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0, 0)
    for k in range(12):
        mp.affine[k] = float(aff[k])
    kp = Kappa()
    kp.kind = _KAPPA[prob.kappa_kind]
    kp.deg = int(getattr(prob, "kappa_deg", 0))
    kp.a = float(getattr(prob, "kappa_a", 1.0))
    kp.b = float(getattr(prob, "kappa_b", 0.0))
    poly = getattr(prob, "kappa_poly", None) or ()
    for k in range(64):
        kp.poly[k] = float(poly[k]) if k < len(poly) else 0.0
    if prob.kappa_kind == "bspline3":
        import torch
        nc = list(prob.kappa_nctrl) + [1] * (3 - len(prob.kappa_nctrl))
        for d in range(3):
            kp.nctrl[d] = int(nc[d])
        if ctrl is None:
            ctrl = torch.tensor(prob.kappa_ctrl, dtype=torch.float64, device="cuda")
        if not (ctrl.is_cuda and ctrl.dtype == torch.float64 and ctrl.is_contiguous()
                and ctrl.numel() == int(np.prod(nc[: prob.dim]))):
            raise ValueError("kappa control values must be a contiguous float64 CUDA tensor of prod(nctrl) entries")
        kp.ctrl = ctrl.data_ptr()
        kp._ctrl_keepalive = ctrl                    # the struct only holds the device pointer
    return pt, mp, kp


def _dtype_code(dtype) -> int:
    if dtype in ("f64", F64, np.float64):
        return F64
    if dtype in ("f32", F32, np.float32):
        return F32
    raise ValueError(f"dtype must be 'f64' or 'f32', got {dtype!r}")


class Matrix:
    """A stencil-ELL matrix owned by libiga (values [S][N] on the device)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)
        N, S, nnz, dt = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
        _check(load().iga_matrix_info(self._h, ctypes.byref(N), ctypes.byref(S), ctypes.byref(nnz), ctypes.byref(dt)))
        self.N, self.S, self.nnz, self.dtype_code = N.value, S.value, nnz.value, dt.value

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    @property
    def np_dtype(self):
        return np.float32 if self.dtype_code == F32 else np.float64

    @property
    def torch_dtype(self):
        import torch
        return torch.float32 if self.dtype_code == F32 else torch.float64

    def apply(self, x, y=None, stream=None):
        """y = A x for device tensors x (and optional y) of the matrix dtype."""
        import torch
        if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == self.torch_dtype and x.numel() == self.N
                and x.is_contiguous()):
            raise ValueError("x must be a contiguous CUDA tensor of N elements of the matrix dtype")
        if y is None:
            y = torch.empty_like(x)
        _check(load().iga_apply(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                ctypes.c_void_p(_stream_ptr(stream))))
        return y

    def apply_host(self, x: np.ndarray, y: Optional[np.ndarray] = None, stream=None) -> np.ndarray:
        """y = A x with host arrays (copies inside the call; returns after the stream syncs)."""
        x = np.ascontiguousarray(x, dtype=self.np_dtype)
        if y is None:
            y = np.empty_like(x)
        _check(load().iga_apply_host(self._h, ctypes.c_void_p(x.ctypes.data), ctypes.c_void_p(y.ctypes.data),
                                     ctypes.c_void_p(_stream_ptr(stream))))
        return y

    def values(self, stream=None):
        """A device copy of the values as a torch tensor [S, N]."""
        import torch
        out = torch.empty((self.S, self.N), dtype=self.torch_dtype, device="cuda")
        _check(load().iga_matrix_copy_values(self._h, ctypes.c_void_p(out.data_ptr()), 0,
                                             ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def values_host(self, stream=None) -> np.ndarray:
        out = np.empty((self.S, self.N), dtype=self.np_dtype)
        _check(load().iga_matrix_copy_values(self._h, ctypes.c_void_p(out.ctypes.data), 1,
                                             ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def cg(self, f, tol: float = 1e-10, maxit: int = 100000, stream=None):
        """Solve the Dirichlet-reduced system A_II u_I = f_I on the GPU (iga_cg).

        f: CUDA float64 tensor of N entries.  Returns (u, iterations, relative residual)."""
        import torch
        if not (isinstance(f, torch.Tensor) and f.is_cuda and f.dtype == torch.float64 and f.numel() == self.N
                and f.is_contiguous()):
            raise ValueError("f must be a contiguous CUDA float64 tensor of N elements")
        u = torch.empty_like(f)
        it = ctypes.c_int()
        rel = ctypes.c_double()
        _check(load().iga_cg(self._h, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(u.data_ptr()), float(tol), int(maxit),
                        ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(it), ctypes.byref(rel)))
        return u, it.value, rel.value

    def device_ptr(self) -> int:
        p = ctypes.c_void_p()
        _check(load().iga_matrix_values(self._h, ctypes.byref(p)))
        return p.value

    def destroy(self):
        if self._h is not None and self._h.value:
            _check(load().iga_matrix_destroy(self._h))
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def _keep(mat: "Matrix", kp) -> "Matrix":
    """The matrix holds the control-value tensor its assembly read (kernels may still run)."""
    mat._kappa_ctrl = getattr(kp, "_ctrl_keepalive", None)
    return mat


def assemble_exact(prob, dtype="f64", stream=None, out: Optional[Matrix] = None, kappa_ctrl=None) -> Matrix:
    """Exact Gauss-quadrature stiffness matrix on the GPU (iga_assemble_exact).

    kappa_ctrl: optional float64 CUDA tensor of B-spline control values (kappa kind 'bspline3');
    by default they are copied from the problem description."""
    pt, mp, kp = _structs(prob, kappa_ctrl)
    h = ctypes.c_void_p(out.handle.value if out is not None else None)
    _check(load().iga_assemble_exact(ctypes.byref(pt), int(prob.p), ctypes.byref(mp), ctypes.byref(kp),
                                     _dtype_code(dtype), ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(h)))
    return _keep(out if out is not None else Matrix(h.value), kp)


DOMAINS = {"common": 0, "per_offset": 1}       # IGA_DOMAINS_COMMON / IGA_DOMAINS_PER_OFFSET


def assemble_surrogate(prob, M: int, q: int, dtype="f64", stream=None, out: Optional[Matrix] = None,
                       domains: str = "common", kappa_ctrl=None) -> Matrix:
    """Symmetric kernel-preserving surrogate stiffness matrix on the GPU.

    domains='common' interpolates on Omega~ (iga_assemble_surrogate); 'per_offset'
    on each Omega~_delta (iga_assemble_surrogate_domains)."""
    pt, mp, kp = _structs(prob, kappa_ctrl)
    h = ctypes.c_void_p(out.handle.value if out is not None else None)
    st = ctypes.c_void_p(_stream_ptr(stream))
    if domains == "common":
        _check(load().iga_assemble_surrogate(ctypes.byref(pt), int(prob.p), ctypes.byref(mp), ctypes.byref(kp),
                                             int(M), int(q), _dtype_code(dtype), st, ctypes.byref(h)))
    else:
        _check(load().iga_assemble_surrogate_domains(ctypes.byref(pt), int(prob.p), ctypes.byref(mp),
                                                     ctypes.byref(kp), int(M), int(q), DOMAINS[domains],
                                                     _dtype_code(dtype), st, ctypes.byref(h)))
    return _keep(out if out is not None else Matrix(h.value), kp)


def assemble_mass(prob, dtype="f64", stream=None, out: Optional[Matrix] = None) -> Matrix:
    """Exact Gauss-quadrature mass matrix on the GPU (iga_assemble_mass); the problem's kappa is not used."""
    pt, mp, _ = _structs(dataclasses.replace(prob, kappa_kind="const"))     # the mass form has no kappa
    h = ctypes.c_void_p(out.handle.value if out is not None else None)
    _check(load().iga_assemble_mass(ctypes.byref(pt), int(prob.p), ctypes.byref(mp), _dtype_code(dtype),
                                    ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(h)))
    return out if out is not None else Matrix(h.value)


def assemble_mass_surrogate(prob, M: int, q: int, dtype="f64", stream=None, out: Optional[Matrix] = None) -> Matrix:
    """Symmetric surrogate mass matrix on the common domain (iga_assemble_mass_surrogate)."""
    pt, mp, _ = _structs(dataclasses.replace(prob, kappa_kind="const"))     # the mass form has no kappa
    h = ctypes.c_void_p(out.handle.value if out is not None else None)
    _check(load().iga_assemble_mass_surrogate(ctypes.byref(pt), int(prob.p), ctypes.byref(mp), int(M), int(q),
                                              _dtype_code(dtype), ctypes.c_void_p(_stream_ptr(stream)),
                                              ctypes.byref(h)))
    return out if out is not None else Matrix(h.value)


def surrogate_plan(prob, M: int, q: int, domains: str = "common") -> dict:
    """Sampling plan of a surrogate assembly, computed on the host (iga_surrogate_plan; no GPU needed).

    Returns {"empty": bool, "samples": [per-direction index arrays],
    "domains": [per direction: [(lo, hi, n_samples, q_used) for delta_d = -p..p]]}."""
    pt, _, _ = _structs(dataclasses.replace(prob, kappa_kind="const"))
    p, W = int(prob.p), 2 * int(prob.p) + 1
    cap = max(prob.m) + 1
    samples = np.zeros((3, cap), dtype=np.int32)
    ns = np.zeros(3, dtype=np.int32)
    lo, hi, dns, dq = (np.zeros((3, W), dtype=np.int32) for _ in range(4))
    empty = ctypes.c_int()
    P32 = ctypes.POINTER(ctypes.c_int32)
    ptr = lambda a: a.ctypes.data_as(P32)                                      # noqa: E731
    _check(load().iga_surrogate_plan(ctypes.byref(pt), p, int(M), int(q), DOMAINS[domains], cap, ptr(samples), ptr(ns),
                                     ptr(lo), ptr(hi), ptr(dns), ptr(dq), ctypes.byref(empty)))
    if empty.value:
        return {"empty": True, "samples": [], "domains": []}
    return {"empty": False,
            "samples": [samples[d, :ns[d]].copy() for d in range(prob.dim)],
            "domains": [[(int(lo[d, v]), int(hi[d, v]), int(dns[d, v]), int(dq[d, v])) for v in range(W)]
                        for d in range(prob.dim)]}


def set_arithmetic(dtype, arith: str):
    """Contraction arithmetic for later assemblies with `dtype` values: 'fp64', 'df64' or 'fp32'."""
    _check(load().iga_set_arithmetic(_dtype_code(dtype), ARITH[arith]))


def get_arithmetic(dtype) -> str:
    code = load().iga_get_arithmetic(_dtype_code(dtype))
    return {v: k for k, v in ARITH.items()}[code]


def launch_count() -> int:
    return int(load().iga_launch_count())


def kernel_names():
    L = load()
    return [L.iga_kernel_name(k).decode() for k in range(L.iga_num_kernels())]


def profile_enable(on: bool = True):
    _check(load().iga_profile_enable(1 if on else 0))


def profile_read():
    """{kernel name: (launches, total ms)} since the last read (synchronises the recorded events)."""
    L = load()
    n = L.iga_num_kernels()
    la = (ctypes.c_int64 * n)()
    ms = (ctypes.c_double * n)()
    _check(L.iga_profile_read(n, la, ms))
    return {L.iga_kernel_name(k).decode(): (int(la[k]), float(ms[k])) for k in range(n)}


def manufactured_load(prob, freq: int = 1, stream=None, kappa_ctrl=None):
    """(F, energy) of the manufactured solution u = prod_d sin(freq pi x_d) (iga_manufactured_load):
    F_i = a(u, B_i) as a float64 CUDA tensor of N entries and a(u, u) as a float64 CUDA scalar tensor."""
    import torch
    pt, mp, kp = _structs(prob, kappa_ctrl)
    N = int(np.prod([int(prob.n_el[d]) + int(prob.p) for d in range(prob.dim)]))
    F = torch.empty(N, dtype=torch.float64, device="cuda")
    en = torch.empty((), dtype=torch.float64, device="cuda")
    _check(load().iga_manufactured_load(ctypes.byref(pt), int(prob.p), ctypes.byref(mp), ctypes.byref(kp),
                                        int(freq), ctypes.c_void_p(F.data_ptr()), ctypes.c_void_p(en.data_ptr()),
                                        ctypes.c_void_p(_stream_ptr(stream))))
    return F, en


def kappa_gradient(prob, ybar, x, M: int = 0, q: int = 3, kappa_ctrl=None, stream=None):
    """dL/dc for L = ybar^T A x and the B-spline control values c of kappa (iga_kappa_gradient).

    A is the exact matrix (M = 0) or the common-domain surrogate (M >= 1, q).  ybar, x:
    float64 CUDA tensors of N entries.  Returns a float64 CUDA tensor of prod(nctrl) entries."""
    import torch
    for v in (ybar, x):
        if not (isinstance(v, torch.Tensor) and v.is_cuda and v.dtype == torch.float64 and v.is_contiguous()
                and v.numel() == prob.N):
            raise ValueError("ybar and x must be contiguous float64 CUDA tensors of N entries")
    pt, mp, kp = _structs(prob, kappa_ctrl)
    nc = int(np.prod(prob.kappa_nctrl[: prob.dim])) if prob.kappa_kind == "bspline3" else 1
    grad = torch.empty(nc, dtype=torch.float64, device=ybar.device)
    _check(load().iga_kappa_gradient(ctypes.byref(pt), int(prob.p), ctypes.byref(mp), ctypes.byref(kp), int(M),
                                     int(q), ctypes.c_void_p(ybar.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                     ctypes.c_void_p(grad.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))))
    return grad


def _stiffness_apply_function():
    import torch

    class StiffnessApply(torch.autograd.Function):
        """y = A(c) x for the exact (M = 0) or surrogate (M >= 1) matrix of a B-spline kappa with
        control values c; backward gives A ybar for x and iga_kappa_gradient for c."""

        @staticmethod
        def forward(ctx, ctrl, x, prob, M, q):
            ctrl = ctrl.detach().contiguous()
            x = x.detach().contiguous()
            if M >= 1:
                A = assemble_surrogate(prob, M, q, dtype="f64", kappa_ctrl=ctrl)
            else:
                A = assemble_exact(prob, dtype="f64", kappa_ctrl=ctrl)
            y = A.apply(x)
            ctx.save_for_backward(ctrl, x)
            ctx.A, ctx.prob, ctx.M, ctx.q = A, prob, M, q
            return y

        @staticmethod
        def backward(ctx, ybar):
            ctrl, x = ctx.saved_tensors
            ybar = ybar.contiguous()
            gc = kappa_gradient(ctx.prob, ybar, x, ctx.M, ctx.q, kappa_ctrl=ctrl) if ctx.needs_input_grad[0] else None
            gx = ctx.A.apply(ybar) if ctx.needs_input_grad[1] else None
            return gc, gx, None, None, None

    return StiffnessApply


_STIFFNESS_APPLY = None


def stiffness_apply(ctrl, x, prob, M: int = 0, q: int = 3):
    """Differentiable y = A(kappa_c) x (torch.autograd): gradients for the control values c
    (float64 CUDA tensor) and for x."""
    global _STIFFNESS_APPLY
    if _STIFFNESS_APPLY is None:
        _STIFFNESS_APPLY = _stiffness_apply_function()
    return _STIFFNESS_APPLY.apply(ctrl, x, prob, M, q)


def assemble_batch(items, dtype="f32", stream=None, out=None):
    """Assemble many patches as one CUDA graph (iga_assemble_batch).

    items: sequence of (problem, M, q) or (problem, M, q, domains); M = 0 is the exact
    matrix.  The first call (out=None) creates the matrices eagerly; passing the returned
    list back as `out` replays a cached, autotuned graph of the whole batch."""
    n = len(items)
    arr = (BatchItem * n)()
    keep = []
    for k, it in enumerate(items):
        prob, M, q = it[0], int(it[1]), int(it[2])
        dom = it[3] if len(it) > 3 else "common"
        pt, mp, kp = _structs(prob)
        arr[k].patch, arr[k].p, arr[k].map, arr[k].kappa = pt, int(prob.p), mp, kp
        arr[k].M, arr[k].q, arr[k].domains = M, q, DOMAINS[dom]
        keep.append(kp)
    H = ctypes.c_void_p * n
    handles = H(*[(m.handle.value if out is not None else None) for m in (out or [None] * n)])
    _check(load().iga_assemble_batch(n, arr, _dtype_code(dtype), ctypes.c_void_p(_stream_ptr(stream)), handles))
    if out is not None:
        return out
    mats = [Matrix(h) for h in handles]
    for m, kp in zip(mats, keep):
        _keep(m, kp)
    return mats


def batch_release():
    """Destroy every cached batch graph (the next batch call re-tunes)."""
    _check(load().iga_batch_release())


def batch_set_modes(branches=True, persistent=True):
    """Restrict the batch autotuner to branch graphs and/or persistent-kernel graphs."""
    _check(load().iga_batch_set_modes(int(bool(branches)), int(bool(persistent))))


def batch_mode():
    """(persistent, resident blocks per SM, items per claim) of this thread's last batch call."""
    p, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().iga_batch_mode(ctypes.byref(p), ctypes.byref(b), ctypes.byref(c)))
    return bool(p.value), b.value, c.value


def batch_status(stream=None):
    """Synchronise the stream; raise IgaError(IGA_ETIMEOUT) if the last persistent replay's wait gave up."""
    _check(load().iga_batch_status(ctypes.c_void_p(_stream_ptr(stream))))


def batch_selftest_timeout(limit_us=20000, stream=None) -> int:
    """Run the persistent kernel on a work item whose dependency never completes; returns the status code
    (IGA_ETIMEOUT = -5 when the bounded wait gave up as it should)."""
    return int(load().iga_batch_selftest_timeout(int(limit_us), ctypes.c_void_p(_stream_ptr(stream))))


def batch_info():
    """(branches, kernels per replay, from cache, tuned replay ms) of this thread's last batch call."""
    b, k, c, ms = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int(), ctypes.c_float()
    _check(load().iga_batch_info(ctypes.byref(b), ctypes.byref(k), ctypes.byref(c), ctypes.byref(ms)))
    return b.value, k.value, bool(c.value), ms.value
