"""Seeded synthetic workloads shared by the tests, the benchmark and the oracle.

This module only *describes* problems (mesh sizes, degree, which geometry map
and which diffusion coefficient, with their parameters) and draws seeded
random vectors.  It holds none of the method's arithmetic: the oracle
(``oracle/``) and the CUDA library (``paper_1904_06971_gb300``) each turn a
``Problem`` into their own input structures.

Workload recipe (stand-ins for the paper's Poisson experiments, Sec. 7.3):
smooth, non-affine single-patch maps of the unit square / cube onto itself,
x_a = xi_a + amp * prod_j sin(pi xi_j), and smooth diffusion coefficients
evaluated at the physical point.  Right-hand sides are discrete load vectors
f_i ~ U[-1, 1]; SpMV inputs are x_i ~ N(0, 1); all drawn from
``numpy.random.default_rng(seed)`` with seed 0 unless stated.
"""
from __future__ import annotations

from dataclasses import dataclass, replace
from typing import Optional, Tuple

import numpy as np


@dataclass(frozen=True)
class Problem:
    dim: int
    p: int
    n_el: Tuple[int, ...]
    map_kind: str = "identity"          # identity | affine | sinprod
    map_amp: float = 0.0
    affine: Optional[Tuple[float, ...]] = None   # 3x3 row-major matrix then 3-vector offset
    kappa_kind: str = "const"           # const | sin2d | expsin3d | poly | bspline3
    kappa_a: float = 1.0
    kappa_b: float = 0.0
    kappa_deg: int = 0
    kappa_poly: Optional[Tuple[float, ...]] = None
    kappa_nctrl: Optional[Tuple[int, ...]] = None    # bspline3: control values per direction
    kappa_ctrl: Optional[Tuple[float, ...]] = None   # bspline3: c[a + n0 (b + n1 c)]

    @property
    def m(self) -> Tuple[int, ...]:
        return tuple(e + self.p for e in self.n_el)

    @property
    def N(self) -> int:
        return int(np.prod(self.m))

    @property
    def S(self) -> int:
        return (2 * self.p + 1) ** self.dim

    @property
    def nnz(self) -> int:
        """Structural nonzeros of the banded tensor pattern: prod_d (m_d(2p+1) - p(p+1))."""
        return int(np.prod([mm * (2 * self.p + 1) - self.p * (self.p + 1) for mm in self.m]))


@dataclass(frozen=True)
class Workload:
    name: str
    problem: Problem
    M: int
    q: int
    dtype: str          # "f64" or "f32": storage type of the matrix values
    seed: int = 0


# 2D: unit square mapped by x = xi + 0.05 sin(pi xi) sin(pi eta) (both components),
# kappa = 1 + 0.5 sin(2 pi x) sin(2 pi y); p = 2, 32 x 32 elements; M = 4, q = 3.
CFG_2D_P2 = Workload(
    "2d_p2_32x32_M4_q3",
    Problem(dim=2, p=2, n_el=(32, 32), map_kind="sinprod", map_amp=0.05,
            kappa_kind="sin2d", kappa_a=1.0, kappa_b=0.5),
    M=4, q=3, dtype="f64")

# 3D: x_i = xi_i + 0.03 prod_j sin(pi xi_j), kappa = exp(0.5 sin(2 pi x) cos(2 pi y) sin(2 pi z));
# p = 3, 64^3 elements; M = 8, q = 3; FP64 values.
CFG_3D_P3 = Workload(
    "3d_p3_64cube_M8_q3",
    Problem(dim=3, p=3, n_el=(64, 64, 64), map_kind="sinprod", map_amp=0.03,
            kappa_kind="expsin3d", kappa_b=0.5),
    M=8, q=3, dtype="f64")

# 3D, p = 4, 96^3 elements (10^6 DoFs, 729-point stencils, 6.8e8 nnz), same map family;
# M = 8, q = 3; FP64 values: the largest single-patch workload, timed at the paper's precision.
CFG_3D_P4_F64 = Workload(
    "3d_p4_96cube_M8_q3",
    Problem(dim=3, p=4, n_el=(96, 96, 96), map_kind="sinprod", map_amp=0.03,
            kappa_kind="expsin3d", kappa_b=0.5),
    M=8, q=3, dtype="f64")

# 3D precision case: same map family, p = 4, 96^3 elements; M = 8, q = 3; FP32 values.
CFG_3D_P4 = Workload(
    "3d_p4_96cube_M8_q3_f32",
    Problem(dim=3, p=4, n_el=(96, 96, 96), map_kind="sinprod", map_amp=0.03,
            kappa_kind="expsin3d", kappa_b=0.5),
    M=8, q=3, dtype="f32")

# Smaller member of the p = 3 family for profiler captures (values 218 MB > L2).
CFG_3D_P3_40 = Workload(
    "3d_p3_40cube_M8_q3",
    Problem(dim=3, p=3, n_el=(40, 40, 40), map_kind="sinprod", map_amp=0.03,
            kappa_kind="expsin3d", kappa_b=0.5),
    M=8, q=3, dtype="f64")

def lognormal_ctrl(nctrl: Tuple[int, ...], seed: int = 0, sigma: float = 0.25) -> Tuple[float, ...]:
    """Control values c ~ exp(N(0, sigma)) of a B-spline diffusion coefficient, colexicographic."""
    rng = np.random.default_rng(seed)
    return tuple(float(v) for v in np.exp(rng.normal(0.0, sigma, size=int(np.prod(nctrl)))))


# Differentiation case: p = 3, 48^3 elements, the 3-D sine-product map, and kappa a cubic
# B-spline on the physical unit cube with 16^3 control values ~ exp(N(0, 0.25)); M = 8, q = 3.
CFG_3D_P3_BSPLINE = Workload(
    "3d_p3_48cube_bspline16_M8_q3",
    Problem(dim=3, p=3, n_el=(48, 48, 48), map_kind="sinprod", map_amp=0.03,
            kappa_kind="bspline3", kappa_nctrl=(16, 16, 16), kappa_ctrl=lognormal_ctrl((16, 16, 16), seed=0)),
    M=8, q=3, dtype="f64")

# Smaller member of the p = 4 FP32 family for profiler captures (values 410 MB > L2).
CFG_3D_P4_48 = Workload(
    "3d_p4_48cube_M8_q3_f32",
    Problem(dim=3, p=4, n_el=(48, 48, 48), map_kind="sinprod", map_amp=0.03,
            kappa_kind="expsin3d", kappa_b=0.5),
    M=8, q=3, dtype="f32")

# Smaller member of the p = 4 FP64 family for profiler captures (values 820 MB > L2).
CFG_3D_P4_48_F64 = Workload(
    "3d_p4_48cube_M8_q3",
    Problem(dim=3, p=4, n_el=(48, 48, 48), map_kind="sinprod", map_amp=0.03,
            kappa_kind="expsin3d", kappa_b=0.5),
    M=8, q=3, dtype="f64")

WORKLOADS = {w.name: w for w in (CFG_2D_P2, CFG_3D_P3, CFG_3D_P4_F64, CFG_3D_P4, CFG_3D_P3_40, CFG_3D_P3_BSPLINE,
                                  CFG_3D_P4_48, CFG_3D_P4_48_F64)}


def scaled(w: Workload, n_el: Tuple[int, ...], M: Optional[int] = None, p: Optional[int] = None) -> Workload:
    """Same map / coefficient family at another mesh size (small parity cases)."""
    prob = replace(w.problem, n_el=tuple(n_el), p=(p if p is not None else w.problem.p))
    return replace(w, name=f"{w.name}@{'x'.join(map(str, n_el))}", problem=prob,
                   M=(M if M is not None else w.M))


def rhs_vector(N: int, seed: int = 0) -> np.ndarray:
    """Discrete load vector f_i ~ U[-1, 1]."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=N)


def normal_vector(N: int, seed: int = 0) -> np.ndarray:
    """SpMV input x_i ~ N(0, 1)."""
    return np.random.default_rng(seed).standard_normal(N)


def sample_rows(N: int, k: int, seed: int = 0) -> np.ndarray:
    """k distinct row indices, sorted (for sampled parity checks at full size)."""
    rng = np.random.default_rng(seed)
    k = min(k, N)
    return np.sort(rng.choice(N, size=k, replace=False)).astype(np.int64)


def random_problem(rng: np.random.Generator, dim: int, p: int, n_el_range=(5, 12),
                   amp_max: float = 0.05) -> Problem:
    """A small random sine-product patch (used by the randomized parity tests)."""
    n_el = tuple(int(rng.integers(n_el_range[0], n_el_range[1] + 1)) for _ in range(dim))
    amp = float(rng.uniform(0.0, amp_max))
    if dim == 2:
        return Problem(dim=2, p=p, n_el=n_el, map_kind="sinprod", map_amp=amp,
                       kappa_kind="sin2d", kappa_a=1.0, kappa_b=float(rng.uniform(0, 0.5)))
    return Problem(dim=3, p=p, n_el=n_el, map_kind="sinprod", map_amp=amp,
                   kappa_kind="expsin3d", kappa_b=float(rng.uniform(0, 0.5)))


def batch_items(n2d: int = 192, n3d: int = 64, seed: int = 0):
    """The batching workload: n2d 2-D patches (p in 2..5, 16..256 elements per direction)
    and n3d 3-D patches (p in 2..4, 8..48 elements per direction), uniform random; each
    with its own sine-product map (amplitude U[0, 0.05]) and coefficient (2-D:
    1 + b sin sin, 3-D: exp(b sin cos sin), b ~ U[0, 0.5]); M in {4, 8}, q = 3.
    Returns a list of (Problem, M, q)."""
    rng = np.random.default_rng(seed)
    items = []
    for k in range(n2d + n3d):
        if k < n2d:
            p = int(rng.integers(2, 6))
            n_el = tuple(int(rng.integers(16, 257)) for _ in range(2))
            amp, b = float(rng.uniform(0.0, 0.05)), float(rng.uniform(0.0, 0.5))
            prob = Problem(dim=2, p=p, n_el=n_el, map_kind="sinprod", map_amp=amp, kappa_kind="sin2d",
                           kappa_a=1.0, kappa_b=b)
        else:
            p = int(rng.integers(2, 5))
            n_el = tuple(int(rng.integers(8, 49)) for _ in range(3))
            amp, b = float(rng.uniform(0.0, 0.05)), float(rng.uniform(0.0, 0.5))
            prob = Problem(dim=3, p=p, n_el=n_el, map_kind="sinprod", map_amp=amp, kappa_kind="expsin3d", kappa_b=b)
        M = int(rng.choice([4, 8]))
        items.append((prob, M, 3))
    return items
