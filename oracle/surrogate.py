"""TEST INFRASTRUCTURE: oracle steps of the symmetric kernel-preserving surrogate.

Follows the paper (Drzisga, Keith & Wohlmuth) in its own order:

1. Sec. 2.2: open uniform knots, B-spline basis, colexicographic numbering.
2. Sec. 3.2, eq. StencilFunction: A_ij = Phi_delta(x~_i) with delta = x~_j - x~_i;
   the exact entries come from (p+1)-point Gauss quadrature (``exact_rows``).
3. Sec. 4, the set Omega~ = [(3p+1)/(2(m-p)), 1-(3p+1)/(2(m-p))]^n on which
   every stencil function is defined.  In 0-based basis indices it is the
   index box [2p, m-2p-1] per direction (``omega_box``).
4. Sec. 6: sampling lattice -- every M-th index of the box from its first
   index, plus the last index when M does not reach it (``sample_indices``);
   stencil values at the samples are exact matrix entries.
5. Sec. 4.1 / Sec. 6: per offset delta, a tensor-product B-spline interpolant
   of degree q through the samples (``surrogate_setup``).  Reading of the
   knot vector (the paper names SciPy's interpolating spline but not its
   knots): the not-a-knot interpolating spline with abscissae = sample
   indices; (q+1)-fold end knots; interior knots at the samples for odd q and
   at sample midpoints for even q; degree lowered to n_s - 1 when there are
   fewer than q + 1 samples.
6. Sec. 5.3, eq. DefinitionOfSurrogateMatrixSymmetricKernel: interpolated
   upper entries inside Omega~, copied lower entries, exact entries elsewhere,
   and the diagonal set to minus the off-diagonal row sum (``surrogate_rows``).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

from . import _lib


# ----------------------------------------------------------------------------
# thin wrappers over the C routines
# ----------------------------------------------------------------------------
def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    rc = _lib.lib().orc_gauss_legendre(n, _lib._dptr(x), _lib._dptr(w))
    assert rc == 0
    return x, w


def open_uniform_knots(p: int, n_el: int) -> np.ndarray:
    t = np.zeros(n_el + 2 * p + 1)
    _lib.lib().orc_open_uniform_knots(p, n_el, _lib._dptr(t))
    return t


def bspline_all(p: int, t: np.ndarray, x: float):
    """Values and derivatives of all B-splines of degree p on knots t at x (C, Cox-de Boor)."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    nb = len(t) - p - 1
    v = np.zeros(nb)
    d = np.zeros(nb)
    rc = _lib.lib().orc_bspline_all(p, len(t), _lib._dptr(t), float(x), _lib._dptr(v), _lib._dptr(d))
    assert rc == 0
    return v, d


def geometry_map(prob, xi: Sequence[float]):
    P = _lib.make_problem(prob)
    xi3 = np.zeros(3)
    xi3[: prob.dim] = xi
    x = np.zeros(3)
    J = np.zeros(9)
    _lib.lib().orc_map(ctypes.byref(P), _lib._dptr(xi3), _lib._dptr(x), _lib._dptr(J))
    return x[: prob.dim], J.reshape(3, 3)[: prob.dim, : prob.dim]


def coefficient(prob, xi: Sequence[float]) -> np.ndarray:
    """K(xi) = kappa(phi(xi)) |det Dphi| Dphi^{-1} Dphi^{-T} (eq. BilinearFormPoissonTensor)."""
    P = _lib.make_problem(prob)
    xi3 = np.zeros(3)
    xi3[: prob.dim] = xi
    K = np.zeros(9)
    _lib.lib().orc_coefficient(ctypes.byref(P), _lib._dptr(xi3), _lib._dptr(K))
    return K.reshape(3, 3)[: prob.dim, : prob.dim]


# ----------------------------------------------------------------------------
# index helpers
# ----------------------------------------------------------------------------
def offsets(dim: int, p: int) -> np.ndarray:
    """[S, dim] offsets delta of each stencil slot, colexicographic (delta_0 fastest)."""
    w = 2 * p + 1
    S = w ** dim
    s = np.arange(S)
    out = np.zeros((S, dim), dtype=np.int64)
    for d in range(dim):
        out[:, d] = (s // w ** d) % w - p
    return out


def center_slot(dim: int, p: int) -> int:
    return ((2 * p + 1) ** dim - 1) // 2


def multi_index(rows: np.ndarray, m: Sequence[int]) -> np.ndarray:
    rows = np.asarray(rows, dtype=np.int64)
    out = np.zeros((len(rows), len(m)), dtype=np.int64)
    rem = rows.copy()
    for d, md in enumerate(m):
        out[:, d] = rem % md
        rem //= md
    return out


def flat_index(mi: np.ndarray, m: Sequence[int]) -> np.ndarray:
    out = np.zeros(mi.shape[0], dtype=np.int64)
    stride = 1
    for d, md in enumerate(m):
        out += mi[:, d] * stride
        stride *= md
    return out


# ----------------------------------------------------------------------------
# exact (Gauss) matrix
# ----------------------------------------------------------------------------
def exact_rows(prob, rows) -> np.ndarray:
    """[len(rows), S] exact quadrature rows (stencil slots)."""
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    S = prob.S
    out = np.zeros((len(rows), S))
    if len(rows) == 0:
        return out
    P = _lib.make_problem(prob)
    rc = _lib.lib().orc_exact_rows(ctypes.byref(P), len(rows),
                                   rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _lib._dptr(out))
    assert rc == 0, rc
    return out


def exact_matrix(prob) -> np.ndarray:
    """Exact matrix in stencil-ELL form, values[s, i] = A_{i, i+delta_s}."""
    return np.ascontiguousarray(exact_rows(prob, np.arange(prob.N)).T)


def elementwise_dense(prob) -> np.ndarray:
    """Dense N x N matrix by the textbook element-by-element loop (tiny meshes)."""
    N = prob.N
    A = np.zeros((N, N))
    P = _lib.make_problem(prob)
    rc = _lib.lib().orc_elementwise_dense(ctypes.byref(P), _lib._dptr(A))
    assert rc == 0, rc
    return A


def ell_to_dense(values: np.ndarray, prob) -> np.ndarray:
    N, m = prob.N, prob.m
    A = np.zeros((N, N))
    mi = multi_index(np.arange(N), m)
    for s, delta in enumerate(offsets(prob.dim, prob.p)):
        mj = mi + delta
        ok = np.all((mj >= 0) & (mj < np.array(m)), axis=1)
        j = flat_index(mj[ok], m)
        A[np.arange(N)[ok], j] = values[s, ok]
    return A


# ----------------------------------------------------------------------------
# Omega~ and the sampling lattice
# ----------------------------------------------------------------------------
def omega_box(p: int, m: int):
    """0-based basis indices k with midpoint x~_k inside Omega~ (Sec. 4): [2p, m-2p-1].

    Returns (k0, k1); the box is empty when k1 < k0.
    """
    return 2 * p, m - 2 * p - 1


def sample_indices(k0: int, k1: int, M: int) -> List[int]:
    """Every M-th index from k0, plus k1 when M does not land on it (Sec. 6)."""
    s = list(range(k0, k1 + 1, M))
    if s[-1] != k1:
        s.append(k1)
    return s


# ----------------------------------------------------------------------------
# 1-D B-spline interpolation (Sec. 4.1)
# ----------------------------------------------------------------------------
def interp_knots(t: Sequence[float], q: int) -> np.ndarray:
    """Not-a-knot knot vector of degree q through abscissae t (see module docstring)."""
    t = np.asarray(t, dtype=np.float64)
    n = len(t)
    assert 0 <= q <= n - 1
    if q % 2 == 1:
        k2 = (q + 1) // 2
        inner = t[k2: n - k2]
    else:
        k2 = q // 2
        mids = 0.5 * (t[1:] + t[:-1])
        inner = mids[k2: (n - 1) - k2]
    return np.concatenate([np.full(q + 1, t[0]), inner, np.full(q + 1, t[-1])])


def bspline_basis(knots: np.ndarray, q: int, x: np.ndarray) -> np.ndarray:
    """[len(x), nb] values of all degree-q B-splines on `knots` at points x.

    Cox-de Boor recursion, N_{i,0} = 1 on [t_i, t_{i+1}); x equal to the last
    knot belongs to the last non-empty interval; 0/0 read as 0.  A knot vector
    with no non-empty interval (one sample, q = 0) has the single basis
    function 1: the interpolant through one sample is that constant.
    """
    knots = np.asarray(knots, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    nt = len(knots)
    nb = nt - q - 1
    nonempty = np.nonzero(knots[1:] > knots[:-1])[0]
    if len(nonempty) == 0:
        # a single abscissa: degree 0 with one basis function, the constant 1
        assert q == 0 and nb == 1
        return np.ones((len(x), 1))
    last = nonempty[-1]
    N = np.zeros((len(x), nt - 1))
    for i in range(nt - 1):
        if knots[i] < knots[i + 1]:
            inside = (knots[i] <= x) & (x < knots[i + 1])
            if i == last:
                inside |= (x == knots[i + 1])
            N[:, i] = inside
    for k in range(1, q + 1):
        Nk = np.zeros((len(x), nt - 1 - k))
        for i in range(nt - 1 - k):
            d1 = knots[i + k] - knots[i]
            d2 = knots[i + k + 1] - knots[i + 1]
            a = (x - knots[i]) / d1 * N[:, i] if d1 > 0 else 0.0
            b = (knots[i + k + 1] - x) / d2 * N[:, i + 1] if d2 > 0 else 0.0
            Nk[:, i] = a + b
        N = Nk
    assert N.shape[1] == nb
    return N


# ----------------------------------------------------------------------------
# surrogate setup: samples, stencil values at samples, coefficients
# ----------------------------------------------------------------------------
@dataclass
class SurrogateSetup:
    empty: bool                     # True when Omega~ has no index in some direction
    k0: List[int]
    k1: List[int]
    samples: List[List[int]]        # sample indices per direction
    q_eff: List[int]
    knots: List[np.ndarray]
    coef: Optional[np.ndarray]      # [S_up, n_s(dir 0), n_s(dir 1), (n_s(dir 2))] spline coefficients
    upper_slots: np.ndarray         # slot numbers s > center, in order


def surrogate_setup(prob, M: int, q: int) -> SurrogateSetup:
    dim, p, m = prob.dim, prob.p, prob.m
    S = prob.S
    c = center_slot(dim, p)
    upper = np.arange(c + 1, S)
    k0 = [omega_box(p, md)[0] for md in m]
    k1 = [omega_box(p, md)[1] for md in m]
    if any(b < a for a, b in zip(k0, k1)):
        return SurrogateSetup(True, k0, k1, [], [], [], None, upper)
    samples = [sample_indices(a, b, M) for a, b in zip(k0, k1)]
    q_eff = [min(q, len(sd) - 1) for sd in samples]
    knots = [interp_knots(sd, qd) for sd, qd in zip(samples, q_eff)]

    # exact stencil values at every sample point: Phi_delta(x~^s) = A_{s, s+delta}
    grids = np.meshgrid(*[np.array(sd) for sd in samples], indexing="ij")   # grids[d][a0, a1, ...]
    smi = np.stack([g.ravel() for g in grids], axis=1)                      # [n_samples, dim], a0 slowest
    srows = flat_index(smi, m)
    Phi = exact_rows(prob, srows)[:, upper]                                 # [n_samples, S_up]
    ns = [len(sd) for sd in samples]
    Phi = Phi.T.reshape([len(upper)] + ns)                                  # [S_up, a0, a1, (a2)]

    # solve the tensor collocation system direction by direction
    coef = Phi.copy()
    for d in range(dim):
        B = bspline_basis(knots[d], q_eff[d], np.array(samples[d], dtype=np.float64))   # [n_s, n_s]
        coef = np.moveaxis(coef, 1 + d, 0)
        shp = coef.shape
        coef = np.linalg.solve(B, coef.reshape(shp[0], -1)).reshape(shp)
        coef = np.moveaxis(coef, 0, 1 + d)
    return SurrogateSetup(False, k0, k1, samples, q_eff, knots, coef, upper)


def _evaluate(setup: SurrogateSetup, slot_pos: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Surrogate stencil function of upper slot index `slot_pos` (position in upper_slots)
    evaluated at index points pts [n, dim]."""
    dim = pts.shape[1]
    bases = [bspline_basis(setup.knots[d], setup.q_eff[d], pts[:, d].astype(np.float64)) for d in range(dim)]
    cf = setup.coef[slot_pos]                                  # [n, a0, a1, (a2)]
    if dim == 2:
        return np.einsum("nab,na,nb->n", cf, bases[0], bases[1])
    return np.einsum("nabc,na,nb,nc->n", cf, bases[0], bases[1], bases[2])


# ----------------------------------------------------------------------------
# surrogate rows (eq. DefinitionOfSurrogateMatrixSymmetricKernel)
# ----------------------------------------------------------------------------
def surrogate_rows(prob, M: int, q: int, rows, setup: Optional[SurrogateSetup] = None) -> np.ndarray:
    rows = np.asarray(rows, dtype=np.int64)
    dim, p, m = prob.dim, prob.p, np.array(prob.m)
    S = prob.S
    c = center_slot(dim, p)
    offs = offsets(dim, p)
    if setup is None:
        setup = surrogate_setup(prob, M, q)
    mi = multi_index(rows, m)
    out = np.zeros((len(rows), S))

    if setup.empty:
        in_box = np.zeros(len(rows), dtype=bool)
    else:
        k0 = np.array(setup.k0)
        k1 = np.array(setup.k1)
        in_box = np.all((mi >= k0) & (mi <= k1), axis=1)

    # exact rows are needed for rows outside Omega~ and for rows with a neighbour outside it
    if setup.empty:
        need_exact = np.ones(len(rows), dtype=bool)
    else:
        need_exact = ~np.all((mi - p >= k0) & (mi + p <= k1), axis=1)
    ex = exact_rows(prob, rows[need_exact])
    out[need_exact] = ex

    if not setup.empty and np.any(in_box):
        idx = np.nonzero(in_box)[0]
        for s in range(S):
            if s == c:
                continue
            mj = mi[idx] + offs[s]
            j_in = np.all((mj >= k0) & (mj <= k1), axis=1)
            sel = idx[j_in]
            if len(sel) == 0:
                continue
            if s > c:      # i < j: surrogate stencil function of delta at x~_i
                vals = _evaluate(setup, np.full(len(sel), s - c - 1), mi[sel])
            else:          # i > j: copy of the (j, i) entry = Phi~_{-delta}(x~_j)
                su = S - 1 - s
                vals = _evaluate(setup, np.full(len(sel), su - c - 1), mj[j_in])
            out[sel, s] = vals
            # entries with j outside Omega~ keep their exact value

    # kernel-preserving diagonal on every row (the equation's i = j case)
    valid = np.ones((len(rows), S), dtype=bool)
    for s in range(S):
        mj = mi + offs[s]
        valid[:, s] = np.all((mj >= 0) & (mj < m), axis=1)
    off = np.where(valid, out, 0.0)
    off[:, c] = 0.0
    out[:, c] = -off.sum(axis=1)
    out[~valid] = 0.0
    return out


def surrogate_matrix(prob, M: int, q: int) -> np.ndarray:
    """Surrogate matrix in stencil-ELL form, values[s, i]."""
    setup = surrogate_setup(prob, M, q)
    return np.ascontiguousarray(surrogate_rows(prob, M, q, np.arange(prob.N), setup).T)
