"""TEST INFRASTRUCTURE: stencil SpMV, Dirichlet reduction and CG for the oracle.

y = A x for a matrix in stencil-ELL form (eq. DiscreteVariationalProblems,
A u = f), homogeneous Dirichlet elimination A_II u_I = f_I (Remark in Sec. 6,
eq. BlockSystem) and plain conjugate gradients on the reduced system.
"""
from __future__ import annotations

import numpy as np

from .surrogate import offsets, multi_index, flat_index


def apply(values: np.ndarray, prob, x: np.ndarray) -> np.ndarray:
    """y_i = sum_s values[s, i] x[i + delta_s] over in-range neighbours."""
    N, m = prob.N, np.array(prob.m)
    x = np.asarray(x, dtype=np.float64)
    mi = multi_index(np.arange(N), m)
    y = np.zeros(N)
    for s, delta in enumerate(offsets(prob.dim, prob.p)):
        mj = mi + delta
        ok = np.all((mj >= 0) & (mj < m), axis=1)
        j = flat_index(mj[ok], m)
        y[ok] += values[s, ok].astype(np.float64) * x[j]
    return y


def interior_dofs(prob) -> np.ndarray:
    """Indices of basis functions that vanish on the boundary (every i_d in [1, m_d - 2])."""
    m = np.array(prob.m)
    mi = multi_index(np.arange(prob.N), m)
    return np.nonzero(np.all((mi >= 1) & (mi <= m - 2), axis=1))[0]


def cg(values: np.ndarray, prob, f: np.ndarray, tol: float = 1e-12, maxiter: int = 100000):
    """Solve A_II u_I = f_I (homogeneous Dirichlet) by unpreconditioned CG in FP64.

    Returns (u [N] with zeros on Dirichlet dofs, iterations, final relative residual).
    """
    I = interior_dofs(prob)

    def matvec(vI):
        v = np.zeros(prob.N)
        v[I] = vI
        return apply(values, prob, v)[I]

    b = np.asarray(f, dtype=np.float64)[I]
    u = np.zeros_like(b)
    r = b - matvec(u)
    d = r.copy()
    rr = r @ r
    bnorm = np.sqrt(b @ b)
    it = 0
    while np.sqrt(rr) > tol * bnorm and it < maxiter:
        Ad = matvec(d)
        alpha = rr / (d @ Ad)
        u += alpha * d
        r -= alpha * Ad
        rr_new = r @ r
        d = r + (rr_new / rr) * d
        rr = rr_new
        it += 1
    out = np.zeros(prob.N)
    out[I] = u
    return out, it, np.sqrt(rr) / bnorm


def relative_entry_error(X: np.ndarray, ref: np.ndarray) -> float:
    """max |X - ref| / max |ref| over all stored entries."""
    X = np.asarray(X, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(X - ref)) / np.max(np.abs(ref)))
