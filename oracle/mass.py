"""TEST INFRASTRUCTURE: oracle of the mass matrix and its symmetric surrogate.

The mass form m(u, v) = int_Omega u v dx pulled back to the parameter domain is
int u v |det Dphi| dxi (Sec. 8, proof of the mass-matrix corollary); with the
(p+1)-point Gauss rule, M_ij = sum_g w_g |det Dphi(g)| B_i(g) B_j(g)
(``mass_rows``, the C oracle's row loop).

The mass matrix is symmetric but has no kernel, so its surrogate is eq.
DefinitionOfSurrogateMatrixSymmetric (Sec. 5.2), not the kernel-preserving
variant: for x~_i, x~_j in Omega~, A~_ij = Phi~_delta(x~_i) when i <= j (the
diagonal included) and the copy A~_ji when i > j; every other entry is exact.
The (2p+1)^n + 1)/2 stencil functions of the offsets delta >= 0 (colexicographic
order, the centre included) are interpolated exactly as in ``surrogate.py``:
the sampling lattice of Sec. 6 on Omega~ and the not-a-knot B-spline of degree q.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import List

import numpy as np

from . import _lib
from .surrogate import (bspline_basis, center_slot, flat_index, interp_knots, multi_index, offsets, omega_box,
                        sample_indices)


def mass_rows(prob, rows) -> np.ndarray:
    """[len(rows), S] mass rows (stencil slots), exact quadrature."""
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    out = np.zeros((len(rows), prob.S))
    if len(rows) == 0:
        return out
    P = _lib.make_problem(prob)
    rc = _lib.lib().orc_mass_rows(ctypes.byref(P), len(rows), rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  _lib._dptr(out))
    assert rc == 0, rc
    return out


def mass_matrix(prob) -> np.ndarray:
    """Mass matrix in stencil-ELL form, values[s, i] = M_{i, i+delta_s}."""
    return np.ascontiguousarray(mass_rows(prob, np.arange(prob.N)).T)


@dataclass
class MassSetup:
    empty: bool
    k0: List[int]
    k1: List[int]
    samples: List[List[int]]
    q_eff: List[int]
    knots: List[np.ndarray]
    coef: np.ndarray              # [S - c, n_s0, n_s1, (n_s2)] for slots c .. S-1


def mass_surrogate_setup(prob, M: int, q: int) -> MassSetup:
    dim, p, m, S = prob.dim, prob.p, prob.m, prob.S
    c = center_slot(dim, p)
    k0 = [omega_box(p, md)[0] for md in m]
    k1 = [omega_box(p, md)[1] for md in m]
    if any(b < a for a, b in zip(k0, k1)):
        return MassSetup(True, k0, k1, [], [], [], None)
    samples = [sample_indices(a, b, M) for a, b in zip(k0, k1)]
    q_eff = [min(q, len(sd) - 1) for sd in samples]
    knots = [interp_knots(sd, qd) for sd, qd in zip(samples, q_eff)]
    grids = np.meshgrid(*[np.array(sd) for sd in samples], indexing="ij")
    smi = np.stack([g.ravel() for g in grids], axis=1)
    Phi = mass_rows(prob, flat_index(smi, m))[:, c:]                    # slots c .. S-1
    coef = Phi.T.reshape([S - c] + [len(sd) for sd in samples])
    for d in range(dim):
        B = bspline_basis(knots[d], q_eff[d], np.array(samples[d], dtype=np.float64))
        coef = np.moveaxis(coef, 1 + d, 0)
        shp = coef.shape
        coef = np.linalg.solve(B, coef.reshape(shp[0], -1)).reshape(shp)
        coef = np.moveaxis(coef, 0, 1 + d)
    return MassSetup(False, k0, k1, samples, q_eff, knots, coef)


def _evaluate(setup: MassSetup, pos: int, pts: np.ndarray) -> np.ndarray:
    dim = pts.shape[1]
    bases = [bspline_basis(setup.knots[d], setup.q_eff[d], pts[:, d].astype(np.float64)) for d in range(dim)]
    cf = setup.coef[pos]
    if dim == 2:
        return np.einsum("ab,na,nb->n", cf, bases[0], bases[1])
    return np.einsum("abc,na,nb,nc->n", cf, bases[0], bases[1], bases[2])


def mass_surrogate_rows(prob, M: int, q: int, rows, setup: MassSetup = None) -> np.ndarray:
    rows = np.asarray(rows, dtype=np.int64)
    dim, p, m, S = prob.dim, prob.p, np.array(prob.m), prob.S
    c = center_slot(dim, p)
    offs = offsets(dim, p)
    if setup is None:
        setup = mass_surrogate_setup(prob, M, q)
    mi = multi_index(rows, m)
    out = mass_rows(prob, rows)                      # exact everywhere, then overwrite inside Omega~
    if setup.empty:
        return out
    k0, k1 = np.array(setup.k0), np.array(setup.k1)
    in_box = np.all((mi >= k0) & (mi <= k1), axis=1)
    idx = np.nonzero(in_box)[0]
    for s in range(S):
        mj = mi[idx] + offs[s]
        j_in = np.all((mj >= k0) & (mj <= k1), axis=1)
        sel = idx[j_in]
        if len(sel) == 0:
            continue
        if s >= c:      # i <= j: Phi~_delta at x~_i
            out[sel, s] = _evaluate(setup, s - c, mi[sel])
        else:           # i > j: the copy Phi~_{-delta}(x~_j)
            out[sel, s] = _evaluate(setup, S - 1 - s - c, mj[j_in])
    return out


def mass_surrogate_matrix(prob, M: int, q: int) -> np.ndarray:
    setup = mass_surrogate_setup(prob, M, q)
    return np.ascontiguousarray(mass_surrogate_rows(prob, M, q, np.arange(prob.N), setup).T)
