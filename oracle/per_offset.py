"""TEST INFRASTRUCTURE: oracle of the surrogate with per-offset interpolation domains.

Sec. 3.2 (the paragraph after the cardinal-basis figure) observes that the
stencil function Phi_delta of an offset delta is defined wherever both basis
functions of the pair are cardinal, a set Omega~_delta that depends on delta;
Sec. 4 then works on the intersection Omega~ of all of them, noting that every
result carries over to Omega~_delta with one interpolation operator per delta.
This module is that per-offset variant of eq.
DefinitionOfSurrogateMatrixSymmetricKernel (Sec. 5.3), in the paper's order:

1. Sec. 2.2: a B-spline of the open uniform knot vector is cardinal (a
   translate of the uniform B-spline) when its p + 2 knots are distinct, i.e.
   for 0-based indices k in [p, m-p-1] per direction (``cardinal_range``).
2. Omega~_delta in indices: the k with k and k + delta_d both cardinal in
   every direction d (``offset_domain``).  The union of all of them is the
   cardinal box, their intersection the box [2p, m-2p-1] of Sec. 4.
3. Sec. 6 sampling, applied to every Omega~_delta on one shared lattice,
   every M-th index from the first cardinal index p: an offset samples the two
   ends k0, k1 of its own domain and the lattice points at least M/2 away from
   both ends (``offset_samples``), so its knot spacing stays between M/2 and
   3M/2 -- quasi-uniform as Sec. 4.1 asks of the knot vector.  All offsets
   together sample the lattice and the p + 1 first and last cardinal indices
   (the ends of every Omega~_delta, ``union_samples``): those are the rows
   assembled by quadrature.
4. Sec. 4.1: per upper offset, the tensor-product not-a-knot B-spline
   interpolant of degree q through its own sample grid (same knot reading as
   ``surrogate.interp_knots``; degree lowered to n_s - 1 with fewer than
   q + 1 samples).
5. Sec. 5.3 with Omega~_delta for Omega~: for i < j with i, j both cardinal,
   A~_ij = Phi~_delta(x~_i) (delta = x~_j - x~_i); for i > j, the copy
   Phi~_{-delta}(x~_j); every entry with a non-cardinal basis function of the
   pair is the exact A_ij; every diagonal is minus its off-diagonal row sum.

Rows of non-cardinal basis functions hold only exact entries, so the rows
that need quadrature are those rows plus the sample rows: the fraction of
exactly assembled rows is 1 - ((m - 2p)/m)^n, the lower bound the paper
shades in its timing plots (Sec. 7).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from .surrogate import (bspline_basis, center_slot, exact_rows, flat_index, interp_knots, multi_index,
                        offsets)


def cardinal_range(p: int, m: int):
    """0-based indices of the cardinal B-splines of one direction: [p, m-p-1] (Sec. 2.2)."""
    return p, m - p - 1


def offset_domain(p: int, m: int, dd: int):
    """Indices k of one direction with k and k + dd both cardinal; (k0, k1), empty if k1 < k0."""
    c0, c1 = cardinal_range(p, m)
    return c0 + max(0, -dd), c1 - max(0, dd)


def union_samples(p: int, m: int, M: int) -> List[int]:
    """Sample indices of one direction shared by all offsets: the lattice p + aM
    in the cardinal range, and the p + 1 first and last cardinal indices."""
    c0, c1 = cardinal_range(p, m)
    lattice = set(range(c0, c1 + 1, M))
    ends = set(range(c0, min(c0 + p, c1) + 1)) | set(range(max(c1 - p, c0), c1 + 1))
    return sorted(lattice | ends)


def offset_samples(p: int, m: int, M: int, dd: int) -> List[int]:
    """Sample indices of Omega~_delta in one direction: its ends k0, k1 and the
    lattice points p + aM with distance >= M/2 from both ends."""
    k0, k1 = offset_domain(p, m, dd)
    if k1 < k0:
        return []
    c0 = cardinal_range(p, m)[0]
    inner = [k for k in range(c0, k1 + 1, M) if 2 * (k - k0) >= M and 2 * (k1 - k) >= M]
    return sorted(set([k0] + inner + [k1]))


@dataclass
class SlotSpline:
    samples: List[List[int]]      # sample indices per direction
    q_eff: List[int]
    knots: List[np.ndarray]
    coef: np.ndarray              # [n_s(dir 0), n_s(dir 1), (n_s(dir 2))]


@dataclass
class PerOffsetSetup:
    c0: List[int]
    c1: List[int]
    upper_slots: np.ndarray
    union: List[List[int]]        # union over offsets of the sample indices, per direction
    slots: List[Optional[SlotSpline]]   # per upper slot (position in upper_slots); None = empty domain


def per_offset_setup(prob, M: int, q: int) -> PerOffsetSetup:
    dim, p, m = prob.dim, prob.p, prob.m
    S = prob.S
    c = center_slot(dim, p)
    upper = np.arange(c + 1, S)
    offs = offsets(dim, p)
    c0 = [cardinal_range(p, md)[0] for md in m]
    c1 = [cardinal_range(p, md)[1] for md in m]

    # sample indices per direction, and those of every offset component
    union = [union_samples(p, md, M) for md in m]
    samp = [{dd: offset_samples(p, m[d], M, dd) for dd in range(-p, p + 1)} for d in range(dim)]

    # exact stencil rows at every point of the union grid
    grids = np.meshgrid(*[np.array(u) for u in union], indexing="ij")
    umi = np.stack([g.ravel() for g in grids], axis=1)
    rows = exact_rows(prob, flat_index(umi, m))                          # [n_union, S]
    nu = [len(u) for u in union]
    table = rows.T.reshape([S] + nu)                                     # [S, u0, u1, (u2)]
    pos = [{k: a for a, k in enumerate(u)} for u in union]

    slots: List[Optional[SlotSpline]] = []
    for s in upper:
        delta = offs[s]
        sd = [samp[d][int(delta[d])] for d in range(dim)]
        if any(len(x) == 0 for x in sd):
            slots.append(None)
            continue
        # Phi_delta at the slot's own sample grid, gathered from the union table
        Phi = table[s]
        for d in range(dim):
            Phi = np.take(Phi, [pos[d][k] for k in sd[d]], axis=d)
        q_eff = [min(q, len(x) - 1) for x in sd]
        knots = [interp_knots(x, qd) for x, qd in zip(sd, q_eff)]
        coef = np.array(Phi, dtype=np.float64)
        for d in range(dim):
            B = bspline_basis(knots[d], q_eff[d], np.array(sd[d], dtype=np.float64))
            coef = np.moveaxis(coef, d, 0)
            shp = coef.shape
            coef = np.linalg.solve(B, coef.reshape(shp[0], -1)).reshape(shp)
            coef = np.moveaxis(coef, 0, d)
        slots.append(SlotSpline(sd, q_eff, knots, coef))
    return PerOffsetSetup(c0, c1, upper, union, slots)


def _evaluate(sp: SlotSpline, pts: np.ndarray) -> np.ndarray:
    """Phi~_delta of one upper slot at index points pts [n, dim]."""
    dim = pts.shape[1]
    bases = [bspline_basis(sp.knots[d], sp.q_eff[d], pts[:, d].astype(np.float64)) for d in range(dim)]
    if dim == 2:
        return np.einsum("ab,na,nb->n", sp.coef, bases[0], bases[1])
    return np.einsum("abc,na,nb,nc->n", sp.coef, bases[0], bases[1], bases[2])


def per_offset_rows(prob, M: int, q: int, rows, setup: Optional[PerOffsetSetup] = None) -> np.ndarray:
    """[len(rows), S] surrogate rows with per-offset interpolation domains."""
    rows = np.asarray(rows, dtype=np.int64)
    dim, p, m = prob.dim, prob.p, np.array(prob.m)
    S = prob.S
    c = center_slot(dim, p)
    offs = offsets(dim, p)
    if setup is None:
        setup = per_offset_setup(prob, M, q)
    c0, c1 = np.array(setup.c0), np.array(setup.c1)
    mi = multi_index(rows, m)
    out = np.zeros((len(rows), S))

    def cardinal(x):
        return np.all((x >= c0) & (x <= c1), axis=1)

    # quadrature for every row that keeps an exact off-diagonal entry
    need_exact = ~np.all((mi - p >= c0) & (mi + p <= c1), axis=1)
    out[need_exact] = exact_rows(prob, rows[need_exact])

    card_i = cardinal(mi)
    for s in range(S):
        if s == c:
            continue
        mj = mi + offs[s]
        sel = np.nonzero(card_i & cardinal(mj))[0]
        if len(sel) == 0:
            continue
        if s > c:       # i < j: Phi~_delta at x~_i
            out[sel, s] = _evaluate(setup.slots[s - c - 1], mi[sel])
        else:           # i > j: Phi~_{-delta} at x~_j
            out[sel, s] = _evaluate(setup.slots[S - 1 - s - c - 1], mj[sel])

    valid = np.ones((len(rows), S), dtype=bool)
    for s in range(S):
        mj = mi + offs[s]
        valid[:, s] = np.all((mj >= 0) & (mj < m), axis=1)
    off = np.where(valid, out, 0.0)
    off[:, c] = 0.0
    out[:, c] = -off.sum(axis=1)
    out[~valid] = 0.0
    return out


def per_offset_matrix(prob, M: int, q: int) -> np.ndarray:
    """Per-offset surrogate in stencil-ELL form, values[s, i]."""
    setup = per_offset_setup(prob, M, q)
    return np.ascontiguousarray(per_offset_rows(prob, M, q, np.arange(prob.N), setup).T)
