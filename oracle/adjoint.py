"""TEST INFRASTRUCTURE: gradients of L(c) = ybar^T A~(kappa_c) x.

kappa_c is the cubic B-spline diffusion coefficient on the physical unit cube
with control values c (kappa kind "bspline3").  The gradient with respect to x
is A~^T ybar = A~ ybar (A~ is symmetric, eq. DefinitionOfSurrogateMatrixSymmetricKernel).

With respect to c, two routes that share nothing but the oracle's forward
assembly and basis routines:

* ``kappa_gradient``: every step of the surrogate is linear in kappa -- the
  Gauss quadrature of the exact rows (eq. ChangeOfVars), the sampling and the
  B-spline interpolation of each stencil function (Sec. 4.1, Sec. 6), the
  symmetric copy and the kernel-preserving diagonal (Sec. 5.3) -- and kappa_c
  is linear in c, so A~(c) = sum_k c_k A~(e_k) and dL/dc_k = ybar^T A~(e_k) x.
  This assembles one matrix per control value (tiny problems only).
* ``exact_kappa_gradient_quadrature``: for the exact matrix,
  ybar^T A x = sum_g w_g kappa(phi(g)) grad u_ybar(g)^T G(g) grad u_x(g) with
  u_v = sum_i v_i B_i and G = |det Dphi| Dphi^{-1} Dphi^{-T} (Sec. 3.2), so
  dL/dc_k = sum_g w_g N_k(phi(g)) grad u_ybar^T G grad u_x, N_k the k-th
  tensor-product cubic B-spline of kappa.
"""
from __future__ import annotations

import ctypes
from dataclasses import replace

import numpy as np

from . import _lib
from .per_offset import per_offset_matrix
from .surrogate import (bspline_all, coefficient, exact_matrix, gauss_legendre, geometry_map, offsets,
                        open_uniform_knots, surrogate_matrix)
from .linalg import apply


def kappa_value(prob, x) -> float:
    """kappa at the physical point x (C oracle)."""
    P = _lib.make_problem(prob)
    x3 = np.zeros(3)
    x3[: prob.dim] = x
    return float(_lib.lib().orc_kappa(ctypes.byref(P), _lib._dptr(x3)))


def _matrix(prob, kind: str, M: int, q: int) -> np.ndarray:
    if kind == "exact":
        return exact_matrix(prob)
    if kind == "per_offset":
        return per_offset_matrix(prob, M, q)
    return surrogate_matrix(prob, M, q)


def loss(prob, kind: str, M: int, q: int, ybar: np.ndarray, x: np.ndarray) -> float:
    """L = ybar^T A x for A the exact ('exact') or surrogate ('common' / 'per_offset') matrix."""
    return float(ybar @ apply(_matrix(prob, kind, M, q), prob, x))


def kappa_gradient(prob, kind: str, M: int, q: int, ybar: np.ndarray, x: np.ndarray) -> np.ndarray:
    """dL/dc_k = ybar^T A(e_k) x, by linearity in the control values."""
    nc = int(np.prod(prob.kappa_nctrl[: prob.dim]))
    g = np.zeros(nc)
    for k in range(nc):
        e = np.zeros(nc)
        e[k] = 1.0
        pk = replace(prob, kappa_ctrl=tuple(e))
        g[k] = ybar @ apply(_matrix(pk, kind, M, q), prob, x)
    return g


def _basis_at_gauss(p: int, n_el: int):
    """Gauss points per element and the values / derivatives of the p+1 active B-splines."""
    xg, wg = gauss_legendre(p + 1)             # nodes and weights on [0, 1]
    t = open_uniform_knots(p, n_el)
    pts, wts, first, val, der = [], [], [], [], []
    for e in range(n_el):
        a, b = e / n_el, (e + 1) / n_el
        for r in range(p + 1):
            xi = a + (b - a) * xg[r]
            v, d = bspline_all(p, t, xi)
            pts.append(xi)
            wts.append((b - a) * wg[r])
            first.append(e)
            val.append(v[e: e + p + 1])
            der.append(d[e: e + p + 1])
    return np.array(pts), np.array(wts), np.array(first), np.array(val), np.array(der)


def exact_kappa_gradient_quadrature(prob, ybar: np.ndarray, x: np.ndarray) -> np.ndarray:
    """dL/dc_k for the exact matrix from the quadrature of grad u_ybar^T G grad u_x."""
    dim, p, m = prob.dim, prob.p, prob.m
    tabs = [_basis_at_gauss(p, ne) for ne in prob.n_el]
    unit = replace(prob, kappa_kind="const", kappa_a=1.0, kappa_nctrl=None, kappa_ctrl=None)
    nck = list(prob.kappa_nctrl[:dim])
    kn = [open_uniform_knots(3, c - 3) for c in nck]
    Y = ybar.reshape(list(reversed(m)))       # [i2][i1][i0] (colexicographic)
    X = x.reshape(list(reversed(m)))
    g = np.zeros(int(np.prod(nck)))
    ranges = [range(len(t[0])) for t in tabs]
    for gi in np.ndindex(*[len(r) for r in ranges]):
        xi = [tabs[d][0][gi[d]] for d in range(dim)]
        w = np.prod([tabs[d][1][gi[d]] for d in range(dim)])
        e = [tabs[d][2][gi[d]] for d in range(dim)]
        V = [tabs[d][3][gi[d]] for d in range(dim)]
        D = [tabs[d][4][gi[d]] for d in range(dim)]
        # gradients of u_ybar and u_x in parametric coordinates
        gu = []
        for F in (Y, X):
            if dim == 2:
                loc = F[e[1]: e[1] + p + 1, e[0]: e[0] + p + 1]        # [a1][a0]
                g0 = np.einsum("ba,a,b->", loc, D[0], V[1])
                g1 = np.einsum("ba,a,b->", loc, V[0], D[1])
                gu.append(np.array([g0, g1]))
            else:
                loc = F[e[2]: e[2] + p + 1, e[1]: e[1] + p + 1, e[0]: e[0] + p + 1]
                g0 = np.einsum("cba,a,b,c->", loc, D[0], V[1], V[2])
                g1 = np.einsum("cba,a,b,c->", loc, V[0], D[1], V[2])
                g2 = np.einsum("cba,a,b,c->", loc, V[0], V[1], D[2])
                gu.append(np.array([g0, g1, g2]))
        G = coefficient(unit, xi)
        s = w * (gu[0] @ G @ gu[1])
        phys, _ = geometry_map(prob, xi)
        Nk = []
        for d in range(dim):
            xd = min(max(phys[d], 0.0), 1.0)
            v, _ = bspline_all(3, kn[d], xd)
            Nk.append(v)
        if dim == 2:
            g += s * np.outer(Nk[1], Nk[0]).ravel()
        else:
            g += s * np.einsum("c,b,a->cba", Nk[2], Nk[1], Nk[0]).ravel()
    return g


__all__ = ["kappa_value", "loss", "kappa_gradient", "exact_kappa_gradient_quadrature", "offsets"]
