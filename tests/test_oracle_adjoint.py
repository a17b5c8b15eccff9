"""Pins of the B-spline diffusion coefficient and of the oracle gradients (no GPU).

* The cubic B-spline kappa equals scipy's BSpline tensor product (an
  independent implementation) at random points; constant control values give
  a constant kappa (partition of unity), and control values sampled from a
  linear function at the Greville abscissae reproduce it (linear precision),
  so the matrix equals the one of the polynomial kappa of degree 1.
* The gradient of L = ybar^T A x with respect to the control values agrees
  between the two independent oracle routes (linearity, and the quadrature of
  grad u_ybar^T G grad u_x) for the exact matrix; for the surrogate it agrees
  with central finite differences of L, and sum_k c_k dL/dc_k = L (L is linear
  in c).
"""
import numpy as np
import pytest
from scipy.interpolate import BSpline

import iga_workloads as W
import oracle
from oracle import adjoint as adj


def _bs_problem(dim, p, n_el, nctrl, seed=0, amp=0.04):
    return W.Problem(dim=dim, p=p, n_el=n_el, map_kind="sinprod", map_amp=amp, kappa_kind="bspline3",
                     kappa_nctrl=nctrl, kappa_ctrl=W.lognormal_ctrl(nctrl, seed=seed))


@pytest.mark.parametrize("dim,nctrl", [(2, (5, 7)), (3, (4, 6, 5)), (3, (16, 16, 16))])
def test_bspline_kappa_matches_scipy(dim, nctrl):
    prob = _bs_problem(dim, 2, (4,) * dim, nctrl, seed=3)
    C = np.array(prob.kappa_ctrl).reshape(list(reversed(nctrl[:dim])))      # [c][b][a]
    kn = [oracle.open_uniform_knots(3, nc - 3) for nc in nctrl[:dim]]
    rng = np.random.default_rng(1)
    for x in rng.uniform(0, 1, size=(25, dim)):
        B = [BSpline(kn[d], np.eye(nctrl[d]), 3)(x[d]) for d in range(dim)]
        ref = np.einsum("ba,a,b->", C, B[0], B[1]) if dim == 2 else np.einsum("cba,a,b,c->", C, B[0], B[1], B[2])
        assert abs(adj.kappa_value(prob, x) - ref) < 1e-13 * abs(ref)


def test_bspline_kappa_partition_of_unity():
    prob = W.Problem(dim=3, p=2, n_el=(5, 4, 6), map_kind="sinprod", map_amp=0.04, kappa_kind="bspline3",
                     kappa_nctrl=(5, 4, 6), kappa_ctrl=tuple(np.full(120, 1.7)))
    ref = W.Problem(dim=3, p=2, n_el=(5, 4, 6), map_kind="sinprod", map_amp=0.04, kappa_kind="const", kappa_a=1.7)
    A, B = oracle.exact_matrix(prob), oracle.exact_matrix(ref)
    assert np.abs(A - B).max() < 1e-14 * np.abs(B).max()


def test_bspline_kappa_linear_precision():
    """Control values alpha + beta . (Greville abscissa) reproduce the linear function."""
    nctrl = (6, 5)
    # Greville abscissae of the open uniform cubic knots: mean of knots t_{k+1..k+3}
    grev = []
    for nc in nctrl:
        t = oracle.open_uniform_knots(3, nc - 3)
        grev.append(np.array([t[k + 1: k + 4].mean() for k in range(nc)]))
    alpha, beta = 1.2, (0.3, -0.4)
    ctrl = np.array([[alpha + beta[0] * grev[0][a] + beta[1] * grev[1][b] for a in range(nctrl[0])]
                     for b in range(nctrl[1])]).ravel()
    prob = W.Problem(dim=2, p=2, n_el=(7, 6), map_kind="sinprod", map_amp=0.04, kappa_kind="bspline3",
                     kappa_nctrl=nctrl, kappa_ctrl=tuple(ctrl))
    poly = np.zeros(64)
    poly[0], poly[1], poly[2] = alpha, beta[0], beta[1]          # x^a y^b at a + 2 b (deg 1)
    ref = W.Problem(dim=2, p=2, n_el=(7, 6), map_kind="sinprod", map_amp=0.04, kappa_kind="poly",
                    kappa_deg=1, kappa_poly=tuple(poly))
    A, B = oracle.exact_matrix(prob), oracle.exact_matrix(ref)
    assert np.abs(A - B).max() < 1e-13 * np.abs(B).max()


CASES = [
    (_bs_problem(2, 2, (9, 8), (5, 6), seed=2), 3, 3),
    (_bs_problem(3, 2, (5, 6, 5), (4, 5, 4), seed=5), 2, 3),
]


@pytest.mark.parametrize("prob,M,q", CASES, ids=["2d", "3d"])
def test_exact_gradient_two_routes_agree(prob, M, q):
    rng = np.random.default_rng(7)
    ybar, x = rng.standard_normal(prob.N), rng.standard_normal(prob.N)
    g1 = adj.kappa_gradient(prob, "exact", M, q, ybar, x)
    g2 = adj.exact_kappa_gradient_quadrature(prob, ybar, x)
    assert np.abs(g1 - g2).max() < 1e-11 * np.abs(g1).max()


@pytest.mark.parametrize("kind", ["common", "per_offset", "exact"])
@pytest.mark.parametrize("prob,M,q", CASES[:1], ids=["2d"])
def test_gradient_matches_finite_differences(prob, M, q, kind):
    rng = np.random.default_rng(8)
    ybar, x = rng.standard_normal(prob.N), rng.standard_normal(prob.N)
    g = adj.kappa_gradient(prob, kind, M, q, ybar, x)
    c = np.array(prob.kappa_ctrl)
    L0 = adj.loss(prob, kind, M, q, ybar, x)
    assert abs(c @ g - L0) < 1e-12 * (np.abs(c) @ np.abs(g))          # Euler: L is linear in c
    h = 1e-3
    for k in rng.choice(len(c), 6, replace=False):
        cp, cm = c.copy(), c.copy()
        cp[k] += h
        cm[k] -= h
        from dataclasses import replace
        Lp = adj.loss(replace(prob, kappa_ctrl=tuple(cp)), kind, M, q, ybar, x)
        Lm = adj.loss(replace(prob, kappa_ctrl=tuple(cm)), kind, M, q, ybar, x)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-9 * np.abs(g).max()
