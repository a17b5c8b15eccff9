"""Pins of the oracle's exact Gauss-quadrature matrix (no GPU).

* Closed forms: on the identity map with constant coefficient every interior
  row equals the tensor sum of 1-D cardinal B-spline mass / stiffness stencils
  (Sec. 3.2, eq. ChangeOfVars with K = I).  The 1-D stencils are derived here
  in exact rational arithmetic from the explicit cardinal B-spline
  N_k(x) = 1/k! sum_j (-1)^j C(k+1, j) (x - j)_+^k and the convolution identity
  int N_p(x) N_p(x - k) dx = N_{2p+1}(p + 1 + k); the (p+1)-point Gauss rule is
  exact for these integrands, so the oracle must reproduce them to rounding.
* Affine maps with a non-symmetric matrix pin K = |det J| J^{-1} J^{-T}
  (eq. BilinearFormPoissonTensor) including the cross terms k != l.
* The Jacobian of the sine-product map against central differences of phi.
* Symmetry and zero row sums of the pure-Neumann matrix (Sec. 5.3: A 1 = 0).
* Brute force: the textbook element-by-element loop on tiny meshes.
* The banded sparsity count (m(2p+1) - p(p+1))^n.
"""
from fractions import Fraction
from math import comb, factorial

import numpy as np
import pytest

import iga_workloads as W
import oracle


# ---------------------------------------------------------------------------
# exact 1-D cardinal stencils
# ---------------------------------------------------------------------------
def _cardinal(k, x, deriv=0):
    """deriv-th derivative of the cardinal B-spline of degree k at rational x."""
    tot = Fraction(0)
    for j in range(k + 2):
        y = x - j
        if y <= 0:
            continue
        e = k - deriv
        if e < 0:
            continue
        c = Fraction(factorial(k), factorial(e))       # d^deriv/dx^deriv y^k
        tot += (-1) ** j * comb(k + 1, j) * c * y ** e
    return tot / factorial(k)


def stencils_1d(p):
    """Dicts over offset k in [-p, p]: F = int N N(.-k), F1 = F', F2 = F''."""
    F, F1, F2 = {}, {}, {}
    for k in range(-p, p + 1):
        x = Fraction(p + 1 + k)
        F[k] = _cardinal(2 * p + 1, x, 0)
        F1[k] = _cardinal(2 * p + 1, x, 1)
        F2[k] = _cardinal(2 * p + 1, x, 2)
    return F, F1, F2


def test_stencils_1d_known_values():
    """Cardinal B-spline values at the integers for p = 2 (mass h [66, 26, 1]/120, stiffness
    [1, -1/3, -1/6]/h, from the B-spline convolution identity) and the sum rules
    (mass sums to h, stiffness to 0)."""
    F, F1, F2 = stencils_1d(2)
    assert [F[k] for k in (0, 1, 2)] == [Fraction(66, 120), Fraction(26, 120), Fraction(1, 120)]
    assert [-F2[k] for k in (0, 1, 2)] == [Fraction(1), Fraction(-2, 6), Fraction(-1, 6)]
    for p in range(1, 6):
        F, F1, F2 = stencils_1d(p)
        assert sum(F.values()) == 1
        assert sum(F2.values()) == 0
        assert sum(F1.values()) == 0


def _factor(F, F1, F2, h, alpha, beta, k):
    """int b_i^(alpha) b_{i+k}^(beta) dx for the cardinal basis of mesh size h."""
    if alpha == 0 and beta == 0:
        return float(F[k]) * h
    if alpha == 1 and beta == 1:
        return -float(F2[k]) / h
    if alpha == 1 and beta == 0:
        return float(F1[k])
    return -float(F1[k])


def closed_form_row(prob, K):
    """Interior-row stencil for a constant tensor K on a uniform mesh."""
    dim, p = prob.dim, prob.p
    F, F1, F2 = stencils_1d(p)
    offs = oracle.offsets(dim, p)
    h = [1.0 / e for e in prob.n_el]
    out = np.zeros(len(offs))
    for s, dl in enumerate(offs):
        tot = 0.0
        for k in range(dim):
            for l in range(dim):
                v = K[k, l]
                for d in range(dim):
                    v *= _factor(F, F1, F2, h[d], int(d == k), int(d == l), int(dl[d]))
                tot += v
        out[s] = tot
    return out


def interior_rows(prob, count=6, seed=0):
    p, m = prob.p, np.array(prob.m)
    rng = np.random.default_rng(seed)
    mi = np.stack([rng.integers(2 * p, md - 2 * p, size=count) for md in m], axis=1)
    stride = np.cumprod([1] + list(m[:-1]))
    return (mi * stride).sum(axis=1)


@pytest.mark.parametrize("dim,p,n_el", [(2, 1, 9), (2, 2, 12), (2, 3, 15), (2, 4, 20), (2, 5, 24),
                                        (3, 1, 7), (3, 2, 9), (3, 3, 14)])
def test_identity_map_closed_form(dim, p, n_el):
    prob = W.Problem(dim=dim, p=p, n_el=tuple([n_el + d for d in range(dim)]))
    rows = interior_rows(prob)
    got = oracle.exact_rows(prob, rows)
    ref = closed_form_row(prob, np.eye(dim))
    scale = np.abs(ref).max()
    for r in range(len(rows)):
        np.testing.assert_allclose(got[r], ref, rtol=0, atol=1e-14 * scale)


@pytest.mark.parametrize("dim,p", [(2, 2), (2, 3), (3, 2), (3, 3)])
def test_affine_map_closed_form(dim, p):
    rng = np.random.default_rng(dim * 7 + p)
    A = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
    b = rng.standard_normal(3)
    aff = tuple(A.ravel()) + tuple(b)
    kap = 1.7
    n_el = (11, 13, 12)[:dim] if p < 3 else (15, 14, 16)[:dim]
    prob = W.Problem(dim=dim, p=p, n_el=n_el, map_kind="affine", affine=aff,
                     kappa_kind="const", kappa_a=kap)
    J = A[:dim, :dim]
    Ji = np.linalg.inv(J)
    K = kap * abs(np.linalg.det(J)) * Ji @ Ji.T
    assert np.abs(K - K.T).max() < 1e-14
    rows = interior_rows(prob, seed=3)
    got = oracle.exact_rows(prob, rows)
    ref = closed_form_row(prob, K)
    scale = np.abs(ref).max()
    for r in range(len(rows)):
        np.testing.assert_allclose(got[r], ref, rtol=0, atol=2e-14 * scale)
    # the coefficient routine itself
    np.testing.assert_allclose(oracle.coefficient(prob, [0.3, 0.6, 0.2][:dim]), K, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_sinprod_jacobian_finite_differences(dim):
    prob = W.Problem(dim=dim, p=2, n_el=(4,) * dim, map_kind="sinprod", map_amp=0.05)
    rng = np.random.default_rng(1)
    for _ in range(5):
        xi = rng.uniform(0.05, 0.95, dim)
        x, J = oracle.geometry_map(prob, xi)
        eps = 1e-6
        Jfd = np.zeros((dim, dim))
        for b in range(dim):
            e = np.zeros(dim)
            e[b] = eps
            Jfd[:, b] = (oracle.geometry_map(prob, xi + e)[0] - oracle.geometry_map(prob, xi - e)[0]) / (2 * eps)
        np.testing.assert_allclose(J, Jfd, atol=1e-9)
        # the map fixes the boundary of the unit cube: x = xi where some xi_j in {0, 1}
        xb = xi.copy()
        xb[0] = 0.0
        np.testing.assert_allclose(oracle.geometry_map(prob, xb)[0], xb, atol=1e-15)


def test_coefficient_from_inverse_jacobian():
    """K computed by the oracle equals kappa |det J| J^{-1} J^{-T} with numpy's inverse."""
    prob = W.CFG_3D_P3.problem
    rng = np.random.default_rng(5)
    for _ in range(5):
        xi = rng.uniform(0, 1, 3)
        x, J = oracle.geometry_map(prob, xi)
        kap = np.exp(0.5 * np.sin(2 * np.pi * x[0]) * np.cos(2 * np.pi * x[1]) * np.sin(2 * np.pi * x[2]))
        Ji = np.linalg.inv(J)
        np.testing.assert_allclose(oracle.coefficient(prob, xi), kap * abs(np.linalg.det(J)) * Ji @ Ji.T,
                                   rtol=1e-13, atol=1e-15)


def _kappa_at(prob, x):
    """kappa at the physical point x, written out from the workload definitions."""
    if prob.kappa_kind == "const":
        return prob.kappa_a
    if prob.kappa_kind == "sin2d":
        return prob.kappa_a + prob.kappa_b * np.sin(2 * np.pi * x[0]) * np.sin(2 * np.pi * x[1])
    if prob.kappa_kind == "poly":
        d = prob.kappa_deg
        xs = list(x) + [0.0] * (3 - len(x))
        return sum(prob.kappa_poly[a + (d + 1) * (b + (d + 1) * c)] * xs[0] ** a * xs[1] ** b * xs[2] ** c
                   for a in range(d + 1) for b in range(d + 1) for c in range(d + 1))
    raise ValueError(prob.kappa_kind)


_POLY = tuple(np.random.default_rng(11).uniform(-0.2, 0.2, 27) + np.eye(1, 27).ravel())


@pytest.mark.parametrize("prob", [
    W.CFG_2D_P2.problem,
    W.Problem(dim=3, p=2, n_el=(4, 4, 4), map_kind="sinprod", map_amp=0.03, kappa_kind="poly", kappa_deg=2,
              kappa_poly=_POLY),
    W.Problem(dim=2, p=2, n_el=(4, 4), map_kind="affine", affine=(1.3, 0.2, 0, -0.4, 0.8, 0, 0, 0, 1, 0.5, -1.0, 0),
              kappa_kind="sin2d", kappa_a=2.0, kappa_b=0.7),
    W.Problem(dim=3, p=1, n_el=(3, 3, 3), map_kind="affine",
              affine=(1.1, 0.2, -0.1, 0.05, 0.9, 0.3, -0.2, 0.1, 1.2, 0.1, -0.2, 0.3), kappa_kind="poly", kappa_deg=2,
              kappa_poly=_POLY),
], ids=["2d_sin2d", "3d_poly_sinprod", "2d_sin2d_affine", "3d_poly_affine"])
def test_coefficient_kappa_at_physical_point(prob):
    """K = kappa(phi(xi)) |det J| J^{-1} J^{-T} for the other kappa kinds and maps, with kappa
    evaluated independently at the physical point and numpy's inverse."""
    rng = np.random.default_rng(6)
    for _ in range(5):
        xi = rng.uniform(0, 1, prob.dim)
        x, J = oracle.geometry_map(prob, xi)
        if prob.map_kind == "affine":
            A = np.array(prob.affine[:9]).reshape(3, 3)[:prob.dim, :prob.dim]
            np.testing.assert_allclose(x, A @ xi + np.array(prob.affine[9:9 + prob.dim]), rtol=1e-15, atol=1e-15)
            np.testing.assert_allclose(J, A, rtol=0, atol=0)
        Ji = np.linalg.inv(J)
        np.testing.assert_allclose(oracle.coefficient(prob, xi), _kappa_at(prob, x) * abs(np.linalg.det(J)) * Ji @ Ji.T,
                                   rtol=1e-13, atol=1e-15)


PROBLEMS_SMALL = [
    W.Problem(dim=2, p=1, n_el=(6, 5), map_kind="sinprod", map_amp=0.05, kappa_kind="sin2d", kappa_a=1.0, kappa_b=0.5),
    W.Problem(dim=2, p=2, n_el=(5, 7), map_kind="sinprod", map_amp=0.04, kappa_kind="sin2d", kappa_a=1.0, kappa_b=0.4),
    W.Problem(dim=2, p=3, n_el=(6, 6), map_kind="sinprod", map_amp=0.05, kappa_kind="sin2d", kappa_a=1.0, kappa_b=0.5),
    W.Problem(dim=3, p=1, n_el=(4, 5, 3), map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d", kappa_b=0.5),
    W.Problem(dim=3, p=2, n_el=(5, 5, 5), map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d", kappa_b=0.5),
]


@pytest.mark.parametrize("prob", PROBLEMS_SMALL, ids=lambda q: f"{q.dim}d_p{q.p}")
def test_brute_force_element_loop(prob):
    """Row-wise quadrature == textbook element-by-element assembly (dense)."""
    dense = oracle.elementwise_dense(prob)
    ell = oracle.exact_matrix(prob)
    D = oracle.ell_to_dense(ell, prob)
    scale = np.abs(dense).max()
    np.testing.assert_allclose(D, dense, rtol=0, atol=1e-14 * scale)
    # the element loop touches nothing outside the stencil pattern
    assert np.count_nonzero(dense) == np.count_nonzero(D)


@pytest.mark.parametrize("prob", PROBLEMS_SMALL + [W.CFG_2D_P2.problem], ids=lambda q: f"{q.dim}d_p{q.p}_{q.N}")
def test_symmetry_and_zero_row_sums(prob):
    ell = oracle.exact_matrix(prob)
    D = oracle.ell_to_dense(ell, prob)
    scale = np.abs(D).max()
    assert np.abs(D - D.T).max() < 1e-14 * scale
    assert np.abs(D.sum(axis=1)).max() < 1e-13 * scale
    # positive semidefinite with a one-dimensional kernel (the constants)
    ev = np.linalg.eigvalsh(0.5 * (D + D.T))
    assert ev[0] > -1e-12 * scale and ev[1] > 1e-8 * scale


@pytest.mark.parametrize("prob", PROBLEMS_SMALL, ids=lambda q: f"{q.dim}d_p{q.p}")
def test_nnz_closed_form(prob):
    ell = oracle.exact_matrix(prob)
    assert np.count_nonzero(ell) == prob.nnz
