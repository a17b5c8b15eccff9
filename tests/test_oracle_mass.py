"""Pins of the oracle's mass matrix and its symmetric surrogate (no GPU).

* Identity map: the mass matrix is the tensor product of 1-D B-spline mass
  matrices, computed here independently with scipy's BSpline and numpy's
  Gauss-Legendre rule; an interior row is the tensor product of the closed-form
  cardinal stencils h N_{2p+1}(k) (B-spline convolution identity).
* Affine map x = A xi + b: M = |det A| M(identity) (change of variables).
* Sine-product map: brute-force element-by-element assembly with a
  finite-difference Jacobian.
* Partition of unity: the sum of all entries is the quadrature of the measure of
  Omega, 1 for the sine-product maps of the unit square / cube (they fix its
  boundary) and |det A| for an affine map.
* Symmetric positive definite.
* Surrogate (eq. DefinitionOfSurrogateMatrixSymmetric): M = 1 reproduces M;
  the mass-matrix corollary (polynomial map of degree p_phi, q >= n p_phi - 1)
  gives M~ = M for affine maps; symmetric; frame rows and the upper entries
  (diagonal included) of the sample rows exact; the H^{q+1} entry-error rate.
"""
import numpy as np
import pytest
from scipy.interpolate import BSpline

import iga_workloads as W
import oracle
from oracle import mass


def _mass_1d(p, n_el):
    """1-D mass matrix of the open uniform B-splines by scipy + numpy Gauss (p+1 points)."""
    t = np.concatenate([np.zeros(p), np.linspace(0, 1, n_el + 1), np.ones(p)])
    m = n_el + p
    xg, wg = np.polynomial.legendre.leggauss(p + 1)
    Mx = np.zeros((m, m))
    basis = BSpline(t, np.eye(m), p)
    for e in range(n_el):
        a, b = e / n_el, (e + 1) / n_el
        x = a + (b - a) * 0.5 * (xg + 1)
        B = basis(x)                                   # [points, m]
        Mx += (B * (0.5 * (b - a) * wg)[:, None]).T @ B
    return Mx


@pytest.mark.parametrize("dim,p,n_el", [(2, 2, (7, 6)), (2, 3, (5, 8)), (3, 2, (4, 5, 3)), (3, 1, (5, 4, 6))])
def test_identity_map_is_tensor_product_of_1d_mass(dim, p, n_el):
    prob = W.Problem(dim=dim, p=p, n_el=n_el)
    D = oracle.ell_to_dense(mass.mass_matrix(prob), prob)
    ref = _mass_1d(p, n_el[0])
    for d in range(1, dim):
        ref = np.kron(_mass_1d(p, n_el[d]), ref)      # colexicographic: direction 0 fastest
    assert np.abs(D - ref).max() < 1e-15 * 10 * np.abs(ref).max()


def _phi_sinprod(xi, amp):
    """x_a = xi_a + amp prod_j sin(pi xi_j) (the map of the sine-product workloads)."""
    return xi + amp * np.prod(np.sin(np.pi * xi), axis=-1, keepdims=True)


@pytest.mark.parametrize("dim,p,n_el", [(2, 2, (5, 4)), (3, 1, (3, 4, 3)), (3, 2, (3, 3, 2))])
def test_brute_force_sinprod(dim, p, n_el):
    """Element-by-element assembly with scipy's B-splines, numpy's Gauss rule and a
    central-difference Jacobian of the map (no formula shared with the oracle)."""
    amp = 0.05
    prob = W.Problem(dim=dim, p=p, n_el=n_el, map_kind="sinprod", map_amp=amp)
    xg, wg = np.polynomial.legendre.leggauss(p + 1)
    knots = [np.concatenate([np.zeros(p), np.linspace(0, 1, ne + 1), np.ones(p)]) for ne in n_el]
    ms = [ne + p for ne in n_el]
    D = np.zeros((prob.N, prob.N))
    h = 1e-5
    for e in np.ndindex(*n_el):
        pts1, w1, B1 = [], [], []
        for d in range(dim):
            a, b = e[d] / n_el[d], (e[d] + 1) / n_el[d]
            x = a + (b - a) * 0.5 * (xg + 1)
            pts1.append(x)
            w1.append(0.5 * (b - a) * wg)
            B1.append(BSpline(knots[d], np.eye(ms[d]), p)(x))          # [points, m_d]
        for g in np.ndindex(*([p + 1] * dim)):
            xi = np.array([pts1[d][g[d]] for d in range(dim)])
            J = np.empty((dim, dim))
            for d in range(dim):
                dx = np.zeros(dim)
                dx[d] = h
                J[:, d] = (_phi_sinprod(xi + dx, amp) - _phi_sinprod(xi - dx, amp)) / (2 * h)
            w = np.prod([w1[d][g[d]] for d in range(dim)]) * abs(np.linalg.det(J))
            B = B1[0][g[0]]
            for d in range(1, dim):
                B = np.kron(B1[d][g[d]], B)                                 # colexicographic
            D += w * np.outer(B, B)
    got = oracle.ell_to_dense(mass.mass_matrix(prob), prob)
    assert np.abs(got - D).max() < 1e-9 * np.abs(D).max()


# Centred cardinal B-spline of degree 2p+1 at the integers 0, 1, ..., p (the
# autocorrelation of the degree-p cardinal B-spline), times (2p+1)!.
_CARDINAL = {2: ([66, 26, 1], 120), 3: ([2416, 1191, 120, 1], 5040), 4: ([156190, 88234, 14608, 502, 1], 362880)}


@pytest.mark.parametrize("p", [2, 3, 4])
def test_interior_stencil_closed_form(p):
    """Identity map: an interior row's entry for offset delta is prod_d h_d N_{2p+1}(delta_d)."""
    num, den = _CARDINAL[p]
    k = np.arange(-p, p + 1)
    n1 = np.array([num[abs(j)] for j in k], dtype=np.float64) / den
    assert abs(n1.sum() - 1.0) < 1e-15                       # each 1-D stencil sums to h
    for dim, n_el in ((2, (4 * p + 3, 4 * p + 5)), (3, (4 * p + 2, 4 * p + 3, 4 * p + 1))):
        prob = W.Problem(dim=dim, p=p, n_el=n_el)
        m = np.array(prob.m)
        row = int(oracle.flat_index(m[None, :] // 2, m)[0])
        got = mass.mass_rows(prob, [row])[0]
        ref = np.ones(1)
        for d in range(dim):                                     # colexicographic slots: direction 0 fastest
            ref = np.kron(n1 / n_el[d], ref)
        assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()      # rounding of (p+1)^n-point sums


def test_affine_map_scales_by_det():
    A = np.array([[1.2, 0.3, 0.0], [-0.1, 0.9, 0.2], [0.05, 0.1, 1.1]])
    aff = tuple(A.ravel()) + (0.1, -0.2, 0.3)
    for dim in (2, 3):
        n_el = (5, 6, 4)[:dim]
        prob = W.Problem(dim=dim, p=2, n_el=n_el, map_kind="affine", affine=aff)
        ref = W.Problem(dim=dim, p=2, n_el=n_el)
        det = abs(np.linalg.det(A[:dim, :dim]))
        M1, M0 = mass.mass_matrix(prob), mass.mass_matrix(ref)
        assert np.abs(M1 - det * M0).max() < 1e-14 * np.abs(M1).max()
        assert abs(M1.sum() - det) < 1e-13


@pytest.mark.parametrize("dim,p,n_el,amp", [(2, 2, (12, 14), 0.05), (3, 2, (8, 7, 9), 0.03), (3, 3, (6, 6, 7), 0.03)])
def test_total_mass_is_the_measure(dim, p, n_el, amp):
    prob = W.Problem(dim=dim, p=p, n_el=n_el, map_kind="sinprod", map_amp=amp)
    M = mass.mass_matrix(prob)
    assert abs(M.sum() - 1.0) < 1e-6
    D = oracle.ell_to_dense(M, prob)
    assert np.abs(D - D.T).max() < 1e-16 * 10
    if prob.N <= 600:
        assert np.linalg.eigvalsh(0.5 * (D + D.T)).min() > 0


SURR = [
    (W.Problem(dim=2, p=2, n_el=(20, 23), map_kind="sinprod", map_amp=0.05), 3, 3),
    (W.Problem(dim=2, p=3, n_el=(25, 22), map_kind="sinprod", map_amp=0.05), 4, 2),
    (W.Problem(dim=3, p=2, n_el=(13, 12, 14), map_kind="sinprod", map_amp=0.03), 3, 3),
]


def test_M1_is_exact():
    for prob, _, q in SURR:
        ref = mass.mass_matrix(prob)
        assert oracle.relative_entry_error(mass.mass_surrogate_matrix(prob, 1, q), ref) < 1e-13


@pytest.mark.parametrize("dim,q", [(2, 1), (3, 2), (2, 3)])
def test_affine_reproduction(dim, q):
    """Mass-matrix corollary: polynomial map of degree 1, q >= n - 1 => M~ = M."""
    A = np.array([[1.1, 0.2, -0.1], [0.05, 0.9, 0.3], [-0.2, 0.1, 1.2]])
    prob = W.Problem(dim=dim, p=2, n_el=(14, 13, 15)[:dim], map_kind="affine", affine=tuple(A.ravel()) + (0, 0, 0))
    ref = mass.mass_matrix(prob)
    assert oracle.relative_entry_error(mass.mass_surrogate_matrix(prob, 3, q), ref) < 1e-12


@pytest.mark.parametrize("prob,M,q", SURR, ids=["2d_p2", "2d_p3", "3d_p2"])
def test_symmetric_surrogate_structure(prob, M, q):
    Ms = mass.mass_surrogate_matrix(prob, M, q)
    ref = mass.mass_matrix(prob)
    D = oracle.ell_to_dense(Ms, prob)
    scale = np.abs(D).max()
    assert np.abs(D - D.T).max() < 1e-15 * 10 * scale
    err = oracle.relative_entry_error(Ms, ref)
    assert 1e-9 < err < 0.1
    setup = mass.mass_surrogate_setup(prob, M, q)
    mi = oracle.multi_index(np.arange(prob.N), prob.m)
    k0, k1 = np.array(setup.k0), np.array(setup.k1)
    frame = ~np.all((mi >= k0) & (mi <= k1), axis=1)
    assert np.abs(Ms[:, frame] - ref[:, frame]).max() < 1e-15 * 10 * scale
    samp = np.ones(prob.N, dtype=bool)
    for d in range(prob.dim):
        samp &= np.isin(mi[:, d], setup.samples[d])
    c = oracle.center_slot(prob.dim, prob.p)
    assert np.abs(Ms[c:, samp] - ref[c:, samp]).max() < 1e-13 * scale


@pytest.mark.slow
def test_entry_error_rate():
    """|M - M~|_max ~ H^{q+1} at fixed h (eq. SurrogateMassBound, q = 3)."""
    prob = W.Problem(dim=2, p=2, n_el=(135, 135), map_kind="sinprod", map_amp=0.05)
    ref = mass.mass_matrix(prob)
    Ms = [4, 8, 16]
    errs = [np.abs(mass.mass_surrogate_matrix(prob, M, 3) - ref).max() for M in Ms]
    slopes = np.diff(np.log(errs)) / np.diff(np.log(Ms))
    assert np.all(slopes > 4 - 0.6) and np.all(slopes < 4 + 1.5), (errs, slopes)
