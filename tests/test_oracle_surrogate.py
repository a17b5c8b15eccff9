"""Pins of the oracle's surrogate assembly (no GPU).

* 1-D interpolation: the not-a-knot spline through the samples equals scipy's
  make_interp_spline (an independent implementation) and reproduces P_q.
* M = 1 samples every point of Omega~, so the surrogate is the exact matrix
  (Sec. 6).
* Polynomial reproduction (Remark rem:PolynomialReproduction,
  prop:PolynomialReproduction): identity map with kappa in Q_r, r <= q, or
  an affine map with constant kappa, gives A~ = A.
* eq. DefinitionOfSurrogateMatrixSymmetricKernel: A~ = A~^T, A~ 1 = 0; rows
  outside Omega~ are exact; the upper entries of sampled rows are exact
  (Sec. 6, the interpolant passes through its samples).
* thm:RegularityOfStencilFunctions: |A - A~|_max decays like H^{q+1} at fixed h.
"""
import numpy as np
import pytest
from scipy.interpolate import make_interp_spline

import iga_workloads as W
import oracle


@pytest.mark.parametrize("q", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("k0,k1,M", [(4, 29, 4), (6, 60, 8), (8, 91, 8), (6, 44, 8), (2, 20, 3), (4, 12, 1)])
def test_interpolant_matches_scipy_not_a_knot(q, k0, k1, M):
    t = np.array(oracle.sample_indices(k0, k1, M), dtype=float)
    n = len(t)
    if q > n - 1:
        pytest.skip("degree lowered below q")
    if q == 0:
        pytest.skip("scipy has no degree-0 not-a-knot")
    rng = np.random.default_rng(q * 100 + k1)
    y = rng.standard_normal(n)
    knots = oracle.interp_knots(t, q)
    ref = make_interp_spline(t, y, k=q)
    np.testing.assert_allclose(knots, ref.t, rtol=0, atol=1e-13)
    B = oracle.bspline_basis(knots, q, t)
    c = np.linalg.solve(B, y)
    xs = np.arange(k0, k1 + 1, dtype=float)
    got = oracle.bspline_basis(knots, q, xs) @ c
    np.testing.assert_allclose(got, ref(xs), rtol=0, atol=1e-12 * max(1, np.abs(y).max()))


@pytest.mark.parametrize("q", [0, 1, 2, 3, 4, 5])
def test_interpolant_reproduces_polynomials(q):
    t = np.array(oracle.sample_indices(6, 60, 8), dtype=float)
    knots = oracle.interp_knots(t, q)
    xs = np.arange(6, 61, dtype=float)
    for deg in range(q + 1):
        y = ((t - 30.0) / 30.0) ** deg
        c = np.linalg.solve(oracle.bspline_basis(knots, q, t), y)
        got = oracle.bspline_basis(knots, q, xs) @ c
        np.testing.assert_allclose(got, ((xs - 30.0) / 30.0) ** deg, atol=1e-12)


def test_sample_lattice_examples():
    """Every M-th index from the first point of Omega~, plus the last (Sec. 6)."""
    assert oracle.sample_indices(6, 60, 8) == [6, 14, 22, 30, 38, 46, 54, 60]
    assert oracle.sample_indices(4, 29, 4) == [4, 8, 12, 16, 20, 24, 28, 29]
    assert oracle.sample_indices(4, 28, 4) == [4, 8, 12, 16, 20, 24, 28]
    assert oracle.sample_indices(5, 5, 3) == [5]
    assert oracle.sample_indices(3, 9, 1) == list(range(3, 10))


def _dense(values, prob):
    return oracle.ell_to_dense(values, prob)


SURR_CASES = [
    (W.Problem(dim=2, p=2, n_el=(20, 23), map_kind="sinprod", map_amp=0.05, kappa_kind="sin2d",
               kappa_a=1.0, kappa_b=0.5), 3, 3),
    (W.Problem(dim=2, p=3, n_el=(25, 22), map_kind="sinprod", map_amp=0.05, kappa_kind="sin2d",
               kappa_a=1.0, kappa_b=0.5), 4, 2),
    (W.Problem(dim=2, p=1, n_el=(14, 15), map_kind="sinprod", map_amp=0.05, kappa_kind="sin2d",
               kappa_a=1.0, kappa_b=0.5), 5, 1),
    (W.Problem(dim=3, p=2, n_el=(13, 12, 14), map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d",
               kappa_b=0.5), 3, 3),
]


def test_M1_is_exact():
    for prob, _, q in SURR_CASES[:3]:
        A = oracle.exact_matrix(prob)
        As = oracle.surrogate_matrix(prob, 1, q)
        assert oracle.relative_entry_error(As, A) < 1e-13


@pytest.mark.parametrize("prob,M,q", SURR_CASES, ids=["2d_p2", "2d_p3", "2d_p1", "3d_p2"])
def test_symmetric_kernel_preserving(prob, M, q):
    As = oracle.surrogate_matrix(prob, M, q)
    A = oracle.exact_matrix(prob)
    D = _dense(As, prob)
    scale = np.abs(D).max()
    assert np.abs(D - D.T).max() < 1e-14 * scale
    assert np.abs(D.sum(axis=1)).max() < 1e-13 * scale
    err = oracle.relative_entry_error(As, A)
    assert 0 < err < 0.5
    # rows outside Omega~ are exact; so are the upper entries of sampled rows
    setup = oracle.surrogate_setup(prob, M, q)
    mi = oracle.multi_index(np.arange(prob.N), prob.m)
    k0, k1 = np.array(setup.k0), np.array(setup.k1)
    frame = ~np.all((mi >= k0) & (mi <= k1), axis=1)
    c = oracle.center_slot(prob.dim, prob.p)
    assert np.abs(As[:, frame] - A[:, frame]).max() < 1e-13 * scale
    samp = np.ones(prob.N, dtype=bool)
    for d in range(prob.dim):
        samp &= np.isin(mi[:, d], setup.samples[d])
    assert np.abs(As[c + 1:, samp] - A[c + 1:, samp]).max() < 1e-13 * scale
    # some interior entries really are interpolated (differ from A)
    assert np.abs(As[c + 1:, ~frame & ~samp] - A[c + 1:, ~frame & ~samp]).max() > 1e-8 * scale


@pytest.mark.parametrize("dim,p,q,r", [(2, 2, 3, 3), (2, 3, 2, 2), (2, 2, 1, 1), (3, 2, 3, 2), (2, 4, 5, 4)])
def test_polynomial_reproduction(dim, p, q, r):
    """Identity map, kappa in Q_r with r <= q: A~ = A (Remark rem:PolynomialReproduction)."""
    rng = np.random.default_rng(11 * p + q)
    coef = np.zeros(64)
    nc = (r + 1) ** dim
    coef[:nc] = rng.uniform(0.1, 1.0, nc) / nc
    coef[0] += 1.0           # keep kappa positive
    n_el = tuple([6 * p + 10 + 2 * d for d in range(dim)])
    prob = W.Problem(dim=dim, p=p, n_el=n_el, kappa_kind="poly", kappa_deg=r, kappa_poly=tuple(coef))
    A = oracle.exact_matrix(prob)
    As = oracle.surrogate_matrix(prob, 3, q)
    assert oracle.relative_entry_error(As, A) < 1e-12
    # one degree too few does NOT reproduce (guards against a vacuous pass)
    if q >= 1 and r == q:
        As_low = oracle.surrogate_matrix(prob, 3, q - 1)
        assert oracle.relative_entry_error(As_low, A) > 1e-9


def test_affine_map_reproduction():
    rng = np.random.default_rng(2)
    Am = np.eye(3) + 0.2 * rng.standard_normal((3, 3))
    prob = W.Problem(dim=2, p=2, n_el=(22, 19), map_kind="affine", affine=tuple(Am.ravel()) + (0.1, 0.2, 0.3),
                     kappa_kind="const", kappa_a=2.0)
    A = oracle.exact_matrix(prob)
    for q in (0, 1, 3):
        assert oracle.relative_entry_error(oracle.surrogate_matrix(prob, 4, q), A) < 1e-12


def test_empty_omega_is_exact():
    prob = W.Problem(dim=2, p=3, n_el=(9, 10), map_kind="sinprod", map_amp=0.05,
                     kappa_kind="sin2d", kappa_a=1.0, kappa_b=0.5)   # m = 12: box [6, 5] is empty
    A = oracle.exact_matrix(prob)
    assert oracle.surrogate_setup(prob, 4, 3).empty
    assert oracle.relative_entry_error(oracle.surrogate_matrix(prob, 4, 3), A) < 1e-13


def test_single_index_omega_is_exact():
    """One index of Omega~ per direction: one sample, a constant interpolant equal to it."""
    prob = W.Problem(dim=2, p=2, n_el=(7, 7), map_kind="sinprod", map_amp=0.05,
                     kappa_kind="sin2d", kappa_a=1.0, kappa_b=0.5)   # m = 9: box [4, 4]
    setup = oracle.surrogate_setup(prob, 4, 3)
    assert setup.samples == [[4], [4]] and setup.q_eff == [0, 0]
    A = oracle.exact_matrix(prob)
    assert oracle.relative_entry_error(oracle.surrogate_matrix(prob, 4, 3), A) < 1e-13


def _offdiag_max(X, prob):
    c = oracle.center_slot(prob.dim, prob.p)
    Y = X.copy()
    Y[c] = 0.0
    return np.abs(Y).max()


@pytest.mark.slow
@pytest.mark.parametrize("q", [1, 2, 3])
def test_entry_error_rate(q):
    """|A - A~|_max ~ H^{q+1} at fixed h (thm:RegularityOfStencilFunctions)."""
    prob = W.Problem(dim=2, p=2, n_el=(135, 135), map_kind="sinprod", map_amp=0.05,
                     kappa_kind="sin2d", kappa_a=1.0, kappa_b=0.5)      # L - 1 = 128
    A = oracle.exact_matrix(prob)
    Ms = [4, 8, 16]
    errs = [_offdiag_max(oracle.surrogate_matrix(prob, M, q) - A, prob) for M in Ms]
    slopes = np.diff(np.log(errs)) / np.diff(np.log(Ms))
    assert np.all(slopes > q + 1 - 0.6), (errs, slopes)
    assert np.all(slopes < q + 1 + 1.5), (errs, slopes)
