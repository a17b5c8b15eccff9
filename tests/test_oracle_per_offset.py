"""Pins of the oracle's per-offset surrogate (Omega~_delta domains; no GPU).

* Sec. 2.2: the cardinal index range [p, m-p-1] is exactly the set of basis
  functions whose p + 2 knots are distinct (checked on the knot vector).
* Sec. 3.2: for an identity map and kappa = 1, A_{i,i+delta} equals the
  interior stencil value whenever i and i + delta are both cardinal (so
  Omega~_delta is large enough to hold only translation-invariant entries),
  and differs from it for some non-cardinal pair (so it is not too large).
* Sec. 3.2 / Sec. 4: the union of the Omega~_delta is the cardinal box and
  their intersection the box [2p, m-2p-1] of Sec. 4.
* Sec. 6: M = 1 samples every point, so the surrogate is exact; the
  interpolant passes through its samples.
* Polynomial reproduction (Remark rem:PolynomialReproduction) with kappa in
  Q_r, r <= q, on the identity map.
* Symmetry and zero row sums (eq. DefinitionOfSurrogateMatrixSymmetricKernel).
* Sec. 7 (timing plots): the rows assembled exactly are the non-cardinal ones,
  N - (m - 2p)^n of them.
* Each slot's interpolant equals scipy's make_interp_spline applied along
  every axis (an independent tensor-product implementation).
* thm:RegularityOfStencilFunctions: the entry error decays like H^{q+1}.
"""
import numpy as np
import pytest
from scipy.interpolate import make_interp_spline

import iga_workloads as W
import oracle
from oracle import per_offset as po


def _sinprod2(n_el, p):
    return W.Problem(dim=2, p=p, n_el=n_el, map_kind="sinprod", map_amp=0.05, kappa_kind="sin2d",
                     kappa_a=1.0, kappa_b=0.5)


CASES = [
    (_sinprod2((20, 23), 2), 3, 3),
    (_sinprod2((25, 22), 3), 4, 2),
    (_sinprod2((14, 15), 1), 5, 1),
    (W.Problem(dim=3, p=2, n_el=(13, 12, 14), map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d",
               kappa_b=0.5), 3, 3),
]


@pytest.mark.parametrize("p,n_el", [(1, 5), (2, 9), (3, 12), (4, 15), (5, 11)])
def test_cardinal_range_from_knots(p, n_el):
    t = oracle.open_uniform_knots(p, n_el)
    m = n_el + p
    card = [k for k in range(m) if np.all(np.diff(t[k: k + p + 2]) > 0)]
    c0, c1 = po.cardinal_range(p, m)
    assert card == list(range(c0, c1 + 1))


@pytest.mark.parametrize("p,m", [(1, 9), (2, 14), (3, 20), (4, 30), (2, 5)])
def test_domain_union_and_intersection(p, m):
    doms = [po.offset_domain(p, m, dd) for dd in range(-p, p + 1)]
    sets = [set(range(a, b + 1)) for a, b in doms]
    c0, c1 = po.cardinal_range(p, m)
    assert set.union(*sets) == set(range(c0, c1 + 1))
    k0, k1 = oracle.omega_box(p, m)
    assert set.intersection(*sets) == set(range(k0, k1 + 1))


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (2, 3), (3, 2)])
def test_domain_holds_the_translation_invariant_entries(dim, p):
    n_el = tuple([4 * p + 5 + d for d in range(dim)])
    prob = W.Problem(dim=dim, p=p, n_el=n_el)
    A = oracle.exact_matrix(prob)
    m = np.array(prob.m)
    mi = oracle.multi_index(np.arange(prob.N), m)
    c0 = np.array([po.cardinal_range(p, md)[0] for md in m])
    c1 = np.array([po.cardinal_range(p, md)[1] for md in m])
    mid = oracle.flat_index((m // 2)[None, :], m)[0]          # a row deep inside
    offs = oracle.offsets(dim, p)
    scale = np.abs(A).max()
    differs = False
    for s, delta in enumerate(offs):
        mj = mi + delta
        inside = np.all((mj >= 0) & (mj < m), axis=1)
        both = np.all((mi >= c0) & (mi <= c1) & (mj >= c0) & (mj <= c1), axis=1)
        assert np.abs(A[s, both] - A[s, mid]).max() < 1e-13 * scale
        if np.any(np.abs(A[s, inside & ~both] - A[s, mid]) > 1e-6 * scale):
            differs = True
    assert differs


def test_sample_examples():
    """Ends of Omega~_delta plus lattice points p + aM at least M/2 from both ends."""
    # p = 2, m = 20: cardinal [2, 17], lattice 2, 6, 10, 14
    assert po.union_samples(2, 20, 4) == [2, 3, 4, 6, 10, 14, 15, 16, 17]
    assert po.offset_samples(2, 20, 4, 0) == [2, 6, 10, 14, 17]
    assert po.offset_samples(2, 20, 4, 2) == [2, 6, 10, 15]
    assert po.offset_samples(2, 20, 4, -1) == [3, 6, 10, 14, 17]
    assert po.offset_samples(2, 20, 4, -2) == [4, 6, 10, 14, 17]
    assert po.offset_samples(2, 20, 1, 1) == list(range(2, 17))
    # p = 3, m = 67, M = 8: cardinal [3, 63]
    assert po.union_samples(3, 67, 8) == [3, 4, 5, 6, 11, 19, 27, 35, 43, 51, 59, 60, 61, 62, 63]
    assert po.offset_samples(3, 67, 8, -3) == [6, 11, 19, 27, 35, 43, 51, 59, 63]
    assert po.offset_samples(3, 67, 8, 3) == [3, 11, 19, 27, 35, 43, 51, 60]
    # end runs that meet: every cardinal index is a sample row
    assert po.union_samples(3, 14, 8) == list(range(3, 11))
    # one cardinal index: offsets other than 0 have no domain
    assert po.offset_samples(2, 5, 4, 0) == [2]
    assert po.offset_samples(2, 5, 4, 1) == []


@pytest.mark.parametrize("p,m,M", [(2, 20, 4), (3, 67, 8), (4, 100, 8), (1, 9, 3), (3, 14, 8), (2, 5, 4),
                                   (5, 45, 6), (2, 34, 40), (4, 100, 3)])
def test_offset_samples_are_quasi_uniform_and_shared(p, m, M):
    """Each domain's ends are samples, spacing stays within [min(M, L)/2, 3M/2], and
    every sample is one of the shared sample rows."""
    union = set(po.union_samples(p, m, M))
    for dd in range(-p, p + 1):
        k0, k1 = po.offset_domain(p, m, dd)
        if k1 < k0:
            continue
        t = po.offset_samples(p, m, M, dd)
        assert t[0] == k0 and t[-1] == k1
        assert set(t) <= union
        gaps = np.diff(t)
        if len(gaps):
            assert gaps.max() <= 1.5 * M
            assert gaps.min() >= min(M, k1 - k0) / 2 or len(gaps) == 1


@pytest.mark.parametrize("p,m,M,q", [(5, 45, 6, 7), (3, 67, 8, 3), (4, 100, 8, 3), (2, 34, 40, 3), (3, 67, 8, 5)])
def test_offset_interpolation_is_well_conditioned(p, m, M, q):
    """Lebesgue constant of every offset's interpolant stays within a small factor of
    the common-domain one (quasi-uniform knots, Sec. 4.1)."""
    def leb(t):
        t = np.asarray(t, dtype=float)
        qe = min(q, len(t) - 1)
        kn = oracle.interp_knots(t, qe)
        Binv = np.linalg.inv(oracle.bspline_basis(kn, qe, t))
        E = oracle.bspline_basis(kn, qe, np.arange(t[0], t[-1] + 1))
        return np.abs(E @ Binv).sum(axis=1).max()
    k0, k1 = oracle.omega_box(p, m)
    common = leb(oracle.sample_indices(k0, k1, M))
    worst = max(leb(po.offset_samples(p, m, M, dd)) for dd in range(-p, p + 1))
    assert worst <= 3.0 * common + 1.0


def test_M1_is_exact():
    for prob, _, q in CASES:
        A = oracle.exact_matrix(prob)
        assert oracle.relative_entry_error(po.per_offset_matrix(prob, 1, q), A) < 1e-13


@pytest.mark.parametrize("prob,M,q", CASES, ids=["2d_p2", "2d_p3", "2d_p1", "3d_p2"])
def test_symmetric_kernel_preserving_and_exact_pattern(prob, M, q):
    As = po.per_offset_matrix(prob, M, q)
    A = oracle.exact_matrix(prob)
    D = oracle.ell_to_dense(As, prob)
    scale = np.abs(D).max()
    assert np.abs(D - D.T).max() < 1e-14 * scale
    assert np.abs(D.sum(axis=1)).max() < 1e-13 * scale
    assert 0 < oracle.relative_entry_error(As, A) < 0.5

    # exact off-diagonal entries: pairs with a non-cardinal member, and upper
    # entries at the slot's own samples; every other entry is interpolated
    setup = po.per_offset_setup(prob, M, q)
    m = np.array(prob.m)
    mi = oracle.multi_index(np.arange(prob.N), m)
    c0, c1 = np.array(setup.c0), np.array(setup.c1)
    c = oracle.center_slot(prob.dim, prob.p)
    offs = oracle.offsets(prob.dim, prob.p)
    for s in range(c + 1, prob.S):
        mj = mi + offs[s]
        inside = np.all((mj >= 0) & (mj < m), axis=1)
        both = np.all((mi >= c0) & (mi <= c1) & (mj >= c0) & (mj <= c1), axis=1)
        sp = setup.slots[s - c - 1]
        on_grid = both.copy()
        if sp is not None:
            for d in range(prob.dim):
                on_grid &= np.isin(mi[:, d], sp.samples[d])
        diff = np.abs(As[s] - A[s])
        assert np.all(diff[inside & ~both] < 1e-13 * scale)
        assert np.all(diff[on_grid] < 1e-13 * scale)
        interp = both & ~on_grid
        if np.any(interp):
            assert diff[interp].max() > 1e-9 * scale


@pytest.mark.parametrize("dim,p,q,r", [(2, 2, 3, 3), (2, 3, 2, 2), (2, 2, 1, 1), (3, 2, 3, 2), (2, 4, 5, 4)])
def test_polynomial_reproduction(dim, p, q, r):
    rng = np.random.default_rng(13 * p + q)
    coef = np.zeros(64)
    nc = (r + 1) ** dim
    coef[:nc] = rng.uniform(0.1, 1.0, nc) / nc
    coef[0] += 1.0
    n_el = tuple([6 * p + 10 + 2 * d for d in range(dim)])
    prob = W.Problem(dim=dim, p=p, n_el=n_el, kappa_kind="poly", kappa_deg=r, kappa_poly=tuple(coef))
    A = oracle.exact_matrix(prob)
    assert oracle.relative_entry_error(po.per_offset_matrix(prob, 3, q), A) < 1e-12
    if q >= 1 and r == q:
        assert oracle.relative_entry_error(po.per_offset_matrix(prob, 3, q - 1), A) > 1e-9


@pytest.mark.parametrize("dim,p,n_el", [(2, 2, (20, 17)), (2, 3, (25, 30)), (3, 2, (9, 10, 11)), (2, 1, (6, 4))])
def test_exact_rows_are_the_non_cardinal_rows(dim, p, n_el):
    """Rows with no interpolated entry number N - (m - 2p)^n (the bound shaded in Sec. 7)."""
    prob = W.Problem(dim=dim, p=p, n_el=n_el, map_kind="sinprod", map_amp=0.03,
                     kappa_kind="sin2d" if dim == 2 else "expsin3d", kappa_a=1.0, kappa_b=0.5)
    M, q = 2, 3
    As = po.per_offset_matrix(prob, M, q)
    A = oracle.exact_matrix(prob)
    setup = po.per_offset_setup(prob, M, q)
    c = oracle.center_slot(dim, p)
    offs = oracle.offsets(dim, p)
    m = np.array(prob.m)
    mi = oracle.multi_index(np.arange(prob.N), m)
    c0, c1 = np.array(setup.c0), np.array(setup.c1)
    has_interp = np.zeros(prob.N, dtype=bool)
    for s in range(prob.S):
        if s == c:
            continue
        mj = mi + offs[s]
        has_interp |= np.all((mi >= c0) & (mi <= c1) & (mj >= c0) & (mj <= c1), axis=1)
    expect = prob.N - int(np.prod([md - 2 * p for md in m]))
    assert int(np.sum(~has_interp)) == expect
    scale = np.abs(A).max()
    assert np.abs(As[:, ~has_interp] - A[:, ~has_interp]).max() < 1e-13 * scale


@pytest.mark.parametrize("q", [1, 2, 3])
def test_slot_interpolant_matches_scipy(q):
    prob = _sinprod2((24, 21), 2)
    M = 4
    setup = po.per_offset_setup(prob, M, q)
    c = oracle.center_slot(2, 2)
    offs = oracle.offsets(2, 2)
    A = oracle.exact_matrix(prob)
    m = prob.m
    checked = 0
    for u, sp in enumerate(setup.slots):
        if sp is None or min(len(x) for x in sp.samples) <= q:
            continue
        s = c + 1 + u
        t0, t1 = (np.array(x, dtype=float) for x in sp.samples)
        rows = oracle.flat_index(np.stack(np.meshgrid(sp.samples[0], sp.samples[1], indexing="ij"),
                                          axis=-1).reshape(-1, 2), m)
        Y = A[s, rows].reshape(len(t0), len(t1))
        # interpolate along direction 1, then direction 0 (scipy, independent)
        sp1 = make_interp_spline(t1, Y, k=q, axis=1)
        k0a, k1a = po.offset_domain(2, m[0], int(offs[s][0]))
        k0b, k1b = po.offset_domain(2, m[1], int(offs[s][1]))
        xa = np.arange(k0a, k1a + 1, dtype=float)
        xb = np.arange(k0b, k1b + 1, dtype=float)
        Z = make_interp_spline(t0, sp1(xb), k=q, axis=0)(xa)               # [len(xa), len(xb)]
        pts = np.stack(np.meshgrid(xa, xb, indexing="ij"), axis=-1).reshape(-1, 2).astype(np.int64)
        got = po._evaluate(sp, pts).reshape(len(xa), len(xb))
        assert np.abs(got - Z).max() < 1e-12 * np.abs(Y).max()
        checked += 1
    assert checked > 0


def _offdiag_max(X, prob):
    c = oracle.center_slot(prob.dim, prob.p)
    Y = X.copy()
    Y[c] = 0.0
    return np.abs(Y).max()


@pytest.mark.slow
@pytest.mark.parametrize("q", [1, 3])
def test_entry_error_rate(q):
    """|A - A~|_max ~ H^{q+1} at fixed h (thm:RegularityOfStencilFunctions, per offset)."""
    prob = _sinprod2((131, 131), 2)          # cardinal box of 129 indices: p + 128
    A = oracle.exact_matrix(prob)
    Ms = [4, 8, 16]
    errs = [_offdiag_max(po.per_offset_matrix(prob, M, q) - A, prob) for M in Ms]
    slopes = np.diff(np.log(errs)) / np.diff(np.log(Ms))
    assert np.all(slopes > q + 1 - 0.6), (errs, slopes)
    assert np.all(slopes < q + 1 + 1.5), (errs, slopes)
