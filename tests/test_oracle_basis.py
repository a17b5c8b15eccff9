"""Pins of the oracle's quadrature rule and B-spline basis (no GPU).

Gauss-Legendre nodes/weights are checked against numpy's leggauss and against
exact monomial integrals; the Cox-de Boor values against scipy's BSpline (an
independent implementation), partition of unity and finite differences; the
knot construction against the worked example of Sec. 2.2 (eq. OpenKnotVectorEg).
"""
import os

import numpy as np
import pytest
from scipy.interpolate import BSpline

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7])
def test_gauss_legendre_matches_numpy_and_is_exact(n):
    x, w = oracle.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, 0.5 * (xr + 1.0), rtol=0, atol=5e-16)
    np.testing.assert_allclose(w, 0.5 * wr, rtol=0, atol=5e-16)
    # exact for monomials up to degree 2n-1 on [0,1]
    for k in range(2 * n):
        assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) < 1e-15
    # and not exact for degree 2n
    assert abs(np.dot(w, x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-12


@pytest.mark.parametrize("p", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("n_el", [1, 3, 7])
def test_cox_de_boor_matches_scipy(p, n_el):
    if n_el < 1:
        pytest.skip()
    t = oracle.open_uniform_knots(p, n_el)
    assert len(t) == n_el + 2 * p + 1
    m = n_el + p
    rng = np.random.default_rng(p * 10 + n_el)
    pts = np.concatenate([rng.uniform(0, 1, 25), [0.0, 1.0, 0.5]])
    for x in pts:
        v, d = oracle.bspline_all(p, t, x)
        assert len(v) == m
        # partition of unity and zero-sum derivatives
        assert abs(v.sum() - 1.0) < 1e-14
        if p > 0:
            assert abs(d.sum()) < 1e-11
        for i in range(m):
            c = np.zeros(m)
            c[i] = 1.0
            spl = BSpline(t, c, p, extrapolate=False)
            ref = spl(x)
            if np.isnan(ref):      # scipy leaves x == 1 outside; compare from the left
                ref = BSpline(t, c, p)(x)
            assert abs(v[i] - ref) < 1e-14, (i, x)
            if p > 0 and 0.0 < x < 1.0:
                assert abs(d[i] - spl.derivative()(x)) < 1e-11 * max(1.0, n_el * p)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_derivative_matches_finite_differences(p):
    n_el = 6
    t = oracle.open_uniform_knots(p, n_el)
    for x in [0.13, 0.41, 0.77]:
        _, d = oracle.bspline_all(p, t, x)
        eps = 1e-6
        vp, _ = oracle.bspline_all(p, t, x + eps)
        vm, _ = oracle.bspline_all(p, t, x - eps)
        np.testing.assert_allclose(d, (vp - vm) / (2 * eps), atol=1e-7 * n_el)


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            out[k] = int(v)
    return out


def test_paper_knot_example_cardinal_count():
    """Sec. 2.2 worked example: 21 functions, 17 identical up to translation."""
    g = _read_golden("paper_knot_example.txt")
    p, n_el = g["p"], g["n_intervals"]
    t = oracle.open_uniform_knots(p, n_el)
    m = n_el + p
    assert m == g["num_basis"]
    h = 1.0 / n_el
    # sample each function on its support, shifted to start at its first knot
    xs = np.linspace(0.0, (p + 1) * h, 61)[1:-1]

    def shape(i):
        return np.array([oracle.bspline_all(p, t, t[i] + x)[0][i] if t[i] + x <= 1.0 else np.nan for x in xs])

    ref = shape(m // 2)
    cardinal = [i for i in range(m) if np.allclose(shape(i), ref, atol=1e-13, equal_nan=False)]
    assert len(cardinal) == g["num_cardinal"]
    assert m - len(cardinal) == g["num_noncardinal"]
    # the cardinal ones are exactly the indices p..m-p-1 (0-based), Sec. 2.2
    assert cardinal == list(range(p, m - p))


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("m_extra", [0, 1, 5, 30])
def test_omega_box_matches_paper_interval(p, m_extra):
    """Sec. 4: Omega~ = [(3p+1)/(2(m-p)), 1-(3p+1)/(2(m-p))]^n holds exactly the midpoints
    x~^(k) = (k - (p+1)/2) h (1-based k in p+1..m-p) of the 0-based index box [2p, m-2p-1]."""
    m = 4 * p + 1 + m_extra
    h = 1.0 / (m - p)
    lo = (3 * p + 1) / (2 * (m - p))
    hi = 1.0 - lo
    inside = []
    for k1 in range(p + 1, m - p + 1):           # 1-based cardinal indices
        xt = (k1 - (p + 1) / 2) * h
        if lo - 1e-12 <= xt <= hi + 1e-12:
            inside.append(k1 - 1)                # 0-based
    k0, k1 = oracle.omega_box(p, m)
    assert inside == list(range(k0, k1 + 1))


def test_stencil_counts():
    """|D| = (2p+1)^n offsets (Sec. 3.2) and ((2p+1)^n + 1)/2 of them on or above the
    diagonal (Sec. 5.2)."""
    for dim in (2, 3):
        for p in range(1, 6):
            offs = oracle.offsets(dim, p)
            assert len(offs) == (2 * p + 1) ** dim
            c = oracle.center_slot(dim, p)
            assert np.all(offs[c] == 0)
            # colexicographic order: slot s > c  <=>  j > i  <=>  last nonzero component > 0
            for s, dl in enumerate(offs):
                nz = np.nonzero(dl)[0]
                if len(nz):
                    assert (s > c) == (dl[nz[-1]] > 0)
            assert len(range(c, len(offs))) == ((2 * p + 1) ** dim + 1) // 2
