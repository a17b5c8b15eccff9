"""Pins of the oracle's manufactured-solution load and error split (no GPU).

u(x) = prod_d sin(k pi x_d), the low- (k = 1) and high-frequency (k = 20)
solutions of the paper's Poisson experiments (Sec. 7.3) for general k.  F_i = a(u, B_i) and a(u, u) by the assembly's Gauss
rule are pinned against quantities fixed independently of the oracle:
  * identity map, kappa = 1: -Laplace u = n (k pi)^2 u, so for basis functions that
    vanish on the boundary F_i = n (k pi)^2 int u B_i, a tensor product of 1-D
    integrals computed here with scipy's adaptive quadrature and scipy's B-splines;
  * a(u, u) = n (k pi)^2 / 2^n for the identity map and kappa = 1;
  * sum_i F_i = a(u, 1) = 0 for any map and coefficient (partition of unity);
  * the discretisation error ||u - u_h||_a, from Galerkin orthogonality, falls
    like h^p under refinement (the H^1 rate of degree-p splines) and equals
    the directly computed energy of u - u_h for the identity map, kappa = 1.
"""
import numpy as np
import pytest

import iga_workloads as W
from oracle import manufactured, exact_matrix, cg, interior_dofs
from oracle.surrogate import multi_index

scipy = pytest.importorskip("scipy")
from scipy.integrate import quad  # noqa: E402
from scipy.interpolate import BSpline  # noqa: E402


def _knots(p, n_el):
    return np.concatenate([np.zeros(p), np.linspace(0.0, 1.0, n_el + 1), np.ones(p)])


def _sin_moments(p, n_el, k=1):
    """int_0^1 sin(k pi x) B_i(x) dx for every B-spline of the open uniform knot vector (element by element)."""
    t = _knots(p, n_el)
    m = n_el + p
    out = np.zeros(m)
    for i in range(m):
        b = BSpline.basis_element(t[i:i + p + 2], extrapolate=False)
        lo, hi = t[i], t[i + p + 1]
        brk = np.unique(t[i:i + p + 2])
        tot = 0.0
        for a, c in zip(brk[:-1], brk[1:]):
            if c > a:
                tot += quad(lambda x: np.sin(k * np.pi * x) * np.nan_to_num(b(x)), a, c, epsabs=1e-15, epsrel=1e-13)[0]
        out[i] = tot
        assert lo <= hi
    return out


@pytest.mark.parametrize("dim,p,n_el,k", [(2, 2, (12, 10), 1), (3, 3, (7, 6, 8), 1), (2, 4, (9, 11), 1),
                                          (2, 3, (24, 22), 3)])
def test_load_identity_map_equals_laplacian_moments(dim, p, n_el, k):
    prob = W.Problem(dim=dim, p=p, n_el=n_el, map_kind="identity", kappa_kind="const", kappa_a=1.0)
    F, en = manufactured.manufactured_load(prob, freq=k)
    mom = [_sin_moments(p, ne, k) for ne in n_el]
    mi = multi_index(np.arange(prob.N), np.array(prob.m))
    ref = dim * (k * np.pi) ** 2 * np.prod([mom[d][mi[:, d]] for d in range(dim)], axis=0)
    I = interior_dofs(prob)
    assert np.abs(F[I] - ref[I]).max() <= 2e-6 * np.abs(ref).max()
    assert abs(en - dim * (k * np.pi) ** 2 / 2 ** dim) <= 1e-6 * en


@pytest.mark.parametrize("prob", [
    W.Problem(dim=2, p=2, n_el=(10, 9), map_kind="sinprod", map_amp=0.05, kappa_kind="sin2d", kappa_a=1.0, kappa_b=0.5),
    W.Problem(dim=3, p=2, n_el=(6, 5, 7), map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d", kappa_b=0.5),
])
def test_load_sums_to_zero(prob):
    F, en = manufactured.manufactured_load(prob)
    assert abs(F.sum()) <= 1e-12 * np.abs(F).sum()
    assert en > 0


def test_discretisation_error_rate_and_orthogonality_identity():
    """||u - u_h||_a from Galerkin orthogonality halves like h^p; on the identity map with kappa = 1 it
    equals sqrt(a(u,u) - 2 F.u_h + u_h^T A u_h) computed term by term."""
    p, errs = 2, []
    for n in (8, 16, 32):
        prob = W.Problem(dim=2, p=p, n_el=(n, n), map_kind="identity", kappa_kind="const", kappa_a=1.0)
        A = exact_matrix(prob)
        F, en = manufactured.manufactured_load(prob)
        disc, cons = manufactured.error_split(prob, A, A, F, en)
        assert cons == 0.0
        u_h, _, _ = cg(A, prob, F, tol=1e-14)
        from oracle import apply
        direct = en - 2 * F @ u_h + u_h @ apply(A, prob, u_h)
        assert abs(direct / en - disc ** 2) <= 1e-9
        errs.append(disc)
    rates = [np.log2(errs[k] / errs[k + 1]) for k in range(2)]
    assert all(abs(r - p) < 0.15 for r in rates), rates


def test_consistency_error_of_surrogate_vanishes_for_M1_and_grows_with_M():
    from oracle import surrogate_matrix
    prob = W.Problem(dim=2, p=2, n_el=(24, 24), map_kind="sinprod", map_amp=0.05, kappa_kind="sin2d", kappa_a=1.0,
                     kappa_b=0.5)
    A = exact_matrix(prob)
    F, en = manufactured.manufactured_load(prob)
    _, c1 = manufactured.error_split(prob, A, surrogate_matrix(prob, 1, 3), F, en)
    _, c4 = manufactured.error_split(prob, A, surrogate_matrix(prob, 4, 3), F, en)
    _, c8 = manufactured.error_split(prob, A, surrogate_matrix(prob, 8, 3), F, en)
    assert c1 <= 1e-10 and 0 < c4 < c8
