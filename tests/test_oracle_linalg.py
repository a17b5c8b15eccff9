"""Pins of the oracle's stencil SpMV and CG (no GPU): dense matvec and dense solve."""
import numpy as np

import iga_workloads as W
import oracle


def test_apply_matches_dense():
    prob = W.CFG_2D_P2.problem
    A = oracle.exact_matrix(prob)
    D = oracle.ell_to_dense(A, prob)
    x = W.normal_vector(prob.N)
    np.testing.assert_allclose(oracle.apply(A, prob, x), D @ x, rtol=0, atol=1e-13 * np.abs(D).max())
    # constants are in the kernel (Sec. 5.3)
    assert np.abs(oracle.apply(A, prob, np.ones(prob.N))).max() < 1e-13


def test_cg_matches_dense_solve():
    prob = W.CFG_2D_P2.problem
    A = oracle.surrogate_matrix(prob, W.CFG_2D_P2.M, W.CFG_2D_P2.q)
    f = W.rhs_vector(prob.N)
    u, it, res = oracle.cg(A, prob, f, tol=1e-13)
    I = oracle.interior_dofs(prob)
    D = oracle.ell_to_dense(A, prob)[np.ix_(I, I)]
    ref = np.linalg.solve(D, f[I])
    assert res < 1e-13
    np.testing.assert_allclose(u[I], ref, rtol=0, atol=1e-10 * np.abs(ref).max())
    assert np.all(u[np.setdiff1d(np.arange(prob.N), I)] == 0.0)
    # interior dofs: every index in [1, m-2]
    assert len(I) == np.prod([m - 2 for m in prob.m])
