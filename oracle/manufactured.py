"""TEST INFRASTRUCTURE (oracle): the manufactured solution of the paper's
Poisson experiments and the split of the surrogate solution's error into a
discretisation and a consistency part (Sec. 7.3).

u(x) = prod_d sin(k pi x_d) (k = 1: the "low-frequency", k = 20: the
"high-frequency" solution of Sec. 7.3; k a positive integer) vanishes on the
boundary of the unit square / cube, so for maps of the unit cube onto
itself it solves the homogeneous Dirichlet problem -div(kappa grad u) = f.
With the load F_i = a(u, B_i) (the Galerkin load of that f, no f needed) and
the same Gauss rule a_h as the stiffness matrix, Galerkin orthogonality gives
the discretisation error of the exact-quadrature solution u_h in the energy
norm without knowing f:
    ||u - u_h||_a^2 = a_h(u, u) - F . u_h .
The consistency error is ||u_h - u~_h||_A with u~_h the surrogate solution
(the two terms of the a-priori bound after eq. APrioriBoundL2).  The paper's
rule of thumb keeps the consistency error at or below 5 % of the
discretisation error.
"""
from __future__ import annotations

import numpy as np

from ._lib import _dptr, lib, make_problem
from .linalg import apply, cg


def manufactured_load(prob, freq: int = 1):
    """(F, energy): F_i = a(u, B_i) for every basis function i (colexicographic), and a(u, u)."""
    P = make_problem(prob)
    N = int(np.prod([e + prob.p for e in prob.n_el]))
    F = np.zeros(N)
    en = np.zeros(1)
    rc = lib().orc_manufactured_load(P, int(freq), _dptr(F), _dptr(en))
    if rc != 0:
        raise ValueError(f"orc_manufactured_load failed ({rc})")
    return F, float(en[0])


def error_split(prob, exact_vals: np.ndarray, surrogate_vals: np.ndarray, F: np.ndarray, energy: float,
                tol: float = 1e-13):
    """Relative energy-norm errors (disc = ||u - u_h||_a / ||u||_a, cons = ||u_h - u~_h||_A / ||u||_a)
    of the Dirichlet-reduced solves with the exact and the surrogate matrix."""
    u_h, _, _ = cg(exact_vals, prob, F, tol=tol)
    u_s, _, _ = cg(surrogate_vals, prob, F, tol=tol)
    disc2 = energy - float(F @ u_h)
    d = u_h - u_s
    cons2 = float(d @ apply(exact_vals, prob, d))
    return np.sqrt(max(disc2, 0.0) / energy), np.sqrt(max(cons2, 0.0) / energy)
