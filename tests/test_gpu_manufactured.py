"""GPU manufactured-solution load (iga_manufactured_load) against the oracle, and the
discretisation / consistency error split of the surrogate solution (Sec. 7.3) from GPU
assembly and GPU CG against the oracle's dense-algebra split."""
import numpy as np
import pytest

import iga_workloads as W
import oracle
from oracle import manufactured

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def iga():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1904_06971_gb300 as m
    m.load()
    return m


CASES = [
    W.CFG_2D_P2.problem,
    W.Problem(dim=3, p=3, n_el=(9, 8, 10), map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d", kappa_b=0.5),
    W.Problem(dim=2, p=4, n_el=(13, 11), map_kind="identity", kappa_kind="const", kappa_a=1.0),
    W.Problem(dim=3, p=2, n_el=(6, 7, 5), map_kind="affine",
              affine=(1.1, 0.2, -0.1, 0.05, 0.9, 0.3, -0.2, 0.1, 1.2, 0.1, 0.2, 0.3), kappa_kind="poly", kappa_deg=1,
              kappa_poly=tuple([1.0, 0.3, 0.2, 0.1, 0.25, 0.0, 0.05, 0.1])),
]


@pytest.mark.parametrize("freq", [1, 20])
@pytest.mark.parametrize("prob", CASES, ids=lambda q: f"{q.dim}d_p{q.p}_{q.map_kind}")
def test_manufactured_load_matches_oracle(iga, prob, freq):
    F, en = iga.manufactured_load(prob, freq=freq)
    Fr, enr = manufactured.manufactured_load(prob, freq=freq)
    assert np.abs(F.cpu().numpy() - Fr).max() <= 1e-12 * np.abs(Fr).max()
    assert abs(en.item() - enr) <= 1e-12 * enr


def test_error_split_matches_oracle(iga):
    """Discretisation error ||u - u_h||_a and consistency error ||u_h - u~_h||_A (relative to ||u||_a)
    from GPU matrices and GPU CG equal the oracle's dense split."""
    prob = W.CFG_2D_P2.problem
    M, q = W.CFG_2D_P2.M, W.CFG_2D_P2.q
    F, en = iga.manufactured_load(prob)
    E = iga.assemble_exact(prob)
    A = iga.assemble_surrogate(prob, M, q)
    u_h, _, _ = E.cg(F, tol=1e-13)
    u_s, _, _ = A.cg(F, tol=1e-13)
    disc = np.sqrt((en.item() - torch.dot(F, u_h).item()) / en.item())
    d = u_h - u_s
    cons = np.sqrt(torch.dot(d, E.apply(d)).item() / en.item())
    dr, cr = manufactured.error_split(prob, oracle.exact_matrix(prob), oracle.surrogate_matrix(prob, M, q),
                                      *manufactured.manufactured_load(prob))
    assert abs(disc - dr) <= 1e-6 * dr
    assert abs(cons - cr) <= 1e-5 * cr
    E.destroy()
    A.destroy()
