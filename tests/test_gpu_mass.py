"""GPU parity of the mass matrix and its symmetric surrogate (Sec. 8, eq.
DefinitionOfSurrogateMatrixSymmetric) against the FP64 oracle (oracle.mass).

Bar: every entry within 1e-12 (FP64 values) or 1e-5 (FP32 values) of the
oracle relative to the largest entry; full-size workloads on sampled rows plus
the properties that hold at any size (symmetry, the sum of all entries is the
measure of Omega).
"""
import numpy as np
import pytest

import iga_workloads as W
import oracle
from oracle import mass

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5


@pytest.fixture(scope="module")
def iga():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1904_06971_gb300 as m
    m.load()
    return m


@pytest.fixture
def arith(iga, request):
    saved = {dt: iga.get_arithmetic(dt) for dt in ("f64", "f32")}
    yield request.param
    for dt, a in saved.items():
        iga.set_arithmetic(dt, a)


def rel(X, ref):
    return oracle.relative_entry_error(X, ref)


def _host(A):
    v = A.values_host()
    A.destroy()
    return v


_AFF = (1.1, 0.2, -0.1, 0.05, 0.9, 0.3, -0.2, 0.1, 1.2, 0.1, -0.2, 0.3)


def _sp(dim, n_el, p, amp=None):
    return W.Problem(dim=dim, p=p, n_el=n_el, map_kind="sinprod", map_amp=amp if amp else (0.05 if dim == 2 else 0.03))


EXACT = [
    _sp(2, (7, 9), 1), _sp(2, (12, 10), 2), _sp(2, (9, 11), 3), _sp(2, (10, 8), 4), _sp(2, (11, 12), 5),
    _sp(3, (5, 6, 4), 1), _sp(3, (7, 6, 8), 2), _sp(3, (6, 7, 5), 3), _sp(3, (5, 5, 6), 4),
    W.Problem(dim=3, p=2, n_el=(6, 5, 7), map_kind="affine", affine=_AFF),
    W.Problem(dim=2, p=3, n_el=(8, 7)),
]

SURR = [
    (_sp(2, (20, 23), 2), 3, 3),
    (_sp(2, (20, 23), 2), 1, 3),             # M = 1: the exact matrix
    (_sp(2, (20, 23), 2), 40, 3),            # one sample (the box's first and last index) per direction
    (_sp(2, (25, 22), 3), 4, 2),
    (_sp(2, (30, 26), 1), 3, 5),
    (_sp(2, (40, 33), 5), 6, 7),
    (_sp(2, (4, 4), 3), 4, 3),               # Omega~ empty: every row exact
    (_sp(2, (10, 11), 3), 2, 3),             # Omega~ of one / two indices
    (_sp(3, (13, 12, 14), 2), 3, 3),
    (_sp(3, (17, 15, 16), 3), 2, 3),
    (_sp(3, (11, 9, 10), 1), 2, 2),
    (_sp(3, (19, 18, 17), 4), 2, 1),
    (_sp(3, (30, 7, 9), 2), 5, 2),           # anisotropic, thin Omega~
]


def _id(x):
    return f"{x.dim}d_p{x.p}_{'x'.join(map(str, x.n_el))}_{x.map_kind}" if hasattr(x, "dim") else str(x)


@pytest.mark.parametrize("arith", ["df64", "fp64"], indirect=True)
@pytest.mark.parametrize("prob", EXACT, ids=_id)
def test_mass_exact_full_matrix(iga, prob, arith):
    iga.set_arithmetic("f64", arith)
    assert rel(_host(iga.assemble_mass(prob)), mass.mass_matrix(prob)) <= TOL64


@pytest.mark.parametrize("arith", ["df64", "fp64"], indirect=True)
@pytest.mark.parametrize("prob,M,q", SURR, ids=_id)
def test_mass_surrogate_full_matrix(iga, prob, M, q, arith):
    iga.set_arithmetic("f64", arith)
    assert rel(_host(iga.assemble_mass_surrogate(prob, M, q)), mass.mass_surrogate_matrix(prob, M, q)) <= TOL64


@pytest.mark.parametrize("arith", ["fp32", "df64"], indirect=True)
@pytest.mark.parametrize("idx", [0, 3, 9])
def test_mass_surrogate_f32(iga, idx, arith):
    iga.set_arithmetic("f32", arith)
    prob, M, q = SURR[idx]
    assert rel(_host(iga.assemble_mass_surrogate(prob, M, q, dtype="f32")), mass.mass_surrogate_matrix(prob, M, q)) \
        <= TOL32
    assert rel(_host(iga.assemble_mass(prob, dtype="f32")), mass.mass_matrix(prob)) <= TOL32


@pytest.mark.parametrize("dim,q", [(2, 1), (3, 2), (3, 3)])
def test_mass_affine_reproduction(iga, dim, q):
    """Mass-matrix corollary (Sec. 8): affine map, q >= dim - 1 => M~ = M, on the GPU."""
    prob = W.Problem(dim=dim, p=2, n_el=(18, 17, 16)[:dim], map_kind="affine", affine=_AFF)
    ex = _host(iga.assemble_mass(prob))
    assert rel(_host(iga.assemble_mass_surrogate(prob, 4, q)), ex) <= TOL64
    assert abs(ex.sum() - abs(np.linalg.det(np.array(_AFF[:9]).reshape(3, 3)[:dim, :dim]))) < 1e-12


def test_mass_handle_reuse_and_bad_args(iga):
    prob, M, q = SURR[0]
    A = iga.assemble_mass(prob)
    iga.assemble_mass_surrogate(prob, M, q, out=A)
    assert rel(A.values_host(), mass.mass_surrogate_matrix(prob, M, q)) <= TOL64
    with pytest.raises(iga.IgaError):
        iga.assemble_mass_surrogate(prob, 0, q)
    with pytest.raises(iga.IgaError):
        iga.assemble_mass_surrogate(_sp(2, (20, 24), 2), M, q, out=A)     # another patch into the same handle
    A.destroy()


def _rows(prob, k, seed):
    p, m = prob.p, np.array(prob.m)
    rows = list(W.sample_rows(prob.N, k, seed))
    stride = np.cumprod([1] + list(m[:-1]))
    special = [np.zeros(prob.dim, dtype=int), m - 1, np.full(prob.dim, 2 * p), np.full(prob.dim, 2 * p - 1),
               np.full(prob.dim, 2 * p + 1), m - 2 * p - 1, m - 2 * p, m - 2 * p - 2, m // 2]
    rows += [int((np.array(s) * stride).sum()) for s in special]
    return np.unique(np.array(rows, dtype=np.int64))


def _symmetry(prob, vals, tol):
    offs = oracle.offsets(prob.dim, prob.p)
    m = np.array(prob.m)
    mi = oracle.multi_index(np.arange(prob.N), m)
    worst = 0.0
    for s in range(prob.S // 2 + 1, prob.S, max(1, prob.S // 40)):
        mj = mi + offs[s]
        ok = np.all((mj >= 0) & (mj < m), axis=1)
        i = torch.from_numpy(np.nonzero(ok)[0]).cuda()
        j = torch.from_numpy(oracle.flat_index(mj[ok], m)).cuda()
        worst = max(worst, (vals[s, i] - vals[prob.S - 1 - s, j]).abs().max().item())
    assert worst <= tol


@pytest.mark.parametrize("wl", [W.CFG_3D_P3, W.CFG_3D_P4], ids=lambda w: w.name)
def test_full_size_mass_surrogate_sampled_rows(iga, wl):
    """64^3 p = 3 (FP64 values) and 96^3 p = 4 (FP32 values): sampled rows against
    the oracle's surrogate rows (its setup needs only the 8^3 / 12^3 exact sample
    rows), symmetry, and the total mass 1 (the sine-product map fixes the unit cube)."""
    prob = wl.problem
    tol = TOL64 if wl.dtype == "f64" else TOL32
    A = iga.assemble_mass_surrogate(prob, wl.M, wl.q, dtype=wl.dtype)
    vals = A.values()
    rows = _rows(prob, 30, seed=6)
    got = vals[:, torch.from_numpy(rows).cuda()].double().cpu().numpy().T
    setup = mass.mass_surrogate_setup(prob, wl.M, wl.q)
    ref = mass.mass_surrogate_rows(prob, wl.M, wl.q, rows, setup)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= tol * scale
    _symmetry(prob, vals, tol * scale)
    ones = torch.ones(prob.N, dtype=A.torch_dtype, device="cuda")
    assert abs(A.apply(ones).double().sum().item() - 1.0) < 1e-3        # within the surrogate's own error
    iga.assemble_mass(prob, dtype=wl.dtype, out=A)                       # the exact matrix into the same handle
    assert abs(A.apply(ones).double().sum().item() - 1.0) < (1e-6 if wl.dtype == "f64" else 1e-4)
    A.destroy()
