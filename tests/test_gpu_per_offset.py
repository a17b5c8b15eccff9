"""GPU parity of the surrogate with per-offset interpolation domains (Omega~_delta).

Same bar as the common-domain surrogate: every entry within 1e-12 (FP64
values) or 1e-5 (FP32 values) of the FP64 oracle relative to the largest
entry; full-size workloads on sampled rows plus zero row sums and symmetry.
"""
import numpy as np
import pytest

import iga_workloads as W
import oracle
from oracle import per_offset as po

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


def gpu_po(iga, prob, M, q, dtype="f64"):
    A = iga.assemble_surrogate(prob, M, q, dtype=dtype, domains="per_offset")
    v = A.values_host()
    A.destroy()
    return v


def _sp2(n_el, p, amp=0.05):
    return W.Problem(dim=2, p=p, n_el=n_el, map_kind="sinprod", map_amp=amp, kappa_kind="sin2d",
                     kappa_a=1.0, kappa_b=0.5)


def _sp3(n_el, p):
    return W.Problem(dim=3, p=p, n_el=n_el, map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d", kappa_b=0.5)


CASES = [
    (W.CFG_2D_P2.problem, 4, 3),
    (W.CFG_2D_P2.problem, 3, 2),
    (W.CFG_2D_P2.problem, 1, 3),             # M = 1: every cardinal index is a sample
    (W.CFG_2D_P2.problem, 40, 3),            # M > cardinal range: each offset samples its two ends
    (_sp2((21, 17), 1), 3, 5),
    (_sp2((30, 26), 3), 4, 4),
    (_sp2((40, 33), 5), 6, 7),
    (_sp2((9, 10), 3), 4, 3),                # end runs meet: every cardinal index sampled
    (_sp2((4, 4), 3), 4, 3),                 # m = 2p + 1: one cardinal index per direction
    (_sp2((5, 6), 3), 2, 3),                 # m = 2p + 2, 2p + 3
    (_sp3((13, 12, 14), 2), 3, 3),
    (_sp3((17, 15, 16), 3), 2, 3),
    (_sp3((11, 9, 10), 1), 2, 2),
    (_sp3((19, 18, 17), 4), 2, 1),
    (_sp3((3, 3, 3), 2), 2, 3),              # m = 2p + 1 in 3-D
    (_sp3((30, 7, 9), 2), 5, 2),             # anisotropic
]


def _id(x):
    return f"{x.dim}d_p{x.p}_{'x'.join(map(str, x.n_el))}" if hasattr(x, "dim") else str(x)


@pytest.mark.parametrize("arith", ["df64", "fp64"], indirect=True)
@pytest.mark.parametrize("prob,M,q", CASES, ids=_id)
def test_per_offset_full_matrix(iga, prob, M, q, arith):
    iga.set_arithmetic("f64", arith)
    ref = po.per_offset_matrix(prob, M, q)
    assert rel(gpu_po(iga, prob, M, q), ref) <= TOL64


@pytest.mark.parametrize("arith", ["fp32", "df64"], indirect=True)
@pytest.mark.parametrize("idx", [5, 11, 13])
def test_per_offset_f32(iga, idx, arith):
    iga.set_arithmetic("f32", arith)
    prob, M, q = CASES[idx]
    ref = po.per_offset_matrix(prob, M, q)
    assert rel(gpu_po(iga, prob, M, q, "f32"), ref) <= TOL32


def test_per_offset_polynomial_reproduction(iga):
    """Identity map, kappa in Q_3, q = 3: per-offset surrogate == exact on the GPU."""
    rng = np.random.default_rng(5)
    coef = rng.uniform(0.1, 1.0, 64) / 64
    coef[0] += 1.0
    prob = W.Problem(dim=3, p=2, n_el=(16, 15, 14), kappa_kind="poly", kappa_deg=3, kappa_poly=tuple(coef))
    A = iga.assemble_exact(prob)
    ex = A.values_host()
    A.destroy()
    assert rel(gpu_po(iga, prob, 3, 3), ex) <= 1e-12


def test_per_offset_bad_domains_rejected(iga):
    with pytest.raises(iga.IgaError) as ei:
        pt, mp, kp = iga._structs(W.CFG_2D_P2.problem)
        import ctypes
        h = ctypes.c_void_p()
        iga._check(iga.load().iga_assemble_surrogate_domains(ctypes.byref(pt), 2, ctypes.byref(mp), ctypes.byref(kp),
                                                             4, 3, 7, 0, None, ctypes.byref(h)))
    assert ei.value.code == -1


def _rows(prob, k, seed):
    p, m = prob.p, np.array(prob.m)
    rows = list(W.sample_rows(prob.N, k, seed))
    stride = np.cumprod([1] + list(m[:-1]))
    special = [np.zeros(prob.dim, dtype=int), m - 1, np.full(prob.dim, p), np.full(prob.dim, p - 1),
               np.full(prob.dim, p + 1), np.full(prob.dim, 2 * p), m - p - 1, m - p, m - p - 2, m // 2]
    rows += [int((np.array(s) * stride).sum()) for s in special]
    return np.unique(np.array(rows, dtype=np.int64))


def _properties(iga, A, vals, prob, tol, scale, f64):
    """Zero row sums and symmetry at full size (eq. DefinitionOfSurrogateMatrixSymmetricKernel)."""
    ones = torch.ones(prob.N, dtype=A.torch_dtype, device="cuda")
    assert A.apply(ones).double().abs().max().item() <= (1e-12 if f64 else 1e-4) * scale
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
    assert worst <= tol * scale


def test_full_size_per_offset_sampled_rows(iga):
    """64^3, p = 3, FP64 values: sampled rows against the full per-offset oracle."""
    wl = W.CFG_3D_P3
    prob = wl.problem
    A = iga.assemble_surrogate(prob, wl.M, wl.q, dtype=wl.dtype, domains="per_offset")
    vals = A.values()
    rows = _rows(prob, 40, seed=3)
    got = vals[:, torch.from_numpy(rows).cuda()].double().cpu().numpy().T
    setup = po.per_offset_setup(prob, wl.M, wl.q)
    ref = po.per_offset_rows(prob, wl.M, wl.q, rows, setup)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= TOL64 * scale
    _properties(iga, A, vals, prob, TOL64, scale, True)
    A.destroy()


def test_full_size_per_offset_f32_exact_entries(iga):
    """96^3, p = 4, FP32 values.  The oracle's interpolants need 8000 exact sample
    rows (minutes on the host), so the sampled rows are checked on the entries the
    method fixes one by one -- entries with a non-cardinal basis function and the
    upper entries of sample rows are exact quadrature values -- plus the
    properties, and the interpolated entries against the exact ones within the
    surrogate's own error."""
    wl = W.CFG_3D_P4
    prob = wl.problem
    p, m = prob.p, np.array(prob.m)
    A = iga.assemble_surrogate(prob, wl.M, wl.q, dtype=wl.dtype, domains="per_offset")
    vals = A.values()
    union = [po.union_samples(p, md, wl.M) for md in m]
    rng = np.random.default_rng(4)
    samp = np.stack([rng.choice(u, 12) for u in union], axis=1)          # sample rows
    rows = np.unique(np.concatenate([_rows(prob, 24, seed=4), oracle.flat_index(samp, m)]))
    got = vals[:, torch.from_numpy(rows).cuda()].double().cpu().numpy().T
    ex = oracle.exact_rows(prob, rows)
    scale = np.abs(ex).max()
    mi = oracle.multi_index(rows, m)
    c0, c1 = p, m - p - 1
    c = oracle.center_slot(prob.dim, p)
    offs = oracle.offsets(prob.dim, p)
    for s in range(prob.S):
        if s == c:
            continue
        mj = mi + offs[s]
        inside = np.all((mj >= 0) & (mj < m), axis=1)
        both = np.all((mi >= c0) & (mi <= c1) & (mj >= c0) & (mj <= c1), axis=1)
        fixed = inside & ~both
        if s > c:       # upper entries at the offset's own sample rows
            own = np.all([np.isin(mi[:, d], po.offset_samples(p, int(m[d]), wl.M, int(offs[s][d])))
                          for d in range(prob.dim)], axis=0)
            fixed |= both & own
        d_fixed = np.abs(got[fixed, s] - ex[fixed, s])
        if d_fixed.size:
            assert d_fixed.max() <= TOL32 * scale, s
        interp = inside & ~fixed
        if np.any(interp):
            assert np.abs(got[interp, s] - ex[interp, s]).max() <= 0.05 * scale
    _properties(iga, A, vals, prob, TOL32, scale, False)
    A.destroy()
