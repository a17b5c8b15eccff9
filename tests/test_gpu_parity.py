"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (relative to the largest stored entry, max |X - ref| / max |ref|):
FP64 values 1e-12, FP32 values 1e-5 (FP64 quadrature rounded to FP32 on store
and FP32 SpMV).  Small cases compare every entry; the full-size workloads
compare sampled rows the oracle computes one by one, plus properties that
hold at any size (symmetry, zero row sums).
"""
import numpy as np
import pytest

import iga_workloads as W
import oracle

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


def rel(X, ref):
    return oracle.relative_entry_error(X, ref)


@pytest.fixture
def arith(iga, request):
    """Run a test under a given contraction arithmetic, restoring the defaults after."""
    saved = {dt: iga.get_arithmetic(dt) for dt in ("f64", "f32")}
    yield request.param
    for dt, a in saved.items():
        iga.set_arithmetic(dt, a)


def use(iga, dtype, arith):
    iga.set_arithmetic(dtype, arith)


def gpu_exact(iga, prob, dtype="f64"):
    A = iga.assemble_exact(prob, dtype=dtype)
    v = A.values_host()
    A.destroy()
    return v


def gpu_surr(iga, prob, M, q, dtype="f64"):
    A = iga.assemble_surrogate(prob, M, q, dtype=dtype)
    v = A.values_host()
    A.destroy()
    return v


SMALL_EXACT = [
    W.CFG_2D_P2.problem,
    W.Problem(dim=2, p=1, n_el=(7, 9), map_kind="sinprod", map_amp=0.05, kappa_kind="sin2d", kappa_a=1.0, kappa_b=0.5),
    W.Problem(dim=2, p=4, n_el=(13, 11), map_kind="sinprod", map_amp=0.04, kappa_kind="sin2d", kappa_a=1.0, kappa_b=0.3),
    W.Problem(dim=2, p=5, n_el=(6, 17), map_kind="sinprod", map_amp=0.05, kappa_kind="sin2d", kappa_a=1.0, kappa_b=0.5),
    W.Problem(dim=3, p=1, n_el=(5, 6, 4), map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d", kappa_b=0.5),
    W.Problem(dim=3, p=2, n_el=(9, 7, 8), map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d", kappa_b=0.5),
    W.Problem(dim=3, p=3, n_el=(6, 7, 5), map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d", kappa_b=0.5),
    W.Problem(dim=3, p=4, n_el=(5, 5, 6), map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d", kappa_b=0.5),
    W.Problem(dim=3, p=2, n_el=(6, 6, 6), map_kind="affine",
              affine=(1.1, 0.2, -0.1, 0.05, 0.9, 0.3, -0.2, 0.1, 1.2, 0.1, 0.2, 0.3), kappa_kind="const", kappa_a=2.0),
]


@pytest.mark.parametrize("arith", ["df64", "fp64"], indirect=True)
@pytest.mark.parametrize("prob", SMALL_EXACT, ids=lambda q: f"{q.dim}d_p{q.p}_{'x'.join(map(str, q.n_el))}")
def test_exact_full_matrix(iga, prob, arith):
    use(iga, "f64", arith)
    ref = oracle.exact_matrix(prob)
    assert rel(gpu_exact(iga, prob), ref) <= TOL64


# Entry error of the FP64-value contractions by degree.  Besides the global
# measure (relative to the largest entry), every stencil slot s is held to its
# own scale, max_i |X_si - ref_si| / max_i |ref_si|: the far-corner slots are
# ~1e-3 of the diagonal, so a global 1e-12 alone would let them carry ~1e-9
# relative errors.  Bounds: native FP64 reaches ~1e-14 (1e-3-term diagonal sums),
# double-float products carry ~2^-48 ~ 3.6e-15 per operation and reach a few 1e-13.
ENTRY_BOUND = {"fp64": 5e-14, "df64": 5e-13}
SLOT_BOUND = {"fp64": 1e-11, "df64": 1e-10}


@pytest.mark.parametrize("arith", ["df64", "fp64"], indirect=True)
@pytest.mark.parametrize("prob", [SMALL_EXACT[i] for i in (1, 2, 3, 4, 5, 6, 7)],
                         ids=lambda q: f"{q.dim}d_p{q.p}_{'x'.join(map(str, q.n_el))}")
def test_entry_error_by_degree(iga, prob, arith):
    use(iga, "f64", arith)
    ref = oracle.exact_matrix(prob)
    got = gpu_exact(iga, prob)
    glob = rel(got, ref)
    scale = np.max(np.abs(ref), axis=1)
    err = np.max(np.abs(got - ref), axis=1)
    live = scale > 0
    per_slot = float(np.max(err[live] / scale[live]))
    print(f"p={prob.p} dim={prob.dim} {arith}: global {glob:.2e}, worst slot {per_slot:.2e}")
    assert glob <= ENTRY_BOUND[arith]
    assert per_slot <= SLOT_BOUND[arith]


@pytest.mark.parametrize("arith", ["fp32", "df64", "fp64"], indirect=True)
@pytest.mark.parametrize("idx", [3, 6, 7])
def test_exact_f32(iga, idx, arith):
    use(iga, "f32", arith)
    prob = SMALL_EXACT[idx]
    ref = oracle.exact_matrix(prob)
    v = gpu_exact(iga, prob, "f32")
    assert v.dtype == np.float32
    assert rel(v, ref) <= TOL32


# patches with rows whose stencil stays among cardinal B-splines in direction 0
# (m_0 >= 4p + 1): the FP32-value stage X of those rows runs on the tensor cores
# under IGA_ARITH_BF16X3; line counts from a partial 128-line tile to many tiles
TC_EXACT = [
    W.Problem(dim=3, p=4, n_el=(20, 6, 5), map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d", kappa_b=0.5),
    W.Problem(dim=2, p=3, n_el=(40, 9), map_kind="sinprod", map_amp=0.05, kappa_kind="sin2d", kappa_a=1.0,
              kappa_b=0.5),
    W.Problem(dim=3, p=2, n_el=(14, 9, 8), map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d", kappa_b=0.4),
    W.Problem(dim=3, p=5, n_el=(24, 6, 6), map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d", kappa_b=0.5),
    W.Problem(dim=3, p=3, n_el=(30, 13, 11), map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d", kappa_b=0.5),
    W.Problem(dim=3, p=4, n_el=(17, 7, 6), map_kind="affine",
              affine=(1.1, 0.2, -0.1, 0.05, 0.9, 0.3, -0.2, 0.1, 1.2, 0.1, 0.2, 0.3), kappa_kind="const", kappa_a=2.0),
]


@pytest.mark.parametrize("arith", ["bf16x3"], indirect=True)
@pytest.mark.parametrize("prob", TC_EXACT, ids=lambda q: f"{q.dim}d_p{q.p}_{'x'.join(map(str, q.n_el))}")
def test_exact_f32_tensor_core_stage(iga, prob, arith):
    """Tensor-core stage X (BF16 parts, FP32 accumulation) against the FP64 oracle at the FP32 tolerance,
    and against the FP32 CUDA-core contraction of the same matrix."""
    iga.set_arithmetic("f32", "fp32")
    ref32 = gpu_exact(iga, prob, "f32")
    use(iga, "f32", arith)
    assert iga.get_arithmetic("f32") == "bf16x3"
    iga.profile_read()
    iga.profile_enable(True)
    v = gpu_exact(iga, prob, "f32")
    iga.profile_enable(False)
    prof = iga.profile_read()
    assert prof["stage_x_tc"][0] >= 1            # the tensor-core kernel ran
    ref = oracle.exact_matrix(prob)
    assert rel(v, ref) <= TOL32
    assert rel(v, ref32.astype(np.float64)) <= 2e-6


@pytest.mark.parametrize("arith", ["df64_tc"], indirect=True)
@pytest.mark.parametrize("prob", TC_EXACT, ids=lambda q: f"{q.dim}d_p{q.p}_{'x'.join(map(str, q.n_el))}")
def test_exact_f64_tensor_core_stage(iga, prob, arith):
    """FP64 values with stage X of the cardinal rows as exact BF16 digit products on the tensor cores:
    the FP64 tolerance against the oracle, and agreement with the double-float CUDA-core contraction."""
    iga.set_arithmetic("f64", "df64")
    ref_df = gpu_exact(iga, prob)
    use(iga, "f64", arith)
    assert iga.get_arithmetic("f64") == "df64_tc"
    iga.profile_read()
    iga.profile_enable(True)
    v = gpu_exact(iga, prob)
    iga.profile_enable(False)
    assert iga.profile_read()["stage_x_tc"][0] >= 2      # group shifts + at least one stage launch
    assert rel(v, oracle.exact_matrix(prob)) <= TOL64
    assert rel(v, ref_df) <= TOL64


SMALL_SURR = [
    (W.CFG_2D_P2.problem, 4, 3),
    (W.CFG_2D_P2.problem, 3, 2),
    (W.CFG_2D_P2.problem, 5, 0),
    (W.CFG_2D_P2.problem, 1, 3),            # M = 1: every Omega~ point is a sample
    (W.CFG_2D_P2.problem, 40, 3),           # M > L: two samples, degree lowered to 1
    (W.Problem(dim=2, p=1, n_el=(21, 17), map_kind="sinprod", map_amp=0.05, kappa_kind="sin2d",
               kappa_a=1.0, kappa_b=0.5), 3, 5),
    (W.Problem(dim=2, p=3, n_el=(30, 26), map_kind="sinprod", map_amp=0.05, kappa_kind="sin2d",
               kappa_a=1.0, kappa_b=0.5), 4, 4),
    (W.Problem(dim=2, p=5, n_el=(40, 33), map_kind="sinprod", map_amp=0.05, kappa_kind="sin2d",
               kappa_a=1.0, kappa_b=0.5), 6, 7),
    (W.Problem(dim=2, p=3, n_el=(9, 10), map_kind="sinprod", map_amp=0.05, kappa_kind="sin2d",
               kappa_a=1.0, kappa_b=0.5), 4, 3),    # Omega~ empty: all rows exact
    (W.Problem(dim=3, p=2, n_el=(13, 12, 14), map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d",
               kappa_b=0.5), 3, 3),
    (W.Problem(dim=3, p=3, n_el=(17, 15, 16), map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d",
               kappa_b=0.5), 2, 3),
    (W.Problem(dim=3, p=1, n_el=(11, 9, 10), map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d",
               kappa_b=0.5), 2, 2),
    (W.Problem(dim=3, p=4, n_el=(19, 18, 17), map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d",
               kappa_b=0.5), 2, 1),
]


@pytest.mark.parametrize("arith", ["df64", "fp64", "df64_tc"], indirect=True)
@pytest.mark.parametrize("prob,M,q", SMALL_SURR,
                         ids=lambda x: f"{x.dim}d_p{x.p}_{'x'.join(map(str, x.n_el))}" if hasattr(x, "dim") else str(x))
def test_surrogate_full_matrix(iga, prob, M, q, arith):
    use(iga, "f64", arith)
    ref = oracle.surrogate_matrix(prob, M, q)
    got = gpu_surr(iga, prob, M, q)
    assert rel(got, ref) <= TOL64


@pytest.mark.parametrize("arith", ["fp32", "df64", "bf16x3"], indirect=True)
@pytest.mark.parametrize("idx", [7, 9, 12])
def test_surrogate_f32(iga, idx, arith):
    use(iga, "f32", arith)
    prob, M, q = SMALL_SURR[idx]
    ref = oracle.surrogate_matrix(prob, M, q)
    assert rel(gpu_surr(iga, prob, M, q, "f32"), ref) <= TOL32


def test_polynomial_reproduction_on_gpu(iga):
    """Identity map, kappa in Q_3, q = 3: GPU surrogate == GPU exact (prop:PolynomialReproduction)."""
    rng = np.random.default_rng(4)
    coef = np.zeros(64)
    coef[:64] = rng.uniform(0.1, 1.0, 64) / 64
    coef[0] += 1.0
    prob = W.Problem(dim=3, p=2, n_el=(16, 15, 14), kappa_kind="poly", kappa_deg=3, kappa_poly=tuple(coef))
    ex = gpu_exact(iga, prob)
    su = gpu_surr(iga, prob, 3, 3)
    assert rel(su, ex) <= 1e-12
    assert rel(ex, oracle.exact_matrix(prob)) <= TOL64


def test_handle_reuse_and_spmv(iga):
    prob = SMALL_SURR[10][0]
    A = iga.assemble_surrogate(prob, 2, 3)
    v1 = A.values_host()
    iga.assemble_surrogate(prob, 2, 3, out=A)
    v2 = A.values_host()
    assert np.array_equal(v1, v2)            # deterministic, storage reused
    x = W.normal_vector(prob.N, seed=3)
    yref = oracle.apply(v1, prob, x)
    y = A.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    scale = np.abs(v1).max() * np.abs(x).max()
    assert np.abs(y - yref).max() <= 1e-13 * scale * prob.S
    yh = A.apply_host(x)
    assert np.array_equal(yh, y)
    ones = torch.ones(prob.N, dtype=torch.float64, device="cuda")
    assert A.apply(ones).abs().max().item() <= 1e-13 * np.abs(v1).max() * prob.S
    A.destroy()


def test_spmv_f32(iga):
    prob = SMALL_EXACT[7]
    A = iga.assemble_exact(prob, dtype="f32")
    v = A.values_host()
    x = W.normal_vector(prob.N, seed=5).astype(np.float32)
    yref = oracle.apply(v.astype(np.float64), prob, x.astype(np.float64))
    y = A.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    scale = np.abs(v).max() * np.abs(x).max() * prob.S
    assert np.abs(y - yref).max() <= 1e-6 * scale
    A.destroy()


# ---------------------------------------------------------------------------
# full-size workloads: sampled rows + properties
# ---------------------------------------------------------------------------
def _sampled_rows(prob, k, seed):
    """k random rows plus rows near the Omega~ boundary and the patch corners."""
    p, m = prob.p, np.array(prob.m)
    rows = list(W.sample_rows(prob.N, k, seed))
    stride = np.cumprod([1] + list(m[:-1]))
    special = [np.zeros(prob.dim, dtype=int), m - 1, np.full(prob.dim, 2 * p), np.full(prob.dim, 2 * p - 1),
               m - 2 * p - 1, m - 2 * p, np.full(prob.dim, 3 * p), m // 2]
    rows += [int((np.array(s) * stride).sum()) for s in special]
    return np.unique(np.array(rows, dtype=np.int64))


@pytest.mark.parametrize("wl,arith", [(W.CFG_3D_P3, "df64"), (W.CFG_3D_P4_F64, "df64"), (W.CFG_3D_P4, "fp32"),
                                     (W.CFG_3D_P4, "bf16x3"), (W.CFG_3D_P4_F64, "df64_tc"), (W.CFG_3D_P3, "df64_tc")],
                         ids=["p3_64", "p4_96_f64", "p4_96_f32", "p4_96_f32_tc", "p4_96_f64_tc", "p3_64_tc"],
                         indirect=["arith"])
def test_full_size_surrogate_sampled_rows(iga, wl, arith):
    use(iga, wl.dtype, arith)
    prob = wl.problem
    tol = TOL64 if wl.dtype == "f64" else TOL32
    A = iga.assemble_surrogate(prob, wl.M, wl.q, dtype=wl.dtype)
    vals = A.values()                                           # device [S, N]
    rows = _sampled_rows(prob, 48, seed=1)
    got = vals[:, torch.from_numpy(rows).cuda()].double().cpu().numpy().T
    setup = oracle.surrogate_setup(prob, wl.M, wl.q)
    ref = oracle.surrogate_rows(prob, wl.M, wl.q, rows, setup)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= tol * scale
    # zero row sums at full size (Sec. 5.3): A~ 1 = 0
    ones = torch.ones(prob.N, dtype=A.torch_dtype, device="cuda")
    rs = A.apply(ones).double().abs().max().item()
    assert rs <= (1e-12 if wl.dtype == "f64" else 1e-4) * scale
    # symmetry at full size: slot s of row i equals slot S-1-s of row i + delta_s
    offs = oracle.offsets(prob.dim, prob.p)
    m = np.array(prob.m)
    mi = oracle.multi_index(np.arange(prob.N), m)
    worst = 0.0
    for s in range(prob.S // 2 + 1, prob.S, max(1, prob.S // 40)):
        mj = mi + offs[s]
        ok = np.all((mj >= 0) & (mj < m), axis=1)
        i = torch.from_numpy(np.nonzero(ok)[0]).cuda()
        j = torch.from_numpy(oracle.surrogate.flat_index(mj[ok], m)).cuda()
        d = (vals[s, i] - vals[prob.S - 1 - s, j]).abs().max().item()
        worst = max(worst, d)
    # frame rows are exact quadrature rows, symmetric only up to the rounding of the contractions
    assert worst <= tol * scale
    if arith in ("df64", "fp32"):
        # the two frame slabs normal to the slowest direction compute one half of their offsets and
        # mirror the other (A_ij = A_ji): the low slab's lower slots and the high slab's upper slots
        # equal their partners' (rows of the same slab) bit for bit
        k0, k1 = oracle.omega_box(prob.p, int(m[-1]))
        mi_t = torch.from_numpy(mi).cuda()
        m_t = torch.from_numpy(m).cuda()
        stride = torch.from_numpy(np.cumprod([1] + list(m[:-1]))).cuda()
        low, high = mi_t[:, -1] < k0, mi_t[:, -1] > k1
        for s in list(range(prob.S // 2)) + list(range(prob.S // 2 + 1, prob.S)):
            mj = mi_t + torch.from_numpy(offs[s]).cuda()
            ok = ((mj >= 0) & (mj < m_t)).all(dim=1) & (low if s < prob.S // 2 else high)
            j = (mj * stride).sum(dim=1)
            assert torch.equal(vals[s][ok], vals[prob.S - 1 - s][j[ok]]), s
    A.destroy()


@pytest.mark.parametrize("wl,arith", [(W.CFG_3D_P3, "df64"), (W.CFG_3D_P4_F64, "df64"), (W.CFG_3D_P4_F64, "df64_tc")],
                         ids=["p3_64", "p4_96", "p4_96_tc"], indirect=["arith"])
def test_full_size_exact_sampled_rows(iga, wl, arith):
    use(iga, "f64", arith)
    prob = wl.problem
    A = iga.assemble_exact(prob, dtype="f64")
    vals = A.values()
    rows = _sampled_rows(prob, 32, seed=2)
    got = vals[:, torch.from_numpy(rows).cuda()].cpu().numpy().T
    ref = oracle.exact_rows(prob, rows)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= TOL64 * scale
    # zero row sums and symmetry of the whole exact matrix at full size (Sec. 3.4, Sec. 5.3)
    ones = torch.ones(prob.N, dtype=torch.float64, device="cuda")
    assert A.apply(ones).abs().max().item() <= TOL64 * scale
    offs = oracle.offsets(prob.dim, prob.p)
    m = np.array(prob.m)
    mi = oracle.multi_index(np.arange(prob.N), m)
    worst = 0.0
    for s in range(prob.S // 2 + 1, prob.S, max(1, prob.S // 40)):
        mj = mi + offs[s]
        ok = np.all((mj >= 0) & (mj < m), axis=1)
        i = torch.from_numpy(np.nonzero(ok)[0]).cuda()
        j = torch.from_numpy(oracle.surrogate.flat_index(mj[ok], m)).cuda()
        worst = max(worst, (vals[s, i] - vals[prob.S - 1 - s, j]).abs().max().item())
    assert worst <= TOL64 * scale
    if arith != "df64_tc":
        # the stages compute the upper offsets only and the lower half is their mirror (A_ij = A_ji):
        # every lower slot equals its partner bit for bit, and is 0 where the partner is outside
        mi_t = torch.from_numpy(mi).cuda()
        m_t = torch.from_numpy(m).cuda()
        stride = torch.from_numpy(np.cumprod([1] + list(m[:-1]))).cuda()
        for s in range(prob.S // 2):
            mj = mi_t + torch.from_numpy(offs[s]).cuda()
            ok = ((mj >= 0) & (mj < m_t)).all(dim=1)
            j = (mj * stride).sum(dim=1)
            assert torch.equal(vals[s][ok], vals[prob.S - 1 - s][j[ok]]), s
            assert bool((vals[s][~ok] == 0).all()), s
    A.destroy()


def test_dfmath_against_cuda_fp64(iga):
    """Double-float Taylor-series sin / cos / exp of the coefficient kernel vs CUDA's FP64 functions."""
    import ctypes
    L = iga.load()
    err = (ctypes.c_double * 3)()
    L.iga_selftest_dfmath.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    assert L.iga_selftest_dfmath(100001, err) == 0
    assert err[0] < 1e-14 and err[1] < 1e-14, list(err)
    assert err[2] < 5e-14, list(err)


@pytest.mark.parametrize("arith", ["df64"], indirect=True)
def test_double_float_coefficients_match_fp64_path(iga, arith):
    """The double-float coefficient path agrees with the FP64 one on the benchmark map family."""
    prob = W.Problem(dim=3, p=3, n_el=(12, 13, 11), map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d",
                     kappa_b=0.5)
    iga.set_arithmetic("f64", "fp64")
    ref = gpu_exact(iga, prob)
    iga.set_arithmetic("f64", "df64")
    got = gpu_exact(iga, prob)
    assert rel(got, ref) <= 1e-12
    assert rel(got, oracle.exact_matrix(prob)) <= TOL64


@pytest.mark.parametrize("kind", ["exact", "surrogate"])
def test_cg_matches_oracle(iga, kind):
    """GPU CG on the Dirichlet-reduced system vs the oracle's CG (same matrix values)."""
    wl = W.CFG_2D_P2
    prob = wl.problem
    A = iga.assemble_exact(prob) if kind == "exact" else iga.assemble_surrogate(prob, wl.M, wl.q)
    vals = A.values_host()
    f = W.rhs_vector(prob.N)
    u, it, rel_res = A.cg(torch.from_numpy(f).cuda(), tol=1e-12)
    A.destroy()
    uref, _, _ = oracle.cg(vals, prob, f, tol=1e-13)
    u = u.cpu().numpy()
    assert rel_res <= 1e-12 and it > 10
    assert np.abs(u - uref).max() <= 1e-9 * np.abs(uref).max()
    assert np.all(u[np.setdiff1d(np.arange(prob.N), oracle.interior_dofs(prob))] == 0.0)


def test_cg_fp32_iterative_refinement(iga):
    """FP32 matrix: FP64-residual refinement reaches an FP64-level residual on the stored system."""
    prob = W.Problem(dim=3, p=2, n_el=(14, 12, 13), map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d",
                     kappa_b=0.5)
    A = iga.assemble_surrogate(prob, 3, 3, dtype="f32")
    v32 = A.values_host()
    f = W.rhs_vector(prob.N, seed=2)
    u, it, rel_res = A.cg(torch.from_numpy(f).cuda(), tol=1e-11)
    A.destroy()
    assert rel_res <= 1e-11
    uref, _, _ = oracle.cg(v32.astype(np.float64), prob, f, tol=1e-13)
    assert np.abs(u.cpu().numpy() - uref).max() <= 1e-8 * np.abs(uref).max()


EDGE = [
    # minimum mesh: n_el = p + 1 (m = 2p + 1), Omega~ empty -> every row exact
    (W.Problem(dim=2, p=3, n_el=(4, 4), map_kind="sinprod", map_amp=0.05, kappa_kind="sin2d", kappa_a=1.0,
               kappa_b=0.5), 2, 3),
    (W.Problem(dim=3, p=2, n_el=(3, 3, 3), map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d", kappa_b=0.5), 2, 3),
    # Omega~ a single index per direction (L = 1): one sample, degree lowered to 0
    (W.Problem(dim=2, p=2, n_el=(7, 7), map_kind="sinprod", map_amp=0.05, kappa_kind="sin2d", kappa_a=1.0,
               kappa_b=0.5), 4, 3),
    # strongly anisotropic meshes
    (W.Problem(dim=3, p=2, n_el=(30, 7, 9), map_kind="sinprod", map_amp=0.03, kappa_kind="expsin3d", kappa_b=0.5), 5, 2),
    (W.Problem(dim=2, p=4, n_el=(120, 17), map_kind="sinprod", map_amp=0.05, kappa_kind="sin2d", kappa_a=1.0,
               kappa_b=0.5), 7, 5),
    # constant and polynomial coefficients on affine geometry
    (W.Problem(dim=3, p=3, n_el=(15, 14, 13), map_kind="affine",
               affine=(1.2, 0.1, 0.0, -0.1, 0.9, 0.2, 0.05, 0.0, 1.1, 0.0, 0.0, 0.0), kappa_kind="poly", kappa_deg=1,
               kappa_poly=tuple([1.0, 0.3, 0.2, 0.1, 0.25, 0.0, 0.05, 0.1])), 3, 1),
]


@pytest.mark.parametrize("prob,M,q", EDGE, ids=lambda x: f"{x.dim}d_p{x.p}_{'x'.join(map(str, x.n_el))}"
                         if hasattr(x, "dim") else str(x))
def test_surrogate_edge_cases(iga, prob, M, q):
    ref = oracle.surrogate_matrix(prob, M, q)
    got = gpu_surr(iga, prob, M, q)
    assert rel(got, ref) <= TOL64
    ex = gpu_exact(iga, prob)
    assert rel(ex, oracle.exact_matrix(prob)) <= TOL64
