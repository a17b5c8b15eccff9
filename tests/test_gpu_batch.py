"""GPU batched assembly (iga_assemble_batch): the graph replays give the same
matrices, bit for bit, as assembling every patch alone (the kernels are
deterministic and see the same inputs), and those match the FP64 oracle."""
from dataclasses import replace

import numpy as np
import pytest

import iga_workloads as W
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def iga():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1904_06971_gb300 as m
    m.load()
    return m


def _sp2(n_el, p, amp=0.05, b=0.5):
    return W.Problem(dim=2, p=p, n_el=n_el, map_kind="sinprod", map_amp=amp, kappa_kind="sin2d", kappa_a=1.0, kappa_b=b)


def _sp3(n_el, p, amp=0.03, b=0.5):
    return W.Problem(dim=3, p=p, n_el=n_el, map_kind="sinprod", map_amp=amp, kappa_kind="expsin3d", kappa_b=b)


ITEMS = [
    (_sp2((20, 23), 2), 3, 3),
    (_sp2((30, 26), 3), 4, 4),
    (_sp2((40, 33), 5, b=0.2), 6, 3),
    (_sp2((9, 10), 3), 4, 3),                       # empty Omega~
    (_sp2((17, 19), 2), 0, 3),                      # exact
    (_sp3((13, 12, 14), 2), 3, 3),
    (_sp3((17, 15, 16), 3, b=0.3), 2, 3),
    (_sp3((11, 9, 10), 2), 0, 3),                   # exact
    (_sp3((14, 13, 12), 2), 3, 3, "per_offset"),
]


def _alone(iga, it, dtype):
    prob, M, q = it[:3]
    dom = it[3] if len(it) > 3 else "common"
    A = iga.assemble_surrogate(prob, M, q, dtype=dtype, domains=dom) if M else iga.assemble_exact(prob, dtype=dtype)
    v = A.values_host()
    A.destroy()
    return v


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batch_graph_matches_single_patch_assembly(iga, dtype):
    ref = [_alone(iga, it, dtype) for it in ITEMS]
    mats = iga.assemble_batch(ITEMS, dtype=dtype)                     # eager, creates the matrices
    for A, r in zip(mats, ref):
        assert np.array_equal(A.values_host(), r)
    # overwrite two matrices through single-patch calls with another coefficient
    for k in (1, 6):
        prob, M, q = ITEMS[k][:3]
        iga.assemble_surrogate(replace(prob, kappa_b=0.1), M, q, dtype=dtype, out=mats[k])
    l0 = iga.launch_count()
    iga.assemble_batch(ITEMS, dtype=dtype, out=mats)                  # capture + autotune
    branches, kernels, cached, tuned_ms = iga.batch_info()
    assert not cached and branches >= 1 and kernels > 0 and tuned_ms > 0
    torch.cuda.synchronize()
    for A, r in zip(mats, ref):
        assert np.array_equal(A.values_host(), r)
    l1 = iga.launch_count()
    iga.assemble_batch(ITEMS, dtype=dtype, out=mats)                  # cached graph
    b2, k2, cached2, _ = iga.batch_info()
    assert cached2 and b2 == branches and k2 == kernels
    assert iga.launch_count() - l1 == kernels
    assert l1 - l0 >= 3 * kernels
    torch.cuda.synchronize()
    for A, r in zip(mats, ref):
        assert np.array_equal(A.values_host(), r)
    for A in mats:
        A.destroy()


def test_batch_against_oracle(iga):
    items = ITEMS[:2] + ITEMS[5:6]
    mats = iga.assemble_batch(items, dtype="f64")
    mats = iga.assemble_batch(items, dtype="f64", out=mats)
    torch.cuda.synchronize()
    for (prob, M, q), A in zip(items, mats):
        ref = oracle.surrogate_matrix(prob, M, q)
        assert oracle.relative_entry_error(A.values_host(), ref) <= 1e-12
        A.destroy()


def test_batch_workload_slice(iga):
    """The first patches of the 256-patch workload (FP32) through eager and graph paths."""
    items = W.batch_items(6, 2, seed=0)
    mats = iga.assemble_batch(items, dtype="f32")
    first = [A.values_host() for A in mats]
    iga.assemble_batch(items, dtype="f32", out=mats)
    torch.cuda.synchronize()
    for A, v in zip(mats, first):
        assert np.array_equal(A.values_host(), v)
        ones = torch.ones(A.N, dtype=torch.float32, device="cuda")
        assert A.apply(ones).abs().max().item() <= 1e-4 * np.abs(v).max()
        A.destroy()


def test_batch_rejects_bad_arguments(iga):
    with pytest.raises(iga.IgaError):
        iga.assemble_batch([], dtype="f32")


@pytest.fixture
def modes(iga):
    yield
    iga.batch_set_modes(True, True)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_batch_persistent_matches_single_patch_assembly(iga, dtype, modes):
    """Persistent quadrature kernel (one launch per dimension/degree/arithmetic over device-side
    patch descriptors): bit-identical to assembling each patch alone, on tuning and cached replays."""
    ref = [_alone(iga, it, dtype) for it in ITEMS]
    iga.batch_set_modes(branches=False, persistent=True)
    mats = iga.assemble_batch(ITEMS, dtype=dtype)
    for k in (0, 5):                                   # stale contents the batch must overwrite
        prob, M, q = ITEMS[k][:3]
        iga.assemble_surrogate(replace(prob, kappa_b=0.1), M, q, dtype=dtype, out=mats[k])
    iga.assemble_batch(ITEMS, dtype=dtype, out=mats)
    persistent, bps, chunk = iga.batch_mode()
    assert persistent and bps >= 1 and chunk >= 1
    iga.batch_status()
    for A, r in zip(mats, ref):
        assert np.array_equal(A.values_host(), r)
    iga.assemble_batch(ITEMS, dtype=dtype, out=mats)   # cached replay
    _, _, cached, _ = iga.batch_info()
    assert cached
    iga.batch_status()
    for A, r in zip(mats, ref):
        assert np.array_equal(A.values_host(), r)
    for A in mats:
        A.destroy()


def test_batch_persistent_workload_slice_against_oracle(iga, modes):
    """A slice of the 256-patch workload (uneven sizes and degrees, FP64 values) through the persistent
    kernel against the FP64 oracle."""
    iga.batch_set_modes(branches=False, persistent=True)
    items = [it for it in W.batch_items(8, 3, seed=3) if it[0].N <= 6000]
    items += [it for it in W.batch_items(0, 8, seed=3) if it[0].N <= 4000]
    assert len(items) == 6 and {it[0].dim for it in items} == {2, 3}
    mats = iga.assemble_batch(items, dtype="f64")
    iga.assemble_batch(items, dtype="f64", out=mats)
    assert iga.batch_mode()[0]
    iga.batch_status()
    for (prob, M, q), A in zip([it[:3] for it in items], mats):
        ref = oracle.surrogate_matrix(prob, M, q) if M else oracle.exact_matrix(prob)
        assert oracle.relative_entry_error(A.values_host(), ref) <= 1e-12
        A.destroy()


def test_persistent_wait_gives_up_with_status(iga):
    """The persistent kernel's dependency wait on a counter nothing increments returns
    IGA_ETIMEOUT after its limit (no hang, no fault), and the device stays usable."""
    import time
    t0 = time.time()
    rc = iga.batch_selftest_timeout(20000)
    assert rc == -5, iga.load().iga_last_error().decode()
    assert time.time() - t0 < 30
    prob = W.CFG_2D_P2.problem
    A = iga.assemble_exact(prob, dtype="f64")
    assert oracle.relative_entry_error(A.values_host(), oracle.exact_matrix(prob)) <= 1e-12
    A.destroy()
