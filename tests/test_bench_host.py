"""Host-side logic of bench.py (no GPU): the max-over-ranks timing and whole-job
aggregation across 2 gloo ranks, the closed-form FMA model of the quadrature
stages against brute-force loop counting, and the oracle reference arm."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

import iga_workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from oracle import per_offset as po  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank))
    dist = bench.init_dist(world, "gloo")
    t = bench.max_over_ranks(dist, 1.0 + rank, torch.device("cpu"))
    bench.barrier(dist)
    q.put((rank, t, bench.aggregate_value(100.0, world, t)))
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.0, 2.0]          # max over ranks
    assert [o[2] for o in out] == [100.0, 100.0]      # 100 units x 2 ranks / 2 s


def _needed(prefix, sym):
    """Whether the partial sum of the offset components `prefix` (slowest direction first) is needed
    by some offset the box computes: sym +1 keeps the offsets at or after the centre in colexicographic
    slot order (first non-zero component from the slowest direction positive), -1 those at or before."""
    if sym == 0:
        return True
    for d in prefix:
        if d != 0:
            return (d > 0) == (sym > 0)
    return True


def _brute_stage_fmas(prob, M, surrogate, domains="common", symmetric=True):
    """Count the multiply-adds the three stage loops need literally (tiny problems)."""
    p, dim = prob.p, prob.dim
    Q, Wd = p + 1, 2 * p + 1
    boxes, ns = bench._boxes(prob, M, surrogate, domains)
    # symmetric stiffness: exact (or no Omega~) over the whole patch, else the two slabs normal to
    # the slowest direction, the low one upper offsets and the high one lower
    syms = [0] * len(boxes)
    if symmetric:
        if not ns:
            syms[0] = 1
        else:
            syms[0], syms[1] = 1, -1
    if ns:
        if domains == "per_offset":
            samples = [po.union_samples(p, prob.m[d], M) for d in range(dim)]
        else:
            k0 = 2 * p
            samples = []
            for d in range(dim):
                k1 = prob.m[d] - 2 * p - 1
                s = list(range(k0, k1 + 1, M))
                if s[-1] != k1:
                    s.append(k1)
                samples.append(s)
        import itertools
        for c in itertools.product(*samples):
            boxes = boxes + [[(ci, 1) for ci in c]]
            syms = syms + [0]
    tot = {"stage_z": 0, "stage_y": 0, "stage_x": 0}
    for bx, sym in zip(boxes, syms):
        G = []
        for d in range(dim):
            lo, R = bx[d]
            elo, ehi = max(0, lo - p), min(prob.n_el[d] - 1, lo + R - 1)
            G.append((ehi - elo + 1) * Q)

        def per_row(i, d, keep):
            n = 0
            for t in range(Q * Q):
                e = i - p + t // Q
                if not (0 <= e < prob.n_el[d]):
                    continue
                for dd in range(Wd):
                    dl = dd - p
                    if max(0, dl) <= t // Q <= p + min(0, dl) and keep(dl):
                        n += 1
            return n
        rows = [range(bx[d][0], bx[d][0] + bx[d][1]) for d in range(dim)]
        offs = range(-p, p + 1)
        if dim == 3:
            tot["stage_z"] += 8 * sum(per_row(i, 2, lambda d2: _needed((d2,), sym)) for i in rows[2]) * G[1] * G[0]
            for _ in rows[2]:
                for d2 in offs:
                    tot["stage_y"] += 9 * sum(per_row(i, 1, lambda d1: _needed((d2, d1), sym))
                                              for i in rows[1]) * G[0]
                    for _ in rows[1]:
                        for d1 in offs:
                            if _needed((d2, d1), sym):
                                tot["stage_x"] += 4 * sum(per_row(i, 0, lambda d0: _needed((d2, d1, d0), sym))
                                                          for i in rows[0])
        else:
            tot["stage_y"] += 4 * sum(per_row(i, 1, lambda d1: _needed((d1,), sym)) for i in rows[1]) * G[0]
            for _ in rows[1]:
                for d1 in offs:
                    if _needed((d1,), sym):
                        tot["stage_x"] += 4 * sum(per_row(i, 0, lambda d0: _needed((d1, d0), sym)) for i in rows[0])
    return tot


@pytest.mark.parametrize("prob,M,surr,domains", [
    (W.Problem(dim=3, p=2, n_el=(13, 12, 14)), 3, True, "common"),
    (W.Problem(dim=3, p=3, n_el=(9, 8, 10)), 2, False, "common"),
    (W.Problem(dim=2, p=2, n_el=(20, 23)), 4, True, "common"),
    (W.Problem(dim=3, p=2, n_el=(13, 12, 14)), 3, True, "per_offset"),
    (W.Problem(dim=2, p=3, n_el=(25, 22)), 4, True, "per_offset"),
    (W.Problem(dim=2, p=2, n_el=(7, 9)), 2, False, "common"),
    (W.Problem(dim=3, p=2, n_el=(5, 4, 6)), 2, True, "common"),      # no Omega~: the whole patch
])
@pytest.mark.parametrize("symmetric", [True, False])
def test_stage_fma_model_matches_loop_count(prob, M, surr, domains, symmetric):
    got = bench.stage_fmas(prob, M, surr, domains, symmetric)
    ref = _brute_stage_fmas(prob, M, surr, domains, symmetric)
    assert got == ref


def test_symmetric_boxes_need_about_half_the_offsets():
    # the exact 3-D patch needs (S + 1) / 2 of the S offsets in stage X, up to the boundary rows
    prob = W.Problem(dim=3, p=2, n_el=(9, 8, 10))
    full = bench.stage_fmas(prob, 2, False, symmetric=False)
    half = bench.stage_fmas(prob, 2, False, symmetric=True)
    S = 5 ** 3
    assert half["stage_x"] < full["stage_x"] * ((S + 1) / (2 * S) + 0.05)
    assert half["stage_x"] > full["stage_x"] * ((S + 1) / (2 * S) - 0.05)


def test_kernel_work_counts_every_offset_with_the_tensor_core_stage():
    # the tensor-core stage X writes every offset of its rows, so the assembly uses no symmetric
    # boxes and stages Z and Y count every offset, in the arithmetic they run in; the CUDA-core
    # modes count the needed half
    wl = W.CFG_3D_P4_F64
    prob = W.Problem(dim=3, p=2, n_el=(13, 12, 14))
    full = bench.stage_fmas(prob, wl.M, True, symmetric=False)
    half = bench.stage_fmas(prob, wl.M, True, symmetric=True)
    for arith, want in (("df64_tc", full), ("bf16x3", full), ("df64", half), ("fp64", half), ("fp32", half)):
        work = bench.kernel_work(prob, wl, arith, surrogate=True)
        per_mac = bench.DF64_FLOPS_PER_MAC if arith in ("df64", "df64_tc") else 2.0
        for k in ("stage_z", "stage_y"):
            assert work[k]["flops"] == per_mac * want[k], (arith, k)
        # stage X: on the tensor cores no FP32-pipe figure, else the CUDA-core count
        if arith in ("df64_tc", "bf16x3"):
            assert "stage_x" not in work
        else:
            assert work["stage_x"]["flops"] == per_mac * want["stage_x"]


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--workload", W.CFG_2D_P2.name, "--ref-rows", "64"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "nnz/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["config"]["workload"] == W.CFG_2D_P2.name


def test_batch_workload_recipe():
    items = W.batch_items()
    assert len(items) == 256
    d2 = [p for p, M, q in items if p.dim == 2]
    d3 = [p for p, M, q in items if p.dim == 3]
    assert len(d2) == 192 and len(d3) == 64
    assert all(2 <= p.p <= 5 and all(16 <= n <= 256 for n in p.n_el) for p in d2)
    assert all(2 <= p.p <= 4 and all(8 <= n <= 48 for n in p.n_el) for p in d3)
    assert all(0.0 <= p.map_amp <= 0.05 for p in d2 + d3)
    assert {M for _, M, _ in items} == {4, 8} and {q for _, _, q in items} == {3}
    again = W.batch_items()
    assert again == items
