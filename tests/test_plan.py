"""The GPU path's host-side sampling plan (iga_surrogate_plan, no GPU needed)
against the oracle's sampling, index for index.

Common domain (Sec. 4, Sec. 6): the sample indices of Omega~ = [2p, m-2p-1]
(every M-th index from 2p, plus the last index) and the degree lowered to the
sample count - 1.  Per-offset domains (Sec. 3.2): the union of the offsets'
samples, and per offset component the domain of Omega~_delta and its samples.
Integer work: the bar is equality.
"""
import numpy as np
import pytest

import iga_workloads as W
import oracle
from oracle import per_offset as po

CASES = [(2, 2, (32, 32), 4, 3), (3, 3, (64, 64, 64), 8, 3), (3, 4, (96, 96, 96), 8, 3), (2, 1, (5, 7), 1, 3),
         (2, 3, (9, 10), 4, 3), (2, 3, (4, 4), 4, 3), (2, 3, (5, 6), 2, 3), (3, 2, (30, 7, 9), 5, 2),
         (2, 5, (40, 33), 6, 7), (2, 2, (20, 23), 40, 3), (3, 2, (3, 3, 3), 2, 3), (2, 4, (200, 150), 7, 5),
         (2, 1, (3, 2), 1, 0), (3, 5, (12, 11, 13), 3, 7)]


@pytest.fixture(scope="module")
def iga():
    import paper_1904_06971_gb300 as m
    m.load()
    return m


def _id(c):
    return f"{c[0]}d_p{c[1]}_{'x'.join(map(str, c[2]))}_M{c[3]}_q{c[4]}"


@pytest.mark.parametrize("case", CASES, ids=_id)
def test_common_domain_plan(iga, case):
    dim, p, n_el, M, q = case
    prob = W.Problem(dim=dim, p=p, n_el=n_el)
    plan = iga.surrogate_plan(prob, M, q, "common")
    boxes = [oracle.omega_box(p, md) for md in prob.m]
    if any(k1 < k0 for k0, k1 in boxes):
        assert plan["empty"]
        return
    assert not plan["empty"]
    for d, (k0, k1) in enumerate(boxes):
        ref = oracle.sample_indices(k0, k1, M)
        assert list(plan["samples"][d]) == ref
        for v in range(2 * p + 1):
            assert plan["domains"][d][v] == (k0, k1, len(ref), min(q, len(ref) - 1))


@pytest.mark.parametrize("case", CASES, ids=_id)
def test_per_offset_plan(iga, case):
    dim, p, n_el, M, q = case
    prob = W.Problem(dim=dim, p=p, n_el=n_el)
    plan = iga.surrogate_plan(prob, M, q, "per_offset")
    cards = [po.cardinal_range(p, md) for md in prob.m]
    if any(c1 < c0 for c0, c1 in cards):
        assert plan["empty"]
        return
    assert not plan["empty"]
    for d, md in enumerate(prob.m):
        assert list(plan["samples"][d]) == po.union_samples(p, md, M)
        for v in range(2 * p + 1):
            dd = v - p
            lo, hi = po.offset_domain(p, md, dd)
            own = po.offset_samples(p, md, M, dd)
            got = plan["domains"][d][v]
            if hi < lo:                                              # no index pair: the plan reports hi = lo - 1
                assert got[:3] == (lo, lo - 1, 0), (d, dd)
                continue
            assert got[:3] == (lo, hi, len(own)), (d, dd)
            if own:
                assert got[3] == min(q, len(own) - 1)
                assert set(own) <= set(plan["samples"][d])       # every offset's samples are sample rows


def test_plan_rejects_what_the_assembly_rejects(iga):
    prob = W.Problem(dim=2, p=2, n_el=(10, 10))
    for M, q, dom in ((0, 3, "common"), (4, 8, "common"), (4, -1, "per_offset")):
        with pytest.raises(iga.IgaError):
            iga.surrogate_plan(prob, M, q, dom)
    with pytest.raises(iga.IgaError):
        iga.surrogate_plan(W.Problem(dim=2, p=2, n_el=(1, 10)), 4, 3)        # n_el < p + 1
