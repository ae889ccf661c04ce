"""Pins for the graph-aware allocation oracle (oracle/allocation.py) and the
library's host-only allocation entry points against it.  CPU only."""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import allocation as oal
from paper_2606_26297_b300 import build_lib, instances as inst

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _figure(intra=2.0, inter=1.0):
    gold = json.load(open(os.path.join(GOLDEN, "allocation_figure.json")))
    n = 6
    H = np.zeros((n, n))
    clusters = [set(vs) for vs in gold["allocations"]["graph_aware"]["qpus"]]
    for u, v in gold["panel_a_edges"]:
        same = any(u in c and v in c for c in clusters)
        H[u - 1, v - 1] = intra if same else inter
    return gold, H


def test_figure_graph_aware_recovers_panel_c():
    """Fig. allocation_strategies: with the intra-cluster edges stronger than
    the inter-cluster ones (as panel (a) draws them), the greedy places
    {1, 4, 5} and {2, 3, 6} together (panel (c)), 2 cross terms, and the
    candidate selection prefers it to contiguous (5) and manual (4)."""
    gold, H = _figure()
    cq = oracle.canonicalize(H, None, 0.0)
    q = oal.graph_aware(cq, [3, 3])
    groups = sorted(sorted(i + 1 for i in range(6) if q[i] == m) for m in range(2))
    assert groups == sorted(sorted(g) for g in gold["allocations"]["graph_aware"]["qpus"])
    manual = [0] * 6
    for m, vs in enumerate(gold["allocations"]["manual"]["qpus"]):
        for v in vs:
            manual[v - 1] = m
    scored, best = oal.candidates(cq, [3, 3], manual)
    assert [s[2] for s in scored] == [5, 2, 4]
    assert scored[best][0] == 1


def test_equal_blocks_recovered_under_permutation():
    """A direct sum of M dense blocks of k variables (non-zero couplings),
    with the variables permuted, and capacities k each: every QPU receives
    exactly one block, so no coupling crosses a QPU."""
    rng = np.random.default_rng(4)
    for M, k in [(3, 4), (2, 5), (4, 3)]:
        n = M * k
        perm = rng.permutation(n)
        H = np.zeros((n, n))
        for blk in range(M):
            vs = perm[blk * k:(blk + 1) * k]
            for a in range(k):
                for b in range(a + 1, k):
                    H[vs[a], vs[b]] = rng.uniform(0.5, 2.0) * rng.choice([-1, 1])
        cq = oracle.canonicalize(H, None, 0.0)
        q = oal.graph_aware(cq, [k] * M)
        assert oal.cross_count(cq, q) == 0
        assert oracle.validate_allocation(q, [k] * M)


def test_uncoupled_equals_contiguous_and_invariants():
    """No couplings: every tie falls to the smaller index, which is the
    contiguous allocation.  Random instances: capacities hold and every QPU
    is used."""
    cq = oracle.canonicalize(np.diag(np.arange(7.0)), None, 0.0)
    assert oal.graph_aware(cq, [3, 2, 2]) == oracle.contiguous_allocation(7, [3, 2, 2])
    rng = np.random.default_rng(9)
    for t in range(20):
        n = int(rng.integers(3, 12))
        M = int(rng.integers(2, min(n, 4) + 1))
        caps = [int(c) for c in rng.integers(1, n, size=M)]
        if sum(caps) < n:
            caps[0] += n - sum(caps)
        Q = inst.upper_int_qubo(n, 700 + t)
        cq = oracle.canonical_of(Q)
        q = oal.graph_aware(cq, caps)
        assert oracle.validate_allocation(q, caps), (caps, q)


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    from paper_2606_26297_b300 import qaoa
    return qaoa


def test_library_graph_aware_and_candidates_match_oracle(lib):
    """qaoa_partition_graph and qaoa_allocation_candidates (host only) against
    the oracle on the figure and on random integer QUBOs."""
    gold, H = _figure()
    got = lib.qaoa_partition_graph(H, None, 0.0, [3, 3])
    assert list(got) == oal.graph_aware(oracle.canonicalize(H, None, 0.0), [3, 3])
    rng = np.random.default_rng(12)
    for t in range(12):
        n = int(rng.integers(4, 14))
        M = int(rng.integers(2, 4))
        caps = [n // M + (1 if m < n % M else 0) for m in range(M)]
        Q = inst.upper_int_qubo(n, 900 + t)
        cq = oracle.canonical_of(Q)
        assert list(lib.qaoa_partition_graph(Q.H, Q.f, Q.c0, caps)) == oal.graph_aware(cq, caps)
        manual = [int(v) for v in rng.permutation(oracle.contiguous_allocation(n, caps))]
        res = lib.qaoa_allocation_candidates(Q.H, Q.f, Q.c0, caps, manual, p=3)
        scored, best = oal.candidates(cq, caps, manual)
        assert res["cross"] == [s[2] for s in scored]
        assert res["remote_cx"] == [2 * 3 * s[2] for s in scored]
        assert res["kind"] == scored[best][0]
        assert list(res["qpu_of"]) == list(scored[best][1])
