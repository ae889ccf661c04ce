"""Oracle for the graph-aware allocation and the allocation candidates of
Sec. 3.1.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
it; the product never imports it and it never imports the product.

Sec. 3.1 builds a weighted adjacency from the quadratic coefficients, places
strongly coupled variables on the same QPU without exceeding a capacity,
forms candidate allocations (contiguous, graph-aware, and the user's manual
one), and keeps the candidate with the fewest cross-QPU couplings, ties broken
by a fixed order of the allocation types.

Readings (the paper names the steps, not their rules):

* Edge weight w_ij = |b_ij|, the magnitude of the canonical coupling.
* Greedy growth: QPUs are filled in order 0 .. M-1.  QPU m opens with the
  unassigned variable of largest weighted degree towards the unassigned
  variables, then repeatedly takes the unassigned variable with the largest
  total weight to the QPU's members (ties: larger weighted degree towards the
  unassigned variables, then smaller index) until it holds
  min(c_m, unassigned - (QPUs still to open)) variables, so that every QPU
  receives at least one variable.
* Candidate priority on equal cross counts: manual, then graph-aware, then
  contiguous.
"""
from __future__ import annotations

import numpy as np


def weights(cq) -> np.ndarray:
    """Symmetric weighted adjacency |b_ij| (zero diagonal)."""
    W = np.abs(np.asarray(cq.b, dtype=np.float64))
    W = np.triu(W, 1)
    return W + W.T


def graph_aware(cq, caps: list[int]) -> list[int]:
    """Greedy graph-aware assignment qpu_of[i] for the capacities caps."""
    n = cq.n
    W = weights(cq)
    M = len(caps)
    qpu = [-1] * n
    free = set(range(n))
    for m in range(M):
        if not free:
            break
        take = min(caps[m], len(free) - (M - m - 1))
        if take <= 0:
            continue
        deg = {v: sum(W[v, u] for u in free if u != v) for v in free}
        seed = min(free, key=lambda v: (-deg[v], v))
        members = [seed]
        free.discard(seed)
        while len(members) < take and free:
            deg = {v: sum(W[v, u] for u in free if u != v) for v in free}
            best = min(free, key=lambda v: (-sum(W[v, u] for u in members), -deg[v], v))
            members.append(best)
            free.discard(best)
        for v in members:
            qpu[v] = m
    return qpu


def cross_count(cq, qpu_of) -> int:
    """Couplings b_ij != 0 (i < j) whose variables sit on different QPUs."""
    n = cq.n
    return sum(1 for i in range(n) for j in range(i + 1, n) if cq.b[i][j] != 0 and qpu_of[i] != qpu_of[j])


def candidates(cq, caps: list[int], manual=None):
    """(kind, qpu_of, cross) for contiguous (0), graph-aware (1) and manual (2)
    candidates, and the index of the selected one."""
    import oracle

    out = [(0, oracle.contiguous_allocation(cq.n, caps)), (1, graph_aware(cq, caps))]
    if manual is not None:
        out.append((2, list(manual)))
    scored = [(kind, q, cross_count(cq, q)) for kind, q in out]
    prio = {2: 0, 1: 1, 0: 2}
    best = min(range(len(scored)), key=lambda k: (scored[k][2], prio[scored[k][0]]))
    return scored, best
