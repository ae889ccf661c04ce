"""The pass schedule on the CPU (qaoa_plan_describe, host only): the passes
apply every layer's cost and every group's mixer once (Eq. qaoa_state), each
reverse pass reads the form of (psi, lambda) the pass before it wrote, the
stored states are the inputs of the last mixer-only passes, and every
gradient term is collected once per mixer and cost layer."""
import math

import pytest

from paper_2606_26297_b300 import qaoa as q

CASES = [(13, 2, 10), (20, 3, 6), (24, 2, 10), (26, 4, 9), (30, 8, 10), (32, 6, 10), (33, 3, 8), (17, 5, 4)]


def _group(ps):
    return (ps["group_type"], ps["loA"], ps["loB"], ps["mask"])


def _split(plan):
    fwd = [ps for ps in plan if ps["kind"] in (0, 1)]
    rev = [ps for ps in plan if ps["kind"] in (2, 3)]
    return fwd, rev


@pytest.mark.parametrize("n,p,maxq", CASES)
def test_forward_passes_cover_every_layer(n, p, maxq):
    G = math.ceil(n / maxq)
    plan, _, _ = q.qaoa_plan_describe(n, p, grad=False, max_fused_qubits=maxq)
    assert all(ps["kind"] == 0 for ps in plan)
    assert len(plan) == 1 + p * (G - 1)
    groups = {_group(ps) for ps in plan}
    assert len(groups) == G
    # the mixed bits of the groups add up to n qubits
    assert sum(bin(g[3]).count("1") for g in groups) == n
    for l in range(p):
        assert sum(ps["cost_layer"] == l for ps in plan) == 1
        for g in groups:
            mixes = sum((ps["pre_layer"] == l) + (ps["post_layer"] == l) for ps in plan if _group(ps) == g)
            assert mixes == 1, (l, g)
    # the first pass synthesises |+>: it reads nothing
    assert plan[0]["bytes_per_amp"] == 12.0


@pytest.mark.parametrize("n,p,maxq", CASES)
@pytest.mark.parametrize("stored", [0, 1, 2, -1])
def test_reverse_sweep_reads_what_the_pass_before_wrote(n, p, maxq, stored):
    G = math.ceil(n / maxq)
    plan, nslots, nmids = q.qaoa_plan_describe(n, p, grad=True, max_fused_qubits=maxq, stored_mids=stored)
    fwd, rev = _split(plan)
    assert len(fwd) == 1 + p * (G - 1) and fwd[-1]["kind"] == 1
    assert len(rev) == len(fwd) - 1
    assert nmids == p * max(G - 2, 0)
    keep = 0 if G < 3 else (nmids if stored < 0 else min(stored, nmids))
    assert sum(ps["kind"] == 3 for ps in rev) == keep
    assert nslots == keep
    # the form each pass writes is the one the next reads: lambda alone before a
    # kind-3 pass, the interleaved (psi, lambda) buffer before a kind-2 pass
    wrote = "lam" if fwd[-1]["lambda_alone_out"] else "pl"
    for ps in rev:
        reads = "lam" if ps["kind"] == 3 else "pl"
        assert reads == wrote
        if ps["kind"] == 3:
            wrote = "pl" if ps["interleaved_out"] else "lam"
        else:
            wrote = "lam" if ps["lambda_alone_out"] else "pl"
    # the kept mixer-only passes are the last ones of the forward sweep; each reads
    # its input from the slot the forward pass before it wrote
    mids = [i for i, ps in enumerate(fwd) if ps["cost_layer"] < 0 and ps["pre_layer"] < 0 and i > 0
            and ps["kind"] == 0 and ps["post_layer"] >= 0]
    kept = mids[len(mids) - keep:] if keep else []
    slots = set()
    for i in kept:
        assert fwd[i]["in_slot"] >= 0 and fwd[i - 1]["out_slot"] == fwd[i]["in_slot"]
        slots.add(fwd[i]["in_slot"])
    assert len(slots) == keep
    assert {ps["psi_slot"] for ps in rev if ps["kind"] == 3} == slots


@pytest.mark.parametrize("n,p,maxq", CASES)
@pytest.mark.parametrize("stored", [0, -1])
def test_every_gradient_term_collected_once(n, p, maxq, stored):
    """dE/dgamma_l from the one pass that undoes cost layer l; dE/dbeta_l from
    the X-terms of every group's mixer of layer l, two slots (the two register
    arrangements) per mixer; the final pass also sums E."""
    G = math.ceil(n / maxq)
    plan, _, _ = q.qaoa_plan_describe(n, p, grad=True, max_fused_qubits=maxq, stored_mids=stored)
    slots = [s for ps in plan if ps["kind"] != 0 for s in ps["slot_param"]]
    for l in range(p):
        assert slots.count(p + l) == 1, l
        assert slots.count(l) == 2 * G, l
    assert slots.count(-2) == 2


def test_bytes_per_evaluation():
    """n = 30, p = 8 with all mixer-only inputs stored moves 772 B per amplitude
    (17 forward passes: 12 + 8 x 16 + 7 x 20 + 20; 8 mixer-only reverse passes of
    32; 7 cost-layer reverse passes of 28 and the first pass's of 20); keeping
    fewer states never moves fewer bytes."""
    totals = []
    for stored in (-1, 4, 1, 0):
        plan, _, _ = q.qaoa_plan_describe(30, 8, grad=True, max_fused_qubits=10, stored_mids=stored)
        totals.append(sum(ps["bytes_per_amp"] for ps in plan))
    assert totals[0] == 772.0
    assert totals == sorted(totals)


def test_rejects_bad_arguments():
    for n, p, maxq in [(12, 2, 10), (34, 2, 10), (20, -1, 10), (20, 2, 2), (20, 2, 11)]:
        with pytest.raises(q.QaoaError):
            q.qaoa_plan_describe(n, p, grad=True, max_fused_qubits=maxq)
