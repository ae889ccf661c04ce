"""GPU parity of the batched forms: many parameter sets and ragged QUBO sizes
in one request (qaoa_grad_batch), and the Adam loop on the exact gradient
replayed as a CUDA graph (qaoa_optimize_adam), against the FP64 oracle.

Tolerances as in test_gpu_parity: |dE| / max|F| <= 1e-5, gradient
max-abs error / max|gradient| <= 1e-4.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_26297_b300 import instances as inst

pytestmark = pytest.mark.gpu

E_TOL = 1e-5
G_TOL = 1e-4


@pytest.fixture(scope="module")
def q():
    from paper_2606_26297_b300 import build_lib
    build_lib.build()
    from paper_2606_26297_b300 import qaoa
    return qaoa


@pytest.fixture(scope="module")
def ctx(q):
    c = q.qaoa_ctx_create(0)
    yield c
    q.qaoa_ctx_destroy(c)


def _cost(q, ctx, Q):
    return q.qaoa_build_cost(ctx, Q.H, Q.f, Q.c0, "i32" if Q.dtype == "i32" else "f32")


def _check_item(F, g, b, E, dg, db):
    Eo, dgo, dbo = oracle.grad_adjoint(F, g, b)
    assert abs(E - Eo) / np.max(np.abs(F)) <= E_TOL
    sc = max(np.max(np.abs(dgo)), np.max(np.abs(dbo)), 1e-12)
    err = max(np.max(np.abs(dg - dgo)), np.max(np.abs(db - dbo))) / sc
    assert err <= G_TOL, err


def test_multistart_batch_vs_oracle_and_single(q, ctx):
    """Many (gamma, beta) sets on one n=16 table: every item against the oracle
    and against the single-item call."""
    n, p, B = 16, 3, 6
    Q = inst.upper_int_qubo(n, 4100)
    g, b = inst.random_angles(p, B, 4101, gamma_scale=1.0 / math.sqrt(n))
    cost = _cost(q, ctx, Q)
    E, dg, db = q.qaoa_grad_batch(ctx, [cost], g, b)
    F = oracle.cost_table(oracle.canonical_of(Q))
    for i in range(B):
        _check_item(F, g[i], b[i], E[i], dg[i], db[i])
        Es, dgs, dbs = q.qaoa_grad(ctx, cost, g[i], b[i])
        assert abs(Es - E[i]) <= 1e-6 * np.max(np.abs(F))
        sc = max(np.abs(dgs).max(), np.abs(dbs).max())
        assert max(np.abs(dgs - dg[i]).max(), np.abs(dbs - db[i]).max()) <= 1e-5 * sc
    q.qaoa_cost_destroy(cost)


def test_ragged_batch_vs_oracle(q, ctx):
    """Uneven sizes in one request: n <= 12 items on the shared-memory kernel,
    two different tables of the same n in one launch, a real-valued table."""
    Qs = [inst.upper_int_qubo(10, 4200), inst.upper_int_qubo(13, 4201), inst.normal_qubo(15, 4202),
          inst.upper_int_qubo(15, 4203), inst.regular_maxcut_qubo(18, 4204)]
    costs = [_cost(q, ctx, Q) for Q in Qs]
    item_cost = [0, 1, 2, 3, 4, 2, 3, 0, 1]
    p = 2
    g, b = inst.random_angles(p, len(item_cost), 4205, gamma_scale=0.3)
    E, dg, db = q.qaoa_grad_batch(ctx, costs, g, b, item_cost=item_cost)
    Fs = [oracle.cost_table(oracle.canonical_of(Q)) for Q in Qs]
    for i, ci in enumerate(item_cost):
        _check_item(Fs[ci], g[i], b[i], E[i], dg[i], db[i])
    Ef = q.qaoa_grad_batch(ctx, costs, g, b, item_cost=item_cost, grad=False)
    for i, ci in enumerate(item_cost):
        Eo = oracle.expectation(Fs[ci], oracle.evolve(Fs[ci], g[i], b[i]))
        assert abs(Ef[i] - Eo) / np.max(np.abs(Fs[ci])) <= E_TOL
    for c in costs:
        q.qaoa_cost_destroy(c)


def test_batch_deterministic(q, ctx):
    Q = inst.upper_int_qubo(17, 4300)
    cost = _cost(q, ctx, Q)
    g, b = inst.random_angles(3, 4, 4301, gamma_scale=0.2)
    r1 = q.qaoa_grad_batch(ctx, [cost], g, b)
    r2 = q.qaoa_grad_batch(ctx, [cost], g, b)
    for a1, a2 in zip(r1, r2):
        assert np.array_equal(a1, a2)
    q.qaoa_cost_destroy(cost)


def _adam_reference(Fs, item_cost, g0, b0, iters, lr, b1=0.9, b2=0.999, eps=1e-8):
    """Adam (bias-corrected moments) on the oracle's exact gradient."""
    g, b = g0.copy(), b0.copy()
    B, p = g.shape
    m = np.zeros((B, 2 * p))
    v = np.zeros((B, 2 * p))
    hist = np.zeros((iters, B))
    for t in range(1, iters + 1):
        for i in range(B):
            E, dg, db = oracle.grad_adjoint(Fs[item_cost[i]], g[i], b[i])
            hist[t - 1, i] = E
            gr = np.concatenate([dg, db])
            m[i] = b1 * m[i] + (1 - b1) * gr
            v[i] = b2 * v[i] + (1 - b2) * gr * gr
            mh = m[i] / (1 - b1 ** t)
            vh = v[i] / (1 - b2 ** t)
            step = lr * mh / (np.sqrt(vh) + eps)
            g[i] -= step[:p]
            b[i] -= step[p:]
    return g, b, hist


def test_adam_graph_vs_eager_vs_oracle(q, ctx):
    Qs = [inst.upper_int_qubo(14, 4400), inst.upper_int_qubo(11, 4401), inst.regular_maxcut_qubo(14, 4402)]
    costs = [_cost(q, ctx, Q) for Q in Qs]
    item_cost = [0, 1, 2, 0]
    p, iters, lr = 2, 6, 0.02
    g0, b0 = inst.random_angles(p, len(item_cost), 4403, gamma_scale=0.2)
    gg, bg, hg, Eg = q.qaoa_optimize_adam(ctx, costs, g0, b0, iters, item_cost=item_cost, lr=lr)
    ge, be, he, Ee = q.qaoa_optimize_adam(ctx, costs, g0, b0, iters, item_cost=item_cost, lr=lr, use_graph=False)
    # the graph replays exactly the eager step's kernels
    assert np.array_equal(gg, ge) and np.array_equal(bg, be)
    assert np.array_equal(hg, he) and np.array_equal(Eg, Ee)
    # the first history entry is the batch evaluation at the starting point
    E0 = q.qaoa_grad_batch(ctx, costs, g0, b0, item_cost=item_cost)[0]
    assert np.array_equal(hg[0], E0)
    Fs = [oracle.cost_table(oracle.canonical_of(Q)) for Q in Qs]
    gr, br, hr = _adam_reference(Fs, item_cost, g0, b0, iters, lr)
    assert np.max(np.abs(gg - gr)) <= 1e-5 and np.max(np.abs(bg - br)) <= 1e-5
    for i, ci in enumerate(item_cost):
        scale = np.max(np.abs(Fs[ci]))
        assert np.max(np.abs(hg[:, i] - hr[:, i])) / scale <= E_TOL
        Ef = oracle.expectation(Fs[ci], oracle.evolve(Fs[ci], gg[i], bg[i]))
        assert abs(Eg[i] - Ef) / scale <= E_TOL
    for c in costs:
        q.qaoa_cost_destroy(c)


def test_adam_graph_several_sizes(q, ctx):
    """Groups of three different n (13, 14, 16) and a shared-memory item in one
    optimisation: the groups of a step run on forked streams that join before
    the Adam update, inside the captured graph as in the eager step.  Graph
    and eager agree bit for bit, and both follow Adam on the oracle gradient."""
    Qs = [inst.upper_int_qubo(13, 4600), inst.normal_qubo(14, 4601), inst.regular_maxcut_qubo(16, 4602),
          inst.upper_int_qubo(9, 4603)]
    costs = [_cost(q, ctx, Q) for Q in Qs]
    item_cost = [2, 0, 1, 3, 2, 1]
    p, iters, lr = 2, 5, 0.02
    g0, b0 = inst.random_angles(p, len(item_cost), 4604, gamma_scale=0.2)
    gg, bg, hg, Eg = q.qaoa_optimize_adam(ctx, costs, g0, b0, iters, item_cost=item_cost, lr=lr)
    ge, be, he, Ee = q.qaoa_optimize_adam(ctx, costs, g0, b0, iters, item_cost=item_cost, lr=lr, use_graph=False)
    assert np.array_equal(gg, ge) and np.array_equal(bg, be)
    assert np.array_equal(hg, he) and np.array_equal(Eg, Ee)
    Fs = [oracle.cost_table(oracle.canonical_of(Q)) for Q in Qs]
    gr, br, hr = _adam_reference(Fs, item_cost, g0, b0, iters, lr)
    assert np.max(np.abs(gg - gr)) <= 1e-5 and np.max(np.abs(bg - br)) <= 1e-5
    for i, ci in enumerate(item_cost):
        assert np.max(np.abs(hg[:, i] - hr[:, i])) / np.max(np.abs(Fs[ci])) <= E_TOL
    for c in costs:
        q.qaoa_cost_destroy(c)


def test_adam_decreases_objective(q, ctx):
    Q = inst.regular_maxcut_qubo(16, 4500)
    cost = _cost(q, ctx, Q)
    g0, b0 = inst.ramp_angles(3, amp=0.4)
    g, b, hist, E = q.qaoa_optimize_adam(ctx, [cost], g0[None, :], b0[None, :], 40, lr=0.03)
    assert E[0] < hist[0, 0] - 0.5
    assert hist[-1, 0] < hist[0, 0]
    q.qaoa_cost_destroy(cost)


def test_autotune_fusion_width(q, ctx):
    """The tuner times every width and keeps the fastest; a context with
    autotune on evaluates exactly as one fixed to that width, and both match
    the oracle."""
    Q = inst.upper_int_qubo(18, 4600)
    g, b = inst.ramp_angles(3, gamma_scale=0.2)
    cost = _cost(q, ctx, Q)
    best, ms = q.qaoa_autotune(ctx, cost, 2)
    assert set(ms) == {10, 9, 8, 7, 6, 5} and best in ms
    assert ms[best] == min(ms.values()) and all(v > 0 for v in ms.values())
    q.qaoa_cost_destroy(cost)
    ca = q.qaoa_ctx_create(0, autotune=True)
    ck = q.qaoa_ctx_create(0, max_fused_qubits=best)
    ka, kk = _cost(q, ca, Q), _cost(q, ck, Q)
    ra = q.qaoa_grad(ca, ka, g, b)
    rk = q.qaoa_grad(ck, kk, g, b)
    F = oracle.cost_table(oracle.canonical_of(Q))
    _check_item(F, g, b, *ra)
    # the autotuned context may pick a different width on its own timing run;
    # whichever it picked, the result equals a fixed-width run of that width
    cw = q.qaoa_ctx_create(0, max_fused_qubits=q.qaoa_autotune(ca, ka, 2)[0])
    kw = _cost(q, cw, Q)
    rw = q.qaoa_grad(cw, kw, g, b)
    ra2 = q.qaoa_grad(ca, ka, g, b)
    assert ra2[0] == rw[0] and np.array_equal(ra2[1], rw[1]) and np.array_equal(ra2[2], rw[2])
    _check_item(F, g, b, *rk)
    for c, k in ((ca, ka), (ck, kk), (cw, kw)):
        q.qaoa_cost_destroy(k)
        q.qaoa_ctx_destroy(c)


def test_autotune_adjoint_form(q, ctx):
    """At n = 24 (three qubit groups, so stored forward states apply) the tuner
    also times the two adjoint forms; a context with autotune on then
    evaluates bit for bit like a context fixed to the chosen width and form."""
    Q = inst.upper_int_qubo(24, 4650)
    g, b = inst.ramp_angles(4, gamma_scale=0.1)
    ca = q.qaoa_ctx_create(0, autotune=True)
    ka = _cost(q, ca, Q)
    best, ms, modes = q.qaoa_autotune(ca, ka, 2, with_modes=True)
    assert modes["stored"] > 0 and modes["uncompute"] > 0
    mode = q.QAOA_ADJ_UNCOMPUTE if modes["uncompute"] < modes["stored"] else q.QAOA_ADJ_AUTO
    cf = q.qaoa_ctx_create(0, max_fused_qubits=best, adjoint_mode=mode)
    kf = _cost(q, cf, Q)
    ra = q.qaoa_grad(ca, ka, g, b)
    rf = q.qaoa_grad(cf, kf, g, b)
    assert ra[0] == rf[0] and np.array_equal(ra[1], rf[1]) and np.array_equal(ra[2], rf[2])
    for c, k in ((ca, ka), (cf, kf)):
        q.qaoa_cost_destroy(k)
        q.qaoa_ctx_destroy(c)


def test_adam_resume_equals_one_run(q, ctx):
    """Checkpointed optimisation: 6 Adam iterations and then 5 more from the
    returned angles, moments and step count give the same angles and history,
    bit for bit, as 11 iterations in one call (a mixed batch: n = 10 items on
    the shared-memory path and n = 14 items on the pass path)."""
    Qa, Qb = inst.upper_int_qubo(10, 4800), inst.upper_int_qubo(14, 4801)
    ca, cb = _cost(q, ctx, Qa), _cost(q, ctx, Qb)
    g0, b0 = inst.random_angles(2, 4, 4802, gamma_scale=0.2)
    ic = [0, 1, 0, 1]
    g1, b1, h1, E1, st = q.qaoa_optimize_adam_resume(ctx, [ca, cb], g0, b0, 6, item_cost=ic, lr=0.02)
    assert st["step"] == 6 and np.any(st["m"] != 0)
    g2, b2, h2, E2, st2 = q.qaoa_optimize_adam_resume(ctx, [ca, cb], g1, b1, 5, state=st, item_cost=ic, lr=0.02)
    assert st2["step"] == 11
    gf, bf, hf, Ef = q.qaoa_optimize_adam(ctx, [ca, cb], g0, b0, 11, item_cost=ic, lr=0.02)
    assert np.array_equal(g2, gf) and np.array_equal(b2, bf)
    assert np.array_equal(np.concatenate([h1, h2]), hf) and np.array_equal(E2, Ef)
    q.qaoa_cost_destroy(ca)
    q.qaoa_cost_destroy(cb)


def test_autograd_functions(q, ctx):
    """torch.autograd.Function wrappers: backward of E (single and batched)
    against the oracle's gradient and against central differences of the
    wrapped forward."""
    import torch
    from paper_2606_26297_b300.autograd import qaoa_expectation, qaoa_expectation_batch
    Q = inst.regular_maxcut_qubo(16, 4700)
    cost = _cost(q, ctx, Q)
    F = oracle.cost_table(oracle.canonical_of(Q))
    g0, b0 = inst.ramp_angles(3)
    g = torch.tensor(g0, dtype=torch.float64, requires_grad=True)
    b = torch.tensor(b0, dtype=torch.float64, requires_grad=True)
    E = qaoa_expectation(g, b, ctx, cost)
    (2.0 * E).backward()
    Eo, dgo, dbo = oracle.grad_adjoint(F, g0, b0)
    assert abs(E.item() - Eo) / np.max(np.abs(F)) <= E_TOL
    sc = max(np.abs(dgo).max(), np.abs(dbo).max())
    assert np.max(np.abs(g.grad.numpy() - 2 * dgo)) <= 2 * G_TOL * sc
    assert np.max(np.abs(b.grad.numpy() - 2 * dbo)) <= 2 * G_TOL * sc
    h = 1e-3
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd = (qaoa_expectation(torch.tensor(g0 + e), torch.tensor(b0), ctx, cost).item()
              - qaoa_expectation(torch.tensor(g0 - e), torch.tensor(b0), ctx, cost).item()) / (2 * h)
        assert abs(fd - dgo[k]) <= 1e-3 * sc
    # batched: weights per item flow into each item's gradient
    G0, B0 = inst.random_angles(3, 4, 4701, gamma_scale=0.3)
    G = torch.tensor(G0, requires_grad=True)
    B = torch.tensor(B0, requires_grad=True)
    Eb = qaoa_expectation_batch(G, B, ctx, [cost])
    w = torch.tensor([1.0, -2.0, 0.5, 3.0], dtype=torch.float64)
    (Eb * w).sum().backward()
    for i in range(4):
        Ei, dgi, dbi = oracle.grad_adjoint(F, G0[i], B0[i])
        assert abs(Eb[i].item() - Ei) / np.max(np.abs(F)) <= E_TOL
        sci = max(np.abs(dgi).max(), np.abs(dbi).max())
        assert np.max(np.abs(G.grad[i].numpy() - w[i].item() * dgi)) <= abs(w[i].item()) * G_TOL * sci
        assert np.max(np.abs(B.grad[i].numpy() - w[i].item() * dbi)) <= abs(w[i].item()) * G_TOL * sci
    q.qaoa_cost_destroy(cost)
