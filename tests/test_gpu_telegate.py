"""GPU parity of the gate-level TeleGate simulation (qaoa_telegate_simulate,
Sec. 3.3) against the oracle's gate-level simulator (oracle/telegate.py) and
the monolithic state.  The GPU evolves complex64 in shared memory; a
measurement draws the same Philox number on both sides, and its outcome is
the same unless P(1) = 1/2 lands within rounding of the draw."""
import math

import numpy as np
import pytest

import oracle
from oracle import telegate as otg
from paper_2606_26297_b300 import instances as inst

pytestmark = pytest.mark.gpu


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
    return q.qaoa_build_cost(ctx, Q.H, Q.f, Q.c0, "i32")


def test_trajectories_match_oracle_n6(q, ctx):
    """Three QPUs, p = 2: each trajectory's data state equals the oracle's
    trajectory (same measurement record, same global sign) within 1e-5, and
    its fidelity with the monolithic state is 1 within 1e-5."""
    Q = inst.upper_int_qubo(6, 7000)
    qpu = [0, 0, 1, 1, 2, 2]
    g, b = [0.22, 0.15], [0.6, 0.35]
    cost = _cost(q, ctx, Q)
    T, seed = 8, 77
    fid, amps, cnt = q.qaoa_telegate_simulate(ctx, cost, qpu, g, b, T, seed, want_amps=True)
    cq = oracle.canonical_of(Q)
    ops = otg.circuit(cq, qpu, g, b)
    for t in range(T):
        psi, outs = otg.run(6, ops, seed, t)
        d = otg.data_state(6, psi)
        assert np.linalg.norm(amps[t] - d) <= 1e-5
        assert abs(fid[t] - 1.0) <= 1e-5
    c = otg.counts(cq, qpu, 2)
    assert cnt["remote_cx"] == c["remote_cx"] and cnt["measurements"] == c["measurements"]
    assert cnt["resets"] == c["resets"] and cnt["cross_zz"] == c["cross_zz"] and cnt["ops"] == len(ops)
    q.qaoa_cost_destroy(cost)


def test_single_qpu_equals_monolithic(q, ctx):
    """One QPU: no remote operations, and the data state equals the oracle's
    monolithic evolution (no sign) within 1e-5."""
    Q = inst.upper_int_qubo(8, 7001)
    cost = _cost(q, ctx, Q)
    g, b = [0.1, 0.05, 0.12], [0.5, 0.4, 0.2]
    fid, amps, cnt = q.qaoa_telegate_simulate(ctx, cost, [0] * 8, g, b, 2, 5, want_amps=True)
    F = oracle.cost_table(oracle.canonical_of(Q))
    assert cnt["remote_cx"] == 0 and cnt["measurements"] == 0
    for t in range(2):
        assert np.linalg.norm(amps[t] - oracle.evolve(F, g, b)) <= 1e-5
    q.qaoa_cost_destroy(cost)


def test_dense12_three_qpus_fidelity_and_counts(q, ctx):
    """The paper's 12-variable size on three QPUs of four (Sec. 3.1 contiguous
    allocation), p = 2, 64 trajectories: every fidelity is 1 within 1e-4
    (about two thousand complex64 operations), trajectory 0 equals the
    oracle's monolithic state up to a global sign, and the remote CNOTs number
    2 x cross x p."""
    Q = inst.upper_int_qubo(12, 7002)
    cost = _cost(q, ctx, Q)
    qpu = [0] * 4 + [1] * 4 + [2] * 4
    g, b = [0.05, 0.03], [0.5, 0.25]
    fid, amps, cnt = q.qaoa_telegate_simulate(ctx, cost, qpu, g, b, 64, 123, want_amps=True)
    assert np.all(np.abs(fid - 1.0) <= 1e-4)
    F = oracle.cost_table(oracle.canonical_of(Q))
    mono = oracle.evolve(F, g, b)
    ov = np.vdot(mono, amps[0].astype(np.complex128))
    assert abs(abs(ov) - 1.0) <= 1e-4
    loc, cross, est = oracle.classify(oracle.canonical_of(Q), qpu, 2)
    assert cnt["remote_cx"] == est == 2 * cross * 2
    q.qaoa_cost_destroy(cost)


def test_telegate_rejects_bad_input(q, ctx):
    cost = _cost(q, ctx, inst.upper_int_qubo(13, 7003))
    with pytest.raises(q.QaoaError):
        q.qaoa_telegate_simulate(ctx, cost, [0] * 13, [0.1], [0.2], 1)
    q.qaoa_cost_destroy(cost)
    cost = _cost(q, ctx, inst.upper_int_qubo(5, 7004))
    with pytest.raises(q.QaoaError):
        q.qaoa_telegate_simulate(ctx, cost, [0, 0, -1, 1, 1], [0.1], [0.2], 1)
    with pytest.raises(q.QaoaError):
        q.qaoa_telegate_simulate(ctx, cost, [0] * 5, [0.1], [0.2], 0)
    q.qaoa_cost_destroy(cost)
