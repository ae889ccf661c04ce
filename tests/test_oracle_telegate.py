"""Pins for the gate-level TeleGate oracle (oracle/telegate.py): the remote
CNOT against the CNOT matrix for every measurement record, the distributed
circuit on one QPU against the (separately pinned) monolithic evolution, and
with remote gates against it up to the protocol's global sign.  CPU only."""
import itertools

import numpy as np
import pytest

import oracle
from oracle import telegate as otg
from paper_2606_26297_b300 import instances as inst


def _cnot_full(n, c, t, psi):
    out = psi.copy()
    idx = np.arange(len(psi))
    sel = idx[((idx >> c) & 1) == 1]
    out[sel] = psi[sel ^ (1 << t)]
    return out


@pytest.mark.parametrize("a,t", [(0, 1), (1, 0), (0, 2), (2, 1)])
def test_remote_cnot_every_record(a, t):
    """For every record (m1, m2) the remote CNOT leaves the data qubits in
    CNOT|psi> times (-1)^(m1 m2), and the communication qubits in |m1 m2>."""
    n = 3
    rng = np.random.default_rng(a * 10 + t)
    data = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    data /= np.linalg.norm(data)
    full = np.zeros(1 << (n + 2), dtype=np.complex128)
    full[: 1 << n] = data
    want = _cnot_full(n, a, t, data)
    ops = otg.remote_cnot(n, a, t)
    for rec in itertools.product([0, 1], repeat=2):
        psi, outs = otg.run_from(n, full, ops, forced=list(rec))
        assert outs == list(rec)
        m1, m2 = rec
        block = psi.reshape(4, 1 << n)
        comm = m1 | (m2 << 1)
        assert np.allclose(block[comm], (-1) ** (m1 * m2) * want, atol=1e-12)
        assert np.allclose(np.delete(block, comm, axis=0), 0, atol=1e-12)


def test_single_qpu_circuit_equals_monolithic():
    """All variables on one QPU: the gate sequence equals exp(-i g F) layer by
    layer, so the data state equals the monolithic evolution exactly."""
    Q = inst.upper_int_qubo(5, 61)
    cq = oracle.canonical_of(Q)
    F = oracle.cost_table(cq)
    g, b = [0.3, -0.2], [0.7, 0.4]
    ops = otg.circuit(cq, [0] * 5, g, b)
    psi, outs = otg.run(5, ops, seed=1, traj=0)
    assert outs == []
    assert np.allclose(otg.data_state(5, psi), oracle.evolve(F, g, b), atol=1e-12)


@pytest.mark.parametrize("traj", [0, 1, 2])
def test_distributed_circuit_equals_monolithic_up_to_sign(traj):
    """Three QPUs with cross couplings: every trajectory's data state is the
    monolithic state up to a global sign, and the protocol counts follow
    2 remote CNOTs per cross coupling per layer (Sec. 3.1's estimate)."""
    Q = inst.upper_int_qubo(6, 62)
    cq = oracle.canonical_of(Q)
    F = oracle.cost_table(cq)
    qpu = [0, 0, 1, 1, 2, 2]
    g, b = [0.25, 0.1], [0.6, 0.3]
    ops = otg.circuit(cq, qpu, g, b)
    psi, outs = otg.run(6, ops, seed=9, traj=traj)
    d = otg.data_state(6, psi)
    mono = oracle.evolve(F, g, b)
    ov = np.vdot(mono, d)
    assert abs(abs(ov) - 1.0) < 1e-12
    assert abs(ov.imag) < 1e-12
    assert np.allclose(d, np.sign(ov.real) * mono, atol=1e-12)
    c = otg.counts(cq, qpu, 2)
    loc, cross, est = oracle.classify(cq, qpu, 2)
    assert c["remote_cx"] == est and c["cross_zz"] == 2 * cross
    assert len(outs) == c["measurements"]
