"""Oracle for the explicit distributed (TeleGate) QAOA circuit of Sec. 3.3:
a plain gate-level statevector simulator over n data qubits plus two
communication qubits, with mid-circuit measurement, reset and classical
feed-forward, run trajectory by trajectory.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
it; the product never imports it and it never imports the product.

The circuit (Sec. 3.3, in the paper's order): every data qubit starts in |+>;
each layer applies the cost terms, then RX(2 beta) on every data qubit.  A
linear term is a phase on its qubit; a quadratic term is the sequence CNOT,
phase rotation, CNOT; when its two variables sit on different QPUs each of
the two CNOTs is a remote CNOT done through the communication pair: reset both
communication qubits, prepare one in superposition and entangle the pair,
couple one to the control and measure it, couple the other to the target and
measure it (in the X basis), then apply the outcome-controlled Pauli
corrections to the data qubits.

Readings:

* Phases in the 0/1 form of the objective, so the circuit equals
  exp(-i g F) exactly: z_i z_j = (z_i + z_j - z_i xor z_j) / 2, so a coupling
  b_ij contributes phase(-g b_ij / 2) on qubits i and j and, between the two
  CNOTs (control i, target j), phase(+g b_ij / 2) on j; phase(t) multiplies
  the |1> amplitude by e^{i t}.  Each qubit's phases are merged into one:
  phase(-g (l_i + sum_j b_ij / 2)).  The constant c0 is the global phase
  e^{-i g c0}.  RX(2 b) = exp(-i b X).
* Remote CNOT (control a, target t): reset cA, cB; H cA; CNOT cA -> cB;
  CNOT a -> cA; measure cA = m1; CNOT cB -> t; H cB; measure cB = m2;
  X^m1 on t; Z^m2 on a.  The data state then equals CNOT applied directly,
  times the global sign (-1)^(m1 m2).
* Reset of a communication qubit: it is in a basis state at that point (the
  previous protocol measured it), so the reset projects on the more likely
  value (P(1) > 1/2 means 1), renormalises, and flips it to 0 when that value
  is 1; it draws no random number.
* Qubit order: data qubit i is bit i, cA is bit n, cB is bit n + 1.
* Measurement k of trajectory t draws u from Philox4x32-10 at counter
  (k, t, 0, 0x54454C45) with key (seed lo, seed hi), u = (w0 + 2^32 w1) >> 11
  times 2^-53, and the outcome is 1 when u < P(1), P(1) summed in FP64.
"""
from __future__ import annotations

import math

import numpy as np

from . import sampling as osm

TAG_TELE = 0x54454C45

# op kinds
PHASE, RX, H, X, Z, CNOT, MEASURE, XIF, ZIF, GPHASE, RESET = range(11)


def remote_cnot(n: int, a: int, t: int) -> list:
    """Op list of one TeleGate remote CNOT (control a, target t)."""
    cA, cB = n, n + 1
    return [(RESET, cA, 0, 0.0), (RESET, cB, 0, 0.0), (H, cA, 0, 0.0), (CNOT, cA, cB, 0.0), (CNOT, a, cA, 0.0), (MEASURE, cA, 0, 0.0),
            (CNOT, cB, t, 0.0), (H, cB, 0, 0.0), (MEASURE, cB, 1, 0.0), (XIF, t, 0, 0.0), (ZIF, a, 1, 0.0)]


def circuit(cq, qpu_of, gamma, beta) -> list:
    """Op list of the distributed circuit.  Ops are (kind, q0, q1, theta);
    MEASURE stores its outcome in slot q1, XIF/ZIF read slot q1."""
    n = cq.n
    ops = []
    for q in range(n):
        ops.append((H, q, 0, 0.0))
    for g, b in zip(gamma, beta):
        ops.append((GPHASE, 0, 0, -g * cq.c0))
        for i in range(n):
            lin = cq.ell[i] + 0.5 * sum(cq.b[min(i, j)][max(i, j)] for j in range(n) if j != i)
            ops.append((PHASE, i, 0, -g * lin))
        for i in range(n):
            for j in range(i + 1, n):
                bij = cq.b[i][j]
                if bij == 0:
                    continue
                cx = [(CNOT, i, j, 0.0)] if qpu_of[i] == qpu_of[j] else remote_cnot(n, i, j)
                ops += cx + [(PHASE, j, 0, 0.5 * g * bij)] + cx
        for q in range(n):
            ops.append((RX, q, 0, b))
    return ops


def uniform(seed: int, k: int, t: int) -> float:
    w = osm.philox4x32_10((k, t, 0, TAG_TELE), (seed & osm.M32, (seed >> 32) & osm.M32))
    return ((w[0] | (w[1] << 32)) >> 11) * 2.0 ** -53


def run(n: int, ops: list, seed: int, traj: int, forced=None):
    """Run one trajectory from |0...0>; returns (state of n + 2 qubits,
    outcomes).  forced: optional list of outcomes to use instead of draws."""
    psi = np.zeros(1 << (n + 2), dtype=np.complex128)
    psi[0] = 1.0
    return run_from(n, psi, ops, seed=seed, traj=traj, forced=forced)


def run_from(n: int, psi0: np.ndarray, ops: list, seed: int = 0, traj: int = 0, forced=None):
    """Run the ops from the state psi0 of n + 2 qubits."""
    N = 1 << (n + 2)
    psi = np.array(psi0, dtype=np.complex128)
    idx = np.arange(N)
    slots = [0, 0]
    outcomes = []
    k = 0
    for kind, q0, q1, th in ops:
        bit0 = (idx >> q0) & 1
        if kind == PHASE:
            psi = np.where(bit0 == 1, psi * np.exp(1j * th), psi)
        elif kind == GPHASE:
            psi = psi * np.exp(1j * th)
        elif kind in (RX, H, X):
            lo = psi[idx[bit0 == 0]]
            hi = psi[idx[bit0 == 0] | (1 << q0)]
            if kind == RX:
                c, s = math.cos(th), math.sin(th)
                nlo, nhi = c * lo - 1j * s * hi, -1j * s * lo + c * hi
            elif kind == H:
                r = 1.0 / math.sqrt(2.0)
                nlo, nhi = r * (lo + hi), r * (lo - hi)
            else:
                nlo, nhi = hi, lo
            psi = psi.copy()
            psi[idx[bit0 == 0]] = nlo
            psi[idx[bit0 == 0] | (1 << q0)] = nhi
        elif kind == Z:
            psi = np.where(bit0 == 1, -psi, psi)
        elif kind == CNOT:
            sel = idx[(bit0 == 1) & (((idx >> q1) & 1) == 0)]
            psi = psi.copy()
            a, b = psi[sel].copy(), psi[sel | (1 << q1)].copy()
            psi[sel], psi[sel | (1 << q1)] = b, a
        elif kind == MEASURE:
            p1 = float(np.sum(np.abs(psi[bit0 == 1]) ** 2))
            if forced is not None:
                m = forced[k]
            else:
                m = 1 if uniform(seed, k, traj) < p1 else 0
            k += 1
            pm = p1 if m == 1 else 1.0 - p1
            psi = np.where(bit0 == m, psi / math.sqrt(pm), 0.0)
            slots[q1] = m
            outcomes.append(m)
        elif kind == RESET:
            p1 = float(np.sum(np.abs(psi[bit0 == 1]) ** 2))
            m = 1 if p1 > 0.5 else 0
            pm = p1 if m == 1 else 1.0 - p1
            psi = np.where(bit0 == m, psi / math.sqrt(pm), 0.0)
            if m:
                lo = idx[bit0 == 0]
                psi = psi.copy()
                a, b = psi[lo].copy(), psi[lo | (1 << q0)].copy()
                psi[lo], psi[lo | (1 << q0)] = b, a
        elif kind in (XIF, ZIF):
            if slots[q1]:
                if kind == XIF:
                    lo = idx[bit0 == 0]
                    psi = psi.copy()
                    a, b = psi[lo].copy(), psi[lo | (1 << q0)].copy()
                    psi[lo], psi[lo | (1 << q0)] = b, a
                else:
                    psi = np.where(bit0 == 1, -psi, psi)
    return psi, outcomes


def data_state(n: int, psi: np.ndarray) -> np.ndarray:
    """Data-qubit amplitudes (the communication qubits end in basis states)."""
    N = 1 << n
    return psi[0:N] + psi[N:2 * N] + psi[2 * N:3 * N] + psi[3 * N:4 * N]


def counts(cq, qpu_of, p: int) -> dict:
    """Gate and protocol counts of the distributed circuit."""
    n = cq.n
    loc = cross = 0
    for i in range(n):
        for j in range(i + 1, n):
            if cq.b[i][j] != 0:
                if qpu_of[i] == qpu_of[j]:
                    loc += 1
                else:
                    cross += 1
    rcx = 2 * cross * p
    return {"local_zz": loc * p, "cross_zz": cross * p, "remote_cx": rcx, "measurements": 2 * rcx,
            "resets": 2 * rcx, "feedforward": 2 * rcx}
