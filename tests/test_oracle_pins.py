"""Pins for the FP64 oracle: each test checks an oracle function against a
fact that does not come from the oracle itself (a closed form, a second
algorithm, a special case that reduces to a textbook result, or the published
p=1 MaxCut formula).  CPU only."""
import json
import math
import os
from fractions import Fraction
from itertools import product

import numpy as np
import pytest

from closed_forms import maxcut_p1_closed_form
import oracle
from paper_2606_26297_b300 import instances as inst

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_int_qubo(n, seed, lo=-6, hi=6):
    """Non-symmetric integer H (both triangles and the diagonal), integer f, c0."""
    rng = inst.SplitMix64(seed)
    H = np.array([[rng.randint(lo, hi) for _ in range(n)] for _ in range(n)], dtype=float)
    f = np.array([rng.randint(lo, hi) for _ in range(n)], dtype=float)
    c0 = float(rng.randint(lo, hi))
    return H, f, c0


# ---- Sec. 2.1: canonical form and objective -----------------------------------

def test_canonical_form_equals_input_form():
    """Eq. qubo_canonical_work must equal Eq. qubo_input_form, evaluated here
    directly as c0 + f.z + z^T H z for every z (exact for integers)."""
    for n, seed in [(1, 1), (5, 2), (9, 3)]:
        H, f, c0 = _rand_int_qubo(n, seed)
        cq = oracle.canonicalize(H, f, c0)
        F = oracle.cost_table(cq)
        Z = ((np.arange(1 << n)[:, None] >> np.arange(n)[None, :]) & 1).astype(float)
        direct = c0 + Z @ f + np.einsum("xi,ij,xj->x", Z, H, Z)
        assert np.array_equal(F, direct)


def test_cost_at_equals_input_form():
    """oracle.cost_at (F at sampled indices, the form used where the full table
    does not fit the host) against the input form c0 + f.z + z^T H z evaluated
    directly for each sampled z, exact for integers; sampled indices include
    0, 2^n - 1 and repeats, at n = 40 (beyond any table) and n = 9."""
    for n, seed in [(9, 5), (40, 6)]:
        H, f, c0 = _rand_int_qubo(n, seed)
        cq = oracle.canonicalize(H, f, c0)
        rng = np.random.default_rng(seed)
        xs = np.concatenate([[0, (1 << n) - 1, 5, 5], rng.integers(0, 1 << n, 60, dtype=np.uint64)]).astype(np.uint64)
        got = oracle.cost_at(cq, xs)
        for x, v in zip(xs.tolist(), got.tolist()):
            z = np.array([(x >> i) & 1 for i in range(n)], dtype=float)
            assert v == c0 + f @ z + z @ H @ z
        if n <= 20:
            assert np.array_equal(got, oracle.cost_table(cq)[xs.astype(np.int64)])


def test_cost_table_gray_code():
    """Objective table vs an independent Gray-code enumeration: flipping bit k
    of z changes F by (1-2 z_k)(l_k + sum_{i != k} b_{ik} z_i).  Bit-exact on
    an integer instance; also pins the brute-force argmin."""
    q = inst.upper_int_qubo(14, 77)
    cq = oracle.canonical_of(q)
    F = oracle.cost_table(cq)
    n = q.n
    bs = cq.b + cq.b.T
    z = np.zeros(n, dtype=np.int64)
    cur = int(cq.c0)
    G = np.empty(1 << n, dtype=np.int64)
    G[0] = cur
    for t in range(1, 1 << n):
        k = (t & -t).bit_length() - 1
        delta = int(cq.ell[k]) + int(bs[k] @ z)
        cur += delta if z[k] == 0 else -delta
        z[k] ^= 1
        x = t ^ (t >> 1)
        G[x] = cur
    assert np.array_equal(F.astype(np.int64), G)
    assert oracle.argmin(F) == int(np.flatnonzero(G == G.min())[0])


def test_uniform_mean_and_variance_closed_form():
    """p=0 (state |+>^n): mean_z F = c0 + sum l_i/2 + sum_{i<j} b_ij/4 and
    var_z F = sum_i h_i^2 + sum_{i<j} J_ij^2 with the Pauli coefficients of
    Eq. cost_hamiltonian_pauli (z = (1-s)/2): h_i = -(l_i/2 + sum_j b_ij/4),
    J_ij = b_ij/4.  Exact rationals on an integer instance."""
    H, f, c0 = _rand_int_qubo(11, 5)
    cq = oracle.canonicalize(H, f, c0)
    F = oracle.cost_table(cq)
    n = cq.n
    ell = [Fraction(int(v)) for v in cq.ell]
    b = [[Fraction(int(cq.b[i, j])) for j in range(n)] for i in range(n)]
    mean = Fraction(int(c0)) + sum(ell) / 2 + sum(b[i][j] for i in range(n) for j in range(i + 1, n)) / 4
    h = [-(ell[i] / 2 + sum(b[min(i, j)][max(i, j)] for j in range(n) if j != i) / 4) for i in range(n)]
    var = sum(x * x for x in h) + sum((b[i][j] / 4) ** 2 for i in range(n) for j in range(i + 1, n))
    Fi = [int(v) for v in F]
    N = len(Fi)
    assert Fraction(sum(Fi), N) == mean
    assert Fraction(sum(v * v for v in Fi), N) - mean * mean == var
    # the expectation routine on the uniform state reproduces the mean
    psi = oracle.evolve(F, [], [])
    assert abs(oracle.expectation(F, psi) - float(mean)) < 1e-9 * max(1.0, abs(float(mean)))


# ---- Sec. 2.3: the state ------------------------------------------------------

@pytest.fixture(scope="module")
def small():
    q = inst.upper_int_qubo(10, 11)
    return oracle.cost_table(oracle.canonical_of(q))


def test_zero_angles_identity(small):
    """gamma = beta = 0: the state stays |+>^n = 2^{-n/2} exactly."""
    psi = oracle.evolve(small, [0.0, 0.0, 0.0], [0.0, 0.0, 0.0])
    assert np.array_equal(psi, np.full(psi.shape, 2.0 ** -5, dtype=complex))


def test_gamma_zero_global_phase(small):
    """gamma = 0: RX(2b)|+> = e^{-ib}|+>, so the state is
    exp(-i n sum beta) 2^{-n/2}."""
    beta = [0.3, -1.1, 0.7]
    psi = oracle.evolve(small, [0.0] * 3, beta)
    ref = np.exp(-1j * 10 * sum(beta)) * 2.0 ** -5
    assert np.max(np.abs(psi - ref)) < 1e-14


def test_beta_zero_uniform_distribution(small):
    """beta = 0: only diagonal phases act, P is uniform and E is the mean."""
    psi = oracle.evolve(small, [0.4, 1.3], [0.0, 0.0])
    P = oracle.probabilities(psi)
    assert np.max(np.abs(P - 2.0 ** -10)) < 1e-16
    assert abs(oracle.expectation(small, psi) - small.mean()) < 1e-10


def test_last_beta_half_pi_is_global_flip(small):
    """beta_p = pi/2: RX(pi) = -iX on every qubit, so the final amplitude at x
    is (-i)^n phi(not x), phi being the state right after U_C(gamma_p)."""
    g, b = [0.37, 0.81], [0.52, math.pi / 2]
    psi = oracle.evolve(small, g, b)
    phi = oracle.evolve(small, g[:1], b[:1]) * np.exp(-1j * g[1] * small)
    flip = np.arange(1 << 10) ^ ((1 << 10) - 1)
    assert np.max(np.abs(psi - (-1j) ** 10 * phi[flip])) < 1e-13


def test_norm_preserved(small):
    for p in range(1, 5):
        g, b = inst.ramp_angles(p, 0.3)
        psi = oracle.evolve(small, g, b)
        assert abs(np.vdot(psi, psi).real - 1.0) < 1e-13


def test_separable_product_state():
    """b = 0: U_C and U_M both factorise over qubits, so the state is a tensor
    product of single-qubit states built from 2x2 matrices (and a global phase
    from c0).  Checked at n=12 with random real l_i and c0."""
    n = 12
    rng = inst.SplitMix64(9)
    ell = np.array(rng.normals(n))
    c0 = 0.75
    H = np.diag(ell)
    F = oracle.cost_table(oracle.canonicalize(H, None, c0))
    g, b = [0.9, -0.4, 1.7], [0.3, 1.1, -0.6]
    psi = oracle.evolve(F, g, b)
    amps = []
    for i in range(n):
        a = np.array([1.0, 1.0], dtype=complex) / math.sqrt(2)
        for gl, bl in zip(g, b):
            a = np.array([1.0, np.exp(-1j * gl * ell[i])]) * a
            rx = np.array([[math.cos(bl), -1j * math.sin(bl)], [-1j * math.sin(bl), math.cos(bl)]])
            a = rx @ a
        amps.append(a)
    ref = np.exp(-1j * sum(g) * c0) * np.ones(1, dtype=complex)
    for i in range(n):  # bit i of x is the fastest-varying factor
        ref = np.kron(amps[i], ref)
    assert np.max(np.abs(psi - ref)) < 1e-13
    # expectation: c0 + sum l_i P_i(1)
    E_ref = c0 + sum(ell[i] * abs(amps[i][1]) ** 2 for i in range(n))
    assert abs(oracle.expectation(F, psi) - E_ref) < 1e-12


def test_block_diagonal_tensor_product():
    """A QUBO with no couplings between two variable blocks evolves as the
    tensor product of the two blocks' states (DQAOA with zero cross terms)."""
    q1, q2 = inst.upper_int_qubo(5, 21), inst.normal_qubo(6, 22)
    q2.c0 = 0.25
    qb = inst.block_diagonal_qubo([q1, q2])
    F1 = oracle.cost_table(oracle.canonical_of(q1))
    F2 = oracle.cost_table(oracle.canonical_of(q2))
    Fb = oracle.cost_table(oracle.canonical_of(qb))
    g, b = [0.2, 0.5, 0.9], [0.8, 0.4, 0.1]
    psi = oracle.evolve(Fb, g, b)
    ref = np.kron(oracle.evolve(F2, g, b), oracle.evolve(F1, g, b))
    assert np.max(np.abs(psi - ref)) < 1e-13
    E = oracle.expectation(Fb, psi)
    E1 = oracle.expectation(F1, oracle.evolve(F1, g, b))
    E2 = oracle.expectation(F2, oracle.evolve(F2, g, b))
    assert abs(E - (E1 + E2)) < 1e-12


# ---- published p=1 MaxCut expectation -----------------------------------------

def _prism():
    return [(0, 1), (1, 2), (0, 2), (3, 4), (4, 5), (3, 5), (0, 3), (1, 4), (2, 5)]


def _cube():
    e = []
    for x in range(8):
        for k in range(3):
            y = x ^ (1 << k)
            if x < y:
                e.append((x, y))
    return e


@pytest.mark.parametrize("name,n,edges", [
    ("K4", 4, [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]),
    ("prism", 6, _prism()),
    ("cube", 8, _cube()),
    ("rand3reg10", 10, None),
    ("rand3reg14", 14, None),
])
def test_maxcut_p1_analytic(name, n, edges):
    if edges is None:
        edges = inst.random_regular_graph(n, 3, 100 + n)
    q = inst.maxcut_qubo(n, edges)
    F = oracle.cost_table(oracle.canonical_of(q))
    for gamma, beta in [(0.3, 0.2), (0.61, 1.17), (-1.4, 0.35), (2.2, -0.9)]:
        E = oracle.expectation(F, oracle.evolve(F, [gamma], [beta]))
        assert abs(E - maxcut_p1_closed_form(n, edges, gamma, beta)) < 1e-11


# ---- gradients ---------------------------------------------------------------

def test_adjoint_matches_central_differences():
    q = inst.normal_qubo(9, 31)
    F = oracle.cost_table(oracle.canonical_of(q))
    g, b = [0.31, 0.72, -0.45], [0.9, 0.2, 0.61]
    E, dg, db = oracle.grad_adjoint(F, g, b)
    fg, fb = oracle.grad_fd(F, g, b, h=1e-5)
    scale = max(np.max(np.abs(dg)), np.max(np.abs(db)))
    assert max(np.max(np.abs(dg - fg)), np.max(np.abs(db - fb))) <= 1e-7 * scale
    assert abs(E - oracle.expectation(F, oracle.evolve(F, g, b))) < 1e-12


def test_adjoint_special_cases():
    """gamma = 0 makes E independent of beta; beta = 0 makes E independent of
    gamma; both derivatives must then vanish."""
    F = oracle.cost_table(oracle.canonical_of(inst.upper_int_qubo(8, 41)))
    _, dg, db = oracle.grad_adjoint(F, [0.0, 0.0], [0.4, 1.2])
    assert np.max(np.abs(db)) < 1e-12
    _, dg, db = oracle.grad_adjoint(F, [0.5, 0.9], [0.0, 0.0])
    assert np.max(np.abs(dg)) < 1e-12


def test_adjoint_matches_analytic_p1_derivative():
    """p=1 MaxCut: the adjoint gradient equals the derivative of the published
    closed form (taken by central differences on the closed form itself)."""
    n = 12
    edges = inst.random_regular_graph(n, 3, 5)
    F = oracle.cost_table(oracle.canonical_of(inst.maxcut_qubo(n, edges)))
    gamma, beta, h = 0.47, 0.33, 1e-6
    _, dg, db = oracle.grad_adjoint(F, [gamma], [beta])
    cf = lambda g_, b_: maxcut_p1_closed_form(n, edges, g_, b_)
    ag = (cf(gamma + h, beta) - cf(gamma - h, beta)) / (2 * h)
    ab = (cf(gamma, beta + h) - cf(gamma, beta - h)) / (2 * h)
    assert abs(dg[0] - ag) < 1e-7 * max(1, abs(ag))
    assert abs(db[0] - ab) < 1e-7 * max(1, abs(ab))


# ---- decoding, top-K, argmin ------------------------------------------------

def test_topk_by_probability_then_index():
    P = np.array([0.1, 0.3, 0.1, 0.3, 0.05, 0.15])
    assert list(oracle.topk(P, 4)) == [1, 3, 5, 0]
    rng = np.random.default_rng(0)
    P = rng.random(4096)
    ref = sorted(range(4096), key=lambda i: (-P[i], i))[:10]
    assert list(oracle.topk(P, 10)) == ref


def test_paper_parameter_layout():
    """x = [gamma_1, beta_1, ..., gamma_p, beta_p] (Sec. 3.4)."""
    assert list(oracle.interleave([0.4, 0.8], [0.7, 0.3])) == [0.4, 0.7, 0.8, 0.3]


# ---- Sec. 3.1-3.2: allocation ---------------------------------------------------

def test_allocation_figure_counts():
    """Fig. allocation_strategies: cross-QPU counts on panel (a)'s graph and the
    remote-CX estimate 2 * cross * p (Sec. 3.1)."""
    gold = json.load(open(os.path.join(GOLDEN, "allocation_figure.json")))
    n = 6
    H = np.zeros((n, n))
    for u, v in gold["panel_a_edges"]:
        H[u - 1, v - 1] = 1.0
    cq = oracle.canonicalize(H, None, 0.0)
    for name, a in gold["allocations"].items():
        qpu_of = [0] * n
        for m, vs in enumerate(a["qpus"]):
            for v in vs:
                qpu_of[v - 1] = m
        assert oracle.validate_allocation(qpu_of, [3, 3])
        loc, cross, est = oracle.classify(cq, qpu_of, p=3)
        assert cross == a["panel_a_cross"], name
        assert loc + cross == len(gold["panel_a_edges"])
        assert est == 2 * cross * 3
    assert oracle.contiguous_allocation(6, oracle.balanced_capacities(6, 2)) == [0, 0, 0, 1, 1, 1]


def test_dense30_partition_counts():
    """Dense n=30, three QPUs of capacity 10, contiguous: 3*C(10,2)=135 local,
    C(30,2)-135 = 300 cross, estimate 2*300*8 = 4800 at p=8."""
    q = inst.normal_qubo(30, 1003)
    cq = oracle.canonical_of(q)
    caps = oracle.balanced_capacities(30, 3)
    assert caps == [10, 10, 10]
    qpu_of = oracle.contiguous_allocation(30, caps)
    assert oracle.validate_allocation(qpu_of, caps)
    assert oracle.classify(cq, qpu_of, 8) == (135, 300, 4800)


def test_validate_allocation_rejects():
    assert not oracle.validate_allocation([0, 0, 0, 0], [3, 3])   # QPU 2 unused / cap exceeded
    assert not oracle.validate_allocation([0, 2, 1], [2, 2])      # unknown QPU
    assert oracle.validate_allocation([0, 1, 1], [2, 2])
