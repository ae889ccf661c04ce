"""Pins for the sampling / sampled-metrics / SPSA oracle (oracle/sampling.py).
Each test checks it against a fact that does not come from the oracle itself:
published known-answer values of the generator, closed forms for dyadic
states, hand-worked metrics, the exactness of the symmetric difference on a
quadratic, the closed-form Adam trajectory on a linear objective, and the
central limit theorem against the (separately pinned) exact expectation.
CPU only."""
import json
import math
import os
from itertools import product

import numpy as np
import pytest

import oracle
from oracle import sampling as osm
from paper_2606_26297_b300 import instances as inst

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    """Philox4x32-10 against the generator authors' published known-answer
    values (tests/golden/philox4x32_10_kat.json)."""
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.json")) as fh:
        kat = json.load(fh)
    for v in kat["vectors"]:
        ctr = [int(w, 16) for w in v["ctr"]]
        key = [int(w, 16) for w in v["key"]]
        assert list(osm.philox4x32_10(ctr, key)) == [int(w, 16) for w in v["out"]]


def test_shot_randoms_uniform():
    """The top 4 bits of 8192 draws fall in 16 equal bins (chi-square, 15 dof,
    far tail at 50) and distinct streams differ."""
    R = osm.shot_randoms(seed=1234, stream=7, shots=8192)
    counts = np.bincount([r >> 60 for r in R], minlength=16)
    chi2 = float(np.sum((counts - 512.0) ** 2 / 512.0))
    assert chi2 < 50.0
    assert osm.shot_randoms(1234, 8, 4) != osm.shot_randoms(1234, 7, 4)
    assert osm.shot_randoms(1234, 7, 4, first=2)[:2] == R[2:4]


def _leading_ones(r):
    k = 0
    while k < 64 and (r >> (63 - k)) & 1:
        k += 1
    return k


def test_sample_dyadic_closed_form():
    """Amplitudes 1/2 + i/2, 1/2, 1/4 + i/4, 1/4 + i/4 give P = (1/2, 1/4,
    1/8, 1/8) exactly: Q = 2^60, T = R >> 4, and the shot is the number of
    leading one bits of R, capped at 3."""
    amps = np.array([0.5 + 0.5j, 0.5 + 0j, 0.25 + 0.25j, 0.25 + 0.25j], dtype=np.complex64)
    assert [int(w) for w in osm.weights(amps)] == [2 ** 59, 2 ** 58, 2 ** 57, 2 ** 57]
    R = osm.shot_randoms(99, 0, 4000) + [0, 2 ** 64 - 1, 2 ** 63, 2 ** 63 - 1, 3 * 2 ** 62, 7 * 2 ** 61]
    x = osm.sample(amps, R)
    assert [int(v) for v in x] == [min(_leading_ones(r), 3) for r in R]


def test_sample_zero_weights_and_basis_state():
    """Indices of zero probability are never drawn; a basis state is always
    drawn."""
    amps = np.zeros(64, dtype=np.complex64)
    amps[37] = 1.0
    R = osm.shot_randoms(5, 1, 500) + [0, 2 ** 64 - 1]
    assert set(int(v) for v in osm.sample(amps, R)) == {37}
    amps = np.zeros(64, dtype=np.complex64)
    amps[[0, 63, 20]] = [0.6, 0.8j, 0.0]
    xs = set(int(v) for v in osm.sample(amps, osm.shot_randoms(5, 2, 2000)))
    assert xs == {0, 63}


def test_sample_brute_force_intervals():
    """Every shot of a random 6-qubit state lies in the half-open weight
    interval its target selects, computed here with Python integers over an
    explicit list of the intervals."""
    rng = np.random.default_rng(3)
    a = (rng.standard_normal(64) + 1j * rng.standard_normal(64)).astype(np.complex64)
    a /= np.float32(np.linalg.norm(a))
    q = [int(np.floor((float(z.real) ** 2 + float(z.imag) ** 2) * 2.0 ** 60)) for z in a]
    Q = sum(q)
    lo = 0
    intervals = []
    for w in q:
        intervals.append((lo, lo + w))
        lo += w
    R = osm.shot_randoms(11, 3, 3000)
    x = osm.sample(a, R)
    for r, xi in zip(R, x):
        T = (r * Q) >> 64
        l, h = intervals[int(xi)]
        assert l <= T < h


def test_sampled_mean_converges_to_expectation():
    """The shot estimate of Eq. training_objective_mean_cost is within five
    standard errors of the exact expectation (Eq. qaoa_expectation_expanded)."""
    q = inst.normal_qubo(10, 21)
    F = oracle.cost_table(oracle.canonical_of(q))
    psi = oracle.evolve(F, [0.3, 0.5], [0.7, 0.2])
    E = oracle.expectation(F, psi)
    P = oracle.probabilities(psi)
    sd = math.sqrt(float(np.sum(P * (F - E) ** 2)))
    S = 20000
    idx = osm.sample(psi, osm.shot_randoms(2024, 0, S))
    assert abs(osm.sampled_mean(F, idx) - E) < 5 * sd / math.sqrt(S)
    counts = np.bincount(idx.astype(np.int64), minlength=len(P))
    big = P > 0.01
    assert np.all(np.abs(counts[big] / S - P[big]) < 5 * np.sqrt(P[big] / S))


def test_metrics_hand_worked():
    """Sec. 3.6 metrics on a hand-worked example: shots on x = 3, 3, 1, 2, 3, 1
    with F = (5, -1, 2, -1)."""
    F = np.array([5.0, -1.0, 2.0, -1.0])
    m = osm.metrics(F, [3, 3, 1, 2, 3, 1], margin=3.0, elite=2, ref_cost=-1.0, ref_index=3)
    assert m["shots"] == 6 and m["distinct"] == 3
    assert m["best_cost"] == -1.0 and m["best_index"] == 1
    assert m["p_best_index"] == pytest.approx(2 / 6)
    assert m["p_best_cost"] == pytest.approx(5 / 6)
    assert m["mean_cost"] == pytest.approx(-0.5)
    assert m["low_cost_mass"] == pytest.approx(1.0)
    assert m["elite"] == [(3, -1.0, 3, 0.5), (1, -1.0, 2, pytest.approx(1 / 3))]
    assert m["p_ref_cost"] == pytest.approx(5 / 6) and m["best_cost_matches_ref"]
    assert m["p_ref_index"] == pytest.approx(0.5) and not m["best_index_matches_ref"]
    m = osm.metrics(F, [0, 2, 2], margin=2.5, elite=5)
    assert m["best_cost"] == 2.0 and m["low_cost_mass"] == pytest.approx(2 / 3)
    assert m["elite"] == [(2, 2.0, 2, pytest.approx(2 / 3)), (0, 5.0, 1, pytest.approx(1 / 3))]


def test_spsa_estimate_quadratic_exact_mean():
    """On J(x) = 1/2 x^T A x (A symmetric) the symmetric difference is exact, so
    the SPSA estimate averaged over all 2^d sign vectors equals A x."""
    rng = np.random.default_rng(0)
    d = 4
    M = rng.standard_normal((d, d))
    A = M + M.T
    x = rng.standard_normal(d)
    J = lambda y: 0.5 * y @ A @ y
    ck = 0.37
    acc = np.zeros(d)
    for signs in product([-1.0, 1.0], repeat=d):
        D = np.array(signs)
        acc += osm.spsa_estimate(J(x + ck * D), J(x - ck * D), D, ck)
    assert np.allclose(acc / 2 ** d, A @ x, rtol=1e-12, atol=1e-12)


def test_spsa_adam_linear_closed_form():
    """On J(x) = a x in one dimension every SPSA estimate is a, so Adam's
    bias-corrected moments are a and a^2 and each step moves x by
    -lr a / (|a| + eps)."""
    a, lr, eps = -2.5, 0.05, 1e-8
    x, hist = osm.spsa_adam(lambda y, k, w: a * float(y[0]), np.array([0.3]), 7, seed=9, lr=lr, eps=eps)
    assert x[0] == pytest.approx(0.3 - 7 * lr * a / (abs(a) + eps), rel=1e-12)
    assert len(hist) == 7


def test_spsa_signs_balanced():
    """Perturbation signs are +-1 and balanced over many draws."""
    s = np.concatenate([osm.spsa_signs(77, k, b, 16) for k in range(40) for b in range(3)])
    assert set(np.unique(s)) == {-1.0, 1.0}
    assert abs(float(s.mean())) < 5 / math.sqrt(len(s))


def test_weights_exact_fractions():
    """q = floor(re^2 2^60) + floor(im^2 2^60) against exact rational
    arithmetic (fractions.Fraction of the stored float) for float32 and float64
    components: random values, zero, +-1, powers of two, float32 denormals."""
    from fractions import Fraction
    rng = np.random.default_rng(8)
    vals32 = np.concatenate([rng.standard_normal(300) * 0.3, [0.0, 1.0, -1.0, 2.0 ** -20, 2.0 ** -31, 2.0 ** -40,
                                                               1e-38, 1e-44, -3e-45]]).astype(np.float32)
    vals64 = np.concatenate([rng.standard_normal(300) * 0.3, [0.0, 1.0, -1.0, 2.0 ** -31, 1e-300]])
    for vals in (vals32, vals64):
        a = vals[: len(vals) // 2 * 2]
        z = (a[0::2] + 1j * a[1::2]).astype(np.complex64 if vals.dtype == np.float32 else np.complex128)
        got = osm.weights(z)
        for k, c in enumerate(z):
            want = sum(math.floor(Fraction(float(v)) ** 2 * 2 ** 60) for v in (c.real, c.imag))
            assert int(got[k]) == want
