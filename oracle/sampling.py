"""Oracle for shot sampling, the sampled metrics and the SPSA-Adam optimiser.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
it; the product never imports it and it never imports the product.

What it follows:

* Sec. 3.4 (training objective): the circuit is measured with a number of shots
  and the mean cost of the measured bitstrings is the objective; several
  averaging passes are averaged.
* Sec. 3.4 (parameter update): SPSA draws one simultaneous perturbation of all
  parameters per iteration, evaluates the objective at the two perturbed
  points, forms a gradient estimate from their difference and feeds it to Adam.
* Sec. 3.6 (final distribution metrics): counts of each decoded bitstring, best
  sampled cost and bitstring, sampled mean cost, probability of the best
  bitstring, low-cost mass within a margin of the best cost, the elite set of
  top sampled bitstrings, and the reference-based quantities.

Readings (the paper does not fix these; the CUDA path implements the same
definitions independently):

* Measurement is inverse-CDF sampling on integer weights.  The weight of
  index x is q_x = floor(re^2 2^60) + floor(im^2 2^60), each square taken
  exactly from the stored amplitude component (float32 or float64), so q_x is
  |psi_x|^2 in units of 2^-60, truncated per component.  With Q = sum_x q_x
  and a 64-bit random integer R per shot, the shot's target is
  T = floor(R * Q / 2^64) and the shot lands on the smallest x whose inclusive
  prefix sum of q exceeds T.  Integer sums are exact, so every order of
  summation gives the same x.
* Random integers come from the counter-based generator Philox4x32-10 (Salmon,
  Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC
  2011), written here from that definition.  Shot s of stream t under seed k
  takes counter (s mod 2^32, s >> 32, t mod 2^32, t >> 32) and key
  (k mod 2^32, k >> 32), and R = out0 + 2^32 out1.
* SPSA perturbation of parameter i (i = 0..2p-1 over x = [g1, b1, ...]) of
  start b at iteration k is +1 when bit 0 of out0 of Philox with counter
  (i, b, k, 0x53505341) and the same key is 0, else -1.  The perturbation size
  is c_k = c / (k + 1)^decay.  The estimate is
  g_i = (J(x + c_k D) - J(x - c_k D)) / (2 c_k D_i).
* Elite order: count descending, then cost ascending, then index ascending.
"""
from __future__ import annotations

import math

import numpy as np

M32 = 0xFFFFFFFF
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
SPSA_TAG = 0x53505341
WEIGHT_BITS = 60


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds (Salmon et al. 2011): each round multiplies
    words 0 and 2 by the two round multipliers, and the new words are
    (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); the key
    is bumped by the two Weyl constants between rounds."""
    c0, c1, c2, c3 = (int(v) & M32 for v in ctr)
    k0, k1 = int(key[0]) & M32, int(key[1]) & M32
    for r in range(10):
        if r:
            k0 = (k0 + PHILOX_W0) & M32
            k1 = (k1 + PHILOX_W1) & M32
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0, p1 & M32, (p0 >> 32) ^ c3 ^ k1, p0 & M32)
    return c0, c1, c2, c3


def shot_randoms(seed: int, stream: int, shots: int, first: int = 0) -> list[int]:
    """R_s for s = first .. first+shots-1 (64-bit integers)."""
    key = (seed & M32, (seed >> 32) & M32)
    out = []
    for s in range(first, first + shots):
        w = philox4x32_10((s & M32, s >> 32, stream & M32, (stream >> 32) & M32), key)
        out.append(w[0] | (w[1] << 32))
    return out


def spsa_signs(seed: int, k: int, b: int, nparam: int) -> np.ndarray:
    """The +-1 perturbation of start b at iteration k (nparam entries)."""
    key = (seed & M32, (seed >> 32) & M32)
    return np.array([1.0 if (philox4x32_10((i, b, k, SPSA_TAG), key)[0] & 1) == 0 else -1.0
                     for i in range(nparam)])


def _sq60(v: np.ndarray) -> np.ndarray:
    """floor(v^2 2^60) of every entry (|v| < 2), exact: v = M 2^(e - d) with an
    integer mantissa M of d bits (24 for float32, 53 for float64), so v^2 2^60
    is M^2 shifted left by 2(e - d) + 60 (right when negative)."""
    m, e = np.frexp(v)
    if v.dtype == np.float32:
        M = np.abs(m.astype(np.float64) * 2.0 ** 24).astype(np.int64)
        sh = 2 * (e.astype(np.int64) - 24) + 60
        M2 = M * M  # < 2^48: exact in int64
        left = M2 << np.clip(sh, 0, 14)
        right = M2 >> np.clip(-sh, 0, 63)
        return np.where(sh >= 0, left, right).astype(np.uint64)
    M = np.abs(m * 2.0 ** 53).astype(np.int64)
    sh = 2 * (e.astype(np.int64) - 53) + 60
    out = [(int(a) * int(a)) << int(t) if t >= 0 else (int(a) * int(a)) >> int(-t) for a, t in zip(M, sh)]
    return np.array(out, dtype=np.uint64)


def weights(amps: np.ndarray) -> np.ndarray:
    """q_x = floor(re^2 2^60) + floor(im^2 2^60) (uint64) of a complex64 or
    complex128 state."""
    a = np.asarray(amps)
    return _sq60(np.ascontiguousarray(a.real)) + _sq60(np.ascontiguousarray(a.imag))


def sample(amps: np.ndarray, R) -> np.ndarray:
    """Inverse-CDF measurement of the state for the random integers R."""
    q = weights(amps)
    cum = np.cumsum(q, dtype=np.uint64)  # exact: Q < 2^63 for a state of norm < 8
    Q = int(cum[-1])
    T = np.array([(int(r) * Q) >> 64 for r in R], dtype=np.uint64)
    return np.searchsorted(cum, T, side="right").astype(np.uint64)


def sampled_mean(F: np.ndarray, idx) -> float:
    """Mean cost of the measured bitstrings (the shot estimate of Eq.
    training_objective_mean_cost)."""
    return float(np.mean(F[np.asarray(idx, dtype=np.int64)]))


def metrics(F: np.ndarray, idx, margin: float, elite: int, ref_cost=None, ref_index=None, tol: float = 1e-9):
    """The sampled metrics of Sec. 3.6 from the measured indices idx."""
    idx = np.asarray(idx, dtype=np.int64)
    S = len(idx)
    xs, counts = np.unique(idx, return_counts=True)
    costs = F[xs]
    best_cost = float(costs.min())
    best_x = int(xs[costs == best_cost].min())
    out = {
        "shots": S,
        "distinct": len(xs),
        "mean_cost": float(np.sum(costs * counts) / S),
        "best_cost": best_cost,
        "best_index": best_x,
        "p_best_index": float(counts[xs == best_x][0] / S),
        "p_best_cost": float(counts[costs == best_cost].sum() / S),
        "low_cost_mass": float(counts[costs <= best_cost + margin].sum() / S),
    }
    order = sorted(range(len(xs)), key=lambda j: (-int(counts[j]), float(costs[j]), int(xs[j])))[:elite]
    out["elite"] = [(int(xs[j]), float(costs[j]), int(counts[j]), float(counts[j] / S)) for j in order]
    if ref_cost is not None:
        out["p_ref_cost"] = float(counts[np.abs(costs - ref_cost) <= tol].sum() / S)
        out["best_cost_matches_ref"] = abs(best_cost - ref_cost) <= tol
    if ref_index is not None:
        hit = counts[xs == ref_index]
        out["p_ref_index"] = float(hit[0] / S) if len(hit) else 0.0
        out["best_index_matches_ref"] = best_x == ref_index
    return out


def adam_step(theta, g, m, v, t, lr, b1, b2, eps):
    """One Adam update with bias-corrected moments (t counts from 1)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def spsa_estimate(jp: float, jm: float, D: np.ndarray, ck: float) -> np.ndarray:
    """g_i = (J(x + c_k D) - J(x - c_k D)) / (2 c_k D_i)."""
    return (jp - jm) / (2.0 * ck * D)


def spsa_adam(objective, x0: np.ndarray, iterations: int, seed: int, b: int = 0, c: float = 0.1,
              decay: float = 0.101, lr: float = 0.01, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """SPSA-Adam of Sec. 3.4 on one start: objective(x, k, which) -> J, with
    which = 0 for x + c_k D and 1 for x - c_k D.  Returns (x, history of the
    estimates (J+, J-) per iteration)."""
    x = np.array(x0, dtype=np.float64)
    m = np.zeros_like(x)
    v = np.zeros_like(x)
    hist = []
    for k in range(iterations):
        D = spsa_signs(seed, k, b, len(x))
        ck = c / (k + 1) ** decay
        jp = objective(x + ck * D, k, 0)
        jm = objective(x - ck * D, k, 1)
        g = spsa_estimate(jp, jm, D, ck)
        x, m, v = adam_step(x, g, m, v, k + 1, lr, b1, b2, eps)
        hist.append((jp, jm))
    return x, hist
