"""Oracle for the depth progression and multi-start search (Algorithm 1,
Sec. 3.5) and its candidate ranking.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use
it; the product never imports it and it never imports the product.

Algorithm 1 in the paper's order: for p = 1 .. p_max, build the initial points
(the previous depth's best lifted to depth p, perturbed copies of it, and fresh
random points), optimise every point, evaluate each result with a final shot-
based execution, rank the candidates and keep the best as the depth's
representative, whose parameters warm-start depth p + 1; finally rank the
representatives with the same rule.

Readings (the paper names these steps but does not define them; the CUDA
library implements the same definitions independently):

* Lifting to the next depth is the INTERP rule of Zhou et al., Phys. Rev. X 10,
  021067 (2020), the reference the paper cites for QAOA: for i = 1 .. p+1,
  x'_i = (i-1)/p x_{i-1} + (p-i+1)/p x_i with x_0 = x_{p+1} = 0, applied to
  gamma and beta separately.
* Random numbers are Philox4x32-10 words (oracle/sampling.py): a uniform in
  [0, 1) is u = (w0 + 2^32 w1) >> 11 times 2^-53, a normal is Box-Muller on the
  uniforms of (w0, w1) and (w2, w3), z = sqrt(-2 ln(1 - u1)) cos(2 pi u2).
  Counter (i, j, p, tag) for entry i of the interleaved x of point j at depth
  p; tag 0x52414E44 for random starts (gamma_i = gamma_range u, beta_i =
  beta_range u), tag 0x57415250 for warm-start perturbations (x + sigma z).
* Start order at a depth: the lifted point (if kept), then the perturbed warm
  starts, then the random starts; start j is item j of its depth's optimiser
  batch, whose SPSA seed is seed + p 0x9E3779B97F4A7C15 (mod 2^64).  The final
  evaluation of start j at depth p uses shot stream 0xF000000000000000 +
  p 2^32 + j under the run's seed.
* Ranking with a reference (the brute-force optimum): best cost matches it,
  best index matches it, probability mass on its cost, probability of its
  index (all larger first); then best sampled cost (smaller first), mass on
  that cost, probability of the best index (larger first), mean cost
  (smaller first).  Without a reference the same sampled criteria, then the
  distribution gap mean - best (smaller first).  Remaining ties keep the
  earlier candidate.
"""
from __future__ import annotations

import math

import numpy as np

from . import sampling as osm

TAG_RAND = 0x52414E44
TAG_WARM = 0x57415250
FINAL_STREAM = 0xF000000000000000


def lift_interp(v) -> np.ndarray:
    """INTERP lifting of one angle sequence from depth p to p + 1."""
    v = np.asarray(v, dtype=np.float64)
    p = len(v)
    ext = np.concatenate([[0.0], v, [0.0]])
    return np.array([((i - 1) / p) * ext[i - 1] + ((p - i + 1) / p) * ext[i] for i in range(1, p + 2)])


def _words(seed, i, j, p, tag):
    return osm.philox4x32_10((i, j, p, tag), (seed & osm.M32, (seed >> 32) & osm.M32))


def uniform(seed, i, j, p, tag) -> float:
    w = _words(seed, i, j, p, tag)
    return ((w[0] | (w[1] << 32)) >> 11) * 2.0 ** -53


def normal(seed, i, j, p, tag) -> float:
    w = _words(seed, i, j, p, tag)
    u1 = ((w[0] | (w[1] << 32)) >> 11) * 2.0 ** -53
    u2 = ((w[2] | (w[3] << 32)) >> 11) * 2.0 ** -53
    return math.sqrt(-2.0 * math.log(1.0 - u1)) * math.cos(2.0 * math.pi * u2)


def initial_points(p: int, prev, seed: int, random_starts: int, warm_perturb: int, include_warm: bool,
                   warm_sigma: float, gamma_range: float, beta_range: float) -> list[np.ndarray]:
    """Interleaved x = [g1, b1, ...] of every start at depth p."""
    pts = []
    j = 0
    if prev is not None:
        g, b = lift_interp(prev[0::2]), lift_interp(prev[1::2])
        lifted = np.empty(2 * p)
        lifted[0::2], lifted[1::2] = g, b
        if include_warm:
            pts.append(lifted.copy())
            j += 1
        for _ in range(warm_perturb):
            pts.append(lifted + warm_sigma * np.array([normal(seed, i, j, p, TAG_WARM) for i in range(2 * p)]))
            j += 1
    for _ in range(random_starts):
        x = np.array([uniform(seed, i, j, p, TAG_RAND) for i in range(2 * p)])
        x[0::2] *= gamma_range
        x[1::2] *= beta_range
        pts.append(x)
        j += 1
    return pts


def rank_key(m: dict, use_reference: bool):
    """Lexicographic key of a candidate's metrics (smaller ranks first)."""
    sampled = (m["best_cost"], -m["p_best_cost"], -m["p_best_index"], m["mean_cost"])
    if use_reference:
        return (-int(m["best_cost_matches_ref"]), -int(m["best_index_matches_ref"]), -m["p_ref_cost"],
                -m["p_ref_index"]) + sampled
    return sampled + (m["mean_cost"] - m["best_cost"],)


def best_of(metrics: list[dict], use_reference: bool) -> int:
    """Index of the best candidate (the earliest among equal keys)."""
    keys = [rank_key(m, use_reference) for m in metrics]
    return min(range(len(keys)), key=lambda k: (keys[k], k))


def depth_seed(seed: int, p: int) -> int:
    return (seed + p * 0x9E3779B97F4A7C15) & ((1 << 64) - 1)


def _optimise(F, x0: np.ndarray, o: dict, j: int, seed: int) -> np.ndarray:
    """Run the configured optimiser from x0 (start j of its depth's batch)."""
    import oracle

    if o["optimizer"] == "adam":
        x = np.array(x0, dtype=np.float64)
        m = np.zeros_like(x)
        v = np.zeros_like(x)
        for t in range(1, o["iterations"] + 1):
            _, dg, db = oracle.grad_adjoint(F, x[0::2], x[1::2])
            g = np.empty_like(x)
            g[0::2], g[1::2] = dg, db
            x, m, v = osm.adam_step(x, g, m, v, t, o["lr"], o["beta1"], o["beta2"], o["eps"])
        return x

    def J(x, k, which):
        psi = oracle.evolve(F, x[0::2], x[1::2])
        if o["shots"] == 0:
            return oracle.expectation(F, psi)
        tot = 0.0
        for a in range(o["averaging"]):
            stream = (k << 32) | (j << 10) | (which << 9) | a
            tot += osm.sampled_mean(F, osm.sample(psi, osm.shot_randoms(seed, stream, o["shots"])))
        return tot / o["averaging"]

    x, _ = osm.spsa_adam(J, x0, o["iterations"], seed, b=j, c=o["c"], decay=o["c_decay"], lr=o["lr"],
                         b1=o["beta1"], b2=o["beta2"], eps=o["eps"])
    return x


def solve(F: np.ndarray, o: dict) -> dict:
    """Algorithm 1 on the objective table F with options o (keys as in the
    library's qaoa_solve_options).  Returns the selected depth, parameters,
    final metrics, and each depth's representative."""
    import oracle

    ref_cost = float(F.min()) if o["use_reference"] else None
    ref_index = oracle.argmin(F) if o["use_reference"] else None
    prev = None
    reps = []
    for p in range(1, o["p_max"] + 1):
        pts = initial_points(p, prev, o["seed"], o["random_starts"], o["warm_perturb"], o["include_warm"],
                             o["warm_sigma"], o["gamma_range"], o["beta_range"])
        cands = []
        for j, x0 in enumerate(pts):
            x = _optimise(F, x0, o, j, depth_seed(o["seed"], p))
            psi = oracle.evolve(F, x[0::2], x[1::2])
            idx = osm.sample(psi, osm.shot_randoms(o["seed"], FINAL_STREAM + (p << 32) + j, o["final_shots"]))
            m = osm.metrics(F, idx, o["margin"], o["elite"], ref_cost=ref_cost, ref_index=ref_index, tol=o["tol"])
            cands.append((x, m))
        k = best_of([c[1] for c in cands], o["use_reference"])
        reps.append({"p": p, "x": cands[k][0], "metrics": cands[k][1], "start": k, "starts": len(pts)})
        prev = cands[k][0]
    k = best_of([r["metrics"] for r in reps], o["use_reference"])
    return {"best_p": reps[k]["p"], "x": reps[k]["x"], "metrics": reps[k]["metrics"], "reps": reps}
