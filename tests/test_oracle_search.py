"""Pins for the Algorithm 1 oracle (oracle/search.py): INTERP lifting against
hand-derived lifts, the Philox uniforms and normals against their moments, the
candidate ranking against hand-ordered candidates, and the composed search on
a tiny instance against brute force.  CPU only."""
import math

import numpy as np
import pytest

import oracle
from oracle import search as osr
from paper_2606_26297_b300 import instances as inst


def test_interp_hand_derived():
    """p=1: [a] -> [a, a]; p=2: [a, b] -> [a, (a+b)/2, b];
    p=3: [a, b, c] -> [a, a/3 + 2b/3, 2b/3 + c/3, c]."""
    a, b, c = 0.3, -0.7, 1.9
    assert np.allclose(osr.lift_interp([a]), [a, a])
    assert np.allclose(osr.lift_interp([a, b]), [a, (a + b) / 2, b])
    assert np.allclose(osr.lift_interp([a, b, c]), [a, a / 3 + 2 * b / 3, 2 * b / 3 + c / 3, c])


def test_interp_keeps_linear_schedules():
    """A linear ramp sampled at the midpoints (i - 1/2)/p stays a linear ramp
    through its endpoints' line at depth p + 1 (INTERP is linear
    interpolation of the piecewise-linear schedule)."""
    p = 5
    v = np.array([(i - 0.5) / p for i in range(1, p + 1)])
    w = osr.lift_interp(v)
    assert np.allclose(np.diff(w[1:-1]), np.diff(w[1:-1])[0])


def test_uniform_normal_moments():
    us = np.array([osr.uniform(7, i, j, 1, osr.TAG_RAND) for i in range(40) for j in range(50)])
    zs = np.array([osr.normal(7, i, j, 2, osr.TAG_WARM) for i in range(40) for j in range(50)])
    assert us.min() >= 0.0 and us.max() < 1.0
    assert abs(us.mean() - 0.5) < 5 * math.sqrt(1 / 12 / len(us))
    assert abs(zs.mean()) < 5 / math.sqrt(len(zs))
    assert abs(zs.var() - 1.0) < 5 * math.sqrt(2 / len(zs))


def _m(best, pbc, pbi, mean, mref=0, iref=0, pref=0.0, pidx=0.0):
    return {"best_cost": best, "p_best_cost": pbc, "p_best_index": pbi, "mean_cost": mean,
            "best_cost_matches_ref": mref, "best_index_matches_ref": iref, "p_ref_cost": pref,
            "p_ref_index": pidx}


def test_ranking_hand_ordered():
    """Sec. 3.5 ranking on hand-made candidates, with and without a reference."""
    c = [_m(-3.0, 0.2, 0.1, -1.0), _m(-4.0, 0.1, 0.1, -0.5), _m(-4.0, 0.3, 0.1, 0.0), _m(-4.0, 0.3, 0.2, 5.0),
         _m(-4.0, 0.3, 0.2, 4.0)]
    order = sorted(range(len(c)), key=lambda k: (osr.rank_key(c[k], False), k))
    assert order == [4, 3, 2, 1, 0]
    assert osr.best_of(c, False) == 4
    r = [_m(-4.0, 0.5, 0.5, -3.0, 0, 0), _m(-3.0, 0.1, 0.1, 0.0, 1, 0, 0.1, 0.0),
         _m(-3.0, 0.1, 0.1, 0.0, 1, 1, 0.1, 0.05), _m(-3.0, 0.1, 0.1, 0.0, 1, 1, 0.2, 0.01)]
    assert osr.best_of(r, True) == 3
    assert osr.best_of(r[:3], True) == 2
    assert osr.best_of([r[0], r[0]], True) == 0


def test_initial_points_layout():
    """Depth 1 has the random starts only; later depths the lifted point,
    its perturbations and the random starts, in that order."""
    pts = osr.initial_points(1, None, 3, 2, 4, True, 0.1, 0.5, 1.5)
    assert len(pts) == 2 and all(len(x) == 2 for x in pts)
    assert all(0 <= x[0] < 0.5 and 0 <= x[1] < 1.5 for x in pts)
    prev = np.array([0.2, 0.6])
    pts = osr.initial_points(2, prev, 3, 1, 2, True, 0.1, 0.5, 1.5)
    assert len(pts) == 4
    assert np.allclose(pts[0], [0.2, 0.6, 0.2, 0.6])
    assert not np.allclose(pts[1], pts[0]) and np.max(np.abs(pts[1] - pts[0])) < 1.0


def test_solve_finds_brute_force_optimum_tiny():
    """Algorithm 1 with exact-gradient Adam on a 5-variable QUBO: the selected
    candidate's best sampled cost is the brute-force minimum (the final shots
    cover every bitstring with non-negligible probability), and each depth's
    representative is the best of its own candidates."""
    Q = inst.upper_int_qubo(5, 77)
    F = oracle.cost_table(oracle.canonical_of(Q))
    o = dict(p_max=2, optimizer="adam", iterations=20, shots=0, averaging=1, random_starts=2, warm_perturb=1,
             include_warm=True, final_shots=2000, elite=4, use_reference=True, lr=0.05, beta1=0.9, beta2=0.999,
             eps=1e-8, c=0.1, c_decay=0.101, warm_sigma=0.05, gamma_range=0.3, beta_range=1.0, margin=0.0,
             tol=1e-9, seed=11)
    r = osr.solve(F, o)
    assert r["metrics"]["best_cost"] == F.min()
    assert [rep["starts"] for rep in r["reps"]] == [2, 4]
    assert r["best_p"] in (1, 2)
