"""CPU checks of qaoa_sample_stats, the host-only entry point that turns
measured indices into the final distribution metrics of Sec. 3.6, against the
oracle's metrics (oracle/sampling.py, pinned in test_oracle_sampling.py).
No GPU is used."""
import math

import numpy as np
import pytest

from oracle import sampling as osm
from paper_2606_26297_b300 import build_lib


@pytest.fixture(scope="module")
def q():
    build_lib.build()
    from paper_2606_26297_b300 import qaoa
    return qaoa


@pytest.mark.parametrize("seed,ncand,shots", [(1, 5, 40), (2, 300, 5000), (3, 1, 7), (4, 4000, 3000)])
def test_stats_vs_oracle(q, seed, ncand, shots):
    rng = np.random.default_rng(seed)
    F = np.round(rng.standard_normal(ncand) * 4) / 2  # ties in cost
    idx = rng.integers(0, ncand, size=shots).astype(np.uint64)
    cost = F[idx.astype(np.int64)]
    ref_x = int(np.argmin(F))
    for margin, elite in [(0.0, 3), (1.0, 10), (2.5, 0)]:
        got = q.qaoa_sample_stats(idx, cost, margin=margin, elite=elite, ref_cost=float(F.min()), ref_index=ref_x)
        want = osm.metrics(F, idx, margin, elite, ref_cost=float(F.min()), ref_index=ref_x)
        for k in ["shots", "distinct", "best_index"]:
            assert got[k] == want[k], k
        for k in ["mean_cost", "best_cost", "p_best_index", "p_best_cost", "low_cost_mass", "p_ref_cost",
                  "p_ref_index"]:
            assert got[k] == pytest.approx(want[k], rel=1e-12, abs=1e-12), k
        assert bool(got["best_cost_matches_ref"]) == want["best_cost_matches_ref"]
        assert bool(got["best_index_matches_ref"]) == want["best_index_matches_ref"]
        assert [(a, b, c) for a, b, c, _ in got["elite"]] == [(a, b, c) for a, b, c, _ in want["elite"]]


def test_stats_without_reference_and_errors(q):
    got = q.qaoa_sample_stats(np.array([3, 3, 1], dtype=np.uint64), np.array([1.0, 1.0, -2.0]), elite=5)
    assert got["best_cost"] == -2.0 and got["best_index"] == 1
    assert math.isnan(got["p_ref_cost"]) and got["best_cost_matches_ref"] == -1
    assert got["elite"] == [(3, 1.0, 2, pytest.approx(2 / 3)), (1, -2.0, 1, pytest.approx(1 / 3))]
    with pytest.raises(q.QaoaError):
        q.qaoa_sample_stats(np.array([], dtype=np.uint64), np.array([]))
    with pytest.raises(q.QaoaError):
        q.qaoa_sample_stats(np.array([1], dtype=np.uint64), np.array([0.0]), margin=-1.0)
