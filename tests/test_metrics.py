"""CPU pins of the accuracy metrics of Sec. IV-B (eqs. RMSE, SAD) and of the
endmember matching they rest on: hand-computed values, a closed-form angle,
invariances, and the optimal assignment cross-checked with scipy's Hungarian
solver (an independent method)."""
import math

import numpy as np
import pytest

from paper_2209_11002_gb300 import metrics


def test_rmse_hand_cases():
    A = np.zeros((2, 3))
    assert metrics.rmse_percent(A, A) == 0.0
    assert math.isclose(metrics.rmse_percent(A, np.ones((2, 3))), 100.0)
    B = np.zeros((2, 3))
    B[0, 0] = 0.6  # one entry off by 0.6: 100 sqrt(0.36 / 6)
    assert math.isclose(metrics.rmse_percent(A, B), 100.0 * math.sqrt(0.36 / 6))


def test_sad_closed_forms():
    E = np.array([[1.0, 0.0], [0.0, 1.0]])
    assert metrics.sad_degrees(E, 3.0 * E) == pytest.approx(0.0, abs=1e-6)  # scale-invariant
    F = np.array([[1.0, 1.0], [math.sqrt(3.0), 0.0]])  # (1, sqrt 3): 60 degrees from e_1; (1, 0): 90 from e_2
    assert metrics.sad_degrees(E, F) == pytest.approx((60.0 + 90.0) / 2.0)
    assert metrics.spectral_angles(E, E[:, ::-1])[0, 0] == pytest.approx(math.pi / 2)


@pytest.mark.parametrize("seed", range(5))
def test_matching_recovers_a_shuffled_copy(seed):
    rng = np.random.default_rng(seed)
    L, p, N = 30, 5, 40
    E = rng.uniform(0.1, 1.0, (L, p))
    A = rng.dirichlet(np.ones(p), N).T
    perm = rng.permutation(p)
    E_hat = 2.5 * E[:, np.argsort(perm)] + 1e-3 * rng.standard_normal((L, p))  # column perm[i] holds E[:, i]
    A_hat = A[np.argsort(perm), :]
    out = metrics.evaluate(E, A, E_hat, A_hat)
    assert out["perm"] == perm.tolist()
    assert out["sad"] < 0.5 and out["rmse"] == pytest.approx(0.0, abs=1e-12)


@pytest.mark.parametrize("seed", range(8))
def test_matching_is_the_optimal_assignment(seed):
    scipy_opt = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(100 + seed)
    p = 2 + seed % 6
    E, F = rng.uniform(0.0, 1.0, (20, p)), rng.uniform(0.0, 1.0, (20, p))
    ang = metrics.spectral_angles(E, F)
    perm = metrics.match_endmembers(E, F)
    r, c = scipy_opt.linear_sum_assignment(ang)
    assert ang[np.arange(p), perm].sum() == pytest.approx(ang[r, c].sum(), rel=1e-12)


def test_selection_quality():
    q = metrics.selection_quality([3.0, 1.0, 2.0, 1.5], selected=2)
    assert q == {"selected": 2, "best_rmse_run": 1, "selected_is_best": False, "rank": 2, "regret": 1.0}
    assert metrics.selection_quality([1.0, 2.0], 0)["selected_is_best"]
