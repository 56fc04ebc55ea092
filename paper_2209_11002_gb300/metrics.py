"""Accuracy of an unmixing against synthetic ground truth (Sec. IV-B).

Host-side evaluation, not part of the solve: the abundance RMSE of eq. (RMSE)
and the spectral angle distance of eq. (SAD), after matching the estimated
endmembers to the true ones.  The paper compares a method's endmember i with
true endmember i; an unsupervised method returns its endmembers in an
arbitrary order, so the estimated columns are first permuted to the order
that minimises the mean spectral angle (an assignment problem on the p x p
matrix of angles), and the abundance rows follow the same permutation.
"""
from __future__ import annotations

import itertools
from typing import Dict, Sequence

import numpy as np


def spectral_angles(E: np.ndarray, E_hat: np.ndarray) -> np.ndarray:
    """p x p matrix of angles (radians) between column i of E and column j of
    E_hat: arccos(<e_i, e^_j> / (||e_i|| ||e^_j||)), the summand of eq. (SAD)."""
    E = np.asarray(E, np.float64)
    F = np.asarray(E_hat, np.float64)
    ne = np.linalg.norm(E, axis=0)
    nf = np.linalg.norm(F, axis=0)
    with np.errstate(invalid="ignore", divide="ignore"):
        c = (E.T @ F) / np.outer(ne, nf)
    c = np.where(np.isfinite(c), c, 0.0)
    return np.arccos(np.clip(c, -1.0, 1.0))


def match_endmembers(E: np.ndarray, E_hat: np.ndarray) -> np.ndarray:
    """perm such that E_hat[:, perm[i]] is matched to E[:, i], minimising the
    mean angle.  Exhaustive over permutations for p <= 8 (at most 40,320),
    else the Hungarian method (scipy)."""
    ang = spectral_angles(E, E_hat)
    p = ang.shape[0]
    if p <= 8:
        best, best_cost = None, np.inf
        rows = np.arange(p)
        for perm in itertools.permutations(range(p)):
            cost = ang[rows, list(perm)].sum()
            if cost < best_cost - 1e-15:
                best, best_cost = perm, cost
        return np.asarray(best, dtype=np.int64)
    from scipy.optimize import linear_sum_assignment
    r, c = linear_sum_assignment(ang)
    return c[np.argsort(r)]


def sad_degrees(E: np.ndarray, E_hat: np.ndarray) -> float:
    """Eq. (SAD): mean spectral angle between matched columns, in degrees
    (E_hat already in the matched order)."""
    ang = spectral_angles(E, E_hat)
    return float(np.degrees(np.mean(np.diag(ang))))


def rmse_percent(A: np.ndarray, A_hat: np.ndarray) -> float:
    """Eq. (RMSE): 100 sqrt(1/(p N) sum_ij (A_ij - A^_ij)^2)."""
    A = np.asarray(A, np.float64)
    B = np.asarray(A_hat, np.float64)
    return float(100.0 * np.sqrt(np.mean((A - B) ** 2)))


def evaluate(E_true: np.ndarray, A_true: np.ndarray, E_hat: np.ndarray, A_hat: np.ndarray) -> Dict[str, object]:
    """Match E_hat's columns to E_true's, then SAD (degrees) and RMSE (%),
    globally and per endmember."""
    perm = match_endmembers(E_true, E_hat)
    Em = np.asarray(E_hat, np.float64)[:, perm]
    Am = np.asarray(A_hat, np.float64)[perm, :]
    ang = np.degrees(np.diag(spectral_angles(E_true, Em)))
    per_rmse = 100.0 * np.sqrt(np.mean((np.asarray(A_true, np.float64) - Am) ** 2, axis=1))
    return {"perm": perm.tolist(), "sad": float(ang.mean()), "rmse": rmse_percent(A_true, Am),
            "sad_per_endmember": ang.tolist(), "rmse_per_endmember": per_rmse.tolist()}


def selection_quality(rmse: Sequence[float], selected: int) -> Dict[str, object]:
    """How good Algorithm 2's pick is among the ensemble's runs: whether it is
    the run of lowest RMSE, its rank (0 = best), and its RMSE excess over the
    best run (regret)."""
    r = np.asarray(rmse, np.float64)
    order = np.argsort(r, kind="stable")
    return {"selected": int(selected), "best_rmse_run": int(order[0]), "selected_is_best": bool(order[0] == selected),
            "rank": int(np.nonzero(order == selected)[0][0]), "regret": float(r[selected] - r[order[0]])}
