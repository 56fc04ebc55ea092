"""CPU check of the near-tie detector the GPU parity tests use to decide when
the GPU's Algorithm 2 choice may differ from the oracle's (Algorithm 2: the
candidate set is every run with fit <= 1.05 min fit; the pick is the lowest
coherence among them)."""
import numpy as np
import pytest

from selection_check import check_selection, selection_near_tie


def test_clear_choice_is_not_a_tie():
    fit = [10.0, 10.2, 12.0, 15.0]   # threshold 10.5: runs 0, 1 are candidates
    mu = [0.9, 0.5, 0.1, 0.0]
    assert not selection_near_tie(fit, mu)


def test_fit_at_the_threshold_is_a_tie():
    fit = [10.0, 10.5 * (1 + 5e-4), 12.0]   # run 1 sits within 1e-3 of 1.05 min fit
    assert selection_near_tie(fit, [0.9, 0.1, 0.0])


def test_equal_coherence_candidates_are_a_tie():
    assert selection_near_tie([10.0, 10.1], [0.5001, 0.5004])


def test_check_selection_accepts_ties_and_rejects_real_disagreements():
    fit, mu = np.array([10.0, 10.2, 12.0]), np.array([0.9, 0.5, 0.1])
    check_selection(1, fit, mu, fit, mu)
    with pytest.raises(AssertionError):  # not Algorithm 2 on the GPU's own vectors
        check_selection(0, fit, mu, fit, mu)
    ref_fit = np.array([10.0, 10.6, 12.0])  # oracle keeps run 1 out of the candidate set: a real disagreement
    with pytest.raises(AssertionError):
        check_selection(1, fit, mu, ref_fit, mu)
