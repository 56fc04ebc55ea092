"""Algorithm 2 checks shared by the GPU parity tests (test helpers, no GPU).

The GPU path computes every run's fit and coherence in FP32/FP64; the oracle
in FP64.  Within the parity tolerances the two can disagree on Algorithm 2's
choice only where the choice itself is fragile: a run whose fit sits at the
threshold 1.05 * min fit, or two candidates of near-equal coherence.  These
helpers make that precise."""
import numpy as np

from oracle import edaa_oracle as O


def selection_near_tie(fit, mu, ratio=1.05, fit_rtol=1e-3, mu_atol=1e-3):
    """True when Algorithm 2's choice on (fit, mu) could flip under errors of
    the size the parity tests allow: a run whose fit lies within fit_rtol of
    the threshold ratio * min fit (its membership in the candidate set is
    undecided), or two candidates whose coherences differ by at most 2 mu_atol."""
    fit = np.asarray(fit, np.float64)
    mu = np.asarray(mu, np.float64)
    thr = ratio * fit[np.isfinite(fit)].min()
    if np.any(np.abs(fit - thr) <= 2 * fit_rtol * thr):
        return True
    cand = np.sort(mu[fit <= thr])
    return cand.size > 1 and cand[1] - cand[0] <= 2 * mu_atol


def check_selection(best, fit, mu, ref_fit, ref_mu):
    """The GPU's index is Algorithm 2 applied to the GPU's own fit and mu, and
    equals the oracle's choice unless either side sits at a near tie."""
    assert best == O.select(fit, mu), (best, O.select(fit, mu))
    ref_best = O.select(ref_fit, ref_mu)
    if best != ref_best:
        tie = selection_near_tie(fit, mu) or selection_near_tie(ref_fit, ref_mu)
        print("selection differs from the oracle's (%d vs %d); near tie: %s" % (best, ref_best, tie))
        assert tie, (best, ref_best, list(fit), list(ref_fit))
