"""Host-side logic of bench.py that needs no GPU."""
import math

import numpy as np

import bench


def test_matched_loss_counts_nonfinite_runs_and_uses_the_selected_run():
    l32 = np.array([10.0, 20.0, 30.0, 40.0])
    l = np.array([10.05, float("nan"), 30.0, 44.0])
    out = bench.matched_loss([l32], [0], [l], [0])
    assert math.isclose(out["selected_run_rel_loss_diff"], 0.005)
    assert out["same_selected_run"] and out["within_1pct"]
    assert out["runs_over_1pct"] == 2 and out["runs"] == 4  # the NaN run and the 10 % run
    assert math.isclose(out["median_run_rel_loss_diff"], 0.0525)


def test_matched_loss_reports_a_different_selection():
    out = bench.matched_loss([np.array([5.0, 4.0])], [1], [np.array([5.0, 4.5])], [0])
    assert not out["same_selected_run"]
    assert math.isclose(out["selected_run_rel_loss_diff"], 0.25) and not out["within_1pct"]
