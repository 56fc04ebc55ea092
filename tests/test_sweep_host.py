"""Host logic of the sweep harness (no GPU): the studies cover the paper's
ablation axes (Sec. IV-E) -- a fixed budget of T (K1 + K2) = 1000 updates
split between the inner and outer loops, T at K1 = K2 = 5, and the ensemble
size M."""
import pytest

from paper_2209_11002_gb300 import sweep


def test_kkt_points_keep_the_update_budget():
    pts = sweep.study_points("kkt")
    assert len(pts) >= 5
    assert all(p["T"] * (p["K1"] + p["K2"]) == 1000 for p in pts)
    assert {"K1": 5, "K2": 5, "T": 100} in pts  # the paper's default (Sec. III-C)


def test_t_and_m_points():
    assert [p["T"] for p in sweep.study_points("t")] == [10, 25, 50, 100, 200]
    assert [p["M"] for p in sweep.study_points("m")] == [10, 20, 50, 100]
    with pytest.raises(ValueError):
        sweep.study_points("nope")


def test_cubes_carry_ground_truth():
    cube = sweep.make_cube("jasper", 7, 4, (0.5, 1.0))
    assert cube.E_true.shape == (cube.L, cube.p) and cube.A_true.shape == (cube.p, cube.N)
    assert cube.M == 4 and set(cube.gammas) <= {0.5, 1.0}
