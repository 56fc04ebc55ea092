"""Checks of the seeded input generator (no EDAA arithmetic lives there)."""
import numpy as np

from paper_2209_11002_gb300 import synth


def test_cube_shapes_and_recipe():
    c = synth.make_cube(40, 5000, 4, alpha=0.3, snr_db=25.0, pure=True, M=6,
                        gamma_choices=(0.5, 1.0, 2.0), seed=7)
    assert c.X.shape == (40, 5000) and c.X.dtype == np.float32
    assert c.E_true.min() >= 0.0 and np.allclose(c.E_true.max(0), 1.0) and np.allclose(c.E_true.min(0), 0.0)
    assert np.allclose(c.A_true.sum(0), 1.0)
    assert np.allclose(c.A_true[:, :4], np.eye(4))
    # Dirichlet(alpha * 1) has mean 1/p per component
    assert np.abs(c.A_true[:, 4:].mean(1) - 0.25).max() < 0.02
    # realised SNR within 0.1 dB of the request
    Y = c.E_true @ c.A_true
    noise = c.X.astype(np.float64) - Y
    snr = 10 * np.log10((Y * Y).sum() / (noise * noise).sum())
    assert abs(snr - 25.0) < 0.1
    assert c.seeds.dtype == np.uint64 and len(set(c.seeds.tolist())) == 6
    assert set(c.gammas.tolist()) <= {0.5, 1.0, 2.0}


def test_determinism_and_uneven_batch():
    a = synth.make_cube(10, 100, 3, seed=3)
    b = synth.make_cube(10, 100, 3, seed=3)
    assert np.array_equal(a.X, b.X)
    cubes = synth.uneven_batch()
    assert len(cubes) == 8
    for c in cubes:
        assert c.L in (156, 162, 188, 198, 224, 285)
        assert 9000 <= c.N <= 94249 and 3 <= c.p <= 6 and c.M == 16
