"""GPU parity: the CUDA library through the C ABI against the FP64 oracle, on
the same seeded inputs.

Tolerances (FP32 path against the FP64 oracle):
  * gradients at each outer-iteration boundary t <= 3: norm-wise relative
    error <= 1e-5;
  * after a full solve: |loss - loss_ref| / loss_ref <= 1e-3 and
    max |A - A_ref| <= 1e-3;
  * initial state: step sizes within 1e-5 relative, B^0 within 1e-6 of the
    oracle's entries (relative to 1/N), A^0 = 1/p to float rounding.
"""
import numpy as np
import pytest

from oracle import edaa_oracle as O
from paper_2209_11002_gb300 import build, edaa, synth
from selection_check import check_selection as _check_selection

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()
    edaa.load_library()


def _ctx(cubes, **cfg):
    return edaa.Context([dict(X=c.pixel_major(), p=c.p, seeds=c.seeds, gammas=c.gammas) for c in cubes], **cfg)


def _oracle(cube, m, T, K1=5, K2=5, record=False):
    X = O.normalize_pixels(cube.X)
    return O.edaa(X, cube.p, T, K1, K2, int(cube.seeds[m]), float(cube.gammas[m]), record=record)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def test_initial_state_matches_oracle():
    cube = synth.make_cube(37, 1531, 3, M=4, gamma_choices=(0.5, 1.0, 2.0), seed=5)
    with _ctx([cube], T=0) as ctx:
        e1, e2 = ctx.step_sizes(0)
        X = O.normalize_pixels(cube.X)
        for m in range(cube.M):
            B0 = O.init_B(O.uniform_u(int(cube.seeds[m]), cube.N, cube.p))
            r1, r2 = O.step_sizes(X, B0, float(cube.gammas[m]))
            assert abs(e1[m] - r1) <= 1e-5 * r1
            assert abs(e2[m] - r2) <= 1e-5 * r2
            E, A, B = ctx.get(0, m, device="cpu")
            assert np.abs(A - 1.0 / cube.p).max() < 1e-7
            assert np.abs(B - B0).max() * cube.N < 1e-5
            assert np.abs(E - X @ B0).max() < 1e-5


@pytest.mark.parametrize("persistent,tile", [(1, None), (0, None), (1, (3, 1, 4, 1)), (0, (3, 1, 4, 2)),
                                             (1, (3, 2, 2, 2)), (1, (2, 4, 1, 8))])
def test_gradients_per_outer_iteration(persistent, tile):
    """grad_A and grad_B (the 2(...) gradients of eqs. update_A / update_B) at
    every outer-iteration boundary t = 0..3, norm-wise relative error <= 1e-5,
    for the built-in launch shape and for explicit ones: four pixels per
    lane, two pixels x two runs, one pixel per lane (ragged last tiles: 2333
    pixels in tiles of 32 and 128)."""
    cube = synth.make_cube(48, 2333, 4, alpha=0.5, snr_db=30, M=3, gamma_choices=(0.5, 1.0, 2.0), seed=6)
    refs = [_oracle(cube, m, 3, record=True)["hist"] for m in range(cube.M)]
    errs = {}
    kw = {} if tile is None else dict(tile=tile)
    with _ctx([cube], T=3, persistent=persistent, **kw) as ctx:
        assert tile is None or ctx.describe(0)["tile"] == tile
        for t in range(4):
            for m in range(cube.M):
                gA, gB = ctx.grad(0, m, device="cpu")
                errs[(t, m)] = (_rel(gA, refs[m]["gA"][t]), _rel(gB, refs[m]["gB"][t]))
            if t < 3:
                ctx.step(1)
    for k, v in sorted(errs.items()):
        print("t=%d run=%d  grad_A rel %.2e  grad_B rel %.2e" % (k[0], k[1], v[0], v[1]))
    assert max(max(v) for v in errs.values()) <= 1e-5


@pytest.mark.parametrize("tile", [None, (2, 1, 4, 1)])
def test_large_step_factors_urban_shape(tile):
    """gamma = 8 and 4, the top of the step-factor set S, on the Urban-shaped
    cube (L=162, N=94249, p=6).  One B-step there moves whole columns of
    logits by tens of nats, to maxima well below zero, so the shifted
    accumulation has to take its reference below the column's mean weight.
    The loss at every outer boundary t <= 3 within 1e-4 of the oracle, and
    A, E within 1e-3 at t = 3; built-in launch shape and four pixels per lane."""
    cube = synth.workload(synth.URBAN_PRECISION, M=2)
    cube.gammas = np.array([8.0, 4.0])
    T = 3
    refs = [_oracle(cube, m, T, record=True) for m in range(2)]
    kw = {} if tile is None else dict(tile=tile)
    with _ctx([cube], T=T, **kw) as ctx:
        for t in range(T + 1):
            loss = ctx.loss(0)
            for m in range(2):
                lr = refs[m]["hist"]["loss"][t]
                assert np.isfinite(loss[m]) and abs(loss[m] - lr) / lr <= 1e-4, (t, m, loss[m], lr)
            if t < T:
                ctx.step(1)
        for m in range(2):
            E, A, B = ctx.get(0, m, device="cpu")
            assert np.abs(A - refs[m]["A"]).max() <= 1e-3
            assert np.abs(E - refs[m]["E"]).max() <= 1e-3


def test_centring_is_an_exact_reparametrisation():
    """Running on X minus its mean pixel leaves EDAA's iterates unchanged."""
    cube = synth.make_cube(40, 1800, 4, alpha=0.4, snr_db=25, M=3, gamma_choices=(0.5, 1.0, 2.0), seed=20)
    outs = []
    for center in (1, 0):
        with _ctx([cube], T=10, center=center) as ctx:
            ctx.solve()
            outs.append([ctx.get(0, m, device="cpu") for m in range(cube.M)] + [ctx.loss(0)])
    for m in range(cube.M):
        for a, b in zip(outs[0][m], outs[1][m]):
            assert np.abs(a - b).max() <= 1e-4 * max(1.0, np.abs(b).max())
    assert np.allclose(outs[0][-1], outs[1][-1], rtol=1e-4)


def test_full_solve_single_run_samson_shape():
    """Full-size plain run (L=156, N=9025, p=3, M=1, gamma=1, T=100)."""
    cube = synth.workload(synth.SAMSON_EDAA)
    ref = _oracle(cube, 0, 100)
    Xn = O.normalize_pixels(cube.X)
    loss_ref = O.objective(Xn, ref["A"], ref["B"])
    with _ctx([cube], T=100) as ctx:
        ctx.solve()
        best, fit, mu = ctx.select(0)
        loss = ctx.loss(0)[0]
        E, A, B = ctx.get(0, 0, device="cpu")
    assert best == 0
    assert abs(loss - loss_ref) / loss_ref <= 1e-3
    assert np.abs(A - ref["A"]).max() <= 1e-3
    assert abs(fit[0] - O.fit_l1(Xn, ref["E"], ref["A"])) / fit[0] <= 1e-3
    assert abs(mu[0] - O.coherence(ref["E"])) <= 1e-3


def test_ensemble_select_and_runs():
    cube = synth.make_cube(40, 2500, 4, alpha=0.3, snr_db=25, M=6, gamma_choices=(0.5, 1.0, 2.0), seed=7)
    T = 20
    Xn = O.normalize_pixels(cube.X)
    refs = [_oracle(cube, m, T) for m in range(cube.M)]
    ref_fit = [O.fit_l1(Xn, r["E"], r["A"]) for r in refs]
    ref_mu = [O.coherence(r["E"]) for r in refs]
    with _ctx([cube], T=T) as ctx:
        ctx.solve()
        best, fit, mu = ctx.select(0)
        loss = ctx.loss(0)
        for m in range(cube.M):
            E, A, B = ctx.get(0, m, device="cpu")
            assert np.abs(A - refs[m]["A"]).max() <= 1e-3
            assert np.abs(E - refs[m]["E"]).max() <= 1e-3
            lr = O.objective(Xn, refs[m]["A"], refs[m]["B"])
            assert abs(loss[m] - lr) / lr <= 1e-3
    assert np.allclose(fit, ref_fit, rtol=1e-3)
    assert np.allclose(mu, ref_mu, atol=1e-3)
    _check_selection(best, fit, mu, ref_fit, ref_mu)


def test_uneven_batch_matches_single_cube_oracles():
    cubes = [synth.make_cube(33, 1111, 3, M=2, gamma_choices=(0.5, 1.0), seed=11),
             synth.make_cube(61, 1700, 5, M=3, gamma_choices=(1.0, 2.0), seed=12),
             synth.make_cube(20, 640, 2, M=1, seed=13)]
    T = 8
    with _ctx(cubes, T=T) as ctx:
        ctx.solve()
        for ci, cube in enumerate(cubes):
            Xn = O.normalize_pixels(cube.X)
            loss = ctx.loss(ci)
            for m in range(cube.M):
                ref = _oracle(cube, m, T)
                E, A, B = ctx.get(ci, m, device="cpu")
                assert np.abs(A - ref["A"]).max() <= 1e-3, (ci, m)
                assert np.abs(B - ref["B"]).max() <= 1e-3 * ref["B"].max() + 1e-6
                lr = O.objective(Xn, ref["A"], ref["B"])
                assert abs(loss[m] - lr) / lr <= 1e-3


def test_persistent_and_per_phase_launches_agree_bitwise():
    cube = synth.make_cube(29, 1999, 3, M=5, gamma_choices=(0.5, 1.0, 2.0), seed=14)
    outs = []
    for persistent in (1, 0):
        with _ctx([cube], T=6, persistent=persistent) as ctx:
            ctx.solve()
            best, fit, mu = ctx.select(0)
            outs.append((best, fit, mu, [ctx.get(0, m, device="cpu") for m in range(cube.M)]))
    assert outs[0][0] == outs[1][0]
    assert np.array_equal(outs[0][1], outs[1][1]) and np.array_equal(outs[0][2], outs[1][2])
    for a, b in zip(outs[0][3], outs[1][3]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_reset_reproduces_solve():
    cube = synth.make_cube(25, 900, 3, M=3, gamma_choices=(0.5, 1.0, 2.0), seed=15)
    with _ctx([cube], T=5) as ctx:
        assert ctx.describe(0)["graph"] == 0
        ctx.solve()
        assert ctx.describe(0)["graph"] == 1  # the solve replayed its captured CUDA graph
        r1 = ctx.select(0)
        A1 = ctx.get(0, 1, device="cpu")[1]
        ctx.reset()
        assert ctx.outer_done() == 0
        ctx.solve()
        r2 = ctx.select(0)
        A2 = ctx.get(0, 1, device="cpu")[1]
    assert r1[0] == r2[0] and np.array_equal(r1[1], r2[1]) and np.array_equal(A1, A2)


@pytest.mark.parametrize("shape", [(5, 3, 1, 2), (1, 50, 2, 1), (17, 33, 8, 2), (319, 77, 4, 1),
                                   (12, 257, 7, 3), (9, 4, 4, 2)])
def test_edge_shapes(shape):
    """p = 1, L = 1, p = 8, L at the compiled maximum, ragged tiles, N = p."""
    L, N, p, M = shape
    cube = synth.make_cube(L, N, p, alpha=0.7, snr_db=30, M=M, gamma_choices=(0.5, 1.0), seed=16 + L)
    T = 4
    with _ctx([cube], T=T) as ctx:
        ctx.solve()
        for m in range(M):
            ref = _oracle(cube, m, T)
            E, A, B = ctx.get(0, m, device="cpu")
            assert np.abs(A - ref["A"]).max() <= 1e-3
            assert np.abs(B.sum(0) - 1).max() < 1e-4 and np.abs(A.sum(0) - 1).max() < 1e-5
            assert np.abs(E - ref["E"]).max() <= 1e-3


def test_k_zero_and_zero_pixel():
    cube = synth.make_cube(30, 500, 3, M=2, gamma_choices=(1.0,), seed=17)
    cube.X[:, 7] = 0.0  # a zero pixel stays zero under normalisation
    for K1, K2 in [(0, 3), (3, 0), (1, 1)]:
        with _ctx([cube], T=3, K1=K1, K2=K2) as ctx:
            ctx.solve()
            for m in range(2):
                ref = _oracle(cube, m, 3, K1, K2)
                E, A, B = ctx.get(0, m, device="cpu")
                assert np.abs(A - ref["A"]).max() <= 1e-4
                assert np.abs(E - ref["E"]).max() <= 1e-4


def test_no_normalisation_flag():
    cube = synth.make_cube(22, 300, 3, alpha=1.0, snr_db=None, pure=True, M=1, seed=18)
    with _ctx([cube], T=10, normalize=0) as ctx:
        ctx.solve()
        E, A, B = ctx.get(0, 0, device="cpu")
    ref = O.edaa(cube.X.astype(np.float64), 3, 10, 5, 5, int(cube.seeds[0]), 1.0)
    assert np.abs(A - ref["A"]).max() <= 1e-3 and np.abs(E - ref["E"]).max() <= 1e-3


def test_nan_input_is_reported_not_crashing():
    cube = synth.make_cube(20, 300, 3, M=2, seed=19)
    cube.X[3, 11] = np.nan
    with _ctx([cube], T=2) as ctx:
        ctx.solve()
        with pytest.raises(edaa.EDAAError) as ei:
            ctx.select(0)
        assert ei.value.status == edaa.EDAA_ERR_NONFINITE


def test_barrier_timeout_returns_status():
    """A grid barrier that can never complete (one arrival short) gives up after
    its time limit and reports EDAA_ERR_TIMEOUT; the device stays usable."""
    assert edaa.selftest_barrier(8, 0, 1000.0) == edaa.EDAA_OK
    assert edaa.selftest_barrier(8, 1, 50.0) == edaa.EDAA_ERR_TIMEOUT
    assert edaa.selftest_barrier(8, 0, 1000.0) == edaa.EDAA_OK


def test_jasper_shape_ensemble_sampled_runs():
    """Full-size ensemble (L=198, N=10000, p=4, M=50, T=100) in the launch
    configuration the benchmark times; three sampled runs against the oracle."""
    cube = synth.workload(synth.JASPER_ENSEMBLE)
    with _ctx([cube], T=100) as ctx:
        ctx.solve()
        best, fit, mu = ctx.select(0)
        loss = ctx.loss(0)
        Xn = O.normalize_pixels(cube.X)
        for m in (0, 17, 49):
            ref = _oracle(cube, m, 100)
            E, A, B = ctx.get(0, m, device="cpu")
            lr = O.objective(Xn, ref["A"], ref["B"])
            assert abs(loss[m] - lr) / lr <= 1e-3, (m, loss[m], lr)
            assert np.abs(A - ref["A"]).max() <= 1e-3
            assert abs(fit[m] - O.fit_l1(Xn, ref["E"], ref["A"])) / fit[m] <= 1e-3
            assert abs(mu[m] - O.coherence(ref["E"])) <= 1e-3
    # Algorithm 2 on the GPU's own 50 fits and coherences, as the oracle states it
    assert np.all(np.isfinite(fit)) and best == O.select(fit, mu)


def test_autotuned_launch_shape_keeps_results():
    """The autotuner times candidate tile shapes at init and keeps the fastest;
    whatever it picks, the result must still match the oracle."""
    cube = synth.make_cube(44, 3000, 4, alpha=0.3, snr_db=25, M=10, gamma_choices=(0.5, 1.0, 2.0), seed=21)
    T = 5
    with _ctx([cube], T=T, autotune=1) as ctx:
        shape = ctx.describe(0)
        ctx.solve()
        loss = ctx.loss(0)
        Xn = O.normalize_pixels(cube.X)
        for m in (0, 9):
            ref = _oracle(cube, m, T)
            E, A, B = ctx.get(0, m, device="cpu")
            assert np.abs(A - ref["A"]).max() <= 1e-3
            lr = O.objective(Xn, ref["A"], ref["B"])
            assert abs(loss[m] - lr) / lr <= 1e-3
    assert shape["runs_per_group"] >= 1 and shape["pixel_tile"] in (32, 64, 128)
