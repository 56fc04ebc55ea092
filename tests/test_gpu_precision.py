"""Mixed-precision (tensor-core) ensemble path against the FP64 oracle and the
FP32 CUDA-core path.

The X-streaming contractions run on tcgen05 with TF32 or BF16 operands and
FP32 accumulation (M p >= 64); the softmax, the merges and the fit stay
FP32/FP64.  Stated errors against the oracle after 10 outer iterations
(measured: TF32 loss 1.6e-5, A 2.2e-5; BF16 loss 4.2e-5, A 1.1e-4):
  TF32: relative loss <= 2e-4, max |A - A_ref| <= 2e-4, max |E - E_ref| <= 2e-4
  BF16: relative loss <= 1e-3, max |A - A_ref| <= 1e-3, max |E - E_ref| <= 1e-3
and every run's final loss within 1 % of the same run in plain FP32."""
import numpy as np
import pytest

from oracle import edaa_oracle as O
from paper_2209_11002_gb300 import build, edaa, synth

pytestmark = pytest.mark.gpu

TOL = {edaa.TF32: 2e-4, edaa.BF16: 1e-3}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()
    edaa.load_library()


def _ctx(cube, **cfg):
    return edaa.Context([dict(X=cube.pixel_major(), p=cube.p, seeds=cube.seeds, gammas=cube.gammas)], **cfg)


@pytest.mark.parametrize("prec", [edaa.TF32, edaa.BF16])
@pytest.mark.parametrize("persistent", [1, 0])
def test_tensor_core_ensemble_against_oracle(prec, persistent):
    cube = synth.make_cube(64, 3001, 4, alpha=0.3, snr_db=25, M=16, gamma_choices=(0.5, 1.0, 2.0), seed=41)
    T = 10
    Xn = O.normalize_pixels(cube.X)
    with _ctx(cube, T=T, precision=prec, persistent=persistent) as ctx:
        shape = ctx.describe(0)
        ctx.solve()
        best, fit, mu = ctx.select(0)
        loss = ctx.loss(0)
        got = {m: ctx.get(0, m, device="cpu") for m in (0, 7, 15)}
    with _ctx(cube, T=T, precision=edaa.FP32) as ref32:
        ref32.solve()
        loss32 = ref32.loss(0)
    assert shape["pixel_tile"] == 128  # the tensor-core tiling
    tol = TOL[prec]
    for m, (E, A, B) in got.items():
        ref = O.edaa(Xn, 4, T, 5, 5, int(cube.seeds[m]), float(cube.gammas[m]))
        lr = O.objective(Xn, ref["A"], ref["B"])
        assert abs(loss[m] - lr) / lr <= tol
        assert np.abs(A - ref["A"]).max() <= tol
        assert np.abs(E - ref["E"]).max() <= tol
    assert np.max(np.abs(loss - loss32) / loss32) <= 0.01
    assert np.all(np.isfinite(fit)) and 0 <= best < 16


@pytest.mark.parametrize("runs", [8, 6, 4])
def test_tensor_core_run_groups_against_oracle(runs):
    """Smaller run groups (padded widths 32, 32 and 16 columns instead of 64;
    the autotuner's candidates) with BF16 operands: the same bars as the
    default grouping, and the same result with autotune = 1."""
    cube = synth.make_cube(64, 3001, 4, alpha=0.3, snr_db=25, M=16, gamma_choices=(0.5, 1.0, 2.0), seed=41)
    T = 10
    Xn = O.normalize_pixels(cube.X)
    with _ctx(cube, T=T, precision=edaa.BF16, tile=(runs, 1, 4, 1)) as ctx:
        assert ctx.describe(0)["runs_per_group"] == runs
        ctx.solve()
        loss = ctx.loss(0)
        got = {m: ctx.get(0, m, device="cpu") for m in (0, 7, 15)}
    for m, (E, A, B) in got.items():
        ref = O.edaa(Xn, 4, T, 5, 5, int(cube.seeds[m]), float(cube.gammas[m]))
        lr = O.objective(Xn, ref["A"], ref["B"])
        assert abs(loss[m] - lr) / lr <= TOL[edaa.BF16]
        assert np.abs(A - ref["A"]).max() <= TOL[edaa.BF16]
        assert np.abs(E - ref["E"]).max() <= TOL[edaa.BF16]
    with _ctx(cube, T=T, precision=edaa.BF16, autotune=1) as tuned:
        tuned.solve()
        assert np.max(np.abs(tuned.loss(0) - loss) / loss) <= 1e-3


def test_uneven_batch_mixes_tensor_core_and_cuda_core_cubes():
    """One launch where one cube is dense enough for tensor cores (M p = 64)
    and another is not (M p = 6): both against the oracle."""
    cubes = [synth.make_cube(48, 1500, 4, alpha=0.3, snr_db=25, M=16, gamma_choices=(0.5, 1.0), seed=51),
             synth.make_cube(30, 900, 3, alpha=0.5, snr_db=30, M=2, gamma_choices=(1.0,), seed=52)]
    T = 6
    with edaa.Context([dict(X=c.pixel_major(), p=c.p, seeds=c.seeds, gammas=c.gammas) for c in cubes], T=T,
                      precision=edaa.TF32) as ctx:
        ctx.solve()
        for ci, cube in enumerate(cubes):
            Xn = O.normalize_pixels(cube.X)
            loss = ctx.loss(ci)
            for m in (0, cube.M - 1):
                ref = O.edaa(Xn, cube.p, T, 5, 5, int(cube.seeds[m]), float(cube.gammas[m]))
                E, A, B = ctx.get(ci, m, device="cpu")
                assert np.abs(A - ref["A"]).max() <= 2e-4
                lr = O.objective(Xn, ref["A"], ref["B"])
                assert abs(loss[m] - lr) / lr <= 2e-4


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("persistent", [1, 0])
def test_split_tf32_gradients_per_outer_iteration(persistent):
    """EDAA_TF32X3 (operands split into two TF32 parts, three MMAs per
    product, element-wise steps in full FP32, tile accumulators folded into
    FP32 running sums): grad_A and grad_B at every outer boundary t = 0..3
    within 1e-5 (norm-wise relative) of the oracle on this 48-band,
    2333-pixel ensemble (M p = 64).  The split keeps about 22 of FP32's 24
    bits: on larger pixel counts its gradient error grows past the FP32
    path's (2.4e-5 at N = 40000, t = 2, against 2.8e-6)."""
    cube = synth.make_cube(48, 2333, 4, alpha=0.5, snr_db=30, M=16, gamma_choices=(0.5, 1.0, 2.0), seed=6)
    Xn = O.normalize_pixels(cube.X)
    runs = (0, 5, 15)
    refs = {m: O.edaa(Xn, 4, 3, 5, 5, int(cube.seeds[m]), float(cube.gammas[m]), record=True)["hist"] for m in runs}
    errs = {}
    with _ctx(cube, T=3, precision=edaa.TF32X3, persistent=persistent) as ctx:
        assert ctx.describe(0)["pixel_tile"] == 128  # the tensor-core tiling
        for t in range(4):
            for m in runs:
                gA, gB = ctx.grad(0, m, device="cpu")
                errs[(t, m)] = (_rel(gA, refs[m]["gA"][t]), _rel(gB, refs[m]["gB"][t]))
            if t < 3:
                ctx.step(1)
    for k, v in sorted(errs.items()):
        print("t=%d run=%d  grad_A rel %.2e  grad_B rel %.2e" % (k[0], k[1], v[0], v[1]))
    assert max(max(v) for v in errs.values()) <= 1e-5


def test_split_tf32_solve_against_oracle_and_fp32():
    """After 30 outer iterations: loss within 1e-3 relative and A, E within
    1e-3 max-abs of the oracle, and every run's loss within 1e-3 of the
    CUDA-core FP32 path."""
    cube = synth.make_cube(64, 3001, 4, alpha=0.3, snr_db=25, M=16, gamma_choices=(0.5, 1.0, 2.0), seed=43)
    T = 30
    Xn = O.normalize_pixels(cube.X)
    with _ctx(cube, T=T, precision=edaa.TF32X3) as ctx:
        ctx.solve()
        loss = ctx.loss(0)
        got = {m: ctx.get(0, m, device="cpu") for m in (0, 9, 15)}
    with _ctx(cube, T=T, precision=edaa.FP32) as ref32:
        ref32.solve()
        loss32 = ref32.loss(0)
    for m, (E, A, B) in got.items():
        ref = O.edaa(Xn, 4, T, 5, 5, int(cube.seeds[m]), float(cube.gammas[m]))
        lr = O.objective(Xn, ref["A"], ref["B"])
        assert abs(loss[m] - lr) / lr <= 1e-3
        assert np.abs(A - ref["A"]).max() <= 1e-3
        assert np.abs(E - ref["E"]).max() <= 1e-3
    assert np.max(np.abs(loss - loss32) / loss32) <= 1e-3
