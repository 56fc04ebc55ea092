"""Every precision mode against the FP64 oracle at the full sizes of the
precision-comparison workloads, after 10 outer iterations (Algorithm 1):

  * the Urban-shaped cube: L=162, N=307x307=94249, p=6, M=64 runs with step
    factors drawn from the paper's set S (eq. eta0A), sampled runs with
    gamma = 1/8, 1/2, 1, 2 and 8;
  * the largest cube the uneven-batch workload allows: L=285, N=94249,
    p=6, M=16 runs (step factors from S).

For each sampled run the test prints the relative loss error, the largest
abundance error max|A - A_ref|, the largest B error relative to the
uniform weight (N max|B - B_ref|) and the largest endmember error
max|E - E_ref|.

Bars.  A step factor gamma <= 1 keeps the step within the Lipschitz bound
the paper's step size is built on; there the iteration contracts and the
error stays at the level of the contraction operands' rounding: 2^-24 for
FP32 and split TF32, 2^-11 for TF32, 2^-9 for BF16 (relative).  The bars
are 5-50x above the errors these cubes show; for TF32 and BF16 they sit a
decade or more below the operands' rounding:
    FP32, split TF32: loss, A, E 1e-6; N|B - B_ref| 1e-3
    TF32:             loss, A, E 2e-5; N|B - B_ref| 1e-2
    BF16:             loss, A, E 1e-4; N|B - B_ref| 1e-1
With gamma = 2 and 8 the step exceeds that bound: the iteration oscillates
and amplifies any rounding (the FP32 path itself ends 1e-3 from the
oracle at gamma = 8), so those runs are reported, must stay finite, and
are bounded only for the FP32-grade modes (loss within 1e-2)."""
import numpy as np
import pytest

from oracle import edaa_oracle as O
from paper_2209_11002_gb300 import build, edaa, synth

pytestmark = pytest.mark.gpu

T = 10
STABLE = {edaa.FP32: (1e-6, 1e-3), edaa.TF32X3: (1e-6, 1e-3), edaa.TF32: (2e-5, 1e-2), edaa.BF16: (1e-4, 1e-1)}
NAMES = {edaa.FP32: "fp32", edaa.TF32: "tf32", edaa.BF16: "bf16", edaa.TF32X3: "split tf32"}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()
    edaa.load_library()


def _refs(cube, runs):
    Xn = O.normalize_pixels(cube.X)
    out = {}
    for m in runs:
        r = O.edaa(Xn, cube.p, T, 5, 5, int(cube.seeds[m]), float(cube.gammas[m]))
        out[m] = (r["E"], r["A"], r["B"], O.objective(Xn, r["A"], r["B"]))
    return out


@pytest.fixture(scope="module")
def urban():
    cube = synth.workload(synth.URBAN_PRECISION)
    runs = (0, 15, 8, 4, 2)  # gamma 1/8, 1/2, 1, 2, 8
    assert [float(cube.gammas[m]) for m in runs] == [0.125, 0.5, 1.0, 2.0, 8.0]
    return cube, runs, _refs(cube, runs)


@pytest.fixture(scope="module")
def largest():
    cube = synth.make_cube(285, 94249, 6, alpha=0.3, snr_db=25.0, M=16, gamma_choices=synth.GAMMA_SET, seed=1044)
    runs = (0, 3, 7)
    return cube, runs, _refs(cube, runs)


def _check(cube, runs, refs, prec):
    with edaa.Context([dict(X=cube.pixel_major(), p=cube.p, seeds=cube.seeds, gammas=cube.gammas)], T=T,
                      precision=prec) as ctx:
        ctx.solve()
        loss = ctx.loss(0)
        best, fit, mu = ctx.select(0)
        got = {m: ctx.get(0, m, device="cpu") for m in runs}
    assert np.all(np.isfinite(loss)) and np.all(np.isfinite(fit))
    assert best == O.select(fit, mu)  # Algorithm 2 on the GPU's own fits and coherences
    tol, tolB = STABLE[prec]
    for m in runs:
        E, A, B = got[m]
        Er, Ar, Br, lr = refs[m]
        g = float(cube.gammas[m])
        e = dict(loss=abs(loss[m] - lr) / lr, A=float(np.abs(A - Ar).max()), B=float(np.abs(B - Br).max()) * cube.N,
                 E=float(np.abs(E - Er).max()))
        print("%-10s L=%d N=%d run %2d gamma %5.3f: loss %.1e  A %.1e  N|B| %.1e  E %.1e"
              % (NAMES[prec], cube.L, cube.N, m, g, e["loss"], e["A"], e["B"], e["E"]))
        if g <= 1.0:
            assert e["loss"] <= tol and e["A"] <= tol and e["E"] <= tol and e["B"] <= tolB, (m, g, e)
        elif prec in (edaa.FP32, edaa.TF32X3):
            assert e["loss"] <= 1e-2, (m, g, e)


@pytest.mark.parametrize("prec", [edaa.FP32, edaa.TF32, edaa.BF16, edaa.TF32X3])
def test_urban_shape_full_size_against_oracle(urban, prec):
    _check(*urban, prec)


@pytest.mark.parametrize("prec", [edaa.FP32, edaa.TF32, edaa.BF16, edaa.TF32X3])
def test_largest_uneven_batch_shape_against_oracle(largest, prec):
    _check(*largest, prec)
