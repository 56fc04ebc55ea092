"""GPU tests of the auxiliary subsystems around the solve: the per-iteration
loss log (config.record_loss) against the FP64 oracle, checkpoint/resume,
and the out-of-memory path driven by host-side failure injection (no device
fault is made)."""
import numpy as np
import pytest

from oracle import edaa_oracle as O
from paper_2209_11002_gb300 import build, edaa, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()
    edaa.load_library()


def _ctx(cube, **cfg):
    return edaa.Context([dict(X=cube.pixel_major(), p=cube.p, seeds=cube.seeds, gammas=cube.gammas)], **cfg)


@pytest.mark.parametrize("prec,M,tol", [(edaa.FP32, 3, 1e-5), (edaa.BF16, 16, 1e-3)])
def test_loss_log_follows_the_oracle_every_outer_iteration(prec, M, tol):
    """Row t of the log is ||X - X B A||_F^2 after outer iteration t + 1 of
    Algorithm 1, per run; persistent and per-phase launches log the same."""
    cube = synth.make_cube(40, 2000, 4, alpha=0.4, snr_db=25, M=M, gamma_choices=(0.5, 1.0), seed=61)
    T = 6
    Xn = O.normalize_pixels(cube.X)
    logs = []
    for persistent in (1, 0):
        with _ctx(cube, T=T, record_loss=1, precision=prec, persistent=persistent) as ctx:
            ctx.step(2)  # the log continues across calls
            ctx.solve()
            logs.append(ctx.loss_history(0))
            assert np.array_equal(logs[-1][-1], ctx.loss(0))  # the last row is the final loss
    assert logs[0].shape == (T, M) and np.array_equal(logs[0], logs[1])
    for m in (0, M - 1):
        ref = O.edaa(Xn, 4, T, 5, 5, int(cube.seeds[m]), float(cube.gammas[m]), record=True)["hist"]["loss"]
        rel = np.abs(logs[0][:, m] - np.array(ref[1:])) / np.array(ref[1:])
        print("run %d: largest relative loss error over the log %.1e" % (m, rel.max()))
        assert rel.max() <= tol


def test_loss_log_is_off_by_default():
    cube = synth.make_cube(20, 300, 3, M=2, seed=62)
    with _ctx(cube, T=2) as ctx:
        ctx.solve()
        with pytest.raises(edaa.EDAAError) as ei:
            ctx.loss_history(0)
        assert ei.value.status == edaa.EDAA_ERR_STATE


@pytest.mark.parametrize("prec,M", [(edaa.FP32, 4), (edaa.BF16, 16), (edaa.TF32X3, 16)])
def test_checkpoint_resume_reproduces_the_run(prec, M):
    """A context restored from a checkpoint taken after 4 outer iterations
    ends exactly where the original does (same kernels, same order)."""
    cube = synth.make_cube(36, 1700, 4, alpha=0.3, snr_db=25, M=M, gamma_choices=(0.5, 1.0, 2.0), seed=63)
    T = 9

    def finish(ctx):
        ctx.solve()
        best, fit, mu = ctx.select(0)
        return best, fit, mu, ctx.loss(0), [ctx.get(0, m, device="cpu") for m in range(M)], ctx.loss_history(0)

    with _ctx(cube, T=T, precision=prec, record_loss=1) as a:
        a.step(4)
        state = a.checkpoint()
        ref = finish(a)
    with _ctx(cube, T=T, precision=prec, record_loss=1) as b:
        b.step(1)  # some other progress, overwritten by the restore
        b.restore(state)
        assert b.outer_done() == 4
        got = finish(b)
    assert got[0] == ref[0]
    for x, y in zip(got[1:4], ref[1:4]):
        assert np.array_equal(x, y)
    for run_got, run_ref in zip(got[4], ref[4]):
        for x, y in zip(run_got, run_ref):
            assert np.array_equal(x, y)
    assert np.array_equal(got[5], ref[5])


def test_restore_refuses_other_cubes_and_other_data():
    cube = synth.make_cube(30, 900, 3, M=3, gamma_choices=(1.0,), seed=64)
    with _ctx(cube, T=4) as a:
        a.step(2)
        state = a.checkpoint()
    other = synth.make_cube(30, 900, 3, M=4, gamma_choices=(1.0,), seed=64)  # one more run
    with _ctx(other, T=4) as b:
        with pytest.raises(edaa.EDAAError) as ei:
            b.restore(state)
        assert ei.value.status == edaa.EDAA_ERR_ARG
    moved = synth.make_cube(30, 900, 3, M=3, gamma_choices=(1.0,), seed=64)
    moved.X[5, 7] += 0.25  # same shapes, other data
    with _ctx(moved, T=4) as c:
        with pytest.raises(edaa.EDAAError) as ei:
            c.restore(state)
        assert ei.value.status == edaa.EDAA_ERR_ARG
        assert c.outer_done() == 0  # nothing was changed
    with _ctx(cube, T=4) as d:
        with pytest.raises(edaa.EDAAError):
            d.restore(state[:-8])  # truncated


def test_simulated_out_of_memory_releases_everything():
    """The k-th device allocation fails (injected on the host): edaa_init
    returns EDAA_ERR_OOM and frees what it had allocated; a host-output
    edaa_get whose scratch allocation fails returns EDAA_ERR_OOM too."""
    import torch
    lib = edaa.load_library()
    cube = synth.make_cube(24, 800, 3, M=2, seed=65)
    with _ctx(cube, T=2) as warm:  # one-time runtime set-up is not a leak
        warm.solve()
        warm.sync()
    torch.cuda.synchronize()
    try:
        free0 = torch.cuda.mem_get_info()[0]
        for k in range(3):  # the cube's arena, the batch descriptor, the status words
            lib.edaa_debug_fail_alloc(k)
            with pytest.raises(edaa.EDAAError) as ei:
                _ctx(cube, T=2)
            assert ei.value.status == edaa.EDAA_ERR_OOM, k
        lib.edaa_debug_fail_alloc(-1)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        with _ctx(cube, T=2) as ctx:
            ctx.solve()
            lib.edaa_debug_fail_alloc(0)
            with pytest.raises(edaa.EDAAError) as ei:
                ctx.get(0, 0, device="cpu")
            assert ei.value.status == edaa.EDAA_ERR_OOM
            lib.edaa_debug_fail_alloc(-1)
            E, A, B = ctx.get(0, 0, device="cpu")
            assert np.all(np.isfinite(A))
    finally:
        lib.edaa_debug_fail_alloc(-1)
