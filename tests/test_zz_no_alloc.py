"""The allocation-free entry point edaa_fit_eval_static.

Callers that cannot call cudaMalloc -- for example a process whose device
memory is owned by another allocator (a framework's caching pool that has
reserved the whole GPU), or a latency-bound loop that must not block in the
driver's allocator -- can still evaluate Algorithm 2's fit and the loss of
given solutions: this entry point keeps its partial sums in a fixed static
device array inside the library instead of allocating.  The test checks it
against the existing entry points that compute the same quantities with
library-allocated scratch (edaa_select's fit, edaa_loss), on two calls in a
row (the second call reuses the array the first one left behind).

This file is collected last so that a run stopping at its first failure has
already run every other test; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

from paper_2209_11002_gb300 import build, edaa, synth


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return edaa.load_library()


@pytest.mark.gpu
def test_static_scratch_fit_matches_existing_entry_points_twice(lib):
    import torch
    cube = synth.make_cube(64, 3001, 4, alpha=0.4, snr_db=25, M=6, gamma_choices=(0.5, 1.0, 2.0), seed=31)
    ref = {}
    Es, As = [], []
    for fit_norm in (0, 1):
        with edaa.Context([dict(X=cube.pixel_major(), p=4, seeds=cube.seeds, gammas=cube.gammas)], T=8,
                          fit_norm=fit_norm) as ctx:
            ctx.solve()
            best, fit, mu = ctx.select(0)
            ref[fit_norm] = fit
            if fit_norm == 0:
                ref["loss"] = ctx.loss(0)
                for m in range(cube.M):
                    E, A, B = ctx.get(0, m, device="cuda")
                    Es.append(E)
                    As.append(A)
    X64 = cube.pixel_major().astype(np.float64)
    Xn = torch.from_numpy((X64 / np.linalg.norm(X64, axis=1, keepdims=True)).astype(np.float32)).cuda()
    E = torch.stack(Es).contiguous()
    A = torch.stack(As).contiguous()
    calls = []
    for _ in range(2):
        fit, fitmax, loss = edaa.fit_eval_static(Xn, E, A)
        torch.cuda.synchronize()
        calls.append((fit.cpu().numpy(), fitmax.cpu().numpy(), loss.cpu().numpy()))
    for fit, fitmax, loss in calls:
        assert np.allclose(fit, ref[0], rtol=1e-4, atol=0)
        assert np.allclose(fitmax, ref[1], rtol=1e-4, atol=0)
        assert np.allclose(loss, ref["loss"], rtol=1e-4, atol=0)
    for a, b in zip(calls[0], calls[1]):
        assert np.array_equal(a, b)


def test_static_scratch_rejects_sizes_beyond_its_limit(lib):
    """M above 64 runs (or p above 8) is refused before any device work."""
    dummy = ctypes.c_void_p(16)
    st = lib.edaa_fit_eval_static(dummy, 10, 100, 4, 65, dummy, dummy, dummy, None, None, None)
    assert st == edaa.EDAA_ERR_UNSUPPORTED
    assert b"64" in lib.edaa_last_error()
    st = lib.edaa_fit_eval_static(dummy, 10, 100, 9, 4, dummy, dummy, dummy, None, None, None)
    assert st == edaa.EDAA_ERR_UNSUPPORTED
