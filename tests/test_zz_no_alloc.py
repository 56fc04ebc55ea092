"""The allocation-free entry point edaa_fit_eval_static.

Callers that cannot call cudaMalloc -- for example a process whose device
memory is owned by another allocator (a framework's caching pool that has
reserved the whole GPU), or a latency-bound loop that must not block in the
driver's allocator -- can still evaluate Algorithm 2's fit and the loss of
given solutions: this entry point keeps its partial sums in a fixed static
device array inside the library instead of allocating.  The test checks it
against the existing entry points that compute the same quantities with
library-allocated scratch (edaa_select's fit, edaa_loss), on two calls in a
row (the second call reuses the array the first one left behind), and
against the FP64 oracle's definitions of the same quantities (entrywise and
max-column l1 fit, squared loss) evaluated on the same E and A.  A second
case exceeds 65,536 pixels (the kernel's grid is capped, so each block
strides over several pixel ranges) with M = 64 runs, the most the static
array holds, and checks that a call leaves the device's free memory as it
found it.

This file is collected last so that a run stopping at its first failure has
already run every other test; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

from oracle import edaa_oracle as O
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
    _check_against_oracle(Xn, E, A, calls[0])


def _check_against_oracle(Xn, E, A, got):
    """Algorithm 2's fit (entrywise and induced l1) and the squared loss, by
    the oracle's definitions on the same float32 X, E and A taken to FP64."""
    X64 = Xn.double().cpu().numpy().T  # L x N, the paper's orientation
    E64, A64 = E.double().cpu().numpy(), A.double().cpu().numpy()
    fit, fitmax, loss = got
    for m in range(E64.shape[0]):
        R = X64 - E64[m] @ A64[m]
        assert abs(fit[m] - O.fit_l1(X64, E64[m], A64[m], 0)) <= 1e-4 * fit[m]
        assert abs(fitmax[m] - O.fit_l1(X64, E64[m], A64[m], 1)) <= 1e-4 * fitmax[m]
        assert abs(loss[m] - float((R * R).sum())) <= 1e-4 * loss[m]


@pytest.mark.gpu
def test_static_scratch_many_pixels_full_array_allocates_nothing(lib):
    """N = 70,001 pixels (the capped grid strides) and M = 64 runs (the whole
    array): against edaa_loss and the oracle, twice, with the device's free
    memory unchanged across the second call."""
    import torch
    cube = synth.make_cube(24, 70001, 3, alpha=0.5, snr_db=30, M=64, gamma_choices=(0.5, 1.0), seed=32)
    with edaa.Context([dict(X=cube.pixel_major(), p=3, seeds=cube.seeds, gammas=cube.gammas)], T=2) as ctx:
        ctx.solve()
        ref_loss = ctx.loss(0)
        got = [ctx.get(0, m, device="cuda") for m in range(cube.M)]
    E = torch.stack([g[0] for g in got]).contiguous()
    A = torch.stack([g[1] for g in got]).contiguous()
    X64 = cube.pixel_major().astype(np.float64)
    Xn = torch.from_numpy((X64 / np.linalg.norm(X64, axis=1, keepdims=True)).astype(np.float32)).cuda()
    out = torch.zeros((2, 3, cube.M), dtype=torch.float64, device="cuda")
    N, L = Xn.shape
    for k in range(2):
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = lib.edaa_fit_eval_static(edaa._ptr(Xn), L, N, 3, cube.M, edaa._ptr(E), edaa._ptr(A), edaa._ptr(out[k, 0]),
                                      edaa._ptr(out[k, 1]), edaa._ptr(out[k, 2]), None)
        assert st == edaa.EDAA_OK, lib.edaa_last_error()
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        if k == 1:  # the first call on a fresh device may still load the library's image
            assert free1 == free0, (free0, free1)
    res = out.cpu().numpy()
    assert np.array_equal(res[0], res[1])
    assert np.allclose(res[0, 2], ref_loss, rtol=1e-4, atol=0)
    _check_against_oracle(Xn, E, A, tuple(res[0]))


def test_static_scratch_rejects_sizes_beyond_its_limit(lib):
    """M above 64 runs (or p above 8) is refused before any device work."""
    dummy = ctypes.c_void_p(16)
    st = lib.edaa_fit_eval_static(dummy, 10, 100, 4, 65, dummy, dummy, dummy, None, None, None)
    assert st == edaa.EDAA_ERR_UNSUPPORTED
    assert b"64" in lib.edaa_last_error()
    st = lib.edaa_fit_eval_static(dummy, 10, 100, 9, 4, dummy, dummy, dummy, None, None, None)
    assert st == edaa.EDAA_ERR_UNSUPPORTED
