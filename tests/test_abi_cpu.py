"""CPU checks of the C-ABI library: it builds, loads, exports every entry point
include/edaa.h declares, its host-side selection rule matches Algorithm 2 as
the oracle states it, and without a GPU its compute calls fail loudly."""
import os
import re

import numpy as np
import pytest

from oracle import edaa_oracle as O
from paper_2209_11002_gb300 import build, edaa

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build_library()
    return edaa.load_library()


def _declared():
    text = open(os.path.join(ROOT, "include", "edaa.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(edaa_[a-z_]+)\s*\(", text)))


def test_header_matches_binding_exports():
    assert _declared() == sorted(edaa.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_config_defaults_are_the_papers(lib):
    cfg = edaa.default_config()
    assert (cfg.T, cfg.K1, cfg.K2) == (100, 5, 5)
    assert cfg.fit_ratio == 1.05 and cfg.normalize == 1


@pytest.mark.parametrize("seed", range(6))
def test_select_rule_matches_oracle(lib, seed):
    rng = np.random.default_rng(seed)
    M = 12
    fit = rng.uniform(10, 12, M)
    mu = rng.uniform(0, 1, M)
    if seed % 2:
        fit[3] = np.nan
        fit[5] = fit.min() * 1.05  # boundary is inclusive
        mu[5] = -1.0
    if seed == 4:
        mu[:] = 0.5  # ties go to the lowest index
    assert edaa.select_rule(fit, mu) == O.select(fit, mu)


def test_select_rule_edge_cases(lib):
    assert edaa.select_rule([np.nan, np.inf], [0.0, 0.0]) == -1
    assert edaa.select_rule([1.0], [float("-inf")]) == 0


def test_compute_calls_fail_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    X = np.ones((40, 5), np.float32)
    with pytest.raises(edaa.EDAAError) as ei:
        edaa.Context([dict(X=X, p=2, seeds=[1], gammas=[1.0])], T=1)
    assert ei.value.status == edaa.EDAA_ERR_CUDA


def test_argument_validation(lib):
    X = np.ones((5, 40), np.float32)  # N=5 pixels, L=40 bands
    bad = [dict(X=X, p=0, seeds=[1], gammas=[1.0]),          # p < 1
           dict(X=X, p=6, seeds=[1], gammas=[1.0]),          # N < p
           dict(X=X, p=2, seeds=[1], gammas=[-1.0]),         # gamma <= 0
           dict(X=np.ones((40, 400), np.float32), p=2, seeds=[1], gammas=[1.0])]  # L > 319
    codes = []
    for c in bad:
        with pytest.raises(edaa.EDAAError) as ei:
            edaa.Context([c], T=1)
        codes.append(ei.value.status)
    assert codes[:3] == [edaa.EDAA_ERR_ARG] * 3
    assert codes[3] == edaa.EDAA_ERR_UNSUPPORTED


def test_trace_read_and_precision_arguments(lib):
    """edaa_trace_read refuses a missing context or an unknown sequence, and
    the precision field accepts exactly FP32, TF32, BF16 and TF32X3."""
    import ctypes
    n = ctypes.c_int(-1)
    assert lib.edaa_trace_read(None, 0, 0, ctypes.byref(n), None, None, None) == edaa.EDAA_ERR_ARG
    assert edaa.default_config().trace == 0
    assert (edaa.FP32, edaa.TF32, edaa.BF16, edaa.TF32X3) == (0, 1, 2, 3)
    X = np.ones((40, 5), np.float32)
    with pytest.raises(edaa.EDAAError) as ei:
        edaa.Context([dict(X=X, p=2, seeds=[1], gammas=[1.0])], T=1, precision=4)
    assert ei.value.status == edaa.EDAA_ERR_ARG


def test_tile_argument_is_validated_before_any_device_call(lib):
    """edaa_config.tile: all zero by default; a launch shape outside the
    compiled register tiles (four pixels per lane needs p >= 3 and one run
    per warp), outside 32..128 pixels, or with more runs than the cube has,
    fails with EDAA_ERR_ARG before the library touches a device."""
    assert list(edaa.default_config().tile) == [0, 0, 0, 0]
    X = np.ones((300, 20), np.float32)
    bad = [(8, 1, 4, 1, 2),   # four pixels per lane with p = 2
           (4, 4, 2, 1, 4),   # 256-pixel tile
           (9, 1, 2, 1, 4),   # more runs per group than runs (M = 8)
           (8, 1, 3, 1, 4),   # three pixels per lane is not compiled
           (8, 0, 2, 1, 4)]   # no phase-1 warps
    for rm, wp1, spt, wp2, p in bad:
        with pytest.raises(edaa.EDAAError) as ei:
            edaa.Context([dict(X=X, p=p, seeds=list(range(8)), gammas=[1.0] * 8)], T=1,
                         tile=(rm, wp1, spt, wp2))
        assert ei.value.status == edaa.EDAA_ERR_ARG, (rm, wp1, spt, wp2, p)
    # a tensor-core cube (BF16, M p = 64) checks tile[0] alone: 1..M
    Xb = np.ones((300, 20), np.float32)
    kw = dict(p=4, seeds=list(range(16)), gammas=[1.0] * 16)
    with pytest.raises(edaa.EDAAError) as ei:
        edaa.Context([dict(X=Xb, **kw)], T=1, precision=edaa.BF16, tile=(17, 0, 0, 0))
    assert ei.value.status == edaa.EDAA_ERR_ARG
    with pytest.raises(edaa.EDAAError) as ei:  # accepted; then no device on this machine
        edaa.Context([dict(X=Xb, **kw)], T=1, precision=edaa.BF16, tile=(12, 0, 0, 0))
    assert ei.value.status != edaa.EDAA_ERR_ARG

