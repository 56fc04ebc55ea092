"""Seeded synthetic hyperspectral cubes (linear mixing model, Sec. III-A, eq. LMM).

This module only draws inputs: endmember spectra, Dirichlet abundances, noise,
per-run seeds and step-size factors.  It holds none of EDAA's arithmetic, so
the FP64 oracle and the CUDA path can both be fed from it without sharing any
part of the method.

Recipe (stand-ins for the paper's real scenes, whose shapes are copied):
  * endmember j: a sum of 3-6 Gaussian bumps over the band index, centres
    U[0, L), widths U[L/20, L/5], amplitudes U[0.2, 1], then min-max scaled
    into [0, 1];
  * abundances: Dirichlet(alpha) per pixel; optionally the first p pixels are
    pure (one-hot), one per endmember;
  * noise: white Gaussian with variance ||E A||_F^2 / (L N 10^(SNR/10));
  * X is returned as float32 in the paper's orientation, L x N (bands x pixels).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

# The paper's step-size factor set S (Sec. III-C, eq. eta0A).
GAMMA_SET = (0.125, 0.25, 0.5, 1.0, 2.0, 4.0, 8.0)


@dataclasses.dataclass
class Cube:
    X: np.ndarray          # L x N float32 (paper orientation)
    E_true: np.ndarray     # L x p float64
    A_true: np.ndarray     # p x N float64
    seeds: np.ndarray      # M uint64: per-run seeds s_m (Algorithm 2)
    gammas: np.ndarray     # M float64: per-run step-size factors gamma_m
    snr_db: float
    name: str = ""

    @property
    def L(self) -> int:
        return self.X.shape[0]

    @property
    def N(self) -> int:
        return self.X.shape[1]

    @property
    def p(self) -> int:
        return self.E_true.shape[1]

    @property
    def M(self) -> int:
        return len(self.seeds)

    def pixel_major(self) -> np.ndarray:
        """X as N x L row-major float32 (pixel i's bands contiguous)."""
        return np.ascontiguousarray(self.X.T)


def endmembers(rng: np.random.Generator, L: int, p: int) -> np.ndarray:
    """Smooth nonnegative spectra scaled into [0, 1], L x p."""
    band = np.arange(L, dtype=np.float64)
    E = np.zeros((L, p))
    for j in range(p):
        nb = int(rng.integers(3, 7))
        centres = rng.uniform(0.0, L, nb)
        widths = rng.uniform(L / 20.0, L / 5.0, nb)
        amps = rng.uniform(0.2, 1.0, nb)
        e = (amps[:, None] * np.exp(-0.5 * ((band[None, :] - centres[:, None]) / widths[:, None]) ** 2)).sum(0)
        lo, hi = e.min(), e.max()
        E[:, j] = (e - lo) / (hi - lo) if hi > lo else e
    return E


def abundances(rng: np.random.Generator, p: int, N: int, alpha: float, pure: bool) -> np.ndarray:
    A = rng.dirichlet(np.full(p, alpha), size=N).T  # p x N
    if pure:
        A[:, :p] = np.eye(p)
    return A


def run_params(seed: int, M: int, gamma_choices: Optional[Sequence[float]]) -> tuple:
    """Per-run seeds and step-size factors, drawn from one generator."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x5EED]))
    seeds = rng.integers(1, 2**63 - 1, size=M, dtype=np.int64).astype(np.uint64)
    if gamma_choices is None:
        gammas = np.ones(M)
    else:
        gammas = np.asarray(rng.choice(np.asarray(gamma_choices, dtype=np.float64), size=M))
    return seeds, gammas


def make_cube(L: int, N: int, p: int, *, alpha: float = 0.5, snr_db: Optional[float] = 30.0,
              pure: bool = False, M: int = 1, gamma_choices: Optional[Sequence[float]] = None,
              seed: int = 0, name: str = "") -> Cube:
    rng = np.random.default_rng(seed)
    E = endmembers(rng, L, p)
    A = abundances(rng, p, N, alpha, pure)
    Y = E @ A
    if snr_db is not None:
        sigma2 = (Y * Y).sum() / (L * N * 10.0 ** (snr_db / 10.0))
        Y = Y + rng.standard_normal(Y.shape) * np.sqrt(sigma2)
    seeds, gammas = run_params(seed, M, gamma_choices)
    return Cube(X=Y.astype(np.float32), E_true=E, A_true=A, seeds=seeds, gammas=gammas,
                snr_db=float(snr_db) if snr_db is not None else float("inf"), name=name)


# ---------------------------------------------------------------------------
# The five workloads.  Shapes copy the paper's scenes (Sec. IV-A): Samson
# 156x9025 p=3, Jasper Ridge 198x10000 p=4, Urban 162x94249 p=6, APEX
# 285x13542 p=4.  Seeds are 1000 + workload number.
# ---------------------------------------------------------------------------
SAMSON_EDAA = dict(L=156, N=95 * 95, p=3, alpha=0.5, snr_db=30.0, pure=True, M=1,
                   gamma_choices=None, seed=1001, name="samson-shape L156 N9025 p3 M1")
JASPER_ENSEMBLE = dict(L=198, N=100 * 100, p=4, alpha=0.3, snr_db=25.0, pure=False, M=50,
                       gamma_choices=(0.5, 1.0, 2.0), seed=1002,
                       name="jasper-shape L198 N10000 p4 M50")
URBAN_PRECISION = dict(L=162, N=307 * 307, p=6, alpha=0.2, snr_db=20.0, pure=False, M=64,
                       gamma_choices=GAMMA_SET, seed=1003, name="urban-shape L162 N94249 p6 M64")
APEX_UNROLLED = dict(L=285, N=111 * 122, p=4, alpha=0.3, snr_db=30.0, pure=False, M=1,
                     gamma_choices=None, seed=1005, name="apex-shape L285 N13542 p4 T20")


def uneven_batch(seed: int = 1004, n_cubes: int = 8, M: int = 16) -> List[Cube]:
    """Eight cubes of uneven (L, N, p): L from the paper's band counts, N in
    [9000, 94249], p in [3, 6], Dirichlet(0.3), SNR U[20, 35] dB."""
    rng = np.random.default_rng(seed)
    Ls = rng.choice(np.array([156, 162, 188, 198, 224, 285]), size=n_cubes)
    Ns = rng.integers(9000, 94250, size=n_cubes)
    ps = rng.integers(3, 7, size=n_cubes)
    snrs = rng.uniform(20.0, 35.0, size=n_cubes)
    cubes = []
    for c in range(n_cubes):
        cubes.append(make_cube(int(Ls[c]), int(Ns[c]), int(ps[c]), alpha=0.3, snr_db=float(snrs[c]),
                               M=M, gamma_choices=GAMMA_SET, seed=seed * 100 + c,
                               name=f"uneven[{c}] L{Ls[c]} N{Ns[c]} p{ps[c]}"))
    return cubes


def workload(spec: dict, **overrides) -> Cube:
    kw = dict(spec)
    kw.update(overrides)
    return make_cube(**kw)
