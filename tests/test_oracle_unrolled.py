"""Pins of the reference gradient of the unrolled solve (torch FP64 CPU autograd
over a second restatement of Algorithm 1): its forward agrees with the numpy
oracle, and its gradients agree with central finite differences of the numpy
oracle's forward (two independent routes)."""
import numpy as np
import pytest
import torch

from oracle import edaa_oracle as O
from oracle.edaa_unrolled_torch import unrolled_edaa
from paper_2209_11002_gb300 import synth


def _setup(L=10, N=60, p=3, T=3, seed=41):
    cube = synth.make_cube(L, N, p, alpha=0.5, snr_db=30, seed=seed)
    X = O.normalize_pixels(cube.X)
    u = O.uniform_u(17, N, p)
    B0 = O.init_B(u)
    e1, e2 = O.step_sizes(X, B0, 1.0)
    rng = np.random.default_rng(seed + 1)
    etaA = e1 * rng.uniform(0.5, 1.5, T)
    etaB = e2 * rng.uniform(0.5, 1.5, T)
    WE = rng.standard_normal((L, p))
    WA = rng.standard_normal((p, N))
    return X, u, etaA, etaB, WE, WA


def _loss_np(X, u, etaA, etaB, WE, WA, K1, K2):
    p = u.shape[1]
    r = O.edaa(X, p, len(etaA), K1, K2, seed=0, B0=O.init_B(u), eta_A=etaA, eta_B=etaB)
    E, A = r["E"], r["A"]
    Rz = X - E @ A
    return 0.5 * (Rz * Rz).sum() + (WE * E).sum() + (WA * A).sum()


def test_torch_forward_matches_numpy_oracle():
    X, u, etaA, etaB, WE, WA = _setup()
    r = O.edaa(X, 3, 3, 2, 2, seed=0, B0=O.init_B(u), eta_A=etaA, eta_B=etaB)
    E, A = unrolled_edaa(torch.tensor(X), torch.tensor(u), torch.tensor(etaA), torch.tensor(etaB), 2, 2)
    assert np.abs(E.numpy() - r["E"]).max() < 1e-12
    assert np.abs(A.numpy() - r["A"]).max() < 1e-12


@pytest.mark.parametrize("K1,K2", [(2, 2), (1, 3)])
def test_torch_gradients_match_finite_differences(K1, K2):
    X, u, etaA, etaB, WE, WA = _setup()
    Xt = torch.tensor(X, requires_grad=True)
    eA = torch.tensor(etaA, requires_grad=True)
    eB = torch.tensor(etaB, requires_grad=True)
    E, A = unrolled_edaa(Xt, torch.tensor(u), eA, eB, K1, K2)
    loss = 0.5 * ((Xt - E @ A) ** 2).sum() + (torch.tensor(WE) * E).sum() + (torch.tensor(WA) * A).sum()
    dX, deA, deB = torch.autograd.grad(loss, [Xt, eA, eB])
    f = lambda X_, a_, b_: _loss_np(X_, u, a_, b_, WE, WA, K1, K2)
    rng = np.random.default_rng(5)
    for _ in range(2):
        V = rng.standard_normal(X.shape)
        V /= np.linalg.norm(V)
        h = 1e-5
        fd = (f(X + h * V, etaA, etaB) - f(X - h * V, etaA, etaB)) / (2 * h)
        ad = float((dX.numpy() * V).sum())
        assert abs(fd - ad) <= 1e-6 * max(1.0, abs(ad))
    for t in range(len(etaA)):
        h = 1e-6 * etaA[t]
        ap, am = etaA.copy(), etaA.copy()
        ap[t] += h
        am[t] -= h
        fd = (f(X, ap, etaB) - f(X, am, etaB)) / (2 * h)
        assert abs(fd - float(deA[t])) <= 1e-5 * max(1.0, abs(fd))
        h = 1e-6 * etaB[t]
        bp, bm = etaB.copy(), etaB.copy()
        bp[t] += h
        bm[t] -= h
        fd = (f(X, etaA, bp) - f(X, etaA, bm)) / (2 * h)
        assert abs(fd - float(deB[t])) <= 1e-5 * max(1.0, abs(fd))
