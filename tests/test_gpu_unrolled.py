"""GPU parity of the differentiable unrolled solve (EDAAUnrolled).

Forward: E_hat, A_hat against the FP64 numpy oracle with the same per-block
step sizes (max-abs 1e-3).  Backward of
    loss = 1/2 ||X - E_hat A_hat||_F^2 + <W_E, E_hat> + <W_A, A_hat>
with respect to X and the 2T step sizes: against torch FP64 autograd over the
independent restatement in oracle/edaa_unrolled_torch.py (norm-wise relative
1e-3), and against central differences (h = 1e-3) of the FP64 numpy forward
along random directions."""
import numpy as np
import pytest
import torch

from oracle import edaa_oracle as O
from oracle.edaa_unrolled_torch import unrolled_edaa
from paper_2209_11002_gb300 import build, edaa, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build_library()
    edaa.load_library()


def _problem(L, N, p, T, seed):
    cube = synth.make_cube(L, N, p, alpha=0.3, snr_db=30, seed=seed)
    X = O.normalize_pixels(cube.X)                      # L x N, FP64
    run_seed = 777 + seed
    u = O.uniform_u(run_seed, N, p)
    e1, e2 = O.step_sizes(X, O.init_B(u), 1.0)
    rng = np.random.default_rng(seed)
    etaA = e1 * rng.uniform(0.5, 1.5, T)
    etaB = e2 * rng.uniform(0.5, 1.5, T)
    WE = rng.standard_normal((L, p))
    WA = rng.standard_normal((p, N)) / np.sqrt(N)
    return X, run_seed, u, etaA, etaB, WE, WA


def _gpu(X, run_seed, etaA, etaB, WE, WA, p, K1, K2):
    from paper_2209_11002_gb300.autograd import EDAAUnrolled
    Xg = torch.tensor(X.T.astype(np.float32), device="cuda", requires_grad=True)   # N x L
    eA = torch.tensor(etaA, dtype=torch.float64, requires_grad=True)
    eB = torch.tensor(etaB, dtype=torch.float64, requires_grad=True)
    E, A = EDAAUnrolled.apply(Xg, eA, eB, p, run_seed, K1, K2)
    R = Xg.t() - E @ A
    loss = 0.5 * (R * R).sum() + (torch.tensor(WE, dtype=torch.float32, device="cuda") * E).sum() \
        + (torch.tensor(WA, dtype=torch.float32, device="cuda") * A).sum()
    loss.backward()
    return E.detach().cpu().numpy(), A.detach().cpu().numpy(), Xg.grad.cpu().numpy().T, eA.grad.numpy(), eB.grad.numpy()


def _reference(X, u, etaA, etaB, WE, WA, K1, K2):
    Xt = torch.tensor(X, requires_grad=True)
    eA = torch.tensor(etaA, requires_grad=True)
    eB = torch.tensor(etaB, requires_grad=True)
    E, A = unrolled_edaa(Xt, torch.tensor(u), eA, eB, K1, K2)
    loss = 0.5 * ((Xt - E @ A) ** 2).sum() + (torch.tensor(WE) * E).sum() + (torch.tensor(WA) * A).sum()
    dX, deA, deB = torch.autograd.grad(loss, [Xt, eA, eB])
    return E.detach().numpy(), A.detach().numpy(), dX.numpy(), deA.numpy(), deB.numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("shape", [(40, 1500, 4, 4, 5, 5), (23, 777, 3, 3, 2, 3)])
def test_unrolled_forward_and_adjoint_small(shape):
    L, N, p, T, K1, K2 = shape
    X, rs, u, etaA, etaB, WE, WA = _problem(L, N, p, T, seed=L)
    E, A, dX, deA, deB = _gpu(X, rs, etaA, etaB, WE, WA, p, K1, K2)
    Er, Ar, dXr, deAr, deBr = _reference(X, u, etaA, etaB, WE, WA, K1, K2)
    ref = O.edaa(X, p, T, K1, K2, seed=rs, eta_A=etaA, eta_B=etaB)
    assert np.abs(A - ref["A"]).max() <= 1e-3 and np.abs(E - ref["E"]).max() <= 1e-3
    assert np.abs(Er - ref["E"]).max() < 1e-10  # the two FP64 restatements agree
    print("dX rel %.2e  d eta_A rel %.2e  d eta_B rel %.2e" % (_rel(dX, dXr), _rel(deA, deAr), _rel(deB, deBr)))
    assert _rel(dX, dXr) <= 1e-3
    assert _rel(deA, deAr) <= 1e-3
    assert _rel(deB, deBr) <= 1e-3


def test_unrolled_adjoint_against_central_differences():
    """Directional derivative of the GPU adjoint against central differences
    (h = 1e-3) of the FP64 numpy forward."""
    L, N, p, T, K1, K2 = 30, 900, 3, 3, 5, 5
    X, rs, u, etaA, etaB, WE, WA = _problem(L, N, p, T, seed=4)
    _, _, dX, deA, deB = _gpu(X, rs, etaA, etaB, WE, WA, p, K1, K2)

    def F(X_, a_, b_):
        r = O.edaa(X_, p, T, K1, K2, seed=rs, eta_A=a_, eta_B=b_)
        R = X_ - r["E"] @ r["A"]
        return 0.5 * (R * R).sum() + (WE * r["E"]).sum() + (WA * r["A"]).sum()

    rng = np.random.default_rng(9)
    h = 1e-3
    for _ in range(2):
        V = rng.standard_normal(X.shape)
        V /= np.linalg.norm(V)
        fd = (F(X + h * V, etaA, etaB) - F(X - h * V, etaA, etaB)) / (2 * h)
        assert abs(fd - (dX * V).sum()) <= 1e-3 * max(1.0, abs(fd))
    va, vb = rng.standard_normal(T) * etaA, rng.standard_normal(T) * etaB
    hh = 1e-3
    fd = (F(X, etaA + hh * va, etaB + hh * vb) - F(X, etaA - hh * va, etaB - hh * vb)) / (2 * hh)
    assert abs(fd - (deA @ va + deB @ vb)) <= 1e-3 * max(1.0, abs(fd))


def test_unrolled_apex_shape_full_size():
    """APEX-shaped cube L=285, N=111x122, p=4, T=20, K1=K2=5 against the FP64
    torch reference gradient."""
    L, N, p, T, K1, K2 = 285, 111 * 122, 4, 20, 5, 5
    X, rs, u, etaA, etaB, WE, WA = _problem(L, N, p, T, seed=1005)
    E, A, dX, deA, deB = _gpu(X, rs, etaA, etaB, WE, WA, p, K1, K2)
    Er, Ar, dXr, deAr, deBr = _reference(X, u, etaA, etaB, WE, WA, K1, K2)
    print("APEX shape: E max %.2e A max %.2e dX rel %.2e d eta_A rel %.2e d eta_B rel %.2e" % (
        np.abs(E - Er).max(), np.abs(A - Ar).max(), _rel(dX, dXr), _rel(deA, deAr), _rel(deB, deBr)))
    assert np.abs(A - Ar).max() <= 1e-3 and np.abs(E - Er).max() <= 1e-3
    assert _rel(dX, dXr) <= 1e-3 and _rel(deA, deAr) <= 1e-3 and _rel(deB, deBr) <= 1e-3


def test_unrolled_engine_reuse_is_bitwise_repeatable():
    """A second forward+backward of the same shape reuses the pooled engine and
    reproduces the first one bit for bit (the sweeps are deterministic)."""
    from paper_2209_11002_gb300 import autograd as AG
    L, N, p, T, K1, K2 = 23, 777, 3, 3, 2, 3
    X, rs, u, etaA, etaB, WE, WA = _problem(L, N, p, T, seed=11)
    first = _gpu(X, rs, etaA, etaB, WE, WA, p, K1, K2)
    pooled = sum(len(v) for k, v in AG._POOL.items() if k[1:7] == (L, N, p, T, K1, K2))
    second = _gpu(X, rs, etaA, etaB, WE, WA, p, K1, K2)
    assert pooled >= 1
    for a, b in zip(first, second):
        assert np.array_equal(a, b)
    AG.free_engines()
    assert not AG._POOL


def test_unrolled_two_live_contexts():
    """Two forwards alive at once (their backwards in reverse order) give the
    same results as two separate forward+backward steps."""
    L, N, p, T, K1, K2 = 23, 777, 3, 3, 2, 3
    X1, rs, u, etaA, etaB, WE, WA = _problem(L, N, p, T, seed=12)
    X2 = X1[:, ::-1].copy()
    ref1 = _gpu(X1, rs, etaA, etaB, WE, WA, p, K1, K2)
    ref2 = _gpu(X2, rs, etaA, etaB, WE, WA, p, K1, K2)
    from paper_2209_11002_gb300.autograd import EDAAUnrolled
    outs, grads = [], []
    for Xh in (X1, X2):
        Xg = torch.tensor(Xh.T.astype(np.float32), device="cuda", requires_grad=True)
        eA = torch.tensor(etaA, dtype=torch.float64, requires_grad=True)
        eB = torch.tensor(etaB, dtype=torch.float64, requires_grad=True)
        E, A = EDAAUnrolled.apply(Xg, eA, eB, p, rs, K1, K2)
        R = Xg.t() - E @ A
        loss = 0.5 * (R * R).sum() + (torch.tensor(WE, dtype=torch.float32, device="cuda") * E).sum() \
            + (torch.tensor(WA, dtype=torch.float32, device="cuda") * A).sum()
        outs.append((E, A, loss))
        grads.append((Xg, eA, eB))
    for (E, A, loss), (Xg, eA, eB), ref in reversed(list(zip(outs, grads, (ref1, ref2)))):
        loss.backward()
        got = (E.detach().cpu().numpy(), A.detach().cpu().numpy(), Xg.grad.cpu().numpy().T, eA.grad.numpy(),
               eB.grad.numpy())
        for a_, b_ in zip(got, ref):
            assert np.array_equal(a_, b_)


@pytest.mark.parametrize("shape", [(200, 50000, 3, 2, 2, 2), (30, 150000, 8, 2, 2, 2)])
def test_unrolled_global_memory_paths(shape):
    """Cubes whose X rows (L=200, N=50000) or X rows and per-pixel state (L=30,
    N=150000, p=8) do not fit in a CTA's shared memory: E, A and d(loss)/dX
    against the FP64 reference.  d(loss)/d eta at these shapes is a small sum
    of large per-pixel terms that cancel: the FP64 restatement itself, run in
    float32, misses its FP64 result by 4e-3 and 0.6 (d eta_A) here, so d eta
    is held only to the order of magnitude (its accuracy is pinned at the APEX
    shape and by central differences above)."""
    L, N, p, T, K1, K2 = shape
    X, rs, u, etaA, etaB, WE, WA = _problem(L, N, p, T, seed=L + p)
    E, A, dX, deA, deB = _gpu(X, rs, etaA, etaB, WE, WA, p, K1, K2)
    Er, Ar, dXr, deAr, deBr = _reference(X, u, etaA, etaB, WE, WA, K1, K2)
    print("global-memory paths %s: E %.2e A %.2e dX %.2e d eta_A %.2e d eta_B %.2e" % (
        shape, np.abs(E - Er).max(), np.abs(A - Ar).max(), _rel(dX, dXr), _rel(deA, deAr), _rel(deB, deBr)))
    assert np.abs(A - Ar).max() <= 1e-3 and np.abs(E - Er).max() <= 1e-3
    assert _rel(dX, dXr) <= 1e-3
    assert np.all(np.isfinite(deA)) and np.all(np.isfinite(deB))
    for got, ref in ((deA, deAr), (deB, deBr)):
        ratio = np.linalg.norm(got) / np.linalg.norm(ref)
        assert 0.1 <= ratio <= 10.0
