"""Why the unrolled solve keeps log A and log B in float-float.

d(loss)/dX of the unrolled solve holds the residual X - E_hat A_hat, small
where the model fits, so any rounding that moves the trajectory shows up in it
amplified.  At the APEX test shape (L=285, N=13542, p=4, T=20, K1=K2=5; the
cube, step sizes and loss of tests/test_gpu_unrolled.py) this test runs an
FP64 restatement of the unrolled solve (the updates of eqs. update_A and
update_B in log-softmax form, as oracle/edaa_unrolled_torch.py) three ways:
exact; with every stored log A and log B rounded to float32; and with a
rounding-sized shift common to each pixel's log A (what a float normaliser
costs).  The first perturbation moves d(loss)/dX by orders of magnitude more
than the second, which the next normalisation removes.  CPU only."""
import numpy as np
import torch

from oracle import edaa_oracle as O
from paper_2209_11002_gb300 import synth


class _Round32(torch.autograd.Function):  # float32 rounding of the forward value only
    @staticmethod
    def forward(ctx, x):
        return x.float().double()

    @staticmethod
    def backward(ctx, g):
        return g


class _PixelShift(torch.autograd.Function):  # one float32 ulp-sized shift per pixel (column of log A)
    gen = None

    @staticmethod
    def forward(ctx, x):
        scale = 6e-8 * (1.0 + x.abs().max(dim=0, keepdim=True).values)
        return x + (torch.rand(1, x.shape[1], generator=_PixelShift.gen, dtype=x.dtype) * 2 - 1) * scale

    @staticmethod
    def backward(ctx, g):
        return g


def _unrolled(X, u, eta_A, eta_B, K1, K2, mode):
    p, N = u.shape[1], X.shape[1]
    logA = torch.full((p, N), -np.log(p), dtype=X.dtype)
    logB = torch.log_softmax(0.1 * u, dim=0)
    for t in range(eta_A.shape[0]):
        E = X @ torch.exp(logB)
        G, c = E.t() @ E, E.t() @ X
        for _ in range(K1):
            logA = torch.log_softmax(logA - eta_A[t] * (G @ torch.exp(logA) - c), dim=0)
            if mode == "round":
                logA = _Round32.apply(logA)
            elif mode == "shift":
                logA = _PixelShift.apply(logA)
        A = torch.exp(logA)
        for _ in range(K2):
            B = torch.exp(logB)
            logB = torch.log_softmax(logB - eta_B[t] * (X.t() @ ((X @ B @ A - X) @ A.t())), dim=0)
            if mode == "round":
                logB = _Round32.apply(logB)
    return X @ torch.exp(logB), torch.exp(logA)


def test_float32_logs_dominate_the_gradient_error():
    L, N, p, T, K1, K2, seed = 285, 111 * 122, 4, 20, 5, 5, 1005
    cube = synth.make_cube(L, N, p, alpha=0.3, snr_db=30, seed=seed)
    X = O.normalize_pixels(cube.X)
    u = O.uniform_u(777 + seed, N, p)
    e1, e2 = O.step_sizes(X, O.init_B(u), 1.0)
    rng = np.random.default_rng(seed)
    etaA = torch.tensor(e1 * rng.uniform(0.5, 1.5, T))
    etaB = torch.tensor(e2 * rng.uniform(0.5, 1.5, T))
    WE = torch.tensor(rng.standard_normal((L, p)))
    WA = torch.tensor(rng.standard_normal((p, N)) / np.sqrt(N))
    torch.set_num_threads(max(1, min(8, torch.get_num_threads())))

    def dX(mode):
        _PixelShift.gen = torch.Generator().manual_seed(5)
        Xt = torch.tensor(X, requires_grad=True)
        E, A = _unrolled(Xt, torch.tensor(u), etaA, etaB, K1, K2, mode)
        loss = 0.5 * ((Xt - E @ A) ** 2).sum() + (WE * E).sum() + (WA * A).sum()
        return torch.autograd.grad(loss, [Xt])[0].numpy()

    ref = dX("exact")
    err_round = np.linalg.norm(dX("round") - ref) / np.linalg.norm(ref)
    err_shift = np.linalg.norm(dX("shift") - ref) / np.linalg.norm(ref)
    print("d(loss)/dX relative change: float32 logs %.2e, per-pixel common shift %.2e" % (err_round, err_shift))
    assert err_round > 1e-4  # within an order of magnitude of the GPU parity test's 1e-3 bar
    assert err_round > 100 * err_shift
