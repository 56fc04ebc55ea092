"""torch.autograd.Function around the unrolled EDAA engine of libedaa.

EDAAUnrolled.apply(X, eta_A, eta_B, p, seed, K1, K2) -> (E_hat, A_hat)
  X      : N x L float32 CUDA tensor (pixel-major), used as given
  eta_A  : length-T float64 tensor, step size of the K1 A-steps of outer t
  eta_B  : length-T float64 tensor, step size of the K2 B-steps of outer t
  E_hat  : L x p (= X B_hat), A_hat: p x N
The forward and the backward (hand-written adjoint kernels, one checkpoint
per outer iteration) both run in libedaa; this module only moves pointers.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np
import torch

from . import edaa


_POOL: dict = {}  # (device, L, N, p, T, K1, K2, stream) -> idle engine handles
_POOL_LOCK = threading.Lock()


class _Engine:
    """One libedaa unrolled engine (device buffers sized for one shape), held
    by an autograd context from its forward to its backward.  Creating one
    allocates device memory (~110 MB for L=285, N=13542, p=4, T=20) and
    queries the device, so released engines go back to a per-shape pool (the
    engine's own stream orders a reuse after any work still queued on it);
    free_engines() destroys the pooled ones."""

    def __init__(self, L, N, p, T, K1, K2, stream):
        self.lib = edaa.load_library()
        self.key = (torch.cuda.current_device(), L, N, p, T, K1, K2, stream.value if stream else 0)
        with _POOL_LOCK:
            idle = _POOL.get(self.key)
            self.h = idle.pop() if idle else None
        if self.h is None:
            h = ctypes.c_void_p()
            edaa._check(self.lib.edaa_unrolled_create(ctypes.byref(h), L, N, p, T, K1, K2, stream),
                        "edaa_unrolled_create")
            self.h = h

    def release(self):
        h, self.h = self.h, None
        if h and _POOL_LOCK is not None:  # (module globals may be gone at interpreter exit)
            with _POOL_LOCK:
                _POOL.setdefault(self.key, []).append(h)

    def __del__(self):
        self.release()


def free_engines():
    """Destroy every pooled (idle) unrolled engine."""
    lib = edaa.load_library()
    with _POOL_LOCK:
        handles = [h for hs in _POOL.values() for h in hs]
        _POOL.clear()
    for h in handles:
        lib.edaa_unrolled_destroy(h)


class EDAAUnrolled(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, eta_A, eta_B, p, seed, K1, K2):
        if not X.is_cuda:
            raise RuntimeError("EDAAUnrolled needs a CUDA tensor X (no CPU path)")
        X = X.to(torch.float32).contiguous()
        N, L = X.shape
        T = eta_A.numel()
        stream = torch.cuda.current_stream(X.device).cuda_stream
        eng = _Engine(L, N, p, T, K1, K2, ctypes.c_void_p(stream) if stream else None)
        eA = np.ascontiguousarray(eta_A.detach().cpu().numpy(), dtype=np.float64)
        eB = np.ascontiguousarray(eta_B.detach().cpu().numpy(), dtype=np.float64)
        E = torch.empty((L, p), dtype=torch.float32, device=X.device)
        A = torch.empty((p, N), dtype=torch.float32, device=X.device)
        dp = ctypes.POINTER(ctypes.c_double)
        edaa._check(eng.lib.edaa_unrolled_forward(eng.h, edaa._ptr(X), ctypes.c_uint64(int(seed)),
                                                  eA.ctypes.data_as(dp), eB.ctypes.data_as(dp),
                                                  edaa._ptr(E), edaa._ptr(A)), "edaa_unrolled_forward")
        ctx.eng = eng
        ctx.shape = (N, L, T)
        ctx.eta_dtype = eta_A.dtype
        ctx.save_for_backward(X)
        return E, A

    @staticmethod
    def backward(ctx, dE, dA):
        (X,) = ctx.saved_tensors
        N, L, T = ctx.shape
        dE = None if dE is None else dE.to(torch.float32).contiguous()
        dA = None if dA is None else dA.to(torch.float32).contiguous()
        dX = torch.empty((N, L), dtype=torch.float32, device=X.device)
        deA = np.zeros(T)
        deB = np.zeros(T)
        dp = ctypes.POINTER(ctypes.c_double)
        eng, ctx.eng = ctx.eng, None
        try:
            edaa._check(eng.lib.edaa_unrolled_backward(eng.h, edaa._ptr(dE), edaa._ptr(dA), edaa._ptr(dX),
                                                       deA.ctypes.data_as(dp), deB.ctypes.data_as(dp)),
                        "edaa_unrolled_backward")
        finally:
            eng.release()  # (the backward synchronises with the engine's stream before it returns)
        return (dX, torch.from_numpy(deA).to(ctx.eta_dtype), torch.from_numpy(deB).to(ctx.eta_dtype),
                None, None, None, None)


def unrolled(X, eta_A, eta_B, p: int, seed: int, K1: int = 5, K2: int = 5):
    return EDAAUnrolled.apply(X, eta_A, eta_B, p, seed, K1, K2)
