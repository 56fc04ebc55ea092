"""Second, independent FP64 restatement of Algorithm 1 in plain PyTorch CPU ops,
used as the reference gradient of the unrolled solve.

TEST INFRASTRUCTURE ONLY (see edaa_oracle.py's header for who may import it).
It shares no code with edaa_oracle.py or with the CUDA library.

The unrolled solve has one step size per block: eta_A[t] for the K1 A-steps
and eta_B[t] for the K2 B-steps of outer iteration t (Algorithm 1).  The
updates are eqs. (update_A) and (update_B) written as
    log z+ = log_softmax(log z - eta * grad)
which is eq. (update_softmax) taken in log space; A^0 = 1/p (eq. initA0) and
B^0 = softmax(0.1 u) (eq. initB0) with u supplied by the caller.
Autograd through this function gives d(loss)/dX and d(loss)/d(eta).
"""
from __future__ import annotations

import torch


def unrolled_edaa(X: torch.Tensor, u: torch.Tensor, eta_A: torch.Tensor, eta_B: torch.Tensor,
                  K1: int, K2: int):
    """X: L x N float64 (already normalised), u: N x p, eta_A/eta_B: length T.
    Returns (E_hat = X B_hat, A_hat)."""
    L, N = X.shape
    p = u.shape[1]
    T = eta_A.shape[0]
    logA = torch.full((p, N), -torch.log(torch.tensor(float(p), dtype=X.dtype)).item(), dtype=X.dtype)
    logB = torch.log_softmax(0.1 * u.to(X.dtype), dim=0)
    for t in range(T):
        B = torch.exp(logB)
        for _ in range(K1):
            A = torch.exp(logA)
            E = X @ B
            G = E.t() @ (E @ A - X)                  # -(B^T X^T (X - X B A))
            logA = torch.log_softmax(logA - eta_A[t] * G, dim=0)
        A = torch.exp(logA)
        for _ in range(K2):
            B = torch.exp(logB)
            E = X @ B
            G = X.t() @ ((E @ A - X) @ A.t())        # -(X^T (X - X B A) A^T)
            logB = torch.log_softmax(logB - eta_B[t] * G, dim=0)
    return X @ torch.exp(logB), torch.exp(logA)
