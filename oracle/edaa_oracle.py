"""Plain FP64 CPU oracle for Entropic Descent Archetypal Analysis (EDAA).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module:
only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
leg may call it.  It shares no code with the CUDA library.

Everything is written in the paper's notation and orientation: X is L x N
(bands x pixels), A is p x N, B is N x p, E = X B is L x p.  Each function
follows one passage of the paper (Zouaoui et al., "Entropic Descent
Archetypal Analysis for Blind Hyperspectral Unmixing", arXiv 2209.11002) and
performs the steps in the paper's order, with numpy matmul as the only
library primitive.

Readings taken where the paper is silent or ambiguous:
  * Step scale: the objective is 1/2||X - XBA||_F^2 (eq. AA) and the updates
    (eqs. update_A, update_B) use its gradient, so the exponent is
    -eta * (E^T E A - E^T X) for A and -eta * X^T (E A A^T - X A^T) for B.
    `grad_A` / `grad_B` return these half-scale gradients; callers that want
    the 2(...) gradient of the unhalved loss multiply by 2.
  * A zero pixel stays zero under the l2 normalisation (eq. normalization).
  * B^0 draws u ~ U[0,1) from SplitMix64 (Steele, Lea & Flood 2014): for run
    seed s, entry (i, j) of the N x p matrix uses output number i*p + j + 1 of
    the generator seeded with s, keeping its top 24 bits: u = (z >> 40) 2^-24.
  * sigma_max is per run (B^0 depends on the run's seed), eq. (eta0A).
  * The fit is the entrywise l1 norm sum |X - E A| (Algorithm 2); the
    induced (max column sum) norm is available as a flag.
  * Coherence (eq. coherence) is the largest cosine between distinct
    columns of E; the raw inner product is available as a flag.  p = 1 gives
    coherence -inf.
  * Algorithm 2's threshold is inclusive; ties in the argmin go to the lowest
    index; runs whose fit is not finite are excluded.
Parity pins for every function live in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional, Sequence

import numpy as np

# ---------------------------------------------------------------------------
# SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): state advances by the golden
# gamma; each output is the state passed through the variant-13 finaliser.
# ---------------------------------------------------------------------------
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MUL1 = np.uint64(0xBF58476D1CE4E5B9)
_MUL2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: np.ndarray) -> np.ndarray:
    """Output number n (n >= 1) of SplitMix64 seeded with `seed` (uint64 array)."""
    n = np.asarray(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.full(n.shape, np.uint64(seed), dtype=np.uint64) + n * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _MUL1
        z = (z ^ (z >> np.uint64(27))) * _MUL2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_u(seed: int, N: int, p: int) -> np.ndarray:
    """u ~ U[0,1)^{N x p} for eq. (initB0): top 24 bits of SplitMix64 outputs."""
    n = np.arange(1, N * p + 1, dtype=np.uint64).reshape(N, p)
    z = splitmix64(seed, n)
    return (z >> np.uint64(40)).astype(np.float64) * 2.0 ** -24


# ---------------------------------------------------------------------------
# Sec. III-C, "Normalization": every pixel (column of X) is divided by its
# l2 norm.
# ---------------------------------------------------------------------------
def normalize_pixels(X: np.ndarray) -> np.ndarray:
    X = np.asarray(X, dtype=np.float64)
    norms = np.sqrt((X * X).sum(axis=0))
    out = X.copy()
    keep = norms > 0
    out[:, keep] = X[:, keep] / norms[keep]
    return out


# ---------------------------------------------------------------------------
# Softmax along the first dimension (Algorithm 1 comment) with the usual max
# subtraction; -inf entries (log 0) map to 0.
# ---------------------------------------------------------------------------
def softmax_columns(Z: np.ndarray) -> np.ndarray:
    Z = np.asarray(Z, dtype=np.float64)
    m = Z.max(axis=0, keepdims=True)
    W = np.exp(Z - m)
    return W / W.sum(axis=0, keepdims=True)


def safe_log(Z: np.ndarray) -> np.ndarray:
    with np.errstate(divide="ignore"):
        return np.log(Z)


# ---------------------------------------------------------------------------
# Eq. (update_softmax): z+ = softmax(log z - eta * grad), applied per column.
# ---------------------------------------------------------------------------
def mirror_step(Z: np.ndarray, G: np.ndarray, eta: float) -> np.ndarray:
    return softmax_columns(safe_log(Z) - eta * G)


# ---------------------------------------------------------------------------
# Gradients of 1/2 ||X - X B A||_F^2 (eq. AA), as they appear (with a minus
# sign) inside eqs. (update_A) and (update_B).
# ---------------------------------------------------------------------------
def grad_A(X: np.ndarray, A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """-(B^T X^T (X - X B A)), p x N."""
    E = X @ B
    return -(E.T @ (X - E @ A))


def grad_B(X: np.ndarray, A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """-(X^T (X - X B A) A^T), N x p.  Parenthesised as X^T ((X - XBA) A^T)."""
    E = X @ B
    return -(X.T @ ((X - E @ A) @ A.T))


def objective(X: np.ndarray, A: np.ndarray, B: np.ndarray) -> float:
    """||X - X B A||_F^2 (unhalved; the paper's eq. AA carries a 1/2)."""
    Rz = X - (X @ B) @ A
    return float((Rz * Rz).sum())


# ---------------------------------------------------------------------------
# Initialisation, eqs. (initA0), (initB0); step sizes, eqs. (eta0A), (eta0B).
# ---------------------------------------------------------------------------
def init_A(p: int, N: int) -> np.ndarray:
    return np.full((p, N), 1.0 / p)


def init_B(u: np.ndarray) -> np.ndarray:
    return softmax_columns(0.1 * np.asarray(u, dtype=np.float64))


def sigma_max_sq(M: np.ndarray) -> float:
    """Largest squared singular value: top eigenvalue of the Gram matrix M^T M."""
    return float(np.linalg.eigvalsh(M.T @ M)[-1])


def step_sizes(X: np.ndarray, B0: np.ndarray, gamma: float) -> tuple:
    N = X.shape[1]
    p = B0.shape[1]
    eta1 = gamma / sigma_max_sq(X @ B0)
    eta2 = math.sqrt(p / N) * eta1
    return eta1, eta2


# ---------------------------------------------------------------------------
# Algorithm 1 (EDAA).
# ---------------------------------------------------------------------------
def edaa(X: np.ndarray, p: int, T: int, K1: int, K2: int, seed: int, gamma: float = 1.0,
         record: bool = False, A0: Optional[np.ndarray] = None, B0: Optional[np.ndarray] = None,
         eta_A: Optional[Sequence[float]] = None, eta_B: Optional[Sequence[float]] = None) -> Dict:
    """Run Algorithm 1 on an already-normalised X.

    Step sizes are eqs. (eta0A)/(eta0B) unless per-block values are given:
    eta_A[t] for the K1 A-steps and eta_B[t] for the K2 B-steps of outer
    iteration t (used by the unrolled, differentiable solve).

    Returns a dict with E, A, B, eta1, eta2 and, when `record`, per outer
    iteration t = 0..T the state's objective and the 2(...) gradients at the
    start of iteration t+1 (t = T: the final state)."""
    X = np.asarray(X, dtype=np.float64)
    L, N = X.shape
    A = init_A(p, N) if A0 is None else np.array(A0, dtype=np.float64)
    B = init_B(uniform_u(seed, N, p)) if B0 is None else np.array(B0, dtype=np.float64)
    eta1, eta2 = step_sizes(X, B, gamma)
    etaA = [eta1] * T if eta_A is None else [float(v) for v in eta_A]
    etaB = [eta2] * T if eta_B is None else [float(v) for v in eta_B]
    hist = {"loss": [], "gA": [], "gB": [], "A": [], "B": []}

    def snap():
        hist["loss"].append(objective(X, A, B))
        hist["gA"].append(2.0 * grad_A(X, A, B))
        hist["gB"].append(2.0 * grad_B(X, A, B))
        hist["A"].append(A.copy())
        hist["B"].append(B.copy())

    for t in range(T):
        if record:
            snap()
        for _ in range(K1):
            A = mirror_step(A, grad_A(X, A, B), etaA[t])
        for _ in range(K2):
            B = mirror_step(B, grad_B(X, A, B), etaB[t])
    if record:
        snap()
    E = X @ B
    out = {"E": E, "A": A, "B": B, "eta1": eta1, "eta2": eta2}
    if record:
        out["hist"] = hist
    return out


# ---------------------------------------------------------------------------
# Model selection (Sec. III-D, eq. coherence, Algorithm 2).
# ---------------------------------------------------------------------------
def fit_l1(X: np.ndarray, E: np.ndarray, A: np.ndarray, mode: int = 0) -> float:
    """||X - E A||_1: entrywise sum (mode 0) or induced max column sum (mode 1)."""
    Rz = np.abs(X - E @ A)
    return float(Rz.sum()) if mode == 0 else float(Rz.sum(axis=0).max())


def coherence(E: np.ndarray, mode: int = 0) -> float:
    """max_{k != k'} <e_k, e_k'> over normalised columns (mode 0) or raw (mode 1)."""
    E = np.asarray(E, dtype=np.float64)
    p = E.shape[1]
    if p < 2:
        return float("-inf")
    if mode == 0:
        nrm = np.sqrt((E * E).sum(axis=0))
        nrm[nrm == 0] = 1.0
        E = E / nrm
    G = E.T @ E
    off = ~np.eye(p, dtype=bool)
    return float(G[off].max())


def select(fits: Sequence[float], mus: Sequence[float], ratio: float = 1.05) -> int:
    """Algorithm 2's rule: among runs with fit <= ratio * min fit, the lowest
    coherence; ties go to the lowest index; non-finite fits are excluded.
    Returns -1 when no run has a finite fit."""
    fits = [float(f) for f in fits]
    finite = [m for m, f in enumerate(fits) if math.isfinite(f)]
    if not finite:
        return -1
    fmin = min(fits[m] for m in finite)
    subset = [m for m in finite if fits[m] <= ratio * fmin]
    best = subset[0]
    for m in subset[1:]:
        if mus[m] < mus[best]:
            best = m
    return best
