"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
published generator outputs, the paper's closed forms and hyper-parameters,
finite differences, brute force on tiny inputs, library routines reached by a
different route, and invariants the method guarantees.  Each test names the
passage it checks."""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import edaa_oracle as O
from paper_2209_11002_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(s=0):
    return np.random.default_rng(s)


def _simplex_cols(rng, rows, cols):
    Z = rng.gamma(1.0, size=(rows, cols))
    return Z / Z.sum(axis=0, keepdims=True)


def _small_X(rng, L=9, N=14):
    return O.normalize_pixels(np.abs(rng.standard_normal((L, N))) + 0.05)


# --- SplitMix64 (B^0 initialisation, eq. initB0) -----------------------------------

def test_splitmix64_published_sequence():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l[0] != "#"]
    n = np.array([int(r[0]) for r in rows], dtype=np.uint64)
    want = [int(r[1], 16) for r in rows]
    got = [int(v) for v in O.splitmix64(0, n)]
    assert got == want


def test_uniform_u_range_and_layout():
    u = O.uniform_u(12345, 1000, 3)
    assert u.shape == (1000, 3)
    assert u.min() >= 0.0 and u.max() < 1.0
    # 24-bit grid: every value times 2^24 is an integer
    assert np.all(np.floor(u * 2**24) == u * 2**24)
    # entry (i, j) is output i*p + j + 1
    z = O.splitmix64(12345, np.array([7 * 3 + 2 + 1], dtype=np.uint64))
    assert u[7, 2] == float(int(z[0]) >> 40) * 2.0**-24
    assert abs(u.mean() - 0.5) < 0.02


# --- Normalisation (Sec. III-C, eq. normalization) --------------------------------

def test_normalize_pixels():
    rng = _rng(1)
    X = rng.standard_normal((6, 5))
    X[:, 3] = 0.0
    Xn = O.normalize_pixels(X)
    norms = np.sqrt((Xn**2).sum(0))
    assert np.allclose(norms[[0, 1, 2, 4]], 1.0, atol=1e-15)
    assert np.all(Xn[:, 3] == 0.0)
    # direction preserved: Xn_i is a positive multiple of X_i
    for i in [0, 1, 2, 4]:
        c = X[:, i] @ Xn[:, i]
        assert c > 0 and np.allclose(X[:, i] / c * 1.0, Xn[:, i] / (Xn[:, i] @ Xn[:, i]))


# --- The mirror step (eqs. EMDA, update, update_softmax) --------------------------

def test_mirror_step_equals_quotient_form():
    """Eq. (update_softmax) equals the explicit quotient of eq. (update)."""
    rng = _rng(2)
    Z = _simplex_cols(rng, 5, 7)
    G = rng.standard_normal((5, 7)) * 3
    eta = 0.37
    want = Z * np.exp(-eta * G) / (Z * np.exp(-eta * G)).sum(0, keepdims=True)
    assert np.allclose(O.mirror_step(Z, G, eta), want, rtol=0, atol=1e-14)


def test_mirror_step_kkt_and_argmin():
    """z+ solves eq. (EMDA): log z+ - log z + eta g is constant over j (KKT),
    and no other simplex point has a lower EMDA objective."""
    rng = _rng(3)
    d = 4
    z = _simplex_cols(rng, d, 1)[:, 0]
    g = rng.standard_normal(d)
    eta = 0.8
    zp = O.mirror_step(z[:, None], g[:, None], eta)[:, 0]
    k = np.log(zp) - np.log(z) + eta * g
    assert np.ptp(k) < 1e-12

    def emda(y):
        y = np.asarray(y)
        kl = np.sum(np.where(y > 0, y * np.log(np.where(y > 0, y, 1) / z), 0.0)) - y.sum() + z.sum()
        return g @ (y - z) + kl / eta

    best = emda(zp)
    cands = rng.dirichlet(np.ones(d), size=20000)
    assert all(emda(c) >= best - 1e-12 for c in cands)
    for j in range(d):  # vertices
        assert emda(np.eye(d)[j]) >= best


def test_mirror_step_keeps_zero_entries():
    Z = np.array([[0.0, 0.5], [0.25, 0.5], [0.75, 0.0]])
    G = np.array([[-100.0, 1.0], [0.0, 2.0], [1.0, -50.0]])
    Zp = O.mirror_step(Z, G, 1.0)
    assert Zp[0, 0] == 0.0 and Zp[2, 1] == 0.0
    assert np.allclose(Zp.sum(0), 1.0, atol=1e-15)


# --- Gradients of the AA objective (eq. AA) against central differences ----------

@pytest.mark.parametrize("seed", [4, 5])
def test_grad_A_finite_differences(seed):
    rng = _rng(seed)
    X = _small_X(rng)
    L, N = X.shape
    p = 3
    A = _simplex_cols(rng, p, N)
    B = _simplex_cols(rng, N, p)
    f = lambda A_: 0.5 * O.objective(X, A_, B)
    G = O.grad_A(X, A, B)
    for _ in range(3):
        V = rng.standard_normal(A.shape)
        h = 1e-6
        fd = (f(A + h * V) - f(A - h * V)) / (2 * h)
        assert abs(fd - (G * V).sum()) <= 1e-7 * max(1.0, abs(fd))


@pytest.mark.parametrize("seed", [6, 7])
def test_grad_B_finite_differences(seed):
    rng = _rng(seed)
    X = _small_X(rng)
    L, N = X.shape
    p = 3
    A = _simplex_cols(rng, p, N)
    B = _simplex_cols(rng, N, p)
    f = lambda B_: 0.5 * O.objective(X, A, B_)
    G = O.grad_B(X, A, B)
    for _ in range(3):
        V = rng.standard_normal(B.shape)
        h = 1e-6
        fd = (f(B + h * V) - f(B - h * V)) / (2 * h)
        assert abs(fd - (G * V).sum()) <= 1e-7 * max(1.0, abs(fd))


def test_objective_brute_force():
    rng = _rng(8)
    X = _small_X(rng, 4, 5)
    A = _simplex_cols(rng, 2, 5)
    B = _simplex_cols(rng, 5, 2)
    s = 0.0
    for l in range(4):
        for i in range(5):
            v = X[l, i]
            for j in range(2):
                for k in range(5):
                    v -= X[l, k] * B[k, j] * A[j, i]
            s += v * v
    assert abs(O.objective(X, A, B) - s) < 1e-13


# --- Initialisation (eqs. initA0, initB0) and step sizes (eqs. eta0A, eta0B) ------

def test_init_values():
    A0 = O.init_A(4, 10)
    assert np.all(A0 == 0.25)
    B0 = O.init_B(O.uniform_u(99, 500, 3))
    assert np.allclose(B0.sum(0), 1.0, atol=1e-14)
    NB = 500 * B0
    assert NB.min() >= math.exp(-0.1) - 1e-12 and NB.max() <= math.exp(0.1) + 1e-12


def test_sigma_max_against_svd_and_rank_one():
    rng = _rng(9)
    M = rng.standard_normal((30, 4))
    assert abs(O.sigma_max_sq(M) - np.linalg.svd(M, compute_uv=False)[0] ** 2) < 1e-10
    u, v = rng.standard_normal(12), rng.standard_normal(3)
    assert abs(O.sigma_max_sq(np.outer(u, v)) - (u @ u) * (v @ v)) < 1e-10


def test_step_sizes_ratio():
    rng = _rng(10)
    X = _small_X(rng, 7, 40)
    B0 = O.init_B(O.uniform_u(5, 40, 3))
    e1, e2 = O.step_sizes(X, B0, 2.0)
    E0 = X @ B0
    assert abs(e1 - 2.0 / np.linalg.svd(E0, compute_uv=False)[0] ** 2) < 1e-12 * e1
    assert abs(e2 / e1 - math.sqrt(3 / 40)) < 1e-14


# --- Convergence of the A sub-problem (Sec. III-B.1): brute-force support search --

def _simplex_ls_bruteforce(E, x):
    """min_{a in simplex} 1/2 ||x - E a||^2 by enumerating supports (p <= 4)."""
    p = E.shape[1]
    G, c = E.T @ E, E.T @ x
    best, best_a = np.inf, None
    for r in range(1, p + 1):
        for S in itertools.combinations(range(p), r):
            S = list(S)
            K = np.zeros((r + 1, r + 1))
            K[:r, :r] = G[np.ix_(S, S)]
            K[:r, r] = 1.0
            K[r, :r] = 1.0
            rhs = np.concatenate([c[S], [1.0]])
            try:
                sol = np.linalg.solve(K, rhs)
            except np.linalg.LinAlgError:
                continue
            a = np.zeros(p)
            a[S] = sol[:r]
            if a.min() < -1e-12:
                continue
            val = 0.5 * np.sum((x - E @ a) ** 2)
            if val < best:
                best, best_a = val, a
    return best, best_a


def test_A_updates_converge_to_simplex_least_squares():
    rng = _rng(11)
    L, N, p = 8, 6, 3
    X = _small_X(rng, L, N)
    B = _simplex_cols(rng, N, p)
    B = np.where(B > 0.2, B, 0.02)
    B /= B.sum(0)
    E = X @ B
    A = O.init_A(p, N)
    eta = 1.0 / O.sigma_max_sq(E)
    for _ in range(20000):
        A = O.mirror_step(A, O.grad_A(X, A, B), eta)
    for i in range(N):
        val, a_star = _simplex_ls_bruteforce(E, X[:, i])
        got = 0.5 * np.sum((X[:, i] - E @ A[:, i]) ** 2)
        assert got - val <= 1e-9 * max(1.0, val) + 1e-12
        assert np.abs(A[:, i] - a_star).max() < 1e-3


def test_B_updates_decrease_to_qp_solution():
    """With A fixed, B-steps (eq. update_B) approach the minimiser of the convex
    B sub-problem, computed independently by scipy's SLSQP."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    rng = _rng(12)
    L, N, p = 5, 6, 2
    X = _small_X(rng, L, N)
    A = _simplex_cols(rng, p, N)
    f = lambda b: 0.5 * O.objective(X, A, b.reshape(N, p))
    cons = [{"type": "eq", "fun": (lambda b, j=j: b.reshape(N, p)[:, j].sum() - 1.0)} for j in range(p)]
    res = scipy_opt.minimize(f, np.full(N * p, 1.0 / N), method="SLSQP", bounds=[(0, 1)] * (N * p),
                             constraints=cons, options={"ftol": 1e-14, "maxiter": 1000})
    B = np.full((N, p), 1.0 / N)
    # l1-smoothness constant of the B sub-problem: the largest entry of its
    # Hessian (A A^T) kron (X^T X); KL is 1-strongly convex w.r.t. l1 (Pinsker).
    L1 = np.abs(A @ A.T).max() * np.abs(X.T @ X).max()
    for _ in range(30000):
        B = O.mirror_step(B, O.grad_B(X, A, B), 1.0 / L1)
    assert f(B.ravel()) - res.fun <= 1e-7 * max(1.0, res.fun)


# --- Monotone A-phase at the paper's step (gamma = 1) -----------------------------

def test_first_A_phase_is_monotone_at_gamma_one():
    """With eta1 = 1/sigma_max^2(X B^0) the A-step is a mirror step with a step no
    larger than 1/(l1-smoothness), so the objective cannot increase while B = B^0."""
    cube = synth.make_cube(20, 400, 3, alpha=0.5, snr_db=30, seed=21)
    X = O.normalize_pixels(cube.X)
    B = O.init_B(O.uniform_u(777, X.shape[1], 3))
    A = O.init_A(3, X.shape[1])
    eta1, _ = O.step_sizes(X, B, 1.0)
    prev = O.objective(X, A, B)
    for _ in range(50):
        A = O.mirror_step(A, O.grad_A(X, A, B), eta1)
        cur = O.objective(X, A, B)
        assert cur <= prev * (1 + 1e-13)
        prev = cur


# --- Algorithm 1 end to end ---------------------------------------------------------

def test_simplex_invariants_after_solve():
    cube = synth.make_cube(16, 300, 3, alpha=0.5, snr_db=30, seed=22)
    X = O.normalize_pixels(cube.X)
    r = O.edaa(X, 3, T=10, K1=5, K2=5, seed=5, gamma=1.0)
    for Z in (r["A"], r["B"]):
        assert Z.min() >= 0.0
        assert np.abs(Z.sum(0) - 1.0).max() < 1e-12
    assert np.allclose(r["E"], X @ r["B"], atol=1e-15)


def test_recovery_of_pure_pixel_archetypes():
    """Noiseless X = E A with one pure pixel per endmember and no normalisation:
    the archetypes are columns of X, so the AA optimum has zero loss.  EDAA's
    loss must fall by orders of magnitude and the endmembers must match."""
    cube = synth.make_cube(30, 500, 3, alpha=1.0, snr_db=None, pure=True, seed=23)
    X = cube.X.astype(np.float64)
    r = O.edaa(X, 3, T=300, K1=5, K2=5, seed=3, gamma=1.0, record=True)
    loss = r["hist"]["loss"]
    assert loss[-1] < 1e-3 * loss[0]
    # each true endmember is matched by an estimated one (spectral angle < 3 deg)
    En = r["E"] / np.linalg.norm(r["E"], axis=0)
    Et = cube.E_true / np.linalg.norm(cube.E_true, axis=0)
    ang = np.degrees(np.arccos(np.clip(Et.T @ En, -1, 1)))
    best = min(sum(ang[j, perm[j]] for j in range(3)) for perm in itertools.permutations(range(3)))
    assert best / 3 < 3.0


def test_history_is_consistent():
    cube = synth.make_cube(12, 200, 2, alpha=0.5, snr_db=30, seed=24)
    X = O.normalize_pixels(cube.X)
    r = O.edaa(X, 2, T=3, K1=2, K2=2, seed=9, gamma=1.0, record=True)
    h = r["hist"]
    assert len(h["loss"]) == 4
    assert abs(h["loss"][-1] - O.objective(X, r["A"], r["B"])) < 1e-12
    assert np.allclose(h["gA"][0], 2 * O.grad_A(X, O.init_A(2, 200), O.init_B(O.uniform_u(9, 200, 2))))


# --- Fit, coherence and Algorithm 2 ------------------------------------------------

def test_fit_l1_brute_force():
    rng = _rng(30)
    X = rng.standard_normal((3, 4))
    E = rng.standard_normal((3, 2))
    A = rng.standard_normal((2, 4))
    s, cols = 0.0, []
    for i in range(4):
        c = 0.0
        for l in range(3):
            c += abs(X[l, i] - E[l, 0] * A[0, i] - E[l, 1] * A[1, i])
        s += c
        cols.append(c)
    assert abs(O.fit_l1(X, E, A, 0) - s) < 1e-13
    assert abs(O.fit_l1(X, E, A, 1) - max(cols)) < 1e-13


def test_coherence_cases():
    assert O.coherence(np.eye(4)[:, :3]) == 0.0
    E = np.array([[1.0, 2.0], [0.0, 0.0]])
    assert abs(O.coherence(E) - 1.0) < 1e-15
    E = np.array([[3.0, 1.0], [4.0, 1.0]])
    assert abs(O.coherence(E) - 7.0 / (5.0 * math.sqrt(2))) < 1e-15
    assert O.coherence(E, mode=1) == 7.0
    assert O.coherence(np.ones((5, 1))) == float("-inf")


def test_algorithm2_selection_rule():
    # threshold is inclusive: 10.5 == 1.05 * 10 is in the subset
    assert O.select([10.0, 10.5, 11.0], [0.9, 0.2, 0.1]) == 1
    # outside the threshold, lower coherence does not win
    assert O.select([10.0, 10.51, 11.0], [0.9, 0.2, 0.1]) == 0
    # ties in coherence go to the lowest index
    assert O.select([10.0, 10.2, 10.1], [0.5, 0.3, 0.3]) == 1
    # non-finite fits are excluded
    assert O.select([float("nan"), 10.0, 10.4], [0.0, 0.5, 0.4]) == 2
    assert O.select([float("nan"), float("inf")], [0.0, 0.1]) == -1
    assert O.select([10.0, 10.4], [0.4, 0.4], ratio=1.0) == 0


def test_paper_hyperparameters_fixture():
    vals = {}
    for l in open(os.path.join(GOLDEN, "paper_hyperparameters.txt")):
        if l.strip() and l[0] != "#":
            k, *v = l.split()
            vals[k] = [float(x) for x in v]
    assert tuple(vals["S"]) == synth.GAMMA_SET
    B0 = O.init_B(np.ones((10, 2)))
    assert np.allclose(B0, 0.1)  # softmax of a constant column is uniform
    assert vals["fit_ratio"] == [1.05]
