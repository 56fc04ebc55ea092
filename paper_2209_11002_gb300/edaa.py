"""Python binding of libedaa (include/edaa.h): argument marshalling only.

Every step of EDAA runs in the CUDA library; this module converts arrays and
tensors to pointers, keeps inputs alive while the library may still read
them, and raises EDAAError on a non-zero status.  There is no CPU fallback:
if libedaa.so is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libedaa.so")

EDAA_OK, EDAA_ERR_ARG, EDAA_ERR_CUDA, EDAA_ERR_OOM, EDAA_ERR_STATE, EDAA_ERR_NONFINITE, \
    EDAA_ERR_TIMEOUT, EDAA_ERR_UNSUPPORTED = range(8)
STATUS_NAMES = ["EDAA_OK", "EDAA_ERR_ARG", "EDAA_ERR_CUDA", "EDAA_ERR_OOM", "EDAA_ERR_STATE",
                "EDAA_ERR_NONFINITE", "EDAA_ERR_TIMEOUT", "EDAA_ERR_UNSUPPORTED"]
FP32, TF32, BF16, TF32X3 = 0, 1, 2, 3

# Every function declared in include/edaa.h (the CPU tests check the export list).
EXPORTS = ["edaa_config_default", "edaa_init", "edaa_reset", "edaa_step", "edaa_solve", "edaa_select",
           "edaa_select_rule", "edaa_get", "edaa_grad", "edaa_loss", "edaa_step_sizes", "edaa_sync",
           "edaa_outer_done", "edaa_describe", "edaa_destroy", "edaa_last_error", "edaa_selftest_barrier",
           "edaa_fit_eval_static", "edaa_unrolled_create", "edaa_unrolled_forward", "edaa_unrolled_backward",
           "edaa_unrolled_destroy", "edaa_trace_read", "edaa_describe_tile", "edaa_measure_fma_peak", "edaa_debug_fail_alloc",
           "edaa_loss_history", "edaa_checkpoint", "edaa_restore"]


class Config(ctypes.Structure):
    _fields_ = [("T", ctypes.c_int), ("K1", ctypes.c_int), ("K2", ctypes.c_int), ("normalize", ctypes.c_int),
                ("precision", ctypes.c_int), ("fit_norm", ctypes.c_int), ("coherence", ctypes.c_int),
                ("fit_ratio", ctypes.c_double), ("persistent", ctypes.c_int), ("autotune", ctypes.c_int),
                ("barrier_timeout_ms", ctypes.c_double), ("center", ctypes.c_int), ("trace", ctypes.c_int),
                ("tile", ctypes.c_int * 4), ("record_loss", ctypes.c_int)]


class CubeDesc(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("L", ctypes.c_int), ("N", ctypes.c_int), ("p", ctypes.c_int),
                ("M", ctypes.c_int), ("seeds", ctypes.POINTER(ctypes.c_uint64)),
                ("gammas", ctypes.POINTER(ctypes.c_double))]


class EDAAError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {msg}")


_lib = None


def load_library():
    """Loads libedaa.so from the package (built by build.build_library)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2209_11002_gb300.build.build_library()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    sig = {
        "edaa_config_default": (None, [ctypes.POINTER(Config)]),
        "edaa_init": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.POINTER(CubeDesc), ctypes.c_int,
                                     ctypes.POINTER(Config), vp]),
        "edaa_reset": (ctypes.c_int, [vp, ctypes.c_int, vp]),
        "edaa_step": (ctypes.c_int, [vp, ctypes.c_int]),
        "edaa_solve": (ctypes.c_int, [vp]),
        "edaa_select": (ctypes.c_int, [vp, ctypes.c_int, ip, dp, dp]),
        "edaa_select_rule": (ctypes.c_int, [dp, dp, ctypes.c_int, ctypes.c_double]),
        "edaa_get": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp]),
        "edaa_grad": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, vp, vp]),
        "edaa_loss": (ctypes.c_int, [vp, ctypes.c_int, dp]),
        "edaa_step_sizes": (ctypes.c_int, [vp, ctypes.c_int, dp, dp]),
        "edaa_sync": (ctypes.c_int, [vp]),
        "edaa_outer_done": (ctypes.c_int, [vp]),
        "edaa_describe": (ctypes.c_int, [vp, ctypes.c_int, ip, ip, ip, ip, ip, ip]),
        "edaa_destroy": (None, [vp]),
        "edaa_last_error": (ctypes.c_char_p, []),
        "edaa_selftest_barrier": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, vp]),
        "edaa_fit_eval_static": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp,
                                                vp, vp, vp, vp]),
        "edaa_unrolled_create": (ctypes.c_int, [ctypes.POINTER(vp)] + [ctypes.c_int] * 6 + [vp]),
        "edaa_unrolled_forward": (ctypes.c_int, [vp, vp, ctypes.c_uint64, dp, dp, vp, vp]),
        "edaa_unrolled_backward": (ctypes.c_int, [vp, vp, vp, vp, dp, dp]),
        "edaa_unrolled_destroy": (None, [vp]),
        "edaa_trace_read": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ip, ip, dp, dp]),
        "edaa_describe_tile": (ctypes.c_int, [vp, ctypes.c_int, ip]),
        "edaa_measure_fma_peak": (ctypes.c_int, [dp, vp]),
        "edaa_debug_fail_alloc": (None, [ctypes.c_int]),
        "edaa_loss_history": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, dp, ip]),
        "edaa_checkpoint": (ctypes.c_int, [vp, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
        "edaa_restore": (ctypes.c_int, [vp, vp, ctypes.c_size_t]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(st: int, where: str):
    if st != EDAA_OK:
        raise EDAAError(st, where, load_library().edaa_last_error().decode())


def default_config(**overrides) -> Config:
    cfg = Config()
    load_library().edaa_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        if not hasattr(cfg, k):
            raise KeyError(k)
        if k == "tile":  # (runs per group, phase-1 pixel warps, pixels per lane, phase-2 pixel warps)
            v = (ctypes.c_int * 4)(*[int(x) for x in v])
        setattr(cfg, k, v)
    return cfg


def _ptr(x):
    """Data pointer of a torch tensor or numpy array (kept alive by the caller)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return ctypes.c_void_p(x.ctypes.data)


def _as_pixel_major(X):
    """N x L float32 contiguous (torch tensor on any device, or numpy)."""
    if hasattr(X, "data_ptr"):
        import torch
        return X.to(torch.float32).contiguous()
    return np.ascontiguousarray(X, dtype=np.float32)


def select_rule(fit: Sequence[float], mu: Sequence[float], ratio: float = 1.05) -> int:
    """Algorithm 2's rule in the library's host code (no device work)."""
    f = np.ascontiguousarray(fit, dtype=np.float64)
    m = np.ascontiguousarray(mu, dtype=np.float64)
    lib = load_library()
    return lib.edaa_select_rule(f.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                m.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(f), ratio)


class Context:
    """One EDAA problem set (one or more cubes, each with M runs) on the GPU.

    cubes: list of dicts with keys X (N x L pixel-major float32, torch tensor
    or numpy array), p, seeds (M uint64), gammas (M float)."""

    def __init__(self, cubes: List[Dict], stream=None, **cfg):
        self.lib = load_library()
        self.cfg = default_config(**cfg)
        self._keep = []
        descs = (CubeDesc * len(cubes))()
        self.shapes = []
        for i, c in enumerate(cubes):
            X = _as_pixel_major(c["X"])
            N, L = X.shape
            seeds = np.ascontiguousarray(c["seeds"], dtype=np.uint64)
            gammas = np.ascontiguousarray(c["gammas"], dtype=np.float64)
            self._keep += [X, seeds, gammas]
            descs[i].X = _ptr(X)
            descs[i].L, descs[i].N, descs[i].p, descs[i].M = L, N, int(c["p"]), len(seeds)
            descs[i].seeds = seeds.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
            descs[i].gammas = gammas.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            self.shapes.append((L, N, int(c["p"]), len(seeds)))
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self.stream = ctypes.c_void_p(stream) if stream else None
        h = ctypes.c_void_p()
        _check(self.lib.edaa_init(ctypes.byref(h), descs, len(cubes), ctypes.byref(self.cfg), self.stream),
               "edaa_init")
        self.h = h

    # -- lifecycle --------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            self.lib.edaa_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- compute ----------------------------------------------------------
    def reset(self, cube: int = -1, X=None):
        if X is not None:
            X = _as_pixel_major(X)
            self._keep.append(X)
        _check(self.lib.edaa_reset(self.h, cube, _ptr(X)), "edaa_reset")

    def step(self, n_outer: int = 1):
        _check(self.lib.edaa_step(self.h, n_outer), "edaa_step")

    def solve(self):
        _check(self.lib.edaa_solve(self.h), "edaa_solve")

    def sync(self):
        _check(self.lib.edaa_sync(self.h), "edaa_sync")
        self._keep = self._keep[:3 * len(self.shapes)]

    def select(self, cube: int = 0):
        M = self.shapes[cube][3]
        fit = np.zeros(M)
        mu = np.zeros(M)
        best = ctypes.c_int(-1)
        _check(self.lib.edaa_select(self.h, cube, ctypes.byref(best),
                                    fit.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "edaa_select")
        return best.value, fit, mu

    def outer_done(self) -> int:
        return self.lib.edaa_outer_done(self.h)

    # -- outputs ----------------------------------------------------------
    def _out(self, shape, device):
        if device == "cpu":
            return np.zeros(shape, dtype=np.float32)
        import torch
        return torch.empty(shape, dtype=torch.float32, device=device)

    def get(self, cube: int = 0, run: int = 0, device="cuda"):
        """(E L x p, A p x N, B N x p) of one run."""
        L, N, p, M = self.shapes[cube]
        E, A, B = self._out((L, p), device), self._out((p, N), device), self._out((N, p), device)
        _check(self.lib.edaa_get(self.h, cube, run, _ptr(E), _ptr(A), _ptr(B)), "edaa_get")
        return E, A, B

    def grad(self, cube: int = 0, run: int = 0, device="cuda"):
        """(2(E^T E A - E^T X) p x N, 2 X^T(E A A^T - X A^T) N x p) at the current state."""
        L, N, p, M = self.shapes[cube]
        gA, gB = self._out((p, N), device), self._out((N, p), device)
        _check(self.lib.edaa_grad(self.h, cube, run, _ptr(gA), _ptr(gB)), "edaa_grad")
        return gA, gB

    def loss(self, cube: int = 0) -> np.ndarray:
        M = self.shapes[cube][3]
        out = np.zeros(M)
        _check(self.lib.edaa_loss(self.h, cube, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "edaa_loss")
        return out

    def checkpoint(self) -> bytes:
        """The iteration state of every run (edaa_checkpoint), as bytes."""
        n = ctypes.c_size_t()
        _check(self.lib.edaa_checkpoint(self.h, None, 0, ctypes.byref(n)), "edaa_checkpoint")
        buf = ctypes.create_string_buffer(n.value)
        _check(self.lib.edaa_checkpoint(self.h, buf, n.value, ctypes.byref(n)), "edaa_checkpoint")
        return buf.raw

    def restore(self, state: bytes):
        """Resume from a checkpoint of a context with the same cubes and X (edaa_restore)."""
        _check(self.lib.edaa_restore(self.h, state, len(state)), "edaa_restore")

    def loss_history(self, cube: int = 0) -> np.ndarray:
        """(outer iterations recorded) x M losses, row t after outer iteration
        t + 1 (needs record_loss=1)."""
        M = self.shapes[cube][3]
        n = ctypes.c_int()
        _check(self.lib.edaa_loss_history(self.h, cube, 0, None, ctypes.byref(n)), "edaa_loss_history")
        out = np.zeros((n.value, M))
        _check(self.lib.edaa_loss_history(self.h, cube, n.value, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          ctypes.byref(n)), "edaa_loss_history")
        return out

    def step_sizes(self, cube: int = 0):
        M = self.shapes[cube][3]
        e1, e2 = np.zeros(M), np.zeros(M)
        _check(self.lib.edaa_step_sizes(self.h, cube, e1.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        e2.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "edaa_step_sizes")
        return e1, e2

    PHASE_NAMES = ["A-pass", "A-merge", "B-pass", "B-merge", "initial B-pass", "initial A-pass", "step sizes",
                   "fit pass", "fit merge", "first B-merge"]

    def trace(self, which: int = 0):
        """Phase trace of the last launch sequence (needs trace=1): which 0 =
        outer iterations, 1 = initialisation, 2 = fit.  Returns (phase ids,
        start us, duration us) as numpy arrays."""
        cap = 4096
        ph, t0, dt, n = np.zeros(cap, np.int32), np.zeros(cap), np.zeros(cap), ctypes.c_int()
        _check(self.lib.edaa_trace_read(self.h, which, cap, ctypes.byref(n),
                                        ph.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                        t0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        dt.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "edaa_trace_read")
        k = min(n.value, cap)
        return ph[:k], t0[:k], dt[:k]

    def describe(self, cube: int = 0) -> Dict[str, int]:
        vals = [ctypes.c_int() for _ in range(6)]
        _check(self.lib.edaa_describe(self.h, cube, *[ctypes.byref(v) for v in vals]), "edaa_describe")
        keys = ["runs_per_group", "pixel_tile", "ctas_per_group", "grid", "launches_per_solve", "graph"]
        out = {k: v.value for k, v in zip(keys, vals)}
        tile = (ctypes.c_int * 4)()
        _check(self.lib.edaa_describe_tile(self.h, cube, tile), "edaa_describe_tile")
        out["tile"] = tuple(tile)  # the edaa_config.tile form of the CUDA-core launch shape
        return out


def fit_eval_static(X, E, A, stream=None):
    """Fit, max-column fit and loss of M given solutions through the
    allocation-free entry point.  X: N x L, E: M x L x p, A: M x p x N, all
    CUDA tensors (float32).  The library allocates nothing for this call; the
    three FP64 output vectors are allocated here by torch."""
    import torch
    N, L = X.shape
    M, _, p = E.shape
    out = torch.zeros((3, M), dtype=torch.float64, device=X.device)
    lib = load_library()
    s = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else stream) if stream else None
    _check(lib.edaa_fit_eval_static(_ptr(X), L, N, p, M, _ptr(E), _ptr(A), _ptr(out[0]), _ptr(out[1]),
                                    _ptr(out[2]), s), "edaa_fit_eval_static")
    return out[0], out[1], out[2]


def measure_fma_peak(stream=None) -> float:
    """FP32 FMA throughput of the current device in TFLOP/s (edaa_measure_fma_peak)."""
    lib = load_library()
    out = ctypes.c_double(0.0)
    s = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else stream) if stream else None
    _check(lib.edaa_measure_fma_peak(ctypes.byref(out), s), "edaa_measure_fma_peak")
    return out.value


def selftest_barrier(grid: int, extra: int, timeout_ms: float, stream=None) -> int:
    """Runs the bounded grid barrier with `extra` missing arrivals; returns the status."""
    lib = load_library()
    return lib.edaa_selftest_barrier(grid, extra, timeout_ms, ctypes.c_void_p(stream) if stream else None)


def solve(X, p: int, seeds: Sequence[int], gammas: Sequence[float], stream=None, **cfg) -> Dict:
    """Algorithm 2 around Algorithm 1 for one cube: returns the selected run's
    E, A, B and every run's fit and coherence."""
    with Context([dict(X=X, p=p, seeds=seeds, gammas=gammas)], stream=stream, **cfg) as ctx:
        ctx.solve()
        best, fit, mu = ctx.select(0)
        E, A, B = ctx.get(0, best)
        return {"best": best, "fit": fit, "mu": mu, "E": E, "A": A, "B": B}
