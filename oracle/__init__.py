"""FP64 oracle for the grid point-process GLM (Zaytsev, Morrison & Deger).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
definition that the CUDA library is checked against.  Only the test suite,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline / reference leg
may import it; the library never does, and it shares no code with the library.

What each function follows:
  * ``filter``        Eq. 13 on the grid (exponential kernel, one-bin delay)
  * ``eval_rows``     Eq. 2/7 (log-likelihood), Eq. 11-12 (gradient in W and
                      b), and the derivative in tau through Y = dX/da
  * ``fit``           Sec. 2.6.3 (per-row L-BFGS; Armijo backtracking and the
                      relative-change stop |dL_i|/|L_i| < eta)
  * ``classify``      Sec. 3.1 (3-component GMM by EM) and Sec. 3.3 (k-means,
                      k = 3), misclassification rate Eq. 20 / Table 2
Parity pins for every function live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .classify import chance_mer, classify, gmm1d, kmeans1d, mer_breakdown  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "glm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libglm_oracle.so")
_lock = threading.Lock()
_lib = None

FIT_CONVERGED, FIT_MAXITER, FIT_STALLED, FIT_DEGENERATE = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP, FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
            lib.oracle_filter.argtypes = [i32, i64, f64, f64, vp, vp, vp, i32]
            lib.oracle_filter.restype = ctypes.c_int
            lib.oracle_eval_rows.argtypes = [i32, i64, f64, f64, vp, vp, vp, vp, i32, vp, vp, vp, vp, vp, i32]
            lib.oracle_eval_rows.restype = ctypes.c_int
            lib.oracle_fit.argtypes = [i32, i64, f64, f64, vp, vp, i32, i32, i32, f64, f64, i32, f64, f64, vp, vp,
                                       vp, vp, i32, i32, vp]
            lib.oracle_fit.restype = ctypes.c_int
            _lib = lib
    return _lib


def _spikes(offs, bins):
    offs = np.ascontiguousarray(offs, dtype=np.int64)
    bins = np.ascontiguousarray(bins, dtype=np.int32)
    if bins.size == 0:
        bins = np.zeros(1, dtype=np.int32)
    return offs, bins


def filter(offs, bins, n_bins: int, dt: float, tau: float, threads: int = 0) -> np.ndarray:
    """X (n x T, float64): X_j[0] = 0, X_j[t] = a X_j[t-1] + S_j[t-1], a = exp(-dt/tau)  (Eq. 13)."""
    offs, bins = _spikes(offs, bins)
    n = offs.size - 1
    X = np.empty((n, int(n_bins)), dtype=np.float64)
    rc = _load().oracle_filter(n, int(n_bins), dt, tau, offs.ctypes.data, bins.ctypes.data, X.ctypes.data,
                               threads)
    if rc != 0:
        raise ValueError(f"oracle_filter: invalid input ({rc})")
    return X


def eval_rows(offs, bins, n_bins: int, dt: float, tau: float, W, b, rows=None, *, grad: bool = True,
              threads: int = 0) -> dict:
    """L_i, dL_i/dW_i., dL_i/db_i and row i's share of dL/dtau for the listed rows (all rows by default).

    Streams over the bins without storing X, so it runs at any size; cost is O(T * n * len(rows))."""
    offs, bins = _spikes(offs, bins)
    n = offs.size - 1
    W = np.ascontiguousarray(W, dtype=np.float64).reshape(n, n)
    b = np.ascontiguousarray(b, dtype=np.float64).reshape(n)
    rows = np.arange(n, dtype=np.int32) if rows is None else np.ascontiguousarray(rows, dtype=np.int32)
    r = rows.size
    L = np.zeros(r)
    G = np.zeros((r, n)) if grad else None
    gb = np.zeros(r)
    gt = np.zeros(r)
    rc = _load().oracle_eval_rows(n, int(n_bins), dt, tau, offs.ctypes.data, bins.ctypes.data, W.ctypes.data,
                                  b.ctypes.data, r, rows.ctypes.data, L.ctypes.data,
                                  G.ctypes.data if grad else None, gb.ctypes.data, gt.ctypes.data, threads)
    if rc != 0:
        raise ValueError(f"oracle_eval_rows failed ({rc})")
    return dict(rows=rows, L=L, G=G, gb=gb, gtau_rows=gt, L_total=float(L.sum()), gtau=float(gt.sum()))


def loglik_grad(offs, bins, n_bins: int, dt: float, tau: float, W, b, threads: int = 0) -> dict:
    """Whole-network log-likelihood L = sum_i L_i (Eq. 1) with its gradient and dL/dtau."""
    return eval_rows(offs, bins, n_bins, dt, tau, W, b, None, grad=True, threads=threads)


def fit(offs, bins, n_bins: int, dt: float, tau: float, *, method: str = "lbfgs", m: int = 10,
        max_iter: int = 500, eta: float = 1e-10, c1: float = 1e-4, max_halvings: int = 60,
        alpha: float = 0.0, eps: float = 1e-6, threads: int = 0, rows=None) -> dict:
    """Maximum-likelihood W, b, one independent row at a time (Sec. 2.2 separability, Sec. 2.6.3); with
    alpha > 0 the maximum a posteriori estimate under the smooth l1 penalty alpha sum_{j != i}
    sqrt(W_ij^2 + eps) (Sec. 2.5, Eq. 16-17).  ``rows``: fit only these rows (W, b, iters and status then
    follow the order of the list)."""
    offs, bins = _spikes(offs, bins)
    n = offs.size - 1
    rl = None if rows is None else np.ascontiguousarray(rows, dtype=np.int32)
    nr = n if rl is None else rl.size
    W = np.zeros((nr, n))
    b = np.zeros(nr)
    iters = np.zeros(nr, dtype=np.int32)
    status = np.zeros(nr, dtype=np.int32)
    meth = {"lbfgs": 0, "ga": 1}[method]
    rc = _load().oracle_fit(n, int(n_bins), dt, tau, offs.ctypes.data, bins.ctypes.data, meth, m, max_iter, eta,
                            c1, max_halvings, float(alpha), float(eps), W.ctypes.data, b.ctypes.data,
                            iters.ctypes.data, status.ctypes.data, threads, nr if rl is not None else 0,
                            rl.ctypes.data if rl is not None else None)
    if rc != 0:
        raise ValueError(f"oracle_fit failed ({rc})")
    return dict(W=W, b=b, iters=iters, status=status)
