"""The oracle's own SVD (one-sided Jacobi in plain C) and the truncation rule.

Test infrastructure only (see ``oracle/__init__``).

App. B: after each step the Schmidt spectrum of every bond of |rho>> is
computed and singular values are discarded under the more severe of two
conditions, ``cut_off_rho`` (maximum discarded weight) and ``max_dim_rho``.
Readings where the paper is silent: the discarded weight is relative to the total weight
sum_i s_i^2; at least one value is kept; equal singular values keep their
original order (stable sort).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle_jacobi.so")
_lib = None


def compile_oracle(force: bool = False) -> str:
    """Compile jacobi.c with gcc (portable flags; no -march=native)."""
    src = os.path.join(_HERE, "jacobi.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(compile_oracle())
        lib.oracle_jacobi_rows.restype = ctypes.c_int
        lib.oracle_jacobi_rows.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_void_p, ctypes.c_double, ctypes.c_int]
        _lib = lib
    return _lib


def jacobi_rows(W: np.ndarray, Z: np.ndarray | None = None, tol: float | None = None,
                max_sweeps: int = 200) -> int:
    """Rotate the rows of W (and Z) in place until mutually orthogonal."""
    assert W.dtype == np.float64 and W.flags.c_contiguous
    c, L = W.shape
    if tol is None:
        tol = np.sqrt(max(L, 1)) * np.finfo(np.float64).eps
    zp = None
    if Z is not None:
        assert Z.dtype == np.float64 and Z.flags.c_contiguous and Z.shape == (c, c)
        zp = Z.ctypes.data
    sweeps = _load().oracle_jacobi_rows(W.ctypes.data, c, L, zp, float(tol), int(max_sweeps))
    if sweeps < 0:
        raise RuntimeError("oracle Jacobi SVD did not converge")
    return sweeps


def svd_right_lapack(M: np.ndarray):
    """The same (s, Vt) as ``svd_right`` from LAPACK's gesdd through numpy,
    multithreaded by the BLAS under numpy: the route of the paper's solver
    (threaded LAPACK, Sec. 2.5), timed as a CPU baseline.  Ties in s keep
    LAPACK's order."""
    _, s, Vt = np.linalg.svd(np.asarray(M, dtype=np.float64), full_matrices=False)
    return s, Vt


def svd_right(M: np.ndarray, tol: float | None = None):
    """Singular values (descending, stable order) and right singular vectors
    (as rows) of M (m x n), from the one-sided Jacobi above.

    m <= n: the rows of M are orthogonalised; row j -> s_j v_j^T.
    m >  n: the rows of M^T (columns of M) are orthogonalised and the
            rotations are accumulated in Z; rows of Z -> v_j^T.
    Returns (s[r], Vt[r, n]) with r = min(m, n)."""
    m, n = M.shape
    if m <= n:
        W = np.array(M, dtype=np.float64, order="C", copy=True)
        jacobi_rows(W, tol=tol)
        s = np.sqrt(np.einsum("ij,ij->i", W, W))
        Vt = np.zeros_like(W)
        nz = s > 0
        Vt[nz] = W[nz] / s[nz, None]
    else:
        W = np.array(M.T, dtype=np.float64, order="C", copy=True)
        Z = np.eye(n)
        jacobi_rows(W, Z, tol=tol)
        s = np.sqrt(np.einsum("ij,ij->i", W, W))
        Vt = Z
    order = np.argsort(-s, kind="stable")
    return s[order], Vt[order]


def truncation_rank(s: np.ndarray, chi_max: int, cutoff: float) -> int:
    """k = min(chi_max, k_cut); k_cut = smallest k >= 1 whose discarded weight
    sum_{i>=k} s_i^2 is <= cutoff * sum_i s_i^2 (App. B: the more severe of
    cut_off_rho and max_dim_rho).  s is sorted descending.  Tail sums run
    from the smallest value up."""
    w = s.astype(np.float64) ** 2
    r = len(w)
    tail = np.zeros(r + 1)
    for i in range(r - 1, -1, -1):
        tail[i] = tail[i + 1] + w[i]
    total = tail[0]
    kcut = r
    for k in range(1, r + 1):
        if tail[k] <= cutoff * total:
            kcut = k
            break
    return int(max(1, min(chi_max, kcut, r)))


def discarded_weight(s: np.ndarray, k: int) -> float:
    w = s.astype(np.float64) ** 2
    tot = w.sum()
    return float(w[k:].sum() / tot) if tot > 0 else 0.0
