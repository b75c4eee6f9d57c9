"""Oracle for the dense LU solve -- TEST INFRASTRUCTURE ONLY.

Only the tests, `__graft_entry__.smoke()` and the bench's CPU-baseline /
reference arm may import this package.  The product path (the CUDA library and
its Python binding) never does: it fails loudly when its extension is missing.

This module is the ctypes face of `lu_oracle.c` (plain FP64 C, compiled with
gcc -O2 -ffp-contract=off -fopenmp).  Every function takes and returns numpy
arrays in column-major (Fortran) order and copies its inputs, so callers'
arrays are never modified.  See `lu_oracle.c` for what each routine computes
and which passage of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lu_oracle.c")
_LIB = os.path.join(_HERE, "liblu_oracle.so")
_lock = threading.Lock()
_lib = None

EPS = 2.0 ** -53  # unit roundoff of FP64


def build(force: bool = False) -> str:
    """Compile lu_oracle.c into liblu_oracle.so next to it (idempotent)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            P = C.c_void_p
            I = C.c_int
            D = C.c_double
            L = C.c_int64
            sig = {
                "orc_num_threads": (I, []),
                "orc_set_threads": (None, [I]),
                "orc_getf2": (I, [I, I, P, I, P]),
                "orc_getrf": (I, [I, P, I, P]),
                "orc_getrf_blocked": (I, [I, I, P, I, P]),
                "orc_getrf_blocked_steps": (I, [I, I, P, I, P, I]),
                "orc_getf2_nopiv": (I, [I, I, P, I]),
                "orc_getrf_nopiv_blocked": (I, [I, I, P, I]),
                "orc_trsm_right_upper": (None, [I, I, P, I, P, I]),
                "orc_laswp": (None, [P, I, I, I, I, I, P]),
                "orc_trsm_unit_lower": (None, [I, I, P, I, P, I]),
                "orc_gemm_update": (None, [I, I, I, P, I, P, I, P, I]),
                "orc_gemm_update_dot2": (None, [I, I, I, P, I, P, I, P, I]),
                "orc_getrs": (None, [I, I, P, I, P, P, I]),
                "orc_residual": (None, [I, I, P, I, P, I, P, I, P, I]),
                "orc_norm_inf_mat": (D, [I, I, P, I]),
                "orc_norm_one_mat": (D, [I, I, P, I]),
                "orc_norm_inf_vec": (D, [I, P]),
                "orc_scaled_residual": (D, [I, D, D, D, D]),
                "orc_paper_residual": (D, [I, D, D]),
                "orc_cond1_est": (D, [I, P, I, P, D]),
                "orc_round_bf16": (None, [L, P, P]),
                "orc_round_fp16": (None, [L, P, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.array(a, dtype=np.float64, order="F", copy=True)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def num_threads() -> int:
    return _load().orc_num_threads()


def set_threads(t: int) -> None:
    _load().orc_set_threads(int(t))


# ----------------------------------------------------------------- factor

def getf2(A):
    """Unblocked GEPP of an m x n block.  Returns (LU, ipiv (1-based, int32), info)."""
    LU = _f64(A)
    m, n = LU.shape
    ipiv = np.zeros(max(1, min(m, n)), dtype=np.int32)
    info = _load().orc_getf2(m, n, _ptr(LU), max(1, m), _ptr(ipiv))
    return LU, ipiv[:min(m, n)], int(info)


def getrf(A, nb: int | None = None, ksteps: int = -1, timed: bool = False):
    """GEPP of a square matrix: unblocked (nb None) or the blocked right-looking
    iteration with block width nb (optionally only its first `ksteps` steps).
    With timed=True a fourth value is the wall time of the C call alone."""
    import time
    LU = _f64(A)
    n = LU.shape[0]
    assert LU.shape == (n, n)
    ipiv = np.zeros(max(1, n), dtype=np.int32)
    lib = _load()
    t0 = time.perf_counter()
    if nb is None:
        info = lib.orc_getrf(n, _ptr(LU), max(1, n), _ptr(ipiv))
    else:
        info = lib.orc_getrf_blocked_steps(n, int(nb), _ptr(LU), max(1, n), _ptr(ipiv), int(ksteps))
    dt = time.perf_counter() - t0
    if timed:
        return LU, ipiv[:n], int(info), dt
    return LU, ipiv[:n], int(info)


def getrf_nopiv(A, nb: int | None = None):
    """LU without pivoting (the paper's HPL-AI variant): unblocked (nb None) or
    the paper's blocked four-kernel iteration.  Returns (LU, info)."""
    LU = _f64(A)
    n = LU.shape[0]
    lib = _load()
    if nb is None:
        info = lib.orc_getf2_nopiv(n, n, _ptr(LU), max(1, n))
    else:
        info = lib.orc_getrf_nopiv_blocked(n, int(nb), _ptr(LU), max(1, n))
    return LU, int(info)


def trsm_right_upper(B, U):
    """B U^-1 for the upper triangle of the square matrix U."""
    X = _f64(B)
    Um = _f64(U)
    m, w = X.shape
    _load().orc_trsm_right_upper(m, w, _ptr(Um), max(1, Um.shape[0]), _ptr(X), max(1, m))
    return X


def laswp(A, c0: int, c1: int, k1: int, k2: int, ipiv):
    out = _f64(A)
    piv = np.ascontiguousarray(ipiv, dtype=np.int32)
    _load().orc_laswp(_ptr(out), max(1, out.shape[0]), c0, c1, k1, k2, _ptr(piv))
    return out


def trsm_unit_lower(L, B):
    """L^-1 B for the unit-lower triangle of the square matrix L."""
    Lm = _f64(L)
    X = _f64(B)
    nb, ncol = X.shape
    _load().orc_trsm_unit_lower(nb, ncol, _ptr(Lm), max(1, Lm.shape[0]), _ptr(X), max(1, nb))
    return X


def gemm_update(Cm, A, B):
    """C - A B in FP64."""
    out = _f64(Cm)
    Am = _f64(A)
    Bm = _f64(B)
    m, k = Am.shape
    k2, n = Bm.shape
    assert k == k2 and out.shape == (m, n)
    _load().orc_gemm_update(m, n, k, _ptr(Am), max(1, m), _ptr(Bm), max(1, k), _ptr(out), max(1, m))
    return out


def gemm_update_dot2(Cm, A, B):
    """C - A B as if computed in twice FP64 precision and rounded once (Dot2)."""
    out = _f64(Cm)
    Am = _f64(A)
    Bm = _f64(B)
    m, k = Am.shape
    k2, n = Bm.shape
    assert k == k2 and out.shape == (m, n)
    _load().orc_gemm_update_dot2(m, n, k, _ptr(Am), max(1, m), _ptr(Bm), max(1, k), _ptr(out), max(1, m))
    return out


def getrs(LU, ipiv, B):
    """X with A X = B from the factors (B is n or n x nrhs)."""
    LUm = _f64(LU)
    X = _f64(B)
    vec = X.ndim == 1
    if vec:
        X = X.reshape(-1, 1, order="F")
    n, nrhs = X.shape
    piv = np.ascontiguousarray(ipiv, dtype=np.int32)
    _load().orc_getrs(n, nrhs, _ptr(LUm), max(1, n), _ptr(piv), _ptr(X), max(1, n))
    return X[:, 0] if vec else X


def solve(A, B, nb: int | None = None):
    """x = A^-1 b by GEPP (blocked when nb is given).  Returns (X, LU, ipiv, info)."""
    LU, ipiv, info = getrf(A, nb)
    return getrs(LU, ipiv, B), LU, ipiv, info


# ----------------------------------------------------------------- residuals

def residual(A, X, B):
    """R = B - A X in FP64."""
    Am = _f64(A)
    Xm = _f64(X)
    Bm = _f64(B)
    vec = Xm.ndim == 1
    if vec:
        Xm = Xm.reshape(-1, 1, order="F")
        Bm = Bm.reshape(-1, 1, order="F")
    n, nrhs = Xm.shape
    R = np.zeros((n, nrhs), dtype=np.float64, order="F")
    _load().orc_residual(n, nrhs, _ptr(Am), max(1, n), _ptr(Xm), max(1, n), _ptr(Bm), max(1, n),
                         _ptr(R), max(1, n))
    return R[:, 0] if vec else R


def norm_inf(A) -> float:
    Am = _f64(A)
    if Am.ndim == 1:
        return float(_load().orc_norm_inf_vec(Am.shape[0], _ptr(Am)))
    return float(_load().orc_norm_inf_mat(Am.shape[0], Am.shape[1], _ptr(Am), max(1, Am.shape[0])))


def norm_one(A) -> float:
    Am = _f64(A)
    return float(_load().orc_norm_one_mat(Am.shape[0], Am.shape[1], _ptr(Am), max(1, Am.shape[0])))


def scaled_residual(A, X, B, anorm: float | None = None):
    """HPL scaled residual per right-hand side (array of length nrhs, or a float for vectors)."""
    lib = _load()
    Xm = _f64(X)
    Bm = _f64(B)
    vec = Xm.ndim == 1
    if vec:
        Xm = Xm.reshape(-1, 1, order="F")
        Bm = Bm.reshape(-1, 1, order="F")
    R = residual(A, Xm, Bm)
    n = Xm.shape[0]
    an = norm_inf(A) if anorm is None else anorm
    out = np.array([lib.orc_scaled_residual(n, norm_inf(R[:, r]), an, norm_inf(Xm[:, r]), norm_inf(Bm[:, r]))
                    for r in range(Xm.shape[1])])
    return float(out[0]) if vec else out


def scaled_residual_from_norms(n: int, rnorm: float, anorm: float, xnorm: float, bnorm: float) -> float:
    return float(_load().orc_scaled_residual(n, rnorm, anorm, xnorm, bnorm))


def paper_residual(n: int, rnorm: float, bnorm: float) -> float:
    return float(_load().orc_paper_residual(n, rnorm, bnorm))


def cond1_est(LU, ipiv, anorm1: float) -> float:
    LUm = _f64(LU)
    piv = np.ascontiguousarray(ipiv, dtype=np.int32)
    return float(_load().orc_cond1_est(LUm.shape[0], _ptr(LUm), max(1, LUm.shape[0]), _ptr(piv), float(anorm1)))


# ----------------------------------------------------------------- 16-bit rounding

def round_bf16(x) -> np.ndarray:
    """FP32 -> bfloat16 round-to-nearest-even, returned as FP64 (same shape)."""
    xf = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(xf.shape, dtype=np.float64)
    _load().orc_round_bf16(xf.size, _ptr(xf), _ptr(out))
    return out


def round_fp16(x) -> np.ndarray:
    """FP32 -> IEEE binary16 round-to-nearest-even, returned as FP64 (same shape)."""
    xf = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(xf.shape, dtype=np.float64)
    _load().orc_round_fp16(xf.size, _ptr(xf), _ptr(out))
    return out
