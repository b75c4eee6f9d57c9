"""Thin ctypes binding of libgb300lu.so (the C ABI in include/lu.h and lu_steps.h).

Only argument marshalling happens here: every step of the solve runs in the
library's CUDA kernels.  PyTorch supplies device memory and the stream.  The
binding refuses to work without the compiled library (there is no fallback).

Matrices are torch CUDA tensors.  The C ABI is column-major: an (n, n) FP64
tensor with strides (1, lda) is passed as is; the step-level entry points take
row-major tensors (strides (ld, 1)).
"""
from __future__ import annotations

import ctypes as C
import os
import threading
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# GB300LU_LIB names another build of the library (the bounds-checking one)
LIB_PATH = os.environ.get("GB300LU_LIB") or os.path.join(_HERE, "libgb300lu.so")

LU_F64, LU_BF16, LU_FP16, LU_F32 = 0, 1, 2, 3
PRECS = {"f64": LU_F64, "bf16": LU_BF16, "fp16": LU_FP16, "f32": LU_F32}
LU_OK, LU_ESINGULAR, LU_ENOMEM, LU_ENOTCONV, LU_ERANGE, LU_ETIMEOUT, LU_EAGAIN, LU_ECUDA, LU_EINTERNAL = range(9)
LU_FACTOR_NOPIV, LU_FACTOR_OZAKI = 1, 2

EXPORTED = [
    "lu_create", "lu_destroy", "lu_strerror", "lu_factor", "lu_fact_info", "lu_fact_ipiv", "lu_fact_lu",
    "lu_solve", "lu_refine", "lu_scaled_residual", "lu_residual_norms", "lu_fact_free",
    "lu_step_panel", "lu_step_trsm", "lu_step_gemm", "lu_ctx_status", "lu_device_sm_count", "lu_build_tag",
    "lu_create_ex", "lu_peak_probe", "lu_default_nb", "lu_generate", "lu_profile_enable", "lu_profile_select", "lu_profile_read", "lu_launch_count", "lu_step_panel_static",
    "lu_batch_create", "lu_batch_run", "lu_batch_shape", "lu_batch_free", "lu_solve_batched",
    "lu_server_create", "lu_server_submit", "lu_server_poll", "lu_server_wait", "lu_server_stats",
    "lu_server_destroy", "lu_fact_bytes", "lu_factor_ex", "lu_step_gemm_ozaki", "lu_step_wait_probe",
]
PHASES = ["panel", "laswp", "trsm", "cast", "gemm", "solve", "residual", "other"]

_lock = threading.Lock()
_lib = None


# device-memory callbacks of lu_create_ex: alloc(user, bytes, stream) -> ptr,
# release(user, ptr, bytes, stream)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)


class LuRequest(C.Structure):
    _fields_ = [("n", C.c_int), ("nrhs", C.c_int), ("dA", C.c_void_p), ("lda", C.c_int), ("dB", C.c_void_p),
                ("ldb", C.c_int), ("dX", C.c_void_p), ("ldx", C.c_int), ("factor_key", C.c_uint64),
                ("keep_factor", C.c_int), ("use_resident", C.c_int)]


class LuResult(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("scaled_resid", C.c_double), ("reused_factor", C.c_int),
                ("refactored", C.c_int), ("slot", C.c_int), ("t_submit_ns", C.c_uint64), ("t_start_ns", C.c_uint64),
                ("t_done_ns", C.c_uint64)]


class LuError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = _lib.lu_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} (code {code})" if what else f"{msg} (code {code})")


def load():
    """Load the library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(the solver has no CPU fallback)")
        lib = C.CDLL(LIB_PATH)
        P, I, D = C.c_void_p, C.c_int, C.c_double
        PP = C.POINTER(C.c_void_p)
        IP = C.POINTER(C.c_int)
        DP = C.POINTER(C.c_double)
        sig = {
            "lu_create": (I, [PP, P]),
            "lu_create_ex": (I, [PP, P, ALLOC_FN, FREE_FN, P]),
            "lu_peak_probe": (I, [I, DP]),
            "lu_default_nb": (I, [I, I, I]),
            "lu_generate": (I, [P, I, I, I, C.c_uint64, I, D, P]),
            "lu_destroy": (None, [P]),
            "lu_strerror": (C.c_char_p, [I]),
            "lu_factor": (I, [P, I, P, I, I, I, PP, IP]),
            "lu_fact_info": (I, [P, IP]),
            "lu_fact_ipiv": (I, [P, P]),
            "lu_fact_lu": (I, [P, P, I]),
            "lu_solve": (I, [P, I, P, I]),
            "lu_refine": (I, [P, P, I, P, I, P, I, I, D, I, IP, DP]),
            "lu_scaled_residual": (I, [P, I, I, P, I, P, I, P, I, DP]),
            "lu_residual_norms": (I, [P, I, I, P, I, P, I, P, I, DP]),
            "lu_fact_free": (None, [P]),
            "lu_step_panel": (I, [P, I, I, I, P, I, P, P]),
            "lu_step_trsm": (I, [P, I, I, I, P, I, P, I]),
            "lu_step_gemm": (I, [P, I, I, I, I, P, I, P, I, P, I]),
            "lu_step_gemm_ozaki": (I, [P, I, I, I, P, I, P, I, P, I]),
            "lu_step_wait_probe": (I, [P, I]),
            "lu_ctx_status": (I, [P]),
            "lu_device_sm_count": (I, [P]),
            "lu_build_tag": (C.c_char_p, []),
            "lu_profile_enable": (I, [P, I]),
            "lu_profile_select": (I, [P, C.c_uint]),
            "lu_profile_read": (I, [P, DP, C.POINTER(C.c_longlong)]),
            "lu_launch_count": (C.c_longlong, [P]),
            "lu_step_panel_static": (I, [P, I, I, I, P, I, P, P, P]),
            "lu_batch_create": (I, [P, I, IP, IP, P, IP, P, IP, P, IP, I, D, I, I, PP]),
            "lu_batch_run": (I, [P, P, P, P]),
            "lu_batch_shape": (I, [P, IP, IP, C.POINTER(C.c_float)]),
            "lu_batch_free": (None, [P]),
            "lu_solve_batched": (I, [P, I, IP, IP, P, IP, P, IP, I, P]),
            "lu_server_create": (I, [PP, C.c_size_t, I, I]),
            "lu_server_submit": (I, [P, C.POINTER(LuRequest), C.POINTER(C.c_uint64)]),
            "lu_server_poll": (I, [P, C.c_uint64, C.POINTER(LuResult)]),
            "lu_server_wait": (I, [P, C.c_uint64, C.POINTER(LuResult)]),
            "lu_server_stats": (I, [P, C.POINTER(C.c_uint64), IP, C.POINTER(C.c_size_t), C.POINTER(C.c_uint64)]),
            "lu_server_destroy": (I, [P]),
            "lu_fact_bytes": (C.c_size_t, [I, I, I, I]),
            "lu_factor_ex": (I, [P, I, P, I, I, I, I, PP, IP]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(rc: int, what: str):
    if rc != LU_OK:
        raise LuError(rc, what)


def _prec(p) -> int:
    return PRECS[p] if isinstance(p, str) else int(p)


def _colmajor(t, name: str, rows: int | None = None):
    """(ptr, ld, ncols) of a column-major CUDA FP64 tensor (1-D = one column)."""
    import torch
    if not (t.is_cuda and t.dtype == torch.float64):
        raise TypeError(f"{name}: expected a CUDA float64 tensor")
    if t.dim() == 1:
        if t.stride(0) != 1:
            raise ValueError(f"{name}: 1-D tensor must be contiguous")
        return t.data_ptr(), max(1, t.shape[0]), 1
    if t.dim() != 2 or (t.stride(0) != 1 and t.shape[0] > 1):
        raise ValueError(f"{name}: expected a column-major (n, k) tensor with strides (1, ld)")
    ld = t.stride(1) if t.shape[1] > 1 else max(1, t.shape[0])
    return t.data_ptr(), max(1, ld), t.shape[1]


def _rowmajor(t, name: str):
    if not t.is_cuda:
        raise TypeError(f"{name}: expected a CUDA tensor")
    if t.dim() != 2 or (t.stride(1) != 1 and t.shape[1] > 1):
        raise ValueError(f"{name}: expected a row-major (m, n) tensor with strides (ld, 1)")
    ld = t.stride(0) if t.shape[0] > 1 else max(1, t.shape[1])
    return t.data_ptr(), max(1, ld)


def generate(out, seed: int, stream_id: int = 0, diag_shift: float = 0.0, cuda_stream=None):
    """Fill the column-major FP64 CUDA tensor `out` (rows x cols) with the
    seeded draws of lu_generate (element (i, j) = draw i + j*rows of the
    stream, + diag_shift on the diagonal): the device form of
    inputs.hpl_matrix / hpl_rhs."""
    import torch
    ptr, ld, cols = _colmajor(out, "out")
    rows = out.shape[0]
    st = cuda_stream if cuda_stream is not None else torch.cuda.current_stream().cuda_stream
    _check(load().lu_generate(C.c_void_p(ptr), rows, cols, ld, C.c_uint64(seed & ((1 << 64) - 1)), int(stream_id),
                              float(diag_shift), C.c_void_p(st)), "lu_generate")
    return out


def default_nb(n: int, prec="f64", ozaki: bool = False) -> int:
    """The block width nb = 0 selects (the library's tuning table)."""
    v = load().lu_default_nb(int(n), _prec(prec), LU_FACTOR_OZAKI if ozaki else 0)
    _check(0 if v > 0 or n == 0 else v, "lu_default_nb")
    return int(v)


def peak_probe(kind: int) -> float:
    """TFLOP/s of an arithmetic-rate probe (0 FP64 FMA, 1 FP64 mma.sync, 2 FP32 FMA) on the current device."""
    out = C.c_double(0.0)
    _check(load().lu_peak_probe(int(kind), C.byref(out)), "lu_peak_probe")
    return float(out.value)


def fact_bytes(n: int, nrhs: int, prec="fp16", nb: int = 0) -> int:
    """Device bytes lu_factor + lu_refine allocate for this system (budgeting)."""
    return int(load().lu_fact_bytes(int(n), int(nrhs), _prec(prec), int(nb)))


def colmajor_empty(n: int, k: int, device="cuda", dtype=None):
    """An uninitialised (n, k) column-major tensor (strides (1, n))."""
    import torch
    return torch.empty((k, n), dtype=dtype or torch.float64, device=device).t()


class Context:
    """A library context bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, stream=None, allocator=None):
        """allocator: None (the library's stream-ordered pool) or a pair of
        callables (alloc(nbytes, stream_handle) -> device pointer int, release(
        ptr, nbytes, stream_handle)) through which every device buffer of this
        context passes (lu_create_ex)."""
        import torch
        lib = load()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        self._h = None
        self._factors = weakref.WeakSet()
        if allocator is None:
            _check(lib.lu_create(C.byref(h), C.c_void_p(stream.cuda_stream)), "lu_create")
        else:
            alloc, release = allocator

            def _alloc(user, nbytes, st):
                try:
                    return int(alloc(int(nbytes), st or 0)) or None
                except Exception:
                    return None

            def _release(user, ptr, nbytes, st):
                release(int(ptr), int(nbytes), st or 0)

            # the ctypes callback objects must live as long as the context
            self._cb = (ALLOC_FN(_alloc), FREE_FN(_release))
            _check(lib.lu_create_ex(C.byref(h), C.c_void_p(stream.cuda_stream), self._cb[0], self._cb[1], None),
                   "lu_create_ex")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        """Free every factorization still alive, then the context."""
        if getattr(self, "_h", None):
            for f in list(self._factors):
                f.free()
            load().lu_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def sm_count(self) -> int:
        return load().lu_device_sm_count(self._h)

    def status(self) -> int:
        return load().lu_ctx_status(self._h)

    def launch_count(self) -> int:
        return int(load().lu_launch_count(self._h))

    def profile(self, enable: bool = True):
        _check(load().lu_profile_enable(self._h, 1 if enable else 0), "lu_profile_enable")

    def profile_select(self, phases=None):
        """Record only these phases while profiling (names from PHASES; None = all)."""
        mask = 0xFFFFFFFF if phases is None else sum(1 << PHASES.index(p) for p in phases)
        _check(load().lu_profile_select(self._h, mask), "lu_profile_select")

    def profile_read(self) -> dict:
        """{phase: (milliseconds, launches)} since the last read (synchronizes)."""
        ms = (C.c_double * len(PHASES))()
        nl = (C.c_longlong * len(PHASES))()
        _check(load().lu_profile_read(self._h, ms, nl), "lu_profile_read")
        return {p: (ms[i], int(nl[i])) for i, p in enumerate(PHASES)}

    def factor(self, A, prec="f64", nb: int = 0, sync: bool = True, nopiv: bool = False,
               ozaki: bool = False) -> "Factor":
        """Factor P A = L U of the column-major FP64 (n, n) tensor A (nopiv: the
        paper's no-pivot variant for diagonally dominant A; ozaki: FP64 trailing
        update on the BF16 tensor cores by error-free splitting, prec f64)."""
        ptr, lda, ncol = _colmajor(A, "A")
        n = A.shape[0]
        if ncol != n:
            raise ValueError("A must be square")
        f = C.c_void_p()
        info = C.c_int(-1)
        flags = (LU_FACTOR_NOPIV if nopiv else 0) | (LU_FACTOR_OZAKI if ozaki else 0)
        rc = load().lu_factor_ex(self._h, n, C.c_void_p(ptr), lda, _prec(prec), int(nb), flags,
                                 C.byref(f), C.byref(info) if sync else None)
        if f.value:
            fac = Factor(self, f, n, _prec(prec))
            self._factors.add(fac)
        else:
            fac = None
        _check(rc, "lu_factor")
        if sync:
            fac._info = info.value
        return fac

    def scaled_residual(self, A, X, B) -> np.ndarray:
        pa, lda, _ = _colmajor(A, "A")
        px, ldx, nrhs = _colmajor(X, "X")
        pb, ldb, _ = _colmajor(B, "B")
        out = (C.c_double * max(1, nrhs))()
        _check(load().lu_scaled_residual(self._h, A.shape[0], nrhs, C.c_void_p(pa), lda, C.c_void_p(px), ldx,
                                         C.c_void_p(pb), ldb, out), "lu_scaled_residual")
        return np.array(out[:nrhs])

    def residual_norms(self, A, X, B) -> np.ndarray:
        """(nrhs, 4) array: ||b - A x||, ||A||, ||x||, ||b|| (infinity norms) per column."""
        pa, lda, _ = _colmajor(A, "A")
        px, ldx, nrhs = _colmajor(X, "X")
        pb, ldb, _ = _colmajor(B, "B")
        out = (C.c_double * max(1, 4 * nrhs))()
        _check(load().lu_residual_norms(self._h, A.shape[0], nrhs, C.c_void_p(pa), lda, C.c_void_p(px), ldx,
                                        C.c_void_p(pb), ldb, out), "lu_residual_norms")
        return np.array(out[:4 * nrhs]).reshape(nrhs, 4)

    # ---- step-level entry points (row-major operands)
    def step_panel(self, P, ipiv, info, prec="f64"):
        pp, ld = _rowmajor(P, "P")
        m, w = P.shape
        _check(load().lu_step_panel(self._h, _prec(prec), m, w, C.c_void_p(pp), ld, C.c_void_p(ipiv.data_ptr()),
                                    C.c_void_p(info.data_ptr())), "lu_step_panel")

    def step_panel_static(self, P, ipiv, info, status, prec="f64"):
        """lu_step_panel_static on this context's stream (allocates nothing)."""
        pp, ld = _rowmajor(P, "P")
        m, w = P.shape
        _check(load().lu_step_panel_static(C.c_void_p(self.stream.cuda_stream), _prec(prec), m, w, C.c_void_p(pp),
                                           ld, C.c_void_p(ipiv.data_ptr()), C.c_void_p(info.data_ptr()),
                                           C.c_void_p(status.data_ptr())), "lu_step_panel_static")

    def step_trsm(self, L, X, prec="f64"):
        pl, ldl = _rowmajor(L, "L")
        px, ldx = _rowmajor(X, "X")
        w, N = X.shape
        _check(load().lu_step_trsm(self._h, _prec(prec), w, N, C.c_void_p(pl), ldl, C.c_void_p(px), ldx),
               "lu_step_trsm")

    def step_gemm(self, Cm, A, B, prec="f64"):
        pc, ldc = _rowmajor(Cm, "C")
        pa, lda = _rowmajor(A, "A")
        pb, ldb = _rowmajor(B, "B")
        m, k = A.shape
        n = B.shape[1]
        _check(load().lu_step_gemm(self._h, _prec(prec), m, n, k, C.c_void_p(pc), ldc, C.c_void_p(pa), lda,
                                   C.c_void_p(pb), ldb), "lu_step_gemm")

    def wait_probe(self, kind: int) -> int:
        """Run one bounded device wait on a condition nothing satisfies (0 flag,
        1 grid barrier, 2 mbarrier); returns the library's code (LU_ETIMEOUT)."""
        rc = load().lu_step_wait_probe(self._h, int(kind))
        if rc < 0:
            _check(rc, "lu_step_wait_probe")
        return rc

    def step_gemm_ozaki(self, Cm, A, B):
        """C -= A B in FP64 with the products on the BF16 tensor cores (row-major FP64, k <= 256)."""
        pc, ldc = _rowmajor(Cm, "C")
        pa, lda = _rowmajor(A, "A")
        pb, ldb = _rowmajor(B, "B")
        m, k = A.shape
        n = B.shape[1]
        _check(load().lu_step_gemm_ozaki(self._h, m, n, k, C.c_void_p(pc), ldc, C.c_void_p(pa), lda,
                                         C.c_void_p(pb), ldb), "lu_step_gemm_ozaki")


class Factor:
    """A factorization owned by the library (freed by free() or garbage collection)."""

    def __init__(self, ctx: Context, handle, n: int, prec: int):
        self.ctx = ctx
        self._h = handle
        self.n = n
        self.prec = prec
        self._info = None

    def free(self):
        if getattr(self, "_h", None):
            load().lu_fact_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def info(self) -> int:
        if self._info is None:
            v = C.c_int(0)
            _check(load().lu_fact_info(self._h, C.byref(v)), "lu_fact_info")
            self._info = v.value
        return self._info

    def ipiv(self):
        import torch
        out = torch.empty(self.n, dtype=torch.int32, device="cuda")
        _check(load().lu_fact_ipiv(self._h, C.c_void_p(out.data_ptr())), "lu_fact_ipiv")
        return out

    def lu(self):
        out = colmajor_empty(self.n, self.n)
        _check(load().lu_fact_lu(self._h, C.c_void_p(out.data_ptr()), max(1, self.n)), "lu_fact_lu")
        return out

    def solve_(self, B):
        """Overwrite B (column-major FP64, (n,) or (n, nrhs)) with the solution."""
        pb, ldb, nrhs = _colmajor(B, "B")
        _check(load().lu_solve(self._h, nrhs, C.c_void_p(pb), ldb), "lu_solve")
        return B

    def refine(self, A, B, X, tol: float = 16.0, max_iter: int = 50, raise_on_notconv: bool = True):
        """Iterative refinement to HPL scaled residual < tol; returns (iters, scaled residual)."""
        pa, lda, _ = _colmajor(A, "A")
        pb, ldb, nrhs = _colmajor(B, "B")
        px, ldx, _ = _colmajor(X, "X")
        it = C.c_int(0)
        sr = C.c_double(0.0)
        rc = load().lu_refine(self._h, C.c_void_p(pa), lda, C.c_void_p(pb), ldb, C.c_void_p(px), ldx, nrhs,
                              float(tol), int(max_iter), C.byref(it), C.byref(sr))
        if rc == LU_ENOTCONV and not raise_on_notconv:
            return it.value, sr.value
        _check(rc, "lu_refine")
        return it.value, sr.value


def _iarr(v):
    a = (C.c_int * max(1, len(v)))()
    for i, x in enumerate(v):
        a[i] = int(x)
    return a


def _parr(tensors):
    a = (C.c_void_p * max(1, len(tensors)))()
    for i, t in enumerate(tensors):
        a[i] = t.data_ptr()
    return a


class Batch:
    """A planned batch of independent solves A_i X_i = B_i (n_i <= 512, nrhs_i <= 8),
    FP32 factor + FP64 refinement, one persistent graph launch per run().

    A, B, X are lists of column-major CUDA FP64 tensors ((n, n), (n, k), (n, k))."""

    def __init__(self, ctx: Context, A, B, X, tol: float = 16.0, max_iter: int = 50, tune: bool = False,
                 prec="f32"):
        self.ctx = ctx
        self._keep = (list(A), list(B), list(X))
        cnt = len(A)
        n, nrhs, lda, ldb, ldx = [], [], [], [], []
        for a, b, x in zip(A, B, X):
            _, la, _ = _colmajor(a, "A")
            _, lb, kb = _colmajor(b, "B")
            _, lx, _ = _colmajor(x, "X")
            n.append(a.shape[0]); nrhs.append(kb); lda.append(la); ldb.append(lb); ldx.append(lx)
        h = C.c_void_p()
        self._h = None
        rc = load().lu_batch_create(ctx.handle, cnt, _iarr(n), _iarr(nrhs), _parr(A), _iarr(lda), _parr(B),
                                    _iarr(ldb), _parr(X), _iarr(ldx), _prec(prec), float(tol), int(max_iter),
                                    1 if tune else 0, C.byref(h))
        _check(rc, "lu_batch_create")
        self._h = h
        self.count = cnt

    def run(self, info, iters=None, resid=None):
        _check(load().lu_batch_run(self._h, C.c_void_p(info.data_ptr()),
                                   C.c_void_p(iters.data_ptr()) if iters is not None else None,
                                   C.c_void_p(resid.data_ptr()) if resid is not None else None), "lu_batch_run")

    def shape(self):
        t, c, ms = C.c_int(0), C.c_int(0), C.c_float(0.0)
        _check(load().lu_batch_shape(self._h, C.byref(t), C.byref(c), C.byref(ms)), "lu_batch_shape")
        return t.value, c.value, ms.value

    def free(self):
        if getattr(self, "_h", None):
            load().lu_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def solve_batched(ctx: Context, A, B, info, prec="f32"):
    """lu_solve_batched: B (list of (n, k) column-major tensors) is overwritten with X."""
    n, nrhs, lda, ldb = [], [], [], []
    for a, b in zip(A, B):
        _, la, _ = _colmajor(a, "A")
        _, lb, kb = _colmajor(b, "B")
        n.append(a.shape[0]); nrhs.append(kb); lda.append(la); ldb.append(lb)
    _check(load().lu_solve_batched(ctx.handle, len(A), _iarr(n), _iarr(nrhs), _parr(A), _iarr(lda), _parr(B),
                                   _iarr(ldb), _prec(prec), C.c_void_p(info.data_ptr())), "lu_solve_batched")


class Server:
    """lu_server_*: continuous-batching solve server on the current device."""

    def __init__(self, hbm_budget_bytes: int, prec="fp16", max_slots: int = 8):
        h = C.c_void_p()
        self._h = None
        _check(load().lu_server_create(C.byref(h), int(hbm_budget_bytes), _prec(prec), int(max_slots)),
               "lu_server_create")
        self._h = h
        self._keep = {}

    def submit(self, A, B, X, factor_key: int = 0, keep_factor: bool = False, use_resident: bool = False) -> int:
        pa, lda, _ = _colmajor(A, "A")
        pb, ldb, nrhs = _colmajor(B, "B")
        px, ldx, _ = _colmajor(X, "X")
        req = LuRequest(A.shape[0], nrhs, pa, lda, pb, ldb, px, ldx, int(factor_key), 1 if keep_factor else 0,
                        1 if use_resident else 0)
        t = C.c_uint64(0)
        _check(load().lu_server_submit(self._h, C.byref(req), C.byref(t)), "lu_server_submit")
        self._keep[t.value] = (A, B, X)
        return t.value

    def poll(self, ticket: int):
        r = LuResult()
        rc = load().lu_server_poll(self._h, int(ticket), C.byref(r))
        if rc == LU_EAGAIN:
            return None
        _check(rc, "lu_server_poll")
        self._keep.pop(int(ticket), None)
        return r

    def wait(self, ticket: int) -> "LuResult":
        r = LuResult()
        _check(load().lu_server_wait(self._h, int(ticket), C.byref(r)), "lu_server_wait")
        self._keep.pop(int(ticket), None)
        return r

    def stats(self) -> dict:
        d, rsd, b, ev = C.c_uint64(0), C.c_int(0), C.c_size_t(0), C.c_uint64(0)
        _check(load().lu_server_stats(self._h, C.byref(d), C.byref(rsd), C.byref(b), C.byref(ev)), "lu_server_stats")
        return {"done": d.value, "resident": rsd.value, "bytes_in_use": b.value, "evictions": ev.value}

    def close(self):
        if getattr(self, "_h", None):
            load().lu_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
