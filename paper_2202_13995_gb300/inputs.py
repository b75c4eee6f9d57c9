"""Seeded synthetic LINPACK inputs, shared by the oracle checks, the GPU tests and the bench.

This module holds no arithmetic of the solver: it only draws the matrix and the
right-hand sides.  The HPL benchmark generates its own input (the paper's HPL
validation section says the input is generated, with the solution chosen as a
vector of ones); here every entry is a pure function of (seed, stream, index),
so any slice of any workload can be regenerated on its own, on the host
(numpy) or on a device (torch), bit for bit the same.

Generator: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used in counter mode: the k-th
draw of a stream is mix64(state0 + (k + 1) * GAMMA), with
state0 = mix64(seed XOR (stream * STREAM_MULT)).  A draw z maps to the uniform
value (z >> 11) * 2**-53 - 0.5, which lies in [-0.5, 0.5) and is exact in FP64.

Layouts: matrices are column-major (element (i, j) has linear index i + j*n),
which is also the device layout of the solver.

Streams: 0 = the matrix A, 1 = the right-hand sides B (n x nrhs, column-major).
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
STREAM_MULT = 0xD1B54A32D192ED03
MASK64 = (1 << 64) - 1

STREAM_A = 0
STREAM_B = 1

__all__ = [
    "mix64_int", "stream_state", "uniform_np", "hpl_matrix", "hpl_rhs",
    "hpl_matrix_torch", "hpl_rhs_torch", "uniform_torch", "batch_shapes", "hpl_batch_torch",
]


def mix64_int(z: int) -> int:
    """SplitMix64 output function on a Python int (reference for the vectorised forms)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * MIX1) & MASK64
    z = ((z ^ (z >> 27)) * MIX2) & MASK64
    return z ^ (z >> 31)


def stream_state(seed: int, stream: int) -> int:
    """Initial SplitMix64 state of one stream of one seed."""
    return mix64_int((seed ^ ((stream * STREAM_MULT) & MASK64)) & MASK64)


def _mix64_np(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
    return z ^ (z >> np.uint64(31))


def uniform_np(seed: int, stream: int, k: np.ndarray) -> np.ndarray:
    """Uniform[-0.5, 0.5) FP64 values for counter indices k (uint64 array)."""
    s0 = np.uint64(stream_state(seed, stream))
    with np.errstate(over="ignore"):
        z = s0 + (k.astype(np.uint64) + np.uint64(1)) * np.uint64(GAMMA)
        z = _mix64_np(z)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) - 0.5


def hpl_matrix(n: int, seed: int, diag_shift: float = 0.0, cols: slice | None = None) -> np.ndarray:
    """A (n x n, column-major FP64): i.i.d. uniform[-0.5, 0.5) plus diag_shift on the diagonal.

    `cols` selects a column range (the full matrix by default); the result is then
    n x len(range), still column-major, with the diagonal shift applied where the
    global column index meets the row index.
    """
    c0, c1 = (0, n) if cols is None else (cols.start or 0, n if cols.stop is None else cols.stop)
    out = np.empty((n, c1 - c0), dtype=np.float64, order="F")
    step = max(1, (1 << 24) // max(n, 1))
    rows = np.arange(n, dtype=np.uint64)
    for j0 in range(c0, c1, step):
        j1 = min(c1, j0 + step)
        jj = np.arange(j0, j1, dtype=np.uint64)
        k = rows[:, None] + jj[None, :] * np.uint64(n)
        out[:, j0 - c0:j1 - c0] = uniform_np(seed, STREAM_A, k)
    if diag_shift != 0.0:
        for j in range(c0, c1):
            out[j, j - c0] += diag_shift
    return out


def hpl_rhs(n: int, nrhs: int, seed: int) -> np.ndarray:
    """B (n x nrhs, column-major FP64): i.i.d. uniform[-0.5, 0.5)."""
    k = np.arange(n * nrhs, dtype=np.uint64)
    return np.asfortranarray(uniform_np(seed, STREAM_B, k).reshape(nrhs, n).T)


# ---------------------------------------------------------------- torch forms
# The same draws computed with int64 tensor arithmetic on any device.  int64
# multiplication wraps modulo 2**64 and the right shifts are made logical with
# a mask, so the bits equal the numpy form.

def _s64(v: int) -> int:
    v &= MASK64
    return v - (1 << 64) if v >= (1 << 63) else v


def _lsr(z, s: int):
    return (z >> s) & ((1 << (64 - s)) - 1)


def _mix64_torch(z):
    z = (z ^ _lsr(z, 30)) * _s64(MIX1)
    z = (z ^ _lsr(z, 27)) * _s64(MIX2)
    return z ^ _lsr(z, 31)


def uniform_torch(seed: int, stream: int, k):
    """Torch form of uniform_np; k is an int64 tensor of counter indices."""
    import torch
    s0 = _s64(stream_state(seed, stream))
    z = (k + 1) * _s64(GAMMA) + s0
    z = _mix64_torch(z)
    return _lsr(z, 11).to(torch.float64) * (2.0 ** -53) - 0.5


def hpl_matrix_torch(n: int, seed: int, diag_shift: float = 0.0, device="cpu", dtype=None):
    """Torch form of hpl_matrix: returns an (n, n) tensor with column-major strides (1, n)."""
    import torch
    dtype = torch.float64 if dtype is None else dtype
    out = torch.empty((n, n), dtype=dtype, device=device)  # out[j] is column j; out.t() is A
    step = max(1, (1 << 26) // max(n, 1))
    rows = torch.arange(n, dtype=torch.int64, device=device)
    for j0 in range(0, n, step):
        j1 = min(n, j0 + step)
        jj = torch.arange(j0, j1, dtype=torch.int64, device=device)
        k = rows[None, :] + jj[:, None] * n  # [col, row]
        out[j0:j1, :] = uniform_torch(seed, STREAM_A, k).to(dtype)
    if diag_shift != 0.0:
        out.diagonal().add_(diag_shift)
    return out.t()  # (n, n) with strides (1, n)


def hpl_rhs_torch(n: int, nrhs: int, seed: int, device="cpu"):
    """Torch form of hpl_rhs: an (n, nrhs) FP64 tensor with column-major strides (1, n)."""
    import torch
    k = torch.arange(n * nrhs, dtype=torch.int64, device=device)
    return uniform_torch(seed, STREAM_B, k).reshape(nrhs, n).t()


def batch_shapes(count: int, seed: int, nmin: int = 32, nmax: int = 512, kmax: int = 8):
    """Sizes of a batched workload: n ~ U{nmin..nmax}, nrhs ~ U{1..kmax} (seeded)."""
    rng = np.random.default_rng(seed)
    return rng.integers(nmin, nmax + 1, size=count), rng.integers(1, kmax + 1, size=count)


def hpl_batch_torch(ns, ks, seed: int, shift_per_n: float = 1.0, device="cuda"):
    """Systems i = 0..count-1: A_i = uniform + shift_per_n * n_i * I (matrix seed
    seed * 100000 + i), B_i uniform (same seed), each a column-major view into
    one device buffer per kind.  Returns (A list, B list)."""
    import torch
    na = int(sum(int(n) * int(n) for n in ns))
    nb = int(sum(int(n) * int(k) for n, k in zip(ns, ks)))
    abuf = torch.empty(na, dtype=torch.float64, device=device)
    bbuf = torch.empty(nb, dtype=torch.float64, device=device)
    As, Bs = [], []
    oa = ob = 0
    for i, (n, k) in enumerate(zip(ns, ks)):
        n, k = int(n), int(k)
        a = abuf[oa:oa + n * n].view(n, n).t()  # column-major view, strides (1, n)
        a.copy_(hpl_matrix_torch(n, seed * 100000 + i, diag_shift=shift_per_n * n, device=device))
        b = bbuf[ob:ob + n * k].view(k, n).t()
        b.copy_(hpl_rhs_torch(n, k, seed * 100000 + i, device=device))
        As.append(a)
        Bs.append(b)
        oa += n * n
        ob += n * k
    return As, Bs
