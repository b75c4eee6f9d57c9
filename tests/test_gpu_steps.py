"""Parity of each step of the blocked LU iteration (CUDA, through the C ABI)
against the oracle, element by element, on seeded inputs.

Steps (the paper's blocked right-looking iteration): the panel (diagonal +
left blocks, partial pivoting), the top-block triangular solve, and the
inner-block matrix-multiplication update (FP64/FP32 on CUDA cores, BF16/FP16
on the tensor cores with FP32 accumulation)."""
import numpy as np
import pytest

import oracle as O
from paper_2202_13995_gb300 import inputs as I

pytestmark = pytest.mark.gpu
EPS64 = 2.0 ** -53
EPS32 = 2.0 ** -24


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2202_13995_gb300 import lu
    c = lu.Context()
    yield c
    torch.cuda.synchronize()
    c.close()


def _rm(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _panel_input(m, w, seed):
    A = I.hpl_matrix(max(m, w), seed)[:m, :w]
    return np.ascontiguousarray(A)


@pytest.mark.parametrize("m,w", [(1, 1), (5, 3), (64, 64), (100, 37), (300, 32), (1000, 64), (2500, 256),
                                 (9000, 100), (20000, 256)])
def test_panel_f64(ctx, m, w):
    import torch
    P = _panel_input(m, w, 1000 + m + w)
    Pd = _rm(P, torch.float64)
    ipiv = torch.zeros(w, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.step_panel(Pd, ipiv, info, "f64")
    LUo, ipo, info_o = O.getf2(P)
    assert info.item() == info_o == 0
    assert np.array_equal(ipiv.cpu().numpy(), ipo)
    LUg = Pd.cpu().numpy()
    scale = max(1.0, np.abs(LUo).max())
    assert np.abs(LUg - LUo).max() <= 64 * max(m, w) * EPS64 * scale
    assert ctx.status() == 0


@pytest.mark.parametrize("m,w", [(64, 64), (333, 48), (3000, 256)])
def test_panel_f32_exact_on_dyadic(ctx, m, w):
    """A = P^T L U with short dyadic entries: elimination is exact in FP32 too,
    so the FP32 panel must return P, L and U bit for bit."""
    import torch
    rng = np.random.default_rng(m + w)
    L = np.tril(rng.integers(-7, 8, size=(m, w)) / 8.0, -1)
    L[np.arange(w), np.arange(w)] = 1.0
    U = np.triu(rng.integers(-8, 9, size=(w, w)).astype(np.float64))
    U[np.arange(w), np.arange(w)] = rng.integers(1, 9, size=w) * rng.choice([-1.0, 1.0], size=w)
    perm = rng.permutation(m)
    P = np.zeros((m, w))
    P[perm] = L @ U
    Pd = _rm(P, torch.float32)
    ipiv = torch.zeros(w, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.step_panel(Pd, ipiv, info, "f32")
    LUo, ipo, _ = O.getf2(P)
    assert np.array_equal(ipiv.cpu().numpy(), ipo)
    assert np.array_equal(Pd.cpu().numpy().astype(np.float64), LUo)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_panel_nan_is_reported(ctx, prec):
    """A NaN in the panel compares as +inf in the pivot search: it becomes the
    pivot of its column (so every column has a candidate row), the non-finite
    pivot raises LU_ERANGE, and every pivot index stays in range."""
    import torch
    from paper_2202_13995_gb300 import lu
    m, w, row, col = 700, 64, 350, 5
    P = _panel_input(m, w, 11)
    P[row, col] = np.nan
    Pd = _rm(P, torch.float64 if prec == "f64" else torch.float32)
    ipiv = torch.zeros(w, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.step_panel(Pd, ipiv, info, prec)
    assert ctx.status() == lu.LU_ERANGE
    ip = ipiv.cpu().numpy()
    assert ((ip >= np.arange(1, w + 1)) & (ip <= m)).all()
    # where the NaN's row stands after the first `col` interchanges: its pivot
    pos = row
    for j in range(col):
        p = ip[j] - 1
        pos = p if pos == j else (j if pos == p else pos)
    assert ip[col] - 1 == pos
    if prec == "f64":
        # the columns before it never see the NaN: the oracle's pivots
        _, ipo, _ = O.getf2(P[:, :col].copy())
        assert np.array_equal(ip[:col], ipo)


def test_panel_zero_pivot(ctx):
    import torch
    P = _panel_input(200, 40, 7)
    P[:, 13] = 0.0
    Pd = _rm(P, torch.float64)
    ipiv = torch.zeros(40, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.step_panel(Pd, ipiv, info, "f64")
    LUo, ipo, info_o = O.getf2(P)
    assert info_o == 14 and info.item() == 14
    assert np.array_equal(ipiv.cpu().numpy(), ipo)
    assert np.allclose(Pd.cpu().numpy(), LUo, rtol=0, atol=1e-12)


@pytest.mark.parametrize("prec", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("w,N", [(1, 1), (32, 31), (64, 257), (100, 40), (256, 1000), (384, 70), (512, 100),
                                 (257, 33), (256, 3000), (200, 5001)])
def test_trsm(ctx, prec, w, N):
    import torch
    rng = np.random.default_rng(w * 7 + N)
    # the unit-lower factor of a real GEPP (|l| <= 1), as the LU produces it
    Lm, _, _ = O.getf2(I.hpl_matrix(w, 300 + w))
    X = rng.uniform(-1, 1, size=(w, N))
    ldb = max(w, N)  # the kernel shares one row stride: embed both in w x ldb buffers
    Lbuf = np.zeros((w, ldb)); Lbuf[:, :w] = Lm
    Xbuf = np.zeros((w, ldb)); Xbuf[:, :N] = X
    # bf16: the mixed factorizations' form (FP32 arithmetic, inverted diagonal
    # blocks; strips of 8 columns below about 2400 columns, 32 above)
    dt = torch.float64 if prec == "f64" else torch.float32
    Ld, Xd = _rm(Lbuf, dt), _rm(Xbuf, dt)
    ctx.step_trsm(Ld[:, :w], Xd[:, :N], prec)
    want = O.trsm_unit_lower(Lbuf[:, :w] if prec == "f64" else Lbuf[:, :w].astype(np.float32),
                             X if prec == "f64" else X.astype(np.float32))
    got = Xd[:, :N].cpu().numpy().astype(np.float64)
    u = EPS64 if prec == "f64" else EPS32
    assert np.abs(got - want).max() <= 32 * w * u * (np.abs(want).max() + 1.0)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (70, 130, 37), (300, 513, 256), (64, 64, 16)])
def test_gemm_simt(ctx, prec, m, n, k):
    import torch
    rng = np.random.default_rng(m + n + k)
    Cm = rng.uniform(-1, 1, (m, n)); Am = rng.uniform(-1, 1, (m, k)); Bm = rng.uniform(-1, 1, (k, n))
    dt = torch.float64 if prec == "f64" else torch.float32
    if prec == "f32":
        Cm, Am, Bm = (x.astype(np.float32).astype(np.float64) for x in (Cm, Am, Bm))
    Cd, Ad, Bd = _rm(Cm, dt), _rm(Am, dt), _rm(Bm, dt)
    ctx.step_gemm(Cd, Ad, Bd, prec)
    want = O.gemm_update(Cm, Am, Bm)
    got = Cd.cpu().numpy().astype(np.float64)
    u = EPS64 if prec == "f64" else EPS32
    bound = (k + 2) * u * (np.abs(Cm) + np.abs(Am) @ np.abs(Bm))
    assert np.all(np.abs(got - want) <= bound)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
@pytest.mark.parametrize("m,n,k", [(128, 256, 64), (200, 300, 100), (1000, 700, 256), (129, 257, 16),
                                   (4096, 4096, 256), (300, 5000, 512)])
def test_gemm_tensor_core(ctx, prec, m, n, k):
    """C -= A B with A, B rounded to BF16/FP16 (RNE) and FP32 accumulation,
    against the FP64 oracle update of the same rounded operands."""
    import torch
    rng = np.random.default_rng(m * 3 + n + k)
    Cm = rng.uniform(-1, 1, (m, n)).astype(np.float32)
    Am = rng.uniform(-1, 1, (m, k)).astype(np.float32)
    Bm = rng.uniform(-1, 1, (k, n)).astype(np.float32)
    ld = max(k, n)
    Ab = np.zeros((m, ld), np.float32); Ab[:, :k] = Am
    Bb = np.zeros((k, ld), np.float32); Bb[:, :n] = Bm
    Cd, Ad, Bd = _rm(Cm, torch.float32), _rm(Ab, torch.float32), _rm(Bb, torch.float32)
    ctx.step_gemm(Cd, Ad[:, :k], Bd[:, :n], prec)
    rnd = O.round_bf16 if prec == "bf16" else O.round_fp16
    Ar, Br = rnd(Am), rnd(Bm)
    want = O.gemm_update(Cm.astype(np.float64), Ar, Br)
    got = Cd.cpu().numpy().astype(np.float64)
    bound = (k + 4) * EPS32 * (np.abs(Cm) + np.abs(Ar) @ np.abs(Br))
    err = np.abs(got - want)
    assert np.all(err <= bound), (err.max(), (err / bound).max())
    assert ctx.status() == 0


@pytest.mark.parametrize("m,n,k,ldc", [(257, 301, 64, 304), (130, 515, 48, 520), (600, 1027, 256, 1032)])
def test_gemm_tensor_core_strided_ragged(ctx, m, n, k, ldc):
    """C a view with 16-byte aligned rows and a width that is not a multiple
    of 4 (the last columns take the element-wise path); the columns past n
    are untouched."""
    import torch
    rng = np.random.default_rng(m + n + k)
    Cfull = rng.uniform(-1, 1, (m, ldc)).astype(np.float32)
    Am = rng.uniform(-1, 1, (m, k)).astype(np.float32)
    Bm = rng.uniform(-1, 1, (k, n)).astype(np.float32)
    ld = max(k, n)
    Ab = np.zeros((m, ld), np.float32); Ab[:, :k] = Am
    Bb = np.zeros((k, ld), np.float32); Bb[:, :n] = Bm
    Cd = _rm(Cfull, torch.float32)
    Ad, Bd = _rm(Ab, torch.float32), _rm(Bb, torch.float32)
    ctx.step_gemm(Cd[:, :n], Ad[:, :k], Bd[:, :n], "bf16")
    Ar, Br = O.round_bf16(Am), O.round_bf16(Bm)
    want = O.gemm_update(Cfull[:, :n].astype(np.float64), Ar, Br)
    got = Cd.cpu().numpy()
    bound = (k + 4) * EPS32 * (np.abs(Cfull[:, :n]) + np.abs(Ar) @ np.abs(Br))
    assert np.all(np.abs(got[:, :n].astype(np.float64) - want) <= bound)
    assert np.array_equal(got[:, n:], Cfull[:, n:])
    assert ctx.status() == 0


def test_gemm_fp16_overflow_is_reported(ctx):
    import torch
    from paper_2202_13995_gb300 import lu
    Cm = np.zeros((128, 256), np.float32)
    Am = np.ones((128, 256), np.float32)
    Am[5, 7] = 70000.0  # beyond the FP16 range
    Bm = np.ones((64, 256), np.float32)
    Cd, Ad, Bd = _rm(Cm, torch.float32), _rm(Am, torch.float32), _rm(Bm, torch.float32)
    ctx.step_gemm(Cd, Ad[:, :64], Bd, "fp16")
    assert ctx.status() == lu.LU_ERANGE
    assert ctx.status() == 0  # cleared by the read


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_bounded_wait_times_out_and_context_survives(ctx, kind):
    """Failure detection without a fault: a solve's flag wait, a panel's grid
    barrier and a tensor-core mbarrier wait, each on a condition nothing
    satisfies, give up after the library's limit with LU_ETIMEOUT; the status
    is cleared and the same context then factors and solves correctly."""
    import time
    from paper_2202_13995_gb300 import lu
    t0 = time.time()
    assert ctx.wait_probe(kind) == lu.LU_ETIMEOUT
    assert 1.5 < time.time() - t0 < 60.0
    assert ctx.status() == lu.LU_OK
    n = 300
    A = I.hpl_matrix(n, 3)
    B = I.hpl_rhs(n, 1, 3)
    import torch
    At = torch.from_numpy(np.asfortranarray(A)).cuda()
    f = ctx.factor(lu.colmajor_empty(n, n).copy_(At), "f64", 64)
    x = lu.colmajor_empty(n, 1)
    x.copy_(torch.from_numpy(np.asfortranarray(B)).cuda())
    f.solve_(x)
    assert O.scaled_residual(A, x.cpu().numpy(), B)[0] < 16.0
