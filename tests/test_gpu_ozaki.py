"""FP64 trailing update by error-free splitting on the BF16 tensor cores
(Ozaki scheme) against the oracle, through the C ABI.

Bars:
  - operands that the slices represent exactly (7-bit integers times a power
    of two): the update equals C - A B bit for bit (every step is exact);
  - any FP64 operands: |C_oz - C_ref| <= u ((1.13 k + 4) 2^(e_i + f_j)
    + (|A||B|)_ij) + 2u |C_ref|, C_ref the compensated (Dot2) update of the
    oracle, u = 2^-53 and 2^e_i, 2^f_j the powers of two just above the
    largest |A(i, :)| and |B(:, j)|: dropped slice pairs (p + q >= 8) < 0.87 k,
    splitting remainders < 0.25 k, the 15 rounded right shifts <= 3.75 (in
    units of u 2^(e_i + f_j)), then the conversion of the integer sum and the
    subtraction round once each;
  - the factorization with this update: the FP64 bars (pivots equal to the
    oracle's, factors and x within the roundoff bounds, scaled residual < 16).
"""
import numpy as np
import pytest

import oracle as O
from paper_2202_13995_gb300 import inputs as I

pytestmark = pytest.mark.gpu
EPS = 2.0 ** -53


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2202_13995_gb300 import lu
    c = lu.Context()
    yield c
    torch.cuda.synchronize()
    c.close()


def _rm(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _dev(a):
    import torch
    from paper_2202_13995_gb300 import lu
    a = np.asarray(a, dtype=np.float64)
    t = lu.colmajor_empty(a.shape[0], a.shape[1])
    t.copy_(torch.from_numpy(np.asfortranarray(a)))
    return t


def _expo(x, axis):
    """e with 2^(e-1) <= max|x| < 2^e along axis (0 for an all-zero line)."""
    mx = np.abs(x).max(axis=axis)
    e = np.zeros(mx.shape, dtype=np.int64)
    nz = mx > 0
    e[nz] = np.frexp(mx[nz])[1]
    return e


def _bound(Am, Bm, ref):
    k = Am.shape[1]
    sc = np.ldexp(1.0, (_expo(Am, 1)[:, None] + _expo(Bm, 0)[None, :]).astype(np.int64))
    return EPS * ((1.13 * k + 4) * sc + np.abs(Am) @ np.abs(Bm)) + 2 * EPS * np.abs(ref)


def _run(ctx, Cm, Am, Bm):
    c = _rm(Cm)
    ctx.step_gemm_ozaki(c, _rm(Am), _rm(Bm))
    return c.cpu().numpy()


# m = 32 takes the kernel's stacked form (four slices of A per 128-row box)
@pytest.mark.parametrize("m,n,k", [(300, 300, 256), (128, 128, 64), (1, 1, 1), (257, 130, 200), (129, 385, 33),
                                   (32, 300, 256), (32, 129, 200), (32, 1300, 64)])
def test_exact_on_sliceable_operands(ctx, m, n, k):
    rng = np.random.default_rng(m * 7 + n + k)
    Am = rng.integers(-127, 128, (m, k)) / 128.0 * 2.0 ** rng.integers(-3, 4, (m, 1))
    Bm = rng.integers(-127, 128, (k, n)) / 128.0 * 2.0 ** rng.integers(-3, 4, (1, n))
    Cm = rng.integers(-2 ** 20, 2 ** 20, (m, n)) * 2.0 ** -14
    want = Cm - Am @ Bm  # exact: every partial sum fits in 53 bits
    got = _run(ctx, Cm, Am, Bm)
    assert np.array_equal(got, want)
    assert ctx.status() == 0


@pytest.mark.parametrize("m,n,k", [(333, 333, 256), (200, 520, 37), (130, 140, 1), (640, 384, 256), (32, 520, 256),
                                   (32, 1000, 37)])
def test_error_bound_against_dot2(ctx, m, n, k):
    rng = np.random.default_rng(m + n + k)
    Am = I.uniform_np(30 + k, 0, np.arange(m * k, dtype=np.uint64)).reshape(m, k)
    Bm = I.uniform_np(30 + k, 1, np.arange(k * n, dtype=np.uint64)).reshape(k, n)
    Cm = rng.standard_normal((m, n))
    ref = O.gemm_update_dot2(Cm, Am, Bm)
    got = _run(ctx, Cm, Am, Bm)
    bound = _bound(Am, Bm, ref)
    err = np.abs(got - ref)
    assert (err <= bound).all(), float((err / bound).max())
    # the plain FP64 update (the oracle's) errs by the same order
    scale = k * np.ldexp(1.0, (_expo(Am, 1)[:, None] + _expo(Bm, 0)[None, :]).astype(np.int64))
    plain = np.abs(O.gemm_update(Cm, Am, Bm) - ref)
    assert (err / scale).max() <= 8 * max((plain / scale).max(), 2.0 ** -56)


def test_wide_dynamic_range_zero_lines(ctx):
    m, n, k = 260, 190, 256
    rng = np.random.default_rng(5)
    Am = rng.standard_normal((m, k)) * 2.0 ** rng.integers(-300, 300, (m, 1))
    Bm = rng.standard_normal((k, n)) * 2.0 ** rng.integers(-300, 300, (1, n))
    Am[7, :] = 0.0
    Bm[:, 11] = 0.0
    Am[9, 3] = 2.0 ** 40  # one dominant entry in a row
    Cm = rng.standard_normal((m, n))
    ref = O.gemm_update_dot2(Cm, Am, Bm)
    got = _run(ctx, Cm, Am, Bm)
    assert (np.abs(got - ref) <= _bound(Am, Bm, ref)).all()
    assert np.array_equal(got[7, :], Cm[7, :])
    assert np.array_equal(got[:, 11], Cm[:, 11])


def test_non_finite_operand_is_reported(ctx):
    from paper_2202_13995_gb300 import lu
    m, n, k = 64, 64, 16
    Am = np.ones((m, k))
    Am[3, 4] = np.nan
    c = _rm(np.zeros((m, n)))
    ctx.step_gemm_ozaki(c, _rm(Am), _rm(np.ones((k, n))))
    assert ctx.status() == lu.LU_ERANGE


def test_k_out_of_range_is_rejected(ctx):
    from paper_2202_13995_gb300 import lu
    with pytest.raises(lu.LuError):
        ctx.step_gemm_ozaki(_rm(np.zeros((4, 4))), _rm(np.zeros((4, 257))), _rm(np.zeros((257, 4))))


@pytest.mark.parametrize("n,nb", [(1, 64), (65, 64), (500, 64), (777, 100), (1500, 256), (2048, 128)])
def test_factor_solve_ozaki(ctx, n, nb):
    A = I.hpl_matrix(n, 40 + n)
    B = I.hpl_rhs(n, 1, 40 + n)
    f = ctx.factor(_dev(A), "f64", nb, ozaki=True)
    assert f.info == 0
    LUo, ipo, info = O.getrf(A, nb)
    assert np.array_equal(f.ipiv().cpu().numpy(), ipo)
    LUg = f.lu().cpu().numpy()
    assert np.abs(LUg - LUo).max() <= 256 * n * EPS * max(1.0, np.abs(LUo).max())
    x = _dev(B)
    f.solve_(x)
    xo = O.getrs(LUo, ipo, B)
    kappa = O.cond1_est(LUo, ipo, O.norm_one(A))
    xg = x.cpu().numpy()
    assert np.abs(xg - xo).max() / np.abs(xo).max() <= max(1e-10, 10 * kappa * EPS), kappa
    assert O.scaled_residual(A, xg, B)[0] < 16.0
    assert ctx.status() == 0


def test_ozaki_nopiv(ctx):
    n = 1024
    A = I.hpl_matrix(n, 9, diag_shift=n / 4.0)
    B = I.hpl_rhs(n, 2, 9)
    f = ctx.factor(_dev(A), "f64", 128, nopiv=True, ozaki=True)
    assert f.info == 0
    LUo, info = O.getrf_nopiv(A, 128)
    LUg = f.lu().cpu().numpy()
    assert np.abs(LUg - LUo).max() <= 256 * n * EPS * max(1.0, np.abs(LUo).max())
    x = _dev(B)
    f.solve_(x)
    assert (O.scaled_residual(A, x.cpu().numpy(), B) < 16.0).all()


def test_ozaki_flag_needs_f64(ctx):
    from paper_2202_13995_gb300 import lu
    A = _dev(I.hpl_matrix(64, 1))
    with pytest.raises(lu.LuError):
        ctx.factor(A, "bf16", 0, ozaki=True)
    with pytest.raises(lu.LuError):
        ctx.factor(A, "f64", 512, ozaki=True)


@pytest.mark.slow
def test_full_size_f64_ozaki_n16384(ctx):
    """n = 16384, nb = 256 with the split update: all 16384 pivots and x
    against the oracle's (the FP64 bars), the first block step's U rows, and
    the scaled residual of the solve."""
    import torch
    from tests.conftest import check_full_size_f64
    n, nb = 16384, 256
    Ad = I.hpl_matrix_torch(n, 2, device="cuda")
    bd = I.hpl_rhs_torch(n, 1, 2, device="cuda")
    f = ctx.factor(Ad, "f64", nb, ozaki=True)
    LUg = f.lu()
    x = bd.clone()
    f.solve_(x)
    torch.cuda.synchronize()
    xg = check_full_size_f64(f, x)
    A = Ad.cpu().numpy()
    O.set_threads(0)
    LU1, ip1, _ = O.getrf(A, nb, ksteps=1)
    U_rows = LUg[:nb, :].cpu().numpy()
    assert np.abs(U_rows - LU1[:nb, :]).max() <= 1e-12 * max(1.0, np.abs(LU1[:nb, :]).max())
    assert O.scaled_residual(A, xg, bd.cpu().numpy()[:, 0]) < 16.0
