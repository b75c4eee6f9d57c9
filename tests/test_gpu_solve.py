"""End-to-end parity of the GPU solve (lu_factor / lu_solve / lu_refine through
the C ABI) against the CPU oracle, on the seeded HPL-shaped workloads.

Bars (the FP64 oracle decides):
  - FP64 path: pivots identical to the oracle's; factors and x within a few
    units of roundoff times the size; HPL scaled residual < 16;
  - mixed path (BF16/FP16/FP32 factor + FP64 refinement): scaled residual < 16
    and ||x - x_oracle||_inf / ||x_oracle||_inf <= 1e-10 (well-conditioned A);
  - full-size cases: the FP64 configuration's pivots (all of them) and x
    against the oracle's cached run of the same seeded system; the mixed
    configuration (1 and 32 right-hand sides) against a closed-form solution.
"""
import numpy as np
import pytest

import oracle as O
from paper_2202_13995_gb300 import inputs as I
from tests.conftest import check_full_size_f64, oracle_cache

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


def _dev(a):
    import torch
    from paper_2202_13995_gb300 import lu
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        return torch.from_numpy(a.copy()).cuda()
    t = lu.colmajor_empty(a.shape[0], a.shape[1])
    t.copy_(torch.from_numpy(np.asfortranarray(a)))
    return t


def _fwd_tol(LU, ipiv, A):
    kappa = O.cond1_est(LU, ipiv, O.norm_one(A))
    return max(1e-10, 10 * kappa * EPS), kappa


@pytest.mark.parametrize("n,nb", [(1, 64), (2, 64), (3, 1), (63, 64), (64, 64), (65, 64), (129, 32), (500, 64),
                                  (1500, 256), (2048, 128), (777, 100)])
def test_factor_solve_f64(ctx, n, nb):
    A = I.hpl_matrix(n, 40 + n)
    B = I.hpl_rhs(n, 1, 40 + n)
    f = ctx.factor(_dev(A), "f64", nb)
    assert f.info == 0
    LUo, ipo, info = O.getrf(A, nb)
    assert info == 0
    assert np.array_equal(f.ipiv().cpu().numpy(), ipo)
    LUg = f.lu().cpu().numpy()
    assert np.abs(LUg - LUo).max() <= 256 * n * EPS * max(1.0, np.abs(LUo).max())
    x = _dev(B)
    f.solve_(x)
    xo = O.getrs(LUo, ipo, B)
    tol, kappa = _fwd_tol(LUo, ipo, A)
    xg = x.cpu().numpy()
    assert np.abs(xg - xo).max() / np.abs(xo).max() <= tol, kappa
    assert O.scaled_residual(A, xg, B)[0] < 16.0
    assert ctx.scaled_residual(_dev(A), x, _dev(B))[0] < 16.0
    assert ctx.status() == 0


def test_config0_n1024_nb64(ctx):
    """The small configuration: n = 1024, nb = 64, A and b uniform[-0.5, 0.5]."""
    n = 1024
    A = I.hpl_matrix(n, 1)
    B = I.hpl_rhs(n, 1, 1)
    f = ctx.factor(_dev(A), "f64", 64)
    xo, LUo, ipo, _ = O.solve(A, B, nb=64)
    assert np.array_equal(f.ipiv().cpu().numpy(), ipo)
    x = _dev(B)
    f.solve_(x)
    tol, _ = _fwd_tol(LUo, ipo, A)
    assert np.abs(x.cpu().numpy() - xo).max() / np.abs(xo).max() <= tol
    assert O.scaled_residual(A, x.cpu().numpy(), B)[0] < 16.0


@pytest.mark.parametrize("nrhs", [3, 32, 40])
def test_multi_rhs_f64(ctx, nrhs):
    n = 700
    A = I.hpl_matrix(n, 77)
    B = I.hpl_rhs(n, nrhs, 78)
    f = ctx.factor(_dev(A), "f64", 64)
    X = _dev(B)
    f.solve_(X)
    Xo, LUo, ipo, _ = O.solve(A, B)
    tol, _ = _fwd_tol(LUo, ipo, A)
    Xg = X.cpu().numpy()
    assert np.abs(Xg - Xo).max() / np.abs(Xo).max() <= tol
    assert np.all(O.scaled_residual(A, Xg, B) < 16.0)


@pytest.mark.parametrize("prec,n", [("f64", 1000), ("f32", 1537), ("bf16", 2049)])
def test_solve_columns_independent_of_batch(ctx, prec, n):
    """A right-hand side's solution does not depend on the others solved with
    it: 32 columns in one call (chunks of 8 or 16 per CTA, the chunks' chains
    interleaved in one launch), 20 columns (a narrower last chunk), each half
    of 16 and a single column give the same bits; and x against the oracle."""
    A = I.hpl_matrix(n, 90 + n, diag_shift=0.25 * n)
    B = I.hpl_rhs(n, 32, 91 + n)
    f = ctx.factor(_dev(A), prec, 0)
    assert f.info == 0

    def solve(Bc):
        X = _dev(Bc)
        f.solve_(X)
        return X.cpu().numpy()

    X32 = solve(B)
    assert np.array_equal(solve(B[:, :20]), X32[:, :20])
    assert np.array_equal(solve(B[:, :16]), X32[:, :16])
    assert np.array_equal(solve(B[:, 16:]), X32[:, 16:])
    assert np.array_equal(solve(B[:, 21:22]), X32[:, 21:22])
    if prec == "f64":
        Xo, LUo, ipo, _ = O.solve(A, B)
        tol, _ = _fwd_tol(LUo, ipo, A)
        assert np.abs(X32 - Xo).max() / np.abs(Xo).max() <= tol
    else:
        # the low-precision factor's solve is an approximation: its error
        # stays within what the factor's precision allows
        Xo, _, _, _ = O.solve(A, B)
        assert np.abs(X32 - Xo).max() / np.abs(Xo).max() <= (1e-4 if prec == "f32" else 1e-1)


def test_residual_norms_against_oracle(ctx):
    """lu_residual_norms: the four infinity norms per column against the
    oracle's, and both checks (HPL's and the paper's shape) built from them."""
    n, nrhs = 900, 3
    A = I.hpl_matrix(n, 31)
    B = I.hpl_rhs(n, nrhs, 32)
    f = ctx.factor(_dev(A), "f64", 64)
    X = _dev(B)
    f.solve_(X)
    Xg = X.cpu().numpy()
    got = ctx.residual_norms(_dev(A), X, _dev(B))
    assert got.shape == (nrhs, 4)
    R = O.residual(A, Xg, B)
    for q in range(nrhs):
        rn, an, xn, bn = got[q]
        ano = O.norm_inf(A)  # row sums: another summation order on the device
        assert abs(an - ano) <= n * 2.0 ** -53 * ano
        assert xn == O.norm_inf(Xg[:, q])  # maxima are exact
        assert bn == O.norm_inf(B[:, q])
        # r is summed in another order on the device: same magnitude, FP64 rounding apart
        ro = O.norm_inf(R[:, q])
        assert abs(rn - ro) <= 4 * n * 2.0 ** -53 * an * xn
        hpl = O.scaled_residual_from_norms(n, rn, an, xn, bn)
        assert abs(hpl - O.scaled_residual_from_norms(n, ro, an, xn, bn)) <= 4.0
        assert hpl < 16.0
        assert O.paper_residual(n, rn, bn) >= 0.0
    assert np.allclose(ctx.scaled_residual(_dev(A), X, _dev(B)),
                       [O.scaled_residual_from_norms(n, *got[q]) for q in range(nrhs)], rtol=1e-12, atol=0)


def test_all_ones_closed_form(ctx):
    """The paper's validation idea: b = A * ones gives x = ones."""
    n = 1200
    A = I.hpl_matrix(n, 5)
    b = O.residual(A, np.ones(n), np.zeros(n)) * -1.0  # b = A * ones, summed by the oracle
    f = ctx.factor(_dev(A), "f64", 128)
    x = _dev(b)
    f.solve_(x)
    LUo, ipo, _ = O.getrf(A, 128)
    tol, _ = _fwd_tol(LUo, ipo, A)
    assert np.abs(x.cpu().numpy() - 1.0).max() <= 10 * tol * n


def test_singular(ctx):
    from paper_2202_13995_gb300 import lu
    n = 300
    A = I.hpl_matrix(n, 9)
    A[:, 150] = 0.0
    f = ctx.factor(_dev(A), "f64", 64)
    _, _, info = O.getrf(A, 64)
    assert f.info == info == 151
    with pytest.raises(lu.LuError) as e:
        f.solve_(_dev(np.ones(n)))
    assert e.value.code == lu.LU_ESINGULAR


@pytest.mark.parametrize("prec", ["bf16", "fp16", "f32"])
@pytest.mark.parametrize("n,nrhs", [(256, 1), (1000, 1), (2048, 32), (3000, 5)])
def test_mixed_refine(ctx, prec, n, nrhs):
    """Low-precision factor + FP64 refinement reaches the FP64 oracle's x."""
    A = I.hpl_matrix(n, 60 + n, diag_shift=n / 4)
    B = I.hpl_rhs(n, nrhs, 61 + n)
    Ad, Bd = _dev(A), _dev(B)
    f = ctx.factor(Ad, prec, 0)
    assert f.info == 0
    assert np.array_equal(f.ipiv().cpu().numpy(), np.arange(1, n + 1))  # diagonal shift: no interchanges
    X = _dev(np.zeros((n, nrhs)))
    iters, res = f.refine(Ad, Bd, X, 16.0, 50)
    assert res < 16.0 and iters <= 10
    Xo, _, _, _ = O.solve(A, B)
    Xg = X.cpu().numpy()
    assert np.abs(Xg - Xo).max() / np.abs(Xo).max() <= 1e-10
    assert np.all(O.scaled_residual(A, Xg, B) < 16.0)
    assert ctx.status() == 0


def test_mixed_refine_with_pivoting(ctx):
    """No diagonal shift: interchanges happen, and refinement still converges."""
    n = 1024
    A = I.hpl_matrix(n, 3)
    B = I.hpl_rhs(n, 2, 4)
    Ad, Bd = _dev(A), _dev(B)
    f = ctx.factor(Ad, "fp16", 128)
    X = _dev(np.zeros((n, 2)))
    iters, res = f.refine(Ad, Bd, X, 16.0, 50)
    assert res < 16.0
    Xo, LUo, ipo, _ = O.solve(A, B)
    # refinement stops once the scaled residual is below 16, i.e. at a backward
    # error of up to 16 n u: the forward distance to the oracle's x is then
    # bounded by about kappa * (16 + 16) * n * u, not by 1e-10 (kappa ~ 1e4 here)
    kappa = O.cond1_est(LUo, ipo, O.norm_one(A))
    tol = max(1e-10, kappa * 32 * n * EPS)
    assert np.abs(X.cpu().numpy() - Xo).max() / np.abs(Xo).max() <= tol


@pytest.mark.slow
def test_full_size_f64_n16384(ctx):
    """The FP64 configuration at full size (n = 16384, nb = 256): all 16384
    pivots and x against the oracle's, the first block step's U rows, and the
    backward stability of the solve."""
    import torch
    n, nb = 16384, 256
    Ad = I.hpl_matrix_torch(n, 2, device="cuda")
    bd = I.hpl_rhs_torch(n, 1, 2, device="cuda")
    f = ctx.factor(Ad, "f64", nb)
    LUg = f.lu()
    x = bd.clone()
    f.solve_(x)
    torch.cuda.synchronize()
    xg = check_full_size_f64(f, x)
    A = Ad.cpu().numpy()
    # first block step by the oracle: rows 0..nb of U are final after it
    O.set_threads(0)
    LU1, ip1, _ = O.getrf(A, nb, ksteps=1)
    U_rows = LUg[:nb, :].cpu().numpy()
    assert np.abs(U_rows - LU1[:nb, :]).max() <= 1e-12 * max(1.0, np.abs(LU1[:nb, :]).max())
    b = bd.cpu().numpy()[:, 0]
    assert O.scaled_residual(A, xg, b) < 16.0


@pytest.fixture(scope="module")
def mixed_n32768():
    """The mixed configuration's matrix at full size (n = 32768, A + (n/4) I,
    seed 3) on the device and on the host, and 32 right-hand sides with a
    known solution: B = A X_true, computed by the oracle, where column 0 of
    X_true is all ones (the paper's validation vector) and the other columns
    are seeded uniform[-0.5, 0.5) draws."""
    import torch
    n, k = 32768, 32
    Ad = I.hpl_matrix_torch(n, 3, diag_shift=n / 4, device="cuda")
    A = Ad.cpu().numpy()
    Xt = np.asfortranarray(np.concatenate([np.ones((n, 1)), I.hpl_rhs(n, k - 1, 33)], axis=1))
    O.set_threads(0)
    Bh = -O.residual(A, Xt, np.zeros((n, k)))  # oracle: B = A X_true
    Bd = _dev(Bh)
    torch.cuda.synchronize()
    yield {"n": n, "Ad": Ad, "A": A, "Xt": Xt, "B": Bh, "Bd": Bd}
    del Ad, Bd
    torch.cuda.empty_cache()


@pytest.mark.slow
@pytest.mark.parametrize("nrhs", [1, 32])
@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_full_size_mixed_n32768(ctx, mixed_n32768, prec, nrhs):
    """The mixed configuration at full size: identity pivots (the diagonal
    shift), and the refined x within 1e-10 of the closed-form solution
    (kappa ~ 1) for 1 and 32 right-hand sides, every column below scaled
    residual 16."""
    from paper_2202_13995_gb300 import lu
    M = mixed_n32768
    n = M["n"]
    f = ctx.factor(M["Ad"], prec, 0)
    assert f.info == 0
    ip = f.ipiv().cpu().numpy()
    assert np.array_equal(ip, np.arange(1, n + 1))
    Bd = M["Bd"][:, :nrhs]
    X = lu.colmajor_empty(n, nrhs)
    iters, res = f.refine(M["Ad"], Bd, X, 16.0, 50)
    f.free()
    assert res < 16.0
    Xg = X.cpu().numpy()
    Xt = M["Xt"][:, :nrhs]
    err = np.abs(Xg - Xt).max() / np.abs(Xt).max()
    assert err <= 1e-10, err
    assert np.all(np.atleast_1d(O.scaled_residual(M["A"], Xg, M["B"][:, :nrhs])) < 16.0)
    assert ctx.status() == 0


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_full_size_mixed_n32768_vs_oracle(ctx, mixed_n32768, prec):
    """The mixed configuration exactly as benchmarked (A + (n/4) I and b of
    seed 3): pivots and the refined x against the oracle's cached FP64 run
    (tests/golden/make_oracle_cache.py), x within 1e-10 (kappa ~ 4)."""
    import torch
    from paper_2202_13995_gb300 import lu
    ref = oracle_cache("hpl_shift_n32768_seed3")
    M = mixed_n32768
    n = M["n"]
    assert int(ref["n"]) == n
    f = ctx.factor(M["Ad"], prec, 0)
    assert f.info == 0
    assert np.array_equal(f.ipiv().cpu().numpy(), ref["ipiv"])
    bd = I.hpl_rhs_torch(n, 1, 3, device="cuda")
    X = lu.colmajor_empty(n, 1)
    iters, res = f.refine(M["Ad"], bd, X, 16.0, 50)
    f.free()
    torch.cuda.synchronize()
    assert res < 16.0
    xo = ref["x"][:, 0]
    err = np.abs(X.cpu().numpy()[:, 0] - xo).max() / np.abs(xo).max()
    assert err <= max(1e-10, 10 * float(ref["kappa1_est"]) * EPS), err
