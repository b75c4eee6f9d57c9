"""The paper's own variant (HPL-AI rules: diagonally dominant A, no pivoting,
its four block operations) on the GPU against the oracle's no-pivot LU."""
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


def _dev(a):
    import torch
    from paper_2202_13995_gb300 import lu
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        a = a.reshape(-1, 1)
    t = lu.colmajor_empty(a.shape[0], a.shape[1])
    t.copy_(torch.from_numpy(np.asfortranarray(a)))
    return t


@pytest.mark.parametrize("n,nb", [(1, 64), (63, 64), (500, 64), (1500, 256), (2049, 128), (700, 100), (1100, 512),
                                  (1000, 384)])
def test_nopiv_f64_vs_oracle(ctx, n, nb):
    A = I.hpl_matrix(n, 80 + n, diag_shift=n / 4)
    B = I.hpl_rhs(n, 2, 80 + n)
    f = ctx.factor(_dev(A), "f64", nb, nopiv=True)
    assert f.info == 0
    assert np.array_equal(f.ipiv().cpu().numpy(), np.arange(1, n + 1))
    LUo, info = O.getrf_nopiv(A, nb)
    assert info == 0
    LUg = f.lu().cpu().numpy()
    assert np.abs(LUg - LUo).max() <= 256 * n * EPS * max(1.0, np.abs(LUo).max())
    X = _dev(B)
    f.solve_(X)
    Xo = O.getrs(LUo, np.arange(1, n + 1, dtype=np.int32), B)
    assert np.abs(X.cpu().numpy() - Xo).max() / np.abs(Xo).max() <= 1e-10
    assert np.all(O.scaled_residual(A, X.cpu().numpy(), B) < 16.0)


@pytest.mark.parametrize("prec", ["bf16", "fp16"])
def test_nopiv_mixed_refined(ctx, prec):
    n = 3000
    A = I.hpl_matrix(n, 90, diag_shift=n / 4)
    B = I.hpl_rhs(n, 4, 91)
    Ad, Bd = _dev(A), _dev(B)
    f = ctx.factor(Ad, prec, 0, nopiv=True)
    X = _dev(np.zeros((n, 4)))
    iters, res = f.refine(Ad, Bd, X, 16.0, 50)
    assert res < 16.0
    Xo, _, _, _ = O.solve(A, B)
    assert np.abs(X.cpu().numpy() - Xo).max() / np.abs(Xo).max() <= 1e-10


def test_nopiv_f32_paper_precision(ctx):
    """FP32 without refinement, as in the paper's bitstreams: the solve is
    accurate to FP32 level on the diagonally dominant matrix."""
    n = 2048
    A = I.hpl_matrix(n, 92, diag_shift=n / 4)
    b = I.hpl_rhs(n, 1, 92)
    f = ctx.factor(_dev(A), "f32", 256, nopiv=True)
    x = _dev(b)
    f.solve_(x)
    xo, _, _, _ = O.solve(A, b)
    assert np.abs(x.cpu().numpy() - xo).max() / np.abs(xo).max() <= 1e-5


def test_nopiv_zero_pivot_info(ctx):
    n = 300
    A = I.hpl_matrix(n, 93, diag_shift=n / 4)
    A[:, 0] = 0.0  # the first pivot is exactly zero
    f = ctx.factor(_dev(A), "f64", 64, nopiv=True)
    _, info = O.getrf_nopiv(A, 64)
    assert info == 1 and f.info == 1
