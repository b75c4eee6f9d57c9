"""The diagonal-pivot check of FP32 panels (the mixed and FP32 factorizations).

Partial pivoting picks the diagonal row of a column when its magnitude is the
largest among the candidates.  The library first factors each FP32 panel as if
every pivot were on the diagonal and keeps the result only when every
multiplier is at most 1/2 in magnitude (so the pivot search would have picked
the diagonal); otherwise it restores the panel and runs the full pivot search.
These tests plant a large entry in one column of an otherwise diagonally
dominant matrix, so that the check passes for the first panels and fails in a
later one -- in its diagonal block (stage 1) or in the rows below it (stage 2)
-- and compare the pivots and the refined solution with the FP64 oracle.
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


def _dev(a):
    import torch
    from paper_2202_13995_gb300 import lu
    a = np.asarray(a, dtype=np.float64)
    t = lu.colmajor_empty(a.shape[0], a.shape[1])
    t.copy_(torch.from_numpy(np.asfortranarray(a)))
    return t


def _planted(n, nb, panel, stage, seed):
    """A + (n/4) I with one entry 10 n/4 planted in column j0 of block column
    `panel`: in the block's own rows (stage 1) or near the bottom (stage 2)."""
    A = I.hpl_matrix(n, seed, diag_shift=n / 4)
    k0 = panel * nb
    j0 = k0 + 5
    i0 = k0 + 20 if stage == 1 else n - 3
    A[i0, j0] = 10.0 * n / 4
    return A, j0, i0


@pytest.mark.parametrize("prec", ["bf16", "fp16", "f32"])
@pytest.mark.parametrize("n,nb,panel,stage", [(1536, 64, 5, 1), (1536, 64, 5, 2), (3000, 256, 3, 1),
                                              (3000, 256, 3, 2), (2100, 128, 0, 2)])
def test_check_fails_in_a_later_panel(ctx, prec, n, nb, panel, stage):
    A, j0, i0 = _planted(n, nb, panel, stage, 500 + 10 * panel + stage)
    B = I.hpl_rhs(n, 2, 77)
    Ad, Bd = _dev(A), _dev(B)
    f = ctx.factor(Ad, prec, nb)
    assert f.info == 0
    ip = f.ipiv().cpu().numpy()
    LUo, ipo, info = O.getrf(A, nb)
    assert info == 0
    assert ipo[j0] == i0 + 1                       # the planted entry is the pivot of its column
    assert np.array_equal(ip[:j0], np.arange(1, j0 + 1))  # every earlier pivot on the diagonal
    assert np.array_equal(ip, ipo)
    X = _dev(np.zeros((n, 2)))
    iters, res = f.refine(Ad, Bd, X, 16.0, 50)
    assert res < 16.0
    Xo = O.getrs(LUo, ipo, B)
    kappa = O.cond1_est(LUo, ipo, O.norm_one(A))
    tol = max(1e-10, kappa * 32 * n * EPS)
    assert np.abs(X.cpu().numpy() - Xo).max() / np.abs(Xo).max() <= tol
    assert ctx.status() == 0


@pytest.mark.parametrize("n,nb", [(1000, 64), (2500, 256), (4100, 256)])
def test_checked_factors_match_oracle(ctx, n, nb):
    """When every panel passes the check, the FP32 factors are the no-interchange
    GEPP factors: compared element by element with the oracle's FP64 LU."""
    A = I.hpl_matrix(n, 900 + n, diag_shift=n / 4)
    f = ctx.factor(_dev(A), "f32", nb)
    assert f.info == 0
    assert np.array_equal(f.ipiv().cpu().numpy(), np.arange(1, n + 1))
    LUo, ipo, _ = O.getrf(A, nb)
    LUg = f.lu().cpu().numpy()
    scale = np.abs(LUo).max()
    assert np.abs(LUg - LUo).max() <= 4 * n * 2.0 ** -24 * scale
