"""The device generator of the seeded inputs (lu_generate) against the host
generator of the package (paper_2202_13995_gb300/inputs.py, itself pinned to
SplitMix64's published outputs in tests/test_inputs.py): the same bits for the
matrix (with and without the diagonal shift, ragged sizes, a leading dimension
larger than the rows) and the right-hand sides."""
import numpy as np
import pytest

from paper_2202_13995_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,seed,shift", [(1, 1, 0.0), (77, 2, 0.0), (300, 3, 75.0), (1024, 12345, 256.0)])
def test_matrix_bits(n, seed, shift):
    import torch
    from paper_2202_13995_gb300 import lu
    A = lu.colmajor_empty(n, n)
    lu.generate(A, seed, 0, shift)
    torch.cuda.synchronize()
    want = I.hpl_matrix(n, seed, diag_shift=shift)
    assert np.array_equal(A.cpu().numpy().view(np.uint64), want.view(np.uint64))


def test_rhs_bits_and_leading_dimension():
    import torch
    from paper_2202_13995_gb300 import lu
    n, k = 513, 7
    buf = torch.full((k, n + 5), 9.0, dtype=torch.float64, device="cuda")
    B = buf.t()[:n, :]  # column-major, ld = n + 5
    lu.generate(B, 4, 1)
    torch.cuda.synchronize()
    want = I.hpl_rhs(n, k, 4)
    assert np.array_equal(B.cpu().numpy(), want)
    assert (buf[:, n:] == 9.0).all()  # the padding rows are untouched
