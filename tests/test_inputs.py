"""The seeded input generator: numpy, torch and plain-int forms agree bit for bit,
and the draws have the distribution the workloads state."""
import numpy as np
import pytest

from paper_2202_13995_gb300 import inputs as I


def test_int_numpy_torch_agree():
    n = 53
    A = I.hpl_matrix(n, 7, diag_shift=3.5)
    s0 = I.stream_state(7, I.STREAM_A)
    for i, j in [(0, 0), (5, 9), (52, 52), (52, 0)]:
        z = I.mix64_int(s0 + (i + j * n + 1) * I.GAMMA)
        want = (z >> 11) * 2.0 ** -53 - 0.5 + (3.5 if i == j else 0.0)
        assert A[i, j] == want
    torch = pytest.importorskip("torch")
    T = I.hpl_matrix_torch(n, 7, diag_shift=3.5)
    assert T.stride() == (1, n)
    assert np.array_equal(T.numpy(), A)
    B = I.hpl_rhs(n, 4, 8)
    assert np.array_equal(I.hpl_rhs_torch(n, 4, 8).numpy(), B)
    # a column slice regenerates the same values
    assert np.array_equal(I.hpl_matrix(n, 7, 3.5, cols=slice(10, 20)), A[:, 10:20])


def test_splitmix64_published_first_outputs():
    # SplitMix64 with state 0: the first outputs of the published generator
    # (Steele, Lea, Flood 2014; the same as java.util.SplittableRandom's mix)
    assert I.mix64_int(I.GAMMA) == 0xE220A8397B1DCDAF
    assert I.mix64_int(2 * I.GAMMA) == 0x6E789E6AA1B965F4


def test_distribution():
    A = I.hpl_matrix(512, 1)
    assert A.min() >= -0.5 and A.max() < 0.5
    assert abs(A.mean()) < 3e-3
    assert abs(A.var() - 1.0 / 12.0) < 2e-3
    assert I.hpl_matrix(8, 1).tobytes() != I.hpl_matrix(8, 2).tobytes()
