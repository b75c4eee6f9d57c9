"""Pins of the CPU oracle against things other than itself.

Each test checks the oracle against something that the paper or mathematics
fixes: a hand-worked example (tests/golden), exact rational elimination by
brute force, factors constructed so that every step is exact, closed forms,
invariants, and LAPACK through scipy/numpy as a library pin.  A plausible slip
in the oracle (a wrong pivot rule, a dropped term, a sign, a transposed
operand) fails at least one of them.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2202_13995_gb300 import inputs as I
from tests.conftest import read_golden

EPS = 2.0 ** -53


# ----------------------------------------------------------------- brute force

def rational_gepp(A):
    """Exact Gaussian elimination with partial pivoting over the rationals.

    Pivot: the first row of largest |a| in the column (the classical rule, as
    in LAPACK).  Returns (ipiv 1-based, L, U, info) with exact Fractions."""
    n = len(A)
    M = [[Fraction(v) for v in row] for row in A]
    ipiv = []
    info = 0
    for j in range(n):
        p = max(range(j, n), key=lambda i: (abs(M[i][j]), -i))
        ipiv.append(p + 1)
        if M[p][j] != 0:
            M[j], M[p] = M[p], M[j]
            for i in range(j + 1, n):
                M[i][j] = M[i][j] / M[j][j]
        elif info == 0:
            info = j + 1
        for i in range(j + 1, n):
            for c in range(j + 1, n):
                M[i][c] -= M[i][j] * M[j][c]
    L = [[M[i][j] if i > j else Fraction(int(i == j)) for j in range(n)] for i in range(n)]
    U = [[M[i][j] if i <= j else Fraction(0) for j in range(n)] for i in range(n)]
    return ipiv, L, U, info


def _frac_mat(rows):
    return np.array([[float(v) for v in r] for r in rows])


def test_golden_textbook_3x3():
    g = read_golden("gepp_3x3_textbook.txt")
    A = _frac_mat(g["A"])
    LU, ipiv, info = O.getrf(A)
    assert info == 0
    assert list(ipiv) == [int(v) for v in g["ipiv"][0]]
    L = _frac_mat(g["L"])
    U = _frac_mat(g["U"])
    assert np.allclose(np.tril(LU, -1) + np.eye(3), L, rtol=0, atol=4 * EPS)
    assert np.allclose(np.triu(LU), U, rtol=0, atol=16 * EPS)
    b = np.array([float(v) for v in g["b"][0]])
    x = O.getrs(LU, ipiv, b)
    assert np.allclose(x, [float(v) for v in g["x"][0]], rtol=0, atol=64 * EPS)
    # the same factors from the brute-force rational elimination
    rp, rl, ru, _ = rational_gepp([[int(v) for v in r] for r in g["A"]])
    assert rp == [int(v) for v in g["ipiv"][0]]
    assert rl == [list(r) for r in g["L"]] and ru == [list(r) for r in g["U"]]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8])
def test_bruteforce_rational_small(n):
    rng = np.random.default_rng(100 + n)
    for trial in range(20):
        A = rng.integers(-9, 10, size=(n, n))
        rp, rl, ru, rinfo = rational_gepp(A.tolist())
        LU, ipiv, info = O.getrf(A.astype(np.float64))
        assert info == rinfo
        if rinfo:
            continue
        # a pivot decision may only differ from the exact one on an exact tie;
        # ties among integer-valued first columns are exact, later ones are
        # checked by the dyadic construction test
        assert list(ipiv) == rp, (A, ipiv, rp)
        L = np.array([[float(v) for v in r] for r in rl])
        U = np.array([[float(v) for v in r] for r in ru])
        scale = max(1.0, np.abs(U).max())
        assert np.allclose(np.tril(LU, -1) + np.eye(n), L, rtol=0, atol=64 * n * EPS)
        assert np.allclose(np.triu(LU), U, rtol=0, atol=64 * n * EPS * scale)


def test_first_index_wins_ties():
    # column 0 holds 3 and -3: the first (row 1, 0-based) must win
    A = np.array([[1.0, 2, 0, 1], [3, 1, 1, 0], [-3, 4, 2, 1], [2, 0, 1, 5]])
    LU, ipiv, _ = O.getrf(A)
    assert ipiv[0] == 2
    rp, _, _, _ = rational_gepp(A.astype(int).tolist())
    assert list(ipiv) == rp


def _dyadic_plu(n, rng, perm=None):
    """A = P^T L U with every value a short dyadic rational, so that elimination
    is exact in FP64; |l_ij| < 1 below the diagonal forces the pivot rows."""
    L = np.tril(rng.integers(-7, 8, size=(n, n)) / 8.0, -1) + np.eye(n)
    U = np.triu(rng.integers(-16, 17, size=(n, n)).astype(np.float64))
    d = rng.integers(1, 17, size=n) * rng.choice([-1.0, 1.0], size=n)
    U[np.arange(n), np.arange(n)] = d
    if perm is None:
        perm = rng.permutation(n)
    # row perm[i] of A holds row i of L U
    A = np.zeros((n, n))
    A[perm] = L @ U
    return A, L, U, perm


def _ipiv_to_perm(ipiv, n):
    rows = np.arange(n)
    for k, p in enumerate(ipiv):
        rows[[k, p - 1]] = rows[[p - 1, k]]
    return rows


@pytest.mark.parametrize("n,nb", [(8, None), (33, None), (64, None), (64, 8), (64, 16), (50, 7)])
def test_constructed_plu_exact(n, nb):
    rng = np.random.default_rng(n * 7 + (nb or 0))
    A, L, U, perm = _dyadic_plu(n, rng)
    LU, ipiv, info = O.getrf(A, nb)
    assert info == 0
    assert np.array_equal(np.tril(LU, -1) + np.eye(n), L)
    assert np.array_equal(np.triu(LU), U)
    # the interchanges rebuild the permutation: position k holds original row perm[k]
    assert np.array_equal(_ipiv_to_perm(ipiv, n), perm)


def test_closed_form_all_ones():
    # the paper's validation input idea: b = A * ones, so x = ones
    n = 64
    A, L, U, _ = _dyadic_plu(n, np.random.default_rng(3))
    b = A @ np.ones(n)  # exact: short dyadic values
    x, LU, ipiv, _ = O.solve(A, b)
    kappa = O.cond1_est(LU, ipiv, O.norm_one(A))
    assert np.abs(x - 1.0).max() <= 10 * kappa * n * EPS


def test_hpl_random_all_ones_and_residual():
    n = 300
    A = I.hpl_matrix(n, 11)
    b = A @ np.ones(n)
    x, LU, ipiv, info = O.solve(A, b, nb=32)
    assert info == 0
    kappa = O.cond1_est(LU, ipiv, O.norm_one(A))
    assert np.abs(x - 1.0).max() <= 10 * kappa * n * EPS
    assert O.scaled_residual(A, x, b) < 16.0


@pytest.mark.parametrize("n", [257, 1000])
def test_lapack_pin(n):
    sl = pytest.importorskip("scipy.linalg")
    A = I.hpl_matrix(n, 20 + n)
    B = I.hpl_rhs(n, 3, 20 + n)
    X, LU, ipiv, info = O.solve(A, B, nb=64)
    lu, piv = sl.lu_factor(A)
    assert np.array_equal(piv + 1, ipiv)
    kappa = O.cond1_est(LU, ipiv, O.norm_one(A))
    Xl = np.linalg.solve(A, B)
    tol = max(1e-10, 10 * kappa * n * EPS)
    assert np.abs(X - Xl).max() / np.abs(Xl).max() <= tol
    assert np.abs(LU - lu).max() <= 1e3 * n * EPS * np.abs(lu).max()


def test_blocked_equals_unblocked_bitwise():
    # the blocked iteration accumulates every element in the same k order
    A = I.hpl_matrix(200, 5)
    LU1, p1, _ = O.getrf(A)
    for nb in (1, 16, 64, 199, 256):
        LU2, p2, _ = O.getrf(A, nb)
        assert np.array_equal(p1, p2) and np.array_equal(LU1, LU2)


def test_blocked_steps_partial():
    A = I.hpl_matrix(96, 8)
    LU, p, _ = O.getrf(A, 32, ksteps=1)
    # after one step rows 0..31 are final; the first 32 columns of L are final
    # up to the later panels' row interchanges
    LUf, pf, _ = O.getrf(A, 32)
    assert np.array_equal(p[:32], pf[:32])
    assert np.array_equal(LU[:32, :], LUf[:32, :])
    assert np.array_equal(O.laswp(LU, 0, 32, 32, 96, pf)[:, :32], LUf[:, :32])


def test_diag_shift_gives_identity_pivots():
    n = 256
    A = I.hpl_matrix(n, 3, diag_shift=n / 4)
    _, ipiv, _ = O.getrf(A, 64)
    assert np.array_equal(ipiv, np.arange(1, n + 1))


def test_singular_info():
    n = 6
    A = I.hpl_matrix(n, 4)
    A[:, 3] = 0.0
    LU, ipiv, info = O.getrf(A)
    assert info == 4
    A2 = I.hpl_matrix(n, 4)
    A2[:, 2] = A2[:, 0] * 2.0 - A2[:, 1] * 0.5  # dependent -> tiny (or zero) pivot
    _, _, info2 = O.getrf(np.zeros((3, 3)))
    assert info2 == 1


def test_scaled_residual_golden():
    g = read_golden("scaled_residual_2x2.txt")
    A = _frac_mat(g["A"])
    x = np.array([float(v) for v in g["x"][0]])
    b = np.array([float(v) for v in g["b"][0]])
    r = O.residual(A, x, b)
    assert np.array_equal(r, [float(v) for v in g["r"][0]])
    want = float(g["scaled_num"][0][0] / g["scaled_den"][0][0])
    got = O.scaled_residual(A, x, b)
    assert abs(got - want) <= 1e-15 * want
    want_p = float(g["paper_num"][0][0] / g["paper_den"][0][0])
    got_p = O.paper_residual(2, O.norm_inf(r), O.norm_inf(b))
    assert abs(got_p - want_p) <= 1e-15 * want_p


def test_residual_and_norms_library_pin():
    rng = np.random.default_rng(9)
    A = rng.standard_normal((40, 40))
    X = rng.standard_normal((40, 3))
    B = rng.standard_normal((40, 3))
    R = O.residual(A, X, B)
    assert np.allclose(R, B - A @ X, rtol=0, atol=1e-12)
    assert O.norm_inf(A) == pytest.approx(np.linalg.norm(A, np.inf), rel=1e-14)
    assert O.norm_one(A) == pytest.approx(np.linalg.norm(A, 1), rel=1e-14)
    assert O.norm_inf(X[:, 1]) == np.abs(X[:, 1]).max()


def test_residual_sums_in_column_order_on_any_thread_count():
    """r_i = b_i - a_i1 x_1 - a_i2 x_2 - ... in that order (one rounding per
    product and per subtraction), bit for bit, whether the oracle's threads
    split the rows or not: the definition, written here with numpy column by
    column, over several row blocks and a ragged tail."""
    rng = np.random.default_rng(17)
    n, k = 600, 3
    A = rng.standard_normal((n, n))
    X = rng.standard_normal((n, k))
    B = rng.standard_normal((n, k))
    want = B.copy()
    for j in range(n):
        want = want - A[:, j:j + 1] * X[j:j + 1, :]
    t0 = O.num_threads()
    try:
        for t in (1, max(2, t0)):
            O.set_threads(t)
            assert np.array_equal(O.residual(A, X, B), want)
    finally:
        O.set_threads(t0)


def test_cond_estimate_against_exact():
    rng = np.random.default_rng(1)
    for n in (5, 20, 60):
        for _ in range(5):
            A = rng.standard_normal((n, n))
            LU, ipiv, _ = O.getrf(A)
            est = O.cond1_est(LU, ipiv, O.norm_one(A))
            exact = np.linalg.cond(A, 1)
            assert est <= exact * (1 + 1e-8)
            assert est >= exact / 10


def test_kernel_steps_library_pins():
    rng = np.random.default_rng(2)
    m, n, k = 37, 29, 11
    Cm = rng.standard_normal((m, n)); Am = rng.standard_normal((m, k)); Bm = rng.standard_normal((k, n))
    assert np.allclose(O.gemm_update(Cm, Am, Bm), Cm - Am @ Bm, rtol=0, atol=1e-12)
    Lm = rng.standard_normal((k, k))
    Bt = rng.standard_normal((k, 7))
    Lu = np.tril(Lm, -1) + np.eye(k)
    assert np.allclose(O.trsm_unit_lower(Lm, Bt), np.linalg.solve(Lu, Bt), rtol=0, atol=1e-9)
    A = rng.standard_normal((10, 6))
    ipiv = np.array([3, 2, 10, 4, 9], dtype=np.int32)
    got = O.laswp(A, 0, 6, 0, 5, ipiv)
    want = A.copy()
    for kk, p in enumerate(ipiv):
        want[[kk, p - 1]] = want[[p - 1, kk]]
    assert np.array_equal(got, want)


def test_round_16bit_library_pin_and_special_values():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    f = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-9, 6, 20000),
                        [0.0, -0.0, 65504.0, 65519.0, 65520.0, 1e-8, 6e-8, 3e-8]]).astype(np.float32)
    assert np.array_equal(O.round_bf16(f), torch.from_numpy(f).bfloat16().double().numpy())
    assert np.array_equal(O.round_fp16(f), f.astype(np.float16).astype(np.float64))
    # ties go to even
    one = np.float32(1.0)
    assert O.round_bf16(np.array([one + np.float32(2.0 ** -8)]))[0] == 1.0
    assert O.round_bf16(np.array([one + np.float32(3 * 2.0 ** -8)]))[0] == 1.0 + 2.0 ** -6
    assert O.round_fp16(np.array([one + np.float32(2.0 ** -11)]))[0] == 1.0
    assert O.round_fp16(np.array([np.float32(65520.0)]))[0] == np.inf
    assert O.round_fp16(np.array([np.float32(65519.0)]))[0] == 65504.0


# ----------------------------------------------------------------- the paper's no-pivot variant

def test_nopiv_recovers_constructed_lu_exactly():
    # A = L U with short dyadic entries (no interchanges): every step is exact
    for n, nb in [(8, None), (64, None), (64, 16), (50, 7)]:
        rng = np.random.default_rng(n + (nb or 0))
        L = np.tril(rng.integers(-7, 8, size=(n, n)) / 8.0, -1) + np.eye(n)
        U = np.triu(rng.integers(-16, 17, size=(n, n)).astype(np.float64))
        U[np.arange(n), np.arange(n)] = rng.integers(1, 17, size=n)
        LU, info = O.getrf_nopiv(L @ U, nb)
        assert info == 0
        assert np.array_equal(np.tril(LU, -1) + np.eye(n), L)
        assert np.array_equal(np.triu(LU), U)


def test_nopiv_equals_gepp_when_pivots_are_diagonal():
    # the diagonal shift makes every partial pivot the diagonal: GEPP performs
    # exactly the no-pivot operations, so the factors agree bit for bit
    n = 300
    A = I.hpl_matrix(n, 31, diag_shift=n / 4)
    LUp, ipiv, _ = O.getrf(A)
    assert np.array_equal(ipiv, np.arange(1, n + 1))
    for nb in (None, 32, 64, 299):
        LUn, info = O.getrf_nopiv(A, nb)
        assert info == 0 and np.array_equal(LUn, LUp)


def test_nopiv_bruteforce_rational():
    for n in (2, 3, 5, 7):
        rng = np.random.default_rng(40 + n)
        A = rng.integers(-9, 10, size=(n, n)) + np.diag(rng.integers(30, 40, size=n))
        M = [[Fraction(int(v)) for v in row] for row in A]
        for j in range(n):
            for i in range(j + 1, n):
                M[i][j] = M[i][j] / M[j][j]
                for c in range(j + 1, n):
                    M[i][c] -= M[i][j] * M[j][c]
        LU, info = O.getrf_nopiv(A.astype(np.float64))
        want = np.array([[float(v) for v in r] for r in M])
        assert np.allclose(LU, want, rtol=0, atol=64 * n * EPS * 40)


def test_trsm_right_upper_library_pin():
    rng = np.random.default_rng(8)
    U = np.triu(rng.uniform(-1, 1, (20, 20))) + 4 * np.eye(20)
    B = rng.uniform(-1, 1, (13, 20))
    assert np.allclose(O.trsm_right_upper(B, U), B @ np.linalg.inv(U), rtol=0, atol=1e-12)


# ----------------------------------------------------------------- compensated update (Dot2)

def _exact_update(Cm, Am, Bm):
    m, k = Am.shape
    n = Bm.shape[1]
    out = [[Fraction(Cm[i, j]) for j in range(n)] for i in range(m)]
    for i in range(m):
        for j in range(n):
            acc = out[i][j]
            for t in range(k):
                acc -= Fraction(Am[i, t]) * Fraction(Bm[t, j])
            out[i][j] = acc
    return out


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (3, 4, 7), (9, 5, 33)])
def test_dot2_update_is_correctly_rounded_up_to_gamma_squared(m, n, k):
    """Against exact rational arithmetic: |dot2 - exact| <= u |exact| + 4 gamma^2 (|C| + |A||B|)."""
    rng = np.random.default_rng(100 + k)
    Cm = rng.standard_normal((m, n)) * 2.0 ** rng.integers(-20, 20, (m, n))
    Am = rng.standard_normal((m, k)) * 2.0 ** rng.integers(-20, 20, (m, k))
    Bm = rng.standard_normal((k, n)) * 2.0 ** rng.integers(-20, 20, (k, n))
    got = O.gemm_update_dot2(Cm, Am, Bm)
    ex = _exact_update(Cm, Am, Bm)
    g = (k + 1) * EPS / (1 - (k + 1) * EPS)
    mag = np.abs(Cm) + np.abs(Am) @ np.abs(Bm)
    for i in range(m):
        for j in range(n):
            err = abs(Fraction(got[i, j]) - ex[i][j])
            assert err <= EPS * abs(ex[i][j]) + 4 * Fraction(g * g) * Fraction(mag[i, j])


def test_dot2_recovers_what_plain_fp64_cancels():
    """1e16 + 1 - 1e16: plain FP64 loses the 1, the compensated sum keeps it."""
    Am = np.array([[1e16, 1.0, -1e16]])
    Bm = np.ones((3, 1))
    Cm = np.zeros((1, 1))
    assert O.gemm_update(Cm, Am, Bm)[0, 0] != -1.0
    assert O.gemm_update_dot2(Cm, Am, Bm)[0, 0] == -1.0
