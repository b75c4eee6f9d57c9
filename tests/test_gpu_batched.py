"""Batched solves (one persistent launch over many independent systems)
against the FP64 oracle, system by system, and against themselves: a system
gives the same bits alone and inside any batch, with any tuned launch shape."""
import numpy as np
import pytest

import oracle as O
from paper_2202_13995_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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


def make_batch(count, seed, nmin=1, nmax=512, shift=True):
    """The batched workload's shape: n ~ U{nmin..nmax}, 1-8 right-hand sides,
    A = U[-0.5, 0.5] + n I (seeded per system)."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(nmin, nmax + 1, size=count)
    ks = rng.integers(1, 9, size=count)
    As = [I.hpl_matrix(int(n), seed * 100000 + i, diag_shift=float(n) if shift else 0.0) for i, n in enumerate(ns)]
    Bs = [I.hpl_rhs(int(n), int(k), seed * 100000 + i) for i, (n, k) in enumerate(zip(ns, ks))]
    return As, Bs


def run_batch(ctx, As, Bs, tune=False):
    import torch
    from paper_2202_13995_gb300 import lu
    Ad = [_dev(a) for a in As]
    Bd = [_dev(b) for b in Bs]
    Xd = [lu.colmajor_empty(b.shape[0], b.shape[1]) for b in Bs]
    bt = lu.Batch(ctx, Ad, Bd, Xd, tune=tune)
    info = torch.full((len(As),), -7, dtype=torch.int32, device="cuda")
    iters = torch.zeros(len(As), dtype=torch.int32, device="cuda")
    resid = torch.zeros(len(As), dtype=torch.float64, device="cuda")
    bt.run(info, iters, resid)
    torch.cuda.synchronize()
    shape = bt.shape()
    bt.free()
    return ([x.cpu().numpy() for x in Xd], info.cpu().numpy(), iters.cpu().numpy(), resid.cpu().numpy(), shape)


def test_batch_matches_oracle(ctx):
    As, Bs = make_batch(48, 1)
    X, info, iters, resid, _ = run_batch(ctx, As, Bs)
    assert np.all(info == 0), info
    assert np.all(resid < 16.0)
    for A, B, x in zip(As, Bs, X):
        xo, _, _, _ = O.solve(A, B)
        assert np.abs(x - xo).max() / np.abs(xo).max() <= 1e-10
        assert np.all(O.scaled_residual(A, x, B) < 16.0)
    assert iters.max() <= 5


def test_edge_sizes(ctx):
    As, Bs = [], []
    for i, (n, k) in enumerate([(1, 1), (2, 8), (31, 3), (32, 1), (33, 2), (255, 4), (256, 8), (257, 1), (512, 8),
                                (511, 5)]):
        As.append(I.hpl_matrix(n, 700 + i, diag_shift=float(n)))
        Bs.append(I.hpl_rhs(n, k, 700 + i))
    X, info, _, resid, _ = run_batch(ctx, As, Bs)
    assert np.all(info == 0)
    for A, B, x in zip(As, Bs, X):
        xo, _, _, _ = O.solve(A, B)
        assert np.abs(x - xo).max() / np.abs(xo).max() <= 1e-10


def test_alone_equals_in_batch_bitwise(ctx):
    As, Bs = make_batch(24, 2)
    X, _, _, _, _ = run_batch(ctx, As, Bs)
    for i in (0, 7, 23):
        Xa, _, _, _, _ = run_batch(ctx, [As[i]], [Bs[i]])
        assert np.array_equal(Xa[0], X[i])
    # a different batch (other systems, other order) around the same system
    As2, Bs2 = make_batch(9, 3)
    As2.insert(4, As[7])
    Bs2.insert(4, Bs[7])
    X2, _, _, _, _ = run_batch(ctx, As2, Bs2)
    assert np.array_equal(X2[4], X[7])


def test_tuned_shape_gives_same_bits(ctx):
    As, Bs = make_batch(64, 4, nmin=200)
    X0, _, _, _, _ = run_batch(ctx, As, Bs, tune=False)
    X1, info, _, _, shape = run_batch(ctx, As, Bs, tune=True)
    assert np.all(info == 0)
    assert shape[0] in (256, 512) and shape[1] in (1, 2)
    for a, b in zip(X0, X1):
        assert np.array_equal(a, b)


def test_pivoting_and_singular_systems(ctx):
    # no diagonal shift: interchanges happen, refinement still converges
    As = [I.hpl_matrix(120, 900), I.hpl_matrix(300, 901), I.hpl_matrix(64, 902)]
    As[2][:, 10] = 0.0  # exactly singular: info = first zero pivot
    Bs = [I.hpl_rhs(120, 2, 900), I.hpl_rhs(300, 1, 901), I.hpl_rhs(64, 1, 902)]
    X, info, _, _, _ = run_batch(ctx, As, Bs)
    assert info[0] == 0 and info[1] == 0
    _, _, info_o = O.getrf(As[2])
    assert info[2] > 0 and info_o > 0
    for A, B, x in zip(As[:2], Bs[:2], X[:2]):
        assert np.all(O.scaled_residual(A, x, B) < 16.0)


def test_solve_batched_in_place(ctx):
    import torch
    from paper_2202_13995_gb300 import lu
    As, Bs = make_batch(10, 5, nmax=200)
    Ad = [_dev(a) for a in As]
    Bd = [_dev(b) for b in Bs]
    info = torch.zeros(len(As), dtype=torch.int32, device="cuda")
    lu.solve_batched(ctx, Ad, Bd, info)
    assert np.all(info.cpu().numpy() == 0)
    for A, B, xd in zip(As, Bs, Bd):
        xo, _, _, _ = O.solve(A, B)
        x = xd.cpu().numpy()
        assert np.abs(x - xo).max() / np.abs(xo).max() <= 1e-10
