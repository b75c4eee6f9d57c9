"""The serving loop (continuous batching): each request's result is the same
alone and in a mix (bitwise), matches the FP64 oracle, resident factors are
reused, evicted under the HBM budget and refactored when asked for again."""
import numpy as np
import pytest

import oracle as O
from paper_2202_13995_gb300 import inputs as I

pytestmark = pytest.mark.gpu
GB = 1 << 30


def _dev(a):
    import torch
    from paper_2202_13995_gb300 import lu
    a = np.asarray(a, dtype=np.float64)
    t = lu.colmajor_empty(a.shape[0], a.shape[1])
    t.copy_(torch.from_numpy(np.asfortranarray(a)))
    return t


def _req(n, k, seed):
    # the served workload's matrices: uniform + (n/4) I
    return I.hpl_matrix(n, seed, diag_shift=n / 4.0), I.hpl_rhs(n, k, seed)


def _solve_one(srv, A, B):
    from paper_2202_13995_gb300 import lu
    Ad, Bd = _dev(A), _dev(B)
    X = lu.colmajor_empty(B.shape[0], B.shape[1])
    r = srv.wait(srv.submit(Ad, Bd, X))
    return r, X.cpu().numpy()


def test_alone_equals_in_mix_and_oracle():
    import torch
    from paper_2202_13995_gb300 import lu
    rng = np.random.default_rng(11)
    # (sizes past 2048 take the server's block width of 256)
    sizes = [(int(n), int(k)) for n, k in zip(np.exp(rng.uniform(np.log(64), np.log(3000), 24)).astype(int),
                                                 rng.integers(1, 17, 24))]
    reqs = [_req(n, k, 500 + i) for i, (n, k) in enumerate(sizes)]
    alone = lu.Server(8 * GB, "fp16", max_slots=1)
    ref = {}
    for i in (0, 5, 13):
        r, x = _solve_one(alone, *reqs[i])
        assert r.status == 0
        ref[i] = x
    alone.close()
    srv = lu.Server(40 * GB, "fp16", max_slots=6)
    dev = [(_dev(A), _dev(B), lu.colmajor_empty(B.shape[0], B.shape[1])) for A, B in reqs]
    tickets = [srv.submit(*d) for d in dev]
    res = [srv.wait(t) for t in tickets]
    torch.cuda.synchronize()
    for i, ((A, B), (Ad, Bd, X), r) in enumerate(zip(reqs, dev, res)):
        assert r.status == 0, (i, r.status)
        assert r.scaled_resid < 16.0
        x = X.cpu().numpy()
        if i in ref:
            assert np.array_equal(x, ref[i]), i  # same bits alone and in the mix
        if A.shape[0] <= 1100:
            xo, _, _, _ = O.solve(A, B)
            assert np.abs(x - xo).max() / np.abs(xo).max() <= 1e-10
    # the slots' work overlapped in time
    spans = sorted((r.t_start_ns, r.t_done_ns) for r in res)
    overlaps = sum(1 for a, b in zip(spans, spans[1:]) if b[0] < a[1])
    assert overlaps > 0
    assert len({r.slot for r in res}) > 1
    srv.close()


def test_resident_factor_reuse_and_eviction():
    from paper_2202_13995_gb300 import lu
    n = 700
    A = I.hpl_matrix(n, 42, diag_shift=n / 4.0)
    B1, B2 = I.hpl_rhs(n, 3, 1), I.hpl_rhs(n, 5, 2)
    Ad = _dev(A)
    # room for two factors of this size at a time
    srv = lu.Server(int(2.5 * lu.fact_bytes(n, 5, "fp16")), "fp16", max_slots=2)
    X1 = lu.colmajor_empty(n, 3)
    r1 = srv.wait(srv.submit(Ad, _dev(B1), X1, factor_key=7, keep_factor=True))
    assert r1.status == 0 and r1.reused_factor == 0
    X2 = lu.colmajor_empty(n, 5)
    r2 = srv.wait(srv.submit(Ad, _dev(B2), X2, factor_key=7, use_resident=True))
    assert r2.status == 0 and r2.reused_factor == 1 and r2.refactored == 0
    xo, _, _, _ = O.solve(A, B2)
    assert np.abs(X2.cpu().numpy() - xo).max() / np.abs(xo).max() <= 1e-10
    # other keep_factor requests push key 7 out of the budget
    for j in range(3):
        Aj = I.hpl_matrix(n, 60 + j, diag_shift=n / 4.0)
        Xj = lu.colmajor_empty(n, 1)
        rj = srv.wait(srv.submit(_dev(Aj), _dev(I.hpl_rhs(n, 1, j)), Xj, factor_key=100 + j, keep_factor=True))
        assert rj.status == 0
    assert srv.stats()["evictions"] >= 1
    X3 = lu.colmajor_empty(n, 5)
    r3 = srv.wait(srv.submit(Ad, _dev(B2), X3, factor_key=7, use_resident=True))
    assert r3.status == 0 and r3.refactored == 1
    assert np.array_equal(X3.cpu().numpy(), X2.cpu().numpy())  # refactored, same bits
    srv.close()


def test_budget_rejects_oversized_request():
    from paper_2202_13995_gb300 import lu
    n = 2048
    A, B = _req(n, 1, 3)
    srv = lu.Server(1 << 20, "fp16", max_slots=1)
    with pytest.raises(lu.LuError) as e:
        srv.submit(_dev(A), _dev(B), lu.colmajor_empty(n, 1))
    assert e.value.code == lu.LU_ENOMEM
    srv.close()


def test_small_requests_take_the_batch_slot():
    """n <= 512 and nrhs <= 8: solved together by the batched solver (slot =
    max_slots), correct against the oracle, same bits alone and in a mix, and
    never resident."""
    from paper_2202_13995_gb300 import lu
    sizes = [(32, 1), (100, 8), (257, 3), (512, 2), (513, 1), (64, 9), (400, 5)]
    reqs = [_req(n, k, 900 + i) for i, (n, k) in enumerate(sizes)]
    alone = lu.Server(8 * GB, "fp16", max_slots=2)
    r0, x0 = _solve_one(alone, *reqs[2])
    assert r0.status == 0 and r0.slot == 2
    alone.close()
    srv = lu.Server(8 * GB, "fp16", max_slots=2)
    dev = [(_dev(A), _dev(B), lu.colmajor_empty(B.shape[0], B.shape[1])) for A, B in reqs]
    tickets = [srv.submit(Ad, Bd, X, factor_key=10 + i, keep_factor=True) for i, (Ad, Bd, X) in enumerate(dev)]
    res = [srv.wait(t) for t in tickets]
    for (n, k), (A, B), (Ad, Bd, X), r in zip(sizes, reqs, dev, res):
        assert r.status == 0 and r.scaled_resid < 16.0
        small = n <= 512 and k <= 8
        assert (r.slot == 2) == small, (n, k, r.slot)
        xo, _, _, _ = O.solve(A, B)
        assert np.abs(X.cpu().numpy() - xo).max() / np.abs(xo).max() <= 1e-10
    assert np.array_equal(dev[2][2].cpu().numpy(), x0)
    # only the two large requests left factors resident
    assert srv.stats()["resident"] == 2
    srv.close()
