"""The workspace allocator of lu_create_ex (the ownership rule of the C ABI:
a context's workspace comes from the caller's allocator, e.g. torch's caching
allocator).  A counting allocator over torch.cuda.caching_allocator_alloc /
caching_allocator_delete is plugged in through the C ABI; factor, solve,
refine, residual, step and batched calls are made; the results equal the
default-allocator context's bitwise; and after the context is destroyed every
byte has been handed back."""
import numpy as np
import pytest

from paper_2202_13995_gb300 import inputs as I

pytestmark = pytest.mark.gpu


class Counting:
    def __init__(self):
        self.live = {}
        self.allocs = 0
        self.bytes_total = 0

    def alloc(self, nbytes, stream):
        import torch
        ptr = torch.cuda.caching_allocator_alloc(nbytes, stream=int(stream) if stream else None)
        self.live[ptr] = nbytes
        self.allocs += 1
        self.bytes_total += nbytes
        return ptr

    def release(self, ptr, nbytes, stream):
        import torch
        assert self.live.pop(ptr) == nbytes
        torch.cuda.caching_allocator_delete(ptr)


def _work(ctx, prec, n=1500, nrhs=3):
    import torch
    from paper_2202_13995_gb300 import lu
    A = I.hpl_matrix_torch(n, 7, diag_shift=n / 4 if prec != "f64" else 0.0, device="cuda")
    B = I.hpl_rhs_torch(n, nrhs, 7, device="cuda").contiguous().t().contiguous().t()
    f = ctx.factor(A, prec, 0)
    X = lu.colmajor_empty(n, nrhs)
    if prec == "f64":
        X.copy_(B)
        f.solve_(X)
    else:
        f.refine(A, B, X, 16.0, 50)
    ip = f.ipiv().cpu().numpy()
    res = ctx.scaled_residual(A, X, B)
    f.free()
    # a step-level call (its workspace is the context's too)
    P = torch.from_numpy(np.ascontiguousarray(I.hpl_matrix(600, 3)[:, :64])).cuda()
    pi = torch.zeros(64, dtype=torch.int32, device="cuda")
    inf = torch.zeros(1, dtype=torch.int32, device="cuda")
    ctx.step_panel(P, pi, inf, "f64")
    torch.cuda.synchronize()
    return ip, X.cpu().numpy(), res, P.cpu().numpy()


@pytest.mark.parametrize("prec", ["f64", "bf16"])
def test_counting_allocator_gets_every_byte_back(prec):
    import torch
    from paper_2202_13995_gb300 import lu
    ref_ctx = lu.Context()
    want = _work(ref_ctx, prec)
    ref_ctx.close()
    cnt = Counting()
    ctx = lu.Context(allocator=(cnt.alloc, cnt.release))
    got = _work(ctx, prec)
    # a batched solve through the same context
    ns, ks = np.array([40, 300, 97]), np.array([1, 2, 3])
    As, Bs = I.hpl_batch_torch(ns, ks, 9)
    Xs = [lu.colmajor_empty(int(n), int(k)) for n, k in zip(ns, ks)]
    bt = lu.Batch(ctx, As, Bs, Xs)
    info = torch.zeros(len(ns), dtype=torch.int32, device="cuda")
    bt.run(info)
    bt.free()
    torch.cuda.synchronize()
    assert (info == 0).all()
    assert cnt.allocs > 0 and cnt.live
    ctx.close()
    torch.cuda.synchronize()
    assert cnt.live == {}, cnt.live  # every block handed back
    for a, b in zip(want, got):
        assert np.array_equal(a, b)
