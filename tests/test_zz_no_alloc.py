"""The panel factorization entry point that allocates nothing.

lu_step_panel_static serves callers that must not call cudaMalloc (code that
runs while a CUDA graph is being captured in global mode, or services that
reserve all device memory at start-up).  It runs the same panel kernel as
lu_step_panel with its scratch in a fixed device array.  This file is
collected last, so a failure here leaves every other test already run.

The check: two calls in a row through the C ABI, each compared with
lu_step_panel on the same panel (same pivots exactly, same factors within the
panel tests' tolerance), the second call reusing the array the first one left
behind."""
import numpy as np
import pytest

from paper_2202_13995_gb300 import inputs as I

pytestmark = pytest.mark.gpu
EPS64 = 2.0 ** -53


def _case(ctx, m, w, seed, prec):
    import torch
    dt = torch.float64 if prec == "f64" else torch.float32
    P = np.ascontiguousarray(I.hpl_matrix(max(m, w), seed)[:m, :w])
    a = torch.from_numpy(P).to(device="cuda", dtype=dt)
    b = a.clone()
    ipa = torch.zeros(w, dtype=torch.int32, device="cuda")
    ipb = torch.zeros(w, dtype=torch.int32, device="cuda")
    infa = torch.full((1,), -5, dtype=torch.int32, device="cuda")
    infb = torch.full((1,), -5, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -5, dtype=torch.int32, device="cuda")
    ctx.step_panel(a, ipa, infa, prec)
    ctx.step_panel_static(b, ipb, infb, status, prec)
    torch.cuda.synchronize()
    assert status.item() == 0
    assert infa.item() == infb.item() == 0
    assert np.array_equal(ipa.cpu().numpy(), ipb.cpu().numpy())
    ra, rb = a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)
    u = EPS64 if prec == "f64" else 2.0 ** -24
    assert np.abs(ra - rb).max() <= 64 * max(m, w) * u * max(1.0, np.abs(ra).max())


def test_static_panel_matches_allocating_panel_twice():
    import torch
    from paper_2202_13995_gb300 import lu
    ctx = lu.Context()
    try:
        _case(ctx, 3000, 256, 11, "f64")   # first call on this device: sets up the array address
        _case(ctx, 1000, 100, 12, "f64")   # second call: the array holds the first call's leftovers
        _case(ctx, 20000, 64, 13, "f32")
    finally:
        torch.cuda.synchronize()
        ctx.close()


def test_static_panel_rejects_oversized_width():
    import torch
    from paper_2202_13995_gb300 import lu
    ctx = lu.Context()
    try:
        P = torch.zeros((600, 513), dtype=torch.float64, device="cuda")
        ip = torch.zeros(513, dtype=torch.int32, device="cuda")
        inf = torch.zeros(1, dtype=torch.int32, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        with pytest.raises(lu.LuError) as e:
            ctx.step_panel_static(P, ip, inf, st, "f64")
        assert e.value.code == -4
    finally:
        ctx.close()
