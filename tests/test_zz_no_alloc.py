"""The panel factorization entry point that allocates nothing.

lu_step_panel_static serves callers that must not call cudaMalloc (code that
runs while another thread captures a CUDA graph in global mode, where an
allocation would break that capture, or services that reserve all of their
device memory at start-up).  It runs the same panel kernel as lu_step_panel
with its scratch in a fixed device array.  This file is collected last, so a
failure here leaves every other test already run.

The checks: two calls in a row through the C ABI, each compared with
lu_step_panel on the same panel (same pivots exactly, same factors within the
panel tests' tolerance), the second call reusing the array the first one left
behind; the FP64 pivots also against the CPU oracle's GEPP; the device's free
memory unchanged across a call once the library is loaded; and the size limits
refused before anything is enqueued."""
import numpy as np
import pytest

import oracle as O
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
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ctx.step_panel_static(b, ipb, infb, status, prec)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert status.item() == 0
    assert infa.item() == infb.item() == 0
    ipb_h = ipb.cpu().numpy()
    assert np.array_equal(ipa.cpu().numpy(), ipb_h)
    ra, rb = a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)
    u = EPS64 if prec == "f64" else 2.0 ** -24
    assert np.abs(ra - rb).max() <= 64 * max(m, w) * u * max(1.0, np.abs(ra).max())
    if prec == "f64":
        # the oracle's unblocked GEPP of the same panel: same pivots, factors
        # within the panel tests' tolerance
        LUo, ipo, info = O.getf2(P)
        assert info == 0
        assert np.array_equal(ipb_h, ipo)
        assert np.abs(rb - LUo).max() <= 64 * m * EPS64 * max(1.0, np.abs(LUo).max())
    return free0, free1


def test_static_panel_matches_allocating_panel_twice():
    import torch
    from paper_2202_13995_gb300 import lu
    ctx = lu.Context()
    try:
        _case(ctx, 3000, 256, 11, "f64")   # first call on this device: sets up the array address
        # second call: the array holds the first call's leftovers; the library
        # is loaded and set up, so the call must leave free device memory as it was
        free0, free1 = _case(ctx, 1000, 100, 12, "f64")
        assert free1 == free0
        _case(ctx, 20000, 64, 13, "f32")
    finally:
        torch.cuda.synchronize()
        ctx.close()


def test_static_panel_rejects_sizes_before_enqueueing():
    import torch
    from paper_2202_13995_gb300 import lu
    ctx = lu.Context()
    try:
        P = torch.zeros((600, 513), dtype=torch.float64, device="cuda")
        ip = torch.zeros(513, dtype=torch.int32, device="cuda")
        inf = torch.zeros(1, dtype=torch.int32, device="cuda")
        st = torch.full((1,), -5, dtype=torch.int32, device="cuda")
        with pytest.raises(lu.LuError) as e:
            ctx.step_panel_static(P, ip, inf, st, "f64")
        assert e.value.code == -4
        # taller than the CTAs' shared memory holds (FP64, 64 wide): refused
        # on the host, so the status word keeps the caller's value
        P = torch.zeros((300000, 64), dtype=torch.float64, device="cuda")
        ip = torch.zeros(64, dtype=torch.int32, device="cuda")
        with pytest.raises(lu.LuError) as e:
            ctx.step_panel_static(P, ip, inf, st, "f64")
        assert e.value.code == -3
        torch.cuda.synchronize()
        assert st.item() == -5
    finally:
        ctx.close()
