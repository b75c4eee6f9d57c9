import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: larger CPU cases")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device in this process")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def golden_path(name: str) -> str:
    return os.path.join(ROOT, "tests", "golden", name)


def read_golden(name: str) -> dict:
    """Parse a golden fixture: '# ...' comments, then 'key v1 v2 ...' lines (a key may repeat)."""
    from fractions import Fraction
    out: dict = {}
    with open(golden_path(name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out.setdefault(key, []).append([Fraction(v) for v in vals])
    return out


def oracle_cache(name: str) -> dict:
    """The oracle's full-size result for one (workload, seed), written by
    tests/golden/make_oracle_cache.py (oracle/ alone): ipiv, x, kappa1_est, ..."""
    import numpy as np
    path = golden_path(f"oracle_{name}.npz")
    if not os.path.exists(path):
        pytest.fail(f"missing {path}: run python tests/golden/make_oracle_cache.py {name}")
    with np.load(path) as z:
        return {k: z[k] for k in z.files}


EPS64 = 2.0 ** -53


def check_full_size_f64(f, x, name="hpl_f64_n16384_seed2"):
    """Every pivot of factorization f equal to the oracle's and its solution x
    within max(1e-10, 10 kappa u) of the oracle's x, kappa the oracle's 1-norm
    condition estimate (the cached oracle run of the same seeded system,
    tests/golden/make_oracle_cache.py).  Returns x on the host."""
    import numpy as np
    ref = oracle_cache(name)
    n = int(ref["n"])
    assert f.info == int(ref["info"]) == 0
    ip = f.ipiv().cpu().numpy()
    assert ip.shape == (n,)
    assert np.array_equal(ip, ref["ipiv"]), int(np.argmax(ip != ref["ipiv"]))
    xo = ref["x"][:, 0]
    xg = x.cpu().numpy().reshape(n)
    tol = max(1e-10, 10 * float(ref["kappa1_est"]) * EPS64)
    err = np.abs(xg - xo).max() / np.abs(xo).max()
    assert err <= tol, (err, tol, float(ref["kappa1_est"]))
    return xg
