"""Write the oracle's full-size results for the seeded workloads to tests/golden/.

    python tests/golden/make_oracle_cache.py [NAME ...]

Each cache file holds what the full-size GPU tests compare against: the
oracle's pivots (LAPACK ipiv, 1-based), its solution x, its condition
estimate (Hager/Higham 1-norm estimate from its own LU) and its scaled
residual, for one (workload, seed).  Everything in it is computed here by
`oracle/` alone (plain FP64 C GEPP, the paper's blocked right-looking
iteration with partial pivoting, then the forward and back substitution);
the inputs come from the seeded generator in paper_2202_13995_gb300/inputs.py,
which holds no solver arithmetic.  The oracle is deterministic (every element
accumulates in a fixed order, compiled with -ffp-contract=off), so the file
is the same on any host.

Runs on all host cores (OpenMP); n = 16384 takes a few minutes, n = 32768
about eight times as long.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2202_13995_gb300 import inputs as I  # noqa: E402

# name -> (n, nb, seed, diagonal shift as a fraction of n, nrhs)
CASES = {
    # the FP64 configuration: n = 16384, nb = 256, A and b uniform[-0.5, 0.5)
    "hpl_f64_n16384_seed2": (16384, 256, 2, 0.0, 1),
    # the mixed configuration's matrix and right-hand side: A + (n/4) I, n = 32768
    "hpl_shift_n32768_seed3": (32768, 256, 3, 0.25, 1),
}


def cache_path(name: str) -> str:
    return os.path.join(HERE, f"oracle_{name}.npz")


def make(name: str) -> str:
    n, nb, seed, shift, nrhs = CASES[name]
    O.set_threads(os.cpu_count() or 1)
    t0 = time.time()
    A = I.hpl_matrix(n, seed, diag_shift=shift * n)
    B = I.hpl_rhs(n, nrhs, seed)
    LU, ipiv, info = O.getrf(A, nb)
    X = O.getrs(LU, ipiv, B)
    kappa = O.cond1_est(LU, ipiv, O.norm_one(A))
    del LU
    res = O.scaled_residual(A, X, B)
    out = cache_path(name)
    np.savez_compressed(out, n=n, nb=nb, seed=seed, shift=shift, nrhs=nrhs, info=info,
                        ipiv=ipiv.astype(np.int32), x=np.asarray(X, dtype=np.float64),
                        kappa1_est=kappa, scaled_residual=np.atleast_1d(res))
    print(f"{name}: {O.num_threads()} threads, {time.time() - t0:.0f} s", flush=True)
    return out


def load(name: str) -> dict:
    with np.load(cache_path(name)) as z:
        return {k: z[k] for k in z.files}


if __name__ == "__main__":
    names = sys.argv[1:] or list(CASES)
    for nm in names:
        t = time.time()
        p = make(nm)
        print(f"{nm}: wrote {os.path.relpath(p, ROOT)} in {time.time() - t:.0f} s", flush=True)
