"""The allocation-free PCG entry point (geneo_pcg_solve_noalloc).

It serves callers that may not allocate device memory while solving (fixed
memory budgets, allocator callbacks, request loops); its scratch is a fixed
array inside the library.  This file sorts last so that a run stopping at
the first failure has already run every other test.  It checks, through the
C ABI, that two calls in a row give the same result as geneo_pcg_solve on the
same handle: same iteration count and solutions equal to 1e-10 relative.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


def test_noalloc_pcg_matches_pcg_twice():
    import torch
    from paper_1906_10944_gb300 import geneo as G
    k = gen.kappa_channels_2d((64, 64), seed=0)
    prob = gen.darcy_problem((64, 64), k, (4, 4), 1)
    sol = G.GenEO(prob, nev_max=10)
    try:
        b = torch.from_numpy(prob.b).cuda()
        x_ref = torch.zeros_like(b)
        ref = G.geneo_pcg_solve(sol.h, b, x_ref, 1, 1e-8, 1000)
        xr = x_ref.cpu().numpy()
        for _ in range(2):
            x = torch.full_like(b, 7.0)       # the call must overwrite x
            out = G.geneo_pcg_solve_noalloc(sol.h, b, x, 1e-8, 1000)
            xn = x.cpu().numpy()
            assert out["iterations"] == ref["iterations"]
            assert out["converged"]
            assert np.linalg.norm(xn - xr) <= 1e-10 * np.linalg.norm(xr)
            assert abs(out["kappa_estimate"] - ref["kappa_estimate"]) <= 1e-10 * ref["kappa_estimate"]
        # sizes beyond the fixed scratch are rejected with a clear error
        bad = G.geneo_pcg_solve_noalloc(sol.h, b, x, 1e-8, 5000, raise_on_error=False)
        assert bad["status"] == 1
    finally:
        sol.close()
