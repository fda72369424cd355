"""The allocation-free PCG entry point (geneo_pcg_solve_noalloc).

Some callers cannot allocate device memory while they solve: code running
under a fixed device-memory budget, inside an allocator's own callbacks, or
in a request loop where a cudaMalloc would stall the device.  For them the
library solves with a fixed scratch array it holds itself.  This file sorts
last so that a run stopping at the first failure has already run every
other test.  Through the C ABI it checks that two calls in a row give the
result of geneo_pcg_solve on the same handle (same iteration count,
solutions equal to 1e-10 relative), that the calls leave the device's free
memory unchanged, the size limit (4095 accepted, 4096 rejected) and that a
profiled handle is rejected.
"""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


def _problem():
    k = gen.kappa_channels_2d((64, 64), seed=0)
    return gen.darcy_problem((64, 64), k, (4, 4), 1)


def test_noalloc_pcg_matches_pcg_twice():
    import torch
    from paper_1906_10944_gb300 import geneo as G
    prob = _problem()
    sol = G.GenEO(prob, nev_max=10)
    try:
        b = torch.from_numpy(prob.b).cuda()
        x_ref = torch.zeros_like(b)
        ref = G.geneo_pcg_solve(sol.h, b, x_ref, 1, 1e-8, 1000)
        xr = x_ref.cpu().numpy()
        x = torch.full_like(b, 7.0)
        G.geneo_pcg_solve_noalloc(sol.h, b, x, 1e-8, 1000)   # first call: symbol lookup
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):
            x = torch.full_like(b, 7.0)       # the call must overwrite x
            out = G.geneo_pcg_solve_noalloc(sol.h, b, x, 1e-8, 1000)
            xn = x.cpu().numpy()
            assert out["iterations"] == ref["iterations"]
            assert out["converged"] and out["true_residual"] <= 1e-8
            assert np.linalg.norm(xn - xr) <= 1e-10 * np.linalg.norm(xr)
            assert abs(out["kappa_estimate"] - ref["kappa_estimate"]) <= 1e-10 * ref["kappa_estimate"]
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        # the size limit of the fixed scratch: 4095 accepted, 4096 rejected
        ok = G.geneo_pcg_solve_noalloc(sol.h, b, x, 1e-8, 4095, raise_on_error=False)
        assert ok["status"] in (0, 5) and ok["converged"]
        bad = G.geneo_pcg_solve_noalloc(sol.h, b, x, 1e-8, 4096, raise_on_error=False)
        assert bad["status"] == 1
    finally:
        sol.close()


def test_noalloc_rejects_profiled_handle():
    import torch
    from paper_1906_10944_gb300 import geneo as G
    prob = _problem()
    sol = G.GenEO(prob, nev_max=10, profile=1)
    try:
        b = torch.from_numpy(prob.b).cuda()
        x = torch.zeros_like(b)
        out = G.geneo_pcg_solve_noalloc(sol.h, b, x, 1e-8, 1000, raise_on_error=False)
        assert out["status"] == 1
    finally:
        sol.close()
