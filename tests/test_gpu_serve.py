"""Serving: a request gives the same solution alone and in a concurrent mix
(worker threads on separate CUDA streams; the kernels use fixed summation
orders, so the results are bitwise identical)."""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


def test_concurrent_requests_match_alone():
    import torch
    from paper_1906_10944_gb300 import geneo as G
    from paper_1906_10944_gb300 import serve as S
    k2 = gen.kappa_channels_2d((64, 64), seed=0, contrast=1e6)
    nel = (18, 14, 12)
    k3 = gen.kappa_grf_layers_3d(nel, seed=4, corr_len=0.2, variance=2.0, contrast=1e4,
                                 slab_z=(30, 80), slab_thickness=1)
    probs = [gen.darcy_problem((64, 64), k2, (4, 4), 1), gen.darcy_problem(nel, k3, (3, 2, 2), 2)]
    entries, keep = [], []
    for prob, ek in zip(probs, (4, 8)):
        dev = {k: torch.from_numpy(v).cuda() for k, v in G.problem_arrays(prob).items()}
        keep.append(dev)
        for prec in (G.GENEO_PREC_FP32, G.GENEO_PREC_FP64):
            opts = G.geneo_default_options(nev_max=8, precision=prec)
            entries.append((G.make_problem(dev, prob.n, prob.n_sub, ek, 1, G.GENEO_MEM_DEVICE), opts,
                            torch.from_numpy(prob.b).cuda(), prob.n))

    torch.cuda.synchronize()

    def solve(req, stream):
        p, opts, b, n = entries[req.payload]
        with torch.cuda.stream(stream):
            x = torch.empty(n, dtype=torch.float64, device="cuda")
        h = G.geneo_setup(p, opts, stream)
        try:
            info = G.geneo_pcg_solve(h, b, x, 1, 1e-8, 2000, G.GENEO_MEM_DEVICE, stream=stream)
        finally:
            G.geneo_destroy(h)
        torch.cuda.synchronize()
        return x.cpu().numpy(), info["iterations"]

    alone = [S.Server(solve, workers=1, make_stream=torch.cuda.Stream).run([S.Request(0, k)])[0].result
             for k in range(len(entries))]
    mix = [S.Request(i, i % len(entries)) for i in range(3 * len(entries))]
    S.Server(solve, workers=3, make_stream=torch.cuda.Stream).run(mix)
    for r in mix:
        assert r.error is None, r.error
        x, it = r.result
        assert np.array_equal(x, alone[r.payload][0]) and it == alone[r.payload][1]
