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


def test_resident_handles_match_alone():
    """Resident serving: handles are set up once per problem and reused; each
    request's right-hand sides (1-3) go to the library in one call; the
    solutions in a concurrent mix equal those of the same request solved
    alone (bitwise: fixed summation orders)."""
    import torch
    from paper_1906_10944_gb300 import geneo as G
    from paper_1906_10944_gb300 import serve as S
    k2 = gen.kappa_channels_2d((64, 64), seed=0, contrast=1e6)
    probs = [gen.darcy_problem((64, 64), k2, (4, 4), 1),
             gen.elasticity_problem((12, 6, 6), (3, 1, 1), 1, layer_thickness=1, seed=7)]
    problems, rhs, keep = [], [], []
    for i, prob in enumerate(probs):
        dev = {k: torch.from_numpy(v).cuda() for k, v in G.problem_arrays(prob).items()}
        keep.append(dev)
        opts = G.geneo_default_options(nev_max=10, precision=G.GENEO_PREC_FP32)
        problems.append((G.make_problem(dev, prob.n, prob.n_sub, prob.elem_dofs.shape[1], prob.ndn,
                                        G.GENEO_MEM_DEVICE), opts, prob.n))
        b = np.random.default_rng(i).uniform(-1, 1, (3, prob.n))
        b[:, prob.dirichlet != 0] = 0.0
        rhs.append(torch.from_numpy(b.reshape(-1)).cuda())
    torch.cuda.synchronize()

    def make_solve(pool):
        def solve(req, stream):
            k = req.payload
            n = problems[k][2]
            with torch.cuda.stream(stream):
                x = torch.empty(n * req.nrhs, dtype=torch.float64, device="cuda")
            e = pool.acquire(k, stream)
            try:
                with e.lock:
                    info = G.geneo_pcg_solve(e.handle, rhs[k], x, req.nrhs, 1e-8, 2000, G.GENEO_MEM_DEVICE,
                                             stream=stream)
            finally:
                pool.release(e)
            torch.cuda.synchronize()
            return x.cpu().numpy(), info["converged"]
        return solve

    alone = {}
    for k in range(2):
        for m in (1, 3):
            pool = S.library_pool(problems, 1e12)
            r = S.Server(make_solve(pool), workers=1, make_stream=torch.cuda.Stream).run([S.Request(0, k, nrhs=m)])[0]
            pool.close()
            assert r.error is None, r.error
            alone[(k, m)] = r.result[0]
    pool = S.library_pool(problems, 1e12)
    mix = [S.Request(i, i % 2, nrhs=1 + 2 * ((i // 2) % 2)) for i in range(12)]
    S.Server(make_solve(pool), workers=3, make_stream=torch.cuda.Stream).run(mix)
    st = pool.stats()
    pool.close()
    assert st["setups"] == 2 and st["resident_hits"] == 10
    for r in mix:
        assert r.error is None, r.error
        x, conv = r.result
        assert conv and np.array_equal(x, alone[(r.payload, r.nrhs)])
