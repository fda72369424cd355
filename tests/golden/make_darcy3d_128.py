"""Write the oracle's results on the 3D Darcy 128^3 workload to
darcy3d_128_oracle.json (the GPU parity test at full size reads them).

Workload: Q1 on 128^3 elements (2,146,689 dofs), kappa = exp(Gaussian field,
seed 1) with four 1e6-contrast slabs, 8 x 8 x 8 boxes of 16^3 elements grown
by two element layers, tau = 0.3, nev_max = 20 (standard partition of unity,
paper form of the eigenproblem, Section 4.3).  Calls only ``gen`` (inputs)
and ``oracle``; the per-subdomain eigenproblems run in forked worker
processes (no CUDA in this process).  About 15 minutes on 8 cores, 30 GB.

    python tests/golden/make_darcy3d_128.py [--workers N]
"""
import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")

import numpy as np  # noqa: E402

import gen  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "darcy3d_128_oracle.json")
N_SAMPLE = 4096


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=os.cpu_count())
    args = ap.parse_args()
    t0 = time.time()
    kap = gen.kappa_grf_layers_3d((128, 128, 128), seed=1)
    prob = gen.darcy_problem((128, 128, 128), kap, (8, 8, 8), 2)
    opts = oracle.OracleOptions(tau=0.3, nev_max=20)
    orc = oracle.GenEOOracle(prob, opts, workers=args.workers, mp_context="fork")
    t_setup = time.time() - t0
    print("setup %.1f s, dim V_H %d" % (t_setup, orc.dim_H), flush=True)
    x, it, hist, kappa = orc.solve(tol=1e-8, maxit=2000)
    bn = np.linalg.norm(prob.b)
    res = float(np.linalg.norm(prob.b - prob.A @ x) / bn)
    first = int(np.argmax(np.asarray(hist) <= 1e-8))
    print("tol 1e-8: %d iterations (%d to the recursive tol), true residual %.3e, kappa %.4f"
          % (it, first, res, kappa), flush=True)
    xs, its, _, _ = orc.solve(tol=1e-12, maxit=4000)
    res_s = float(np.linalg.norm(prob.b - prob.A @ xs) / bn)
    print("tol 1e-12: %d iterations, true residual %.3e" % (its, res_s), flush=True)
    rng = np.random.default_rng(20240601)
    free = np.nonzero(prob.dirichlet == 0)[0]
    idx = np.sort(rng.choice(free, size=N_SAMPLE, replace=False))
    nev = opts.nev_max
    out = {
        "what": "FP64 CPU oracle on 3D Darcy Q1 128^3 (2,146,689 dofs), kappa = exp(GRF l=0.1 "
                "s2=4, seed 1) x 1e6 slabs, 8x8x8 boxes of 16^3 grown by 2, tau 0.3, nev_max 20; "
                "written by tests/golden/make_darcy3d_128.py",
        "n": int(prob.n), "n_sub": int(prob.n_sub), "dim_coarse": int(orc.dim_H),
        "pcg_tol": 1e-8, "pcg_iterations": int(it), "pcg_iterations_recursive": first,
        "kappa_estimate": float(kappa), "true_residual": res,
        "x_norm": float(np.linalg.norm(x)),
        "ref_tol": 1e-12, "ref_iterations": int(its), "ref_true_residual": res_s,
        "ref_x_norm": float(np.linalg.norm(xs)),
        "sample_index": idx.tolist(),
        "x_sample": [float(v) for v in x[idx]],
        "ref_x_sample": [float(v) for v in xs[idx]],
        "m": [int(orc.ms[j]) for j in range(prob.n_sub)],
        "lambda": [[float(v) for v in orc.lams[j][:nev + 1]] for j in range(prob.n_sub)],
        "seconds": time.time() - t0,
    }
    with open(OUT, "w") as f:
        json.dump(out, f, separators=(",", ":"))
    print("wrote %s (%.0f s)" % (OUT, time.time() - t0))


if __name__ == "__main__":
    main()
