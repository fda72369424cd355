"""Parity at the benchmark's full size (3D Darcy 128^3, 512 subdomains), in
the launch configuration bench.py times (mixed path, FP32 factors) and on the
FP64 path, against the oracle's own run of the same workload stored by
tests/golden/make_darcy3d_128.py (every subdomain's selected count and
eigenvalues, the PCG iteration count, the solution at 4096 sampled dofs and a
reference solution at tol 1e-12), plus four sampled subdomains whose coarse
vectors the oracle computes here (ARPACK shift-invert, Section 4.4) for the
principal angles between the coarse spaces.

Bars: eigenvalues |lambda - lambda*| <= 1e-6 max(|lambda*|, 1e-3 tau) on all
512 subdomains, m_j equal unless an eigenvalue sits within 1e-6 tau of tau;
principal angles <= 1e-4 rad; PCG iterations within +-2 of the oracle's
(FP64) or 10 % + 2 (FP32 factors); true residual <= 1e-8; sampled solution
error against the reference <= max(1e-7, 10 x the oracle's own)."""
import json
import os

import numpy as np
import pytest

import gen
import oracle
from gpu_helpers import principal_angle

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "darcy3d_128_oracle.json")


@pytest.fixture(scope="module")
def c2():
    kap = gen.kappa_grf_layers_3d((128, 128, 128), seed=1)
    return gen.darcy_problem((128, 128, 128), kap, (8, 8, 8), 2)


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.mark.parametrize("precision", [1, 0])
def test_darcy_128_parity(c2, golden, precision):
    import torch
    from paper_1906_10944_gb300 import geneo as G
    prob = c2
    tau, nev = 0.3, 20
    assert golden["n"] == prob.n and golden["n_sub"] == prob.n_sub
    sol = G.GenEO(prob, nev_max=nev, tau=tau, precision=precision)
    try:
        # properties over all subdomains, and every subdomain's eigenvalues
        s = np.zeros(prob.n)
        worst = 0.0
        for j in range(prob.n_sub):
            g = sol.subdomain(j)
            N = prob.sub_dofs(j)
            s[N] += g["pu"]
            if g["m"]:
                assert np.allclose(np.linalg.norm(g["Z"], axis=0), 1.0, atol=1e-12)
            lo = np.asarray(golden["lambda"][j])
            m_or = golden["m"][j]
            assert g["m"] == m_or or np.any(np.abs(lo - tau) <= 1e-6 * tau), (j, g["m"], m_or)
            m = min(g["m"], m_or)
            bar = np.maximum(np.abs(lo[:m]), 1e-3 * tau)
            err = np.abs(g["lambda"][:m] - lo[:m]) / bar
            assert np.all(err <= 1e-6), (j, g["lambda"][:m], lo[:m])
            worst = max(worst, float(err.max()) if m else 0.0)
        free = prob.dirichlet == 0
        assert np.abs(s[free] - 1.0).max() < 1e-12 and np.all(s[~free] == 0.0)
        # coarse spaces of sampled subdomains: interior, face, edge, corner
        sets = oracle.subdomain_sets(prob)
        e_tau = oracle.element_multiplicity(prob)
        _, xs = oracle.partition_of_unity(prob, sets)
        angle = 0.0
        for j in (0, 7, 73, 273):
            g = sol.subdomain(j)
            assert np.array_equal(g["D"], sets[j]["D"].astype(np.int32))
            At, B = oracle.geneo_pencil(prob, j, sets, xs, e_tau)
            lo, P = oracle.local_eigenpairs(At, B, nev + min(10, nev), -0.01, 0)
            m = min(g["m"], oracle.select_count(lo, tau, nev))
            Zo = oracle.coarse_vectors(P, xs[j], m)[sets[j]["dpos"], :]
            a = principal_angle(g["Z"], Zo, lo, m)
            assert a <= 1e-4, (j, a)
            angle = max(angle, a)
        # the solve against the oracle's
        b = torch.from_numpy(prob.b).cuda()
        x = torch.zeros_like(b)
        info = sol.solve(b, x, tol=1e-8, maxit=2000)
        xr = x.cpu().numpy()
        bn = np.linalg.norm(prob.b)
        res = np.linalg.norm(prob.b - prob.A @ xr) / bn
        ev = np.finfo(np.float64).eps * np.linalg.norm(abs(prob.A) @ np.abs(xr)) / bn
        assert info["converged"] and info["true_residual"] <= 1e-8 and res <= 1e-8 + 2 * ev, \
            (info["rel_residual"], info["true_residual"], res, ev)
        ito = golden["pcg_iterations"]
        slack = 2 if precision == 0 else 2 + 0.1 * ito
        assert abs(info["iterations"] - ito) <= slack, (info["iterations"], ito)
        idx = np.asarray(golden["sample_index"])
        xref = np.asarray(golden["ref_x_sample"])
        err = np.linalg.norm(xr[idx] - xref) / np.linalg.norm(xref)
        err_o = np.linalg.norm(np.asarray(golden["x_sample"]) - xref) / np.linalg.norm(xref)
        assert err <= max(1e-7, 10 * err_o), (err, err_o)
        print("PARITY darcy3d-128 prec=%d: eig rel err %.2e (all 512 subdomains), coarse angle %.2e "
              "rad (4 sampled), sampled solution err %.2e (oracle %.2e), true residual %.2e, "
              "iterations %d (oracle %d), kappa %.3f (oracle %.3f)"
              % (precision, worst, angle, err, err_o, res, info["iterations"], ito,
                 info["kappa_estimate"], golden["kappa_estimate"]))
    finally:
        sol.close()
