"""Shared helpers for the GPU parity tests (compare the CUDA library with the oracle)."""
import numpy as np
import scipy.sparse.linalg as spla

import oracle


def run_gpu(prob, pu_weights=None, **opts):
    """Set up the GPU preconditioner for prob and return (wrapper, torch)."""
    import torch
    from paper_1906_10944_gb300 import geneo as G
    return G.GenEO(prob, pu_weights=pu_weights, **opts), torch


def gpu_solve(sol, prob, tol=1e-8, maxit=2000):
    import torch
    b = torch.from_numpy(prob.b).cuda()
    x = torch.zeros_like(b)
    info = sol.solve(b, x, tol=tol, maxit=maxit, hist_cap=maxit + 1)
    return x.cpu().numpy(), info


def lam_close(lg, lo, tau):
    """|lambda - lambda*| <= 1e-6 max(|lambda*|, 1e-3 tau) elementwise."""
    return np.abs(lg - lo) <= 1e-6 * np.maximum(np.abs(lo), 1e-3 * tau)


def check_selection(lg_all, lo_all, m_gpu, m_or, tau, nev):
    """m_j must agree unless an eigenvalue sits within 1e-6 tau of tau
    (a tie at the threshold: either choice is correct)."""
    if m_gpu == m_or:
        return True
    lo = lo_all[:nev + 1]
    return bool(np.any(np.abs(lo - tau) <= 1e-6 * tau))


def principal_angle(Zg, Zo, lam, m):
    """Largest principal angle (radians) between the spans of the first m'
    columns of Zg and Zo, m' <= m the largest count whose next eigenvalue is
    separated by a relative gap above 1e-2 (a cluster split at m' leaves its
    subspace undetermined); 0 when there is no such m'."""
    mm = 0
    for k in range(m, 0, -1):
        nxt = lam[k] if k < lam.size else np.inf
        if (nxt - lam[k - 1]) > 1e-2 * max(abs(nxt), 1e-3):
            mm = k
            break
    if mm == 0:
        return 0.0
    qg, _ = np.linalg.qr(Zg[:, :mm])
    qo, _ = np.linalg.qr(Zo[:, :mm])
    s = np.linalg.svd(qo.T @ qg, compute_uv=False)
    return float(np.arccos(np.clip(s.min(), -1.0, 1.0)))


def compare_setup(prob, sol, orc, tau, nev, fixed=False, stats=None):
    """Per-subdomain parity of D_j, X_j, selected eigenvalues and coarse
    vectors; stats (a dict) receives the largest relative eigenvalue error
    and the largest principal angle between the coarse spaces."""
    worst_lam = 0.0
    worst_angle = 0.0
    for j in range(prob.n_sub):
        g = sol.subdomain(j)
        s = orc.sets[j]
        assert np.array_equal(g["D"], s["D"].astype(np.int32)), j
        assert np.array_equal(g["pu"], orc.xs[j]), j
        lo = orc.lams[j]
        m_or = orc.ms[j]
        assert check_selection(g["lambda"], lo, g["m"], m_or, tau, nev), (j, g["lambda"][:nev + 1], lo[:nev + 1])
        m = min(g["m"], m_or)
        if m:
            ok = lam_close(g["lambda"][:m], lo[:m], tau)
            assert np.all(ok), (j, g["lambda"][:m], lo[:m])
            worst_lam = max(worst_lam, float(np.max(np.abs(g["lambda"][:m] - lo[:m]) /
                                                     np.maximum(np.abs(lo[:m]), 1e-3 * tau))))
            # coarse vectors: compare where the eigenvalue is well separated
            Zo = orc.Zloc[j][s["dpos"], :]
            ang = principal_angle(g["Z"], Zo, lo, m)
            assert ang <= 1e-4, (j, ang)
            worst_angle = max(worst_angle, ang)
            for k in range(m):
                gap = np.min(np.abs(np.delete(lo[:nev + 5], k) - lo[k])) / max(abs(lo[k]), 1e-3)
                zg = g["Z"][:, k]
                # sign rule of the library: entry of largest magnitude positive
                assert zg[np.argmax(np.abs(zg))] > 0 or np.sort(np.abs(zg))[-2] >= (1 - 1e-9) * np.abs(zg).max()
                assert abs(np.linalg.norm(zg) - 1.0) < 1e-12
                if gap > 1e-2:
                    # up to sign: when the two largest entries tie to rounding the
                    # rule may pick either
                    err = min(np.linalg.norm(zg - Zo[:, k]), np.linalg.norm(zg + Zo[:, k]))
                    assert err < 1e-4, (j, k, err, gap)
    if stats is not None:
        stats["eig_rel_err"] = worst_lam
        stats["coarse_angle"] = worst_angle
    return worst_lam


def oracle_reference_solution(prob):
    return spla.spsolve(prob.A.tocsc(), prob.b)
