"""Failure paths of the C ABI, each made on the host (bad data, a small
iteration cap): the kernels record the first error in the device status word
and finish; no test faults, traps or hangs the GPU.

  - a NaN in one element matrix          -> GENEO_ERR_NONFINITE (subdomain, element)
  - a negated, scaled element matrix     -> GENEO_ERR_NOT_SPD (subdomain, pivot row)
  - maxit = 2                            -> GENEO_ERR_PCG_NOCONV, 2 iterations
  - eig_maxit = 1 with eig_strict = 1    -> GENEO_ERR_EIG_NOCONV; without: a count
  - nev_max above a subdomain's size     -> the block is clipped, parity holds
"""
import copy

import numpy as np
import pytest

import gen
import oracle
from gpu_helpers import gpu_solve, run_gpu

pytestmark = pytest.mark.gpu

NONFINITE, NOT_SPD, EIG_NOCONV, PCG_NOCONV = 9, 3, 4, 5


def _c1():
    k = gen.kappa_channels_2d((64, 64), seed=0)
    return gen.darcy_problem((64, 64), k, (4, 4), 1)


def _elem_of_sub(prob, j):
    """An element of subdomain j that lies in no other subdomain."""
    counts = np.bincount(prob.sub_elem, minlength=prob.n_elem)
    el = prob.sub_elems(j)
    return int(el[counts[el] == 1][len(el[counts[el] == 1]) // 2])


def test_nan_coefficient_is_nonfinite():
    from paper_1906_10944_gb300 import geneo as G
    prob = copy.copy(_c1())
    e = _elem_of_sub(prob, 5)
    prob.elem_mats = prob.elem_mats.copy()
    prob.elem_mats[e, 1, 2] = np.nan
    with pytest.raises(G.GenEOError) as ex:
        G.GenEO(prob, nev_max=10)
    assert ex.value.code == NONFINITE
    code, where, index = G.geneo_last_error(None)
    assert (code, where, index) == (NONFINITE, 5, e)


def test_negated_element_is_not_spd():
    from paper_1906_10944_gb300 import geneo as G
    prob = copy.copy(_c1())
    e = _elem_of_sub(prob, 6)
    prob.elem_mats = prob.elem_mats.copy()
    prob.elem_mats[e] *= -100.0
    with pytest.raises(G.GenEOError) as ex:
        G.GenEO(prob, nev_max=10)
    assert ex.value.code == NOT_SPD
    code, where, index = G.geneo_last_error(None)
    assert code == NOT_SPD and where == 6 and 0 <= index < prob.sub_dofs(6).size


def test_pcg_iteration_cap():
    from paper_1906_10944_gb300 import geneo as G
    prob = _c1()
    sol, torch = run_gpu(prob, nev_max=10)
    try:
        b = torch.from_numpy(prob.b).cuda()
        x = torch.zeros_like(b)
        out = G.geneo_pcg_solve(sol.h, b, x, 1, 1e-8, 2, raise_on_error=False)
        assert out["status"] == PCG_NOCONV and out["iterations"] == 2 and not out["converged"]
        assert out["true_residual"] > 1e-8
        # the handle stays usable
        x2, info = gpu_solve(sol, prob)
        assert info["converged"]
    finally:
        sol.close()


def test_eigensolver_cap():
    from paper_1906_10944_gb300 import geneo as G
    prob = _c1()
    with pytest.raises(G.GenEOError) as ex:
        G.GenEO(prob, nev_max=10, eig_maxit=1, eig_strict=1)
    assert ex.value.code == EIG_NOCONV
    sol, _ = run_gpu(prob, nev_max=10, eig_maxit=1)
    try:
        q = sol.query()
        assert 0 < q["eig_unconverged"] <= prob.n_sub
        x, info = gpu_solve(sol, prob)   # a weaker coarse space still solves
        assert info["converged"]
    finally:
        sol.close()
    sol, _ = run_gpu(prob, nev_max=10)
    try:
        assert sol.query()["eig_unconverged"] == 0
    finally:
        sol.close()


def test_nev_above_subdomain_size():
    """8 x 8 elements on 4 x 4 subdomains with one layer of overlap: corner
    subdomains hold 9 free dofs, fewer than nev_max = 30; the eigensolver
    block is clipped to the subdomain and the results match the oracle."""
    prob = gen.darcy_problem((8, 8), gen.kappa_channels_2d((8, 8), seed=1, n_channels=1, n_incl=2),
                             (4, 4), 1)
    orc = oracle.GenEOOracle(prob, oracle.OracleOptions(nev_max=30))
    sol, _ = run_gpu(prob, nev_max=30)
    try:
        for j in range(prob.n_sub):
            g = sol.subdomain(j)
            assert g["m"] == orc.ms[j], (j, g["m"], orc.ms[j])
            m = g["m"]
            lo = orc.lams[j][:m]
            assert np.all(np.abs(g["lambda"][:m] - lo) <= 1e-6 * np.maximum(np.abs(lo), 3e-4))
        x, info = gpu_solve(sol, prob)
        _, ito, _, _ = orc.solve(tol=1e-8)
        assert info["converged"] and abs(info["iterations"] - ito) <= 2
    finally:
        sol.close()


def test_deterministic_off_matches():
    """options.deterministic = 0 (atomic inner products in PCG) converges to
    the same solution as the fixed-order mode within rounding."""
    prob = _c1()
    xs = []
    for det in (1, 0):
        sol, _ = run_gpu(prob, nev_max=10, deterministic=det)
        try:
            x, info = gpu_solve(sol, prob)
            assert info["converged"] and info["true_residual"] <= 1e-8
            xs.append((x, info["iterations"]))
        finally:
            sol.close()
    assert abs(xs[0][1] - xs[1][1]) <= 1
    assert np.linalg.norm(xs[0][0] - xs[1][0]) <= 1e-6 * np.linalg.norm(xs[0][0])
