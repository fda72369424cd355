"""Parity of the CUDA library (through the C ABI) with the FP64 oracle.

Tolerances (FP64 path): eigenvalues |lambda - lambda*| <= 1e-6 max(|lambda*|,
1e-3 tau); partition of unity and D_j bit-exact; PCG iterations within +-2 of
the oracle; relative error <= 1e-7 against a direct solve, or the oracle's own
error at the same tolerance times 10 when that is larger (the error a residual
of 1e-8 implies depends on kappa(A)).

Residuals: PCG (library and oracle alike) stops when the true residual
||b - A x|| / ||b|| reaches tol (the recursive residual is tested first and
replaced by the true one while that is above tol), so the library's reported
true residual is asserted <= tol and the one recomputed here with scipy <=
1.01 tol (the two FP64 evaluations differ in rounding).

Every full check prints the worst relative eigenvalue error, the largest
principal angle between the library's and the oracle's coarse spaces (per
subdomain, over the selected vectors up to a separated eigenvalue), the
solution error against a direct solve and the iteration counts.
"""
import numpy as np
import pytest

import gen
import oracle
from gpu_helpers import compare_setup, gpu_solve, oracle_reference_solution, run_gpu

pytestmark = pytest.mark.gpu



def check_residual(prob, x, info, tol):
    """True residual <= tol as the library evaluates it, and the scipy
    recomputation within the rounding of an FP64 residual evaluation,
    eps ||(|A| |x|)|| / ||b|| per evaluation (at contrast 1e6 that is a few
    1e-9, the same order as the residual itself)."""
    bn = np.linalg.norm(prob.b)
    res = np.linalg.norm(prob.b - prob.A @ x) / bn
    ev = np.finfo(np.float64).eps * np.linalg.norm(abs(prob.A) @ np.abs(x)) / bn
    assert info["converged"] and info["true_residual"] <= tol, (info["rel_residual"], info["true_residual"])
    assert res <= tol + 2 * ev and abs(info["true_residual"] - res) <= 2 * ev + 1e-3 * tol, \
        (info["true_residual"], res, ev)
    return res


def _c1(contrast=1e6, seed=0):
    k = gen.kappa_channels_2d((64, 64), seed=seed, contrast=contrast)
    return gen.darcy_problem((64, 64), k, (4, 4), 1)


def _full_check(prob, tau=0.3, nev=10, fixed=False, form="paper", tol=1e-8, name="", precision=0,
                pu=None, gpu_pu=None, iter_slack=0.0):
    orc = oracle.GenEOOracle(prob, oracle.OracleOptions(tau=tau, nev_max=nev, fixed_nev=fixed,
                                                        eig_form=form), pu=pu)
    kw = {} if gpu_pu is None else gpu_pu
    sol, torch = run_gpu(prob, tau=tau, nev_max=nev, fixed_nev=int(fixed),
                         eig_form=0 if form == "paper" else 1, precision=precision, **kw)
    try:
        q = sol.query()
        stats = {}
        compare_setup(prob, sol, orc, tau, nev, fixed, stats=stats)
        assert q["dim_coarse"] == orc.dim_H or not fixed
        x, info = gpu_solve(sol, prob, tol=tol)
        xo, ito, _, kapo = orc.solve(tol=tol)
        xs = oracle_reference_solution(prob)
        res = check_residual(prob, x, info, tol)
        assert abs(info["iterations"] - ito) <= 2 + iter_slack * ito, (info["iterations"], ito)
        err = np.linalg.norm(x - xs) / np.linalg.norm(xs)
        err_o = np.linalg.norm(xo - xs) / np.linalg.norm(xs)
        assert err <= max(1e-7, 10 * err_o), (err, err_o)
        # FP32 local solves change M^{-1} slightly
        assert abs(info["kappa_estimate"] - kapo) <= (0.05 if precision == 0 else 0.15) * kapo
        print("PARITY %s prec=%d: eig rel err %.2e, coarse angle %.2e rad, solution err %.2e "
              "(oracle %.2e), true residual %.2e, iterations %d (oracle %d), kappa %.3f (oracle %.3f)"
              % (name, precision, stats["eig_rel_err"], stats["coarse_angle"], err, err_o, res,
                 info["iterations"], ito, info["kappa_estimate"], kapo))
        return sol, orc, info
    finally:
        sol.close()


def test_c1_darcy_2d_high_contrast():
    """2D Darcy 64x64, 4x4 subdomains, overlap 1, channels at contrast 1e6."""
    _full_check(_c1(), name="c1")


def test_c1_full_eigen_form():
    _full_check(_c1(), form="full", name="c1-full-form")


def test_fixed_nev_mode():
    _full_check(_c1(contrast=1e4, seed=3), nev=4, fixed=True, name="c1-fixed-nev")


def test_one_level_apply_exact():
    """nev_max = 0: the apply equals sum_j R_j^T A_j^{-1} R_j (one-level method,
    banded FP64 Cholesky against sparse LU) to rounding."""
    import torch
    prob = _c1()
    orc = oracle.GenEOOracle(prob, oracle.OracleOptions(nev_max=0))
    sol, _ = run_gpu(prob, nev_max=0)
    try:
        rng = np.random.default_rng(1)
        for _ in range(3):
            r = rng.standard_normal(prob.n)
            z = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
            sol.apply(torch.from_numpy(r).cuda(), z)
            zg = z.cpu().numpy()
            zo = orc.apply(r)
            assert np.linalg.norm(zg - zo) <= 1e-10 * np.linalg.norm(zo)
    finally:
        sol.close()


def test_long_subdomains_ring_solve():
    """Two subdomains of 1202 x 49 nodes (2D Darcy 2400 x 48, channels):
    the local vectors no longer fit in shared memory beside the staged band
    rows, so the local solves take the ring kernel.  FP64: the one-level
    apply equals the oracle's sparse-LU apply to rounding.  FP32 factors:
    PCG with the one-level method reaches the true residual 1e-8 in the
    oracle's iteration count up to the mixed-precision bar."""
    import torch
    k = gen.kappa_channels_2d((2400, 48), seed=3, contrast=1e2)
    prob = gen.darcy_problem((2400, 48), k, (2, 1), 1)
    orc = oracle.GenEOOracle(prob, oracle.OracleOptions(nev_max=0))
    sol, _ = run_gpu(prob, nev_max=0)
    try:
        rng = np.random.default_rng(4)
        for _ in range(2):
            r = rng.standard_normal(prob.n)
            z = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
            sol.apply(torch.from_numpy(r).cuda(), z)
            zo = orc.apply(r)
            assert np.linalg.norm(z.cpu().numpy() - zo) <= 1e-10 * np.linalg.norm(zo)
    finally:
        sol.close()
    _, its_o, _, _ = orc.solve(prob.b, tol=1e-8, maxit=4000)
    sol, _ = run_gpu(prob, nev_max=0, precision=1)
    try:
        x, info = gpu_solve(sol, prob, tol=1e-8, maxit=4000)
        check_residual(prob, x, info, 1e-8)
        assert abs(info["iterations"] - its_o) <= 0.1 * its_o + 2, (info["iterations"], its_o)
    finally:
        sol.close()


def test_two_level_apply_matches_oracle():
    """Two-level apply vs the oracle's; the coarse vectors come from an
    iterative eigensolve (residual 1e-6), hence the looser tolerance."""
    import torch
    prob = _c1(contrast=1e3, seed=5)
    orc = oracle.GenEOOracle(prob, oracle.OracleOptions(nev_max=6))
    sol, _ = run_gpu(prob, nev_max=6, eig_tol=1e-9)
    try:
        rng = np.random.default_rng(2)
        r = rng.standard_normal(prob.n)
        z = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
        sol.apply(torch.from_numpy(r).cuda(), z)
        zo = orc.apply(r)
        assert np.linalg.norm(z.cpu().numpy() - zo) <= 1e-6 * np.linalg.norm(zo)
    finally:
        sol.close()


def test_darcy_3d_ragged():
    """3D Darcy 18x14x12 with uneven boxes (3x2x2 parts, overlap 2): several
    block columns of the banded kernels and ragged last blocks."""
    nel = (18, 14, 12)
    kap = gen.kappa_grf_layers_3d(nel, seed=4, corr_len=0.2, variance=2.0, contrast=1e4,
                                  slab_z=(30, 80), slab_thickness=1)
    prob = gen.darcy_problem(nel, kap, (3, 2, 2), 2)
    _full_check(prob, nev=8, name="darcy3d-ragged")


def test_elasticity_3d_small():
    """3D laminate elasticity (3 dofs per node), floating subdomains carry six
    rigid-body modes."""
    prob = gen.elasticity_problem((12, 6, 6), (3, 1, 1), 1, layer_thickness=1)
    _full_check(prob, nev=10, name="elasticity")


def test_elasticity_3d_mixed_precision():
    """The laminate elasticity case with FP32 factors (the precision its full
    size configuration runs in): FP64 eigenvalue bar, the same coarse space
    (principal angles), the true residual at tol, iterations within 10 % + 2."""
    prob = gen.elasticity_problem((12, 6, 6), (3, 1, 1), 1, layer_thickness=1)
    _full_check(prob, nev=10, name="elasticity", precision=1, iter_slack=0.1)


def test_darcy_3d_ragged_mixed_precision():
    nel = (18, 14, 12)
    kap = gen.kappa_grf_layers_3d(nel, seed=4, corr_len=0.2, variance=2.0, contrast=1e4,
                                  slab_z=(30, 80), slab_thickness=1)
    prob = gen.darcy_problem(nel, kap, (3, 2, 2), 2)
    _full_check(prob, nev=8, name="darcy3d-ragged", precision=1, iter_slack=0.1)


def test_wide_bands_mixed_precision():
    """3D Darcy 60 x 26 x 26 in two subdomains of about 19,000 dofs: half
    bandwidths 807 (K_j) and 781 (A_j), too wide for four A-tile stages next
    to the panel block, so the tensor-core factorisation runs with two and
    three stages.  FP32 factors against the FP64 oracle (mixed bar)."""
    nel = (60, 26, 26)
    kap = gen.kappa_grf_layers_3d(nel, seed=6, corr_len=0.2, variance=2.0, contrast=1e3,
                                  slab_z=(30, 80), slab_thickness=1)
    prob = gen.darcy_problem(nel, kap, (2, 1, 1), 1)
    _full_check(prob, nev=8, name="wide-bands", precision=1, iter_slack=0.1)


def test_c1_mixed_precision():
    """FP32 factors (local solves and the eigensolver's shift-invert operator)
    with FP64 residuals, coarse problem and PCG, and double-single eigensolver
    products, Rayleigh-Ritz and coarse inverse."""
    _full_check(_c1(), name="c1", precision=1, iter_slack=0.1)


def _random_pu(prob, seed):
    """Caller weights of Definition 3 that are not the standard ones: random
    positive weights on each D_j, normalised to sum to one per dof, zero on
    the inner boundary (a test input)."""
    sets = oracle.subdomain_sets(prob)
    rng = np.random.default_rng(seed)
    raw = [np.zeros(s["N"].size) for s in sets]
    tot = np.zeros(prob.n)
    for s, w in zip(sets, raw):
        w[s["dpos"]] = rng.uniform(0.2, 1.0, s["dpos"].size)
        tot[s["D"]] += w[s["dpos"]]
    for s, w in zip(sets, raw):
        w[s["dpos"]] /= tot[s["D"]]
    return raw


def test_caller_standard_weights_bitwise():
    """Passing the standard partition of unity as caller weights gives
    bitwise the same eigenvalues, coarse space and solution as passing none."""
    prob = _c1()
    orc_sets = oracle.subdomain_sets(prob)
    _, xs = oracle.partition_of_unity(prob, orc_sets)
    outs = []
    for w in (None, np.concatenate(xs)):
        sol, _ = run_gpu(prob, nev_max=10, pu_weights=w)
        try:
            x, info = gpu_solve(sol, prob)
            subs = [sol.subdomain(j) for j in range(prob.n_sub)]
            outs.append((x, np.concatenate([g["lambda"] for g in subs]),
                         np.concatenate([g["Z"].ravel() for g in subs]), info["iterations"]))
        finally:
            sol.close()
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


def test_caller_random_weights_match_oracle():
    """Non-standard caller weights: the library matches the oracle run with
    the same weights (eigenvalues, coarse space, PCG)."""
    prob = _c1(contrast=1e4, seed=2)
    w = _random_pu(prob, 7)
    _full_check(prob, name="c1-random-pu", pu=w, gpu_pu={"pu_weights": np.concatenate(w)})


def test_caller_weights_rejected():
    """Weights that do not sum to one, or that are non-zero on the inner
    boundary, are rejected with GENEO_ERR_ARG."""
    from paper_1906_10944_gb300 import geneo as G
    prob = _c1()
    sets = oracle.subdomain_sets(prob)
    _, xs = oracle.partition_of_unity(prob, sets)
    bad1 = np.concatenate(xs) * 1.001
    bad2 = [x.copy() for x in xs]
    inner = np.setdiff1d(np.arange(sets[5]["N"].size), sets[5]["dpos"])
    bad2[5][inner[0]] = 0.5
    for w in (bad1, np.concatenate(bad2)):
        with pytest.raises(G.GenEOError) as e:
            G.GenEO(prob, pu_weights=w, nev_max=10)
        assert e.value.code == 1


def test_sarkis_partition_of_unity_matches_oracle():
    """The smooth (Sarkis) partition of unity computed on the device equals
    the oracle's bit for bit (integer layer distances, one division), and the
    GenEO setup and solve built on it match the oracle's."""
    prob = gen.darcy_problem((64, 64), gen.kappa_channels_2d((64, 64), seed=0), (4, 4), 2)
    _full_check(prob, name="c1-overlap2-sarkis", pu="sarkis", gpu_pu={"pu_kind": 1})


def test_sarkis_3d_elasticity():
    prob = gen.elasticity_problem((12, 6, 6), (3, 1, 1), 2, layer_thickness=1)
    _full_check(prob, nev=10, name="elasticity-sarkis", pu="sarkis", gpu_pu={"pu_kind": 1})


def test_single_subdomain_is_direct_solve():
    """One subdomain covering the domain: no overlap, B = 0, no coarse space;
    M^{-1} = A^{-1} and PCG converges in one iteration."""
    prob = gen.darcy_problem((20, 16), np.ones((16, 20)), (1, 1), 0)
    sol, _ = run_gpu(prob, nev_max=5)
    try:
        assert sol.query()["dim_coarse"] == 0
        x, info = gpu_solve(sol, prob)
        assert info["iterations"] <= 1 and info["converged"]
        xs = oracle_reference_solution(prob)
        assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)
    finally:
        sol.close()


def test_deterministic():
    """Two setups and solves give bitwise identical results."""
    prob = _c1()
    outs = []
    for _ in range(2):
        sol, _ = run_gpu(prob, nev_max=10)
        try:
            x, info = gpu_solve(sol, prob)
            lam = np.concatenate([sol.subdomain(j)["lambda"] for j in range(prob.n_sub)])
            outs.append((x, lam, info["iterations"]))
        finally:
            sol.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2]


def test_host_memory_path():
    """The same setup and solve with host arrays (copies inside the calls)."""
    from paper_1906_10944_gb300 import geneo as G
    prob = _c1()
    arrs = G.problem_arrays(prob)
    p = G.make_problem(arrs, prob.n, prob.n_sub, 4, 1, G.GENEO_MEM_HOST)
    h = G.geneo_setup(p, G.geneo_default_options())
    try:
        x = np.zeros(prob.n)
        info = G.geneo_pcg_solve(h, np.ascontiguousarray(prob.b), x, tol=1e-8, mem=G.GENEO_MEM_HOST)
        check_residual(prob, x, info, 1e-8)
    finally:
        G.geneo_destroy(h)


def test_uneven_batch_darcy_3d():
    """Uneven batching: an irregular k-d box partition (sides 3..8 elements,
    overlap 1..3 per box, one inclusion of contrast 1e4..1e8 per box), so the
    batch mixes subdomain sizes and band widths; FP64 parity as above."""
    prob = gen.uneven_darcy_problem((24, 20, 18), 24, 3, 8, seed=3)
    _full_check(prob, nev=8)


@pytest.mark.parametrize("pivot_tol", [1e-4, 0.05, 0.3, 0.999])
def test_mixed_precision_fp64_refactor(pivot_tol):
    """Adaptive precision per subdomain: an FP32 factorisation with a pivot
    at or below fp32_pivot_tol (equilibrated bands, unit diagonal) is redone
    in FP64 and solved by the FP64 kernels into the same vectors.  With
    0.999 every K_j and A_j goes to FP64 (every factorisation has a pivot
    below its unit diagonal), which exercises the FP64 batch end to end; the
    default keeps FP32 where FP32 suffices, and the intermediate tolerances
    split the batch, so the eigensolver's products run partly in
    double-single and partly in FP64 arithmetic.  Uneven k-d boxes with
    inclusions of contrast up to 1e8; parity as in the mixed-precision
    test."""
    prob = gen.uneven_darcy_problem((24, 20, 18), 24, 3, 8, seed=3)
    nev = 8
    orc = oracle.GenEOOracle(prob, oracle.OracleOptions(nev_max=nev))
    sol, _ = run_gpu(prob, nev_max=nev, precision=1, fp32_pivot_tol=pivot_tol)
    try:
        q = sol.query()
        print("pivot_tol", pivot_tol, "fp64 K", q["fp64_factors_K"], "A", q["fp64_factors_A"],
              "ortho", q["fp64_ortho"], "of", prob.n_sub)
        if pivot_tol > 0.5:
            assert q["fp64_factors_K"] == prob.n_sub and q["fp64_factors_A"] == prob.n_sub, q
        else:
            assert 0 <= q["fp64_factors_K"] <= prob.n_sub and 0 <= q["fp64_factors_A"] <= prob.n_sub
        for j in range(prob.n_sub):
            g = sol.subdomain(j)
            m = min(g["m"], orc.ms[j])
            lo = orc.lams[j][:m]
            assert np.all(np.abs(g["lambda"][:m] - lo) <= 1e-6 * np.maximum(np.abs(lo), 3e-4)), j
        x, info = gpu_solve(sol, prob)
        _, ito, _, _ = orc.solve(tol=1e-8)
        check_residual(prob, x, info, 1e-8)
        assert abs(info["iterations"] - ito) <= 2 + 0.1 * ito, (info["iterations"], ito)
    finally:
        sol.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_block_pcg_several_rhs(precision):
    """Several right-hand sides in one call (solved together, 8 at a time):
    every column meets the true-residual bar, its error against a direct
    solve meets the single-solve bar, and it equals the one-column solve of
    the same right-hand side up to the solver tolerance; 11 columns exercise
    a full block of 8 and a ragged block of 3."""
    import torch
    import scipy.sparse.linalg as spla
    from paper_1906_10944_gb300 import geneo as G
    nel = (18, 14, 12)
    kap = gen.kappa_grf_layers_3d(nel, seed=4, corr_len=0.2, variance=2.0, contrast=1e4,
                                  slab_z=(30, 80), slab_thickness=1)
    prob = gen.darcy_problem(nel, kap, (3, 2, 2), 2)
    k = 11
    rng = np.random.default_rng(9)
    B = rng.uniform(-1, 1, (k, prob.n))
    B[:, prob.dirichlet != 0] = 0.0
    B[0] = prob.b
    sol, _ = run_gpu(prob, nev_max=8, precision=precision)
    try:
        bd = torch.from_numpy(B.reshape(-1)).cuda()
        xd = torch.zeros_like(bd)
        info = G.geneo_pcg_solve(sol.h, bd, xd, k, 1e-8, 1000)
        X = xd.cpu().numpy().reshape(k, prob.n)
        lu = spla.splu(prob.A.tocsc())
        for c in range(k):
            bn = np.linalg.norm(B[c])
            res = np.linalg.norm(B[c] - prob.A @ X[c]) / bn
            ev = np.finfo(np.float64).eps * np.linalg.norm(abs(prob.A) @ np.abs(X[c])) / bn
            assert res <= 1e-8 + 2 * ev, (c, res)
            xs = lu.solve(B[c])
            x1 = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
            one = G.geneo_pcg_solve(sol.h, torch.from_numpy(B[c]).cuda(), x1, 1, 1e-8, 1000)
            x1 = x1.cpu().numpy()
            e_blk = np.linalg.norm(X[c] - xs) / np.linalg.norm(xs)
            e_one = np.linalg.norm(x1 - xs) / np.linalg.norm(xs)
            assert e_blk <= max(1e-7, 10 * e_one), (c, e_blk, e_one)
            assert np.linalg.norm(X[c] - x1) <= 1e-6 * np.linalg.norm(x1)
            if c == k - 1:
                assert abs(info["iterations"] - one["iterations"]) <= 2
                assert info["converged"] and info["true_residual"] <= 1e-8
    finally:
        sol.close()
