"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these tests retypes the oracle's formulas: each compares the oracle
with an independent construction (pointwise finite-element quadrature and box
geometry), a closed form, a brute-force dense computation, an exact special
case, or a qualitative invariant the paper reports (Section 5.2, Table 1).
"""
import itertools

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import gen
import oracle


# ----------------------------------------------------------------------------
# Independent brute-force finite-element construction (2D, boxes).
# ----------------------------------------------------------------------------
def _hat(t):
    return np.maximum(0.0, 1.0 - np.abs(t))


def _dhat(t):
    return np.where(np.abs(t) < 1.0, -np.sign(t), 0.0)


def _brute_pencil(prob, j):
    """Atilde_j, A_j^o and X_j built from their continuous definitions:
    integrals of kappa grad(phi_a).grad(phi_b) over Omega_j and over the
    overlap zone, evaluated pointwise with a 3x3 Gauss rule per element, with
    Omega_j, the overlap zone and D_j taken from box geometry."""
    nx, ny = prob.nel
    h = prob.h
    boxes = prob.boxes_grown
    kap = prob.coeff.reshape(ny, nx)
    g1 = np.array([0.5 - np.sqrt(0.15), 0.5, 0.5 + np.sqrt(0.15)])
    w1 = np.array([5.0, 8.0, 5.0]) / 18.0

    def in_box(bx, x, y):  # open box test (quadrature points are interior)
        (x0, y0), (x1, y1) = bx
        return x0 * h < x < x1 * h and y0 * h < y < y1 * h

    def node_in_D(bx, i, k):
        (x0, y0), (x1, y1) = bx
        okx = (x0 < i < x1) or (i == 0 and x0 == 0) or (i == nx and x1 == nx)
        oky = (y0 < k < y1) or (k == 0 and y0 == 0) or (k == ny and y1 == ny)
        return okx and oky

    (x0, y0), (x1, y1) = boxes[j]
    nodes = [(i, k) for k in range(y0, y1 + 1) for i in range(x0, x1 + 1)]
    dofs = [i + (nx + 1) * k for i, k in nodes]
    keep = [q for q, d in enumerate(dofs) if prob.dirichlet[d] == 0]
    nodes = [nodes[q] for q in keep]
    m = len(nodes)
    mult = {}
    for jj, bx in enumerate(boxes):
        for k in range(ny + 1):
            for i in range(nx + 1):
                if node_in_D(bx, i, k):
                    mult[(i, k)] = mult.get((i, k), 0) + 1
    mu = np.array([1.0 / mult[(i, k)] if node_in_D(boxes[j], i, k) else 0.0 for i, k in nodes])
    At = np.zeros((m, m))
    Ao = np.zeros((m, m))
    for ey in range(y0, y1):
        for ex in range(x0, x1):
            for qa, qb in itertools.product(range(3), range(3)):
                x = (ex + g1[qa]) * h
                y = (ey + g1[qb]) * h
                w = w1[qa] * w1[qb] * h * h
                grads = np.array([[_dhat(x / h - i) / h * _hat(y / h - k),
                                   _hat(x / h - i) * _dhat(y / h - k) / h] for i, k in nodes])
                contrib = w * kap[ey, ex] * grads @ grads.T
                At += contrib
                if any(in_box(bx, x, y) for jj, bx in enumerate(boxes) if jj != j):
                    Ao += contrib
    return At, Ao, mu, np.array([dofs[q] for q in keep]), nodes


@pytest.fixture(scope="module")
def small2d():
    rng = np.random.default_rng(7)
    nel = (8, 6)
    kap = 10.0 ** rng.uniform(-2, 3, size=(nel[1], nel[0]))
    return gen.darcy_problem(nel, kap, (2, 2), 1, dirichlet="top1_bottom0")


def test_q1_reference_element():
    for dim in (2, 3):
        k = gen.q1_reference_stiffness(dim, 0.25)
        assert np.allclose(k, k.T)
        assert np.abs(k.sum(axis=1)).max() < 1e-14  # constants in the kernel
        ev = np.linalg.eigvalsh(k)
        assert abs(ev[0]) < 1e-14 and ev[1] > 1e-3  # only constants
    # known 2D entries: diagonal 2/3, edge -1/6, diagonal neighbour -1/3
    k2 = gen.q1_reference_stiffness(2, 1.0)
    assert np.isclose(k2[0, 0], 2 / 3) and np.isclose(k2[0, 1], -1 / 6) and np.isclose(k2[0, 3], -1 / 3)
    # elasticity element: exactly 6 rigid body modes
    ke = gen.q1_elasticity_element(gen.isotropic_stiffness(3.0, 0.35), 0.5)
    ev = np.linalg.eigvalsh(ke)
    assert np.all(np.abs(ev[:6]) < 1e-12 * ev[-1]) and ev[6] > 1e-6 * ev[-1]


def test_patch_test_linear_field():
    """Assembled Neumann stiffness annihilates linear functions at interior
    nodes for constant kappa (consistency of the Q1 discretisation)."""
    nel = (6, 5, 4)
    p = gen.darcy_problem(nel, np.ones(nel[::-1]), (1, 1, 1), 0)
    import scipy.sparse as sp
    k = p.elem_dofs.shape[1]
    A = sp.csr_matrix((p.elem_mats.reshape(-1), (np.repeat(p.elem_dofs, k, 1).ravel(),
                       np.tile(p.elem_dofs, (1, k)).ravel())), shape=(p.n, p.n))
    nn = [v + 1 for v in nel]
    i, j, l = np.meshgrid(np.arange(nn[0]), np.arange(nn[1]), np.arange(nn[2]), indexing="ij")
    u = np.zeros(p.n)
    ids = (i + nn[0] * j + nn[0] * nn[1] * l).ravel()
    u[ids] = (1.0 + 2.0 * i - 3.0 * j + 0.5 * l).ravel() * p.h
    r = A @ u
    inner = ((i > 0) & (i < nel[0]) & (j > 0) & (j < nel[1]) & (l > 0) & (l < nel[2])).ravel()
    assert np.abs(r[ids[inner]]).max() < 1e-12


def test_sets_pu_and_pencil_match_bruteforce(small2d):
    """N_j, D_j, X_j, Atilde_j and A_j^o agree entrywise with the pointwise
    construction from the continuous definitions (Sections 3 and 4.3)."""
    p = small2d
    sets = oracle.subdomain_sets(p)
    e_tau = oracle.element_multiplicity(p)
    c, xs = oracle.partition_of_unity(p, sets)
    for j in range(p.n_sub):
        At_b, Ao_b, mu_b, dofs_b, _ = _brute_pencil(p, j)
        assert np.array_equal(sets[j]["N"], dofs_b)
        assert np.allclose(xs[j], mu_b, rtol=0, atol=1e-15)
        At = oracle.neumann_matrix(p, j, sets).toarray()
        Ao = oracle.overlap_matrix(p, j, sets, e_tau).toarray()
        scale = np.abs(At_b).max()
        assert np.abs(At - At_b).max() < 1e-12 * scale
        assert np.abs(Ao - Ao_b).max() < 1e-12 * scale
        _, B = oracle.geneo_pencil(p, j, sets, xs, e_tau, "paper")
        assert np.abs(B.toarray() - np.diag(mu_b) @ Ao_b @ np.diag(mu_b)).max() < 1e-12 * scale


def test_dirichlet_matrix_is_restriction(small2d):
    """A_j = R_j A R_j^T with R_j the 0/1 matrix picking D_j (Section 3)."""
    p = small2d
    sets = oracle.subdomain_sets(p)
    Ad = p.A.toarray()
    for j in range(p.n_sub):
        D = sets[j]["D"]
        R = np.zeros((D.size, p.n))
        R[np.arange(D.size), D] = 1.0
        assert np.array_equal(oracle.dirichlet_matrix(p.A, D).toarray(), R @ Ad @ R.T)


def test_partition_of_unity_sums_to_one():
    """sum_j R_j^T X_j = 1 on free dofs, 0 on Dirichlet dofs (Section 4.3)."""
    for nel, parts, ov in [((16, 12), (3, 2), 1), ((8, 8, 8), (2, 2, 2), 2)]:
        kap = np.ones(nel[::-1])
        p = gen.darcy_problem(nel, kap, parts, ov)
        sets = oracle.subdomain_sets(p)
        _, xs = oracle.partition_of_unity(p, sets)
        s = np.zeros(p.n)
        for j, st in enumerate(sets):
            s[st["N"]] += xs[j]
            # zero on the subdomain boundary (dofs of N_j outside D_j)
            outside = np.setdiff1d(np.arange(st["N"].size), st["dpos"])
            assert np.all(xs[j][outside] == 0.0)
        assert np.all(s[p.dirichlet == 0] == 1.0)
        assert np.all(s[p.dirichlet > 0] == 0.0)


def _closed_form_q1_dirichlet(nel, h):
    """Eigenvalues of the 2D Q1 Dirichlet stiffness with B = identity and with
    B = the Q1 mass matrix, from the 1D factors k = (2/h)(1 - cos t),
    m = (h/3)(2 + cos t), t = k pi / n (tensor-product structure)."""
    th = [np.arange(1, n) * np.pi / n for n in nel]
    kx, ky = [(2 / h) * (1 - np.cos(t)) for t in th]
    mx, my = [(h / 3) * (2 + np.cos(t)) for t in th]
    std = np.sort((kx[:, None] * my[None, :] + mx[:, None] * ky[None, :]).ravel())
    mass = np.sort((kx / mx)[:, None] + (ky / my)[None, :]).ravel()
    return std, np.sort(mass)


@pytest.mark.parametrize("dense_max", [100000, 0])
def test_eigensolver_closed_form(dense_max):
    """The shift-and-invert eigensolver (Section 4.4) reproduces the closed-form
    spectrum of a constant-coefficient Dirichlet box for a standard (B = I)
    and a mass-matrix (B = M) pencil, dense and ARPACK paths."""
    import scipy.sparse as sp
    nel = (12, 9)
    h = 1.0 / 12
    p = gen.darcy_problem(nel, np.ones(nel[::-1]), (1, 1), 0)
    free = np.nonzero(p.dirichlet == 0)[0]
    K = p.A[free][:, free].tocsr()
    std, mass = _closed_form_q1_dirichlet(nel, h)
    lam, V = oracle.local_eigenpairs(K, sp.identity(K.shape[0], format="csr"), 8, -0.01, dense_max)
    assert np.allclose(lam, std[:8], rtol=1e-10)
    m1 = [sp.diags([np.full(n - 2, h / 6), np.full(n - 1, 4 * h / 6), np.full(n - 2, h / 6)],
                   [-1, 0, 1]) for n in (nel[0], nel[1])]
    M = sp.kron(m1[1], m1[0]).tocsr()
    lam, _ = oracle.local_eigenpairs(K, M, 8, -0.01, dense_max)
    assert np.allclose(lam, mass[:8], rtol=1e-10)


def _geneo_spectra(p, form="paper", k=12):
    sets = oracle.subdomain_sets(p)
    e_tau = oracle.element_multiplicity(p)
    _, xs = oracle.partition_of_unity(p, sets)
    out = []
    for j in range(p.n_sub):
        At, B = oracle.geneo_pencil(p, j, sets, xs, e_tau, form)
        lam, _ = oracle.local_eigenpairs(At, B, k, -0.01, 100000)
        out.append(lam)
    return out


def test_zero_eigenvalues_floating_subdomains_darcy():
    """Floating subdomains have exactly one zero eigenvalue (constants); those
    touching the Dirichlet boundary have none."""
    nel = (12, 12)
    rng = np.random.default_rng(3)
    p = gen.darcy_problem(nel, 10.0 ** rng.uniform(0, 2, size=nel), (3, 3), 1)
    spectra = _geneo_spectra(p)
    for j, lam in enumerate(spectra):
        nz = np.count_nonzero(np.abs(lam) < 1e-9)
        assert nz == (1 if j == 4 else 0), (j, lam[:3])


def test_zero_eigenvalues_floating_subdomain_elasticity():
    """A floating 3D elasticity subdomain has exactly six zero eigenvalues
    (rigid body modes); the clamped one has none."""
    p = gen.elasticity_problem((8, 3, 3), (2, 1, 1), 1, layer_thickness=1)
    spectra = _geneo_spectra(p, k=10)
    assert np.count_nonzero(np.abs(spectra[0]) < 1e-9) == 0
    assert np.count_nonzero(np.abs(spectra[1]) < 1e-9) == 6
    assert spectra[1][6] > 1e-6


def test_two_copies_of_the_domain_give_lambda_four():
    """Two subdomains both equal to Omega: every dof has multiplicity 2, so
    X = 1/2 and every element is an overlap element, hence B = Atilde/4 and
    every eigenvalue equals 4 exactly (both eigenproblem forms)."""
    nel = (6, 5)
    rng = np.random.default_rng(1)
    p = gen.darcy_problem(nel, 10.0 ** rng.uniform(-3, 3, size=nel[::-1]), (1, 1), 0)
    p.sub_elem_ptr = np.array([0, p.n_elem, 2 * p.n_elem], dtype=np.int64)
    p.sub_elem = np.concatenate([np.arange(p.n_elem)] * 2).astype(np.int32)
    free = np.nonzero(p.dirichlet == 0)[0].astype(np.int32)
    p.sub_dof_ptr = np.array([0, free.size, 2 * free.size], dtype=np.int64)
    p.sub_dof = np.concatenate([free, free])
    for form in ("paper", "full"):
        for lam in _geneo_spectra(p, form, k=10):
            assert np.allclose(lam, 4.0, rtol=1e-10)


def test_arpack_agrees_with_dense():
    """Section 4.4's ARPACK shift-invert path equals the dense solve."""
    k = gen.kappa_channels_2d((64, 64), seed=0)
    p = gen.darcy_problem((64, 64), k, (4, 4), 1)
    sets = oracle.subdomain_sets(p)
    e_tau = oracle.element_multiplicity(p)
    _, xs = oracle.partition_of_unity(p, sets)
    for j in (0, 5):
        At, B = oracle.geneo_pencil(p, j, sets, xs, e_tau)
        l1, V1 = oracle.local_eigenpairs(At, B, 12, -0.01, 100000)
        l2, V2 = oracle.local_eigenpairs(At, B, 12, -0.01, 0)
        assert np.all(np.abs(l1 - l2) <= 1e-9 * np.maximum(np.abs(l1), 1e-3))


def test_coarse_space_properties():
    """Unit basis vectors (Section 4.4), A_H symmetric positive definite and
    zero between non-overlapping subdomains (Section 4.5)."""
    k = gen.kappa_channels_2d((48, 48), seed=2, contrast=1e4)
    p = gen.darcy_problem((48, 48), k, (4, 4), 1)
    o = oracle.GenEOOracle(p, oracle.OracleOptions(nev_max=6))
    norms = np.sqrt(np.asarray(o.Zg.multiply(o.Zg).sum(axis=0))).ravel()
    assert np.allclose(norms, 1.0, rtol=1e-14)
    assert np.allclose(o.AH, o.AH.T, rtol=0, atol=1e-13 * np.abs(o.AH).max())
    assert np.linalg.eigvalsh(o.AH)[0] > 0
    boxes = p.boxes_grown
    for i in range(p.n_sub):
        for j in range(p.n_sub):
            (a0, b0), (a1, b1) = boxes[i]
            (c0, d0), (c1, d1) = boxes[j]
            disjoint = a1 <= c0 or c1 <= a0 or b1 <= d0 or d1 <= b0
            if disjoint:
                blk = o.AH[o.offsets[i]:o.offsets[i] + o.ms[i], o.offsets[j]:o.offsets[j] + o.ms[j]]
                assert np.all(blk == 0.0)


def test_apply_matches_dense_operator(small2d):
    """M^{-1} r equals the dense sum_j R_j^T A_j^{-1} R_j + Z A_H^{-1} Z^T built
    from explicit 0/1 restriction matrices and dense inverses (Definition 2)."""
    p = small2d
    o = oracle.GenEOOracle(p, oracle.OracleOptions(nev_max=3))
    Ad = p.A.toarray()
    M = np.zeros_like(Ad)
    for j, st in enumerate(o.sets):
        D = st["D"]
        R = np.zeros((D.size, p.n))
        R[np.arange(D.size), D] = 1.0
        M += R.T @ np.linalg.inv(R @ Ad @ R.T) @ R
    Z = o.Zg.toarray()
    M += Z @ np.linalg.inv(Z.T @ Ad @ Z) @ Z.T
    dmask = p.dirichlet > 0
    M[dmask, :] = 0.0
    M[:, dmask] = 0.0
    M[dmask, dmask] = 1.0
    rng = np.random.default_rng(0)
    for _ in range(3):
        r = rng.standard_normal(p.n)
        assert np.allclose(o.apply(r), M @ r, rtol=1e-11, atol=1e-11 * np.abs(M @ r).max())
    assert np.allclose(M, M.T, atol=1e-12 * np.abs(M).max())


def test_pcg_solution_and_condition_estimate(small2d):
    """PCG reaches the direct solution, and its Lanczos estimate of
    kappa(M^{-1}A) matches the dense eigenvalues of M^{-1}A."""
    p = small2d
    o = oracle.GenEOOracle(p, oracle.OracleOptions(nev_max=2))
    x, it, hist, kap = o.solve(tol=1e-12)
    xs = spla.spsolve(p.A.tocsc(), p.b)
    assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)
    free = np.nonzero(p.dirichlet == 0)[0]
    Minv = np.stack([o.apply(e) for e in np.eye(p.n)], axis=1)
    ev = np.sort(np.real(sla.eigvals(Minv[np.ix_(free, free)] @ p.A.toarray()[np.ix_(free, free)])))
    assert abs(kap - ev[-1] / ev[0]) <= 1e-6 * ev[-1] / ev[0]


def test_theorem1_bound_and_flat_condition_number():
    """Theorem 1: with tau_j = delta_j/H_j the estimated condition number stays
    below the bound and does not grow with the contrast, while the one-level
    estimate grows in proportion to it (Section 5.2 and Table 1)."""
    kg, k1, its = [], [], []
    for c in (1e4, 1e6, 1e8):
        k = gen.kappa_channels_2d((48, 48), seed=4, contrast=c)
        p = gen.darcy_problem((48, 48), k, (4, 4), 1)
        H, delta = 12 + 2, 1
        o = oracle.GenEOOracle(p, oracle.OracleOptions(tau=delta / H, nev_max=40))
        _, _, hist, kap = o.solve(tol=1e-8)
        # iterations until the recursive residual first reaches tol (at
        # contrast 1e8 the true residual then stops at the FP64 rounding
        # floor of x, which is not a property of the preconditioner)
        it = int(np.argmax(np.asarray(hist) <= 1e-8))
        assert kap <= oracle.theorem1_bound(4, [H / delta])
        kg.append(kap)
        its.append(it)
        o1 = oracle.GenEOOracle(p, oracle.OracleOptions(nev_max=0))
        _, _, _, kap1 = o1.solve(tol=1e-8)
        k1.append(kap1)
    assert max(kg) < 1.1 * min(kg)
    assert its[-1] <= 1.3 * its[0]
    assert k1[-1] > 1e3 * k1[0]


def test_layers_need_exactly_four_eigenvectors():
    """Section 5.2: 40 horizontal layers on 8x8 subdomains with a two-cell
    overlap become robust exactly at four eigenvectors per subdomain."""
    kap = {}
    for c in (1.0, 1e6):
        k = gen.kappa_layers_2d((80, 80), c, n_layers=40)
        p = gen.darcy_problem((80, 80), k, (8, 8), 2, dirichlet="top1_bottom0")
        for nev in (3, 4):
            o = oracle.GenEOOracle(p, oracle.OracleOptions(nev_max=nev, fixed_nev=True))
            _, it, _, kp = o.solve(tol=1e-8)
            kap[(c, nev)] = kp
    assert kap[(1e6, 3)] > 1e3 * kap[(1.0, 3)]      # three: not robust
    assert kap[(1e6, 4)] < 3.0 * kap[(1.0, 4)]      # four: robust


def test_one_level_iterations_grow_with_subdomains():
    """Table 1 shape: one-level iterations grow with N faster than GenEO's,
    whose condition estimate stays bounded."""
    k = gen.kappa_channels_2d((64, 64), seed=0, contrast=1e3)
    it1, itg, kg = [], [], []
    for parts in ((2, 2), (4, 4), (8, 8)):
        p = gen.darcy_problem((64, 64), k, parts, 1)
        _, a, _, _ = oracle.GenEOOracle(p, oracle.OracleOptions(nev_max=0)).solve(tol=1e-8)
        _, b, _, kb = oracle.GenEOOracle(p, oracle.OracleOptions(nev_max=8)).solve(tol=1e-8)
        it1.append(a)
        itg.append(b)
        kg.append(kb)
    assert it1[2] > 1.8 * it1[0]
    assert it1[2] / it1[0] > itg[2] / itg[0]
    assert max(kg) < 2.0 * min(kg)


def _two_copies_problem():
    nel = (6, 5)
    rng = np.random.default_rng(1)
    p = gen.darcy_problem(nel, 10.0 ** rng.uniform(-3, 3, size=nel[::-1]), (1, 1), 0)
    p.sub_elem_ptr = np.array([0, p.n_elem, 2 * p.n_elem], dtype=np.int64)
    p.sub_elem = np.concatenate([np.arange(p.n_elem)] * 2).astype(np.int32)
    free = np.nonzero(p.dirichlet == 0)[0].astype(np.int32)
    p.sub_dof_ptr = np.array([0, free.size, 2 * free.size], dtype=np.int64)
    p.sub_dof = np.concatenate([free, free])
    return p


def test_selection_cap_and_strict_threshold():
    """R4 on the exact special case where every eigenvalue is 4: with tau
    just above 4 every eigenvalue is below the threshold, so m_j is the cap
    nev_max (3 here, out of 6 computed pairs); with tau just below 4 none is,
    so m_j = 0 and the method is one-level; fixed-count mode takes nev_max
    whatever tau is.  (The two subdomains are identical, so their coarse
    vectors coincide and A_H would be singular: only the local steps run.)"""
    p = _two_copies_problem()
    for tau, fixed, want in ((4.0 + 1e-9, False, 3), (4.0 - 1e-9, False, 0), (4.0 - 1e-9, True, 3)):
        o = oracle.GenEOOracle(p, oracle.OracleOptions(tau=tau, nev_max=3, fixed_nev=fixed),
                               subdomains=[0, 1])
        assert [o.ms[j] for j in range(2)] == [want, want], (tau, fixed, o.ms)
        assert [o.Zloc[j].shape[1] for j in range(2)] == [want, want]
        assert all(o.lams[j].size == 6 for j in range(2))


def test_selection_cap_on_layers():
    """Section 5.2: on 40 layers with 8 x 8 subdomains the subdomains crossed
    by the layers have at least four small eigenvalues; with nev_max = 3 and
    a threshold above them each such subdomain takes exactly three."""
    k = gen.kappa_layers_2d((80, 80), 1e6, n_layers=40)
    p = gen.darcy_problem((80, 80), k, (8, 8), 2, dirichlet="top1_bottom0")
    o = oracle.GenEOOracle(p, oracle.OracleOptions(tau=0.5, nev_max=3), subdomains=[27, 36])
    for j in (27, 36):
        assert np.count_nonzero(o.lams[j] < 0.5) >= 4, o.lams[j][:6]
        assert o.ms[j] == 3


def test_sarkis_partition_of_unity_ramp():
    """R11 on a strip of two subdomains (16 x 4 elements, parts split at
    x = 8, overlap 2): across the overlap the weights fall linearly from 1 to
    0 over 2 delta = 4 element layers, X_1(i) = (8 + 2 - i) / 4 at node column
    i, they sum to one on every free dof and vanish on the inner boundary."""
    p = gen.darcy_problem((16, 4), np.ones((4, 16)), (2, 1), 2)
    sets = oracle.subdomain_sets(p)
    _, xs = oracle.sarkis_partition_of_unity(p, sets)
    tot = np.zeros(p.n)
    for s, x in zip(sets, xs):
        tot[s["N"]] += x
        inner = np.setdiff1d(np.arange(s["N"].size), s["dpos"])
        assert np.all(x[inner] == 0.0)
    free = p.dirichlet == 0
    assert np.allclose(tot[free], 1.0, rtol=0, atol=1e-15) and np.all(tot[~free] == 0.0)
    col = sets[0]["N"] % 17
    want = np.clip((10.0 - col) / 4.0, 0.0, 1.0)
    assert np.allclose(xs[0], want, rtol=0, atol=1e-15), (xs[0], want)


def test_sarkis_partition_of_unity_gives_robust_geneo():
    """The coarse space built with the smooth partition of unity is as robust
    as with the standard one (Section 3 reports no large influence): the
    condition estimate stays flat in the contrast."""
    kap = []
    for c in (1e2, 1e6):
        k = gen.kappa_channels_2d((48, 48), seed=4, contrast=c)
        p = gen.darcy_problem((48, 48), k, (4, 4), 2)
        o = oracle.GenEOOracle(p, oracle.OracleOptions(nev_max=10), pu="sarkis")
        _, _, _, kp = o.solve(tol=1e-8)
        kap.append(kp)
    assert kap[1] < 2.0 * kap[0], kap


def test_pcg_true_residual_replacement():
    """R8: at contrast 1e6 the solve stops with the true residual below tol;
    at contrast 1e8 the recursive residual reaches tol while the true one is
    still far above it; replacing it lowers the true residual to the rounding
    floor of x in FP64 (about 3e-7 here), where the solve stops instead of
    iterating on."""
    for c, converged in ((1e6, True), (1e8, False)):
        k = gen.kappa_channels_2d((48, 48), seed=4, contrast=c)
        p = gen.darcy_problem((48, 48), k, (4, 4), 1)
        o = oracle.GenEOOracle(p, oracle.OracleOptions(tau=1 / 14, nev_max=40))
        x, it, hist, _ = o.solve(tol=1e-8)
        res = np.linalg.norm(p.b - p.A @ x) / np.linalg.norm(p.b)
        if converged:
            assert res <= 1e-8
        else:
            first = int(np.argmax(np.asarray(hist) <= 1e-8))
            x0, _, _, _ = oracle.pcg(p.A, p.b, o.apply, tol=1e-8, maxit=first)
            res0 = np.linalg.norm(p.b - p.A @ x0) / np.linalg.norm(p.b)
            assert res0 > 1e-7 and res < res0 and it < first + 100, (res0, res, first, it)
