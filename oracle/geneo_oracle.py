"""FP64 CPU oracle of the GenEO two-level overlapping Schwarz preconditioner.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the CUDA library or its
binding.  It is deliberately plain and slow: numpy/scipy, float64 throughout,
each step written the way the paper states it, library primitives (sparse
products, sparse LU, dense ``eigh``, ARPACK) used as whole steps.

Citations refer to the paper "A High-Performance Implementation of a Robust
Preconditioner for Heterogeneous Problems" (Seelinger, Reinarz, Scheichl):
Section 3 (definitions of R_j, A_j, the two-level additive Schwarz operator,
the partition of unity, the GenEO eigenproblem eq. 5, the coarse space and
Theorem 1), Section 4.3 (discrete eigenproblem, Neumann and overlap matrices,
discrete partition of unity), Section 4.4 (shift-and-invert eigensolve and the
l2 normalisation of the basis), Section 4.5 (coarse matrix, R_H and R_H^T).

Readings where the paper is silent or ambiguous (each one is stated where it
is used):
  R1  Eigenproblem right-hand side: X_j A_j^o X_j ("paper" form, Section 4.3);
      the "full" form X_j Atilde_j X_j is kept as an option.
  R2  The left-hand matrix of the eigenproblem is the Neumann matrix
      Atilde_j (no Dirichlet condition on the subdomain boundary, Section 4.3);
      the local solves of the preconditioner use the Dirichlet A_j (Section 3).
  R3  Shift sigma = -0.01 ("near zero", Section 4.4; sigma = 0 is not usable
      because Atilde_j is singular on floating subdomains).
  R4  Selection: m_j = #{k : lambda_k < tau}, capped at nev_max (Theorem 1
      with a scaled threshold, end of Section 3); fixed-count mode takes nev.
  R5  Overlap elements: elements that belong to more than one subdomain (the
      set definition of Omega_j^o in Section 3), counted per element.
  R6  Global Dirichlet dofs are eliminated: they belong to no N_j and no D_j,
      the partition of unity is zero there, and the preconditioner acts as the
      identity on them.
  R7  Basis vectors are X_j p / ||X_j p||_2 with the sign chosen so that the
      entry of largest magnitude is positive (first such entry on ties).
  R8  PCG starts from x0 = 0 and stops when ||r_k||_2 <= tol ||b||_2
      (Section 5.3 states a residual reduction): the recursively updated
      residual is tested first, then the true residual b - A x, which
      replaces the recursive one when it is still above tol.
  R9  The condition number reported by the paper is estimated from the CG
      coefficients (Lanczos tridiagonal matrix).
  R11 The smooth partition of unity Section 3 shows (Sarkis) is the ratio of
      element-layer distances to the inner subdomain boundaries.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


@dataclasses.dataclass
class OracleOptions:
    tau: float = 0.3            # selection threshold (R4)
    nev_max: int = 10           # cap on eigenvectors per subdomain
    fixed_nev: bool = False     # take exactly nev_max per subdomain
    sigma: float = -0.01        # shift (R3)
    eig_form: str = "paper"     # "paper": X A^o X; "full": X Atilde X (R1)
    dense_max: int = 2500       # dense generalized eigh up to this local size
    guard: int = -1             # extra ARPACK vectors (default min(10, nev_max))
    arpack_tol: float = 1e-12


# ----------------------------------------------------------------------------
# Section 3: subdomains, restriction sets and partition of unity.
# ----------------------------------------------------------------------------
def subdomain_sets(prob):
    """Dof sets of each overlapping subdomain Omega_j (Section 3).

    N_j: dofs of the closure of Omega_j without global Dirichlet dofs (R6);
         this is the space V_h(Omega_j) of the eigenproblem.
    D_j: dofs of N_j whose every element lies in Omega_j; these are the dofs
         of V_{h,0}(Omega_j) (functions vanishing on the subdomain boundary),
         i.e. the range of R_j.
    Returns a list of dicts with global index arrays 'N', 'D' and 'dpos'
    (positions of D_j inside N_j).
    """
    n = prob.n
    count_all = np.bincount(prob.elem_dofs.ravel(), minlength=n)
    out = []
    for j in range(prob.n_sub):
        e = prob.sub_elems(j)
        count_j = np.bincount(prob.elem_dofs[e].ravel(), minlength=n)
        nodes = np.nonzero(count_j)[0]
        N = nodes[prob.dirichlet[nodes] == 0]
        interior = count_j[N] == count_all[N]
        out.append({"N": N, "D": N[interior], "dpos": np.nonzero(interior)[0]})
    return out


def element_multiplicity(prob):
    """e_tau = number of subdomains containing element tau (R5)."""
    return np.bincount(prob.sub_elem, minlength=prob.n_elem)


def partition_of_unity(prob, sets):
    """Discrete partition of unity X_j (Section 4.3, Definition 3).

    c_k = number of subdomains whose D_j contains dof k ("adding vectors of
    ones across subdomains"); X_j(k) = 1/c_k on D_j and 0 on the remaining
    dofs of N_j (the subdomain boundary).  Returns (c, [X_j on N_j]).
    """
    c = np.zeros(prob.n)
    for s in sets:
        c[s["D"]] += 1.0
    xs = []
    for s in sets:
        x = np.zeros(s["N"].size)
        x[s["dpos"]] = 1.0 / c[s["D"]]
        xs.append(x)
    return c, xs


def sarkis_partition_of_unity(prob, sets):
    """Smooth (Sarkis) partition of unity, the second example of Section 3
    (Fig. 2, right), read as R11: d_j(k) is the number of element layers
    between dof k and the inner boundary of Omega_j (the dofs of N_j that
    are not in D_j, i.e. that touch an element outside Omega_j), measured as
    breadth-first distance over the elements of Omega_j (two dofs are
    neighbours when one element holds both); X_j(k) = d_j(k) / sum_i d_i(k).
    X_j vanishes on the inner boundary and ramps up linearly across the
    overlap.  A subdomain without inner boundary takes d_j = 1 everywhere.
    Returns (sum_i d_i, [X_j on N_j])."""
    dist = []
    for j, s in enumerate(sets):
        N = s["N"]
        el = prob.sub_elems(j)
        ed = prob.elem_dofs[el]
        loc = np.searchsorted(N, ed)
        loc = np.where(loc < N.size, loc, 0)
        valid = N[loc] == ed
        k = ed.shape[1]
        rows = np.repeat(loc, k, axis=1)[np.repeat(valid, k, axis=1) & np.tile(valid, (1, k))]
        cols = np.tile(loc, (1, k))[np.repeat(valid, k, axis=1) & np.tile(valid, (1, k))]
        G = sp.csr_matrix((np.ones(rows.size), (rows, cols)), shape=(N.size, N.size))
        d = np.full(N.size, -1, dtype=np.int64)
        inner = np.ones(N.size, dtype=bool)
        inner[s["dpos"]] = False
        if not inner.any():
            dist.append(np.ones(N.size))
            continue
        d[inner] = 0
        frontier = np.nonzero(inner)[0]
        level = 0
        while frontier.size:
            level += 1
            reach = np.unique(G[frontier].indices)
            frontier = reach[d[reach] < 0]
            d[frontier] = level
        dist.append(d.astype(np.float64))
    total = np.zeros(prob.n)
    for s, d in zip(sets, dist):
        total[s["N"]] += d
    xs = []
    for s, d in zip(sets, dist):
        x = np.zeros(s["N"].size)
        x[s["dpos"]] = d[s["dpos"]] / total[s["D"]]
        xs.append(x)
    return total, xs


# ----------------------------------------------------------------------------
# Local matrices (Sections 3 and 4.3).
# ----------------------------------------------------------------------------
def dirichlet_matrix(A, D):
    """A_j = R_j A R_j^T: the rows and columns D_j of A (Section 3)."""
    return A[D][:, D].tocsr()


def _assemble_local(prob, elems, N):
    """Sum of the element matrices of ``elems`` in the local numbering of N;
    dofs outside N (global Dirichlet dofs) are dropped (R6)."""
    k = prob.elem_dofs.shape[1]
    ed = prob.elem_dofs[elems]
    loc = np.searchsorted(N, ed)
    loc = np.where(loc < N.size, loc, 0)
    valid = N[loc] == ed
    rows = np.repeat(loc, k, axis=1)
    cols = np.tile(loc, (1, k))
    ok = np.repeat(valid, k, axis=1) & np.tile(valid, (1, k))
    vals = prob.elem_mats[elems].reshape(len(elems), k * k)
    m = sp.coo_matrix((vals[ok], (rows[ok], cols[ok])), shape=(N.size, N.size))
    return m.tocsr()


def neumann_matrix(prob, j, sets):
    """Atilde_j: assembled over all elements of Omega_j with no Dirichlet
    condition on the subdomain boundary, global Dirichlet dofs removed
    (Section 4.3, R2, R6)."""
    return _assemble_local(prob, prob.sub_elems(j), sets[j]["N"])


def overlap_matrix(prob, j, sets, e_tau):
    """A_j^o: assembled only over the overlap elements of Omega_j, i.e. those
    that also belong to another subdomain (Section 4.3, R5)."""
    el = prob.sub_elems(j)
    return _assemble_local(prob, el[e_tau[el] > 1], sets[j]["N"])


def geneo_pencil(prob, j, sets, xs, e_tau, form="paper"):
    """The pencil (Atilde_j, B_j) of the discrete GenEO eigenproblem
    Atilde_j p = lambda X_j A_j^o X_j p (Section 4.3; R1 for the "full" form)."""
    At = neumann_matrix(prob, j, sets)
    if form == "paper":
        Ao = overlap_matrix(prob, j, sets, e_tau)
    elif form == "full":
        Ao = At
    else:
        raise ValueError(form)
    X = sp.diags(xs[j])
    B = (X @ Ao @ X).tocsr()
    return At, B


def local_eigenpairs(At, B, k, sigma, dense_max=2500, tol=1e-12):
    """The k eigenpairs of Atilde p = lambda B p of smallest lambda (Section 4.4).

    Shift and invert: eigenvalues nu of (Atilde - sigma B)^{-1} B satisfy
    nu = 1/(lambda - sigma) with the same eigenvectors; the wanted lambda are
    the largest nu.  Small problems use a dense generalized symmetric
    eigensolver on (B, K) with K = Atilde - sigma B; larger ones ARPACK in
    shift-invert mode exactly as in the paper.  Eigenvalues with nu <= 0 are
    infinite (B-null directions).  Returns (lambda ascending, P) with P
    normalised so that p^T K p = 1.
    """
    n = At.shape[0]
    k = min(k, n)
    if n <= dense_max:
        K = (At - sigma * B).toarray()
        nu, V = sla.eigh(B.toarray(), K)
        nu, V = nu[::-1][:k], V[:, ::-1][:, :k]
    else:
        kk = min(k, n - 2)
        lam, V = spla.eigsh(At.tocsc(), k=kk, M=B.tocsc(), sigma=sigma, which="LM", tol=tol)
        with np.errstate(divide="ignore"):
            nu = 1.0 / (lam - sigma)
        order = np.argsort(-nu)
        nu, V = nu[order], V[:, order]
        K = (At - sigma * B).tocsr()
        V = V / np.sqrt(np.einsum("ij,ij->j", V, K @ V))[None, :]
    with np.errstate(divide="ignore"):
        lam = np.where(nu > 0, sigma + 1.0 / np.where(nu > 0, nu, 1.0), np.inf)
    return lam, V


def select_count(lam, tau, nev_max, fixed_nev=False):
    """m_j: number of eigenvectors taken (Theorem 1 and the remark after it, R4)."""
    if fixed_nev:
        return int(min(nev_max, lam.size))
    return int(min(nev_max, np.count_nonzero(lam < tau)))


def coarse_vectors(P, x, m):
    """Local parts of the coarse basis: X_j p_k / ||X_j p_k||_2 (Definition 4
    and Section 4.4), sign fixed by R7.  Returns an array (|N_j|, m)."""
    Z = np.zeros((P.shape[0], m))
    for k in range(m):
        v = x * P[:, k]
        nrm = np.linalg.norm(v)
        if nrm == 0.0:
            continue
        v = v / nrm
        if v[np.argmax(np.abs(v))] < 0:
            v = -v
        Z[:, k] = v
    return Z


def coarse_matrix(A, Zg):
    """A_H = R_H A R_H^T with R_H^T = Z (Section 3 and Section 4.5)."""
    return (Zg.T @ (A @ Zg)).toarray()


# ----------------------------------------------------------------------------
# Krylov solver (Section 5.3 / 5.4: preconditioned CG, R8, R9).
# ----------------------------------------------------------------------------
def lanczos_condition_estimate(alphas, betas):
    """Condition-number estimate of M^{-1}A from the CG coefficients: the
    extreme eigenvalues of the Lanczos tridiagonal matrix (R9)."""
    m = len(alphas)
    if m == 0:
        return 1.0
    d = np.zeros(m)
    e = np.zeros(max(m - 1, 0))
    for i in range(m):
        d[i] = 1.0 / alphas[i] + (betas[i - 1] / alphas[i - 1] if i > 0 else 0.0)
        if i < m - 1:
            e[i] = np.sqrt(betas[i]) / alphas[i]
    ev = sla.eigvalsh_tridiagonal(d, e)
    return float(ev[-1] / ev[0])


def pcg(A, b, apply_M, tol=1e-8, maxit=1000, x0=None, max_replace=5):
    """Textbook preconditioned conjugate gradients (R8).

    The iteration updates the residual recursively; when that recursive
    residual reaches tol, the true residual b - A x is formed.  If it is
    still above tol, it replaces the recursive residual and CG restarts from
    the current x (p = M^{-1} r), at most max_replace times; the solve stops
    unconverged when a replacement did not at least halve the true residual
    (the rounding floor of x in FP64 is reached).  A replacement breaks the
    Lanczos relation of the CG coefficients, so the condition estimate uses
    the coefficients up to the first replacement.  hist holds the recursive
    residuals ||r_k|| / ||b||.
    """
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A @ x
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x, 0, [0.0], 1.0
    z = apply_M(r)
    p = z.copy()
    rz = r @ z
    hist = [np.linalg.norm(r) / bn]
    alphas, betas = [], []
    it = 0
    replaced = 0
    n_lanczos = None
    last_true = np.inf
    while it < maxit:
        q = A @ p
        pq = p @ q
        if pq <= 0:
            break
        alpha = rz / pq
        x += alpha * p
        r -= alpha * q
        it += 1
        hist.append(np.linalg.norm(r) / bn)
        if n_lanczos is None:
            alphas.append(alpha)
        if hist[-1] <= tol:
            r_true = b - A @ x
            rel_true = np.linalg.norm(r_true) / bn
            if rel_true <= tol or replaced >= max_replace or rel_true > 0.5 * last_true:
                break
            last_true = rel_true
            replaced += 1
            if n_lanczos is None:
                n_lanczos = len(alphas)
            r = r_true
            z = apply_M(r)
            rz = r @ z
            p = z.copy()
            continue
        z = apply_M(r)
        rz_new = r @ z
        beta = rz_new / rz
        if n_lanczos is None:
            betas.append(beta)
        rz = rz_new
        p = z + beta * p
    return x, it, hist, lanczos_condition_estimate(alphas, betas)


def theorem1_bound(k0, H_over_delta):
    """Right-hand side of the condition-number bound of Theorem 1."""
    return (1 + k0) * (2 + k0 * (2 * k0 + 1) * max(1.0 + h for h in H_over_delta))


# ----------------------------------------------------------------------------
# The whole method.
# ----------------------------------------------------------------------------
# state handed to forked worker processes (see GenEOOracle, workers > 1)
_WORK = None


def _local_part(j):
    """Eigenproblem, selection and coarse vectors of subdomain j (the
    per-subdomain steps of Sections 4.3 and 4.4)."""
    prob, sets, xs, e_tau, o, guard = _WORK
    if o.nev_max <= 0:
        return j, np.zeros(0), 0, np.zeros((sets[j]["N"].size, 0))
    At, B = geneo_pencil(prob, j, sets, xs, e_tau, o.eig_form)
    lam, P = local_eigenpairs(At, B, o.nev_max + guard, o.sigma, o.dense_max, o.arpack_tol)
    m = select_count(lam, o.tau, o.nev_max, o.fixed_nev)
    return j, lam, m, coarse_vectors(P, xs[j], m)


class GenEOOracle:
    """Setup and application of M^{-1}_{AS,2} (Section 3, Definition 2).

    pu: None (the standard partition of unity of Section 4.3), "sarkis"
    (R11), or a list of weight vectors X_j on N_j given by the caller (any
    weights of Definition 3).  workers > 1 runs the independent
    per-subdomain eigenproblems in that many processes of the given
    multiprocessing start method ("fork" shares the problem without copying
    it; use it only in a process that has not initialised CUDA)."""

    def __init__(self, prob, opts=None, subdomains=None, pu=None, workers=1, mp_context="fork"):
        global _WORK
        self.prob = prob
        self.opts = opts or OracleOptions()
        o = self.opts
        A = prob.A
        self.sets = subdomain_sets(prob)
        self.e_tau = element_multiplicity(prob)
        if pu is None:
            self.c, self.xs = partition_of_unity(prob, self.sets)
        elif isinstance(pu, str) and pu == "sarkis":
            self.c, self.xs = sarkis_partition_of_unity(prob, self.sets)
        else:
            self.c, self.xs = None, [np.asarray(x, dtype=np.float64) for x in pu]
        guard = o.guard if o.guard >= 0 else min(10, o.nev_max)
        sel = list(range(prob.n_sub) if subdomains is None else subdomains)
        self.local_lu = {}
        self.lams, self.ms, self.Zloc = {}, {}, {}
        _WORK = (prob, self.sets, self.xs, self.e_tau, o, guard)
        try:
            if workers > 1 and len(sel) > 1:
                import multiprocessing as mp
                with mp.get_context(mp_context).Pool(workers) as pool:
                    parts = pool.map(_local_part, sel, chunksize=1)
            else:
                parts = [_local_part(j) for j in sel]
        finally:
            _WORK = None
        for j, lam, m, Z in parts:
            self.lams[j] = lam
            self.ms[j] = m
            self.Zloc[j] = Z
        for j in sel:
            Aj = dirichlet_matrix(A, self.sets[j]["D"])
            self.local_lu[j] = spla.splu(Aj.tocsc())
        self.subdomains = sel
        if subdomains is None:
            self._build_coarse()

    def _build_coarse(self):
        prob = self.prob
        rows, cols, vals = [], [], []
        off = 0
        self.offsets = {}
        for j in self.subdomains:
            Z = self.Zloc[j]
            N = self.sets[j]["N"]
            self.offsets[j] = off
            for k in range(Z.shape[1]):
                nz = np.nonzero(Z[:, k])[0]
                rows.append(N[nz])
                cols.append(np.full(nz.size, off + k))
                vals.append(Z[nz, k])
            off += Z.shape[1]
        self.dim_H = off
        if off > 0:
            self.Zg = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows),
                                     np.concatenate(cols))), shape=(prob.n, off))
            self.AH = coarse_matrix(prob.A, self.Zg)
            self.AH_chol = sla.cho_factor(self.AH, lower=True)
        else:
            self.Zg = sp.csr_matrix((prob.n, 0))
            self.AH = np.zeros((0, 0))
            self.AH_chol = None

    def apply(self, r):
        """z = M^{-1}_{AS,2} r = R_H^T A_H^{-1} R_H r + sum_j R_j^T A_j^{-1} R_j r,
        identity on global Dirichlet dofs (R6)."""
        z = np.zeros_like(r)
        for j in self.subdomains:
            D = self.sets[j]["D"]
            z[D] += self.local_lu[j].solve(r[D])
        if self.dim_H > 0:
            c = self.Zg.T @ r
            y = sla.cho_solve(self.AH_chol, c)
            z += self.Zg @ y
        dmask = self.prob.dirichlet > 0
        z[dmask] = r[dmask]
        return z

    def solve(self, b=None, tol=1e-8, maxit=1000):
        b = self.prob.b if b is None else b
        return pcg(self.prob.A, b, self.apply, tol, maxit)
