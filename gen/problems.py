"""Structured Q1 problems, coefficient fields and box partitions (inputs only).

Conventions shared by every consumer of these arrays:

* Nodes of an ``nel = (nx, ny[, nz])`` element grid are numbered
  lexicographically, x fastest: ``node = i + (nx+1)*j + (nx+1)*(ny+1)*k``.
* Elements are numbered the same way over the element grid.
* Local node ``a`` of an element is ``a = ax + 2*ay + 4*az`` with ``ax, ay, az``
  in {0, 1} the offsets of the node from the element's lower corner.
* Degrees of freedom: ``dof = ndn*node + c`` for ``c < ndn`` (ndn = 1 for Darcy,
  3 for elasticity).  Element dof ``ndn*a + c`` is dof ``c`` of local node ``a``.
* Element matrices are the unconstrained element stiffness matrices
  K_tau (Section 2, eqs. 2 and 3, on one element).  The global matrix A is
  their sum with the Dirichlet rows and columns replaced by identity rows
  (homogeneous elimination; a non-zero Dirichlet value g is lifted into b).
"""
from __future__ import annotations

import dataclasses
import itertools

import numpy as np
import scipy.sparse as sp

MASK64 = (1 << 64) - 1


# ----------------------------------------------------------------------------
# Counter-based generator (SplitMix64, Steele, Lea and Flood, OOPSLA 2014).
# ----------------------------------------------------------------------------
def splitmix64(x):
    """SplitMix64 finaliser applied to ``x`` (uint64 array or int).

    z = x + 0x9E3779B97F4A7C15; z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB; return z ^ (z >> 31).
    """
    z = np.asarray(x, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


# ----------------------------------------------------------------------------
# Reference Q1 element integrals.
# ----------------------------------------------------------------------------
_GAUSS2 = (0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0))  # on [0, 1]


def _q1_shape_grads(dim, xi):
    """Values and reference gradients of the 2**dim Q1 shape functions at xi."""
    nloc = 2 ** dim
    val = np.ones(nloc)
    grad = np.ones((nloc, dim))
    for a in range(nloc):
        bits = [(a >> d) & 1 for d in range(dim)]
        for d in range(dim):
            f = xi[d] if bits[d] else 1.0 - xi[d]
            df = 1.0 if bits[d] else -1.0
            val[a] *= f
            for e in range(dim):
                grad[a, e] *= df if e == d else f
    return val, grad


def q1_reference_stiffness(dim, h):
    """Element matrix of a(v, w) = int grad v . grad w on a cube of side h.

    Computed with the 2-point Gauss rule per direction, which is exact here.
    The entries scale as h**(dim-2).
    """
    nloc = 2 ** dim
    k = np.zeros((nloc, nloc))
    for q in itertools.product(_GAUSS2, repeat=dim):
        _, g = _q1_shape_grads(dim, q)
        k += (g @ g.T) * (0.5 ** dim)  # Gauss weights 1/2 per direction
    return k * h ** (dim - 2)


def q1_reference_load(dim, h):
    """int phi_a dx on a cube of side h (all local nodes equal: h**dim / 2**dim)."""
    return np.full(2 ** dim, h ** dim / 2 ** dim)


def isotropic_stiffness(E, nu):
    """6x6 Voigt stiffness (order xx, yy, zz, yz, xz, xy; engineering shear)."""
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    c = np.zeros((6, 6))
    c[:3, :3] = lam
    c[np.arange(3), np.arange(3)] += 2 * mu
    c[np.arange(3, 6), np.arange(3, 6)] = mu
    return c


def orthotropic_stiffness(E1, E2, E3, nu12, nu13, nu23, G12, G13, G23):
    """6x6 Voigt stiffness of an orthotropic material, axes 1, 2, 3 = x, y, z."""
    s = np.zeros((6, 6))
    s[0, 0], s[1, 1], s[2, 2] = 1 / E1, 1 / E2, 1 / E3
    s[0, 1] = s[1, 0] = -nu12 / E1
    s[0, 2] = s[2, 0] = -nu13 / E1
    s[1, 2] = s[2, 1] = -nu23 / E2
    s[3, 3], s[4, 4], s[5, 5] = 1 / G23, 1 / G13, 1 / G12
    return np.linalg.inv(s)


def rotate_voigt_z90(c):
    """Stiffness of the same material turned by 90 degrees about z (x <-> y)."""
    p = [1, 0, 2, 4, 3, 5]
    return c[np.ix_(p, p)]


def q1_elasticity_element(c, h):
    """24x24 element matrix of int C eps(u) : eps(v) on a cube of side h.

    Element dof ordering 3*a + component.  2x2x2 Gauss rule (exact for Q1).
    """
    k = np.zeros((24, 24))
    for q in itertools.product(_GAUSS2, repeat=3):
        _, g = _q1_shape_grads(3, q)
        g = g / h
        b = np.zeros((6, 24))
        for a in range(8):
            gx, gy, gz = g[a]
            b[0, 3 * a + 0] = gx
            b[1, 3 * a + 1] = gy
            b[2, 3 * a + 2] = gz
            b[3, 3 * a + 1], b[3, 3 * a + 2] = gz, gy
            b[4, 3 * a + 0], b[4, 3 * a + 2] = gz, gx
            b[5, 3 * a + 0], b[5, 3 * a + 1] = gy, gx
        k += b.T @ c @ b * (h ** 3) * 0.125
    return k


# ----------------------------------------------------------------------------
# Meshes and partitions.
# ----------------------------------------------------------------------------
def structured_mesh(nel):
    """Element -> node connectivity of a structured grid (int64 [n_elem, 2**d])."""
    nel = tuple(int(v) for v in nel)
    dim = len(nel)
    nn = [v + 1 for v in nel]
    strides = [1, nn[0], nn[0] * (nn[1] if dim > 1 else 1)]
    grids = np.meshgrid(*[np.arange(v) for v in nel[::-1]], indexing="ij")
    lower = np.zeros(grids[0].size, dtype=np.int64)
    for d in range(dim):
        lower += grids[dim - 1 - d].ravel().astype(np.int64) * strides[d]
    offs = np.zeros(2 ** dim, dtype=np.int64)
    for a in range(2 ** dim):
        offs[a] = sum(((a >> d) & 1) * strides[d] for d in range(dim))
    return lower[:, None] + offs[None, :]


def _split(n, p):
    """Split range(n) into p contiguous, nearly equal parts; returns bounds."""
    return [(n * i) // p for i in range(p + 1)]


def box_partition(nel, parts, overlap):
    """Non-overlapping box partition of the element grid, grown by layers.

    Each box Omega'_j is grown by ``overlap`` layers of elements; one layer adds
    every element sharing a vertex with the current set, which for a box extends
    it by one element per side, clipped to the grid (Section 3).
    Subdomains are numbered lexicographically (x fastest).
    Returns (boxes_core, boxes_grown) as lists of (lo, hi) per dimension,
    hi exclusive, in element indices.
    """
    dim = len(nel)
    bounds = [_split(nel[d], parts[d]) for d in range(dim)]
    cores, grown = [], []
    for idx in itertools.product(*[range(p) for p in parts[::-1]]):
        idx = idx[::-1]
        lo = [bounds[d][idx[d]] for d in range(dim)]
        hi = [bounds[d][idx[d] + 1] for d in range(dim)]
        cores.append((tuple(lo), tuple(hi)))
        glo = [max(0, lo[d] - overlap) for d in range(dim)]
        ghi = [min(nel[d], hi[d] + overlap) for d in range(dim)]
        grown.append((tuple(glo), tuple(ghi)))
    return cores, grown


def kd_partition(nel, n_parts, min_side, max_side, seed):
    """Irregular box partition by recursive bisection (k-d splits).

    The box with the longest side that can still be split is cut at a
    seeded random position so that both halves keep sides >= min_side, until
    n_parts boxes exist or no box can be split; boxes with a side above
    max_side are split first.  Returns a list of (lo, hi) element boxes."""
    rng = np.random.default_rng(seed)
    boxes = [(tuple(0 for _ in nel), tuple(nel))]
    while len(boxes) < n_parts:
        best, bd, blen = -1, -1, 0
        for i, (lo, hi) in enumerate(boxes):
            for d in range(len(nel)):
                L = hi[d] - lo[d]
                score = L + (10 ** 6 if L > max_side else 0)
                if L >= 2 * min_side and score > blen:
                    best, bd, blen = i, d, score
        if best < 0:
            break
        lo, hi = boxes.pop(best)
        L = hi[bd] - lo[bd]
        cut = lo[bd] + int(rng.integers(min_side, L - min_side + 1))
        hi1 = list(hi); hi1[bd] = cut
        lo2 = list(lo); lo2[bd] = cut
        boxes.append((lo, tuple(hi1)))
        boxes.append((tuple(lo2), hi))
    boxes.sort(key=lambda b: (b[0][::-1], b[1][::-1]))
    return boxes


def _box_ids(lo, hi, strides):
    grids = np.meshgrid(*[np.arange(lo[d], hi[d]) for d in range(len(lo))][::-1], indexing="ij")
    ids = np.zeros(grids[0].size, dtype=np.int64)
    for d in range(len(lo)):
        ids += grids[len(lo) - 1 - d].ravel().astype(np.int64) * strides[d]
    return ids


# ----------------------------------------------------------------------------
# Problem container.
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Problem:
    """All arrays the GenEO setup consumes (host copies, numpy)."""

    dim: int
    nel: tuple
    ndn: int                      # dofs per node
    n: int                        # global dofs
    elem_dofs: np.ndarray         # int32 [n_elem, k]
    elem_mats: np.ndarray         # float64 [n_elem, k, k]
    dirichlet: np.ndarray         # uint8 [n]
    A: sp.csr_matrix              # float64, int64 indptr, int32 indices
    b: np.ndarray                 # float64 [n]
    sub_elem_ptr: np.ndarray      # int64 [N+1]
    sub_elem: np.ndarray          # int32
    sub_dof_ptr: np.ndarray       # int64 [N+1]
    sub_dof: np.ndarray           # int32, sorted per subdomain, no Dirichlet dofs
    boxes_core: list
    boxes_grown: list
    overlap: int
    h: float
    coeff: np.ndarray | None = None
    name: str = ""

    @property
    def n_sub(self):
        return len(self.sub_elem_ptr) - 1

    @property
    def n_elem(self):
        return self.elem_dofs.shape[0]

    def sub_elems(self, j):
        return self.sub_elem[self.sub_elem_ptr[j]:self.sub_elem_ptr[j + 1]]

    def sub_dofs(self, j):
        return self.sub_dof[self.sub_dof_ptr[j]:self.sub_dof_ptr[j + 1]]


def _assemble(elem_dofs, elem_mats, n):
    k = elem_dofs.shape[1]
    rows = np.repeat(elem_dofs, k, axis=1).ravel()
    cols = np.tile(elem_dofs, (1, k)).ravel()
    a = sp.csr_matrix((elem_mats.reshape(-1), (rows, cols)), shape=(n, n))
    a.sum_duplicates()
    a.sort_indices()
    return a


def _finish(dim, nel, ndn, elem_nodes, elem_mats, load, dir_nodes_mask, dir_values,
            parts, overlap, h, coeff, name, cores=None, overlaps=None):
    nn = [v + 1 for v in nel]
    n_nodes = int(np.prod(nn))
    n = ndn * n_nodes
    if ndn == 1:
        elem_dofs = elem_nodes
    else:
        elem_dofs = (elem_nodes[:, :, None] * ndn + np.arange(ndn)[None, None, :]).reshape(
            elem_nodes.shape[0], -1)
    elem_dofs = elem_dofs.astype(np.int32)
    dirichlet = np.repeat(dir_nodes_mask.astype(np.uint8), ndn)
    g = np.repeat(dir_values, ndn) if dir_values is not None else np.zeros(n)
    g = np.where(dirichlet > 0, g, 0.0)
    a_full = _assemble(elem_dofs, elem_mats, n)
    # load vector
    k = elem_dofs.shape[1]
    f = np.zeros(n)
    np.add.at(f, elem_dofs.ravel(), np.broadcast_to(load, (elem_dofs.shape[0], k)).ravel())
    # lifting of non-homogeneous Dirichlet values, then symmetric elimination
    b = f - a_full @ g
    b = np.where(dirichlet > 0, g, b)
    # Eliminate in place so that A keeps the full element pattern (explicit
    # zeros included): every element coupling (k, l) has a slot in A.
    a = a_full
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(a.indptr))
    cols = a.indices.astype(np.int64)
    hit = (dirichlet[rows] > 0) | (dirichlet[cols] > 0)
    a.data[hit] = 0.0
    a.data[hit & (rows == cols)] = 1.0
    a.indptr = a.indptr.astype(np.int64)
    a.indices = a.indices.astype(np.int32)
    # partition
    if cores is None:
        cores, grown = box_partition(nel, parts, overlap)
    else:
        ovs = overlaps if overlaps is not None else [overlap] * len(cores)
        grown = [(tuple(max(0, lo[d] - o) for d in range(dim)),
                  tuple(min(nel[d], hi[d] + o) for d in range(dim))) for (lo, hi), o in zip(cores, ovs)]
    estrides = [1, nel[0], nel[0] * (nel[1] if dim > 1 else 1)]
    nstrides = [1, nn[0], nn[0] * (nn[1] if dim > 1 else 1)]
    se_ptr, se, sd_ptr, sdv = [0], [], [0], []
    for lo, hi in grown:
        el = _box_ids(lo, hi, estrides)
        se.append(el)
        se_ptr.append(se_ptr[-1] + el.size)
        nodes = _box_ids(lo, tuple(v + 1 for v in hi), nstrides)
        dofs = (nodes[:, None] * ndn + np.arange(ndn)[None, :]).ravel()
        dofs = dofs[dirichlet[dofs] == 0]
        sdv.append(np.sort(dofs))
        sd_ptr.append(sd_ptr[-1] + dofs.size)
    return Problem(
        dim=dim, nel=tuple(nel), ndn=ndn, n=n, elem_dofs=elem_dofs,
        elem_mats=np.ascontiguousarray(elem_mats), dirichlet=dirichlet, A=a, b=b,
        sub_elem_ptr=np.array(se_ptr, dtype=np.int64), sub_elem=np.concatenate(se).astype(np.int32),
        sub_dof_ptr=np.array(sd_ptr, dtype=np.int64), sub_dof=np.concatenate(sdv).astype(np.int32),
        boxes_core=cores, boxes_grown=grown, overlap=overlap, h=h, coeff=coeff, name=name)


def _boundary_node_mask(nel, faces):
    """Mask of nodes on the requested faces; faces = list of (dim, side)."""
    dim = len(nel)
    nn = [v + 1 for v in nel]
    idx = np.meshgrid(*[np.arange(v) for v in nn[::-1]], indexing="ij")
    idx = [idx[dim - 1 - d].ravel() for d in range(dim)]
    mask = np.zeros(idx[0].size, dtype=bool)
    for d, side in faces:
        mask |= idx[d] == (0 if side == 0 else nel[d])
    return mask, idx


def darcy_problem(nel, kappa, parts, overlap, dirichlet="all", f=1.0, name="darcy", cores=None,
                  overlaps=None):
    """Q1 Darcy -div(kappa grad u) = f on the unit square/cube (Section 2, eq. 2).

    ``kappa``: per-element coefficient, shape ``nel`` (x fastest in the flat
    order).  ``dirichlet``: "all" (u = 0 on the whole boundary) or
    "top1_bottom0" (u = 1 on the top face y = 1 (2D) / z = 1 (3D), u = 0 on the
    bottom face, natural conditions elsewhere).
    """
    nel = tuple(int(v) for v in nel)
    dim = len(nel)
    h = 1.0 / nel[0]
    kflat = np.asarray(kappa, dtype=np.float64).reshape(-1)
    assert kflat.size == int(np.prod(nel))
    kref = q1_reference_stiffness(dim, h)
    elem_nodes = structured_mesh(nel)
    elem_mats = kflat[:, None, None] * kref[None, :, :]
    load = f * q1_reference_load(dim, h)
    if dirichlet == "all":
        mask, _ = _boundary_node_mask(nel, [(d, s) for d in range(dim) for s in (0, 1)])
        vals = np.zeros(mask.size)
    elif dirichlet == "top1_bottom0":
        top = dim - 1
        mask, idx = _boundary_node_mask(nel, [(top, 0), (top, 1)])
        vals = np.where(idx[top] == nel[top], 1.0, 0.0)
    else:
        raise ValueError(dirichlet)
    return _finish(dim, nel, 1, elem_nodes, elem_mats, load, mask, vals, parts, overlap, h,
                   kflat, name, cores, overlaps)


def uneven_darcy_problem(nel, n_parts, min_side, max_side, seed=3, contrast_range=(1e4, 1e8),
                         overlap_range=(1, 3), name="uneven"):
    """3D Darcy on an irregular k-d box partition with per-box overlap drawn
    from overlap_range and, per box, one inclusion of log-uniform contrast in
    contrast_range (uneven subdomain sizes for batching)."""
    rng = np.random.default_rng(seed)
    cores = kd_partition(nel, n_parts, min_side, max_side, seed)
    overlaps = [int(rng.integers(overlap_range[0], overlap_range[1] + 1)) for _ in cores]
    kap = np.ones(nel[::-1])
    for lo, hi in cores:
        c = 10.0 ** rng.uniform(np.log10(contrast_range[0]), np.log10(contrast_range[1]))
        a = [int(rng.integers(lo[d], max(lo[d] + 1, hi[d] - 1))) for d in range(3)]
        b = [min(hi[d], a[d] + int(rng.integers(1, max(2, (hi[d] - lo[d]) // 2)))) for d in range(3)]
        kap[a[2]:b[2], a[1]:b[1], a[0]:b[0]] = c
    return darcy_problem(nel, kap, None, None, cores=cores, overlaps=overlaps, name=name)


def elasticity_problem(nel, parts, overlap, layer_thickness=2, body_force=(0.0, 0.0, -1.0),
                       name="laminate", seed=None):
    """Q1 hexahedral linear elasticity of a fibre/resin laminate (Section 2, eq. 3).

    Domain [0, nx*h] x [0, ny*h] x [0, nz*h] with h = 1/nz.  Layers of
    ``layer_thickness`` elements in z alternate fibre (orthotropic, E1 = 135,
    E2 = E3 = 10, nu12 = nu13 = 0.3, nu23 = 0.4, G12 = G13 = 5,
    G23 = E2/(2(1+nu23)), units GPa) and resin (isotropic E = 3, nu = 0.35);
    successive fibre layers turn by 90 degrees about z.  Clamped at x = 0.
    With a seed the laminate is a random sample: each fibre layer's
    orientation (0 or 90 degrees) is drawn, and each resin layer's modulus is
    scaled by a log-uniform factor in [1/2, 2] (SplitMix64 stream).
    """
    nel = tuple(int(v) for v in nel)
    assert len(nel) == 3
    h = 1.0 / nel[2]
    fib = orthotropic_stiffness(135.0, 10.0, 10.0, 0.3, 0.3, 0.4, 5.0, 5.0, 10.0 / (2 * 1.4))
    res = isotropic_stiffness(3.0, 0.35)
    k_fib0 = q1_elasticity_element(fib, h)
    k_fib90 = q1_elasticity_element(rotate_voigt_z90(fib), h)
    k_res = q1_elasticity_element(res, h)
    elem_nodes = structured_mesh(nel)
    ez = np.arange(elem_nodes.shape[0]) // (nel[0] * nel[1])
    layer = ez // layer_thickness
    kind = np.where(layer % 2 == 1, 0, np.where((layer // 2) % 2 == 0, 1, 2))  # 0 resin, 1/2 fibre
    table = np.stack([k_res, k_fib0, k_fib90])
    if seed is None:
        elem_mats = table[kind]
    else:
        nl = int(layer.max()) + 1
        u = splitmix64(np.arange(2 * nl, dtype=np.uint64) + np.uint64(seed << 20)).astype(np.float64) / 2.0 ** 64
        orient = np.where(u[:nl] < 0.5, 1, 2)
        scale = 2.0 ** (2.0 * u[nl:] - 1.0)
        kind = np.where(layer % 2 == 1, 0, orient[layer])
        elem_mats = table[kind] * np.where(kind == 0, scale[layer], 1.0)[:, None, None]
    load = np.zeros(24)
    load[2::3] = body_force[2] * h ** 3 / 8
    load[0::3] = body_force[0] * h ** 3 / 8
    load[1::3] = body_force[1] * h ** 3 / 8
    mask, _ = _boundary_node_mask(nel, [(0, 0)])
    return _finish(3, nel, 3, elem_nodes, elem_mats, load, mask, np.zeros(mask.size), parts,
                   overlap, h, kind.astype(np.float64), name)


# ----------------------------------------------------------------------------
# Coefficient fields (all seeded).
# ----------------------------------------------------------------------------
def kappa_channels_2d(nel, seed=0, contrast=1e6, n_channels=4, n_incl=8):
    """kappa = 1 background with horizontal channels (1 element high, 48..60
    long) and rectangular inclusions (2..6 elements per side), kappa = contrast.
    Returns shape (ny, nx) (row = y)."""
    nx, ny = nel
    rng = np.random.default_rng(seed)
    k = np.ones((ny, nx))
    for _ in range(n_channels):
        length = int(rng.integers(min(48, nx), min(60, nx) + 1))
        y = int(rng.integers(1, ny - 1))
        x0 = int(rng.integers(0, nx - length + 1))
        k[y, x0:x0 + length] = contrast
    for _ in range(n_incl):
        wx, wy = (int(v) for v in rng.integers(2, 7, size=2))
        x0 = int(rng.integers(0, nx - wx + 1))
        y0 = int(rng.integers(0, ny - wy + 1))
        k[y0:y0 + wy, x0:x0 + wx] = contrast
    return k


def kappa_skyscrapers_2d(nel, contrast, seed=0, n_sky=24):
    """High-contrast 'skyscrapers' (tall thin inclusions) and channels, seeded."""
    nx, ny = nel
    rng = np.random.default_rng(seed)
    k = np.ones((ny, nx))
    for _ in range(n_sky):
        w = max(1, nx // 80)
        hgt = int(rng.integers(ny // 8, ny // 2))
        x0 = int(rng.integers(0, nx - w))
        y0 = int(rng.integers(0, ny - hgt))
        k[y0:y0 + hgt, x0:x0 + w] = contrast
    for _ in range(4):
        y = int(rng.integers(1, ny - 1))
        k[y:y + max(1, ny // 160), :] = contrast
    return k


def kappa_layers_2d(nel, contrast, n_layers=40):
    """n_layers horizontal layers of equal thickness alternating 1 / contrast."""
    nx, ny = nel
    y = np.arange(ny)
    lay = (y * n_layers) // ny
    col = np.where(lay % 2 == 1, contrast, 1.0)
    return np.repeat(col[:, None], nx, axis=1)


def gaussian_random_field(nel, corr_len, variance, seed):
    """Stationary Gaussian field with covariance variance*exp(-r/corr_len) at
    element centroids of the unit cube, by circulant embedding on a grid padded
    to twice the size (negative embedding eigenvalues clipped to zero).
    Returns a float64 array of shape nel[::-1] (z, y, x)."""
    dim = len(nel)
    m = [2 * v for v in nel]
    h = 1.0 / nel[0]
    axes = [np.minimum(np.arange(mm), mm - np.arange(mm)) * h for mm in m[::-1]]
    grids = np.meshgrid(*axes, indexing="ij")
    r = np.sqrt(sum(g * g for g in grids))
    c = variance * np.exp(-r / corr_len)
    lam = np.fft.fftn(c).real
    lam = np.maximum(lam, 0.0)
    rng = np.random.default_rng(seed)
    xi = rng.standard_normal(lam.shape) + 1j * rng.standard_normal(lam.shape)
    field = np.fft.fftn(np.sqrt(lam / lam.size) * xi).real
    sl = tuple(slice(0, v) for v in nel[::-1])
    return np.ascontiguousarray(field[sl])


def kappa_grf_layers_3d(nel, seed=1, corr_len=0.1, variance=4.0, contrast=1e6,
                        slab_z=(24, 56, 88, 120), slab_thickness=2):
    """kappa = exp(g) (g a Gaussian field as above) times ``contrast`` in
    horizontal slabs ``slab_thickness`` elements thick starting at the z
    element indices ``slab_z`` (scaled to the grid when nz != 128)."""
    g = gaussian_random_field(nel, corr_len, variance, seed)
    k = np.exp(g)
    nz = nel[2]
    for z0 in slab_z:
        z = (z0 * nz) // 128
        k[z:z + slab_thickness] *= contrast
    return k
