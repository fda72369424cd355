"""The C ABI library builds, loads and exports every entry point declared in
include/geneo.h; host-only entry points work without a GPU."""
import os
import re

import numpy as np

import gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "geneo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(geneo_[a-z_]+)\s*\(", src)))


def _lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1906_10944_gb300 import geneo
    return geneo, geneo.load_library()


def test_every_declared_symbol_is_exported():
    geneo, lib = _lib()
    names = _declared()
    assert len(names) >= 12
    for nm in names:
        assert hasattr(lib, nm), nm
    assert sorted(geneo.EXPORTED) == names


def test_status_strings_and_defaults():
    geneo, _ = _lib()
    assert geneo.geneo_status_str(0) == "ok"
    assert "pivot" in geneo.geneo_status_str(3)
    o = geneo.geneo_default_options()
    assert (o.tau, o.sigma, o.nev_max, o.eig_tol) == (0.3, -0.01, 10, 1e-6)


def test_setup_rejects_bad_arguments_without_gpu():
    import ctypes as C
    geneo, lib = _lib()
    h = C.c_void_p()
    p = geneo.geneo_problem_t()          # all zero: n = 0
    o = geneo.geneo_default_options()
    assert lib.geneo_setup(C.byref(p), C.byref(o), None, C.byref(h)) == 1
    assert lib.geneo_setup(None, C.byref(o), None, C.byref(h)) == 1
    assert not h.value


def test_grow_partition_matches_box_growth():
    """geneo_grow_partition (vertex-neighbour layers, Section 3) reproduces
    the box partition grown by whole element layers, 2D and 3D."""
    geneo, _ = _lib()
    for nel, parts, ov in [((16, 12), (4, 3), 2), ((8, 6, 6), (2, 3, 2), 1)]:
        kap = np.ones(nel[::-1])
        p0 = gen.darcy_problem(nel, kap, tuple([1] * len(nel)), 0)
        cores, _ = gen.box_partition(nel, parts, 0)
        part = np.zeros(p0.n_elem, dtype=np.int32)
        estr = [1, nel[0], nel[0] * nel[1]]
        for j, (lo, hi) in enumerate(cores):
            rng = [np.arange(lo[d], hi[d]) for d in range(len(nel))]
            g = np.meshgrid(*rng, indexing="ij")
            ids = sum(g[d].ravel() * estr[d] for d in range(len(nel)))
            part[ids] = j
        ep, el, dp, dl = geneo.geneo_grow_partition(p0.n, p0.elem_dofs, p0.dirichlet, part,
                                                     len(cores), ov)
        q = gen.darcy_problem(nel, kap, parts, ov)
        assert np.array_equal(ep, q.sub_elem_ptr) and np.array_equal(el, q.sub_elem)
        assert np.array_equal(dp, q.sub_dof_ptr) and np.array_equal(dl, q.sub_dof)


def test_option_limits_rejected_without_gpu():
    """Options outside the supported range return GENEO_ERR_ARG before any
    device work (nev_max > 34, sigma >= 0, unknown precision)."""
    import ctypes as C
    geneo, lib = _lib()
    p = gen.darcy_problem((4, 4), np.ones((4, 4)), (1, 1), 0)
    arrs = geneo.problem_arrays(p)
    prob = geneo.make_problem(arrs, p.n, p.n_sub, 4, 1, geneo.GENEO_MEM_HOST)
    for kw in ({"nev_max": 35}, {"sigma": 0.0}, {"precision": 7}, {"eig_form": 3}):
        o = geneo.geneo_default_options(**kw)
        h = C.c_void_p()
        assert lib.geneo_setup(C.byref(prob), C.byref(o), None, C.byref(h)) == 1, kw


def test_binding_struct_layouts_match_the_library():
    import ctypes
    geneo, _ = _lib()
    sizes = geneo.geneo_struct_sizes()
    assert sizes == [ctypes.sizeof(geneo.geneo_problem_t), ctypes.sizeof(geneo.geneo_options_t),
                     ctypes.sizeof(geneo.geneo_solve_info_t), ctypes.sizeof(geneo.geneo_coarse_info_t)]
    o = geneo.geneo_default_options()
    assert (o.first_nev, o.guard, o.fp32_pivot_tol, o.precision) == (-1, -1, 1e-4, geneo.GENEO_PREC_FP64)
