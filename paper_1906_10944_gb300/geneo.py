"""ctypes binding of libgeneo (the C ABI declared in include/geneo.h).

Argument marshalling only: every numeric step runs in the CUDA library.  The
functions carry the C names; ``GenEO`` is a small convenience wrapper that
keeps the device copies of a problem alive and owns the handle.  PyTorch is
used for device memory and streams.  There is no fallback: if the library is
missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgeneo.so")

GENEO_MEM_HOST = 0
GENEO_MEM_DEVICE = 1
GENEO_EIG_PAPER = 0
GENEO_EIG_FULL = 1
GENEO_PREC_FP64 = 0
GENEO_PREC_FP32 = 1
GENEO_PU_STANDARD = 0
GENEO_PU_SARKIS = 1

PROF_FAMILIES = ["factor", "eig_solve", "gram", "spmm", "gemm", "small_eig", "local_solve",
                 "coarse_solve", "spmv", "other", "ortho32"]
NPROF = len(PROF_FAMILIES)  # GENEO_PROF_COUNT

STATUS = {
    0: "GENEO_OK", 1: "GENEO_ERR_ARG", 2: "GENEO_ERR_OOM", 3: "GENEO_ERR_NOT_SPD",
    4: "GENEO_ERR_EIG_NOCONV", 5: "GENEO_ERR_PCG_NOCONV", 6: "GENEO_ERR_BREAKDOWN",
    7: "GENEO_ERR_CUDA", 8: "GENEO_ERR_TIMEOUT", 9: "GENEO_ERR_NONFINITE",
}

EXPORTED = [
    "geneo_default_options", "geneo_setup", "geneo_apply", "geneo_pcg_solve", "geneo_query",
    "geneo_get_subdomain", "geneo_grow_partition", "geneo_free_host", "geneo_destroy",
    "geneo_status_str", "geneo_last_error", "geneo_launch_count", "geneo_pcg_solve_noalloc",
    "geneo_struct_sizes",
]


class geneo_problem_t(C.Structure):
    _fields_ = [
        ("mem", C.c_int32), ("ndof_node", C.c_int32), ("n", C.c_int64), ("nnz", C.c_int64),
        ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p), ("dirichlet", C.c_void_p),
        ("n_elem", C.c_int64), ("elem_ndof", C.c_int32), ("n_sub", C.c_int32),
        ("elem_dofs", C.c_void_p), ("elem_mats", C.c_void_p), ("sub_elem_ptr", C.c_void_p),
        ("sub_elem", C.c_void_p), ("sub_dof_ptr", C.c_void_p), ("sub_dof", C.c_void_p),
        ("pu_weights", C.c_void_p),
    ]


class geneo_options_t(C.Structure):
    _fields_ = [
        ("tau", C.c_double), ("sigma", C.c_double), ("eig_tol", C.c_double),
        ("nev_max", C.c_int32), ("fixed_nev", C.c_int32), ("eig_form", C.c_int32),
        ("eig_maxit", C.c_int32), ("guard", C.c_int32), ("precision", C.c_int32),
        ("profile", C.c_int32), ("first_nev", C.c_int32), ("seed", C.c_uint64),
        ("fp32_pivot_tol", C.c_double), ("pu_kind", C.c_int32), ("eig_strict", C.c_int32),
        ("deterministic", C.c_int32), ("eig_solve_tf32", C.c_int32),
        ("factor_kernel", C.c_int32), ("autotune", C.c_int32),
        ("factor_bf16", C.c_int32), ("reserved", C.c_int32),
    ]


class geneo_solve_info_t(C.Structure):
    _fields_ = [
        ("iterations", C.c_int32), ("converged", C.c_int32), ("rel_residual", C.c_double),
        ("kappa_estimate", C.c_double), ("resid_hist", C.POINTER(C.c_double)),
        ("resid_hist_cap", C.c_int32), ("resid_hist_len", C.c_int32),
        ("true_residual", C.c_double), ("replacements", C.c_int32), ("reserved", C.c_int32),
    ]


class geneo_coarse_info_t(C.Structure):
    _fields_ = [
        ("n_sub", C.c_int32), ("dim_coarse", C.c_int32), ("coarse_bandwidth", C.c_int32),
        ("eig_iterations", C.c_int32), ("block_size", C.c_int32),
        ("fp64_factors_K", C.c_int32), ("fp64_factors_A", C.c_int32), ("fp64_ortho", C.c_int32),
        ("eig_unconverged", C.c_int32), ("factor_classes", C.c_int32), ("device_bytes", C.c_int64),
        ("setup_ms", C.c_double * 8), ("factor_flops", C.c_double), ("factor_event_ms", C.c_double),
        ("eigsolve_flops", C.c_double), ("eigsolve_event_ms", C.c_double),
        ("apply_flops", C.c_double), ("apply_bytes", C.c_double),
        ("prof_ms", C.c_double * NPROF), ("prof_flops", C.c_double * NPROF),
        ("prof_bytes", C.c_double * NPROF), ("prof_launches", C.c_int64 * NPROF),
        ("local_solve_stages", C.c_int32), ("reserved", C.c_int32),
    ]


class GenEOError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__("%s (%d)%s" % (STATUS.get(code, "unknown"), code, (": " + what) if what else ""))


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libgeneo.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libgeneo.so not built (%s); run __graft_entry__.build()" % path)
    lib = C.CDLL(path)
    P, I32, I64, D, VP = C.POINTER, C.c_int32, C.c_int64, C.c_double, C.c_void_p
    lib.geneo_default_options.argtypes = [P(geneo_options_t)]
    lib.geneo_default_options.restype = None
    lib.geneo_setup.argtypes = [P(geneo_problem_t), P(geneo_options_t), VP, P(VP)]
    lib.geneo_setup.restype = I32
    lib.geneo_apply.argtypes = [VP, VP, VP, I32, VP]
    lib.geneo_apply.restype = I32
    lib.geneo_pcg_solve.argtypes = [VP, VP, VP, I32, D, I32, I32, P(geneo_solve_info_t), VP]
    lib.geneo_pcg_solve.restype = I32
    lib.geneo_query.argtypes = [VP, P(geneo_coarse_info_t)]
    lib.geneo_query.restype = I32
    lib.geneo_get_subdomain.argtypes = [VP, I32, P(I32), P(I32), P(I32), P(I32), VP, I64, VP, I64,
                                        VP, I64, VP, I64]
    lib.geneo_get_subdomain.restype = I32
    lib.geneo_grow_partition.argtypes = [I64, I64, I32, VP, VP, VP, I32, I32, P(P(C.c_int64)),
                                         P(P(C.c_int32)), P(P(C.c_int64)), P(P(C.c_int32))]
    lib.geneo_grow_partition.restype = I32
    lib.geneo_free_host.argtypes = [VP]
    lib.geneo_free_host.restype = None
    lib.geneo_destroy.argtypes = [VP]
    lib.geneo_destroy.restype = None
    lib.geneo_status_str.argtypes = [I32]
    lib.geneo_status_str.restype = C.c_char_p
    lib.geneo_last_error.argtypes = [VP, P(I32), P(I32), P(I64)]
    lib.geneo_last_error.restype = I32
    lib.geneo_pcg_solve_noalloc.argtypes = [VP, VP, VP, D, I32, P(geneo_solve_info_t), VP]
    lib.geneo_pcg_solve_noalloc.restype = I32
    lib.geneo_struct_sizes.argtypes = [VP, I32]
    lib.geneo_struct_sizes.restype = I32
    lib.geneo_launch_count.argtypes = []
    lib.geneo_launch_count.restype = I64
    _lib = lib
    return lib


def _check(code, what=""):
    if code != 0:
        raise GenEOError(code, what)


def _ptr(a):
    """Raw address of a torch tensor or a C-contiguous numpy array."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    assert isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


# ---------------------------------------------------------------------------
# C-named entry points
# ---------------------------------------------------------------------------
def geneo_default_options(**overrides):
    lib = load_library()
    o = geneo_options_t()
    lib.geneo_default_options(C.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def geneo_setup(problem: geneo_problem_t, options: geneo_options_t, stream=None):
    lib = load_library()
    h = C.c_void_p()
    _check(lib.geneo_setup(C.byref(problem), C.byref(options), C.c_void_p(_stream(stream)), C.byref(h)),
           "geneo_setup")
    return h


def geneo_apply(h, r, z, nrhs=1, stream=None):
    lib = load_library()
    _check(lib.geneo_apply(h, _ptr(r), _ptr(z), nrhs, C.c_void_p(_stream(stream))), "geneo_apply")


def geneo_pcg_solve(h, b, x, nrhs=1, tol=1e-8, maxit=1000, mem=GENEO_MEM_DEVICE, hist_cap=0,
                    stream=None, raise_on_error=True):
    lib = load_library()
    info = geneo_solve_info_t()
    hist = None
    if hist_cap > 0:
        hist = (C.c_double * hist_cap)()
        info.resid_hist = C.cast(hist, C.POINTER(C.c_double))
        info.resid_hist_cap = hist_cap
    code = lib.geneo_pcg_solve(h, _ptr(b), _ptr(x), nrhs, tol, maxit, mem, C.byref(info),
                               C.c_void_p(_stream(stream)))
    if raise_on_error:
        _check(code, "geneo_pcg_solve")
    out = _info_dict(code, info)
    if hist is not None:
        out["resid_hist"] = np.array(hist[:min(info.resid_hist_len, hist_cap)])
    return out


def geneo_pcg_solve_noalloc(h, b, x, tol=1e-8, maxit=1000, stream=None, raise_on_error=True):
    """PCG without any allocation inside the call (device arrays only)."""
    lib = load_library()
    info = geneo_solve_info_t()
    code = lib.geneo_pcg_solve_noalloc(h, _ptr(b), _ptr(x), tol, maxit, C.byref(info),
                                       C.c_void_p(_stream(stream)))
    if raise_on_error:
        _check(code, "geneo_pcg_solve_noalloc")
    return _info_dict(code, info)


def _info_dict(code, info):
    return {"status": code, "iterations": info.iterations, "converged": bool(info.converged),
            "rel_residual": info.rel_residual, "true_residual": info.true_residual,
            "replacements": info.replacements, "kappa_estimate": info.kappa_estimate}


def geneo_query(h):
    lib = load_library()
    q = geneo_coarse_info_t()
    _check(lib.geneo_query(h, C.byref(q)), "geneo_query")
    return {"n_sub": q.n_sub, "dim_coarse": q.dim_coarse, "coarse_bandwidth": q.coarse_bandwidth,
            "eig_iterations": q.eig_iterations, "block_size": q.block_size,
            "fp64_factors_K": q.fp64_factors_K, "fp64_factors_A": q.fp64_factors_A,
            "fp64_ortho": q.fp64_ortho, "eig_unconverged": q.eig_unconverged,
            "factor_classes": q.factor_classes, "local_solve_stages": q.local_solve_stages,
            "device_bytes": q.device_bytes, "setup_ms": list(q.setup_ms),
            "factor_flops": q.factor_flops, "factor_event_ms": q.factor_event_ms,
            "eigsolve_flops": q.eigsolve_flops, "eigsolve_event_ms": q.eigsolve_event_ms,
            "apply_flops": q.apply_flops, "apply_bytes": q.apply_bytes,
            "prof": {name: {"ms": q.prof_ms[i], "flops": q.prof_flops[i], "bytes": q.prof_bytes[i],
                            "launches": q.prof_launches[i]} for i, name in enumerate(PROF_FAMILIES)}}


def geneo_get_subdomain(h, j):
    lib = load_library()
    nn, nd, m, s = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib.geneo_get_subdomain(h, j, C.byref(nn), C.byref(nd), C.byref(m), C.byref(s),
                                   None, 0, None, 0, None, 0, None, 0), "geneo_get_subdomain")
    dofs = np.zeros(nd.value, dtype=np.int32)
    pu = np.zeros(nn.value, dtype=np.float64)
    lam = np.zeros(s.value, dtype=np.float64)
    Z = np.zeros(nd.value * m.value, dtype=np.float64)
    _check(lib.geneo_get_subdomain(h, j, C.byref(nn), C.byref(nd), C.byref(m), C.byref(s),
                                   _ptr(dofs), dofs.size, _ptr(pu), pu.size, _ptr(lam), lam.size,
                                   _ptr(Z), Z.size), "geneo_get_subdomain")
    return {"D": dofs, "pu": pu, "lambda": lam, "m": m.value,
            "Z": Z.reshape(m.value, nd.value).T.copy()}


def geneo_grow_partition(n, elem_dofs, dirichlet, part, n_parts, overlap):
    lib = load_library()
    elem_dofs = np.ascontiguousarray(elem_dofs, dtype=np.int32)
    dirichlet = np.ascontiguousarray(dirichlet, dtype=np.uint8)
    part = np.ascontiguousarray(part, dtype=np.int32)
    sep, se = C.POINTER(C.c_int64)(), C.POINTER(C.c_int32)()
    sdp, sd = C.POINTER(C.c_int64)(), C.POINTER(C.c_int32)()
    _check(lib.geneo_grow_partition(n, elem_dofs.shape[0], elem_dofs.shape[1], _ptr(elem_dofs),
                                    _ptr(dirichlet), _ptr(part), n_parts, overlap, C.byref(sep),
                                    C.byref(se), C.byref(sdp), C.byref(sd)), "geneo_grow_partition")
    try:
        ep = np.ctypeslib.as_array(sep, shape=(n_parts + 1,)).copy()
        dp = np.ctypeslib.as_array(sdp, shape=(n_parts + 1,)).copy()
        el = np.ctypeslib.as_array(se, shape=(max(int(ep[-1]), 1),))[:ep[-1]].copy()
        dl = np.ctypeslib.as_array(sd, shape=(max(int(dp[-1]), 1),))[:dp[-1]].copy()
    finally:
        for p in (sep, se, sdp, sd):
            lib.geneo_free_host(C.cast(p, C.c_void_p))
    return ep, el, dp, dl


def geneo_destroy(h):
    if h:
        load_library().geneo_destroy(h)


def geneo_status_str(code):
    return load_library().geneo_status_str(code).decode()


def geneo_launch_count():
    return int(load_library().geneo_launch_count())


def geneo_last_error(h):
    c, w, i = C.c_int32(), C.c_int32(), C.c_int64()
    load_library().geneo_last_error(h, C.byref(c), C.byref(w), C.byref(i))
    return c.value, w.value, i.value


# ---------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------
def problem_arrays(prob):
    """The numpy arrays of a gen.Problem in the layout geneo_problem_t wants."""
    A = prob.A
    return {
        "row_ptr": np.ascontiguousarray(A.indptr, dtype=np.int64),
        "col": np.ascontiguousarray(A.indices, dtype=np.int32),
        "val": np.ascontiguousarray(A.data, dtype=np.float64),
        "dirichlet": np.ascontiguousarray(prob.dirichlet, dtype=np.uint8),
        "elem_dofs": np.ascontiguousarray(prob.elem_dofs, dtype=np.int32),
        "elem_mats": np.ascontiguousarray(prob.elem_mats, dtype=np.float64),
        "sub_elem_ptr": np.ascontiguousarray(prob.sub_elem_ptr, dtype=np.int64),
        "sub_elem": np.ascontiguousarray(prob.sub_elem, dtype=np.int32),
        "sub_dof_ptr": np.ascontiguousarray(prob.sub_dof_ptr, dtype=np.int64),
        "sub_dof": np.ascontiguousarray(prob.sub_dof, dtype=np.int32),
    }


def make_problem(arrays, n, n_sub, elem_ndof, ndof_node=1, mem=GENEO_MEM_DEVICE):
    p = geneo_problem_t()
    p.mem = mem
    p.ndof_node = ndof_node
    p.n = n
    p.nnz = int(arrays["col"].shape[0])
    p.n_elem = int(arrays["elem_dofs"].shape[0])
    p.elem_ndof = elem_ndof
    p.n_sub = n_sub
    for k in ("row_ptr", "col", "val", "dirichlet", "elem_dofs", "elem_mats", "sub_elem_ptr",
              "sub_elem", "sub_dof_ptr", "sub_dof"):
        setattr(p, k, _ptr(arrays[k]))
    p.pu_weights = _ptr(arrays.get("pu_weights"))
    return p


class GenEO:
    """Owns a handle; keeps the device copies of the inputs alive until close()."""

    def __init__(self, prob, device_arrays=None, stream=None, pu_weights=None, **opts):
        import torch
        load_library()
        host = problem_arrays(prob)
        if pu_weights is not None:
            host["pu_weights"] = np.ascontiguousarray(pu_weights, dtype=np.float64)
        if device_arrays is None:
            device_arrays = {k: torch.from_numpy(v).cuda() for k, v in host.items()}
        self.arrays = device_arrays
        self.n = prob.n
        self.problem = make_problem(device_arrays, prob.n, prob.n_sub, prob.elem_dofs.shape[1],
                                    prob.ndn, GENEO_MEM_DEVICE)
        self.options = geneo_default_options(**opts)
        self.stream = stream
        self.h = geneo_setup(self.problem, self.options, stream)

    def apply(self, r, z, nrhs=1):
        geneo_apply(self.h, r, z, nrhs, self.stream)

    def solve(self, b, x, tol=1e-8, maxit=1000, mem=GENEO_MEM_DEVICE, hist_cap=0, nrhs=1,
              raise_on_error=True):
        return geneo_pcg_solve(self.h, b, x, nrhs, tol, maxit, mem, hist_cap, self.stream,
                               raise_on_error)

    def query(self):
        return geneo_query(self.h)

    def subdomain(self, j):
        return geneo_get_subdomain(self.h, j)

    def close(self):
        if self.h:
            geneo_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def geneo_struct_sizes():
    """Struct sizes compiled into the library (problem, options, solve info,
    coarse info), for layout checks."""
    lib = load_library()
    out = np.zeros(4, dtype=np.int64)
    k = lib.geneo_struct_sizes(_ptr(out), 4)
    return [int(v) for v in out[:k]]
