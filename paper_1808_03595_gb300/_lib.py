"""ctypes declarations of the semmg C ABI (include/semmg.h).

Loading fails loudly when libsemmg.so has not been built: there is no CPU or
Python fallback for any entry point.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsemmg.so")

c_int, c_double, c_void_p, c_int64 = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64
P_double = ctypes.POINTER(ctypes.c_double)

SEMMG_OK = 0
ERRORS = {
    -1: "SEMMG_ERR_INVALID_ARG",
    -2: "SEMMG_ERR_UNSUPPORTED",
    -3: "SEMMG_ERR_CUDA",
    -4: "SEMMG_ERR_NOT_CONVERGED",
    -5: "SEMMG_ERR_NONFINITE",
    -6: "SEMMG_ERR_TIMEOUT",
    -7: "SEMMG_ERR_NOMEM",
    -8: "SEMMG_ERR_DIVERGED",
}
SEMMG_ERR_NOT_CONVERGED, SEMMG_ERR_NONFINITE, SEMMG_ERR_TIMEOUT, SEMMG_ERR_DIVERGED = -4, -5, -6, -8
SEMMG_FP64, SEMMG_MIXED, SEMMG_MIXED_FP32, SEMMG_MIXED_TC, SEMMG_MIXED_FP32_TC, SEMMG_MIXED_BF16 = 0, 1, 2, 3, 4, 5
SEMMG_MIXED_FF, SEMMG_MIXED_FF_TC = 6, 7
SEMMG_SOLVER_MG, SEMMG_SOLVER_KMG = 0, 1
SEMMG_SMOOTHER_STAR, SEMMG_SMOOTHER_ELEMENT, SEMMG_SMOOTHER_ELEMENT_MULT = 0, 1, 2
SEMMG_BC_DIRICHLET, SEMMG_BC_NEUMANN, SEMMG_BC_PERIODIC = 0, 1, 2
SEMMG_F64, SEMMG_F32 = 0, 1
SEMMG_NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024


class semmg_mesh(ctypes.Structure):
    _fields_ = [("n", c_int * 3), ("h", P_double * 3), ("bc", c_int * 6)]


class semmg_opts(ctypes.Structure):
    _fields_ = [("p0", c_int), ("nu_pre", c_int), ("nu_post", c_int), ("precision", c_int), ("max_iter", c_int),
                ("solver", c_int), ("nu_vary", c_int), ("smoother", c_int)]


class semmg_kstat(ctypes.Structure):
    _fields_ = [("ms", c_double), ("launches", c_int64), ("flops", c_double), ("bytes", c_double),
                ("xflops", c_double)]


KSTAT_KINDS = ["star", "star_gather", "elem_schur", "assemble", "transfer", "coarse", "condense", "recover",
               "vector"]


class semmg_info(ctypes.Structure):
    _fields_ = [("iters", c_int), ("res0", c_double), ("res_final", c_double), ("rho", c_double), ("status", c_int)]


# name -> (restype, argtypes); every function declared in include/semmg.h
SIGNATURES = {
    "semmg_default_opts": (None, [ctypes.POINTER(semmg_opts)]),
    "semmg_setup": (c_int, [ctypes.POINTER(semmg_mesh), c_int, c_double, ctypes.POINTER(semmg_opts), c_void_p,
                            ctypes.POINTER(c_void_p)]),
    "semmg_destroy": (None, [c_void_p]),
    "semmg_num_levels": (c_int, [c_void_p, ctypes.POINTER(c_int)]),
    "semmg_level_degree": (c_int, [c_void_p, c_int, ctypes.POINTER(c_int)]),
    "semmg_condensed_size": (c_int, [c_void_p, c_int, ctypes.POINTER(c_int64)]),
    "semmg_nodal_size": (c_int, [c_void_p, c_int, ctypes.POINTER(c_int64)]),
    "semmg_pack": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "semmg_unpack": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "semmg_pack_dirichlet": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "semmg_apply_condensed": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p]),
    "semmg_residual": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "semmg_residual_cycle": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "semmg_smooth": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "semmg_restrict": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "semmg_prolong_add": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "semmg_coarse_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "semmg_vcycle": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "semmg_condense_rhs": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "semmg_recover": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "semmg_solve": (c_int, [c_void_p, c_void_p, c_void_p, c_double, ctypes.POINTER(semmg_info), c_void_p]),
    "semmg_solve_dirichlet": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_double, ctypes.POINTER(semmg_info),
                                      c_void_p]),
    "semmg_solve_host": (c_int, [c_void_p, c_void_p, c_void_p, c_double, ctypes.POINTER(semmg_info), c_void_p]),
    "semmg_smooth_noalloc": (c_int, [c_void_p, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "semmg_batch_create": (c_int, [ctypes.POINTER(c_void_p), c_int, ctypes.POINTER(c_void_p),
                                   ctypes.POINTER(c_void_p), c_double, c_void_p, ctypes.POINTER(c_void_p)]),
    "semmg_batch_create_dirichlet": (c_int, [ctypes.POINTER(c_void_p), c_int, ctypes.POINTER(c_void_p),
                                             ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p), c_double, c_void_p,
                                             ctypes.POINTER(c_void_p)]),
    "semmg_batch_solve": (c_int, [c_void_p, ctypes.POINTER(semmg_info), c_void_p]),
    "semmg_batch_graph_nodes": (c_int, [c_void_p, ctypes.POINTER(c_int64)]),
    "semmg_batch_destroy": (None, [c_void_p]),
    "semmg_autotune": (c_int, [c_void_p, c_void_p]),
    "semmg_get_launch": (c_int, [c_void_p, c_int, c_int, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                 ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    "semmg_set_launch": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, c_int]),
    "semmg_set_timing": (c_int, [c_void_p, c_int]),
    "semmg_get_kstat": (c_int, [c_void_p, c_int, ctypes.POINTER(semmg_kstat)]),
    "semmg_reset_kstats": (c_int, [c_void_p]),
    "semmg_set_guards": (c_int, [c_void_p, c_double, ctypes.c_longlong]),
    "semmg_peak_tflops": (c_int, [c_int, ctypes.POINTER(c_double), c_void_p]),
    "semmg_strerror": (ctypes.c_char_p, [c_int]),
    "semmg_last_error": (ctypes.c_char_p, [c_void_p]),
}

_lib = None


def load(path=LIB_PATH):
    """Load libsemmg.so and declare every entry point; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1808_03595_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
