"""ctypes prototypes of the C interface in include/nnmg.h (argument marshalling only)."""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnnmg.so")

OK, INVALID_ARG, BAD_MESH, POINT_NOT_FOUND, CHOLESKY_FAIL, OUT_OF_MEMORY, CUDA_ERROR, \
    NOT_CONVERGED, BREAKDOWN = range(9)
F32, F64, F64_DW = 0, 1, 2
FP64_MG, FP32_MG_FP64_CG, FP32_MG_DW_CG = 0, 1, 2
# columns of nnmg_vcycle_profile
PROF_COLUMNS = ("pre_smoother", "residual", "restrictor", "coarse_solver", "prolongator",
                "post_smoother", "operator", "vector")


class LevelDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_vertices", C.c_int64), ("vertices", C.c_void_p),
                ("n_cells", C.c_int64), ("cells", C.c_void_p), ("dirichlet_vertex", C.c_void_p),
                ("degree", C.c_int)]


class Options(C.Structure):
    _fields_ = [("degree", C.c_int), ("n_components", C.c_int), ("lam", C.c_double),
                ("mu", C.c_double), ("cheb_degree", C.c_int), ("smoothing_range", C.c_double),
                ("lanczos_steps", C.c_int), ("eig_safety", C.c_double), ("max_nrhs", C.c_int),
                ("deterministic", C.c_int)]


# name -> (restype, argtypes); every symbol declared in include/nnmg.h
PROTOTYPES = {
    "nnmg_default_options": (None, [C.POINTER(Options)]),
    "nnmg_setup_hierarchy": (C.c_int, [C.POINTER(LevelDesc), C.c_int, C.POINTER(Options),
                                       C.c_void_p, C.POINTER(C.c_void_p)]),
    "nnmg_destroy": (C.c_int, [C.c_void_p]),
    "nnmg_n_levels": (C.c_int, [C.c_void_p]),
    "nnmg_level_info": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int64),
                                  C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "nnmg_hierarchy_bytes": (C.c_size_t, [C.c_void_p]),
    "nnmg_solve_bytes": (C.c_size_t, [C.c_void_p, C.c_int]),
    "nnmg_estimate_bytes": (C.c_int, [C.POINTER(LevelDesc), C.c_int, C.POINTER(Options), C.c_int,
                                      C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "nnmg_support_points": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "nnmg_constrained_nodes": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "nnmg_cell_nodes": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "nnmg_color_cells": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int, C.c_void_p,
                                   C.POINTER(C.c_int)]),
    "nnmg_level_colors": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_int)]),
    "nnmg_quadrature_points": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "nnmg_transfer_points": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "nnmg_pcg_device_loop": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "nnmg_setup_seconds": (C.c_int, [C.c_void_p, C.c_void_p]),
    "nnmg_operator_choice": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "nnmg_eigen_estimates": (C.c_int, [C.c_void_p, C.c_void_p]),
    "nnmg_load_vector": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p,
                                   C.c_int, C.c_int, C.c_void_p]),
    "nnmg_apply_operator": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                      C.c_int, C.c_void_p]),
    "nnmg_prolongate": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                  C.c_int, C.c_void_p]),
    "nnmg_restrict": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                C.c_int, C.c_void_p]),
    "nnmg_restrict_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                        C.c_int, C.c_void_p]),
    "nnmg_vcycle": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                              C.c_void_p]),
    "nnmg_vcycle_profile": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                      C.c_void_p, C.c_void_p, C.c_void_p]),
    "nnmg_pcg_solve": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                 C.c_double, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "nnmg_pcg_solve_host": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                      C.c_double, C.c_int, C.c_void_p, C.c_void_p,
                                      C.c_void_p]),
    "nnmg_set_nested": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "nnmg_batch_reset": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_int, C.c_void_p]),
    "nnmg_batch_admit": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p]),
    "nnmg_batch_step": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "nnmg_batch_poll": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p]),
    "nnmg_batch_retire": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p]),
    "nnmg_batch_admit_cols": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int,
                                        C.c_void_p]),
    "nnmg_batch_repack": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "nnmg_pipe_rate": (C.c_int, [C.c_int, C.c_int, C.c_void_p, C.POINTER(C.c_double)]),
    "nnmg_last_error": (C.c_char_p, []),
}

_lib = None


def load():
    """Load libnnmg.so from the package directory; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                "libnnmg.so is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
