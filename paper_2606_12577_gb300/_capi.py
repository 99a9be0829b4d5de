"""ctypes declarations of the C ABI in include/cascade_mg.h.

Argument marshalling only: every computation happens in libcascade_mg.so.
Loading fails with an exception when the library has not been built; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libcascade_mg.so")

CS_OK, CS_ERR_ARG, CS_ERR_CUDA, CS_ERR_NOMEM, CS_ERR_SINGULAR = 0, -1, -2, -3, -4
CS_ERR_DIVERGED, CS_ERR_TIMEOUT, CS_ERR_UNSUPPORTED, CS_ERR_NOTCONV = -5, -6, -7, -8
STATUS_NAMES = {0: "CS_OK", -1: "CS_ERR_ARG", -2: "CS_ERR_CUDA", -3: "CS_ERR_NOMEM", -4: "CS_ERR_SINGULAR",
                -5: "CS_ERR_DIVERGED", -6: "CS_ERR_TIMEOUT", -7: "CS_ERR_UNSUPPORTED", -8: "CS_ERR_NOTCONV"}
CS_ADDITIVE, CS_MULTIPLICATIVE = 0, 1
CS_FP64, CS_FP32, CS_BF16 = 0, 1, 2
CS_FF, CS_RF = 0, 1
CS_STATIONARY, CS_GMRES, CS_REFINE, CS_GMRES_RIGHT, CS_PCG = 0, 1, 2, 3, 4
PRESCALE = {"none": 0, "elliptic": 1, "stokes1": 2, "stokes2": 3, "stokesinf": 4, False: 0, True: 1}


class cs_stencil(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("nst", C.c_int), ("off", (C.c_int * 3) * 27),
                ("coeff", C.c_void_p), ("coeff_on_host", C.c_int), ("periodic", C.c_int)]


class cs_hierarchy_opts(C.Structure):
    _fields_ = [("coarse_max", C.c_int), ("max_levels", C.c_int), ("block", C.c_int), ("no_reuse", C.c_int)]


class cs_cascade_opts(C.Structure):
    _fields_ = [("kind", C.c_int), ("nu", C.c_int), ("prescale", C.c_int), ("alpha", C.c_int), ("lowp", C.c_int),
                ("no_reuse", C.c_int), ("model", C.c_void_p), ("model_tol", C.c_double), ("setup_precision", C.c_int),
                ("sketch", C.c_int), ("sketch_exact_first", C.c_int), ("sketch_seed", C.c_uint64)]


class cs_vcycle_opts(C.Structure):
    _fields_ = [("mu_pre", C.c_int), ("mu_post", C.c_int), ("order", C.c_int), ("precision", C.c_int)]


class cs_solve_opts(C.Structure):
    _fields_ = [("method", C.c_int), ("restart", C.c_int), ("maxit", C.c_int), ("tol", C.c_double),
                ("cycle", cs_vcycle_opts), ("host_buffers", C.c_int), ("hist", C.POINTER(C.c_double)),
                ("hist_cap", C.c_int)]


class cs_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("final_rel_residual", C.c_double),
                ("nhist", C.c_int)]


class cs_level_info(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("N", C.c_int64), ("nst", C.c_int),
                ("off", (C.c_int * 3) * 27), ("nlevels", C.c_int), ("block", C.c_int), ("lamsize", C.c_int64),
                ("sym32", C.c_int)]


class cs_csr(C.Structure):
    _fields_ = [("n", C.c_int), ("m", C.c_int), ("rowptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p),
                ("on_host", C.c_int)]


class cs_batch_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("order", C.c_int), ("mu_pre", C.c_int), ("mu_post", C.c_int),
                ("autotune", C.c_int), ("threads", C.c_int), ("tiles_per_cta", C.c_int), ("method", C.c_int),
                ("restart", C.c_int)]


class cs_batch_tune(C.Structure):
    _fields_ = [("threads", C.c_int), ("tiles_per_cta", C.c_int), ("ms", C.c_float)]


_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "cs_setup_hierarchy": (C.c_int, [C.POINTER(cs_stencil), C.POINTER(cs_hierarchy_opts), C.c_void_p,
                                     C.POINTER(C.c_void_p)]),
    "cs_setup_cascade": (C.c_int, [C.c_void_p, C.POINTER(cs_cascade_opts), C.c_void_p, C.POINTER(C.c_void_p)]),
    "cs_vcycle": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(cs_vcycle_opts), C.c_void_p, C.c_void_p, C.c_void_p]),
    "cs_smooth": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cs_sweep": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                           C.c_void_p, C.c_void_p]),
    "cs_kernel_launches": (C.c_int64, []),
    "cs_sweep_rhs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                               C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cs_smooth_noalloc": (C.c_int, [C.c_int, C.POINTER(C.c_int), C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                    C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cs_residual_restrict": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cs_prolong_correct": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cs_residual_restrict_lowp": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.c_void_p]),
    "cs_prolong_correct_lowp": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                          C.c_void_p]),
    "cs_coarse_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cs_gsetup_hierarchy": (C.c_int, [C.POINTER(cs_csr), C.c_int, C.POINTER(cs_csr), C.c_double, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p,
                                      C.POINTER(C.c_void_p)]),
    "cs_tc_gemm_bf16": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cs_gsetup_cascade": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                    C.POINTER(C.c_void_p)]),
    "cs_gsweep": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                            C.c_void_p]),
    "cs_gsmooth": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cs_gvcycle": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(cs_vcycle_opts), C.c_void_p, C.c_void_p, C.c_void_p]),
    "cs_gsolve": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(cs_solve_opts), C.c_void_p, C.c_void_p,
                            C.POINTER(cs_solve_info), C.c_void_p]),
    "cs_gquery_level": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.c_int),
                                  C.POINTER(C.c_int)]),
    "cs_gnlevels": (C.c_int, [C.c_void_p]),
    "cs_gexport_operator": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cs_gexport_colours": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "cs_gexport_blocks": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "cs_glamsize": (C.c_int64, [C.c_void_p, C.c_int]),
    "cs_gexport_lambda": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "cs_gdestroy_hierarchy": (None, [C.c_void_p]),
    "cs_gdestroy_cascade": (None, [C.c_void_p]),
    "cs_residual": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                              C.c_void_p]),
    "cs_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(cs_solve_opts), C.c_void_p, C.c_void_p,
                           C.POINTER(cs_solve_info), C.c_void_p]),
    "cs_query_level": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(cs_level_info)]),
    "cs_export_operator": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "cs_export_colours": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "cs_export_lambda": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "cs_hierarchy_bytes": (C.c_int64, [C.c_void_p]),
    "cs_cascade_bytes": (C.c_int64, [C.c_void_p]),
    "cs_mlp_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64, C.POINTER(C.c_void_p)]),
    "cs_mlp_destroy": (None, [C.c_void_p]),
    "cs_mlp_nparam": (C.c_int64, [C.c_void_p]),
    "cs_mlp_get_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "cs_mlp_set_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "cs_mlp_forward": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "cs_mlp_gradients": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.POINTER(C.c_float), C.c_void_p]),
    "cs_mlp_train_step": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_float, C.POINTER(C.c_float),
                                    C.c_void_p]),
    "cs_block_features": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "cs_block_targets": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "cs_learned_status": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "cs_learned_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                   C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "cs_setup_many": (C.c_int, [C.c_int, C.POINTER(cs_stencil), C.POINTER(cs_hierarchy_opts),
                                C.POINTER(cs_cascade_opts), C.c_int, C.c_void_p, C.POINTER(C.c_void_p),
                                C.POINTER(C.c_void_p)]),
    "cs_batch_create": (C.c_int, [C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_int),
                                  C.POINTER(cs_batch_opts), C.c_void_p, C.POINTER(C.c_void_p)]),
    "cs_batch_solve": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_double, C.c_int,
                                 C.POINTER(cs_solve_info), C.c_void_p]),
    "cs_batch_config": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int),
                                  C.POINTER(cs_batch_tune), C.c_int, C.POINTER(C.c_int)]),
    "cs_batch_set_config": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "cs_batch_bytes": (C.c_int64, [C.c_void_p]),
    "cs_batch_destroy": (None, [C.c_void_p]),
    "cs_solve_batched": (C.c_int, [C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(cs_solve_opts),
                                   C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_int),
                                   C.POINTER(cs_solve_info), C.c_void_p]),
    "cs_last_error": (C.c_char_p, []),
    "cs_destroy_hierarchy": (None, [C.c_void_p]),
    "cs_destroy_cascade": (None, [C.c_void_p]),
}

EXPORTED = tuple(_SIGS)


def lib():
    """Load libcascade_mg.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


class CascadeError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int, where: str):
    if status != CS_OK:
        raise CascadeError(status, where, lib().cs_last_error().decode(errors="replace"))
