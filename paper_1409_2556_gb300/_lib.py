"""ctypes binding of the C ABI in include/lt.h (argument marshalling only).

Every computation runs in liblt.so; this module never falls back to Python
or CPU arithmetic.  Loading fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblt.so")

LT_OK = 0
LT_ERR_INVALID_ARG = -1
LT_ERR_OOM = -2
LT_ERR_CUDA = -3
LT_ERR_NOT_CONVERGED = -4
LT_ERR_TIMEOUT = -5
LT_ERR_STATE = -6

LT_BC_DIRICHLET = 0
LT_BC_NEUMANN = 1
LT_TAU_SINGLE = 0
LT_TAU_FLEXIBLE = 1
LT_PREC_FP64 = 0
LT_PREC_FP32 = 1
LT_KRYLOV_GMRES = 0
LT_KRYLOV_FOM = 1
LT_STOP_SHIFT = 0
LT_STOP_QUADRATURE = 1

# kernel classes (lt_stats.work, lt_opts.timing_class)
KC_NAMES = ["rbgs", "restrict", "prolong", "coarse", "exact_res", "update_u", "dots", "ortho", "normalize",
            "shift_ls", "xk", "true_res", "fused_down", "fused_up", "other", "inner"]
KC_COUNT = len(KC_NAMES)
KC = {n: i for i, n in enumerate(KC_NAMES)}


class LtOpts(C.Structure):
    _fields_ = [("Nz", C.c_int), ("tol", C.c_double), ("maxit", C.c_int), ("tau_policy", C.c_int),
                ("tau_project", C.c_int), ("groups", C.c_int), ("mg_pre", C.c_int), ("mg_post", C.c_int),
                ("inner_cycles", C.c_int), ("inner_rounds", C.c_int), ("inner_tol", C.c_double),
                ("true_residual", C.c_int), ("check_every", C.c_int), ("timing_class", C.c_int),
                ("inner_relax", C.c_double), ("graphs", C.c_int), ("mg_tile", C.c_int), ("precond", C.c_int),
                ("mg_tma", C.c_int), ("mg_cluster", C.c_int), ("precision", C.c_int), ("krylov", C.c_int),
                ("stop_rule", C.c_int), ("tma_wait_polls", C.c_int), ("gram_schmidt", C.c_int),
                ("block", C.c_int)]


class LtStats(C.Structure):
    _fields_ = [("n_bases", C.c_int), ("n_shift_solves", C.c_int), ("n_converged", C.c_int),
                ("outer_iters_max", C.c_int), ("outer_iters_sum", C.c_int), ("inner_cycles_total", C.c_int),
                ("max_true_residual", C.c_double), ("max_proj_residual", C.c_double),
                ("max_inner_residual", C.c_double), ("ms_total", C.c_float), ("kernel_launches", C.c_int),
                ("timed_ms", C.c_float), ("timed_launches", C.c_int), ("work", C.c_ulonglong * 16)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "work"}
        d["work"] = [int(x) for x in self.work[:KC_COUNT]]
        return d


EXPORTS = {
    "lt_default_options": (C.c_int, [C.POINTER(LtOpts)]),
    "lt_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int]),
    "lt_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lt_setup_grid": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lt_set_sources": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "lt_set_receivers": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "lt_set_source_rates": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lt_set_initial_state": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lt_set_options": (C.c_int, [C.c_void_p, C.POINTER(LtOpts)]),
    "lt_forward": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(LtStats)]),
    "lt_forward_batch": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                   C.c_void_p]),
    "lt_adjoint_batch": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_void_p]),
    "lt_crank_nicolson": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                                    C.POINTER(LtStats)]),
    "lt_geostat_step": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_double,
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(LtStats)]),
    "lt_forward_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(LtStats)]),
    "lt_forward_fields": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.POINTER(LtStats)]),
    "lt_adjoint_jacobian": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(LtStats)]),
    "lt_adjoint_vjp": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                 C.POINTER(LtStats)]),
    "lt_unet_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_ulonglong]),
    "lt_unet_num_params": (C.c_int, [C.c_void_p]),
    "lt_unet_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "lt_unet_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "lt_unet_forward": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "lt_unet_grad": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                               C.POINTER(C.c_double)]),
    "lt_unet_train_step": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_float,
                                     C.POINTER(C.c_double)]),
    "lt_unet_set_wait_polls": (C.c_int, [C.c_void_p, C.c_uint]),
    "lt_unet_last_error": (C.c_char_p, [C.c_void_p]),
    "lt_unet_destroy": (None, [C.c_void_p]),
    "lt_precond_apply": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "lt_set_learned_preconditioner": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lt_contour_nodes": (C.c_int, [C.c_double, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "lt_learned_pairs": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "lt_krylov_vectors": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]),
    "lt_strerror": (C.c_char_p, [C.c_int]),
    "lt_last_error": (C.c_char_p, [C.c_void_p]),
    "lt_destroy": (None, [C.c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load liblt.so and declare every exported symbol; raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run paper_1409_2556_gb300.build.build() (CUDA extension not built)")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
