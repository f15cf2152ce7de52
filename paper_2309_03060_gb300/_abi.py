"""ctypes declarations of the C ABI in include/cola.h (argument marshalling only).

Loading fails loudly when the shared library has not been built: there is no
CPU or Python fallback for any call.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcola_gb300.so")

COLA_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "SHAPE", 3: "DTYPE", 4: "BREAKDOWN",
                5: "NOT_CONVERGED", 6: "TIMEOUT", 7: "CUDA", 8: "OOM", 9: "UNSUPPORTED"}
F64, F32 = 0, 1
PREC_F64, PREC_F32, PREC_MIXED = 0, 1, 2
LEAF_DENSE, LEAF_DIAG, LEAF_SCALAR, LEAF_LOWRANK = 0, 1, 2, 3


class cola_cg_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("maxiter", C.c_int64), ("precision", C.c_int32),
                ("refine", C.c_int32), ("reliable_delta", C.c_double),
                ("max_updates", C.c_int32), ("split_factor_terms", C.c_int32),
                ("split_vector_terms", C.c_int32), ("graph_chunk", C.c_int32),
                ("jacobi", C.c_int32), ("x0_given", C.c_int32),
                ("kron_precond", C.c_int32), ("reorth_residuals", C.c_int32)]


class cola_cg_info(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("rel_residual", C.c_double),
                ("updates", C.c_int32), ("status", C.c_int32)]


P = C.c_void_p
PP = C.POINTER(C.c_void_p)
I64 = C.c_int64
I32 = C.c_int32
D = C.c_double

SIGNATURES = {
    "cola_last_error": (C.c_char_p, []),
    "cola_create": (I32, [C.c_int, PP]),
    "cola_destroy": (I32, [P]),
    "cola_linop_dense": (I32, [P, I64, I64, P, I64, I32, PP]),
    "cola_linop_diag": (I32, [P, I64, P, I64, I32, PP]),
    "cola_linop_lowrank": (I32, [P, I64, I64, P, P, I32, PP]),
    "cola_linop_kron": (I32, [P, C.c_int, PP, PP]),
    "cola_linop_kronsum": (I32, [P, C.c_int, PP, PP]),
    "cola_linop_sum": (I32, [P, C.c_int, PP, C.POINTER(D), PP]),
    "cola_linop_product": (I32, [P, C.c_int, PP, PP]),
    "cola_linop_set_spd": (I32, [P, C.c_int]),
    "cola_linop_shape": (I32, [P, C.POINTER(I64), C.POINTER(I64)]),
    "cola_linop_num_leaves": (I32, [P, C.POINTER(C.c_int)]),
    "cola_linop_leaf_info": (I32, [P, C.c_int, C.POINTER(C.c_int), C.POINTER(I64),
                                   C.POINTER(I64)]),
    "cola_linop_release": (I32, [P]),
    "cola_matvec": (I32, [P, P, P, P, I64, I32, P]),
    "cola_cg_opts_default": (None, [C.POINTER(cola_cg_opts)]),
    "cola_cg_solve": (I32, [P, P, P, P, I64, C.POINTER(cola_cg_opts), C.POINTER(cola_cg_info), P]),
    "cola_cg_solve_batched": (I32, [P, I32, PP, PP, PP, C.POINTER(I64), C.POINTER(cola_cg_opts),
                                    C.POINTER(cola_cg_info), P]),
    "cola_lanczos": (I32, [P, P, P, I64, I32, I32, I32, P, P, P, P]),
    "cola_slq_logdet": (I32, [P, P, I32, I32, C.c_uint64, P, I32, I32, C.POINTER(D), C.POINTER(D),
                              P, C.POINTER(I32), P]),
    "cola_bilinear_grad": (I32, [P, P, P, P, C.POINTER(D), I64, I32, PP, I32, P]),
    "cola_solve_backward": (I32, [P, P, P, P, P, I64, PP, C.POINTER(cola_cg_opts),
                                  C.POINTER(cola_cg_info), P]),
    "cola_logdet_backward": (I32, [P, P, P, P, I64, D, PP, I32, C.POINTER(cola_cg_opts), P]),
    "cola_rademacher": (I32, [P, C.c_uint64, I64, I64, P, I32, P]),
    "cola_diag_estimate": (I32, [P, P, I32, C.c_uint64, I32, I32, P, C.POINTER(D), P]),
    "cola_arnoldi_householder": (I32, [P, P, P, I64, I32, I32, P, P, P]),
    "cola_kernel_launches": (I32, [P, C.POINTER(I64)]),
    "cola_get_stream": (I32, [P, C.POINTER(P)]),
    "cola_kron_eig_solve": (I32, [P, P, P, P, I64, I32, P]),
    "cola_kron_eig_logdet": (I32, [P, P, C.POINTER(C.c_double), P]),
    "cola_product_solve": (I32, [P, P, P, P, I64, P, I32, P, P]),
    "cola_linop_cache_prepared": (I32, [P, I32]),
    "cola_linop_touch": (I32, [P]),
    "cola_batch_tile_table": (I32, [I32, P, P, P, I32, P, P, I64, P]),
    "cola_sym_eig": (I32, [I64, P, P, P]),
    "cola_set_split_terms": (I32, [P, I32, I32]),
    "cola_test_stall_next_launch": (I32, [P, I64]),
    "cola_kron_eigs": (I32, [P, P, P, P, P, P]),
    "cola_gp_objective": (I32, [P, P, P, P, I64, I32, C.POINTER(cola_cg_opts), P,
                                C.POINTER(D), C.POINTER(D), C.POINTER(D),
                                C.POINTER(cola_cg_info), P]),
    "cola_gp_objective_backward": (I32, [P, P, P, P, I64, D, I32, PP, P, P]),
    "cola_kron_matvec_noalloc": (I32, [C.c_int, C.POINTER(I64), C.POINTER(I64), PP, P, P, I64, P]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the library (once) and attach argument types to every entry point."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build the CUDA library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class ColaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def check(status: int):
    if status != COLA_OK:
        msg = _lib.cola_last_error().decode() if _lib is not None else ""
        raise ColaError(status, msg)
    return status
