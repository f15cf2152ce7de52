"""CPU-side checks of the C ABI: the library builds, loads without a GPU and
exports every entry point include/cola.h declares; host logic that needs no
device (option defaults, error reporting without a device)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cola.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cola_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2309_03060_gb300 import build, _abi
    build.build()
    return _abi.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["cola_linop_dense", "cola_linop_diag", "cola_linop_lowrank", "cola_linop_kron",
                     "cola_linop_kronsum", "cola_linop_sum", "cola_linop_product", "cola_matvec",
                     "cola_cg_solve", "cola_lanczos", "cola_slq_logdet", "cola_solve_backward"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2309_03060_gb300 import _abi
    out = subprocess.run(["nm", "-D", "--defined-only", _abi.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (cola_[a-z0-9_]+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)
        assert n in _abi.SIGNATURES, f"binding lacks {n}"


def test_opts_defaults(lib):
    from paper_2309_03060_gb300 import _abi
    o = _abi.cola_cg_opts()
    lib.cola_cg_opts_default(ctypes.byref(o))
    assert o.tol == 1e-8 and o.maxiter == 100000 and o.precision == _abi.PREC_MIXED
    assert o.refine == 1 and o.split_factor_terms == 3 and o.split_vector_terms == 3
    assert o.graph_chunk == 64
    assert o.jacobi == 0 and o.x0_given == 0 and o.kron_precond == 0
    assert o.reorth_residuals == 0
    assert ctypes.sizeof(o) == 64  # sizeof(cola_cg_opts) in C (fields appended at the end)


def test_null_arguments_are_rejected_without_a_device(lib):
    from paper_2309_03060_gb300 import _abi
    h = ctypes.c_void_p()
    st = lib.cola_linop_dense(None, 4, 4, None, 4, 0, ctypes.byref(h))
    assert st == 1  # INVALID_ARG, before any CUDA call
    assert b"NULL" in lib.cola_last_error()
    assert lib.cola_linop_release(None) == 1
    assert lib.cola_destroy(None) == 1


def test_new_entry_points_reject_null_without_a_device(lib):
    """The structured, product, estimator and Householder calls check their
    arguments before touching the device."""
    from paper_2309_03060_gb300 import _abi
    o = _abi.cola_cg_opts()
    lib.cola_cg_opts_default(ctypes.byref(o))
    assert lib.cola_product_solve(None, None, None, None, 1, ctypes.byref(o), 1, None, None) == 1
    d = ctypes.c_double()
    assert lib.cola_diag_estimate(None, None, 4, 0, 1, 0, None, ctypes.byref(d), None) == 1
    assert lib.cola_arnoldi_householder(None, None, None, 1, 4, 0, None, None, None) == 1
    assert lib.cola_kron_eig_solve(None, None, None, None, 1, 0, None) == 1
    assert lib.cola_kron_eig_logdet(None, None, ctypes.byref(d), None) == 1


def test_sym_eig_runs_on_the_host(lib):
    """cola_sym_eig needs no GPU: A V = V diag(w) for a small symmetric matrix."""
    import numpy as np
    r = np.random.default_rng(3)
    A = r.standard_normal((7, 7))
    A = np.ascontiguousarray(A + A.T)
    V = np.zeros((7, 7))
    w = np.zeros(7)
    st = lib.cola_sym_eig(7, A.ctypes.data, V.ctypes.data, w.ctypes.data)
    assert st == 0
    np.testing.assert_allclose(A @ V, V * w, atol=1e-12)
    np.testing.assert_allclose(V.T @ V, np.eye(7), atol=1e-13)


def test_noalloc_rejects_oversize_and_overflow_without_a_device(lib):
    """The allocation-free Kronecker MVM checks its scratch bound before it
    looks at the device, with sizes that cannot wrap around: a huge nrhs, and
    factor shapes whose product overflows int64, are refused with
    COLA_ERR_INVALID_ARG and nothing is launched (the device pointers here are
    placeholders that are never dereferenced)."""
    fake = ctypes.c_void_p(256)
    rows = (ctypes.c_int64 * 2)(64, 64)
    cols = (ctypes.c_int64 * 2)(64, 64)
    ptrs = (ctypes.c_void_p * 2)(256, 512)
    huge = (1 << 62) // 64
    st = lib.cola_kron_matvec_noalloc(2, rows, cols, ptrs, fake, ctypes.c_void_p(1024), huge,
                                      None)
    assert st == 1 and b"scratch" in lib.cola_last_error()
    big = (ctypes.c_int64 * 3)(1 << 30, 1 << 30, 1 << 30)
    ptrs3 = (ctypes.c_void_p * 3)(256, 512, 768)
    st = lib.cola_kron_matvec_noalloc(3, big, big, ptrs3, fake, ctypes.c_void_p(1024), 1, None)
    assert st == 1 and b"overflow" in lib.cola_last_error()
    # nrhs = 2 with a 2048 x 2048 intermediate fits in 4 Mi floats only once
    r2 = (ctypes.c_int64 * 2)(2048, 2048)
    st = lib.cola_kron_matvec_noalloc(2, r2, r2, ptrs, fake, ctypes.c_void_p(1024), 2, None)
    assert st == 1 and b"scratch" in lib.cola_last_error()
