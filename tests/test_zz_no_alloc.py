"""The allocation-free Kronecker MVM entry point.

cola_kron_matvec_noalloc is for callers that cannot let a library allocate
device memory: a framework that owns all device memory through its own pool,
code where an allocation would synchronise the device, and callers without a
context.  Its intermediate results live in a fixed file-scope device array.
This test calls it through the C ABI twice in a row and checks each result
against the regular cola_matvec (FP32) on the same inputs, which runs the same
SIMT mode products with the same shapes and strides, so the two must agree bit
for bit; it also checks the result against the oracle's Kronecker MVM at the
FP32 parity tolerance.  The file sorts last so a failure here comes after
every other test has run.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as wl
from oracle import linop as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib_and_cola():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_03060_gb300 as cola
    from paper_2309_03060_gb300 import _abi, build
    build.build()
    lib = _abi.load()
    fn = lib.cola_kron_matvec_noalloc
    fn.restype = C.c_int32
    fn.argtypes = [C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_void_p),
                   C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]
    return lib, cola


def _call(lib, factors, X, Y):
    n = len(factors)
    rows = (C.c_int64 * n)(*[f.shape[0] for f in factors])
    cols = (C.c_int64 * n)(*[f.shape[1] for f in factors])
    ptrs = (C.c_void_p * n)(*[f.data_ptr() for f in factors])
    st = lib.cola_kron_matvec_noalloc(n, rows, cols, ptrs, C.c_void_p(X.data_ptr()),
                                      C.c_void_p(Y.data_ptr()), X.shape[0],
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.cola_last_error().decode()


def _factor_sets():
    r = np.random.default_rng(11)
    return {
        "three_rect": [r.standard_normal((37, 29)), wl.rbf_factor(wl.uniform(5, (64,)), 0.2),
                       r.standard_normal((5, 7))],
        "one_factor": [r.standard_normal((50, 33))],
    }


@pytest.mark.parametrize("name", list(_factor_sets().keys()))
def test_noalloc_matches_matvec_twice(lib_and_cola, name):
    lib, cola = lib_and_cola
    dev = torch.device("cuda", 0)
    r = np.random.default_rng(12)
    mats = _factor_sets()[name]
    F32 = [torch.tensor(m, dtype=torch.float32, device=dev) for m in mats]
    ctx = cola.Context(0)
    op = cola.cola_linop_kron(ctx, *[cola.cola_linop_dense(ctx, f) for f in F32])
    rows, cols = op.shape
    ref_op = O.Kron([O.Dense(f.double().cpu().numpy()) for f in F32])
    for call in range(2):
        Xh = r.standard_normal((3, cols))
        X = torch.tensor(Xh, dtype=torch.float32, device=dev)
        Y = torch.full((3, rows), float("nan"), dtype=torch.float32, device=dev)
        _call(lib, F32, X, Y)
        ref = cola.cola_matvec(ctx, op, X, cola.PREC_F32)
        torch.cuda.synchronize()
        assert torch.equal(Y, ref), (call, float((Y - ref).abs().max()))
        y = Y.double().cpu().numpy()
        exact = ref_op.mvm(X.double().cpu().numpy())
        assert np.max(np.abs(y - exact)) <= 2e-6 * np.max(np.abs(exact)), call


def test_noalloc_rejects_oversize(lib_and_cola):
    lib, _ = lib_and_cola
    dev = torch.device("cuda", 0)
    F = [torch.ones((1024, 1024), dtype=torch.float32, device=dev) for _ in range(2)]
    X = torch.zeros((8, 1024 * 1024), dtype=torch.float32, device=dev)
    Y = torch.zeros_like(X)
    n = 2
    st = lib.cola_kron_matvec_noalloc(n, (C.c_int64 * n)(1024, 1024), (C.c_int64 * n)(1024, 1024),
                                      (C.c_void_p * n)(*[f.data_ptr() for f in F]),
                                      C.c_void_p(X.data_ptr()), C.c_void_p(Y.data_ptr()), 8, None)
    assert st == 1 and b"scratch" in lib.cola_last_error()
