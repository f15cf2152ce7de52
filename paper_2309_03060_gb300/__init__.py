"""GB300 (sm_103a) compositional linear algebra: Python binding of the C ABI.

Operators are trees of linear maps defined by their MVM (CoLA Sec. 3.1-3.2);
CG, Lanczos / SLQ and the adjoint rules of App. B.2 run on them inside the
CUDA library ``libcola_gb300.so``.  This module only marshals arguments:
PyTorch provides device memory and the current stream.  Every function keeps
the C entry point's name.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _abi
from ._abi import (F32, F64, PREC_F32, PREC_F64, PREC_MIXED, ColaError, check,
                   cola_cg_info, cola_cg_opts)

__all__ = [
    "Context", "LinOp", "cola_create", "cola_linop_dense", "cola_linop_diag",
    "cola_linop_lowrank", "cola_linop_kron", "cola_linop_kronsum", "cola_linop_sum",
    "cola_linop_product", "cola_matvec", "cola_cg_solve", "cola_cg_solve_batched",
    "cola_lanczos", "cola_slq_logdet", "cola_bilinear_grad", "cola_solve_backward",
    "cola_logdet_backward", "cola_rademacher", "cola_cg_opts_default", "ColaError",
    "cola_kron_eig_solve", "cola_kron_eig_logdet", "cola_sym_eig", "cola_product_solve",
    "cola_diag_estimate", "cola_arnoldi_householder",
    "PREC_F64", "PREC_F32", "PREC_MIXED",
]


def _lib():
    return _abi.load()


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor) -> C.c_void_p:
    if not t.is_cuda:
        raise ValueError("tensor must live on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return C.c_void_p(t.data_ptr())


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"unsupported dtype {t.dtype}")


def _vec_dtype(precision: int, refine: bool = False) -> torch.dtype:
    return torch.float64 if (precision == PREC_F64 or refine) else torch.float32


class Context:
    """Owns a cola_ctx (device workspace, cached plans and graphs)."""

    def __init__(self, device: int = 0):
        lib = _lib()
        h = C.c_void_p()
        check(lib.cola_create(int(device), C.byref(h)))
        self.handle = h
        self.device = torch.device("cuda", device)

    def close(self):
        if self.handle:
            check(_lib().cola_destroy(self.handle))
            self.handle = None

    def kernel_launches(self) -> int:
        n = C.c_int64()
        check(_lib().cola_kernel_launches(self.handle, C.byref(n)))
        return n.value

    def test_stall_next_launch(self, wait_ns: int) -> None:
        """Arms cola_test_stall_next_launch (time-out path test hook)."""
        check(_lib().cola_test_stall_next_launch(self.handle, int(wait_ns)))

    def stream(self) -> "torch.cuda.ExternalStream":
        """The library's launch stream (for timing kernels with events)."""
        s = C.c_void_p()
        check(_lib().cola_get_stream(self.handle, C.byref(s)))
        return torch.cuda.ExternalStream(s.value, device=self.device)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cola_create(device: int = 0) -> Context:
    return Context(device)


class LinOp:
    """A cola_linop handle; keeps the borrowed tensors and children alive.

    Leaves keep their prepared copies (working-precision and split images)
    across calls; reading ``handle`` first compares every borrowed tensor's
    version counter with the one last seen and reports a change to the
    library (cola_linop_touch), so in-place updates are picked up."""

    def __init__(self, ctx: Context, handle, keep=(), children=()):
        self.ctx = ctx
        self._h = handle
        self._keep = list(keep)
        self._seen = [t._version for t in self._keep]
        self._children = list(children)
        if self._keep and handle:
            check(_lib().cola_linop_cache_prepared(handle, 1))

    def _sync(self):
        for i, t in enumerate(self._keep):
            if t._version != self._seen[i]:
                check(_lib().cola_linop_touch(self._h))
                self._seen = [u._version for u in self._keep]
                break
        for ch in self._children:
            ch._sync()

    @property
    def handle(self):
        if self._h:
            self._sync()
        return self._h

    @handle.setter
    def handle(self, h):
        self._h = h

    @property
    def shape(self):
        r, c = C.c_int64(), C.c_int64()
        check(_lib().cola_linop_shape(self.handle, C.byref(r), C.byref(c)))
        return (r.value, c.value)

    def leaves(self):
        """[(kind, rows, cols)] in tree order."""
        lib = _lib()
        n = C.c_int()
        check(lib.cola_linop_num_leaves(self.handle, C.byref(n)))
        out = []
        for i in range(n.value):
            k, r, c = C.c_int(), C.c_int64(), C.c_int64()
            check(lib.cola_linop_leaf_info(self.handle, i, C.byref(k), C.byref(r), C.byref(c)))
            out.append((k.value, r.value, c.value))
        return out

    def set_spd(self, spd: bool = True) -> "LinOp":
        check(_lib().cola_linop_set_spd(self.handle, int(bool(spd))))
        return self

    def release(self):
        if self._h:
            check(_lib().cola_linop_release(self._h))
            self._h = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def _new(ctx, fn, *args, keep=(), children=()):
    h = C.c_void_p()
    check(fn(ctx.handle, *args, C.byref(h)))
    return LinOp(ctx, h, keep, children)


def cola_linop_dense(ctx: Context, M: torch.Tensor) -> LinOp:
    rows, cols = M.shape
    return _new(ctx, _lib().cola_linop_dense, rows, cols, _ptr(M), M.stride(0), _dtype_code(M),
                keep=[M])


def cola_linop_diag(ctx: Context, d: torch.Tensor, n: int | None = None) -> LinOp:
    """Vector d (n entries) -> Diag(d); a one-element d with n given -> d[0] * I_n."""
    if n is None:
        return _new(ctx, _lib().cola_linop_diag, d.numel(), _ptr(d), 1, _dtype_code(d), keep=[d])
    return _new(ctx, _lib().cola_linop_diag, int(n), _ptr(d), 0, _dtype_code(d), keep=[d])


def cola_linop_lowrank(ctx: Context, U: torch.Tensor, V: torch.Tensor | None = None) -> LinOp:
    n, k = U.shape
    vp = _ptr(V) if V is not None else None
    return _new(ctx, _lib().cola_linop_lowrank, n, k, _ptr(U), vp, _dtype_code(U),
                keep=[U] + ([V] if V is not None else []))


def _handles(ops):
    arr = (C.c_void_p * len(ops))(*[o.handle for o in ops])
    return arr


def cola_linop_kron(ctx: Context, *factors: LinOp) -> LinOp:
    return _new(ctx, _lib().cola_linop_kron, len(factors), _handles(factors), children=factors)


def cola_linop_kronsum(ctx: Context, *factors: LinOp) -> LinOp:
    return _new(ctx, _lib().cola_linop_kronsum, len(factors), _handles(factors), children=factors)


def cola_linop_sum(ctx: Context, terms, coeffs=None) -> LinOp:
    cptr = None if coeffs is None else (C.c_double * len(terms))(*[float(c) for c in coeffs])
    return _new(ctx, _lib().cola_linop_sum, len(terms), _handles(terms), cptr, children=terms)


def cola_linop_product(ctx: Context, terms) -> LinOp:
    return _new(ctx, _lib().cola_linop_product, len(terms), _handles(terms), children=terms)


def cola_matvec(ctx: Context, op: LinOp, X: torch.Tensor, precision: int = PREC_F64,
                out: torch.Tensor | None = None, split_terms: int = 2) -> torch.Tensor:
    X2 = X if X.dim() == 2 else X.reshape(1, -1)
    rows, cols = op.shape
    if X2.shape[1] != cols:
        raise ValueError(f"X has {X2.shape[1]} columns, operator has {cols}")
    want = _vec_dtype(precision)
    if X2.dtype != want:
        raise TypeError(f"precision {precision} needs {want} vectors")
    Y = out if out is not None else torch.empty((X2.shape[0], rows), dtype=want, device=X.device)
    ft, vt = (split_terms, split_terms) if isinstance(split_terms, int) else split_terms
    check(_lib().cola_set_split_terms(ctx.handle, int(ft), int(vt)))
    check(_lib().cola_matvec(ctx.handle, op.handle, _ptr(X2), _ptr(Y), X2.shape[0], precision,
                             _stream()))
    return Y if X.dim() == 2 else Y.reshape(-1)


def cola_kron_eig_solve(ctx: Context, op: LinOp, B: torch.Tensor, precision: int = PREC_F64,
                        out: torch.Tensor | None = None) -> torch.Tensor:
    """X = A^-1 B from the factor eigendecompositions (A = c K_1 (x) ... (x) K_d [+ s I])."""
    B2 = B if B.dim() == 2 else B.reshape(1, -1)
    rows, cols = op.shape
    if B2.shape[1] != rows:
        raise ValueError(f"B has {B2.shape[1]} columns, operator has {rows} rows")
    want = torch.float64 if precision == PREC_F64 else torch.float32
    if B2.dtype != want or precision not in (PREC_F64, PREC_F32):
        raise TypeError("precision F64 needs float64 vectors, F32 float32 vectors")
    X = out if out is not None else torch.empty_like(B2)
    check(_lib().cola_kron_eig_solve(ctx.handle, op.handle, _ptr(B2), _ptr(X), B2.shape[0],
                                     precision, _stream()))
    return X if B.dim() == 2 else X.reshape(-1)


def cola_product_solve(ctx: Context, op: LinOp, B: torch.Tensor,
                       opts: cola_cg_opts | None = None, use_structure: bool = True,
                       raise_on_error: bool = True):
    """Solve A X = B for a product A = A_1 ... A_m one factor at a time.
    Returns (X, info list, status)."""
    opts = opts or cola_cg_opts_default()
    B2 = B if B.dim() == 2 else B.reshape(1, -1)
    R = B2.shape[0]
    want = _vec_dtype(opts.precision, bool(opts.refine))
    if B2.dtype != want:
        raise TypeError(f"this precision/refine setting needs {want} vectors")
    X = torch.empty_like(B2)
    info = (cola_cg_info * R)()
    st = _lib().cola_product_solve(ctx.handle, op.handle, _ptr(B2), _ptr(X), R, C.byref(opts),
                                   int(use_structure), info, _stream())
    if raise_on_error and st not in (0, 5):
        check(st)
    X = X if B.dim() == 2 else X.reshape(-1)
    return X, _info_list(info, R), st


def cola_kron_eig_logdet(ctx: Context, op: LinOp) -> float:
    """Exact log det A from the factor eigenvalues."""
    v = C.c_double()
    check(_lib().cola_kron_eig_logdet(ctx.handle, op.handle, C.byref(v), _stream()))
    return v.value


def cola_kron_eigs(ctx: Context, op: LinOp, want_evals: bool = True):
    """Kronecker-form eigendecomposition: (factor eigenvalues [w_1, ..],
    factor eigenvector matrices [V_1, ..] (columns = eigenvectors), and the N
    eigenvalues of A in flat index order, or None when want_evals is False)."""
    # the factors are the operator's dense leaves (a scalar shift is the other)
    sizes = [r for k, r, _ in op.leaves() if k == 0]
    dev = ctx.device
    w = torch.empty(sum(sizes), dtype=torch.float64, device=dev)
    V = torch.empty(sum(n * n for n in sizes), dtype=torch.float64, device=dev)
    N = op.shape[0]
    ev = torch.empty(N, dtype=torch.float64, device=dev) if want_evals else None
    check(_lib().cola_kron_eigs(ctx.handle, op.handle, _ptr(w), _ptr(V),
                                _ptr(ev) if ev is not None else None, _stream()))
    ws, Vs, ow, ov = [], [], 0, 0
    for n in sizes:
        ws.append(w[ow:ow + n])
        Vs.append(V[ov:ov + n * n].reshape(n, n))
        ow += n
        ov += n * n
    return ws, Vs, ev


def cola_sym_eig(A):
    """(w, V) with A = V diag(w) V^T for a symmetric matrix in host memory
    (a numpy array); the routine applied to every Kronecker factor."""
    import numpy as np
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    if A.shape != (n, n):
        raise ValueError("A must be square")
    V = np.empty((n, n))
    w = np.empty(n)
    check(_lib().cola_sym_eig(n, A.ctypes.data, V.ctypes.data, w.ctypes.data))
    return w, V


def cola_cg_opts_default(**kw) -> cola_cg_opts:
    o = cola_cg_opts()
    _lib().cola_cg_opts_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _info_list(info, n):
    return [dict(iterations=info[i].iterations, rel_residual=info[i].rel_residual,
                 updates=info[i].updates, status=info[i].status) for i in range(n)]


def cola_cg_solve(ctx: Context, op: LinOp, B: torch.Tensor, opts: cola_cg_opts | None = None,
                  X0: torch.Tensor | None = None, raise_on_error: bool = True):
    """Solve A X = B.  Returns (X, info list, status)."""
    opts = opts or cola_cg_opts_default()
    B2 = B if B.dim() == 2 else B.reshape(1, -1)
    R = B2.shape[0]
    want = _vec_dtype(opts.precision, bool(opts.refine))
    if B2.dtype != want:
        raise TypeError(f"this precision/refine setting needs {want} vectors")
    X = torch.empty_like(B2) if X0 is None else X0.reshape(B2.shape).clone()
    opts.x0_given = 0 if X0 is None else 1
    info = (cola_cg_info * R)()
    st = _lib().cola_cg_solve(ctx.handle, op.handle, _ptr(B2), _ptr(X), R, C.byref(opts), info,
                              _stream())
    if raise_on_error and st not in (0, 5):
        check(st)
    X = X if B.dim() == 2 else X.reshape(-1)
    return X, _info_list(info, R), st


def cola_cg_solve_batched(ctx: Context, ops, Bs, opts: cola_cg_opts | None = None):
    opts = opts or cola_cg_opts_default()
    n = len(ops)
    Xs = [torch.empty_like(b) for b in Bs]
    R = [b.shape[0] for b in Bs]
    info = (cola_cg_info * sum(R))()
    st = _lib().cola_cg_solve_batched(
        ctx.handle, n, _handles(ops), (C.c_void_p * n)(*[b.data_ptr() for b in Bs]),
        (C.c_void_p * n)(*[x.data_ptr() for x in Xs]), (C.c_int64 * n)(*R), C.byref(opts), info,
        _stream())
    if st not in (0, 5):
        check(st)
    return Xs, _info_list(info, sum(R)), st


def cola_arnoldi_householder(ctx: Context, op: LinOp, Q0: torch.Tensor, m: int,
                             precision: int = PREC_F64):
    """Householder Arnoldi (Algorithm 2).  Returns (H [nvec, m+1, m] FP64, m_eff)."""
    Q2 = Q0 if Q0.dim() == 2 else Q0.reshape(1, -1)
    nv = Q2.shape[0]
    H = torch.zeros((nv, m + 1, m), dtype=torch.float64, device=Q2.device)
    meff = torch.zeros(nv, dtype=torch.int32, device=Q2.device)
    check(_lib().cola_arnoldi_householder(ctx.handle, op.handle, _ptr(Q2), nv, m, precision,
                                          _ptr(H), _ptr(meff), _stream()))
    return H, meff


def cola_lanczos(ctx: Context, op: LinOp, Q0: torch.Tensor, m: int, precision: int = PREC_F64,
                 reorth: int = 0, split_terms=2):
    """reorth: 0 none, 1 full reorthogonalisation, 2 Householder basis;
    split_terms (MIXED) as in cola_matvec."""
    nv = Q0.shape[0]
    ft, vt = (split_terms, split_terms) if isinstance(split_terms, int) else split_terms
    check(_lib().cola_set_split_terms(ctx.handle, int(ft), int(vt)))
    alpha = torch.zeros((nv, m), dtype=torch.float64, device=Q0.device)
    beta = torch.zeros((nv, m), dtype=torch.float64, device=Q0.device)
    meff = torch.zeros(nv, dtype=torch.int32, device=Q0.device)
    check(_lib().cola_lanczos(ctx.handle, op.handle, _ptr(Q0), nv, m, precision, int(reorth),
                              _ptr(alpha), _ptr(beta), _ptr(meff), _stream()))
    return alpha, beta, meff


def cola_slq_logdet(ctx: Context, op: LinOp, nprobes: int, m: int, seed: int = 0,
                    probes: torch.Tensor | None = None, precision: int = PREC_F64,
                    reorth: int = 0, split_terms=2):
    """Returns (logdet, std_err, per_probe tensor, clamped count); split_terms
    (MIXED) as in cola_matvec."""
    ft, vt = (split_terms, split_terms) if isinstance(split_terms, int) else split_terms
    check(_lib().cola_set_split_terms(ctx.handle, int(ft), int(vt)))
    ld, se = C.c_double(), C.c_double()
    cl = C.c_int32()
    pp = torch.empty(nprobes, dtype=torch.float64, device=ctx.device)
    check(_lib().cola_slq_logdet(ctx.handle, op.handle, nprobes, m, C.c_uint64(seed & (2**64 - 1)),
                                 _ptr(probes) if probes is not None else None, precision,
                                 int(reorth), C.byref(ld), C.byref(se), _ptr(pp), C.byref(cl),
                                 _stream()))
    return ld.value, se.value, pp, cl.value


def cola_diag_estimate(ctx: Context, op: LinOp, nprobes: int, seed: int = 0,
                       doubly: bool = True, precision: int = PREC_F64, split_terms=2):
    """Stochastic Diag(A) (FP64 device tensor [N]) and Tr(A) estimates;
    split_terms (MIXED) as in cola_matvec.  Returns (diag, trace)."""
    diag = torch.empty(op.shape[0], dtype=torch.float64, device=ctx.device)
    tr = C.c_double()
    ft, vt = (split_terms, split_terms) if isinstance(split_terms, int) else split_terms
    check(_lib().cola_set_split_terms(ctx.handle, int(ft), int(vt)))
    check(_lib().cola_diag_estimate(ctx.handle, op.handle, nprobes,
                                    C.c_uint64(seed & (2**64 - 1)), int(doubly), precision,
                                    _ptr(diag), C.byref(tr), _stream()))
    return diag, tr.value


def _leaf_grad_buffers(op: LinOp, dtypes, device):
    out = []
    for (kind, r, c), dt in zip(op.leaves(), dtypes):
        shape = (r, c) if kind in (_abi.LEAF_DENSE, _abi.LEAF_LOWRANK) else ((r,) if kind == _abi.LEAF_DIAG else (1,))
        out.append(torch.zeros(shape, dtype=dt, device=device))
    return out


def cola_bilinear_grad(ctx: Context, op: LinOp, U: torch.Tensor, X: torch.Tensor, weights=None,
                       precision: int = PREC_F64, leaf_dtypes=None):
    """[sum_r w_r u_r^T (dA/dtheta_l) x_r for every leaf l] as tensors."""
    nl = len(op.leaves())
    leaf_dtypes = leaf_dtypes or [U.dtype] * nl
    grads = _leaf_grad_buffers(op, leaf_dtypes, U.device)
    R = U.shape[0]
    w = None if weights is None else (C.c_double * R)(*[float(v) for v in weights])
    check(_lib().cola_bilinear_grad(ctx.handle, op.handle, _ptr(U), _ptr(X), w, R, precision,
                                    (C.c_void_p * nl)(*[g.data_ptr() for g in grads]), 0,
                                    _stream()))
    return grads


def cola_gp_objective(ctx: Context, op: LinOp, y: torch.Tensor, Z: torch.Tensor,
                      slq_steps: int, opts: cola_cg_opts | None = None):
    """L = 1/2 y^T A^-1 y + 1/2 log det A.  Returns (L, Sol = A^-1 [y, Z],
    logdet, logdet standard error, info list, status)."""
    opts = opts or cola_cg_opts_default()
    want = _vec_dtype(opts.precision, bool(opts.refine))
    if y.dtype != want or Z.dtype != want:
        raise TypeError(f"this precision/refine setting needs {want} vectors")
    m = Z.shape[0]
    N = y.numel()
    Sol = torch.empty((1 + m, N), dtype=want, device=y.device)
    info = (cola_cg_info * (1 + m))()
    v, ld, se = C.c_double(), C.c_double(), C.c_double()
    st = _lib().cola_gp_objective(ctx.handle, op.handle, _ptr(y.contiguous()), _ptr(Z.contiguous()),
                                  m, int(slq_steps), C.byref(opts), _ptr(Sol), C.byref(v),
                                  C.byref(ld), C.byref(se), info, _stream())
    if st not in (0, 5):
        check(st)
    return v.value, Sol, ld.value, se.value, _info_list(info, 1 + m), st


def cola_gp_objective_backward(ctx: Context, op: LinOp, Sol: torch.Tensor, Z: torch.Tensor,
                               g: float, precision: int = PREC_F64, leaf_dtypes=None):
    """(leaf gradients, grad_y) of g * L from the forward solution block."""
    m = Z.shape[0]
    nl = len(op.leaves())
    grads = _leaf_grad_buffers(op, leaf_dtypes or [Sol.dtype] * nl, Sol.device)
    gy = torch.empty(Sol.shape[1], dtype=Sol.dtype, device=Sol.device)
    check(_lib().cola_gp_objective_backward(
        ctx.handle, op.handle, _ptr(Sol), _ptr(Z), m, float(g), precision,
        (C.c_void_p * nl)(*[t.data_ptr() for t in grads]), _ptr(gy), _stream()))
    return grads, gy


def cola_solve_backward(ctx: Context, op: LinOp, X: torch.Tensor, gradX: torch.Tensor,
                        opts: cola_cg_opts | None = None, leaf_dtypes=None):
    """Returns (gradB, leaf grads, info, status)."""
    opts = opts or cola_cg_opts_default()
    R = X.shape[0]
    nl = len(op.leaves())
    grads = _leaf_grad_buffers(op, leaf_dtypes or [torch.float64] * nl, X.device)
    gradB = torch.empty_like(gradX)
    info = (cola_cg_info * R)()
    st = _lib().cola_solve_backward(ctx.handle, op.handle, _ptr(X), _ptr(gradX), _ptr(gradB), R,
                                    (C.c_void_p * nl)(*[g.data_ptr() for g in grads]),
                                    C.byref(opts), info, _stream())
    if st not in (0, 5):
        check(st)
    return gradB, grads, _info_list(info, R), st


def cola_logdet_backward(ctx: Context, op: LinOp, Z: torch.Tensor, AinvZ: torch.Tensor | None,
                         scale: float = 1.0, opts: cola_cg_opts | None = None, leaf_dtypes=None):
    opts = opts or cola_cg_opts_default()
    nl = len(op.leaves())
    grads = _leaf_grad_buffers(op, leaf_dtypes or [torch.float64] * nl, Z.device)
    st = _lib().cola_logdet_backward(ctx.handle, op.handle, _ptr(Z),
                                     _ptr(AinvZ) if AinvZ is not None else None, Z.shape[0],
                                     float(scale),
                                     (C.c_void_p * nl)(*[g.data_ptr() for g in grads]), 0,
                                     C.byref(opts), _stream())
    if st not in (0, 5):
        check(st)
    return grads


def cola_rademacher(ctx: Context, seed: int, count: int, offset: int = 0,
                    dtype=torch.float64) -> torch.Tensor:
    out = torch.empty(count, dtype=dtype, device=ctx.device)
    check(_lib().cola_rademacher(ctx.handle, C.c_uint64(seed & (2**64 - 1)), offset, count,
                                 _ptr(out), F64 if dtype == torch.float64 else F32, _stream()))
    return out
