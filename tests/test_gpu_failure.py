"""Failure detection on the GPU path, without a GPU fault.

* Time-out path of the tensor-core kernels: cola_test_stall_next_launch makes
  one launch's MMA role wait on a barrier that nothing completes, with a short
  limit (20 ms).  The launch takes its ordinary time-out path (every role
  stops, each CTA waits for its own copies and MMAs, frees tensor memory and
  exits); the host sees COLA_ERR_TIMEOUT on the context's next call, and the
  call after that is bit-identical to one made before the stall and matches
  the oracle.  Both kernels of a single MVM: factor-stationary (sides <= 128)
  and the split GEMM (a side above 128); and the table-driven kernel of a
  batched solve, which then ends with COLA_ERR_TIMEOUT and succeeds when run
  again.
* Breakdown, injected on the host: a right-hand side with a NaN or an Inf
  entry, and an operator annotated spd that is not (p^T A p < 0 in the first
  iteration), end with COLA_ERR_BREAKDOWN in that right-hand side's info while
  the other right-hand side still converges.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import krylov
from oracle import linop as O
from tests._trees import gpu_tree, oracle_tree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda"
TIMEOUT = 6
BREAKDOWN = 4


@pytest.fixture(scope="module")
def cola():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2309_03060_gb300 as c
    from paper_2309_03060_gb300 import build
    build.build()
    return c


@pytest.fixture(scope="module")
def ctx(cola):
    return cola.Context(0)


def _rbf(n, seed):
    return wl.rbf_factor(wl.uniform(wl.substream(seed, n), (n,)), 0.2)


@pytest.mark.parametrize("sides", [(64, 48, 32), (160, 24, 16)],
                         ids=["factor_stationary", "split_gemm"])
def test_tensor_core_timeout_reported_and_context_recovers(cola, ctx, sides):
    F = [_rbf(n, 70 + k) for k, n in enumerate(sides)]
    op = cola.cola_linop_kron(ctx, *[cola.cola_linop_dense(ctx, torch.tensor(f, device=DEV))
                                     for f in F])
    N = int(np.prod(sides))
    X = torch.tensor(np.random.default_rng(3).standard_normal((2, N)), dtype=torch.float32,
                     device=DEV)
    good = cola.cola_matvec(ctx, op, X, cola.PREC_MIXED, split_terms=3)
    torch.cuda.synchronize()
    ctx.test_stall_next_launch(20_000_000)
    cola.cola_matvec(ctx, op, X, cola.PREC_MIXED, split_terms=3)  # stalls, returns at once
    torch.cuda.synchronize()
    with pytest.raises(cola.ColaError) as e:
        cola.cola_matvec(ctx, op, X, cola.PREC_MIXED, split_terms=3)
    assert e.value.status == TIMEOUT
    torch.cuda.synchronize()
    after = cola.cola_matvec(ctx, op, X, cola.PREC_MIXED, split_terms=3)
    torch.cuda.synchronize()
    assert torch.equal(after, good)
    ref = O.Kron([O.Dense(f) for f in F])
    Xh = X.double().cpu().numpy()
    bound = O.Kron([O.Dense(np.abs(f)) for f in F]).mvm(np.abs(Xh))
    assert np.max(np.abs(after.double().cpu().numpy() - ref.mvm(Xh)) / bound) < 1e-5


def test_batched_timeout_reported_and_context_recovers(cola, ctx):
    """The table-driven kernel of batched solves (every factor size) takes the
    same time-out path: a batched solve whose first tensor-core launch is made
    to stall ends with COLA_ERR_TIMEOUT, and the same solve run again reaches
    1e-8 by the oracle's FP64 true residual."""
    probs = []
    for k, (n1, n2, R) in enumerate([(40, 48, 2), (150, 24, 1)]):
        F = [_rbf(n1, 90 + k), _rbf(n2, 95 + k)]
        spec = ("sum", [("kron", [("dense", f) for f in F]), ("scalar", 0.05, n1 * n2)], None)
        B = np.random.default_rng(20 + k).standard_normal((R, n1 * n2))
        probs.append((spec, B))
    ops = [gpu_tree(cola, ctx, sp, torch.float64, DEV).set_spd() for sp, _ in probs]
    Bs = [torch.tensor(B, device=DEV) for _, B in probs]
    opts = cola.cola_cg_opts_default(precision=cola.PREC_MIXED, refine=1, tol=1e-8,
                                     maxiter=3000, graph_chunk=16)
    torch.cuda.synchronize()
    ctx.test_stall_next_launch(20_000_000)
    with pytest.raises(cola.ColaError) as e:
        cola.cola_cg_solve_batched(ctx, ops, Bs, opts)
    assert e.value.status == TIMEOUT
    torch.cuda.synchronize()
    Xs, info, st = cola.cola_cg_solve_batched(ctx, ops, Bs, opts)
    assert st == 0, info
    for (spec, B), X in zip(probs, Xs):
        res = krylov.true_relative_residual(oracle_tree(spec), B, X.cpu().numpy())
        assert np.all(res <= 1e-8), res


def _kron_shift(n1, n2, shift, seed):
    F = [_rbf(n1, seed), _rbf(n2, seed + 1)]
    return ("sum", [("kron", [("dense", f) for f in F]), ("scalar", shift, n1 * n2)], None)


@pytest.mark.parametrize("bad", ["nan", "inf"])
@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_cg_nonfinite_rhs_is_breakdown(cola, ctx, bad, prec):
    spec = _kron_shift(40, 48, 0.05, 81)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    B = np.random.default_rng(4).standard_normal((2, 40 * 48))
    B[1, 17] = np.nan if bad == "nan" else np.inf
    P = cola.PREC_F64 if prec == "f64" else cola.PREC_MIXED
    opts = cola.cola_cg_opts_default(precision=P, refine=0 if prec == "f64" else 1, tol=1e-8,
                                     maxiter=5000)
    X, info, st = cola.cola_cg_solve(ctx, op, torch.tensor(B, device=DEV), opts,
                                     raise_on_error=False)
    assert st == BREAKDOWN
    assert info[1]["status"] == BREAKDOWN
    assert info[0]["status"] == 0
    res = krylov.true_relative_residual(oracle_tree(spec), B[:1], X[:1].cpu().numpy())
    assert res[0] <= 1e-8


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_cg_indefinite_operator_flagged_spd_is_breakdown(cola, ctx, prec):
    """A = D1 (x) D2 with diagonal factors of mixed sign, annotated spd: for a
    right-hand side supported where A is negative, p^T A p = b^T A b < 0 in
    the first iteration."""
    n1, n2 = 32, 48
    s1 = np.where(np.arange(n1) % 3 == 0, -1.0, 1.0) * (1.0 + np.arange(n1) / n1)
    s2 = 0.5 + np.arange(n2) / n2
    spec = ("kron", [("dense", np.diag(s1)), ("dense", np.diag(s2))])
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    dA = np.kron(s1, s2)
    B = np.zeros((2, n1 * n2))
    B[0] = np.where(dA > 0, 1.0, 0.0)    # SPD on its support: converges
    B[1] = np.where(dA < 0, 1.0, 0.0)    # negative on its support: breakdown
    P = cola.PREC_F64 if prec == "f64" else cola.PREC_MIXED
    opts = cola.cola_cg_opts_default(precision=P, refine=0 if prec == "f64" else 1, tol=1e-8,
                                     maxiter=2000)
    X, info, st = cola.cola_cg_solve(ctx, op, torch.tensor(B, device=DEV), opts,
                                     raise_on_error=False)
    assert st == BREAKDOWN
    assert info[1]["status"] == BREAKDOWN and info[1]["iterations"] <= 1
    assert info[0]["status"] == 0
    res = krylov.true_relative_residual(oracle_tree(spec), B[:1], X[:1].cpu().numpy())
    assert res[0] <= 1e-8
