"""Adjoint gradients through torch.autograd (App. B.2) and the large-factor
tensor-core path, against the FP64 oracle.

The GP objective's gradient has an exact quadratic part and a Hutchinson trace
part; the GPU value is compared with the oracle's evaluation of the SAME
estimator on the same probes (deterministic), and the exact eigenbasis
gradient is reported against it.
"""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import exact, grad, krylov
from oracle import linop as O
from tests._trees import gpu_tree, oracle_tree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


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


DEV = "cuda"


def rbf_t(x, ell):
    d = x[:, None] - x[None, :]
    return torch.exp(-(d * d) / (2.0 * ell * ell))


def test_solve_autograd_matches_vjp(cola, ctx):
    from paper_2309_03060_gb300 import autograd as cag
    r = np.random.default_rng(3)
    A = r.standard_normal((6, 6))
    A = A @ A.T / 6 + np.eye(6)
    Bm = r.standard_normal((7, 7))
    Bm = Bm @ Bm.T / 7 + np.eye(7)
    K1 = torch.tensor(A, device=DEV, requires_grad=True)
    K2 = torch.tensor(Bm, device=DEV, requires_grad=True)
    s = torch.tensor([0.2], dtype=torch.float64, device=DEV, requires_grad=True)
    op = cola.cola_linop_sum(ctx, [cola.cola_linop_kron(ctx, cola.cola_linop_dense(ctx, K1.detach()),
                                                        cola.cola_linop_dense(ctx, K2.detach())),
                                   cola.cola_linop_diag(ctx, s.detach(), n=42)]).set_spd()
    b = r.standard_normal((2, 42))
    w = r.standard_normal((2, 42))
    B = torch.tensor(b, device=DEV, requires_grad=True)
    opts = cola.cola_cg_opts_default(precision=cola.PREC_F64, refine=0, tol=1e-13, maxiter=5000,
                                     graph_chunk=4)
    X = cag.solve(ctx, op, B, [K1, K2, s], opts)
    loss = (X * torch.tensor(w, device=DEV)).sum()
    loss.backward()
    ref = O.Sum([O.Kron([O.Dense(A), O.Dense(Bm)]), O.Diag(np.float64(0.2), 42)])
    Ad = ref.dense()
    x = exact.dense_solve(Ad, b)
    u = exact.dense_solve(Ad.T, w)
    g = [-v for v in grad.bilinear_grad(ref, u, x)]
    np.testing.assert_allclose(K1.grad.cpu().numpy(), g[0], rtol=1e-7, atol=1e-10)
    np.testing.assert_allclose(K2.grad.cpu().numpy(), g[1], rtol=1e-7, atol=1e-10)
    np.testing.assert_allclose(s.grad.cpu().numpy()[0], g[2], rtol=1e-7)
    np.testing.assert_allclose(B.grad.cpu().numpy(), u, rtol=1e-8, atol=1e-11)


def _gp_setup(n, nprobes, seed):
    x1 = wl.uniform(wl.substream(seed, 10), (n,))
    x2 = wl.uniform(wl.substream(seed, 11), (n,))
    y = wl.normal(wl.substream(seed, 1), (n * n,))
    Z = wl.rademacher(wl.substream(seed, 2), (nprobes, n * n))
    return x1, x2, y, Z


def _gp_gpu(cola, ctx, x1, x2, y, Z, l1, l2, s2, opts, slq_steps=20):
    from paper_2309_03060_gb300 import autograd as cag
    L1 = torch.tensor(l1, dtype=torch.float64, device=DEV, requires_grad=True)
    L2 = torch.tensor(l2, dtype=torch.float64, device=DEV, requires_grad=True)
    S2 = torch.tensor([s2], dtype=torch.float64, device=DEV, requires_grad=True)
    K1 = rbf_t(torch.tensor(x1, device=DEV), L1)
    K2 = rbf_t(torch.tensor(x2, device=DEV), L2)
    N = len(x1) * len(x2)
    op = cola.cola_linop_sum(ctx, [cola.cola_linop_kron(ctx, cola.cola_linop_dense(ctx, K1.detach()),
                                                        cola.cola_linop_dense(ctx, K2.detach())),
                                   cola.cola_linop_diag(ctx, S2.detach(), n=N)]).set_spd()
    loss = cag.gp_objective(ctx, op, torch.tensor(y, device=DEV), [K1, K2, S2],
                            torch.tensor(Z, device=DEV), opts, slq_steps=slq_steps, seed=1)
    loss.backward()
    return [L1.grad.item(), L2.grad.item(), S2.grad.item()]


def _gp_oracle_same_probes(x1, x2, y, Z, l1, l2, s2):
    """Oracle value of the same estimator: exact quadratic part plus the
    Hutchinson trace on the given probes with exact solves."""
    K1, K2 = wl.rbf_factor(x1, l1), wl.rbf_factor(x2, l2)
    op = O.Sum([O.Kron([O.Dense(K1), O.Dense(K2)]), O.Diag(np.float64(s2), len(y))])
    a = exact.kron_shift_solve([K1, K2], s2, y)
    U = exact.kron_shift_solve([K1, K2], s2, Z)
    m = Z.shape[0]
    g = grad.bilinear_grad(op, np.vstack([a, U]), np.vstack([a, Z]),
                           np.array([-0.5] + [0.5 / m] * m))
    return [float(np.sum(g[0] * wl.rbf_factor_dell(x1, l1))),
            float(np.sum(g[1] * wl.rbf_factor_dell(x2, l2))), float(g[2])]


def test_gp_objective_gradient_f64_small(cola, ctx):
    n, m = 32, 16
    x1, x2, y, Z = _gp_setup(n, m, 71)
    l1, l2, s2 = 0.1, 0.2, 0.1
    opts = cola.cola_cg_opts_default(precision=cola.PREC_F64, refine=0, tol=1e-12, maxiter=20000,
                                     graph_chunk=16)
    g = _gp_gpu(cola, ctx, x1, x2, y, Z, l1, l2, s2, opts)
    ref = _gp_oracle_same_probes(x1, x2, y, Z, l1, l2, s2)
    np.testing.assert_allclose(g, ref, rtol=1e-6)
    # and the exact gradient is within the estimator's spread
    K1, K2 = wl.rbf_factor(x1, l1), wl.rbf_factor(x2, l2)
    e1, e2, es = exact.gp_gradient(K1, K2, s2, y)
    ex = [float(np.sum(e1 * wl.rbf_factor_dell(x1, l1))),
          float(np.sum(e2 * wl.rbf_factor_dell(x2, l2))), es]
    for a, b in zip(g, ex):
        assert abs(a - b) <= 0.2 * abs(b) + 5.0


@pytest.mark.parametrize("prec", ["mixed"])
def test_matvec_mixed_large_factors(cola, ctx, prec):
    """1024 x 1024 factors (output columns in chunks, K streamed) against rows
    of the operator computed one by one."""
    n = 1024
    x1 = wl.uniform(wl.substream(5, 1), (n,))
    x2 = wl.uniform(wl.substream(5, 2), (64,))
    K1, K2 = wl.rbf_factor(x1, 0.1), wl.rbf_factor(x2, 0.2)
    spec = ("sum", [("kron", [("dense", K1), ("dense", K2)]), ("scalar", 0.1, n * 64)], None)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV)
    X = wl.normal(wl.substream(5, 3), (3, n * 64))
    Y = cola.cola_matvec(ctx, op, torch.tensor(X, dtype=torch.float32, device=DEV),
                         cola.PREC_MIXED, split_terms=3).double().cpu().numpy()
    idx = np.random.default_rng(9).integers(0, n * 64, 50)
    for r in range(3):
        Xr = X[r].reshape(n, 64)
        for I in idx:
            i1, i2 = I // 64, I % 64
            row = np.outer(K1[i1], K2[i2])
            ref = float(np.sum(row * Xr)) + 0.1 * Xr[i1, i2]
            bound = float(np.sum(row * np.abs(Xr))) + 0.1 * abs(Xr[i1, i2])
            assert abs(Y[r, I] - ref) <= 1e-5 * bound


def test_gp_full_scale_mixed(cola, ctx):
    """The differentiation workload at full size: two 1024-point RBF factors
    (l1 = 0.1, l2 = 0.2, sigma^2 = 0.1, N = 1,048,576), y and 32 Rademacher
    probes solved as one 33-RHS block to 1e-8 (MIXED + FP64 refinement), and
    the gradient in (l1, l2, sigma^2) against the oracle's evaluation of the
    same estimator."""
    w = wl.config5()
    x1, x2 = w.points
    l1, l2 = w.ells
    opts = cola.cola_cg_opts_default(precision=cola.PREC_MIXED, refine=1, tol=1e-8,
                                     maxiter=60000)
    g = _gp_gpu(cola, ctx, x1, x2, w.y, w.Z, l1, l2, w.sigma2, opts, slq_steps=30)
    ref = _gp_oracle_same_probes(x1, x2, w.y, w.Z, l1, l2, w.sigma2)
    np.testing.assert_allclose(g, ref, rtol=2e-4)
