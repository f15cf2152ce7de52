"""CG with re-orthogonalised residuals (the low-precision CG variant Sec. 3.4 /
App. C.3 cite; cola_cg_opts.reorth_residuals) against the oracle's
cg_reorth_residuals.

Workload: K1 (x) K2 + 1e-3 I with 64- and 48-point RBF factors (l = 0.2,
N = 3072, kappa ~ 1e4, clustered small eigenvalues), 2 right-hand sides.
* FP64: the solution matches the oracle's to 1e-9 and the iteration counts
  agree within 1 (the same recursion up to rounding order).
* MIXED (3 x 3 split-BF16 tensor-core MVM, FP32 vectors), no refinement, the
  recursion run until its residual meets 1e-5 (max_updates = 0: no
  verify-and-continue on the true residual, which FP32 cannot bring below
  about u kappa here): the re-orthogonalised solve takes within a few
  iterations of the oracle's FP64 count (exact arithmetic up to rounding), at
  most half the plain MIXED CG's count on the same system, and its true
  residual (oracle MVM) is within the FP32 floor max(tol, 10 u kappa)
  (Higham ch. 12).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import exact, krylov
from tests._trees import gpu_tree, oracle_tree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda"


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


@pytest.fixture(scope="module")
def problem():
    x1 = wl.uniform(wl.substream(77, 1), (64,))
    x2 = wl.uniform(wl.substream(77, 2), (48,))
    F = [wl.rbf_factor(x1, 0.2), wl.rbf_factor(x2, 0.2)]
    spec = ("sum", [("kron", [("dense", f) for f in F]), ("scalar", 1e-3, 64 * 48)], None)
    B = wl.normal(wl.substream(77, 3), (2, 64 * 48))
    lam = exact.kron_eigenvalues(F, 1e-3)
    return F, spec, B, lam.max() / lam.min()


def test_reorth_cg_fp64_matches_oracle(cola, ctx, problem):
    F, spec, B, _ = problem
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    opts = cola.cola_cg_opts_default(precision=cola.PREC_F64, refine=0, tol=1e-8, maxiter=2000,
                                     reorth_residuals=600, graph_chunk=16)
    X, info, st = cola.cola_cg_solve(ctx, op, torch.tensor(B, device=DEV), opts)
    assert st == 0
    ref = oracle_tree(spec)
    for r in range(2):
        x_ref, it_ref, _ = krylov.cg_reorth_residuals(ref, B[r], tol=1e-8, maxiter=2000)
        assert abs(info[r]["iterations"] - it_ref) <= 1
        np.testing.assert_allclose(X[r].cpu().numpy(), x_ref, rtol=0,
                                   atol=1e-9 * np.max(np.abs(x_ref)))


def test_reorth_cg_mixed_tracks_exact_arithmetic(cola, ctx, problem):
    F, spec, B, kappa = problem
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    B32 = torch.tensor(B, dtype=torch.float32, device=DEV)
    common = dict(precision=cola.PREC_MIXED, refine=0, tol=1e-5, maxiter=5000, graph_chunk=16,
                  split_factor_terms=3, split_vector_terms=3, max_updates=0)
    X, info, st = cola.cola_cg_solve(ctx, op, B32,
                                     cola.cola_cg_opts_default(reorth_residuals=600, **common),
                                     raise_on_error=False)
    assert st in (0, 5)  # 5: the FP32 true residual sits above tol (checked below)
    Xp, info_p, st_p = cola.cola_cg_solve(ctx, op, B32, cola.cola_cg_opts_default(**common),
                                          raise_on_error=False)
    ref = oracle_tree(spec)
    res = krylov.true_relative_residual(ref, B, X.double().cpu().numpy())
    assert np.all(res <= max(1e-5, 10 * 2.0 ** -24 * kappa)), res
    for r in range(2):
        _, it_ref, _ = krylov.cg_reorth_residuals(ref, B[r], tol=1e-5, maxiter=5000)
        assert abs(info[r]["iterations"] - it_ref) <= 5, (info[r], it_ref)
        assert info[r]["iterations"] * 2 <= info_p[r]["iterations"], (info[r], info_p[r])


def test_reorth_cg_rejects_refinement_and_preconditioning(cola, ctx, problem):
    _, spec, B, _ = problem
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    for kw in (dict(refine=1), dict(refine=0, jacobi=1)):
        opts = cola.cola_cg_opts_default(precision=cola.PREC_MIXED, reorth_residuals=50, **kw)
        Bt = torch.tensor(B, dtype=torch.float64 if kw.get("refine") else torch.float32,
                          device=DEV)
        with pytest.raises(cola.ColaError) as e:
            cola.cola_cg_solve(ctx, op, Bt, opts)
        assert e.value.status == 1
