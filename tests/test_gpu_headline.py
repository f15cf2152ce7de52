"""Oracle parity at the full 128^3 workload the bench times:
A = K1 (x) K2 (x) K3 + 0.01 I, three 128-point RBF factors (l = 0.1),
N = 2,097,152.

* Unpreconditioned MIXED CG (3 x 3 split-BF16 terms, FP32 recurrences, FP64
  reliable updates) to 1e-8 on 2 right-hand sides: the oracle's FP64 true
  residual ||b - A x|| / ||b|| is <= 1e-8 for each, and the forward error
  against the exact eigen-structured solve (Table 3 Inverse rule) is within
  the bound kappa * tol.
* Lanczos for SLQ (Table 5; App. A.2 LogDet = Tr log) in F32 and MIXED on the
  same Rademacher probes as the FP64 oracle (no reorthogonalisation on either
  side), 2 probes x 100 steps.  Tolerances (from a CPU run of FP32 against
  FP64 Lanczos on this operator):
    - alpha_j, beta_j for j < 12 within 1e-5 relative: while the basis is
      still orthogonal the coefficients are a well-conditioned function of the
      operator and probe, and single-precision rounding (measured drift
      <= 1e-6 up to j = 15) stays far below 1e-5.  From j ~ 20 on, loss of
      orthogonality (the top Ritz value converges first) makes FP32 and FP64
      sequences diverge entry by entry; even FP64 with and without
      reorthogonalisation differ by tens of percent from j ~ 40.
    - the per-probe Gauss quadrature ||z||^2 e_1^T log(T_m) e_1 within 5e-3
      relative of the oracle's: finite-precision Lanczos is exact Lanczos on
      a nearby operator, so the quadrature stays close although the
      coefficients do not (measured FP32 vs FP64 gap 1.2e-3, below the m = 100
      quadrature bias of ~6e-3 against the exact log-det).
    - no Ritz value is clamped (3 x 3 split terms keep A positive definite in
      working precision).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import exact, krylov, rng
from tests._trees import gpu_tree, oracle_tree

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda"
M_STEPS = 100
N_PROBES = 2
J_EARLY = 12


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
def work():
    w = wl.config2(nrhs=2)
    spec = ("sum", [("kron", [("dense", f) for f in w.factors]), ("scalar", w.shift, w.N)], None)
    return w, spec


@pytest.fixture(scope="module")
def oracle_lanczos(work):
    """The oracle's Lanczos (FP64, no reorthogonalisation) on the bench's
    first two SLQ probes, and its per-probe quadrature values."""
    w, spec = work
    ref = oracle_tree(spec)
    seed = wl.substream(w.seed, 2)
    Z = rng.rademacher_probes(seed, N_PROBES, w.N)
    out = []
    for v in range(N_PROBES):
        a, b, _ = krylov.lanczos(ref, Z[v], M_STEPS, reorth=False)
        out.append((a, b, krylov.quadrature_logdet_from_tridiag(a, b, float(Z[v] @ Z[v]))))
    return seed, Z, out


def test_cg_mixed_full_size_unpreconditioned(cola, ctx, work):
    w, spec = work
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    opts = cola.cola_cg_opts_default(precision=cola.PREC_MIXED, refine=1, tol=w.tol,
                                     maxiter=60000, split_factor_terms=3, split_vector_terms=3)
    X, info, st = cola.cola_cg_solve(ctx, op, torch.tensor(w.B, device=DEV), opts)
    assert st == 0, info
    Xh = X.cpu().numpy()
    res = krylov.true_relative_residual(oracle_tree(spec), w.B, Xh)
    assert np.all(res <= w.tol), res
    for i, r in zip(info, res):
        assert i["rel_residual"] <= w.tol and i["updates"] >= 1
        # the residual the library reports is its FP64 true residual at the
        # returned x: it agrees with the oracle's
        assert abs(i["rel_residual"] - r) <= 0.05 * max(i["rel_residual"], r)
    x_ref = exact.kron_shift_solve(w.factors, w.shift, w.B)
    lam = exact.kron_eigenvalues(w.factors, w.shift)
    kappa = lam.max() / lam.min()
    fe = np.linalg.norm(Xh - x_ref, axis=1) / np.linalg.norm(x_ref, axis=1)
    assert np.all(fe <= kappa * w.tol), (fe, kappa)


@pytest.mark.parametrize("prec", ["f32", "mixed"])
def test_lanczos_full_size_matches_oracle(cola, ctx, work, oracle_lanczos, prec):
    w, spec = work
    seed, Z, ref = oracle_lanczos
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    P = cola.PREC_F32 if prec == "f32" else cola.PREC_MIXED
    Zd = torch.tensor(Z, dtype=torch.float32, device=DEV)
    al, be, me = cola.cola_lanczos(ctx, op, Zd, M_STEPS, P, reorth=0, split_terms=3)
    al, be, me = al.cpu().numpy(), be.cpu().numpy(), me.cpu().numpy()
    for v in range(N_PROBES):
        a, b, _ = ref[v]
        assert me[v] == M_STEPS == len(a)
        np.testing.assert_allclose(al[v, :J_EARLY], a[:J_EARLY], rtol=1e-5)
        np.testing.assert_allclose(be[v, :J_EARLY], b[:J_EARLY], rtol=1e-5)
    # the SLQ path on the same probes: per-probe quadrature and no clamping
    ld, se, pp, clamped = cola.cola_slq_logdet(ctx, op, N_PROBES, M_STEPS, probes=Zd,
                                               precision=P, split_terms=3)
    pp = pp.cpu().numpy()
    q_ref = np.array([r[2] for r in ref])
    np.testing.assert_allclose(pp, q_ref, rtol=5e-3)
    assert clamped == 0
    assert abs(ld - q_ref.mean()) <= 5e-3 * abs(q_ref.mean())


def test_slq_mixed_seeded_probes_match_given_probes(cola, ctx, work, oracle_lanczos):
    """Probes drawn on the device from the seed are the oracle's SplitMix64
    Rademacher probes: the seeded call gives the same per-probe values as the
    call with the probes passed in."""
    w, spec = work
    seed, Z, _ = oracle_lanczos
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    _, _, pp_seed, _ = cola.cola_slq_logdet(ctx, op, N_PROBES, 20, seed=seed,
                                            precision=cola.PREC_MIXED, split_terms=3)
    _, _, pp_given, _ = cola.cola_slq_logdet(
        ctx, op, N_PROBES, 20, probes=torch.tensor(Z, dtype=torch.float32, device=DEV),
        precision=cola.PREC_MIXED, split_terms=3)
    assert torch.equal(pp_seed, pp_given)
