"""The Kronecker eigen-structured solve and log-determinant (cola_kron_eig_*,
Table 3 Inverse / Eigs / LogDet rules) against the FP64 oracle.

Referees: dense LU and dense Cholesky at N = 4096 (independent of any
eigendecomposition), the oracle's eigen-based exact solve and log-det at
N = 2^21, and the true residual computed by the oracle's MVM."""
import numpy as np
import pytest

import workloads as wl
from oracle import exact, krylov
from oracle import linop as O
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


def _spec(factors, shift, N, coeffs=None):
    return ("sum", [("kron", [("dense", f) for f in factors]), ("scalar", shift, N)], coeffs)


def _residual_bound(factors, shift, X, B, u):
    """Rounding level of a computed solution's residual: evaluating b - A x and
    rounding x itself each leave about (sum_k n_k) u |A| |x| per entry, so
    ||b - A x|| / ||b|| is bounded by 4 (sum_k n_k) u || |A| |x| || / ||b||."""
    N = B.shape[1]
    absA = O.Sum([O.Kron([O.Dense(np.abs(f)) for f in factors]),
                  O.Diag(np.float64(abs(shift)), N)])
    AX = absA.mvm(np.abs(X))
    nk = sum(f.shape[0] for f in factors)
    return 4.0 * nk * u * np.linalg.norm(AX, axis=1) / np.linalg.norm(B, axis=1)


def test_eig_solve_and_logdet_config1_vs_dense(cola, ctx):
    """K1 (x) K2 + 0.1 I, 64-point factors (N = 4096): FP64 direct solve against
    dense LU, log-det against dense Cholesky."""
    w = wl.config1()
    spec = _spec(w.factors, w.shift, w.N)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV)
    X = cola.cola_kron_eig_solve(ctx, op, torch.tensor(w.B, device=DEV), cola.PREC_F64)
    Ad = oracle_tree(spec).dense()
    ref = exact.dense_solve(Ad, w.B)
    Xh = X.cpu().numpy()
    assert np.abs(Xh - ref).max() <= 1e-11 * np.abs(ref).max()
    res = krylov.true_relative_residual(oracle_tree(spec), w.B, Xh)
    assert np.all(res <= _residual_bound(w.factors, w.shift, Xh, w.B, 2.0 ** -53)), res
    ld = cola.cola_kron_eig_logdet(ctx, op)
    ld_ref = exact.cholesky_logdet(Ad)
    assert abs(ld - ld_ref) <= 1e-11 * abs(ld_ref)


def test_eig_solve_kron3_full_size(cola, ctx):
    """K1 (x) K2 (x) K3 + 0.01 I, three 128-point factors (N = 2^21, kappa 3.2e6):
    FP64 and FP32 direct solves against the oracle's exact solve, and the log-det."""
    w = wl.config2(nrhs=2)
    spec = _spec(w.factors, w.shift, w.N)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV)
    ref = exact.kron_shift_solve(w.factors, w.shift, w.B)
    X64 = cola.cola_kron_eig_solve(ctx, op, torch.tensor(w.B, device=DEV), cola.PREC_F64)
    X64 = X64.cpu().numpy()
    # forward error within ~kappa * u (orthogonal transforms, one division per entry)
    assert np.abs(X64 - ref).max() <= 1e-8 * np.abs(ref).max()
    res = krylov.true_relative_residual(oracle_tree(spec), w.B, X64)
    assert np.all(res <= _residual_bound(w.factors, w.shift, X64, w.B, 2.0 ** -53)), res
    assert np.all(res <= 1e-8)  # the accuracy the CG path is asked for
    X32 = cola.cola_kron_eig_solve(ctx, op, torch.tensor(w.B, dtype=torch.float32, device=DEV),
                                   cola.PREC_F32).double().cpu().numpy()
    # FP32 mode products: the same bound at FP32 unit roundoff
    res32 = krylov.true_relative_residual(oracle_tree(spec), w.B, X32)
    assert np.all(res32 <= _residual_bound(w.factors, w.shift, X32, w.B, 2.0 ** -24)), res32
    ld = cola.cola_kron_eig_logdet(ctx, op)
    ld_ref = exact.kron_shift_logdet(w.factors, w.shift)
    assert abs(ld - ld_ref) <= 1e-10 * abs(ld_ref)


def test_eig_solve_coefficients_and_fp32_factors(cola, ctx):
    """Sum coefficients (2 Kron + 0.5 s I) and factors stored in FP32."""
    K1, K2 = wl.config1().factors
    K1 = K1.astype(np.float32).astype(np.float64)
    K2 = K2.astype(np.float32).astype(np.float64)
    N = K1.shape[0] * K2.shape[0]
    B = wl.normal(wl.substream(11, 3), (3, N))
    spec = _spec([K1, K2], 0.1, N, [2.0, 0.5])
    op = gpu_tree(cola, ctx, spec, torch.float32, DEV)
    X = cola.cola_kron_eig_solve(ctx, op, torch.tensor(B, device=DEV), cola.PREC_F64)
    s = 0.5 * float(np.float32(0.1))  # the shift as stored (FP32 leaf)
    ref = exact.kron_shift_solve([2.0 * K1, K2], s, B)
    assert np.abs(X.cpu().numpy() - ref).max() <= 1e-11 * np.abs(ref).max()
    ld = cola.cola_kron_eig_logdet(ctx, op)
    assert abs(ld - exact.kron_shift_logdet([2.0 * K1, K2], s)) <= 1e-11 * abs(ld)


def test_eig_path_rejects_what_it_cannot_diagonalise(cola, ctx):
    K1, K2 = wl.config1().factors
    N = K1.shape[0] * K2.shape[0]
    d = wl.uniform(wl.substream(12, 1), (N,)) + 0.5
    op = gpu_tree(cola, ctx, ("sum", [("kron", [("dense", K1), ("dense", K2)]), ("diag", d)], None),
                  torch.float64, DEV)
    B = torch.ones(1, N, dtype=torch.float64, device=DEV)
    with pytest.raises(cola.ColaError, match="UNSUPPORTED"):
        cola.cola_kron_eig_solve(ctx, op, B, cola.PREC_F64)
    A = K1.copy()
    A[0, 1] += 1e-3  # not symmetric
    op2 = gpu_tree(cola, ctx, ("kron", [("dense", A), ("dense", K2)]), torch.float64, DEV)
    with pytest.raises(cola.ColaError, match="INVALID_ARG"):
        cola.cola_kron_eig_solve(ctx, op2, B, cola.PREC_F64)


@pytest.mark.parametrize("kind", ["kron", "kronsum"])
def test_kron_eigs_small_dense(cola, ctx, kind):
    """cola_kron_eigs (Table 3 Eigs rule) on 2.5 * (K1 op K2) + 0.3 I with op
    the Kronecker product or sum of a 7 x 7 and a 9 x 9 symmetric factor:
    the N = 63 eigenvalues equal the dense matrix's (LAPACK eigvalsh, no
    Kronecker structure used), each factor pair satisfies K V = V diag(w) with
    orthonormal V, and column (i, j) of V1 (x) V2 is an eigenvector of A with
    the eigenvalue at flat index i n2 + j."""
    r = np.random.default_rng(31)
    M1, M2 = r.standard_normal((7, 7)), r.standard_normal((9, 9))
    K1, K2 = M1 @ M1.T / 7 + 0.2 * np.eye(7), M2 @ M2.T / 9 + 0.1 * np.eye(9)
    spec = ("sum", [(kind, [("dense", K1), ("dense", K2)]), ("scalar", 0.3, 63)], [2.5, 1.0])
    ref = oracle_tree(spec)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV)
    ws, Vs, ev = cola.cola_kron_eigs(ctx, op)
    ev = ev.cpu().numpy()
    np.testing.assert_allclose(np.sort(ev), np.linalg.eigvalsh(ref.dense()), rtol=1e-12,
                               atol=1e-12)
    for K, w, V in zip((K1, K2), ws, Vs):
        w, V = w.cpu().numpy(), V.cpu().numpy()
        np.testing.assert_allclose(K @ V, V * w, atol=1e-12)
        np.testing.assert_allclose(V.T @ V, np.eye(len(w)), atol=1e-13)
    V1, V2 = Vs[0].cpu().numpy(), Vs[1].cpu().numpy()
    for i, j in [(0, 0), (3, 5), (6, 8)]:
        q = np.kron(V1[:, i], V2[:, j])
        np.testing.assert_allclose(ref @ q, ev[i * 9 + j] * q, atol=1e-11)


def test_kron_eigs_full_size(cola, ctx):
    """At the 128^3 workload the 2,097,152 eigenvalues equal the oracle's
    (products of the factors' LAPACK eigenvalues plus the shift), as sets."""
    w = wl.config2(nrhs=1)
    op = gpu_tree(cola, ctx, _spec(w.factors, w.shift, w.N), torch.float64, DEV)
    _, _, ev = cola.cola_kron_eigs(ctx, op)
    ref = np.sort(exact.kron_eigenvalues(w.factors, w.shift))
    got = np.sort(ev.cpu().numpy())
    np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-12 * ref.max())
