"""Pins for the FP64 oracle: checks against facts the paper and mathematics fix.

Nothing here trusts the oracle against itself.  Each pin compares an oracle
routine with an independent referee: a brute-force loop over the definition,
a closed form, a LAPACK routine solving a different formulation, or an
invariant.  The ``planted`` tests swap a plausible mistake into the oracle on
the CPU and check that some pin catches it.
"""
import math
import os

import numpy as np
import pytest

from oracle import exact, grad, krylov, rng, stochastic
from oracle.linop import (Dense, Diag, Kron, KronSum, LowRank, Product, Sum,
                          derivative)
import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rs(seed):
    return np.random.default_rng(seed)


def _spd(n, seed, shift=0.5):
    M = _rs(seed).standard_normal((n, n))
    return M @ M.T / n + shift * np.eye(n)


# ---------------------------------------------------------------------------
# Kronecker MVM (Sec. 3.2, Table 3)
# ---------------------------------------------------------------------------

def kron_bruteforce(mats):
    """Entry ((i_1..i_d),(j_1..j_d)) = prod_k M_k[i_k, j_k] by explicit loops."""
    rows = [m.shape[0] for m in mats]
    cols = [m.shape[1] for m in mats]
    out = np.zeros((int(np.prod(rows)), int(np.prod(cols))))
    for I, ii in enumerate(np.ndindex(*rows)):
        for J, jj in enumerate(np.ndindex(*cols)):
            v = 1.0
            for m, a, b in zip(mats, ii, jj):
                v *= m[a, b]
            out[I, J] = v
    return out


def test_kron_dense_matches_bruteforce_rectangular():
    r = _rs(1)
    mats = [r.standard_normal((2, 3)), r.standard_normal((3, 2)), r.standard_normal((2, 2))]
    op = Kron([Dense(m) for m in mats])
    np.testing.assert_allclose(op.dense(), kron_bruteforce(mats), rtol=0, atol=1e-13)
    np.testing.assert_allclose(op.dense(), np.kron(np.kron(mats[0], mats[1]), mats[2]),
                               rtol=0, atol=1e-13)


def test_kron_2x2_worked_by_hand():
    # A (x) B for A = [[1,2],[3,4]], B = [[0,1],[1,0]]: block (i,j) is A_ij * B.
    A = np.array([[1.0, 2.0], [3.0, 4.0]])
    B = np.array([[0.0, 1.0], [1.0, 0.0]])
    expect = np.array([[0, 1, 0, 2],
                       [1, 0, 2, 0],
                       [0, 3, 0, 4],
                       [3, 0, 4, 0]], dtype=float)
    np.testing.assert_array_equal(Kron([Dense(A), Dense(B)]).dense(), expect)
    # and applied to x = (1, 2, 3, 4): A X B^T with X = [[1,2],[3,4]]
    np.testing.assert_array_equal(Kron([Dense(A), Dense(B)]) @ np.array([1.0, 2, 3, 4]),
                                  np.array([2.0 + 8, 1 + 6, 6 + 16, 3 + 12]))


def kron_vec_identity_error(op_factory, square=False):
    r = _rs(2)
    A = r.standard_normal((3, 3) if square else (4, 3))
    B = r.standard_normal((2, 2) if square else (5, 2))
    X = r.standard_normal((3, 2))
    y = op_factory([Dense(A), Dense(B)]) @ X.ravel()
    e1 = np.max(np.abs(y - (A @ X @ B.T).ravel()))                 # row-major vec
    e2 = np.max(np.abs(y - (B @ X.T @ A.T).ravel(order="F")))      # column-major vec(B X' A^T)
    return max(e1, e2)


def test_kron_vec_identities():
    assert kron_vec_identity_error(Kron) < 1e-13
    assert kron_vec_identity_error(Kron, square=True) < 1e-13


def test_kron_eigenvalues_are_products():
    """App. A.1.2: Eigs(A (x) B) = Lambda_A (x) Lambda_B."""
    mats = [_spd(3, 3), _spd(4, 4), _spd(2, 5)]
    dense = Kron([Dense(m) for m in mats]).dense()
    ev = np.sort(np.linalg.eigvalsh(dense))
    np.testing.assert_allclose(np.sort(exact.kron_eigenvalues(mats)), ev, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(np.sort(exact.kron_eigenvalues(mats, 0.3)), ev + 0.3, rtol=1e-12)


# ---------------------------------------------------------------------------
# Kronecker sum with the Dirichlet Laplacian: closed-form eigenpairs
# ---------------------------------------------------------------------------

def laplacian_eigpairs(n):
    k = np.arange(1, n + 1)
    lam = 2.0 - 2.0 * np.cos(k * math.pi / (n + 1))
    i = np.arange(1, n + 1)
    S = np.sin(np.outer(i, k) * math.pi / (n + 1))
    S /= np.linalg.norm(S, axis=0)
    return lam, S


def test_laplacian_closed_form():
    n = 7
    L = wl.dirichlet_laplacian(n)
    lam, S = laplacian_eigpairs(n)
    np.testing.assert_allclose(L @ S, S * lam, atol=1e-13)
    np.testing.assert_allclose(Dense(L) @ S[:, 2], lam[2] * S[:, 2], atol=1e-13)


def test_kronsum_eigenpairs():
    """App. A.1.2: Eigs(A (+) B) = Lambda_A (+) Lambda_B with vectors V_A (x) V_B."""
    n1, n2 = 5, 6
    L1, L2 = wl.dirichlet_laplacian(n1), wl.dirichlet_laplacian(n2)
    l1, S1 = laplacian_eigpairs(n1)
    l2, S2 = laplacian_eigpairs(n2)
    op = KronSum([Dense(L1), Dense(L2)])
    for i in range(n1):
        for j in range(n2):
            v = np.kron(S1[:, i], S2[:, j])
            np.testing.assert_allclose(op @ v, (l1[i] + l2[j]) * v, atol=1e-12)


def test_kronsum_three_factors_definition():
    r = _rs(6)
    mats = [r.standard_normal((n, n)) for n in (2, 3, 2)]
    I = [np.eye(m.shape[0]) for m in mats]
    expect = (np.kron(np.kron(mats[0], I[1]), I[2]) + np.kron(np.kron(I[0], mats[1]), I[2])
              + np.kron(np.kron(I[0], I[1]), mats[2]))
    np.testing.assert_allclose(KronSum([Dense(m) for m in mats]).dense(), expect, atol=1e-13)


# ---------------------------------------------------------------------------
# Diag rules (App. A.1.4) and transpose rules (App. A.1.5)
# ---------------------------------------------------------------------------

def _zoo():
    r = _rs(7)
    A, B, C = r.standard_normal((3, 3)), r.standard_normal((4, 4)), r.standard_normal((2, 2))
    U, V = r.standard_normal((12, 2)), r.standard_normal((12, 2))
    d = r.standard_normal(12)
    return [
        Kron([Dense(A), Dense(B)]),
        KronSum([Dense(A), Dense(B)]),
        Kron([Dense(A), Diag(np.array([1.0, -2.0, 0.5, 3.0]))]),
        Sum([Kron([Dense(A), Dense(B)]), Diag(0.25, 12), LowRank(U, V), Diag(d)], [1.0, 2.0, -0.5, 1.5]),
        Sum([KronSum([Dense(A), Dense(B)]), Diag(d), LowRank(U)]),
        Product([Kron([Dense(A), Dense(B)]), Sum([Diag(d), LowRank(U, V)])]),
        Kron([Dense(C), Dense(A), Dense(C)]),
    ]


@pytest.mark.parametrize("k", range(7))
def test_diag_rules_match_bruteforce(k):
    op = _zoo()[k]
    np.testing.assert_allclose(op.diag(), op.diag_bruteforce(), atol=1e-12)


@pytest.mark.parametrize("k", range(7))
def test_transpose_rules_inner_product(k):
    op = _zoo()[k]
    r = _rs(8)
    u = r.standard_normal(op.rows)
    v = r.standard_normal(op.cols)
    lhs = u @ (op @ v)
    rhs = (op.transpose() @ u) @ v
    assert abs(lhs - rhs) < 1e-11 * (1 + abs(lhs))
    np.testing.assert_allclose(op.transpose().dense(), op.dense().T, atol=1e-12)


def test_woodbury_low_rank_plus_diagonal():
    """(D + U U^T)^-1 = D^-1 - D^-1 U (I + U^T D^-1 U)^-1 U^T D^-1 (App. A.1.1)."""
    r = _rs(9)
    n, k = 20, 3
    d = 0.5 + r.random(n)
    U = r.standard_normal((n, k)) / math.sqrt(n)
    b = r.standard_normal(n)
    op = Sum([Diag(d), LowRank(U)])
    Dinv_b = b / d
    Dinv_U = U / d[:, None]
    core = np.eye(k) + U.T @ Dinv_U
    x_wood = Dinv_b - Dinv_U @ np.linalg.solve(core, U.T @ Dinv_b)
    np.testing.assert_allclose(exact.dense_solve(op.dense(), b)[0], x_wood, rtol=1e-12)
    x_cg, _ = krylov.cg(op, b, tol=1e-13, maxiter=200)
    np.testing.assert_allclose(x_cg, x_wood, rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------------------
# Solves: CG vs dense LU, exact Kronecker solve vs dense
# ---------------------------------------------------------------------------

def test_cg_matches_dense_lu():
    mats = [_spd(4, 11), _spd(5, 12)]
    op = Sum([Kron([Dense(m) for m in mats]), Diag(0.1, 20)])
    b = _rs(13).standard_normal(20)
    x_cg, it = krylov.cg(op, b, tol=1e-13, maxiter=200)
    x_lu = exact.dense_solve(op.dense(), b)[0]
    np.testing.assert_allclose(x_cg, x_lu, rtol=1e-10)
    assert it <= 40


def test_cg_reorth_residuals_fp64_is_cg():
    """In FP64 on a well-conditioned operator the re-orthogonalised CG takes
    the textbook CG's iterations (exact-arithmetic CG residuals are already
    orthogonal) and solves the system (dense LU)."""
    mats = [_spd(4, 11), _spd(5, 12)]
    op = Sum([Kron([Dense(m) for m in mats]), Diag(0.1, 20)])
    b = _rs(13).standard_normal(20)
    x_cg, it = krylov.cg(op, b, tol=1e-12, maxiter=200)
    x_ro, it_ro, R = krylov.cg_reorth_residuals(op, b, tol=1e-12, maxiter=200)
    # n = 20: exact-arithmetic CG ends within 20 steps; the textbook
    # recursion may need one more to absorb rounding
    assert it_ro <= 20 and abs(it_ro - it) <= 1 and R.shape == (it_ro + 1, 20)
    np.testing.assert_allclose(x_ro, x_cg, rtol=1e-9)
    np.testing.assert_allclose(x_ro, exact.dense_solve(op.dense(), b)[0], rtol=1e-9)


def test_cg_reorth_residuals_keeps_them_orthogonal_in_fp32():
    """The point of the variant: in FP32 the residuals it uses stay mutually
    orthogonal to rounding level (|cos| <= 1e-5) on an ill-conditioned RBF
    operator (kappa ~ 1e4, clustered small eigenvalues), so it takes within a
    few iterations of the FP64 re-orthogonalised count (exact arithmetic up to
    rounding), while even FP64 textbook CG, whose residuals lose
    orthogonality, needs several times more; the FP32 solution meets the
    tolerance against a dense LU solve."""
    x = wl.uniform(5, (24,))
    y = wl.uniform(6, (20,))
    op = Sum([Kron([Dense(wl.rbf_factor(x, 0.2)), Dense(wl.rbf_factor(y, 0.2))]),
              Diag(1e-3, 480)])
    b = _rs(15).standard_normal(480)
    _, it64 = krylov.cg(op, b, tol=1e-5, maxiter=2000)
    _, it64_ro, _ = krylov.cg_reorth_residuals(op, b, tol=1e-5, maxiter=2000)
    x32, it32, R = krylov.cg_reorth_residuals(op, b, tol=1e-5, maxiter=2000, dtype=np.float32)
    Q = R.astype(np.float64)
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    G = Q @ Q.T - np.eye(len(Q))
    assert np.max(np.abs(G)) <= 1e-5
    assert abs(it32 - it64_ro) <= 3
    assert it64 >= 2 * it64_ro
    # the true residual of an FP32 recursion stalls near u kappa (Higham,
    # Accuracy and Stability, ch. 12), above the recursive 1e-5
    lam = np.linalg.eigvalsh(op.dense())
    kappa = lam.max() / lam.min()
    u32 = 2.0 ** -24
    res = np.linalg.norm(b - op @ x32) / np.linalg.norm(b)
    assert res <= max(1e-5, 10 * u32 * kappa)


def test_jacobi_pcg_matches_dense_lu():
    n = 6
    L = wl.dirichlet_laplacian(n)
    r = _rs(14)
    d = 0.5 + r.random(n * n)
    U = r.standard_normal((n * n, 2)) / n
    op = Sum([KronSum([Dense(L), Dense(L)]), Diag(d), LowRank(U)])
    b = r.standard_normal(n * n)
    x, _ = krylov.cg(op, b, tol=1e-13, maxiter=500, precond_diag=op.diag())
    np.testing.assert_allclose(x, exact.dense_solve(op.dense(), b)[0], rtol=1e-9)


def _kron_precond(factors, d):
    """M^-1 for M = (x)_k K_k + mean(d) I by the exact Kronecker solve."""
    s = float(np.mean(d))
    return lambda r: exact.kron_shift_solve(factors, s, r)[0]


def test_pcg_with_exact_preconditioner_takes_one_step():
    """M = A: the first search direction is A^-1 b, so CG ends after one step."""
    mats = [_spd(5, 21), _spd(7, 22)]
    d = np.full(35, 0.3)
    op = Sum([Kron([Dense(m) for m in mats]), Diag(d)])
    b = _rs(23).standard_normal(35)
    x, it = krylov.cg(op, b, tol=1e-12, maxiter=50, precond=_kron_precond(mats, d))
    assert it == 1
    np.testing.assert_allclose(x, exact.dense_solve(op.dense(), b)[0], rtol=1e-11)


def test_kron_mean_shift_pcg_meets_condition_number_bound():
    """A = K_1 (x) K_2 + Diag(d), M = K_1 (x) K_2 + mean(d) I.  The Rayleigh
    quotient x^T A x / x^T M x lies between min(1, d_min/mean) and
    max(1, d_max/mean), so kappa(M^-1 A) <= d_max / d_min, and the PCG error
    contracts by rho = (sqrt(kappa) - 1) / (sqrt(kappa) + 1) per step in the A
    norm.  With ||r|| <= sqrt(lambda_max(A)) ||e||_A the relative residual
    after k steps is at most 2 rho^k sqrt(kappa(A)): the iteration count may
    not exceed the k where that reaches tol (+2 for rounding)."""
    w = wl.kron_diag("pin", [12, 15], [0.2, 0.2], 0.05, 0.15, 1, 1e-10, 31)
    d = w.extra["d"]
    op = Sum([Kron([Dense(f) for f in w.factors]), Diag(d)])
    b = w.B[0]
    x, it = krylov.cg(op, b, tol=1e-10, maxiter=500, precond=_kron_precond(w.factors, d))
    np.testing.assert_allclose(x, exact.dense_solve(op.dense(), b)[0], rtol=1e-8)
    ev = np.linalg.eigvalsh(op.dense())
    kappa = d.max() / d.min()
    rho = (math.sqrt(kappa) - 1) / (math.sqrt(kappa) + 1)
    bound = math.ceil(math.log(2 * math.sqrt(ev[-1] / ev[0]) / 1e-10) / math.log(1 / rho))
    assert it <= bound + 2, (it, bound)
    _, it_plain = krylov.cg(op, b, tol=1e-10, maxiter=2000)
    assert it_plain > 2 * it


def test_kronsum_eigenvalues_match_laplacian_closed_form():
    """L (+) L with L = tridiag(-1, 2, -1) of size n: eigenvalues
    (2 - 2 cos(i pi/(n+1))) + (2 - 2 cos(j pi/(n+1))) (textbook Dirichlet
    Laplacian spectrum)."""
    n = 9
    L = wl.dirichlet_laplacian(n)
    lam = 2.0 - 2.0 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
    closed = np.sort(np.add.outer(lam, lam).ravel())
    np.testing.assert_allclose(np.sort(exact.kronsum_eigenvalues([L, L])), closed, rtol=1e-13,
                               atol=1e-13)


def test_exact_kronsum_solve_matches_dense():
    mats = [_spd(4, 41), _spd(3, 42), _spd(5, 43)]
    op = Sum([KronSum([Dense(m) for m in mats]), Diag(0.3, 60)])
    B = _rs(44).standard_normal((2, 60))
    np.testing.assert_allclose(exact.kronsum_shift_solve(mats, 0.3, B),
                               exact.dense_solve(op.dense(), B), rtol=1e-10)


def test_product_split_solve_order():
    """A = A_1 A_2 with non-commuting Kronecker-sum factors: solving A_1 first,
    then A_2, matches dense LU of the product; the reversed order does not."""
    f1 = [_spd(4, 45), _spd(5, 46)]
    f2 = [_spd(4, 47), _spd(5, 48)]
    A1 = KronSum([Dense(m) for m in f1])
    A2 = Sum([KronSum([Dense(m) for m in f2]), Diag(0.2, 20)])
    B = _rs(49).standard_normal((2, 20))
    s1 = lambda X: exact.kronsum_shift_solve(f1, 0.0, X)
    s2 = lambda X: exact.kronsum_shift_solve(f2, 0.2, X)
    ref = exact.dense_solve(Product([A1, A2]).dense(), B)
    np.testing.assert_allclose(exact.product_split_solve([s1, s2], B), ref, rtol=1e-9)
    assert np.abs(exact.product_split_solve([s2, s1], B) - ref).max() > 1e-3 * np.abs(ref).max()


# ---------------------------------------------------------------------------
# Stochastic diagonal / trace estimators (Sec. 3.3, App. B.1)
# ---------------------------------------------------------------------------

def _hypercube(N):
    """All 2^N sign vectors, shape (2^N, N)."""
    idx = np.arange(2 ** N)[:, None]
    return np.where((idx >> np.arange(N)[None, :]) & 1, -1.0, 1.0)


def test_hutchinson_over_the_full_hypercube_is_exact():
    """Averaging z (.) A z over every sign vector gives Diag(A) exactly (the
    off-diagonal products z_k z_l cancel over the hypercube); the doubly
    stochastic form with a full hypercube per term gives Diag of the sum."""
    A1, A2 = _spd(4, 51), _rs(52).standard_normal((4, 4))
    A2 = A2 + A2.T
    Z = _hypercube(4)
    np.testing.assert_allclose(stochastic.hutchinson_diag(Dense(A1), Z), np.diag(A1),
                               rtol=1e-14, atol=1e-14)
    Zs = np.stack([Z, Z[::-1]])
    est = stochastic.doubly_stochastic_diag([Dense(A1), Dense(A2)], [0.5, 2.0], Zs)
    np.testing.assert_allclose(est, 0.5 * np.diag(A1) + 2.0 * np.diag(A2), rtol=1e-14,
                               atol=1e-14)


def test_rademacher_trace_variance_by_enumeration():
    """Var[z^T B z] over the uniform hypercube equals 2 sum_{k != l} B_kl^2."""
    B = _rs(53).standard_normal((5, 5))
    B = B + B.T
    Z = _hypercube(5)
    q = np.einsum("vk,kl,vl->v", Z, B, Z)
    assert abs(np.var(q) - stochastic.rademacher_trace_variance(B)) < 1e-10 * np.var(q)


def test_doubly_stochastic_trace_variance_statistics():
    """1500 independent draws on a sum of three Kronecker products of RBF
    factors (a multi-task kernel): the sample variances of the base and doubly
    stochastic trace estimates match their formulas within 15 %, and the doubly
    stochastic one is the smaller: with entrywise positive terms the cross
    terms 4 c_i c_k sum_{k != l} (A_i)_kl (A_k)_kl of the base variance are
    positive.  (For terms with off-diagonal entries of both signs they can be
    negative, and the doubly stochastic variance is then not always smaller.)"""
    r = _rs(59)
    terms_m = [np.kron(wl.rbf_factor(r.random(4), 0.2 + 0.2 * i),
                       wl.rbf_factor(r.random(5), 0.5 - 0.1 * i)) for i in range(3)]
    coeffs = [1.0, 0.5, 2.0]
    terms = [Dense(m) for m in terms_m]
    A = sum(c * m for c, m in zip(coeffs, terms_m))
    n, N, trials = 4, 20, 1500
    base, dbl = [], []
    for t in range(trials):
        Zs = stochastic.probes(1000 + t, 3, n, N)
        base.append(np.sum(stochastic.hutchinson_diag(Dense(A), Zs[0])))
        dbl.append(np.sum(stochastic.doubly_stochastic_diag(terms, coeffs, Zs)))
    v_base = stochastic.rademacher_trace_variance(A) / n
    v_dbl = sum(c * c * stochastic.rademacher_trace_variance(m)
                for c, m in zip(coeffs, terms_m)) / n
    assert abs(np.mean(base) - np.trace(A)) < 4 * np.sqrt(v_base / trials)
    assert abs(np.mean(dbl) - np.trace(A)) < 4 * np.sqrt(v_dbl / trials)
    assert abs(np.var(base) / v_base - 1) < 0.15
    assert abs(np.var(dbl) / v_dbl - 1) < 0.15
    assert v_dbl < 0.8 * v_base


# ---------------------------------------------------------------------------
# Householder Arnoldi (Algorithm 2)
# ---------------------------------------------------------------------------

def test_householder_arnoldi_relation_and_orthogonality():
    """Nonsymmetric A (30 x 30), 12 steps: Q has orthonormal columns, its first
    column is nu_0 / ||nu_0||, H is upper Hessenberg, and A Q_T = Q_{T+1} H."""
    r = _rs(80)
    A = r.standard_normal((30, 30))
    nu0 = r.standard_normal(30)
    H, Q = krylov.householder_arnoldi(Dense(A), nu0, 12)
    np.testing.assert_allclose(Q.T @ Q, np.eye(13), atol=1e-13)
    np.testing.assert_allclose(Q[:, 0], nu0 / np.linalg.norm(nu0), atol=1e-14)
    assert np.all(np.tril(H, -2) == 0.0)
    np.testing.assert_allclose(A @ Q[:, :12], Q @ H, atol=1e-12)


def test_householder_arnoldi_symmetric_is_lanczos():
    """Symmetric A: H is tridiagonal to rounding and its diagonal and
    sub-diagonal are Lanczos' alpha and beta (full reorthogonalisation) from
    the same start."""
    A = _spd(40, 81)
    z = _rs(82).standard_normal(40)
    H, _ = krylov.householder_arnoldi(Dense(A), z, 15)
    band = np.triu(np.tril(H, 1), -1)
    assert np.abs(H - band).max() < 1e-12 * np.abs(A).max()
    a, b, _ = krylov.lanczos(Dense(A), z, 15, reorth=True)
    np.testing.assert_allclose(np.diag(H[:15, :15]), a, rtol=1e-11, atol=1e-13)
    np.testing.assert_allclose(np.abs(np.diag(H, -1))[:14], b, rtol=1e-11)


def test_householder_vector_zeroes_the_tail():
    w = _rs(83).standard_normal(9)
    u = krylov.householder_vector(w, 3)
    h = w - 2.0 * u * (u @ w)
    np.testing.assert_allclose(h[:3], w[:3], atol=1e-15)
    assert abs(h[3] - np.linalg.norm(w[3:])) < 1e-14
    np.testing.assert_allclose(h[4:], 0.0, atol=1e-14)


def test_exact_kron_solve_matches_dense():
    mats = [_spd(3, 15), _spd(4, 16), _spd(2, 17)]
    s = 0.05
    op = Sum([Kron([Dense(m) for m in mats]), Diag(s, 24)])
    B = _rs(18).standard_normal((3, 24))
    np.testing.assert_allclose(exact.kron_shift_solve(mats, s, B),
                               exact.dense_solve(op.dense(), B), rtol=1e-10)


def test_exact_logdet_matches_cholesky():
    mats = [_spd(5, 19), _spd(6, 20)]
    op = Sum([Kron([Dense(m) for m in mats]), Diag(0.2, 30)])
    assert abs(exact.kron_shift_logdet(mats, 0.2) - exact.cholesky_logdet(op.dense())) < 1e-10


@pytest.fixture(scope="module")
def cfg1():
    return wl.config1()


def test_config1_cg_and_logdet_against_dense(cfg1):
    """The FP64 single-solve workload (N = 4096): CG to 1e-10, exact solve and
    exact log-det against dense LU / Cholesky of the assembled matrix."""
    K1, K2 = cfg1.factors
    op = Sum([Kron([Dense(K1), Dense(K2)]), Diag(cfg1.shift, cfg1.N)])
    A = np.kron(K1, K2) + cfg1.shift * np.eye(cfg1.N)
    b = cfg1.B[0]
    x_exact = exact.kron_shift_solve(cfg1.factors, cfg1.shift, b)[0]
    x_lu = exact.dense_solve(A, b)[0]
    assert np.linalg.norm(x_exact - x_lu) / np.linalg.norm(x_lu) < 1e-9
    x_cg, it = krylov.cg(op, b, tol=cfg1.tol)
    assert krylov.true_relative_residual(op, b, x_cg)[0] < 3 * cfg1.tol
    assert 50 < it < 1000
    ld = exact.kron_shift_logdet(cfg1.factors, cfg1.shift)
    assert abs(ld - exact.cholesky_logdet(A)) < 1e-8 * abs(ld)


# ---------------------------------------------------------------------------
# Lanczos, Gauss quadrature, SLQ
# ---------------------------------------------------------------------------

def test_lanczos_relation_and_orthogonality():
    A = _spd(30, 21)
    op = Dense(A)
    z = _rs(22).standard_normal(30)
    m = 10
    a, b, Q = krylov.lanczos(op, z, m + 1)
    T = krylov.tridiagonal(a[:m], b[:m - 1])
    # A Q_m^T = Q_m^T T_m + beta_m q_m e_m^T
    lhs = A @ Q[:m].T
    rhs = Q[:m].T @ T
    rhs[:, -1] += b[m - 1] * Q[m]
    np.testing.assert_allclose(lhs, rhs, atol=1e-11)
    np.testing.assert_allclose(Q @ Q.T, np.eye(m + 1), atol=1e-12)


@pytest.mark.parametrize("p", [0, 1, 2, 5, 9, 11])
def test_gauss_quadrature_exact_for_polynomials(p):
    """The m-point Gauss rule from Lanczos integrates t^p exactly for p <= 2m - 1."""
    A = _spd(25, 23) / 2.0
    op = Dense(A)
    z = _rs(24).standard_normal(25)
    m = 6
    a, b, _ = krylov.lanczos(op, z, m)
    q, _, _ = krylov.gauss_quadrature(a, b, lambda t: t ** p)
    v = z.copy()
    for _ in range(p):
        v = A @ v
    assert abs((z @ z) * q - z @ v) < 1e-10 * max(1.0, abs(z @ v))


def test_gauss_quadrature_not_exact_beyond_degree():
    A = _spd(25, 23) / 2.0
    z = _rs(24).standard_normal(25)
    m = 3
    a, b, _ = krylov.lanczos(Dense(A), z, m)
    q, _, _ = krylov.gauss_quadrature(a, b, lambda t: t ** (2 * m + 2))
    v = np.linalg.matrix_power(A, 2 * m + 2) @ z
    assert abs((z @ z) * q - z @ v) > 1e-6 * abs(z @ v)


def test_slq_full_krylov_reaches_quadratic_form():
    A = _spd(16, 25)
    z = rng.rademacher_probes(5, 1, 16)[0]
    val, se, vals = krylov.slq_logdet(Dense(A), z[None, :], 16)
    w, V = np.linalg.eigh(A)
    exact_q = z @ (V @ (np.log(w) * (V.T @ z)))
    assert abs(vals[0] - exact_q) < 1e-9 * abs(exact_q)


def test_slq_config1_zscore(cfg1):
    """SLQ with 16 Rademacher probes x 50 steps vs the exact log-det."""
    op = Sum([Kron([Dense(f) for f in cfg1.factors]), Diag(cfg1.shift, cfg1.N)])
    Z = rng.rademacher_probes(wl.substream(cfg1.seed, 2), cfg1.slq_probes, cfg1.N)
    est, se, _ = krylov.slq_logdet(op, Z, cfg1.slq_steps)
    ld = exact.kron_shift_logdet(cfg1.factors, cfg1.shift)
    assert abs(est - ld) / se < 4.0
    assert abs(est - ld) / abs(ld) < 2e-2


def test_hutchinson_gaussian_variance():
    """App. B.1: Var[z^T A z] = 2 Tr(A^2) for Gaussian probes."""
    A = _spd(8, 26)
    r = _rs(27)
    Z = r.standard_normal((40000, 8))
    q = np.einsum("ij,jk,ik->i", Z, A, Z)
    assert abs(q.mean() - np.trace(A)) < 5 * math.sqrt(2 * np.trace(A @ A) / len(q))
    assert abs(q.var() / (2 * np.trace(A @ A)) - 1.0) < 0.05


# ---------------------------------------------------------------------------
# Gradients (App. B.2)
# ---------------------------------------------------------------------------

def _grad_zoo():
    r = _rs(30)
    A, B = _spd(3, 31), _spd(4, 32)
    NA = r.standard_normal((3, 3))
    U, V = r.standard_normal((12, 2)), r.standard_normal((12, 2))
    d = 1.0 + r.random(12)
    return [
        Sum([Kron([Dense(A), Dense(B)]), Diag(0.3, 12)]),
        Sum([Kron([Dense(NA), Dense(B)]), Diag(d), LowRank(U)], [2.0, 1.0, 0.5]),
        Sum([KronSum([Dense(A), Dense(B)]), LowRank(U, V)]),
        Product([Kron([Dense(NA), Dense(B)]), Sum([Diag(d), LowRank(U, V)])]),
        Kron([Dense(A), Diag(np.array([1.0, 2.0, 3.0, 4.0]))]),
    ]


@pytest.mark.parametrize("k", range(5))
def test_bilinear_grad_contracted_matches_definition(k):
    op = _grad_zoo()[k]
    r = _rs(33)
    U = r.standard_normal((3, op.rows))
    X = r.standard_normal((3, op.cols))
    w = np.array([1.0, -0.5, 2.0])
    for g1, g2 in zip(grad.bilinear_grad(op, U, X, w), grad.bilinear_grad_bruteforce(op, U, X, w)):
        np.testing.assert_allclose(g1, g2, atol=1e-11)


def _with_leaf(op, leaf, value):
    """Rebuild the tree with one leaf's parameter replaced."""
    if op is leaf:
        return op.replaced(value)
    if isinstance(op, Sum):
        return Sum([_with_leaf(t, leaf, value) for t in op.terms], op.coeffs)
    if isinstance(op, Product):
        return Product([_with_leaf(t, leaf, value) for t in op.terms])
    if isinstance(op, Kron):
        return Kron([_with_leaf(t, leaf, value) for t in op.factors])
    if isinstance(op, KronSum):
        return KronSum([_with_leaf(t, leaf, value) for t in op.factors])
    return op


def solve_vjp_fd_error(op, vjp):
    """max |vjp - central FD| of f(theta) = w^T A(theta)^-1 b over all leaf entries."""
    r = _rs(34)
    b = r.standard_normal(op.cols)
    w = r.standard_normal(op.rows)
    g = vjp(op, b, w)
    h = 1e-6
    worst = 0.0
    for leaf, gl in zip(op.leaves(), g):
        p = np.asarray(leaf.param(), dtype=float)
        for e in (np.ndindex(*p.shape) if p.ndim else [()]):
            pp, pm = p.copy(), p.copy()
            pp[e] += h
            pm[e] -= h
            fp = w @ exact.dense_solve(_with_leaf(op, leaf, pp).dense(), b)[0]
            fm = w @ exact.dense_solve(_with_leaf(op, leaf, pm).dense(), b)[0]
            worst = max(worst, abs((fp - fm) / (2 * h) - np.asarray(gl)[e]))
    return worst


def oracle_solve_vjp(op, b, w):
    A = op.dense()
    x = exact.dense_solve(A, b)
    u = exact.dense_solve(A.T, w)
    return [-g for g in grad.bilinear_grad(op, u, x)]


@pytest.mark.parametrize("k", [0, 1, 2, 4])
def test_solve_vjp_matches_finite_differences(k):
    op = _grad_zoo()[k]
    assert solve_vjp_fd_error(op, oracle_solve_vjp) < 1e-6


def test_gp_gradient_matches_fd_and_dense():
    """Exact GP objective gradient (eigenbasis) vs central FD in (l1, l2, sigma2)
    and vs the dense FP64 gradient at n1 = n2 = 32."""
    n = 32
    x1 = wl.uniform(wl.substream(99, 1), (n,))
    x2 = wl.uniform(wl.substream(99, 2), (n,))
    l1, l2, s = 0.1, 0.2, 0.1
    y = wl.normal(wl.substream(99, 3), (n * n,))

    def L(a, b, c):
        return exact.gp_objective(wl.rbf_factor(x1, a), wl.rbf_factor(x2, b), c, y)

    K1, K2 = wl.rbf_factor(x1, l1), wl.rbf_factor(x2, l2)
    g1, g2, gs = exact.gp_gradient(K1, K2, s, y)
    dl1 = float(np.sum(g1 * wl.rbf_factor_dell(x1, l1)))
    dl2 = float(np.sum(g2 * wl.rbf_factor_dell(x2, l2)))
    h = 1e-5
    fd = [(L(l1 + h, l2, s) - L(l1 - h, l2, s)) / (2 * h),
          (L(l1, l2 + h, s) - L(l1, l2 - h, s)) / (2 * h),
          (L(l1, l2, s + h) - L(l1, l2, s - h)) / (2 * h)]
    np.testing.assert_allclose([dl1, dl2, gs], fd, rtol=1e-5)
    # dense gradient: dL/dtheta = -1/2 a^T dA a + 1/2 Tr(A^-1 dA)
    A = np.kron(K1, K2) + s * np.eye(n * n)
    Ainv = np.linalg.inv(A)
    a = Ainv @ y
    dA1 = np.kron(wl.rbf_factor_dell(x1, l1), K2)
    dA2 = np.kron(K1, wl.rbf_factor_dell(x2, l2))
    dense = [-0.5 * a @ dA1 @ a + 0.5 * np.sum(Ainv * dA1.T),
             -0.5 * a @ dA2 @ a + 0.5 * np.sum(Ainv * dA2.T),
             -0.5 * a @ a + 0.5 * np.trace(Ainv)]
    np.testing.assert_allclose([dl1, dl2, gs], dense, rtol=1e-8)


def test_gp_gradient_hutchinson_estimate():
    """Tr(A^-1 dA/dtheta) via Rademacher probes reusing A^-1 z (App. B.1/B.2)
    lies within 4 standard errors of the exact eigenbasis trace."""
    n = 16
    x1 = wl.uniform(wl.substream(98, 1), (n,))
    x2 = wl.uniform(wl.substream(98, 2), (n,))
    K1, K2, s = wl.rbf_factor(x1, 0.2), wl.rbf_factor(x2, 0.3), 0.1
    op = Sum([Kron([Dense(K1), Dense(K2)]), Diag(s, n * n)])
    Z = rng.rademacher_probes(7, 400, n * n)
    U = exact.kron_shift_solve([K1, K2], s, Z)
    per = [grad.bilinear_grad(op, U[i:i + 1], Z[i:i + 1]) for i in range(len(Z))]
    y = np.zeros(n * n)
    g1, g2, gs = exact.gp_gradient(K1, K2, s, y)      # y = 0: only the trace term
    for leaf, ex in ((0, g1), (1, g2), (2, gs)):
        samples = np.array([0.5 * p[leaf] for p in per])
        m = samples.mean(axis=0)
        se = samples.std(axis=0, ddof=1) / math.sqrt(len(samples)) + 1e-12
        assert np.max(np.abs(m - ex) / se) < 4.5


# ---------------------------------------------------------------------------
# Counter generator (published outputs) and workload generator agreement
# ---------------------------------------------------------------------------

def test_splitmix64_published_outputs():
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        vals = [int(l, 16) for l in f if l.strip() and not l.startswith("#")]
    assert [rng.output(0, i) for i in range(3)] == vals
    assert [int(v) for v in wl.splitmix64(0, 3)] == vals


def test_probe_generator_definition():
    Z = rng.rademacher_probes(12345, 3, 50)
    for v in range(3):
        for i in range(50):
            bit = rng.output(12345, v * 50 + i) >> 63
            assert Z[v, i] == (1.0 if bit == 0 else -1.0)


# ---------------------------------------------------------------------------
# Planted mistakes: each plausible oracle bug is caught by some pin above.
# ---------------------------------------------------------------------------

class _KronTransposed(Kron):
    def mvm(self, X):
        R = X.shape[0]
        T = X.reshape((R,) + tuple(f.cols for f in self.factors))
        for k, f in enumerate(self.factors):
            T = np.moveaxis(np.tensordot(f.dense().T, T, axes=([1], [1 + k])), 0, 1 + k)
        return T.reshape(R, self.rows)


def test_planted_transposed_factor_is_caught():
    assert kron_vec_identity_error(_KronTransposed, square=True) > 1e-3


def test_planted_dropped_shift_is_caught():
    mats = [_spd(3, 15), _spd(4, 16)]
    b = _rs(18).standard_normal((1, 12))
    op = Sum([Kron([Dense(m) for m in mats]), Diag(0.05, 12)])
    wrong = exact.kron_shift_solve(mats, 0.0, b)
    assert np.max(np.abs(wrong - exact.dense_solve(op.dense(), b))) > 1e-3


def test_planted_gradient_sign_is_caught():
    op = _grad_zoo()[0]

    def wrong_vjp(op, b, w):
        return [-g for g in oracle_solve_vjp(op, b, w)]

    assert solve_vjp_fd_error(op, wrong_vjp) > 1e-3


def test_planted_missing_probe_norm_is_caught():
    A = _spd(16, 25)
    z = rng.rademacher_probes(5, 1, 16)[0]
    a, b, _ = krylov.lanczos(Dense(A), z, 16)
    without_norm = krylov.quadrature_logdet_from_tridiag(a, b, 1.0)
    w, V = np.linalg.eigh(A)
    exact_q = z @ (V @ (np.log(w) * (V.T @ z)))
    assert abs(without_norm - exact_q) > 1e-2 * abs(exact_q)


def test_derivative_operator_is_linear_direction():
    op = _grad_zoo()[1]
    leaf = op.leaves()[0]
    r = _rs(40)
    E1, E2 = r.standard_normal((3, 3)), r.standard_normal((3, 3))
    x = r.standard_normal(op.cols)
    lhs = derivative(op, leaf, E1 + 2 * E2) @ x
    rhs = derivative(op, leaf, E1) @ x + 2 * (derivative(op, leaf, E2) @ x)
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)
