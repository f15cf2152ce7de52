"""Closed forms the iterative results must reach (FP64).  Test infrastructure only.

Kronecker sums K_1 (+) ... (+) K_d = sum_k I (x) .. (x) K_k (x) .. (x) I share
the eigenvectors (x)_k V_k, with eigenvalues lam_1[i_1] + ... + lam_d[i_d]
(App. A.1.2); a product's inverse is the product of the factor inverses in
reverse order (Sec. 3.2).

App. A.1.2: Eigs(A (x) B) = (Lambda_A (x) Lambda_B, V_A (x) V_B), so for
A = K_1 (x) ... (x) K_d + s I with symmetric factors K_k = V_k diag(lam_k) V_k^T
    A^-1 b = V (Lambda + s)^-1 V^T b,  V = V_1 (x) ... (x) V_d,
    log det A = sum over multi-indices of log(lam_1[i_1] ... lam_d[i_d] + s)
(App. A.2: LogDet(A) = Tr(Log(A))).  V and V^T are applied by mode products.
Factor eigendecompositions use numpy's symmetric eigensolver (a library step).

The GP objective (Sec. 4 / App. D GP training) is
    L = 1/2 y^T A^-1 y + 1/2 log det A,   A = K_1 (x) K_2 + sigma^2 I,
with dL/dtheta = -1/2 alpha^T (dA/dtheta) alpha + 1/2 Tr(A^-1 dA/dtheta),
alpha = A^-1 y (App. B.2, rules 1 and 4).  In the eigenbasis:
    d/dK_1  1/2 log det A = 1/2 V_1 diag(c) V_1^T,  c_a = sum_b mu_b / (lam_a mu_b + s)
    d/dK_2  1/2 log det A = 1/2 V_2 diag(c') V_2^T, c'_b = sum_a lam_a / (lam_a mu_b + s)
    d/ds    1/2 log det A = 1/2 sum_ab 1 / (lam_a mu_b + s)
and, with alpha reshaped row-major to (n_1, n_2),
    d/dK_1 1/2 y^T A^-1 y = -1/2 alpha K_2 alpha^T,  d/dK_2 = -1/2 alpha^T K_1 alpha,
    d/ds = -1/2 alpha^T alpha.
"""
from __future__ import annotations

import numpy as np

from .linop import _mode_product


def _eig(factors):
    return [np.linalg.eigh(np.asarray(K, dtype=np.float64)) for K in factors]


def kron_eigenvalues(factors, shift=0.0):
    """All eigenvalues of K_1 (x) ... (x) K_d + shift I in row-major order."""
    lam = np.ones(1)
    for w, _ in _eig(factors):
        lam = np.outer(lam, w).ravel()
    return lam + shift


def _apply_modes(mats, X, shape):
    R = X.shape[0]
    T = X.reshape((R,) + tuple(shape))
    for k, M in enumerate(mats):
        T = _mode_product(M, T, k)
    return T.reshape(R, -1)


def kron_shift_solve(factors, shift, B):
    """Exact A^-1 B for A = (x)_k K_k + shift I (rows of B are right-hand sides)."""
    B = np.atleast_2d(np.asarray(B, dtype=np.float64))
    eig = _eig(factors)
    shape = [K.shape[0] for K in factors]
    lam = np.ones(1)
    for w, _ in eig:
        lam = np.outer(lam, w).ravel()
    C = _apply_modes([V.T for _, V in eig], B, shape)
    C = C / (lam + shift)
    return _apply_modes([V for _, V in eig], C, shape)


def kron_shift_logdet(factors, shift):
    lam = kron_eigenvalues(factors, shift)
    if np.any(lam <= 0):
        raise FloatingPointError("operator is not positive definite")
    return float(np.sum(np.log(lam)))


def kronsum_eigenvalues(factors, shift=0.0):
    """All eigenvalues of K_1 (+) ... (+) K_d + shift I in row-major order:
    lam_1[i_1] + ... + lam_d[i_d] (App. A.1.2, the Kronecker-sum rule)."""
    lam = np.zeros(1)
    for w, _ in _eig(factors):
        lam = np.add.outer(lam, w).ravel()
    return lam + shift


def kronsum_shift_solve(factors, shift, B):
    """Exact A^-1 B for A = (+)_k K_k + shift I: same eigenvectors as the
    Kronecker product, eigenvalues summed."""
    B = np.atleast_2d(np.asarray(B, dtype=np.float64))
    eig = _eig(factors)
    shape = [K.shape[0] for K in factors]
    lam = np.zeros(1)
    for w, _ in eig:
        lam = np.add.outer(lam, w).ravel()
    C = _apply_modes([V.T for _, V in eig], B, shape)
    C = C / (lam + shift)
    return _apply_modes([V for _, V in eig], C, shape)


def product_split_solve(factor_solvers, B):
    """A^-1 B for A = A_1 A_2 ... A_m given solvers for each factor
    (Sec. 3.2: Inverse(A_1 ... A_m) = A_m^-1 ... A_1^-1): A_1 is solved first."""
    X = np.atleast_2d(np.asarray(B, dtype=np.float64))
    for solve in factor_solvers:
        X = solve(X)
    return X


def dense_solve(A, B):
    """Dense LU solve (numpy/LAPACK), the reference for small systems."""
    return np.linalg.solve(A, np.atleast_2d(B).T).T


def cholesky_logdet(A):
    """log det A = 2 sum log L_ii for A = L L^T."""
    L = np.linalg.cholesky(A)
    return float(2.0 * np.sum(np.log(np.diag(L))))


def gp_objective(K1, K2, sigma2, y):
    """L = 1/2 y^T A^-1 y + 1/2 log det A for A = K1 (x) K2 + sigma2 I."""
    a = kron_shift_solve([K1, K2], sigma2, y)[0]
    return 0.5 * float(y @ a) + 0.5 * kron_shift_logdet([K1, K2], sigma2)


def gp_gradient(K1, K2, sigma2, y):
    """Exact (dL/dK1, dL/dK2, dL/dsigma2) for the GP objective above."""
    (lam, V1), (mu, V2) = _eig([K1, K2])
    n1, n2 = K1.shape[0], K2.shape[0]
    den = lam[:, None] * mu[None, :] + sigma2
    c1 = np.sum(mu[None, :] / den, axis=1)
    c2 = np.sum(lam[:, None] / den, axis=0)
    dld_K1 = 0.5 * (V1 * c1) @ V1.T
    dld_K2 = 0.5 * (V2 * c2) @ V2.T
    dld_s = 0.5 * float(np.sum(1.0 / den))
    a = kron_shift_solve([K1, K2], sigma2, y)[0].reshape(n1, n2)
    dq_K1 = -0.5 * a @ K2 @ a.T
    dq_K2 = -0.5 * a.T @ K1 @ a
    dq_s = -0.5 * float(np.sum(a * a))
    return dld_K1 + dq_K1, dld_K2 + dq_K2, dld_s + dq_s
