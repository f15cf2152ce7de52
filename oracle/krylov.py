"""Krylov base cases in FP64: CG, Lanczos, Gauss quadrature, SLQ.  Test infrastructure only.

Table 5 (App. C.2) names CG as the base case for PSD solves, Lanczos for
self-adjoint eigenproblems and stochastic Lanczos quadrature (SLQ) for f(A)
of self-adjoint A.  App. A.2 defines log det A = Tr(log A), which SLQ
estimates with Rademacher probes z: E[z^T log(A) z] = Tr(log A) (Sec. 3.3 /
App. B.1 trace estimator).  The Lanczos stopping rule mirrors the Arnoldi
breakdown test of Algorithm 1 (stop when the new off-diagonal falls below a
tolerance).  The Householder Arnoldi iteration of Algorithm 2 keeps the basis
orthogonal to rounding by building it from reflectors; for symmetric A its
Hessenberg matrix is Lanczos' tridiagonal.
"""
from __future__ import annotations

import numpy as np


def cg(op, b, tol=1e-10, maxiter=None, precond_diag=None, x0=None, precond=None):
    """Textbook (preconditioned) conjugate gradients on one right-hand side.

    Stops when the recursive residual satisfies ||r|| <= tol * ||b||.
    Returns (x, iterations).  ``precond_diag`` is the Jacobi diagonal M;
    ``precond`` (exclusive with it) is any function r -> M^-1 r of a
    symmetric positive definite M.
    """
    if precond is None:
        precond = (lambda r: r / precond_diag) if precond_diag is not None else (lambda r: r.copy())
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    maxiter = n if maxiter is None else maxiter
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - (op @ x) if x0 is not None else b.copy()
    z = precond(r)
    p = z.copy()
    rz = float(r @ z)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return x, 0
    it = 0
    while np.linalg.norm(r) > tol * bnorm and it < maxiter:
        Ap = op @ p
        pAp = float(p @ Ap)
        if not pAp > 0.0:
            raise FloatingPointError("CG breakdown: p^T A p <= 0")
        alpha = rz / pAp
        x = x + alpha * p
        r = r - alpha * Ap
        z = precond(r)
        rz_new = float(r @ z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
        it += 1
    return x, it


def cg_reorth_residuals(op, b, tol=1e-10, maxiter=None, dtype=np.float64):
    """Conjugate gradients with re-orthogonalised residuals, the low-precision
    CG variant of Maddox, Potapczynski & Wilson (UAI 2022) that Sec. 3.4 /
    App. C.3 cite: every new residual r_{k+1} = r_k - alpha_k A p_k is made
    orthogonal, by two passes of classical Gram-Schmidt, to all earlier
    residuals r_0 .. r_k before it enters beta_k = r_{k+1}^T r_{k+1} / r_k^T r_k
    and p_{k+1} = r_{k+1} + beta_k p_k.  In exact arithmetic CG's residuals are
    already mutually orthogonal, so the iterates are those of ``cg``; in low
    precision the projection restores that orthogonality.  Unpreconditioned.

    ``dtype`` is the working precision of the vectors and the MVM (the
    projections' dot products accumulate in FP64).  Returns (x, iterations,
    R) with R the (iterations + 1, n) array of the residuals used.
    """
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    maxiter = n if maxiter is None else maxiter
    x = np.zeros(n, dtype=dtype)
    r = b.astype(dtype)
    p = r.copy()
    rr = float(r.astype(np.float64) @ r.astype(np.float64))
    bnorm = float(np.linalg.norm(b))
    res = [r.copy()]
    if bnorm == 0.0:
        return x.astype(np.float64), 0, np.array(res)
    it = 0
    while np.sqrt(rr) > tol * bnorm and it < maxiter:
        Ap = (op @ p.astype(np.float64)).astype(dtype)
        pAp = float(p.astype(np.float64) @ Ap.astype(np.float64))
        if not pAp > 0.0:
            raise FloatingPointError("CG breakdown: p^T A p <= 0")
        alpha = rr / pAp
        x = (x + dtype(alpha) * p).astype(dtype)
        r = (r - dtype(alpha) * Ap).astype(dtype)
        for _ in range(2):
            for q in res:
                q64 = q.astype(np.float64)
                c = float(q64 @ r.astype(np.float64)) / float(q64 @ q64)
                r = (r - dtype(c) * q).astype(dtype)
        rr_new = float(r.astype(np.float64) @ r.astype(np.float64))
        beta = rr_new / rr
        rr = rr_new
        p = (r + dtype(beta) * p).astype(dtype)
        res.append(r.copy())
        it += 1
    return x.astype(np.float64), it, np.array(res)


def true_relative_residual(op, B, X):
    """||b - A x|| / ||b|| per right-hand side (rows of B, X)."""
    B = np.atleast_2d(B)
    X = np.atleast_2d(X)
    R = B - op.mvm(X)
    return np.linalg.norm(R, axis=1) / np.linalg.norm(B, axis=1)


def lanczos(op, z, m, reorth=True, breakdown_tol=1e-10):
    """m steps of symmetric Lanczos from q_0 = z / ||z||.

    Recurrence: w = A q_j - beta_{j-1} q_{j-1}; alpha_j = q_j^T w;
    w -= alpha_j q_j; (full reorthogonalisation against all previous q when
    ``reorth``); beta_j = ||w||; stop when beta_j <= breakdown_tol * max|alpha|;
    q_{j+1} = w / beta_j.

    Returns (alpha[m_eff], beta[m_eff - 1], Q[m_eff, N]).
    """
    z = np.asarray(z, dtype=np.float64)
    q = z / np.linalg.norm(z)
    Q = [q]
    alphas, betas = [], []
    q_prev = np.zeros_like(q)
    beta_prev = 0.0
    for j in range(m):
        w = op @ Q[j] - beta_prev * q_prev
        a = float(Q[j] @ w)
        w = w - a * Q[j]
        if reorth:
            for _ in range(2):
                for qi in Q:
                    w = w - float(qi @ w) * qi
        alphas.append(a)
        if j == m - 1:
            break
        beta = float(np.linalg.norm(w))
        if beta <= breakdown_tol * max(abs(x) for x in alphas):
            break
        betas.append(beta)
        q_prev = Q[j]
        beta_prev = beta
        Q.append(w / beta)
    return np.array(alphas), np.array(betas), np.array(Q[: len(alphas)])


def householder_vector(w, k):
    """Unit u with (I - 2 u u^T) w = (w_0, .., w_{k-1}, ||w_{k:}||, 0, .., 0)
    (the GET_HOUSEHOLDER_VEC step of Algorithm 2: u_i = 0 below k, u_k =
    w_k - ||w_{k:}||, u_i = w_i above k, then normalised)."""
    u = np.zeros_like(w)
    u[k + 1:] = w[k + 1:]
    u[k] = w[k] - np.linalg.norm(w[k:])
    n = np.linalg.norm(u)
    return u / n if n > 0 else u


def householder_arnoldi(op, nu0, T):
    """Householder Arnoldi iteration (Algorithm 2) for T steps from nu_0.

    For j = 0..T: u_j = householder_vector(nu_j, j), R_j = I - 2 u_j u_j^T,
    h_j = R_j nu_j, q_j = R_0 ... R_j e_j and, for j < T,
    nu_{j+1} = R_j ... R_0 (A q_j).  Column j - 1 of the (T+1) x T
    Hessenberg matrix H holds h_j[0..j] (j >= 1), so A Q[:, :T] = Q H.
    Returns (H, Q) with Q of shape (N, T+1)."""
    nu = np.asarray(nu0, dtype=np.float64).copy()
    N = nu.shape[0]
    us = []
    H = np.zeros((T + 1, T))
    Q = np.zeros((N, T + 1))
    for j in range(T + 1):
        u = householder_vector(nu, j)
        us.append(u)
        h = nu - 2.0 * u * float(u @ nu)
        if j >= 1:
            H[: j + 1, j - 1] = h[: j + 1]
        q = np.zeros(N)
        q[j] = 1.0
        for i in range(j, -1, -1):          # R_0 ... R_j e_j: R_j acts first
            q = q - 2.0 * us[i] * float(us[i] @ q)
        Q[:, j] = q
        if j < T:
            v = op @ q
            for i in range(j + 1):           # R_j ... R_0 (A q_j): R_0 acts first
                v = v - 2.0 * us[i] * float(us[i] @ v)
            nu = v
    return H, Q


def tridiagonal(alpha, beta):
    T = np.diag(alpha)
    if len(beta):
        T += np.diag(beta, 1) + np.diag(beta, -1)
    return T


def gauss_quadrature(alpha, beta, f):
    """sum_k S_{0k}^2 f(theta_k) with T_m = S diag(theta) S^T: the m-point Gauss
    rule for q_0^T f(A) q_0 (exact for polynomials of degree <= 2m - 1)."""
    theta, S = np.linalg.eigh(tridiagonal(alpha, beta))
    return float(np.sum(S[0, :] ** 2 * f(theta))), theta, S[0, :]


def slq_logdet(op, probes, m, reorth=True):
    """Stochastic Lanczos quadrature for log det A = Tr(log A).

    For each probe z: ||z||^2 * sum_k S_{0k}^2 log(theta_k).  Returns
    (mean over probes, standard error of the mean, per-probe values).
    A Ritz value <= 0 is an error (A must be positive definite).
    """
    vals = []
    for z in np.atleast_2d(probes):
        a, b, _ = lanczos(op, z, m, reorth=reorth)
        theta, S = np.linalg.eigh(tridiagonal(a, b))
        if np.any(theta <= 0.0):
            raise FloatingPointError("non-positive Ritz value in SLQ")
        vals.append(float(z @ z) * float(np.sum(S[0, :] ** 2 * np.log(theta))))
    vals = np.array(vals)
    se = float(np.std(vals, ddof=1) / np.sqrt(len(vals))) if len(vals) > 1 else float("nan")
    return float(np.mean(vals)), se, vals


def quadrature_logdet_from_tridiag(alpha, beta, znorm2):
    """Per-probe SLQ value from given Lanczos coefficients."""
    theta, S = np.linalg.eigh(tridiagonal(alpha, beta))
    return znorm2 * float(np.sum(S[0, :] ** 2 * np.log(theta)))
