"""The host eigensolver behind the Kronecker eigen-structured path
(cola_sym_eig: Householder tridiagonalisation + implicit symmetric QR, FP64),
pinned on CPU against LAPACK, closed forms and invariants."""
import math

import numpy as np
import pytest

import workloads as wl


@pytest.fixture(scope="module")
def cola():
    try:
        import paper_2309_03060_gb300 as c
        c._lib()
    except ImportError as e:
        pytest.skip(f"library not built: {e}")
    return c


@pytest.mark.parametrize("n", [1, 2, 3, 8, 65, 128])
def test_sym_eig_matches_lapack_and_invariants(cola, n):
    r = np.random.default_rng(n)
    A = r.standard_normal((n, n))
    A = A + A.T
    w, V = cola.cola_sym_eig(A)
    scale = max(1.0, np.abs(A).max() * n)
    np.testing.assert_allclose(np.sort(w), np.linalg.eigvalsh(A), atol=1e-13 * scale)
    assert np.abs(A @ V - V * w).max() <= 1e-13 * scale
    assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-13 * n


def test_sym_eig_dirichlet_laplacian_closed_form(cola):
    """tridiag(-1, 2, -1) of order n has eigenvalues 2 - 2 cos(k pi / (n + 1))."""
    n = 50
    L = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    w, V = cola.cola_sym_eig(L)
    exact = np.array([2 - 2 * math.cos(k * math.pi / (n + 1)) for k in range(1, n + 1)])
    np.testing.assert_allclose(np.sort(w), exact, atol=1e-13)
    # eigenvector of the smallest eigenvalue: sin(j pi / (n + 1)) up to sign
    j = np.argmin(w)
    s = np.sin(np.arange(1, n + 1) * math.pi / (n + 1))
    s /= np.linalg.norm(s)
    assert abs(abs(float(V[:, j] @ s)) - 1.0) <= 1e-12


@pytest.mark.parametrize("A", [np.eye(6), np.diag([2.0, 2.0, 1.0, 1.0, 3.0]),
                               np.ones((4, 4))])
def test_sym_eig_repeated_eigenvalues(cola, A):
    w, V = cola.cola_sym_eig(A)
    np.testing.assert_allclose(np.sort(w), np.linalg.eigvalsh(A), atol=1e-14)
    assert np.abs(A @ V - V * w).max() <= 1e-14
    assert np.abs(V.T @ V - np.eye(len(A))).max() <= 1e-14


def test_sym_eig_rbf_factor(cola):
    """The bench workload's factor: RBF on 128 points, lengthscale 0.1
    (eigenvalues spread over 16 decades, many near rounding level)."""
    x = wl.uniform(wl.substream(7, 1), (128,))
    K = wl.rbf_factor(x, 0.1)
    w, V = cola.cola_sym_eig(K)
    assert np.abs(K @ V - V * w).max() <= 1e-12 * np.abs(K).sum(1).max()
    np.testing.assert_allclose(np.sort(w), np.linalg.eigvalsh(K), atol=1e-12 * np.abs(w).max())
