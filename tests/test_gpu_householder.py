"""Householder Arnoldi / Lanczos (Algorithm 2; cola_arnoldi_householder and
cola_lanczos(reorth=2)) against the FP64 oracle.

The CUDA path takes the cancellation-free reflector sign, so its Hessenberg
matrix equals the oracle's (Algorithm 2 as printed) up to a +-1 diagonal
similarity: diagonals are compared directly, other entries in absolute
value.  In FP32 the point of the method is a basis that stays orthogonal:
plain FP32 Lanczos repeats converged Ritz values (ghosts) on an operator
with a well separated top of the spectrum, the Householder iteration does
not."""
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


def _sym_spec():
    r = np.random.default_rng(90)
    K1, K2 = wl.rbf_factor(r.random(24), 0.2), wl.rbf_factor(r.random(20), 0.3)
    return ("sum", [("kron", [("dense", K1), ("dense", K2)]), ("scalar", 0.05, 480)], None)


def test_householder_arnoldi_symmetric_f64(cola, ctx):
    spec = _sym_spec()
    ref_tree = oracle_tree(spec)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV)
    Z = np.random.default_rng(91).standard_normal((3, 480))
    m = 25
    H, meff = cola.cola_arnoldi_householder(ctx, op, torch.tensor(Z, device=DEV), m,
                                            cola.PREC_F64)
    H = H.cpu().numpy()
    assert np.all(meff.cpu().numpy() == m)
    scale = np.abs(ref_tree.dense()).max()
    for p in range(3):
        Href, _ = krylov.householder_arnoldi(ref_tree, Z[p], m)
        np.testing.assert_allclose(np.diag(H[p]), np.diag(Href), rtol=1e-9, atol=1e-12 * scale)
        assert np.abs(np.abs(H[p]) - np.abs(Href)).max() <= 1e-9 * scale
        assert np.all(np.tril(H[p], -2) == 0.0)


def test_householder_arnoldi_nonsymmetric_f64(cola, ctx):
    """Product(K1 (x) K2, Diag(d)) is not symmetric: full upper Hessenberg H."""
    r = np.random.default_rng(92)
    K1, K2 = wl.rbf_factor(r.random(16), 0.2), wl.rbf_factor(r.random(12), 0.3)
    d = 0.5 + r.random(192)
    spec = ("product", [("kron", [("dense", K1), ("dense", K2)]), ("diag", d)])
    ref_tree = oracle_tree(spec)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV)
    Z = r.standard_normal((2, 192))
    m = 20
    H, _ = cola.cola_arnoldi_householder(ctx, op, torch.tensor(Z, device=DEV), m, cola.PREC_F64)
    H = H.cpu().numpy()
    scale = np.abs(ref_tree.dense()).max()
    for p in range(2):
        Href, _ = krylov.householder_arnoldi(ref_tree, Z[p], m)
        assert np.abs(np.abs(H[p]) - np.abs(Href)).max() <= 1e-9 * scale
        # the Ritz values (eigenvalues of the square part) are similarity-invariant
        ev = np.sort_complex(np.linalg.eigvals(H[p][:m, :m]))
        ev_ref = np.sort_complex(np.linalg.eigvals(Href[:m, :m]))
        np.testing.assert_allclose(ev, ev_ref, rtol=1e-7, atol=1e-10 * scale)


def test_lanczos_reorth2_matches_oracle_lanczos_f64(cola, ctx):
    spec = _sym_spec()
    ref_tree = oracle_tree(spec)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    Z = np.random.default_rng(93).standard_normal((2, 480))
    a, b, meff = cola.cola_lanczos(ctx, op, torch.tensor(Z, device=DEV), 30, cola.PREC_F64,
                                   reorth=2)
    a, b = a.cpu().numpy(), b.cpu().numpy()
    for p in range(2):
        a_ref, b_ref, _ = krylov.lanczos(ref_tree, Z[p], 30, reorth=True)
        k = len(a_ref)
        assert int(meff[p]) == k
        np.testing.assert_allclose(a[p, :k], a_ref, rtol=1e-9)
        np.testing.assert_allclose(b[p, :k - 1], b_ref, rtol=1e-9)


def _ritz(a, b):
    T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
    return np.sort(np.linalg.eigvalsh(T))[::-1]


def test_fp32_householder_has_no_ghosts(cola, ctx):
    """K1 (x) K2 (x) K3 + 1e-4 I, three 24-point RBF factors (N = 13824), one
    Rademacher start, 80 steps in FP32: the Householder iteration's top Ritz
    values match the FP64 reorthogonalised oracle and the largest eigenvalue
    appears once; plain FP32 Lanczos repeats it."""
    r = np.random.default_rng(5)
    facs = [wl.rbf_factor(r.random(24), 0.15) for _ in range(3)]
    N = 24 ** 3
    spec = ("sum", [("kron", [("dense", f) for f in facs]), ("scalar", 1e-4, N)], None)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    z = np.where(r.random(N) < 0.5, -1.0, 1.0)
    m = 80
    a64, b64, _ = krylov.lanczos(oracle_tree(spec), z, m, reorth=True)
    r64 = _ritz(a64, b64)
    top = float(np.max(exact.kron_eigenvalues(facs, 1e-4)))
    Z = torch.tensor(z[None, :], dtype=torch.float32, device=DEV)
    res = {}
    for reorth in (0, 2):
        a, b, meff = cola.cola_lanczos(ctx, op, Z, m, cola.PREC_F32, reorth=reorth)
        k = int(meff[0])
        res[reorth] = _ritz(a[0, :k].cpu().numpy(), b[0, :k - 1].cpu().numpy())
    near = {k: int(np.sum(np.abs(v - top) < 1e-3 * top)) for k, v in res.items()}
    assert near[2] == 1, near
    assert near[0] >= 2, near
    np.testing.assert_allclose(res[2][:8], r64[:8], rtol=1e-4)
