"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: F64 results within 1e-11 relative (rounding order only); F32
MVMs within 2e-6 of max|A x| (n_k-term FP32 dot products per mode); solves by
their relative residual and the forward-error bound kappa * tol; SLQ per-probe
values from the same probes within 1e-8 (F64).
"""
import math

import numpy as np
import pytest

import workloads as wl
from oracle import exact, grad, krylov, rng
from oracle import linop as O
from tests._trees import gpu_tree, leaf_params, oracle_tree

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


def _rs(seed):
    return np.random.default_rng(seed)


def _spd(n, seed, shift=0.5):
    M = _rs(seed).standard_normal((n, n))
    return M @ M.T / n + shift * np.eye(n)


def rel_max_err(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _zoo():
    r = _rs(100)
    A = r.standard_normal((37, 29))
    B = r.standard_normal((131, 129))
    C3 = r.standard_normal((5, 7))
    S1, S2 = _spd(33, 101), _spd(40, 102)
    n = 37
    L = wl.dirichlet_laplacian(n)
    U = r.standard_normal((n * n, 5)) / n
    V = r.standard_normal((n * n, 5)) / n
    d = 0.5 + r.random(n * n)
    return {
        "kron_rect": ("kron", [("dense", A), ("dense", B), ("dense", C3)]),
        "kron_shift": ("sum", [("kron", [("dense", S1), ("dense", S2)]), ("scalar", 0.1, 33 * 40)],
                       None),
        "kronsum_tridiag_lowrank": ("sum", [("kronsum", [("dense", L), ("dense", L)]), ("diag", d),
                                            ("lowrank", U, None)], [1.0, 1.0, 1.0]),
        "kronsum_dense": ("kronsum", [("dense", S1[:7, :7]), ("dense", _spd(9, 3)),
                                      ("dense", _spd(11, 4))]),
        "lowrank_uv": ("sum", [("lowrank", U, V), ("diag", d)], [2.0, -1.0]),
        "product": ("product", [("kron", [("dense", S1[:6, :6]), ("dense", S2[:7, :7])]),
                                ("sum", [("diag", d[:42]), ("lowrank", U[:42], V[:42])], None)]),
        "dense_big": ("dense", r.standard_normal((300, 257))),
    }


@pytest.mark.parametrize("name", list(_zoo().keys()))
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_matvec_parity(cola, ctx, name, prec):
    spec = _zoo()[name]
    ref = oracle_tree(spec)
    dt = torch.float64 if prec == "f64" else torch.float32
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV)
    X = _rs(5).standard_normal((3, ref.cols))
    Y_ref = ref.mvm(X)
    Y = cola.cola_matvec(ctx, op, torch.tensor(X, dtype=dt, device=DEV),
                         cola.PREC_F64 if prec == "f64" else cola.PREC_F32)
    err = rel_max_err(Y.double().cpu().numpy(), Y_ref)
    assert err < (1e-12 if prec == "f64" else 2e-6), err


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_matvec_kron3_full_size_sampled(cola, ctx, prec):
    """The three-factor 128^3 workload (N = 2,097,152) in the launch layout
    the solver uses, checked on sampled rows computed one by one."""
    w = wl.config2(nrhs=2)
    spec = ("sum", [("kron", [("dense", f) for f in w.factors]), ("scalar", w.shift, w.N)], None)
    dt = torch.float64 if prec == "f64" else torch.float32
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV)
    X = torch.tensor(w.B, dtype=dt, device=DEV)
    Y = cola.cola_matvec(ctx, op, X, cola.PREC_F64 if prec == "f64" else cola.PREC_F32)
    Yh = Y.double().cpu().numpy()
    K1, K2, K3 = w.factors
    n = 128
    idx = _rs(7).integers(0, w.N, size=40)
    for r in range(2):
        Xr = w.B[r].reshape(n, n, n)
        scale = np.max(np.abs(Yh[r]))
        for I in idx:
            i1, i2, i3 = I // (n * n), (I // n) % n, I % n
            # row (i1, i2, i3) of K1 (x) K2 (x) K3 by its definition
            row = np.einsum("a,b,c->abc", K1[i1], K2[i2], K3[i3])
            ref = float(np.sum(row * Xr)) + w.shift * Xr[i1, i2, i3]
            assert abs(Yh[r, I] - ref) <= (1e-11 if prec == "f64" else 2e-6) * scale


def test_rademacher_bit_exact(cola, ctx):
    z = cola.cola_rademacher(ctx, seed=987654321, count=5000, offset=123).cpu().numpy()
    ref = rng.rademacher_probes(987654321, 1, 5123)[0, 123:]
    assert np.array_equal(z, ref)


def _kron_shift_problem(n1, n2, shift, nrhs, seed):
    x1 = wl.uniform(wl.substream(seed, 1), (n1,))
    x2 = wl.uniform(wl.substream(seed, 2), (n2,))
    K1, K2 = wl.rbf_factor(x1, 0.2), wl.rbf_factor(x2, 0.2)
    B = wl.normal(wl.substream(seed, 3), (nrhs, n1 * n2))
    spec = ("sum", [("kron", [("dense", K1), ("dense", K2)]), ("scalar", shift, n1 * n2)], None)
    return K1, K2, B, spec


def test_cg_config1_fp64(cola, ctx):
    """FP64 CG on K1 (x) K2 + 0.1 I with 64-point factors (N = 4096) to 1e-10."""
    w = wl.config1()
    spec = ("sum", [("kron", [("dense", f) for f in w.factors]), ("scalar", w.shift, w.N)], None)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    opts = cola.cola_cg_opts_default(precision=cola.PREC_F64, refine=0, tol=w.tol, maxiter=5000)
    X, info, st = cola.cola_cg_solve(ctx, op, torch.tensor(w.B, device=DEV), opts)
    assert st == 0
    x_ref = exact.kron_shift_solve(w.factors, w.shift, w.B)
    lam = exact.kron_eigenvalues(w.factors, w.shift)
    kappa = lam.max() / lam.min()
    assert info[0]["rel_residual"] <= w.tol
    assert krylov.true_relative_residual(oracle_tree(spec), w.B, X.cpu().numpy())[0] <= 1.5 * w.tol
    fe = np.linalg.norm(X.cpu().numpy() - x_ref) / np.linalg.norm(x_ref)
    assert fe <= kappa * w.tol * 2
    _, it_ref = krylov.cg(oracle_tree(spec), w.B[0], tol=w.tol)
    assert abs(info[0]["iterations"] - it_ref) <= max(3, 0.05 * it_ref) + opts.graph_chunk


@pytest.mark.parametrize("prec", ["f32"])
def test_cg_refined_reaches_1e8(cola, ctx, prec):
    K1, K2, B, spec = _kron_shift_problem(45, 70, 0.01, 4, 11)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    opts = cola.cola_cg_opts_default(precision=cola.PREC_F32, refine=1, tol=1e-8, maxiter=20000)
    X, info, st = cola.cola_cg_solve(ctx, op, torch.tensor(B, device=DEV), opts)
    assert st == 0, info
    res = krylov.true_relative_residual(oracle_tree(spec), B, X.cpu().numpy())
    assert np.all(res <= 1e-8), res
    for i in info:
        assert i["rel_residual"] <= 1e-8 and i["updates"] >= 1
    x_ref = exact.kron_shift_solve([K1, K2], 0.01, B)
    assert np.allclose(X.cpu().numpy(), x_ref, rtol=0, atol=1e-3 * np.max(np.abs(x_ref)))


def test_cg_plain_fp32_to_1e4(cola, ctx):
    K1, K2, B, spec = _kron_shift_problem(30, 50, 0.1, 3, 12)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    opts = cola.cola_cg_opts_default(precision=cola.PREC_F32, refine=0, tol=1e-4, maxiter=5000)
    X, info, st = cola.cola_cg_solve(ctx, op, torch.tensor(B, dtype=torch.float32, device=DEV), opts)
    res = krylov.true_relative_residual(oracle_tree(spec), B, X.double().cpu().numpy())
    assert np.all(res <= 2e-4), res


def test_jacobi_pcg_poisson_lowrank(cola, ctx):
    n = 64
    w = wl.config3(n=n, rank=8, nrhs=3)
    spec = ("sum", [("kronsum", [("dense", w.L), ("dense", w.L)]), ("diag", w.d),
                    ("lowrank", w.U, None)], None)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    opts = cola.cola_cg_opts_default(precision=cola.PREC_F32, refine=0, tol=1e-6, jacobi=1,
                                     maxiter=2000, graph_chunk=8)
    X, info, st = cola.cola_cg_solve(ctx, op, torch.tensor(w.B, dtype=torch.float32, device=DEV),
                                     opts)
    ref = oracle_tree(spec)
    res = krylov.true_relative_residual(ref, w.B, X.double().cpu().numpy())
    assert np.all(res <= 1e-5), res
    # iteration count close to the oracle's Jacobi PCG
    _, it = krylov.cg(ref, w.B[0], tol=1e-6, precond_diag=ref.diag())
    assert info[0]["iterations"] <= it + 8 + 5


def test_cg_not_converged_reports_status(cola, ctx):
    K1, K2, B, spec = _kron_shift_problem(30, 30, 1e-3, 1, 13)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    opts = cola.cola_cg_opts_default(precision=cola.PREC_F64, refine=0, tol=1e-12, maxiter=5,
                                     graph_chunk=2)
    X, info, st = cola.cola_cg_solve(ctx, op, torch.tensor(B, device=DEV), opts)
    assert st == 5 and info[0]["status"] == 5
    assert np.all(np.isfinite(X.cpu().numpy()))


def test_cg_rejects_non_spd_annotation(cola, ctx):
    K1, K2, B, spec = _kron_shift_problem(8, 8, 0.1, 1, 14)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV)
    with pytest.raises(cola.ColaError) as e:
        cola.cola_cg_solve(ctx, op, torch.tensor(B, device=DEV),
                           cola.cola_cg_opts_default(precision=cola.PREC_F64, refine=0))
    assert e.value.status == 1


def test_lanczos_matches_oracle(cola, ctx):
    w = wl.config1(scale=20)
    spec = ("sum", [("kron", [("dense", f) for f in w.factors]), ("scalar", w.shift, w.N)], None)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    Z = rng.rademacher_probes(3, 4, w.N)
    m = 30
    al, be, me = cola.cola_lanczos(ctx, op, torch.tensor(Z, device=DEV), m, cola.PREC_F64,
                                   reorth=True)
    al, be, me = al.cpu().numpy(), be.cpu().numpy(), me.cpu().numpy()
    ref = oracle_tree(spec)
    for v in range(4):
        a, b, _ = krylov.lanczos(ref, Z[v], m, reorth=True)
        assert me[v] == len(a)
        np.testing.assert_allclose(al[v, :len(a)], a, rtol=1e-9, atol=1e-9)
        np.testing.assert_allclose(be[v, :len(b)], b, rtol=1e-9, atol=1e-9)


def test_slq_config1_fp64(cola, ctx):
    """16 probes x 50 steps on the N = 4096 workload.  With full
    reorthogonalisation on both sides the per-probe quadrature values match
    the oracle's on the same probes to 1e-9; without it (the default), loss of
    orthogonality amplifies reduction-order differences, so they agree to
    1e-5.  The estimate lies within 4 SE of the exact log-det."""
    w = wl.config1()
    spec = ("sum", [("kron", [("dense", f) for f in w.factors]), ("scalar", w.shift, w.N)], None)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    seed = wl.substream(w.seed, 2)
    Z = rng.rademacher_probes(seed, w.slq_probes, w.N)
    ld_r, se_r, pp_r, cl = cola.cola_slq_logdet(ctx, op, w.slq_probes, w.slq_steps, seed=seed,
                                                precision=cola.PREC_F64, reorth=True)
    _, _, pp_ref_r = krylov.slq_logdet(oracle_tree(spec), Z, w.slq_steps, reorth=True)
    np.testing.assert_allclose(pp_r.cpu().numpy(), pp_ref_r, rtol=1e-9)
    ld, se, pp, cl = cola.cola_slq_logdet(ctx, op, w.slq_probes, w.slq_steps, seed=seed,
                                          precision=cola.PREC_F64)
    ld_ref, se_ref, pp_ref = krylov.slq_logdet(oracle_tree(spec), Z, w.slq_steps, reorth=False)
    np.testing.assert_allclose(pp.cpu().numpy(), pp_ref, rtol=1e-5)
    assert cl == 0
    exact_ld = exact.kron_shift_logdet(w.factors, w.shift)
    assert abs(ld - exact_ld) / se < 4.0
    assert abs(ld_r - exact_ld) / se_r < 4.0


def _grad_specs():
    r = _rs(200)
    A, B = _spd(7, 201), _spd(9, 202)
    NA = r.standard_normal((7, 7))
    n = 63
    U = r.standard_normal((n, 3))
    d = 1 + r.random(n)
    return {
        "kron_shift": ("sum", [("kron", [("dense", A), ("dense", B)]), ("scalar", 0.3, n)], None),
        "kron_diag_lowrank": ("sum", [("kron", [("dense", NA), ("dense", B)]), ("diag", d),
                                      ("lowrank", U, None)], [2.0, 1.0, 0.5]),
        "kronsum": ("sum", [("kronsum", [("dense", A), ("dense", B)]), ("scalar", 0.2, n)], None),
        "product": ("product", [("kron", [("dense", NA), ("dense", B)]), ("diag", d)]),
    }


@pytest.mark.parametrize("name", list(_grad_specs().keys()))
def test_bilinear_grad_parity(cola, ctx, name):
    spec = _grad_specs()[name]
    ref = oracle_tree(spec)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV)
    r = _rs(210)
    U = r.standard_normal((3, ref.rows))
    X = r.standard_normal((3, ref.cols))
    wts = [1.0, -0.5, 2.0]
    g = cola.cola_bilinear_grad(ctx, op, torch.tensor(U, device=DEV), torch.tensor(X, device=DEV),
                                wts, cola.PREC_F64)
    g_ref = grad.bilinear_grad(ref, U, X, np.array(wts))
    for a, b in zip(g, g_ref):
        np.testing.assert_allclose(a.cpu().numpy().reshape(np.shape(b)) if np.ndim(b) else
                                   a.cpu().numpy()[0], b, rtol=1e-10, atol=1e-10)


def test_solve_backward_parity(cola, ctx):
    spec = _grad_specs()["kron_shift"]
    ref = oracle_tree(spec)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    r = _rs(220)
    B = r.standard_normal((2, ref.rows))
    W = r.standard_normal((2, ref.rows))
    opts = cola.cola_cg_opts_default(precision=cola.PREC_F64, refine=0, tol=1e-12, maxiter=2000,
                                     graph_chunk=4)
    X, _, st = cola.cola_cg_solve(ctx, op, torch.tensor(B, device=DEV), opts)
    gB, g, info, st2 = cola.cola_solve_backward(ctx, op, X, torch.tensor(W, device=DEV), opts)
    A = ref.dense()
    x_ref = exact.dense_solve(A, B)
    u_ref = exact.dense_solve(A.T, W)
    np.testing.assert_allclose(gB.cpu().numpy(), u_ref, rtol=1e-8, atol=1e-10)
    g_ref = [-x for x in grad.bilinear_grad(ref, u_ref, x_ref)]
    for a, b in zip(g, g_ref):
        np.testing.assert_allclose(a.cpu().numpy().reshape(np.shape(b)), b, rtol=1e-7, atol=1e-9)


def test_logdet_backward_parity(cola, ctx):
    spec = _grad_specs()["kron_shift"]
    ref = oracle_tree(spec)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    Z = rng.rademacher_probes(5, 6, ref.rows)
    opts = cola.cola_cg_opts_default(precision=cola.PREC_F64, refine=0, tol=1e-12, maxiter=2000,
                                     graph_chunk=4)
    g = cola.cola_logdet_backward(ctx, op, torch.tensor(Z, device=DEV), None, 1.0, opts)
    U = exact.dense_solve(ref.dense(), Z)
    g_ref = grad.bilinear_grad(ref, U, Z, np.full(6, 1.0 / 6))
    for a, b in zip(g, g_ref):
        np.testing.assert_allclose(a.cpu().numpy().reshape(np.shape(b)), b, rtol=1e-7, atol=1e-9)


def test_batched_systems_uneven(cola, ctx):
    probs = [_kron_shift_problem(n1, n2, s, r, 300 + i)
             for i, (n1, n2, s, r) in enumerate([(16, 20, 0.1, 1), (33, 17, 0.05, 3),
                                                  (40, 41, 0.01, 2)])]
    ops = [gpu_tree(cola, ctx, p[3], torch.float64, DEV).set_spd() for p in probs]
    Bs = [torch.tensor(p[2], device=DEV) for p in probs]
    opts = cola.cola_cg_opts_default(precision=cola.PREC_F32, refine=1, tol=1e-8, maxiter=20000,
                                     graph_chunk=16)
    Xs, info, st = cola.cola_cg_solve_batched(ctx, ops, Bs, opts)
    assert st == 0
    for p, X in zip(probs, Xs):
        res = krylov.true_relative_residual(oracle_tree(p[3]), p[2], X.cpu().numpy())
        assert np.all(res <= 1e-8)


# ----------------------------------------------------------------- tensor cores
# Split-BF16 contraction error: with T terms per operand the unrepresented
# remainder is below 2^-(8T+1) of each entry and dropped cross terms are of
# the same order, so per mode the error is < ~3 * 2^-(8T) of sum|K||x|.
MIXED_TOL = {1: 2e-2, 2: 2e-4, 3: 3e-6}


@pytest.mark.parametrize("name", ["kron_rect", "kron_shift"])
@pytest.mark.parametrize("terms", [1, 2, 3])
def test_matvec_mixed_parity(cola, ctx, name, terms):
    spec = _zoo()[name]
    ref = oracle_tree(spec)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV)
    X = _rs(6).standard_normal((3, ref.cols))
    absop = oracle_tree(_abs_spec(spec))
    scale = np.max(absop.mvm(np.abs(X)))
    Y = cola.cola_matvec(ctx, op, torch.tensor(X, dtype=torch.float32, device=DEV),
                         cola.PREC_MIXED, split_terms=terms)
    err = float(np.max(np.abs(Y.double().cpu().numpy() - ref.mvm(X))))
    assert err < MIXED_TOL[terms] * scale, (err / scale)


def _abs_spec(spec):
    k = spec[0]
    if k in ("dense", "diag"):
        return (k, np.abs(spec[1]))
    if k == "scalar":
        return (k, abs(spec[1]), spec[2])
    if k == "lowrank":
        return spec
    if k in ("kron", "kronsum", "product"):
        return (k, [_abs_spec(s) for s in spec[1]])
    return (k, [_abs_spec(s) for s in spec[1]], spec[2])


def test_matvec_mixed_kron3_full_size_sampled(cola, ctx):
    w = wl.config2(nrhs=2)
    spec = ("sum", [("kron", [("dense", f) for f in w.factors]), ("scalar", w.shift, w.N)], None)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV)
    X = torch.tensor(w.B, dtype=torch.float32, device=DEV)
    Yh = cola.cola_matvec(ctx, op, X, cola.PREC_MIXED, split_terms=3).double().cpu().numpy()
    K1, K2, K3 = w.factors
    n = 128
    idx = _rs(8).integers(0, w.N, size=40)
    for r in range(2):
        Xr = w.B[r].reshape(n, n, n)
        for I in idx:
            i1, i2, i3 = I // (n * n), (I // n) % n, I % n
            row = np.einsum("a,b,c->abc", K1[i1], K2[i2], K3[i3])
            ref = float(np.sum(row * Xr)) + w.shift * Xr[i1, i2, i3]
            bound = float(np.sum(row * np.abs(Xr))) + w.shift * abs(Xr[i1, i2, i3])
            assert abs(Yh[r, I] - ref) <= MIXED_TOL[3] * 3 * bound


@pytest.mark.parametrize("n1", [1, 24, 128])
@pytest.mark.parametrize("terms", [2, 3])
def test_matvec_mixed_slab_path_parity(cola, ctx, n1, terms):
    """A three-factor Kronecker product with 128 x 128 second and third
    factors runs as the first mode step (slab-major output) and the slab
    kernel (modes 2 and 3 on chip): every entry matches the oracle's mode
    products within the split-term bound, for a first factor of side 1 (one
    slab per right-hand side), a ragged 24 and the full 128, with a
    coefficient on the product."""
    F = [wl.rbf_factor(wl.uniform(wl.substream(640 + n1, k), (n,)), 0.15)
         for k, n in enumerate((n1, 128, 128))]
    spec = ("sum", [("kron", [("dense", f) for f in F])], [2.5])
    ref = oracle_tree(spec)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV)
    X = _rs(641).standard_normal((3, ref.cols))
    Y = cola.cola_matvec(ctx, op, torch.tensor(X, dtype=torch.float32, device=DEV),
                         cola.PREC_MIXED, split_terms=terms).double().cpu().numpy()
    bound = oracle_tree(_abs_spec(spec)).mvm(np.abs(X))
    err = np.abs(Y - ref.mvm(X))
    assert np.all(err <= 3 * MIXED_TOL[terms] * bound + 1e-30), float(np.max(err / bound))


def _tridiag(n, seed):
    r = _rs(seed)
    T = np.diag(2.0 + r.random(n))
    if n > 1:
        T += np.diag(-0.5 - r.random(n - 1), 1) + np.diag(-0.5 - r.random(n - 1), -1)
    return T


@pytest.mark.parametrize("sides", [(1, 4), (5, 44), (37, 44), (130, 128)],
                         ids=lambda s: f"{s[0]}x{s[1]}")
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("diag", ["per_element", "scalar"])
def test_matvec_tridiag_kronsum_stencil_parity(cola, ctx, sides, prec, diag):
    """A Kronecker sum of two (non-symmetric) tridiagonal factors with a
    diagonal term runs as the two-factor stencil (one row quad per thread at
    these sizes): every entry matches the oracle, for one row, and column-quad
    counts that are not multiples of a warp."""
    _stencil_case(cola, ctx, sides, prec, diag, 3)


def _stencil_case(cola, ctx, sides, prec, diag, nrhs):
    n1, n2 = sides
    T1, T2 = _tridiag(n1, 650 + n1), _tridiag(n2, 651 + n2)
    N = n1 * n2
    dterm = ("diag", 0.5 + _rs(652).random(N)) if diag == "per_element" else ("scalar", 0.3, N)
    spec = ("sum", [("kronsum", [("dense", T1), ("dense", T2)]), dterm], [1.5, 0.5])
    ref = oracle_tree(spec)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV)
    X = _rs(653).standard_normal((nrhs, N))
    P = cola.PREC_F64 if prec == "f64" else cola.PREC_F32
    dt = torch.float64 if prec == "f64" else torch.float32
    Y = cola.cola_matvec(ctx, op, torch.tensor(X, dtype=dt, device=DEV), P).double().cpu().numpy()
    Yr = ref.mvm(X)
    tol = 1e-13 if prec == "f64" else 1e-6
    bound = oracle_tree(_abs_spec(spec)).mvm(np.abs(X))
    assert np.all(np.abs(Y - Yr) <= tol * bound + 1e-300), float(np.max(np.abs(Y - Yr) / bound))


@pytest.mark.parametrize("prec,diag", [("f32", "per_element"), ("f64", "scalar")])
def test_matvec_tridiag_kronsum_strips_parity(cola, ctx, prec, diag):
    """Enough rows for the stencil's strip form (a thread walks 16 rows of one
    column quad): 1037 rows (a ragged last strip of 13), 1028 columns (257
    quads per row, so warps straddle rows and strips), 8 right-hand sides;
    every entry against the oracle."""
    _stencil_case(cola, ctx, (1037, 1028), prec, diag, 8)


def test_matvec_on_library_stream_matches_joined_call(cola, ctx):
    """A caller working on the context's own stream (no cross-stream join)
    gets bit-identical results to a call from another stream, also for calls
    queued back to back before the device reaches them."""
    w = wl.config2(nrhs=2)
    spec = ("sum", [("kron", [("dense", f) for f in w.factors]), ("scalar", w.shift, w.N)], None)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV)
    X = torch.tensor(w.B, dtype=torch.float32, device=DEV)
    ref = cola.cola_matvec(ctx, op, X, cola.PREC_MIXED, split_terms=3)
    torch.cuda.synchronize()
    ls = ctx.stream()
    outs = [torch.empty_like(X) for _ in range(3)]
    with torch.cuda.stream(ls):
        torch.cuda._sleep(2_000_000)
        for o in outs:
            cola.cola_matvec(ctx, op, X, cola.PREC_MIXED, out=o, split_terms=3)
    torch.cuda.synchronize()
    for o in outs:
        assert torch.equal(o, ref)


@pytest.mark.parametrize("terms", [(2, 2), (3, 2), (3, 3)])
def test_cg_mixed_reaches_1e8(cola, ctx, terms):
    K1, K2, B, spec = _kron_shift_problem(64, 96, 0.01, 4, 15)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    opts = cola.cola_cg_opts_default(precision=cola.PREC_MIXED, refine=1, tol=1e-8,
                                     maxiter=20000, split_factor_terms=terms[0],
                                     split_vector_terms=terms[1])
    X, info, st = cola.cola_cg_solve(ctx, op, torch.tensor(B, device=DEV), opts)
    assert st == 0, info
    res = krylov.true_relative_residual(oracle_tree(spec), B, X.cpu().numpy())
    assert np.all(res <= 1e-8), res


def test_batched_mixed_uneven_one_launch_per_step(cola, ctx):
    """Table-driven batched solve: systems of uneven factor sizes (16..200,
    so some need two output chunks) and 1..5 right-hand sides advance together
    through one tensor-core launch per mode step; every right-hand side reaches
    1e-8 (FP64 true residual) and matches the exact Kronecker solve."""
    shapes = [(16, 16, 0.1, 1), (200, 24, 0.05, 3), (33, 130, 0.01, 2), (64, 64, 0.003, 5),
              (17, 45, 0.02, 1), (128, 96, 0.001, 2)]
    probs = [_kron_shift_problem(n1, n2, s, r, 400 + i) for i, (n1, n2, s, r) in enumerate(shapes)]
    ops = [gpu_tree(cola, ctx, p[3], torch.float64, DEV).set_spd() for p in probs]
    Bs = [torch.tensor(p[2], device=DEV) for p in probs]
    opts = cola.cola_cg_opts_default(precision=cola.PREC_MIXED, refine=1, tol=1e-8, maxiter=40000,
                                     graph_chunk=16)
    Xs, info, st = cola.cola_cg_solve_batched(ctx, ops, Bs, opts)
    assert st == 0, [i for i in info if i["status"] != 0][:3]
    for (K1, K2, B, spec), X, (n1, n2, s, r) in zip(probs, Xs, shapes):
        res = krylov.true_relative_residual(oracle_tree(spec), B, X.cpu().numpy())
        assert np.all(res <= 1e-8), res
        x_ref = exact.kron_shift_solve([K1, K2], s, B)
        assert np.max(np.abs(X.cpu().numpy() - x_ref)) <= 1e-4 * np.max(np.abs(x_ref))
    assert all(i["rel_residual"] <= 1e-8 for i in info)


@pytest.mark.parametrize("n,k,nrhs", [(40004, 36, 11), (4096, 4, 8), (1048576, 32, 8)])
def test_lowrank_vectorised_parity(cola, ctx, n, k, nrhs):
    """The FP32 low-rank product on its 16-byte paths (n and k multiples of 4),
    added to a diagonal term's output: a ragged last 128-row stage, a partial
    second 32-column group, a partial second group of 8 right-hand sides, and
    the 2^20 x 32 PDE-workload shape."""
    r = _rs(150)
    U = r.standard_normal((n, k)) / np.sqrt(n)
    V = r.standard_normal((n, k)) / np.sqrt(n)
    spec = ("sum", [("diag", 0.5 + r.random(n)), ("lowrank", U, V)], [1.0, 1.5])
    ref = oracle_tree(spec)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV)
    X = r.standard_normal((nrhs, n))
    Y = cola.cola_matvec(ctx, op, torch.tensor(X, dtype=torch.float32, device=DEV),
                         cola.PREC_F32)
    err = rel_max_err(Y.double().cpu().numpy(), ref.mvm(X))
    assert err < 2e-6, err


def test_poisson_lowrank_full_size(cola, ctx):
    """A = (L (+) L) + D + U U^T with the 1024-point Dirichlet Laplacian
    (N = 1,048,576), U 32 columns, 8 right-hand sides: Jacobi PCG in FP32 to
    1e-6, checked with the oracle's FP64 residual; the Kronecker-sum factor is
    applied as a stencil (tridiagonal detected at construction)."""
    w = wl.config3()
    spec = ("sum", [("kronsum", [("dense", w.L), ("dense", w.L)]), ("diag", w.d),
                    ("lowrank", w.U, None)], None)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    opts = cola.cola_cg_opts_default(precision=cola.PREC_F32, refine=0, tol=w.tol, jacobi=1,
                                     maxiter=1000, graph_chunk=8)
    X, info, st = cola.cola_cg_solve(ctx, op, torch.tensor(w.B, dtype=torch.float32, device=DEV),
                                     opts)
    assert st == 0, info[:2]
    res = krylov.true_relative_residual(oracle_tree(spec), w.B, X.double().cpu().numpy())
    assert np.all(res <= 2e-6), res
    assert max(i["iterations"] for i in info) < 200


def test_prepared_copies_reused_and_refreshed_after_in_place_update(cola, ctx):
    """A MIXED MVM reuses the leaves' FP32 copies and split images across calls
    (only the 2 mode steps launch the second time), and an in-place update of
    a factor tensor is picked up on the next call (version counter -> touch)."""
    r = _rs(140)
    K1 = torch.tensor(_spd(32, 141), device=DEV)
    K2 = torch.tensor(_spd(48, 142), device=DEV)
    op = cola.cola_linop_kron(ctx, cola.cola_linop_dense(ctx, K1), cola.cola_linop_dense(ctx, K2))
    X = torch.tensor(r.standard_normal((2, 32 * 48)), dtype=torch.float32, device=DEV)
    Y1 = cola.cola_matvec(ctx, op, X, cola.PREC_MIXED, split_terms=3)
    torch.cuda.synchronize()
    l0 = ctx.kernel_launches()
    Y1b = cola.cola_matvec(ctx, op, X, cola.PREC_MIXED, split_terms=3)
    torch.cuda.synchronize()
    assert ctx.kernel_launches() - l0 == 2
    assert torch.equal(Y1, Y1b)
    K1.mul_(2.0)
    Y2 = cola.cola_matvec(ctx, op, X, cola.PREC_MIXED, split_terms=3)
    ref = oracle_tree(("kron", [("dense", K1.cpu().numpy()), ("dense", K2.cpu().numpy())]))
    err = np.abs(Y2.double().cpu().numpy() - ref.mvm(X.double().cpu().numpy())).max()
    assert err <= 1e-5 * np.abs(Y2.double().cpu().numpy()).max()
    torch.testing.assert_close(Y2, 2.0 * Y1, rtol=1e-5, atol=1e-5)


@pytest.mark.parametrize("sides", [(24, 20, 16), (160, 24)], ids=["factor_stationary", "split_gemm"])
def test_lanczos_mixed_fused_matches_oracle(cola, ctx, sides):
    """MIXED Lanczos on K (x) ... + 0.05 I runs the recurrence fused into the
    tensor-core MVM (normalisation in the first mode step's prologue, shift,
    three-term subtraction and alpha partials in the last one's epilogue).  Its
    coefficients match the oracle's Lanczos on the same probes for the steps
    before orthogonality is lost (3 x 3 split terms: FP32-level rounding)."""
    F = [_spd(n, 500 + n) for n in sides]
    N = int(np.prod(sides))
    spec = ("sum", [("kron", [("dense", f) for f in F]), ("scalar", 0.05, N)], None)
    ref = oracle_tree(spec)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    Z = rng.rademacher_probes(9, 3, N)
    m, j0 = 12, 8
    al, be, me = cola.cola_lanczos(ctx, op, torch.tensor(Z, dtype=torch.float32, device=DEV), m,
                                   cola.PREC_MIXED, reorth=0, split_terms=3)
    al, be, me = al.cpu().numpy(), be.cpu().numpy(), me.cpu().numpy()
    for v in range(3):
        a, b, _ = krylov.lanczos(ref, Z[v], m, reorth=False)
        assert me[v] == m
        np.testing.assert_allclose(al[v, :j0], a[:j0], rtol=1e-5)
        np.testing.assert_allclose(be[v, :j0], b[:j0], rtol=1e-5)


@pytest.mark.parametrize("shapes", [[(132, 120), (40, 36)], [(128, 128), (128, 128), (128, 128)]],
                         ids=["ragged", "cube128"])
def test_matvec_f32_mode_kernel_parity(cola, ctx, shapes):
    """The FP32 SIMT mode-product kernel (double-buffered 128 x 128 tiles)
    on shapes with M, N and K tails (132 x 120 and 40 x 36 factors) and on
    the 128^3 cube, against the oracle's mode products: within 2e-6 of
    max |A x| (an n-term FP32 dot product per mode)."""
    r = _rs(600)
    F = [r.standard_normal(s) / np.sqrt(s[1]) for s in shapes]
    spec = ("kron", [("dense", f) for f in F])
    ref = oracle_tree(spec)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV)
    X = r.standard_normal((2, ref.cols))
    Y = cola.cola_matvec(ctx, op, torch.tensor(X, dtype=torch.float32, device=DEV),
                         cola.PREC_F32).double().cpu().numpy()
    Y_ref = ref.mvm(X)
    assert rel_max_err(Y, Y_ref) < 2e-6


def test_cg_and_lanczos_mixed_slab_path(cola, ctx):
    """K1 (x) K2 (x) K3 + 0.02 I with 128 x 128 second and third factors: the
    fused Lanczos MVM runs through the slab kernel (steps 2 and 3 of the
    Kronecker product on chip per (right-hand side, i1) slab) and its
    coefficients match the oracle's on the same probes for the steps before
    orthogonality is lost; the fused three-step CG on the same operator (MIXED
    3 x 3 with FP64 refinement) reaches 1e-8 (oracle FP64 true residual) and
    matches the exact eigen-structured solve within the forward-error bound."""
    sides = (24, 128, 128)
    F = [wl.rbf_factor(wl.uniform(wl.substream(610, k), (n,)), 0.15) for k, n in enumerate(sides)]
    N = int(np.prod(sides))
    spec = ("sum", [("kron", [("dense", f) for f in F]), ("scalar", 0.02, N)], None)
    ref = oracle_tree(spec)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    B = wl.normal(wl.substream(610, 9), (3, N))
    opts = cola.cola_cg_opts_default(precision=cola.PREC_MIXED, refine=1, tol=1e-8,
                                     maxiter=40000, split_factor_terms=3, split_vector_terms=3)
    X, info, st = cola.cola_cg_solve(ctx, op, torch.tensor(B, device=DEV), opts)
    assert st == 0, info
    Xh = X.cpu().numpy()
    res = krylov.true_relative_residual(ref, B, Xh)
    assert np.all(res <= 1e-8), res
    lam = exact.kron_eigenvalues(F, 0.02)
    x_ref = exact.kron_shift_solve(F, 0.02, B)
    fe = np.linalg.norm(Xh - x_ref, axis=1) / np.linalg.norm(x_ref, axis=1)
    assert np.all(fe <= lam.max() / lam.min() * 1e-8), fe
    Z = rng.rademacher_probes(611, 2, N)
    al, be, me = cola.cola_lanczos(ctx, op, torch.tensor(Z, dtype=torch.float32, device=DEV), 12,
                                   cola.PREC_MIXED, reorth=0, split_terms=3)
    al, be = al.cpu().numpy(), be.cpu().numpy()
    for v in range(2):
        a, b, _ = krylov.lanczos(ref, Z[v], 12, reorth=False)
        np.testing.assert_allclose(al[v, :8], a[:8], rtol=1e-5)
        np.testing.assert_allclose(be[v, :8], b[:8], rtol=1e-5)


@pytest.mark.parametrize("terms", [1, 2, 3])
@pytest.mark.parametrize("shapes", [[(257, 131), (24, 16), (150, 200)], [(257, 131), (150, 200)]],
                         ids=["three_factor", "two_factor_chained"])
def test_matvec_mixed_split_gemm_parity(cola, ctx, terms, shapes):
    """Factors with a side above 128 take the split GEMM mode step (the mode
    step's input pre-split into K-major BF16 images, both operands moved by
    copy engines, double-buffered accumulators): a three-factor product that
    mixes it with the factor-stationary kernel (257 x 131, 24 x 16 and
    150 x 200 factors: ragged row tiles, k blocks and 128-output chunks), and
    a two-factor product whose first step's epilogue writes the second step's
    split image; 3 right-hand sides, per entry within the mode steps' split
    error of sum |K||x|."""
    r = _rs(700)
    F = [r.standard_normal(sh) / np.sqrt(sh[1]) for sh in shapes]
    spec = ("kron", [("dense", f) for f in F])
    ref = oracle_tree(spec)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV)
    X = r.standard_normal((3, ref.cols)).astype(np.float32).astype(np.float64)
    Y = cola.cola_matvec(ctx, op, torch.tensor(X, dtype=torch.float32, device=DEV),
                         cola.PREC_MIXED, split_terms=terms).double().cpu().numpy()
    bound = oracle_tree(_abs_spec(spec)).mvm(np.abs(X))
    assert np.max(np.abs(Y - ref.mvm(X)) / bound) < 3 * MIXED_TOL[terms]


def test_cg_and_lanczos_mixed_split_gemm(cola, ctx):
    """K1 (x) K2 + 0.05 I with 200- and 150-point RBF factors, both mode
    steps on the split GEMM path.  CG (p = r + beta p formed in the pre-split
    pass, the shift term and the p . Ap partials in the GEMM epilogue; MIXED
    3 x 3 with FP64 refinement) reaches 1e-8 by the oracle's FP64 true
    residual and matches the exact eigen-structured solve within the
    forward-error bound; Lanczos (q = w / beta in the pre-split pass, the
    three-term subtraction and alpha partials in the epilogue) matches the
    oracle's coefficients on the same probes before orthogonality is lost."""
    sides = (200, 150)
    F = [wl.rbf_factor(wl.uniform(wl.substream(710, k), (n,)), 0.2) for k, n in enumerate(sides)]
    N = int(np.prod(sides))
    spec = ("sum", [("kron", [("dense", f) for f in F]), ("scalar", 0.05, N)], None)
    ref = oracle_tree(spec)
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV).set_spd()
    B = wl.normal(wl.substream(710, 9), (3, N))
    opts = cola.cola_cg_opts_default(precision=cola.PREC_MIXED, refine=1, tol=1e-8,
                                     maxiter=40000, split_factor_terms=3, split_vector_terms=3)
    X, info, st = cola.cola_cg_solve(ctx, op, torch.tensor(B, device=DEV), opts)
    assert st == 0, info
    Xh = X.cpu().numpy()
    res = krylov.true_relative_residual(ref, B, Xh)
    assert np.all(res <= 1e-8), res
    lam = exact.kron_eigenvalues(F, 0.05)
    x_ref = exact.kron_shift_solve(F, 0.05, B)
    fe = np.linalg.norm(Xh - x_ref, axis=1) / np.linalg.norm(x_ref, axis=1)
    assert np.all(fe <= lam.max() / lam.min() * 1e-8), fe
    Z = rng.rademacher_probes(11, 3, N)
    m, j0 = 12, 8
    al, be, me = cola.cola_lanczos(ctx, op, torch.tensor(Z, dtype=torch.float32, device=DEV), m,
                                   cola.PREC_MIXED, reorth=0, split_terms=3)
    al, be, me = al.cpu().numpy(), be.cpu().numpy(), me.cpu().numpy()
    for v in range(3):
        a, b, _ = krylov.lanczos(ref, Z[v], m, reorth=False)
        assert me[v] == m
        np.testing.assert_allclose(al[v, :j0], a[:j0], rtol=1e-5)
        np.testing.assert_allclose(be[v, :j0], b[:j0], rtol=1e-5)
