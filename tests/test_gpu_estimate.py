"""Stochastic diagonal and trace estimators (cola_diag_estimate, Sec. 3.3 /
App. B.1) against the FP64 oracle.

With the same probes (the counter-based Rademacher stream both sides
generate bit-exactly) the estimate is a deterministic function of the
operator, so the CUDA result is compared entry by entry with the oracle's;
at the multi-task workload size the oracle computes sampled entries one by
one.  The statistical behaviour (unbiasedness within 4 standard errors of the
Rademacher variance formula) is checked at many probes."""
import numpy as np
import pytest

import workloads as wl
from oracle import stochastic
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


def _small_multitask():
    w = wl.multitask(terms=3, tasks=6, n=40)
    spec = ("sum", [("kron", [("dense", b), ("dense", k)]) for b, k in zip(w.B, w.K)],
            [float(c) for c in w.coeffs])
    return w, spec


@pytest.mark.parametrize("doubly", [True, False])
def test_estimate_parity_same_probes_f64(cola, ctx, doubly):
    w, spec = _small_multitask()
    N, n, seed = w.N, 8, 7
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV)
    diag, tr = cola.cola_diag_estimate(ctx, op, n, seed=seed, doubly=doubly,
                                       precision=cola.PREC_F64)
    ref_tree = oracle_tree(spec)
    if doubly:
        ref = stochastic.doubly_stochastic_diag(ref_tree.terms, ref_tree.coeffs,
                                                stochastic.probes(seed, 3, n, N))
    else:
        ref = stochastic.hutchinson_diag(ref_tree, stochastic.probes(seed, 1, n, N)[0])
    got = diag.cpu().numpy()
    scale = np.abs(ref_tree.dense()).sum(axis=1).max()
    assert np.abs(got - ref).max() <= 1e-13 * scale
    assert abs(tr - ref.sum()) <= 1e-12 * N * scale


@pytest.mark.parametrize("prec,tol", [("F32", 1e-5), ("MIXED", 2e-3)])
def test_estimate_parity_same_probes_low_precision(cola, ctx, prec, tol):
    w, spec = _small_multitask()
    N, n, seed = w.N, 8, 11
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV)
    diag, _ = cola.cola_diag_estimate(ctx, op, n, seed=seed, doubly=True,
                                      precision=getattr(cola, "PREC_" + prec))
    ref_tree = oracle_tree(spec)
    ref = stochastic.doubly_stochastic_diag(ref_tree.terms, ref_tree.coeffs,
                                            stochastic.probes(seed, 3, n, N))
    # each product is a sum of |A_i| |z| terms; bound relative to that scale
    scale = sum(c * np.abs(t.dense()).sum(axis=1).max()
                for c, t in zip(ref_tree.coeffs, ref_tree.terms))
    assert np.abs(diag.cpu().numpy() - ref).max() <= tol * scale


def test_estimate_unbiased_at_many_probes(cola, ctx):
    """n = 4096 probes per term: the trace estimates lie within 4 standard
    deviations (Rademacher variance formula) of the exact trace, and the
    diagonal estimate's mean squared error is of the predicted size."""
    w, spec = _small_multitask()
    op = gpu_tree(cola, ctx, spec, torch.float64, DEV)
    ref_tree = oracle_tree(spec)
    A = ref_tree.dense()
    n = 4096
    terms = [t.dense() for t in ref_tree.terms]
    v_base = stochastic.rademacher_trace_variance(A) / n
    v_dbl = sum(c * c * stochastic.rademacher_trace_variance(m)
                for c, m in zip(ref_tree.coeffs, terms)) / n
    for doubly, var in ((True, v_dbl), (False, v_base)):
        diag, tr = cola.cola_diag_estimate(ctx, op, n, seed=123, doubly=doubly,
                                           precision=cola.PREC_F64)
        assert abs(tr - np.trace(A)) <= 4 * np.sqrt(var), (doubly, tr, np.trace(A), var)
        # E ||diag_est - diag||^2 = sum_k Var[z_k (A z)_k] / n = sum_k sum_{l != k} A_kl^2 / n
        off = A - np.diag(np.diag(A))
        if doubly:
            mse = sum(c * c * np.sum((m - np.diag(np.diag(m))) ** 2)
                      for c, m in zip(ref_tree.coeffs, terms)) / n
        else:
            mse = np.sum(off ** 2) / n
        err = np.sum((diag.cpu().numpy() - np.diag(A)) ** 2)
        assert 0.5 * mse < err < 2.0 * mse, (doubly, err, mse)


def test_estimate_multitask_full_size_sampled(cola, ctx):
    """The multi-task workload (8 terms, 128 tasks x 1024 points, N = 131072),
    MIXED with 3 split terms, 16 probes per term: 40 sampled entries against
    the oracle computing (A_q z)_k = B_q[t] Z K_q[x]^T one entry at a time."""
    w = wl.multitask()
    T, n_pts = w.B[0].shape[0], w.K[0].shape[0]
    N, n, seed = w.N, 16, 5
    kids = []
    keep = []
    for b, k in zip(w.B, w.K):
        tb = torch.tensor(b, device=DEV)
        tk = torch.tensor(k, device=DEV)
        keep += [tb, tk]
        kids.append(cola.cola_linop_kron(ctx, cola.cola_linop_dense(ctx, tb),
                                         cola.cola_linop_dense(ctx, tk)))
    op = cola.cola_linop_sum(ctx, kids, [float(c) for c in w.coeffs])
    diag, tr = cola.cola_diag_estimate(ctx, op, n, seed=seed, doubly=True,
                                       precision=cola.PREC_MIXED, split_terms=3)
    got = diag.cpu().numpy()
    Zs = stochastic.probes(seed, len(w.B), n, N)
    idx = np.random.default_rng(9).integers(0, N, size=40)
    for k in idx:
        t, x = k // n_pts, k % n_pts
        ref = 0.0
        bound = 0.0
        for q, (b, kq, c) in enumerate(zip(w.B, w.K, w.coeffs)):
            Zq = Zs[q].reshape(n, T, n_pts)
            az = np.einsum("a,vab,b->v", b[t], Zq, kq[x])
            ref += c * np.mean(Zq[:, t, x] * az)
            bound += c * float(np.abs(b[t]).sum() * np.abs(kq[x]).sum())
        assert abs(got[k] - ref) <= 3 * 3e-6 * bound, (k, got[k], ref)
