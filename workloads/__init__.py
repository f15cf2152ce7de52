"""Seeded synthetic inputs for the composed-operator workloads.

This module only draws numbers and lays out the input arrays (points, kernel
factors, right-hand sides, probes, diagonals, low-rank factors).  It holds
none of the method's arithmetic (no MVM, no Krylov step, no quadrature), so
both the FP64 oracle and the CUDA path consume identical bytes from it.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), evaluated counter-style:
output i of a stream seeded with ``s`` is ``mix64(s + (i + 1) * GAMMA)``,
which equals the i-th draw of the sequential generator.

* uniform in [0, 1): top 53 bits times 2^-53
* normal: Box-Muller on pairs of uniforms (FP64)
* Rademacher: +1 when the top bit is 0, else -1

The RBF factor is k(x, x') = exp(-(x - x')^2 / (2 l^2)) with output scale 1 on
1-D points, the reading taken for the paper's unspecified "RBF kernel"
(Appendix D, Fig. 2a / Fig. 3b settings).  Every factor draws its own points.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
BASE_SEED = 20230906
_M64 = (1 << 64) - 1


def _mix64_int(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset .. offset+count-1 of SplitMix64 seeded with ``seed``."""
    i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed & _M64) + i * np.uint64(GAMMA)
    return _mix64(state)


def substream(seed: int, tag: int) -> int:
    """Seed of an independent sub-stream, one per array of a workload."""
    return _mix64_int((seed ^ ((tag * 0xD1B54A32D192ED03) & _M64)) & _M64)


def uniform(seed: int, shape) -> np.ndarray:
    n = int(np.prod(shape))
    v = splitmix64(seed, n)
    return ((v >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)).reshape(shape)


def normal(seed: int, shape, std: float = 1.0) -> np.ndarray:
    n = int(np.prod(shape))
    m = (n + 1) // 2
    u = uniform(seed, (2 * m,))
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = rad * np.cos(2.0 * math.pi * u2)
    z[1::2] = rad * np.sin(2.0 * math.pi * u2)
    return (std * z[:n]).reshape(shape)


def rademacher(seed: int, shape) -> np.ndarray:
    n = int(np.prod(shape))
    v = splitmix64(seed, n)
    return np.where((v >> np.uint64(63)) == 0, 1.0, -1.0).reshape(shape)


def rbf_factor(points: np.ndarray, ell: float) -> np.ndarray:
    d = points[:, None] - points[None, :]
    return np.exp(-(d * d) / (2.0 * ell * ell))


def rbf_factor_dell(points: np.ndarray, ell: float) -> np.ndarray:
    """d/d ell of the RBF factor (input-side chain rule for lengthscale gradients)."""
    d = points[:, None] - points[None, :]
    k = np.exp(-(d * d) / (2.0 * ell * ell))
    return k * (d * d) / ell ** 3


def dirichlet_laplacian(n: int) -> np.ndarray:
    """The n x n 1-D Dirichlet Laplacian, tridiag(-1, 2, -1)."""
    L = 2.0 * np.eye(n)
    i = np.arange(n - 1)
    L[i, i + 1] = -1.0
    L[i + 1, i] = -1.0
    return L


# --------------------------------------------------------------------------
# The five workloads.  Each returns plain arrays; the operator they define is
# assembled by whoever consumes them (oracle tree or C-ABI handles).
# --------------------------------------------------------------------------

@dataclass
class KronShiftWorkload:
    """A = K_1 (x) ... (x) K_d + shift * I with RBF factors."""
    name: str
    factors: list          # list of (n_k, n_k) float64
    points: list
    ells: list
    shift: float
    B: np.ndarray          # (nrhs, N) float64
    tol: float
    slq_probes: int = 0
    slq_steps: int = 0
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(np.prod([f.shape[0] for f in self.factors]))


def kron_shift(name: str, sizes, ells, shift: float, nrhs: int, tol: float,
               seed: int, slq_probes: int = 0, slq_steps: int = 0) -> KronShiftWorkload:
    pts, facs = [], []
    for k, (n, ell) in enumerate(zip(sizes, ells)):
        x = uniform(substream(seed, 10 + k), (n,))
        pts.append(x)
        facs.append(rbf_factor(x, ell))
    N = int(np.prod(sizes))
    B = normal(substream(seed, 1), (nrhs, N))
    return KronShiftWorkload(name, facs, pts, list(ells), shift, B, tol,
                             slq_probes, slq_steps, seed)


def config1(scale: int = 64) -> KronShiftWorkload:
    """FP64 single solve: K1 (x) K2 + 0.1 I, 64-point RBF factors (l = 0.2)."""
    return kron_shift("kron2_rbf64_fp64", [scale, scale], [0.2, 0.2], 0.1, 1, 1e-10,
                      BASE_SEED + 1, slq_probes=16, slq_steps=50)


def config2(n: int = 128, nrhs: int = 16) -> KronShiftWorkload:
    """Mixed precision: K1 (x) K2 (x) K3 + 0.01 I, three n-point RBF factors (l = 0.1)."""
    return kron_shift(f"kron3_rbf{n}_mixed", [n, n, n], [0.1, 0.1, 0.1], 0.01, nrhs, 1e-8,
                      BASE_SEED + 2, slq_probes=32, slq_steps=100)


def kron_diag(name: str, sizes, ells, dmin: float, dmax: float, nrhs: int, tol: float,
              seed: int) -> KronShiftWorkload:
    """A = K_1 (x) ... (x) K_d + Diag(d): RBF factors as in kron_shift and a
    per-point noise variance d drawn uniformly from [dmin, dmax] (a
    heteroscedastic GP).  d is extra["d"]; shift is 0."""
    w = kron_shift(name, sizes, ells, 0.0, nrhs, tol, seed)
    w.extra["d"] = dmin + (dmax - dmin) * uniform(substream(seed, 3), (w.N,))
    return w


def config2_hetero(n: int = 128, nrhs: int = 16) -> KronShiftWorkload:
    """The mixed-precision Kronecker workload with per-point noise:
    K1 (x) K2 (x) K3 + Diag(d), d in [0.005, 0.015], three n-point RBF factors."""
    return kron_diag(f"kron3_rbf{n}_hetero", [n, n, n], [0.1, 0.1, 0.1], 0.005, 0.015, nrhs,
                     1e-8, BASE_SEED + 6)


@dataclass
class PoissonLowRankWorkload:
    """A = (L (+) L) + D + U U^T with the 1-D Dirichlet Laplacian L."""
    name: str
    L: np.ndarray
    d: np.ndarray
    U: np.ndarray
    B: np.ndarray
    tol: float

    @property
    def N(self) -> int:
        return self.L.shape[0] ** 2


def config3(n: int = 1024, rank: int = 32, nrhs: int = 8) -> PoissonLowRankWorkload:
    seed = BASE_SEED + 3
    N = n * n
    L = dirichlet_laplacian(n)
    d = 0.5 + uniform(substream(seed, 20), (N,))
    U = normal(substream(seed, 21), (N, rank), std=1.0 / math.sqrt(N))
    B = normal(substream(seed, 1), (nrhs, N))
    return PoissonLowRankWorkload("poisson2d_lowrank", L, d, U, B, 1e-6)


@dataclass
class BatchedWorkload:
    name: str
    systems: list          # list of KronShiftWorkload (2 factors each)
    tol: float


def config4(nsys: int = 512, nmin: int = 16, nmax: int = 256, rmax: int = 8) -> BatchedWorkload:
    seed = BASE_SEED + 4
    u = uniform(substream(seed, 30), (nsys, 6))
    systems = []
    for i in range(nsys):
        n1 = nmin + int(u[i, 0] * (nmax - nmin + 1))
        n2 = nmin + int(u[i, 1] * (nmax - nmin + 1))
        l1 = 0.05 + 0.45 * u[i, 2]
        l2 = 0.05 + 0.45 * u[i, 3]
        s = 10.0 ** (-3.0 + 2.0 * u[i, 4])
        r = 1 + int(u[i, 5] * rmax)
        systems.append(kron_shift(f"sys{i}", [n1, n2], [l1, l2], s, r, 1e-8,
                                  substream(seed, 1000 + i)))
    return BatchedWorkload("batched_kron2_uneven", systems, 1e-8)


@dataclass
class GPWorkload:
    name: str
    points: list
    ells: list
    sigma2: float
    y: np.ndarray          # (N,)
    Z: np.ndarray          # (nprobes, N) Rademacher
    tol: float

    @property
    def N(self) -> int:
        return int(np.prod([len(p) for p in self.points]))


def config5(n: int = 1024, nprobes: int = 32) -> GPWorkload:
    seed = BASE_SEED + 5
    pts = [uniform(substream(seed, 10 + k), (n,)) for k in range(2)]
    N = n * n
    y = normal(substream(seed, 1), (N,))
    Z = rademacher(substream(seed, 2), (nprobes, N))
    return GPWorkload("gp_kron2_rbf_grad", pts, [0.1, 0.2], 0.1, y, Z, 1e-8)


@dataclass
class BiPoissonWorkload:
    """The Bi-Poisson operator (L (+) L)^2 on an n x n Dirichlet grid, as the
    product of two Kronecker sums, with N(0, 1) right-hand sides."""
    name: str
    L: np.ndarray          # (n, n) tridiag(-1, 2, -1)
    B: np.ndarray          # (nrhs, n * n)
    tol: float
    maxiter: int

    @property
    def N(self) -> int:
        return self.L.shape[0] ** 2


def bipoisson(n: int = 1000, nrhs: int = 1) -> BiPoissonWorkload:
    """Fig. 2(b) setting: grid up to 1000^2, CG tolerance 1e-11.  The paper caps
    CG at 10K iterations; the residual bound for kappa(L (+) L) = 4.1e5 at
    n = 1000 allows up to ~10.4K per solve, so the cap here is 20K."""
    seed = BASE_SEED + 7
    B = normal(substream(seed, 1), (nrhs, n * n))
    return BiPoissonWorkload(f"bipoisson_{n}x{n}", dirichlet_laplacian(n), B, 1e-11, 20000)


@dataclass
class MultiTaskWorkload:
    """A multi-task GP covariance (linear model of coregionalisation):
    A = sum_q c_q B_q (x) K_q with task covariances B_q = a_q a_q^T + diag(k_q)
    (T x T) and RBF data kernels K_q (n x n) on shared 1-D points."""
    name: str
    B: list                # task factors (T, T)
    K: list                # data factors (n, n)
    coeffs: list

    @property
    def N(self) -> int:
        return self.B[0].shape[0] * self.K[0].shape[0]


def multitask(terms: int = 8, tasks: int = 128, n: int = 1024) -> MultiTaskWorkload:
    """The doubly stochastic estimators' workload (Sec. 3.3 names multi-task GPs
    as the Sum structure it targets): lengthscales 0.02..0.3, task loadings
    |N(0, 1)| (positively correlated tasks), task noise U[0.1, 1], coefficients
    U[0.5, 1.5]."""
    seed = BASE_SEED + 8
    x = uniform(substream(seed, 1), (n,))
    ells = 0.02 + 0.28 * uniform(substream(seed, 2), (terms,))
    coeffs = list(0.5 + uniform(substream(seed, 3), (terms,)))
    Bs, Ks = [], []
    for q in range(terms):
        a = np.abs(normal(substream(seed, 100 + q), (tasks,)))
        k = 0.1 + 0.9 * uniform(substream(seed, 200 + q), (tasks,))
        Bs.append(np.outer(a, a) + np.diag(k))
        Ks.append(rbf_factor(x, float(ells[q])))
    return MultiTaskWorkload(f"multitask_lmc{terms}_{tasks}x{n}", Bs, Ks, coeffs)
