"""Stochastic diagonal and trace estimators in FP64 (Sec. 3.3; App. B.1).
Test infrastructure only.

Hutchinson's estimator of Diag(A) averages z (.) A z over probe vectors z with
identity covariance; its sum is the trace estimate z^T A z.  For a sum
A = sum_i c_i A_i the doubly stochastic variant draws independent probes for
every term: Diag ~ sum_i c_i (1/n) sum_j z_ij (.) A_i z_ij.  The probes here
are Rademacher vectors.  For symmetric B and a Rademacher z,
Var[z^T B z] = 2 sum_{k != l} B_kl^2 (Hutchinson 1989), so
    Var[base trace]   = (2/n) sum_{k != l} A_kl^2,
    Var[doubly trace] = (2/n) sum_i c_i^2 sum_{k != l} (A_i)_kl^2,
the Rademacher form of the Gaussian-probe variances 2 Tr(A^2) / n and
(2/(nm)) Tr(S(A)) derived in App. B.1.

Probe layout shared with the CUDA path (a counter-based stream, see rng.py):
term i, probe v, entry k is output (i * n + v) * N + k of the stream seeded
with ``seed``; the base estimator uses term index 0.
"""
from __future__ import annotations

import numpy as np

from . import rng


def probes(seed: int, nterms: int, nprobes: int, N: int) -> np.ndarray:
    """Rademacher probe blocks, shape (nterms, nprobes, N)."""
    return rng.rademacher_probes(seed, nterms * nprobes, N).reshape(nterms, nprobes, N)


def hutchinson_diag(op, Z: np.ndarray) -> np.ndarray:
    """(1/n) sum_v z_v (.) A z_v for the probes Z (n, N)."""
    AZ = op.mvm(Z)
    return np.mean(Z * AZ, axis=0)


def doubly_stochastic_diag(terms, coeffs, Zs: np.ndarray) -> np.ndarray:
    """sum_i c_i (1/n) sum_v z_iv (.) A_i z_iv, Zs (nterms, n, N)."""
    out = np.zeros(Zs.shape[2])
    for c, t, Z in zip(coeffs, terms, Zs):
        out += c * hutchinson_diag(t, Z)
    return out


def rademacher_trace_variance(B: np.ndarray) -> float:
    """Var[z^T B z] for one Rademacher z and symmetric B."""
    off = B - np.diag(np.diag(B))
    return 2.0 * float(np.sum(off * off))
