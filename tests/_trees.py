"""Builds one operator tree twice: as an oracle tree (numpy, FP64) and as
C-ABI handles (device tensors).  Test-side helper; it holds no arithmetic.

Spec grammar (nested tuples):
  ("dense", M) | ("diag", d) | ("scalar", s, n) | ("lowrank", U, V_or_None)
  ("kron", [specs]) | ("kronsum", [specs]) | ("sum", [specs], coeffs_or_None)
  ("product", [specs])
"""
import numpy as np

from oracle import linop as O


def oracle_tree(spec):
    kind = spec[0]
    if kind == "dense":
        return O.Dense(spec[1])
    if kind == "diag":
        return O.Diag(spec[1])
    if kind == "scalar":
        return O.Diag(np.float64(spec[1]), spec[2])
    if kind == "lowrank":
        return O.LowRank(spec[1], spec[2])
    if kind == "kron":
        return O.Kron([oracle_tree(s) for s in spec[1]])
    if kind == "kronsum":
        return O.KronSum([oracle_tree(s) for s in spec[1]])
    if kind == "sum":
        return O.Sum([oracle_tree(s) for s in spec[1]], spec[2])
    if kind == "product":
        return O.Product([oracle_tree(s) for s in spec[1]])
    raise ValueError(kind)


def gpu_tree(cola, ctx, spec, dtype, device):
    import torch

    def t(a):
        return torch.tensor(np.asarray(a), dtype=dtype, device=device)

    kind = spec[0]
    if kind == "dense":
        return cola.cola_linop_dense(ctx, t(spec[1]))
    if kind == "diag":
        return cola.cola_linop_diag(ctx, t(spec[1]))
    if kind == "scalar":
        return cola.cola_linop_diag(ctx, t([spec[1]]), n=spec[2])
    if kind == "lowrank":
        return cola.cola_linop_lowrank(ctx, t(spec[1]), None if spec[2] is None else t(spec[2]))
    kids = [gpu_tree(cola, ctx, s, dtype, device) for s in spec[1]]
    if kind == "kron":
        return cola.cola_linop_kron(ctx, *kids)
    if kind == "kronsum":
        return cola.cola_linop_kronsum(ctx, *kids)
    if kind == "sum":
        return cola.cola_linop_sum(ctx, kids, spec[2])
    if kind == "product":
        return cola.cola_linop_product(ctx, kids)
    raise ValueError(kind)


def leaf_params(spec):
    """Leaf parameter arrays in tree order (matches cola_linop_leaf_info order)."""
    kind = spec[0]
    if kind in ("dense", "diag", "lowrank"):
        return [np.asarray(spec[1])]
    if kind == "scalar":
        return [np.asarray([spec[1]])]
    out = []
    for s in spec[1]:
        out.extend(leaf_params(s))
    return out
