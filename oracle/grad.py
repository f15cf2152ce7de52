"""Parameter gradients of bilinear forms u^T A x (FP64).  Test infrastructure only.

App. B.2 flattens an operator into its differentiable leaves theta and gives,
for y = A^-1 b,  w^T dy/dtheta = -(A^-1 w)^T (dA/dtheta) (A^-1 b)  (rule 1),
and for y = log det A,  dy/dtheta = Tr(A^-1 dA/dtheta)  (rule 4), which the
Hutchinson estimator (App. B.1) turns into mean_k (A^-1 z_k)^T (dA/dtheta) z_k.

Both reduce to the weighted bilinear form
    g(theta) = sum_r w_r u_r^T (dA/dtheta) x_r,
computed here per leaf, in the leaf's own shape.

``bilinear_grad_bruteforce`` follows the definition entry by entry: it builds
dA/dtheta_e for every entry e of every leaf (the tree with that leaf replaced
by the unit direction E_e, see ``linop.derivative``) and applies it.  It is
O(#entries * MVM) and meant for tiny trees.

``bilinear_grad`` evaluates the same sums in contracted form for larger trees
(the contraction over all modes but one for Kronecker factors).
"""
from __future__ import annotations

import numpy as np

from .linop import (Dense, Diag, Kron, KronSum, LowRank, Product, Sum,
                    _mode_product, derivative)


def bilinear_grad_bruteforce(op, U, X, w=None):
    U = np.atleast_2d(U)
    X = np.atleast_2d(X)
    w = np.ones(U.shape[0]) if w is None else np.asarray(w, dtype=np.float64)
    out = []
    for leaf in op.leaves():
        p = np.asarray(leaf.param())
        g = np.zeros(p.shape)
        for e in np.ndindex(*p.shape) if p.ndim else [()]:
            E = np.zeros(p.shape)
            E[e] = 1.0
            D = derivative(op, leaf, E)
            g[e] = float(np.sum(w * np.sum(U * D.mvm(X), axis=1)))
        out.append(g)
    return out


def bilinear_grad(op, U, X, w=None):
    """Same result as ``bilinear_grad_bruteforce`` by contractions."""
    U = np.atleast_2d(np.asarray(U, dtype=np.float64))
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    w = np.ones(U.shape[0]) if w is None else np.asarray(w, dtype=np.float64)
    grads = {}
    _walk(op, U * w[:, None], X, 1.0, grads)
    return [grads[id(l)] for l in op.leaves()]


def _acc(grads, leaf, g):
    grads[id(leaf)] = grads.get(id(leaf), 0.0) + g


def _walk(op, Uw, X, scale, grads):
    """Accumulate d/dtheta [sum_r Uw_r^T (scale * op) X_r] into grads."""
    if isinstance(op, Dense):
        _acc(grads, op, scale * (Uw.T @ X))
    elif isinstance(op, Diag):
        if op.is_scalar:
            _acc(grads, op, np.asarray(scale * float(np.sum(Uw * X))))
        else:
            _acc(grads, op, scale * np.sum(Uw * X, axis=0))
    elif isinstance(op, LowRank):
        V = op._V()
        g = Uw.T @ (X @ V)                     # d/dU of u^T U V^T x
        if op.V is None:
            g = g + X.T @ (Uw @ op.U)          # U U^T: second occurrence of U
        _acc(grads, op, scale * g)
    elif isinstance(op, Sum):
        for c, t in zip(op.coeffs, op.terms):
            _walk(t, Uw, X, scale * c, grads)
    elif isinstance(op, Product):
        # u^T A_1 ... A_m x: leaf in A_i sees left vector (A_1..A_{i-1})^T u
        # and right vector A_{i+1} ... A_m x.
        m = len(op.terms)
        rights = [None] * m
        v = X
        for i in range(m - 1, -1, -1):
            rights[i] = v
            v = op.terms[i].mvm(v)
        left = Uw
        for i in range(m):
            _walk(op.terms[i], left, rights[i], scale, grads)
            left = op.terms[i].transpose().mvm(left)
    elif isinstance(op, Kron):
        R = X.shape[0]
        d = len(op.factors)
        xs = (R,) + tuple(f.cols for f in op.factors)
        us = (R,) + tuple(f.rows for f in op.factors)
        Xt = X.reshape(xs)
        Ut = Uw.reshape(us)
        for k, f in enumerate(op.factors):
            Z = Xt
            for m_, g in enumerate(op.factors):
                if m_ != k:
                    Z = _mode_product(g.dense(), Z, m_)
            axes = [0] + [1 + m_ for m_ in range(d) if m_ != k]
            # G[i, j] = sum over all other axes of U[.., i, ..] Z[.., j, ..]
            G = np.tensordot(Ut, Z, axes=(axes, axes))
            _leaf_from_mode_grad(f, G, scale, grads)
    elif isinstance(op, KronSum):
        R = X.shape[0]
        d = len(op.factors)
        shape = (R,) + tuple(f.rows for f in op.factors)
        Xt = X.reshape(shape)
        Ut = Uw.reshape(shape)
        for k, f in enumerate(op.factors):
            axes = [0] + [1 + m_ for m_ in range(d) if m_ != k]
            G = np.tensordot(Ut, Xt, axes=(axes, axes))
            _leaf_from_mode_grad(f, G, scale, grads)
    else:
        raise TypeError(type(op))


def _leaf_from_mode_grad(f, G, scale, grads):
    """Gradient wrt a factor acting on one mode, given G = dF/d(factor matrix)."""
    if isinstance(f, Dense):
        _acc(grads, f, scale * G)
    elif isinstance(f, Diag):
        if f.is_scalar:
            _acc(grads, f, np.asarray(scale * float(np.trace(G))))
        else:
            _acc(grads, f, scale * np.diag(G).copy())
    else:
        raise TypeError("Kronecker factors must be Dense or Diag leaves")
