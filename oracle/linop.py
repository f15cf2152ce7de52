"""Operator tree with MVM by definition (FP64).  Test infrastructure only.

Sec. 3.1: a linear operator is defined by its MVM; its dense form is obtained
by applying the MVM to each unit vector e_i.
Sec. 3.2: compositions Sum (MVM = sum of MVMs), Product (chained MVMs),
Kronecker A (x) B and Kronecker sum A (+) B = A (x) I + I (x) B.
App. A.1.4: Diag rules; App. A.1.5: transpose rules.

Vectors are row-major (C order): entry (i_1, ..., i_d) of a Kronecker-shaped
vector sits at index ((i_1 n_2 + i_2) n_3 + ...) .  With this convention
(K_1 (x) K_2) vec(X) = vec(K_1 X K_2^T) for X of shape (n_1, n_2), and
Diag(A (x) B) = vec(Diag(A) Diag(B)^T) as App. A.1.4 writes it.

Multi-RHS arrays have shape (nrhs, N).
"""
from __future__ import annotations

import numpy as np


class Op:
    rows: int
    cols: int

    # --- MVM -----------------------------------------------------------------
    def mvm(self, X: np.ndarray) -> np.ndarray:  # X: (R, cols) -> (R, rows)
        raise NotImplementedError

    def __matmul__(self, x):
        x = np.asarray(x, dtype=np.float64)
        if x.ndim == 1:
            return self.mvm(x[None, :])[0]
        return self.mvm(x)

    # --- derived by definition ---------------------------------------------
    def dense(self) -> np.ndarray:
        """Sec. 3.1: column i of the dense matrix is MVM(e_i)."""
        E = np.eye(self.cols)
        return self.mvm(E).T.copy()

    def diag_bruteforce(self) -> np.ndarray:
        """App. A.1.4 base case: Diag(A)_i = e_i^T A e_i."""
        n = min(self.rows, self.cols)
        out = np.empty(n)
        for i in range(n):
            e = np.zeros((1, self.cols))
            e[0, i] = 1.0
            out[i] = self.mvm(e)[0, i]
        return out

    # --- tree structure ----------------------------------------------------
    def children(self):
        return []

    def leaves(self):
        """Differentiable leaves in tree order (depth first, left to right):
        the flattened parameter tree of App. B.2."""
        out = []
        for c in self.children():
            out.extend(c.leaves())
        return out


# ============================================================================
# Base operators (Sec. 3.1)
# ============================================================================

class Dense(Op):
    """[A v]_i = sum_j A_ij v_j."""

    def __init__(self, M):
        self.M = np.asarray(M, dtype=np.float64)
        self.rows, self.cols = self.M.shape

    def mvm(self, X):
        return X @ self.M.T

    def transpose(self):
        return Dense(self.M.T)

    def dense(self):
        return self.M.copy()

    def diag(self):
        return np.diag(self.M).copy()

    def leaves(self):
        return [self]

    def param(self):
        return self.M

    def replaced(self, value):
        return Dense(value)


class Diag(Op):
    """[Diag(d) v]_i = d_i v_i.  A 0-d ``d`` means the scalar multiple d * I."""

    def __init__(self, d, n=None):
        self.d = np.asarray(d, dtype=np.float64)
        if self.d.ndim == 0:
            assert n is not None
            self.rows = self.cols = int(n)
        else:
            self.rows = self.cols = self.d.shape[0]

    @property
    def is_scalar(self):
        return self.d.ndim == 0

    def mvm(self, X):
        return X * self.d

    def transpose(self):
        return self

    def diag(self):
        return np.broadcast_to(self.d, (self.rows,)).astype(np.float64).copy()

    def leaves(self):
        return [self]

    def param(self):
        return self.d

    def replaced(self, value):
        return Diag(value, self.rows)


class LowRank(Op):
    """U V^T (V omitted means U U^T), the low-rank term of the Woodbury rule."""

    def __init__(self, U, V=None):
        self.U = np.asarray(U, dtype=np.float64)
        self.V = None if V is None else np.asarray(V, dtype=np.float64)
        self.rows = self.U.shape[0]
        self.cols = self.U.shape[0] if V is None else self.V.shape[0]

    def _V(self):
        return self.U if self.V is None else self.V

    def mvm(self, X):
        return (X @ self._V()) @ self.U.T

    def transpose(self):
        return self if self.V is None else LowRank(self.V, self.U)

    def diag(self):
        return np.sum(self.U * self._V(), axis=1)

    def leaves(self):
        return [self]

    def param(self):
        return self.U

    def replaced(self, value):
        return LowRank(value, self.V)


# ============================================================================
# Compositions (Sec. 3.2)
# ============================================================================

class Sum(Op):
    """MVM_Sum(v) = sum_i c_i MVM_i(v)."""

    def __init__(self, terms, coeffs=None):
        self.terms = list(terms)
        self.coeffs = [1.0] * len(self.terms) if coeffs is None else [float(c) for c in coeffs]
        self.rows, self.cols = self.terms[0].rows, self.terms[0].cols
        for t in self.terms:
            assert (t.rows, t.cols) == (self.rows, self.cols)

    def children(self):
        return self.terms

    def mvm(self, X):
        Y = np.zeros((X.shape[0], self.rows))
        for c, t in zip(self.coeffs, self.terms):
            Y += c * t.mvm(X)
        return Y

    def transpose(self):
        return Sum([t.transpose() for t in self.terms], self.coeffs)

    def diag(self):
        return sum(c * t.diag() for c, t in zip(self.coeffs, self.terms))


class Product(Op):
    """(A_1 A_2 ... A_m) v, applied right to left."""

    def __init__(self, terms):
        self.terms = list(terms)
        self.rows, self.cols = self.terms[0].rows, self.terms[-1].cols
        for a, b in zip(self.terms[:-1], self.terms[1:]):
            assert a.cols == b.rows

    def children(self):
        return self.terms

    def mvm(self, X):
        for t in reversed(self.terms):
            X = t.mvm(X)
        return X

    def transpose(self):
        return Product([t.transpose() for t in reversed(self.terms)])

    def diag(self):
        return self.diag_bruteforce()


def _mode_product(K: np.ndarray, X: np.ndarray, mode: int) -> np.ndarray:
    """Y[r, ..., i, ...] = sum_j K[i, j] X[r, ..., j, ...] along axis 1 + mode."""
    Y = np.tensordot(K, X, axes=([1], [1 + mode]))      # (m, r, ..., rest)
    return np.moveaxis(Y, 0, 1 + mode)


class Kron(Op):
    """K_1 (x) K_2 (x) ... (x) K_d; entry ((i_1..i_d),(j_1..j_d)) = prod_k K_k[i_k, j_k]."""

    def __init__(self, factors):
        self.factors = list(factors)
        self.rows = int(np.prod([f.rows for f in self.factors]))
        self.cols = int(np.prod([f.cols for f in self.factors]))

    def children(self):
        return self.factors

    def mvm(self, X):
        R = X.shape[0]
        T = X.reshape((R,) + tuple(f.cols for f in self.factors))
        for k, f in enumerate(self.factors):
            T = _mode_product(f.dense(), T, k)
        return T.reshape(R, self.rows)

    def transpose(self):
        return Kron([f.transpose() for f in self.factors])

    def diag(self):
        """Diag(A (x) B) = vec(Diag(A) Diag(B)^T), applied recursively."""
        out = np.ones(1)
        for f in self.factors:
            out = np.outer(out, f.diag()).ravel()
        return out


class KronSum(Op):
    """A_1 (+) ... (+) A_d = sum_k I (x) ... (x) A_k (x) ... (x) I (square A_k)."""

    def __init__(self, factors):
        self.factors = list(factors)
        for f in self.factors:
            assert f.rows == f.cols
        self.rows = self.cols = int(np.prod([f.rows for f in self.factors]))

    def children(self):
        return self.factors

    def mvm(self, X):
        R = X.shape[0]
        shape = (R,) + tuple(f.cols for f in self.factors)
        T = X.reshape(shape)
        Y = np.zeros(shape)
        for k, f in enumerate(self.factors):
            Y += _mode_product(f.dense(), T, k)
        return Y.reshape(R, self.rows)

    def transpose(self):
        return KronSum([f.transpose() for f in self.factors])

    def diag(self):
        """Diag(A (+) B) = vec(Diag(A) 1^T + 1 Diag(B)^T), applied recursively."""
        out = np.zeros(1)
        for f in self.factors:
            out = (out[:, None] + f.diag()[None, :]).ravel()
        return out


def identity(n):
    return Dense(np.eye(n))


# ============================================================================
# Derivative of the operator in the direction of one leaf (App. B.2).
# Every leaf occurs once in a tree, so A is linear in each Dense / Diag leaf:
# dA/dtheta_k [E] is the tree with leaf k replaced by E and every Sum term
# that does not contain leaf k dropped.  U U^T is quadratic in U, so its
# derivative in direction E is E U^T + U E^T.
# ============================================================================

def leaf_index_map(op):
    return {id(l): i for i, l in enumerate(op.leaves())}


def derivative(op, leaf, E):
    """Operator dA/d(leaf) applied to the direction E (same shape as the leaf),
    or None when ``leaf`` is not inside ``op``."""
    if op is leaf:
        if isinstance(op, LowRank):
            if op.V is None:
                return Sum([LowRank(E, op.U), LowRank(op.U, E)])
            return LowRank(E, op.V)
        return op.replaced(E)
    if isinstance(op, Sum):
        for c, t in zip(op.coeffs, op.terms):
            d = derivative(t, leaf, E)
            if d is not None:
                return Sum([d], [c])
        return None
    if isinstance(op, (Product, Kron)):
        kids = op.factors if isinstance(op, Kron) else op.terms
        for i, t in enumerate(kids):
            d = derivative(t, leaf, E)
            if d is not None:
                new = list(kids)
                new[i] = d
                return Kron(new) if isinstance(op, Kron) else Product(new)
        return None
    if isinstance(op, KronSum):
        for i, t in enumerate(op.factors):
            d = derivative(t, leaf, E)
            if d is not None:
                new = [identity(f.rows) for f in op.factors]
                new[i] = d
                return Kron(new)
        return None
    return None
