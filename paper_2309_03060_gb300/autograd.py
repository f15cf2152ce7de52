"""torch.autograd wrappers of the adjoint rules (CoLA App. B.2).

* ``solve``: X = A^-1 B.  Backward: gradB = A^-T gradX (a second CG solve with
  the same kernels) and, for every leaf theta of A,
  dL/dtheta = -(A^-T gradX)^T (dA/dtheta) X  (rule 1).  Only X is saved; no
  Krylov iterate is stored.
* ``gp_objective``: L = 1/2 y^T A^-1 y + 1/2 log det A (cola_gp_objective).
  The forward solves [y, z_1 .. z_m] as one block (the probes reuse the
  solve, App. D GP training) and estimates log det A by SLQ; the backward
  (cola_gp_objective_backward) is one weighted bilinear-gradient call:
      dL/dtheta = -1/2 a^T (dA/dtheta) a + 1/2 (1/m) sum_k u_k^T (dA/dtheta) z_k,
  a = A^-1 y, u_k = A^-1 z_k (rules 1 and 4 with the Hutchinson trace of App. B.1),
  and dL/dy = a.

Operators are built by the caller from the leaf tensors that are passed in;
gradients come back in the leaves' shapes and dtypes.  All arithmetic runs in
the CUDA library.
"""
from __future__ import annotations

import torch

from . import (PREC_F64, ColaError, cola_cg_opts_default, cola_cg_solve, cola_gp_objective,
               cola_gp_objective_backward, cola_solve_backward)


def _require_converged(st, info):
    if st != 0:
        bad = [i for i in info if i["status"] != 0][:3]
        raise ColaError(st, f"forward solve did not converge: {bad}")


def _reshape_like(grads, leaves):
    return [g.reshape(l.shape).to(l.dtype) for g, l in zip(grads, leaves)]


class _Solve(torch.autograd.Function):
    @staticmethod
    def forward(fctx, cctx, op, opts, B, *leaves):
        X, info, st = cola_cg_solve(cctx, op, B.detach(), opts)
        _require_converged(st, info)
        fctx.cctx, fctx.op, fctx.opts = cctx, op, opts
        fctx.save_for_backward(X)
        fctx.leaf_meta = [(l.shape, l.dtype) for l in leaves]
        fctx.info = info
        return X

    @staticmethod
    def backward(fctx, gradX):
        (X,) = fctx.saved_tensors
        gradB, grads, _, _ = cola_solve_backward(
            fctx.cctx, fctx.op, X, gradX.contiguous().to(X.dtype), fctx.opts,
            leaf_dtypes=[d for _, d in fctx.leaf_meta])
        lg = [g.reshape(s) for g, (s, _) in zip(grads, fctx.leaf_meta)]
        return (None, None, None, gradB, *lg)


def solve(cctx, op, B, leaves, opts=None):
    """X = A^-1 B with gradients for B and for every leaf tensor in ``leaves``
    (the tensors the operator was built from, in tree order)."""
    opts = opts or cola_cg_opts_default()
    return _Solve.apply(cctx, op, opts, B, *leaves)


class _GPObjective(torch.autograd.Function):
    @staticmethod
    def forward(fctx, cctx, op, opts, Z, slq_steps, y, *leaves):
        want = torch.float64 if (opts.precision == PREC_F64 or opts.refine) else torch.float32
        Zs = Z.to(want).contiguous()
        val, Sol, ld, se, info, st = cola_gp_objective(
            cctx, op, y.detach().reshape(-1).to(want).contiguous(), Zs, slq_steps, opts)
        _require_converged(st, info)
        fctx.cctx, fctx.op = cctx, op
        fctx.save_for_backward(Sol, Zs)
        fctx.leaf_meta = [(l.shape, l.dtype) for l in leaves]
        fctx.y_meta = (y.shape, y.dtype)
        fctx.logdet, fctx.logdet_se, fctx.info = ld, se, info
        return torch.tensor(val, dtype=y.dtype, device=y.device)

    @staticmethod
    def backward(fctx, g):
        Sol, Zs = fctx.saved_tensors
        # FP64 contractions whenever the solve returned FP64 vectors: the
        # lengthscale gradients are differences of O(1e7) terms
        prec = PREC_F64 if Sol.dtype == torch.float64 else 1
        grads, gy = cola_gp_objective_backward(
            fctx.cctx, fctx.op, Sol, Zs, float(g), prec,
            leaf_dtypes=[d for _, d in fctx.leaf_meta])
        lg = [gr.reshape(s) for gr, (s, _) in zip(grads, fctx.leaf_meta)]
        ys, yd = fctx.y_meta
        return (None, None, None, None, None, gy.reshape(ys).to(yd), *lg)


def gp_objective(cctx, op, y, leaves, Z, opts=None, slq_steps=30, seed=0):
    """L = 1/2 y^T A^-1 y + 1/2 log det A with the adjoint backward above (both
    computed by the library: cola_gp_objective / cola_gp_objective_backward).
    ``Z`` holds the Rademacher probes (nprobes x N) shared by the trace
    estimate of the gradient and the SLQ log-det; ``seed`` is accepted for
    compatibility and not used (both estimates always take Z)."""
    opts = opts or cola_cg_opts_default()
    return _GPObjective.apply(cctx, op, opts, Z, slq_steps, y, *leaves)
