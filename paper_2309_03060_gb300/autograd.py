"""torch.autograd wrappers of the adjoint rules (CoLA App. B.2).

* ``solve``: X = A^-1 B.  Backward: gradB = A^-T gradX (a second CG solve with
  the same kernels) and, for every leaf theta of A,
  dL/dtheta = -(A^-T gradX)^T (dA/dtheta) X  (rule 1).  Only X is saved; no
  Krylov iterate is stored.
* ``gp_objective``: L = 1/2 y^T A^-1 y + 1/2 log det A.  The forward solves
  [y, z_1 .. z_m] as one block (the probes reuse the solve, App. D GP
  training) and estimates log det A by SLQ; the backward is one weighted
  bilinear-gradient call:
      dL/dtheta = -1/2 a^T (dA/dtheta) a + 1/2 (1/m) sum_k u_k^T (dA/dtheta) z_k,
  a = A^-1 y, u_k = A^-1 z_k (rules 1 and 4 with the Hutchinson trace of App. B.1),
  and dL/dy = a.

Operators are built by the caller from the leaf tensors that are passed in;
gradients come back in the leaves' shapes and dtypes.  All arithmetic runs in
the CUDA library.
"""
from __future__ import annotations

import torch

from . import (PREC_F64, ColaError, cola_bilinear_grad, cola_cg_opts_default, cola_cg_solve,
               cola_slq_logdet, cola_solve_backward)


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
    def forward(fctx, cctx, op, opts, Z, slq_steps, seed, y, *leaves):
        m = Z.shape[0]
        block = torch.cat([y.detach().reshape(1, -1), Z], dim=0).contiguous()
        Sol, info, st = cola_cg_solve(cctx, op, block, opts)
        _require_converged(st, info)
        a = Sol[0]
        quad = 0.5 * torch.dot(y.detach().reshape(-1).to(a.dtype), a)
        prec = opts.precision
        # the SLQ log-det and the Hutchinson gradient use the same probes Z
        ld, se, _, _ = cola_slq_logdet(cctx, op, m, slq_steps, seed=seed,
                                       probes=Z.to(torch.float64 if prec == PREC_F64 else
                                                   torch.float32).contiguous(),
                                       precision=prec)
        fctx.cctx, fctx.op, fctx.opts = cctx, op, opts
        fctx.save_for_backward(Sol, Z)
        fctx.leaf_meta = [(l.shape, l.dtype) for l in leaves]
        fctx.logdet, fctx.logdet_se, fctx.info = ld, se, info
        return quad + 0.5 * torch.tensor(ld, dtype=quad.dtype, device=quad.device)

    @staticmethod
    def backward(fctx, g):
        Sol, Z = fctx.saved_tensors
        m = Z.shape[0]
        U = Sol                                     # [a, u_1 .. u_m]
        Xr = torch.cat([Sol[:1], Z.to(Sol.dtype)], dim=0).contiguous()
        w = [-0.5] + [0.5 / m] * m
        # FP64 contractions whenever the solve returned FP64 vectors: the
        # lengthscale gradients are differences of O(1e7) terms
        prec = PREC_F64 if Sol.dtype == torch.float64 else 1
        Uw = U if prec == PREC_F64 else U.float().contiguous()
        Xw = Xr if prec == PREC_F64 else Xr.float().contiguous()
        grads = cola_bilinear_grad(fctx.cctx, fctx.op, Uw.contiguous(), Xw, w, prec,
                                   leaf_dtypes=[d for _, d in fctx.leaf_meta])
        gs = float(g)
        lg = [gs * gr.reshape(s) for gr, (s, _) in zip(grads, fctx.leaf_meta)]
        return (None, None, None, None, None, None, gs * Sol[0], *lg)


def gp_objective(cctx, op, y, leaves, Z, opts=None, slq_steps=30, seed=0):
    """L = 1/2 y^T A^-1 y + 1/2 log det A with the adjoint backward above.
    ``Z`` holds the Rademacher probes (nprobes x N) shared by the trace
    estimate of the gradient and the SLQ log-det (``seed`` is not used to draw
    probes: both estimates always take Z)."""
    opts = opts or cola_cg_opts_default()
    return _GPObjective.apply(cctx, op, opts, Z, slq_steps, seed, y, *leaves)
