"""Benchmark: Kronecker-operator CG solves/s (and iterations/s) to a 1e-8
relative residual, mixed precision vs plain FP32, on one GB300.

Workload (one step = the whole hot path over one batch of synthetic input):
  A = K1 (x) K2 (x) K3 + 0.01 I, three 128 x 128 RBF factors (lengthscale 0.1,
  points uniform in [0,1]), N = 2,097,152; 16 right-hand sides ~ N(0, 1);
  CG with split-BF16 tensor-core Kronecker contractions, FP32 recurrences and
  FP64 reliable-update refinement to ||b - A x|| / ||b|| <= 1e-8 for every RHS;
  then stochastic Lanczos quadrature of log det A with 32 Rademacher probes and
  100 Lanczos steps.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead (bounded sample per step).  Under torchrun every rank runs its
own replica of the workload (independent right-hand sides, no collective on the
data path); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = "Kron-operator CG solves/s and iters/s to 1e-8 residual, mixed vs FP32 plain"
UNIT = "solves/s"
WORKLOAD = "kron3_rbf128_mixed: K1(x)K2(x)K3 + 0.01 I, n=128^3 (N=2,097,152), 16 RHS, tol 1e-8; SLQ 32x100"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(gpus: int):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if gpus > 0 else "gloo")
        pg = dist
    return rank, world, local, pg


def max_over_ranks(pg, value: float, device) -> float:
    if pg is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def barrier(pg):
    if pg is not None:
        pg.barrier()


def rank_rhs(w, rank: int):
    """Right-hand sides of one rank: the workload's own block on rank 0, an
    independent seeded block of the same shape on every other rank (replicas
    of the workload, no data shared between ranks)."""
    return w.B if rank == 0 else wl.normal(wl.substream(w.seed, 100 + rank), w.B.shape)


def rank_probe_seed(w, rank: int) -> int:
    """Seed of the SLQ probes of one rank (rank 0 keeps the workload's own)."""
    return wl.substream(w.seed, 2) if rank == 0 else wl.substream(w.seed, 200 + rank)


# ----------------------------------------------------------------- our arm
def build_operator(cola, ctx, w, device):
    import torch
    K = [torch.tensor(f, device=device) for f in w.factors]
    s = torch.tensor([w.shift], dtype=torch.float64, device=device)
    kron = cola.cola_linop_kron(ctx, *[cola.cola_linop_dense(ctx, k) for k in K])
    op = cola.cola_linop_sum(ctx, [kron, cola.cola_linop_diag(ctx, s, n=w.N)]).set_spd()
    return op, kron


def run_batched_workload(cola, ctx, device, hbm_peak, stream):
    """The batched uneven-systems workload (512 systems K1 (x) K2 + s I, factor
    sides 16..256, 1..8 right-hand sides each) in one cola_cg_solve_batched
    call, MIXED + FP64 refinement to 1e-8: one untimed call (tile tuning,
    graph capture, factor splits), one timed with CUDA events.  The roofline
    counts 32 N bytes per CG iteration of every right-hand side."""
    import statistics as st_
    import torch
    w4 = wl.config4()
    ops, Bs = [], []
    for s in w4.systems:
        K = [torch.tensor(f, device=device) for f in s.factors]
        sh = torch.tensor([s.shift], dtype=torch.float64, device=device)
        kron = cola.cola_linop_kron(ctx, *[cola.cola_linop_dense(ctx, k) for k in K])
        ops.append(cola.cola_linop_sum(ctx, [kron, cola.cola_linop_diag(ctx, sh, n=s.N)]).set_spd())
        Bs.append(torch.tensor(s.B, device=device))
    opts = cola.cola_cg_opts_default(precision=cola.PREC_MIXED, refine=1, tol=w4.tol,
                                     maxiter=60000, split_factor_terms=3, split_vector_terms=3,
                                     graph_chunk=64)
    cola.cola_cg_solve_batched(ctx, ops, Bs, opts)
    torch.cuda.synchronize()
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    Xs, info, status = cola.cola_cg_solve_batched(ctx, ops, Bs, opts)
    b1.record(stream)
    torch.cuda.synchronize()
    t = b0.elapsed_time(b1) / 1e3
    its = [i["iterations"] for i in info]
    sizes = [s.N for s, b in zip(w4.systems, Bs) for _ in range(b.shape[0])]
    alg = sum(32.0 * n * k for n, k in zip(sizes, its))
    return {"workload": "batched_kron2_uneven: 512 systems K1(x)K2 + s I, n1, n2 in 16..256, "
                        "1..8 RHS each, tol 1e-8", "systems": len(ops), "rhs": len(its),
            "seconds": round(t, 3), "solves_per_s": round(len(its) / t, 2), "status": status,
            "iterations": {"min": min(its), "mean": round(st_.mean(its), 1), "max": max(its)},
            "worst_rel_residual": max(i["rel_residual"] for i in info),
            "alg_bytes": alg, "achieved_gbs": round(alg / t / 1e9, 1),
            "roofline_frac": round(alg / t / 1e9 / hbm_peak, 4)}


def run_kron_precond(cola, ctx, device, args, stream):
    """The heteroscedastic variant of the workload, K1 (x) K2 (x) K3 + Diag(d)
    with d in [0.005, 0.015] (no scalar shift: the eigen-structured solve does
    not apply), solved by MIXED CG + FP64 refinement to 1e-8 preconditioned with
    M = Kron + mean(d) I, M^-1 applied by the eigen-structured solve.  One
    untimed solve (factor eigendecompositions, graph capture), one timed."""
    import torch
    w = wl.config2_hetero(nrhs=args.nrhs)
    K = [torch.tensor(f, device=device) for f in w.factors]
    d = torch.tensor(w.extra["d"], device=device)
    kron = cola.cola_linop_kron(ctx, *[cola.cola_linop_dense(ctx, k) for k in K])
    op = cola.cola_linop_sum(ctx, [kron, cola.cola_linop_diag(ctx, d)]).set_spd()
    B = torch.tensor(w.B, device=device)
    opts = cola.cola_cg_opts_default(precision=cola.PREC_MIXED, refine=1, tol=w.tol,
                                     maxiter=2000, split_factor_terms=args.fterms,
                                     split_vector_terms=args.vterms, graph_chunk=8,
                                     reliable_delta=args.delta, kron_precond=1)
    cola.cola_cg_solve(ctx, op, B, opts)
    torch.cuda.synchronize()
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    X, info, st = cola.cola_cg_solve(ctx, op, B, opts)
    k1.record(stream)
    torch.cuda.synchronize()
    t = k0.elapsed_time(k1) / 1e3
    return {"workload": f"{w.name}: K1(x)K2(x)K3 + Diag(d), d in [0.005, 0.015], "
                        f"{args.nrhs} RHS, tol {w.tol}",
            "preconditioner": "M = Kron + mean(d) I, applied by the eigen-structured solve",
            "seconds": round(t, 4), "solves_per_s": round(args.nrhs / t, 2), "status": st,
            "iterations": max(i["iterations"] for i in info),
            "fp64_replacements": max(i["updates"] for i in info),
            "worst_rel_residual": max(i["rel_residual"] for i in info)}


def run_bipoisson(cola, ctx, device, args, stream):
    """Product splitting on the Bi-Poisson operator (L (+) L)^2, 1000 x 1000
    grid (N = 1e6), tol 1e-11, FP64 (Sec. 3.2 / Fig. 2(b)): the split solve
    (one CG per Kronecker-sum factor), one CG on the product itself with the
    same iteration budget, and the split solve with the eigen-structured rule
    for each factor.  Each timed call follows an untimed one (graph capture,
    factor eigendecomposition)."""
    import torch
    w = wl.bipoisson(1000, nrhs=1)
    Ld = torch.tensor(w.L, device=device)
    Lop = cola.cola_linop_dense(ctx, Ld)
    ks = cola.cola_linop_kronsum(ctx, Lop, Lop).set_spd()
    op = cola.cola_linop_product(ctx, [ks, ks]).set_spd()
    B = torch.tensor(w.B, device=device)
    opts = cola.cola_cg_opts_default(precision=cola.PREC_F64, refine=0, tol=w.tol,
                                     maxiter=w.maxiter, graph_chunk=64)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) / 1e3

    (_, info_s, st_s), t_s = timed(lambda: cola.cola_product_solve(ctx, op, B, opts,
                                                                   use_structure=False))
    budget = info_s[0]["iterations"]
    mono = cola.cola_cg_opts_default(precision=cola.PREC_F64, refine=0, tol=w.tol,
                                     maxiter=budget, graph_chunk=64)
    (_, info_m, st_m), t_m = timed(lambda: cola.cola_cg_solve(ctx, op, B, mono,
                                                              raise_on_error=False))
    (_, info_e, st_e), t_e = timed(lambda: cola.cola_product_solve(ctx, op, B, opts,
                                                                   use_structure=True))
    return {"workload": f"{w.name}: (L(+)L)^2, N = {w.N}, tol {w.tol}, FP64",
            "split_cg": {"seconds": round(t_s, 4), "status": st_s,
                         "iterations": budget, "rel_residual": info_s[0]["rel_residual"]},
            "monolithic_cg_same_budget": {"seconds": round(t_m, 4), "status": st_m,
                                          "iterations": info_m[0]["iterations"],
                                          "rel_residual": info_m[0]["rel_residual"]},
            "split_eigen": {"seconds": round(t_e, 4), "status": st_e,
                            "rel_residual": info_e[0]["rel_residual"]}}


def run_diag_estimate(cola, ctx, device, args, stream):
    """Doubly stochastic vs Hutchinson diagonal estimation (Sec. 3.3 / App. B.1)
    on the multi-task covariance sum_q c_q B_q (x) K_q (8 terms, 128 tasks x
    1024 points, N = 131072), 16 Rademacher probes per term, MIXED with 3 split
    terms: time per estimate, error against the exact diagonal (Diag rule:
    Diag(B (x) K) = diag(B) (x) diag(K)), and the error the Rademacher variance
    formula predicts (Frobenius norms from the Kronecker structure)."""
    import numpy as np
    import torch
    w = wl.multitask()
    n = 16
    kids, keep = [], []
    for b, k in zip(w.B, w.K):
        tb, tk = torch.tensor(b, device=device), torch.tensor(k, device=device)
        keep += [tb, tk]
        kids.append(cola.cola_linop_kron(ctx, cola.cola_linop_dense(ctx, tb),
                                         cola.cola_linop_dense(ctx, tk)))
    op = cola.cola_linop_sum(ctx, kids, [float(c) for c in w.coeffs])
    exact = sum(c * np.kron(np.diag(b), np.diag(k)) for b, k, c in zip(w.B, w.K, w.coeffs))
    fro2 = sum(cq * cr * np.sum(bq * br) * np.sum(kq * kr)
               for bq, kq, cq in zip(w.B, w.K, w.coeffs)
               for br, kr, cr in zip(w.B, w.K, w.coeffs))
    off_base = fro2 - float(np.sum(exact ** 2))
    off_dbl = sum(c * c * (np.sum(b * b) * np.sum(k * k)
                           - float(np.sum(np.kron(np.diag(b), np.diag(k)) ** 2)))
                  for b, k, c in zip(w.B, w.K, w.coeffs))
    out = {"workload": f"{w.name}: sum of {len(w.B)} Kron(task 128, RBF 1024) terms, "
                       f"N = {w.N}, {n} probes per term, MIXED (3 split terms)"}
    for doubly, off in ((False, off_base), (True, off_dbl)):
        def call():
            return cola.cola_diag_estimate(ctx, op, n, seed=17, doubly=doubly,
                                           precision=cola.PREC_MIXED, split_terms=3)
        call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d, tr = call()
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        err = float(np.linalg.norm(d.cpu().numpy() - exact) / np.linalg.norm(exact))
        pred = float(np.sqrt(off / n) / np.linalg.norm(exact))
        out["doubly" if doubly else "base"] = {
            "seconds": round(t, 4), "estimates_per_s": round(1.0 / t, 2),
            "diag_rel_error": round(err, 5), "predicted_rel_error": round(pred, 5),
            "trace_rel_error": abs(tr - float(exact.sum())) / float(exact.sum())}
    return out


def run_householder(cola, ctx, device, args, stream):
    """SLQ log-det of the bench operator (K1 (x) K2 (x) K3 + 0.01 I, 128^3) with 8
    Rademacher probes x 100 steps in MIXED precision, plain Lanczos against the
    Householder basis (Algorithm 2): time, and error against the exact log-det
    from the factor eigenvalues."""
    import torch
    w = wl.config2(nrhs=1)
    op, _ = build_operator(cola, ctx, w, device)
    exact_ld = cola.cola_kron_eig_logdet(ctx, op)
    out = {"workload": "SLQ on kron3_rbf128 (N = 2^21), 8 probes x 100 steps, MIXED",
           "logdet_exact": exact_ld}
    for name, reorth in (("plain", 0), ("householder", 2)):
        def call():
            return cola.cola_slq_logdet(ctx, op, 8, 100, seed=3, precision=cola.PREC_MIXED,
                                        reorth=reorth)
        call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ld, se, _, clamped = call()
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        out[name] = {"seconds": round(t, 4), "logdet": ld,
                     "rel_error": abs(ld - exact_ld) / abs(exact_ld), "stderr": se,
                     "clamped": clamped}
    # reflector reads per step j: Y^T u_j (j reflectors), q_j = e_j + Y c, Y^T A q_j and
    # nu_{j+1} = A q_j + Y t (j + 1 each); 8 probes x N FP32 entries per reflector
    refl = float(sum(j + 3 * (j + 1) for j in range(100))) * 8 * w.N * 4
    out["householder"]["reflector_bytes"] = refl
    out["householder"]["reflector_tbs"] = round(refl / out["householder"]["seconds"] / 1e12, 2)
    return out


def run_config1(cola, ctx, device, stream):
    """The FP64 single-solve workload: K1 (x) K2 + 0.1 I, two 64-point RBF factors
    (l = 0.2), N = 4096, one RHS, CG to 1e-10, then SLQ with 16 Rademacher probes
    x 50 Lanczos steps.  The whole working set fits on chip, so the bound is
    latency: reported as microseconds per CG iteration and per Lanczos step.
    One untimed call of each (graph capture), one timed."""
    import torch
    w = wl.config1()
    K = [torch.tensor(f, device=device) for f in w.factors]
    s = torch.tensor([w.shift], dtype=torch.float64, device=device)
    kron = cola.cola_linop_kron(ctx, *[cola.cola_linop_dense(ctx, k) for k in K])
    op = cola.cola_linop_sum(ctx, [kron, cola.cola_linop_diag(ctx, s, n=w.N)]).set_spd()
    B = torch.tensor(w.B, device=device)
    opts = cola.cola_cg_opts_default(precision=cola.PREC_F64, refine=0, tol=w.tol, maxiter=5000)
    seed = wl.substream(w.seed, 2)

    def solve():
        return cola.cola_cg_solve(ctx, op, B, opts)

    def slq():
        return cola.cola_slq_logdet(ctx, op, w.slq_probes, w.slq_steps, seed=seed,
                                    precision=cola.PREC_F64)
    (_, info, st), t_cg = timed_call(torch, stream, solve)
    (ld, se, _, clamped), t_slq = timed_call(torch, stream, slq)
    exact_ld = cola.cola_kron_eig_logdet(ctx, op)
    it = info[0]["iterations"]
    steady = steady_iteration_time(
        cola, ctx, torch, stream, op, B,
        lambda n: cola.cola_cg_opts_default(precision=cola.PREC_F64, refine=0, tol=0.0,
                                            maxiter=n, max_updates=0), 64, 192)
    return {"workload": f"{w.name}: K1(x)K2 + 0.1 I, 64-point RBF factors (l 0.2), N = {w.N}, "
                        "1 RHS, CG to 1e-10; SLQ 16 x 50, FP64",
            "bound": "latency (the FP64 working set, ~192 KB, fits on chip)",
            "cg": {"seconds": round(t_cg, 5), "iterations": it, "status": st,
                   "us_per_iteration": round(1e6 * t_cg / max(it, 1), 2),
                   "us_per_iteration_steady": round(1e6 * steady, 2),
                   "rel_residual": info[0]["rel_residual"]},
            "slq": {"seconds": round(t_slq, 5), "logdets_per_s": round(1.0 / t_slq, 2),
                    "us_per_lanczos_step": round(1e6 * t_slq / w.slq_steps, 2),
                    "logdet": ld, "stderr": se, "logdet_exact": exact_ld,
                    "z_score": (ld - exact_ld) / se if se > 0 else None,
                    "rel_error": abs(ld - exact_ld) / abs(exact_ld), "clamped": clamped}}


def run_config3(cola, ctx, device, stream, hbm_peak):
    """The PDE-style composed operator: (L (+) L) + D + U U^T with the 1024-point
    Dirichlet Laplacian (N = 2^20), D ~ U[0.5, 1.5], U 32 columns ~ N(0, 1/N); 8
    RHS, Jacobi-preconditioned FP32 CG to 1e-6.  Algorithmic bytes per CG
    iteration: U read twice (2 N 32 x 4 B) + d and M^-1 (2 N x 4 B) + the
    vectors (32 N B per RHS) = 545 MB."""
    import torch
    w = wl.config3()
    Ld = torch.tensor(w.L, device=device)
    Lop = cola.cola_linop_dense(ctx, Ld)
    d = torch.tensor(w.d, device=device)
    U = torch.tensor(w.U, device=device)
    op = cola.cola_linop_sum(ctx, [cola.cola_linop_kronsum(ctx, Lop, Lop),
                                   cola.cola_linop_diag(ctx, d),
                                   cola.cola_linop_lowrank(ctx, U, None)]).set_spd()
    B = torch.tensor(w.B, dtype=torch.float32, device=device)
    opts = cola.cola_cg_opts_default(precision=cola.PREC_F32, refine=0, tol=w.tol, jacobi=1,
                                     maxiter=1000, graph_chunk=8)
    (_, info, st), t = timed_call(torch, stream, lambda: cola.cola_cg_solve(ctx, op, B, opts))
    it = max(i["iterations"] for i in info)
    R, N = w.B.shape[0], w.N
    alg = 2.0 * N * 32 * 4 + 2.0 * N * 4 + 32.0 * N * R
    per_it = steady_iteration_time(
        cola, ctx, torch, stream, op, B,
        lambda n: cola.cola_cg_opts_default(precision=cola.PREC_F32, refine=0, tol=0.0,
                                            jacobi=1, maxiter=n, graph_chunk=8,
                                            max_updates=0), 32, 96)
    return {"workload": f"{w.name}: L(+)L + D + U U^T, n 1024 (N = {N}), U 32 columns, "
                        f"{R} RHS, Jacobi PCG FP32 to {w.tol}",
            "seconds": round(t, 5), "iterations": it, "status": st,
            "solves_per_s": round(R / t, 2), "us_per_iteration_solve": round(1e6 * t / it, 2),
            "us_per_iteration": round(1e6 * per_it, 2),
            "per_iteration": "steady state: difference of 96- and 32-iteration solves",
            "worst_rel_residual": max(i["rel_residual"] for i in info),
            "roofline": {"bound": "hbm", "alg_bytes_per_iteration": alg,
                         "roofline_us": round(1e6 * alg / (hbm_peak * 1e9), 1),
                         "achieved_gbs": round(alg / per_it / 1e9, 1),
                         "frac": round(alg / per_it / 1e9 / hbm_peak, 4)}}


def run_config5(cola, ctx, device, stream, hbm_peak, tflops):
    """The differentiation workload: A = K1(l1) (x) K2(l2) + s2 I, two 1024-point
    RBF factors (l1 0.1, l2 0.2, s2 0.1; N = 2^20); y and 32 Rademacher probes
    solved as one 33-RHS block to 1e-8 (MIXED + FP64 refinement), then the
    backward: one weighted bilinear-gradient call (App. B.2 rules 1 and 4 with
    the Hutchinson trace) giving dL/dK1, dL/dK2 and dL/ds2.  Roofline per CG
    iteration: max(32 N R bytes / HBM, 2 N (n1 + n2) R flop / BF16 peak)."""
    import torch
    w = wl.config5()
    K = [torch.tensor(wl.rbf_factor(p, l), device=device) for p, l in zip(w.points, w.ells)]
    s2 = torch.tensor([w.sigma2], dtype=torch.float64, device=device)
    kron = cola.cola_linop_kron(ctx, *[cola.cola_linop_dense(ctx, k) for k in K])
    op = cola.cola_linop_sum(ctx, [kron, cola.cola_linop_diag(ctx, s2, n=w.N)]).set_spd()
    block = torch.tensor(np.vstack([w.y[None, :], w.Z]), device=device)
    R = block.shape[0]
    opts = cola.cola_cg_opts_default(precision=cola.PREC_MIXED, refine=1, tol=w.tol,
                                     maxiter=60000, split_factor_terms=3, split_vector_terms=3)
    (Sol, info, st), t = timed_call(torch, stream, lambda: cola.cola_cg_solve(ctx, op, block, opts),
                                    warm=False)
    m = w.Z.shape[0]
    Xr = torch.cat([Sol[:1], block[1:]], dim=0).contiguous()
    wts = [-0.5] + [0.5 / m] * m
    grads, t_bw = timed_call(torch, stream, lambda: cola.cola_bilinear_grad(
        ctx, op, Sol, Xr, wts, cola.PREC_F64), warm=False)
    it = max(i["iterations"] for i in info)
    per_it = t / max(it, 1)
    N = w.N
    Xf = torch.randn(R, N, dtype=torch.float32, device=device)
    Yf = torch.empty_like(Xf)
    (_, t_mvm) = timed_call(torch, stream, lambda: cola.cola_matvec(
        ctx, op, Xf, cola.PREC_MIXED, out=Yf, split_terms=3))
    byts = 32.0 * N * R
    flop = 2.0 * N * (1024 + 1024) * R
    roof = max(byts / (hbm_peak * 1e9), flop / (tflops * 1e12))
    return {"workload": f"{w.name}: K1(l1)(x)K2(l2) + s2 I, n 1024^2 (N = {N}), [y, 32 probes] "
                        "= 33 RHS to 1e-8, MIXED 3x3 + FP64 refinement; backward = one "
                        "bilinear-gradient call",
            "forward": {"seconds": round(t, 4), "iterations": it, "status": st,
                        "fp64_replacements": max(i["updates"] for i in info),
                        "us_per_iteration": round(1e6 * per_it, 2),
                        "worst_rel_residual": max(i["rel_residual"] for i in info)},
            "backward_seconds": round(t_bw, 4),
            "mvm": {"us": round(1e6 * t_mvm, 1),
                    "tensor_tflops_split": round(6 * 2.0 * N * 2048 * R / t_mvm / 1e12, 1),
                    "note": "one MIXED MVM of the 33-RHS block (2 mode steps, 6 split MMAs "
                            "per product)"},
            "grad_s2": float(grads[2].double().sum()),
            "roofline": {"bound": "hbm (algorithmic); near the ridge",
                         "alg_bytes_per_iteration": byts, "alg_flop_per_iteration": flop,
                         "roofline_us": round(1e6 * roof, 1),
                         "frac": round(roof / per_it, 4)}}


def steady_iteration_time(cola, ctx, torch, stream, op, B, make_opts, lo, hi):
    """Seconds per CG iteration in steady state: the difference of two solves
    that run exactly `hi` and `lo` iterations (tol 0, so they stop at maxiter),
    which cancels the per-solve set-up (preparation, first restate, final true
    residual)."""
    def run(n):
        return cola.cola_cg_solve(ctx, op, B, make_opts(n), raise_on_error=False)
    (_, info_hi, _), t_hi = timed_call(torch, stream, lambda: run(hi))
    (_, info_lo, _), t_lo = timed_call(torch, stream, lambda: run(lo))
    d_it = max(i["iterations"] for i in info_hi) - max(i["iterations"] for i in info_lo)
    return (t_hi - t_lo) / max(d_it, 1)


def timed_call(torch, stream, fn, warm=True):
    """(result, seconds) of fn() timed with CUDA events on `stream`, after one
    untimed call (graph capture, workspace, factor preparation) when warm."""
    if warm:
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1) / 1e3


def optional_section(fn, enabled):
    """Runs one secondary workload; None when disabled, {"error": ...} when it raised."""
    if not enabled:
        return None
    try:
        return fn()
    except Exception as e:  # noqa: BLE001 - reported in the JSON line
        return {"error": f"{type(e).__name__}: {e}"[:300]}


def time_queued(torch, ctx, fn, reps):
    """Device time of `reps` calls of fn, on the library's launch stream (the
    calls are issued on that stream, so no cross-stream join sits between
    them), with every launch queued before the device reaches the first one (a
    device-side sleep holds the stream while the host enqueues), so host
    overhead between calls is not timed.  Returns seconds per call."""
    ls = ctx.stream()
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(ls):
        torch.cuda._sleep(50_000_000)      # ~25 ms at 2 GHz
        k0.record(ls)
        for _ in range(reps):
            fn()
        k1.record(ls)
    torch.cuda.synchronize()
    return k0.elapsed_time(k1) / 1e3 / reps


def run_mvm_only(args):
    """A few MIXED Kronecker MVMs of the bench operator (for profiler captures)."""
    import torch
    import paper_2309_03060_gb300 as cola
    device = torch.device("cuda", 0)
    ctx = cola.Context(0)
    w = wl.config2(nrhs=1)
    op, kron = build_operator(cola, ctx, w, device)
    X = torch.randn(args.nrhs, w.N, dtype=torch.float32, device=device)
    Y = torch.empty_like(X)
    target = op if args.with_shift else kron
    for _ in range(args.reps):
        cola.cola_matvec(ctx, target, X, cola.PREC_MIXED, out=Y,
                         split_terms=(args.fterms, args.vterms))
    t = time_queued(torch, ctx, lambda: cola.cola_matvec(
        ctx, target, X, cola.PREC_MIXED, out=Y, split_terms=(args.fterms, args.vterms)),
        args.reps)
    print(json.dumps({"mode": "mvm-only", "nrhs": args.nrhs, "reps": args.reps,
                      "ms_per_mvm": t * 1e3, "launches": ctx.kernel_launches()}))
    ctx.close()


def run_cg_short(args):
    """A CG solve of the bench operator capped at --maxiter iterations (the
    solve's kernels in their launch configuration, for profiler captures)."""
    import torch
    import paper_2309_03060_gb300 as cola
    device = torch.device("cuda", 0)
    ctx = cola.Context(0)
    w = wl.config2(nrhs=args.nrhs)
    op, _ = build_operator(cola, ctx, w, device)
    B = torch.tensor(w.B, device=device)
    opts = cola.cola_cg_opts_default(precision=cola.PREC_MIXED, refine=1, tol=w.tol,
                                     maxiter=args.maxiter, split_factor_terms=args.fterms,
                                     split_vector_terms=args.vterms, graph_chunk=args.chunk)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, info, st = cola.cola_cg_solve(ctx, op, B, opts)
    torch.cuda.synchronize()
    print(json.dumps({"mode": "cg-short", "nrhs": args.nrhs, "status": st,
                      "iterations": max(i["iterations"] for i in info),
                      "seconds": time.perf_counter() - t0, "launches": ctx.kernel_launches()}))
    ctx.close()


def bench_config(args, world):
    """The `config` object of the JSON line, shared by both arms."""
    return {"workload": WORKLOAD, "nrhs_per_gpu": args.nrhs, "N": 128 ** 3,
            "split_terms": {"factor": args.fterms, "vector": args.vterms},
            "slq": {"probes": 32, "steps": 100,
                    "split_terms": {"factor": args.fterms, "vector": args.vterms}},
            "tol": 1e-8,
            "l2": "inputs larger than L2 (16 x 2M FP32 vectors, 134 MB each)",
            "parallelism": f"replicas x{world}"}


def run_ours(args):
    import torch
    import paper_2309_03060_gb300 as cola

    rank, world, local, pg = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    ctx = cola.Context(local)
    w = wl.config2(nrhs=args.nrhs)
    op, kron = build_operator(cola, ctx, w, device)
    # each rank solves its own independent block of right-hand sides
    B_host = torch.tensor(rank_rhs(w, rank)).pin_memory()
    B = B_host.to(device)
    opts = cola.cola_cg_opts_default(precision=cola.PREC_MIXED, refine=1, tol=w.tol,
                                     maxiter=args.maxiter, split_factor_terms=args.fterms,
                                     split_vector_terms=args.vterms, graph_chunk=args.chunk,
                                     reliable_delta=args.delta)
    seed = rank_probe_seed(w, rank)
    stream = torch.cuda.current_stream()
    terms = (args.fterms, args.vterms)
    marks = []

    def step(record=False):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)] if record else None
        if record:
            ev[0].record(stream)
        X, info, st = cola.cola_cg_solve(ctx, op, B, opts)
        if st != 0:
            raise RuntimeError(f"solve status {st}: {info[:2]}")
        if record:
            ev[1].record(stream)
        ld, se, _, clamped = cola.cola_slq_logdet(ctx, op, w.slq_probes, w.slq_steps, seed=seed,
                                                  precision=cola.PREC_MIXED, split_terms=terms)
        if record:
            ev[2].record(stream)
            marks.append(ev)
        return X, info, ld, se, clamped

    for _ in range(args.warmup):
        X, info, ld, se, clamped = step()
    barrier(pg)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = ctx.kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    iters = []
    ev0.record(stream)
    for _ in range(args.steps):
        X, info, ld, se, clamped = step(record=True)
        iters.append(max(i["iterations"] for i in info))
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(pg)
    t_local = ev0.elapsed_time(ev1) / 1e3
    launches = ctx.kernel_launches() - l0
    clk = clocks.stop()
    t = max_over_ranks(pg, t_local, device)
    t_cg = sum(e[0].elapsed_time(e[1]) for e in marks) / 1e3
    t_slq = sum(e[1].elapsed_time(e[2]) for e in marks) / 1e3
    R = args.nrhs
    solves = R * args.steps * world
    value = solves / t
    it_per_solve = statistics.mean(iters)
    worst_res = max(i["rel_residual"] for i in info)
    fp64_updates = statistics.mean(i["updates"] for i in info)

    # end to end through the public API: pinned host B in, host X out, timed per step
    e2e_t = 0.0
    Xh = torch.empty_like(B_host).pin_memory()
    for k in range(args.e2e_steps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Bd = B_host.to(device, non_blocking=True)
        Xd, info_e, st = cola.cola_cg_solve(ctx, op, Bd, opts)
        ld_e, _, _, _ = cola.cola_slq_logdet(ctx, op, w.slq_probes, w.slq_steps, seed=seed,
                                             precision=cola.PREC_MIXED, split_terms=terms)
        Xh.copy_(Xd, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_t += e0.elapsed_time(e1) / 1e3
    e2e_t = max_over_ranks(pg, e2e_t, device)
    e2e = ({"value": R * args.e2e_steps * world / e2e_t, "unit": UNIT,
            "h2d_bytes_per_step": B_host.numel() * 8, "d2h_bytes_per_step": Xh.numel() * 8 + 16}
           if args.e2e_steps > 0 else None)

    # dominant work: one MIXED Kronecker MVM of the bench operator, timed alone
    # in the launch configuration the solve uses: the first mode step
    # (k_kron_tc_fs, slab-major output) and the slab kernel (k_kron_tc_slab,
    # steps 2 and 3 on chip), two launches.  Algorithmic bytes of an MVM:
    # 8 R N (X read once, Y written once, FP32; the intermediate excluded).
    hbm, tflops, peak_src = peaks()
    Xf = torch.randn(R, w.N, dtype=torch.float32, device=device)
    Yf = torch.empty_like(Xf)
    for _ in range(3):
        cola.cola_matvec(ctx, kron, Xf, cola.PREC_MIXED, out=Yf, split_terms=terms)
    l_mvm = ctx.kernel_launches()
    cola.cola_matvec(ctx, kron, Xf, cola.PREC_MIXED, out=Yf, split_terms=terms)
    launches_per_mvm = ctx.kernel_launches() - l_mvm
    reps = 20
    per_mvm = time_queued(torch, ctx, lambda: cola.cola_matvec(
        ctx, kron, Xf, cola.PREC_MIXED, out=Yf, split_terms=terms), reps)
    alg_mvm = 8.0 * R * w.N
    achieved = alg_mvm / per_mvm / 1e9
    roofline = {"kernel": "one MIXED Kronecker MVM: k_kron_tc_fs (mode 1, slab-major output) + "
                          "k_kron_tc_slab (modes 2 and 3 on chip)",
                "bound": "hbm",
                "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "peak_source": peak_src,
                "traffic": args.traffic_bytes, "mvm_us": round(per_mvm * 1e6, 2),
                "launches_per_mvm": launches_per_mvm,
                "alg_bytes_per_mvm": alg_mvm,
                "accounting": "8 R N bytes per MVM (X read, Y written; the slab-major "
                              "intermediate excluded) / event-timed MVM",
                "moved_gbs": round(2 * alg_mvm / per_mvm / 1e9, 1)}
    # CG iteration roofline: 32 N R algorithmic bytes per iteration of the block
    cg_iters = sum(iters)
    it_time = t_cg / max(cg_iters, 1)
    iter_alg = 32.0 * w.N * R
    iteration_roofline = {"alg_bytes_per_iter": iter_alg, "iter_us": round(1e6 * it_time, 2),
                          "roofline_us": round(1e6 * iter_alg / (hbm * 1e9), 1),
                          "achieved_gbs": round(iter_alg / it_time / 1e9, 1),
                          "frac": round(iter_alg / it_time / 1e9 / hbm, 4),
                          "includes": "FP64 residual replacements, alpha/beta kernels"}
    # SLQ roofline: 6 vector touches (4 B) per probe entry per Lanczos step
    slq_each = t_slq / args.steps
    slq_alg = 6.0 * 4 * w.N * w.slq_probes * w.slq_steps
    slq_out = {"seconds": round(slq_each, 4), "logdets_per_s": round(1.0 / slq_each, 3),
               "alg_bytes": slq_alg, "roofline_s": round(slq_alg / (hbm * 1e9), 4),
               "frac": round(slq_alg / slq_each / 1e9 / hbm, 4),
               "split_terms": {"factor": args.fterms, "vector": args.vterms},
               "logdet": ld, "stderr": se, "clamped": clamped}

    cpu = cpu_baseline(args) if (rank == 0 and not args.no_cpu) else None

    # the structured path: direct solve from the factor eigendecompositions
    # (Table 3 Inverse / Eigs rules) on the same right-hand sides, and the
    # exact log-det that the SLQ estimate is compared with
    def eig_section():
        Xe = cola.cola_kron_eig_solve(ctx, op, B, cola.PREC_F64)  # eigendecompositions here
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(3):
            cola.cola_kron_eig_solve(ctx, op, B, cola.PREC_F64, out=Xe)
        g1.record(stream)
        torch.cuda.synchronize()
        te = g0.elapsed_time(g1) / 1e3 / 3
        Ae = cola.cola_matvec(ctx, op, Xe, cola.PREC_F64)
        rel_e = float(((B - Ae).norm(dim=1) / B.norm(dim=1)).max())
        ld_exact = cola.cola_kron_eig_logdet(ctx, op)
        return {"solves_per_s": round(R / te, 2), "worst_rel_residual": rel_e,
                "path": "FP64 mode products with the factor eigenvectors + eigenvalue scaling",
                "logdet_exact": ld_exact,
                "slq_rel_error": abs(ld - ld_exact) / abs(ld_exact)}

    eig = optional_section(eig_section, rank == 0 and args.eig)

    # the secondary workloads run after the timed region; a failure in one is
    # reported in its field and does not cost the bench line
    cfg1 = optional_section(lambda: run_config1(cola, ctx, device, stream),
                            rank == 0 and args.configs)
    cfg3 = optional_section(lambda: run_config3(cola, ctx, device, stream, hbm),
                            rank == 0 and args.configs)
    cfg5 = optional_section(lambda: run_config5(cola, ctx, device, stream, hbm, tflops),
                            rank == 0 and args.configs)
    batched = optional_section(lambda: run_batched_workload(cola, ctx, device, hbm, stream),
                               rank == 0 and args.batched)
    kprec = optional_section(lambda: run_kron_precond(cola, ctx, device, args, stream),
                             rank == 0 and args.kron_precond)
    bipo = optional_section(lambda: run_bipoisson(cola, ctx, device, args, stream),
                            rank == 0 and args.bipoisson)
    dest = optional_section(lambda: run_diag_estimate(cola, ctx, device, args, stream),
                            rank == 0 and args.diag_est)
    hh = optional_section(lambda: run_householder(cola, ctx, device, args, stream),
                          rank == 0 and args.householder)

    def plain_section():
        popts = cola.cola_cg_opts_default(precision=cola.PREC_F32, refine=1, tol=w.tol,
                                          maxiter=args.maxiter, graph_chunk=args.chunk,
                                          reliable_delta=args.delta)
        torch.cuda.synchronize()
        p0 = time.perf_counter()
        Xp, pinfo, pst = cola.cola_cg_solve(ctx, op, B, popts)
        torch.cuda.synchronize()
        pt = time.perf_counter() - p0
        pit = max(i["iterations"] for i in pinfo)
        # the plain path's own mode step: FP32 SIMT GEMM, 2 R N n flop per launch
        per_mvm32 = time_queued(torch, ctx, lambda: cola.cola_matvec(
            ctx, kron, Xf, cola.PREC_F32, out=Yf), 5)
        flop = 2.0 * R * w.N * 128
        fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12  # SMs x FP32 lanes x FMA x max clock
        return {"solves_per_s": R / pt, "iterations": pit, "status": pst,
                "worst_rel_residual": max(i["rel_residual"] for i in pinfo),
                "path": "FP32 SIMT mode products, same CG with FP64 replacements, 1 solve",
                "mixed_speedup_cg_only": round((R * args.steps / t_cg) / (R / pt), 3),
                "mode_step_us": round(1e6 * per_mvm32 / 3, 2),
                "mode_step_fp32_tflops": round(flop / (per_mvm32 / 3) / 1e12, 2),
                "fp32_peak_tflops": round(fp32_peak, 1),
                "mode_step_frac_of_fp32_peak": round(flop / (per_mvm32 / 3) / 1e12 / fp32_peak, 4),
                "mode_step_frac_of_hbm": round(alg_mvm / per_mvm32 / 1e9 / hbm, 4)}

    plain = optional_section(plain_section, rank == 0 and args.plain)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * t / args.steps, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3-split/f32/f64",
            "data": "synthetic (seeded SplitMix64; RBF factors on uniform points, N(0,1) RHS)",
            "config": bench_config(args, world),
            "iters_per_s": round(cg_iters * world / t, 2),
            "cg_only": {"seconds_per_solve_block": round(t_cg / args.steps, 4),
                        "solves_per_s": round(R * args.steps / t_cg, 4),
                        "iters_per_s": round(cg_iters / t_cg, 2)},
            "cg_iterations_per_solve": it_per_solve,
            "fp64_replacements_per_solve": fp64_updates,
            "logdets_per_s": round(args.steps * world / t, 4),
            "worst_rel_residual": worst_res,
            "slq": slq_out,
            "roofline": roofline,
            "iteration_roofline": iteration_roofline,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clk, "plain_fp32": plain, "kron_eig": eig, "config1_fp64": cfg1,
            "config3_pde": cfg3, "config5_gp": cfg5, "batched": batched,
            "kron_precond": kprec, "bipoisson": bipo, "diag_estimate": dest,
            "householder_slq": hh,
        }
        print(json.dumps(line))
    ctx.close()


# ------------------------------------------------------------- CPU oracle
def _oracle_cg_sample(w, iters: int, threads: int):
    """FP64 oracle CG iterations on all RHS; returns seconds per iteration."""
    os.environ["OPENBLAS_NUM_THREADS"] = str(threads)
    from oracle import krylov  # noqa: F401  (oracle imported only on this leg)
    from oracle.linop import Dense, Diag, Kron, Sum
    op = Sum([Kron([Dense(f) for f in w.factors]), Diag(w.shift, w.N)])
    t0 = time.perf_counter()
    for r in range(w.B.shape[0]):
        krylov.cg(op, w.B[r], tol=0.0, maxiter=iters)
    return (time.perf_counter() - t0) / iters


# Iterations per solve that both CPU legs extrapolate to: the exact-arithmetic
# CG iteration count to 1e-8 on this operator's spectrum (kappa ~ 3.2e6), the
# count an FP64 CG needs up to rounding.  The GPU's own count (reported as
# cg_iterations_per_solve) is higher: its FP32 recursion loses some of the
# Krylov space's orthogonality.
CPU_ITERS_PER_SOLVE = 12400


def cores_available() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_leg(args, threads: int):
    """Seconds per all-RHS oracle CG iteration, measured in a child process
    with `threads` BLAS threads (the oracle as it stands: numpy FP64)."""
    code = (
        "import sys,json,os; sys.path.insert(0, %r);"
        "import bench, workloads as wl;"
        "w = wl.config2(nrhs=%d);"
        "print(json.dumps(bench._oracle_cg_sample(w, %d, %d)))"
    ) % (ROOT, args.nrhs, args.cpu_iters, threads)
    env = dict(os.environ, OPENBLAS_NUM_THREADS=str(threads), OMP_NUM_THREADS=str(threads),
               MKL_NUM_THREADS=str(threads))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=900)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-300:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def _cpu_leg_record(args, threads: int, sec_per_iter: float):
    solve_time = sec_per_iter * CPU_ITERS_PER_SOLVE
    return {"value": args.nrhs / solve_time, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": (f"{args.cpu_iters} FP64 oracle CG iterations on each of the {args.nrhs} "
                       f"RHS of the 128^3 workload ({sec_per_iter:.3f} s per all-RHS iteration, "
                       f"{threads} BLAS threads), extrapolated to {CPU_ITERS_PER_SOLVE} "
                       f"iterations per solve (exact-arithmetic CG count to 1e-8)")}


def cpu_baseline(args):
    """The oracle on all host cores (the reported baseline) and on one core."""
    try:
        n = cores_available()
        out = _cpu_leg_record(args, n, _oracle_leg(args, n))
        out["single_thread"] = _cpu_leg_record(args, 1, _oracle_leg(args, 1))
        return out
    except (RuntimeError, subprocess.TimeoutExpired) as e:
        return {"error": str(e)[-300:]}


def run_reference(args):
    """The reference arm: the FP64 oracle as it stands, on the host cores, on a
    bounded sample of the same workload per step, in the same metric and
    config as our arm (solves/s extrapolated on the same iteration basis as
    cpu_baseline)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = wl.config2(nrhs=args.nrhs)
    n = cores_available()
    for _ in range(args.warmup):
        _oracle_cg_sample(w, 1, n)
    t = 0.0
    for _ in range(args.steps):
        t += _oracle_cg_sample(w, args.cpu_iters, n)
    sec_per_iter = t / args.steps
    rec = _cpu_leg_record(args, n, sec_per_iter)
    value = rec["value"]
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sec_per_iter * args.cpu_iters,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded SplitMix64; RBF factors on uniform points, N(0,1) RHS)",
        "config": bench_config(args, 1),
        "cpu_baseline": rec,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nrhs", type=int, default=16)
    ap.add_argument("--fterms", type=int, default=3)
    ap.add_argument("--vterms", type=int, default=3)
    ap.add_argument("--chunk", type=int, default=64)
    ap.add_argument("--delta", type=float, default=0.1)
    ap.add_argument("--maxiter", type=int, default=60000)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--cpu-iters", type=int, default=2)
    # DRAM bytes (reads + writes) of one MIXED MVM of this workload (both
    # launches), from the ncu capture of the current kernel build summarised in
    # profiles/mvm_kron_tc_fs_slab_kron3_rbf128_r16.md
    ap.add_argument("--traffic-bytes", type=float, default=431.2e6)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--batched-only", action="store_true",
                    help="run only the 512-system batched workload (for profiler captures)")
    ap.add_argument("--batched", action=argparse.BooleanOptionalAction, default=True,
                    help="also run the 512-system batched workload once")
    ap.add_argument("--kron-precond", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the preconditioned solve of the per-point-noise variant")
    ap.add_argument("--kron-precond-only", action="store_true",
                    help="run only the preconditioned per-point-noise solve")
    ap.add_argument("--bipoisson", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the product-splitting Bi-Poisson solves")
    ap.add_argument("--bipoisson-only", action="store_true",
                    help="run only the product-splitting Bi-Poisson solves")
    ap.add_argument("--diag-est", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the doubly stochastic diagonal estimator")
    ap.add_argument("--diag-est-only", action="store_true",
                    help="run only the doubly stochastic diagonal estimator")
    ap.add_argument("--householder", action=argparse.BooleanOptionalAction, default=True,
                    help="also time SLQ with the Householder Lanczos basis")
    ap.add_argument("--householder-only", action="store_true",
                    help="run only the Householder-basis SLQ comparison")
    ap.add_argument("--configs", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the N = 4096 FP64, PDE-style and GP-gradient workloads")
    ap.add_argument("--configs-only", action="store_true",
                    help="run only those three workload sections")
    ap.add_argument("--config", type=int, choices=[1, 3, 5], default=None,
                    help="run only one of those sections (profiler captures)")
    ap.add_argument("--mvm-gp", action="store_true",
                    help="only run --reps MIXED MVMs of the GP workload's 33-RHS block "
                         "(1024-point factors; profiler captures of the streaming kernel)")
    ap.add_argument("--slq-only", action="store_true",
                    help="run only --reps SLQ log-dets (32 probes x 100 steps, MIXED 3x3) "
                         "of the bench operator (profiler captures)")
    ap.add_argument("--eig", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the eigen-structured direct solve and exact log-det")
    ap.add_argument("--plain", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the plain FP32 path once (--no-plain skips it)")
    ap.add_argument("--mvm-only", action="store_true",
                    help="only run --reps MIXED MVMs of the bench operator (profiler captures)")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--cg-short", action="store_true",
                    help="one CG solve of the bench operator capped at --maxiter iterations "
                         "(for profiler captures)")
    ap.add_argument("--with-shift", action="store_true")
    args = ap.parse_args()
    if args.cg_short:
        run_cg_short(args)
        return
    if args.mvm_only:
        run_mvm_only(args)
    elif args.mvm_gp:
        import torch
        import paper_2309_03060_gb300 as cola
        ctx = cola.Context(0)
        dev, st = torch.device("cuda", 0), torch.cuda.current_stream()
        w = wl.config5()
        K = [torch.tensor(wl.rbf_factor(p_, l), device=dev) for p_, l in zip(w.points, w.ells)]
        s2 = torch.tensor([w.sigma2], dtype=torch.float64, device=dev)
        kron = cola.cola_linop_kron(ctx, *[cola.cola_linop_dense(ctx, k) for k in K])
        op = cola.cola_linop_sum(ctx, [kron, cola.cola_linop_diag(ctx, s2, n=w.N)])
        X = torch.randn(33, w.N, dtype=torch.float32, device=dev)
        Y = torch.empty_like(X)
        ts = []
        for _ in range(args.reps):
            _, t = timed_call(torch, st, lambda: cola.cola_matvec(
                ctx, op, X, cola.PREC_MIXED, out=Y, split_terms=3), warm=False)
            ts.append(round(t * 1e6, 1))
        print(json.dumps({"mode": "mvm-gp", "us": ts}))
    elif args.slq_only:
        import torch
        import paper_2309_03060_gb300 as cola
        ctx = cola.Context(0)
        w = wl.config2(nrhs=1)
        op, _ = build_operator(cola, ctx, w, torch.device("cuda", 0))
        st = torch.cuda.current_stream()
        out = []
        for _ in range(args.reps):
            (ld, se, _, cl), t = timed_call(torch, st, lambda: cola.cola_slq_logdet(
                ctx, op, w.slq_probes, w.slq_steps, seed=5, precision=cola.PREC_MIXED,
                split_terms=(3, 3)), warm=False)
            out.append(round(t, 4))
        print(json.dumps({"mode": "slq-only", "seconds": out, "logdet": ld, "clamped": cl}))
    elif args.config is not None:
        import torch
        import paper_2309_03060_gb300 as cola
        ctx = cola.Context(0)
        hbm, tflops, _ = peaks()
        dev, st = torch.device("cuda", 0), torch.cuda.current_stream()
        fn = {1: lambda: run_config1(cola, ctx, dev, st),
              3: lambda: run_config3(cola, ctx, dev, st, hbm),
              5: lambda: run_config5(cola, ctx, dev, st, hbm, tflops)}[args.config]
        print(json.dumps(fn()))
    elif args.configs_only:
        import torch
        import paper_2309_03060_gb300 as cola
        ctx = cola.Context(0)
        hbm, tflops, _ = peaks()
        dev, st = torch.device("cuda", 0), torch.cuda.current_stream()
        print(json.dumps({"config1_fp64": optional_section(
            lambda: run_config1(cola, ctx, dev, st), True),
            "config3_pde": optional_section(lambda: run_config3(cola, ctx, dev, st, hbm), True),
            "config5_gp": optional_section(
                lambda: run_config5(cola, ctx, dev, st, hbm, tflops), True)}))
    elif args.batched_only:
        import torch
        import paper_2309_03060_gb300 as cola
        ctx = cola.Context(0)
        hbm, _, _ = peaks()
        print(json.dumps(run_batched_workload(cola, ctx, torch.device("cuda", 0), hbm,
                                              torch.cuda.current_stream())))
    elif args.householder_only:
        import torch
        import paper_2309_03060_gb300 as cola
        ctx = cola.Context(0)
        print(json.dumps(run_householder(cola, ctx, torch.device("cuda", 0), args,
                                         torch.cuda.current_stream())))
    elif args.diag_est_only:
        import torch
        import paper_2309_03060_gb300 as cola
        ctx = cola.Context(0)
        print(json.dumps(run_diag_estimate(cola, ctx, torch.device("cuda", 0), args,
                                           torch.cuda.current_stream())))
    elif args.bipoisson_only:
        import torch
        import paper_2309_03060_gb300 as cola
        ctx = cola.Context(0)
        print(json.dumps(run_bipoisson(cola, ctx, torch.device("cuda", 0), args,
                                       torch.cuda.current_stream())))
    elif args.kron_precond_only:
        import torch
        import paper_2309_03060_gb300 as cola
        ctx = cola.Context(0)
        print(json.dumps(run_kron_precond(cola, ctx, torch.device("cuda", 0), args,
                                          torch.cuda.current_stream())))
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
