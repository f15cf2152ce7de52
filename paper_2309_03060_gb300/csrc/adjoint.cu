// Adjoint rules of App. B.2 on the CG solver:
//  * solve VJP: for X = A^-1 B, gradB = A^-T gradX (a second CG solve with the
//    same kernels; transpose rules of App. A.1.5 give A^T = A for the SPD
//    operators CG accepts) and, per leaf theta,
//    dL/dtheta = -(A^-T gradX)^T (dA/dtheta) X, with no Krylov iterate stored;
//  * log-det gradient Tr(A^-1 dA/dtheta) through Hutchinson probes
//    (App. B.1), (1/m) sum_k (A^-1 z_k)^T (dA/dtheta) z_k, reusing A^-1 Z when
//    the forward pass solved the probes in the same block;
//  * many independent systems (one CG per system, driven in turn).
#include <string.h>

#include <vector>

#include "internal.h"

namespace cola {

// FP32 copies of FP64 vectors for the gradient contractions when the solve
// ran in F32/MIXED (the contractions then run in FP32).
static const void* as_working(Ctx* c, const void* v, int64_t n, bool io64, bool f64work,
                              const char* name) {
  if (io64 == f64work) return v;
  if (io64 && !f64work) {
    float* t = (float*)c->ws.get(name, 4 * n);
    convert<double, float>(c, (const double*)v, t, n);
    return t;
  }
  double* t = (double*)c->ws.get(name, 8 * n);
  convert<float, double>(c, (const float*)v, t, n);
  return t;
}

cola_status batched_cg_fast(Ctx* c, int32_t nsys, const cola_linop* const* ops,
                            const void* const* Bin, void* const* Xout, const int64_t* nrhs,
                            const cola_cg_opts& o, cola_cg_info* info, bool* handled);

cola_status batched_cg_impl(Ctx* c, int32_t nsys, const cola_linop* const* ops,
                            const void* const* B, void* const* X, const int64_t* nrhs,
                            const cola_cg_opts& o, cola_cg_info* info) {
  // every system of the form c_k K1 (x) K2 + c_d Diag under MIXED + refinement:
  // all systems advance together through table-driven batched kernels
  bool handled = false;
  const cola_status st = batched_cg_fast(c, nsys, ops, B, X, nrhs, o, info, &handled);
  if (handled) return st;
  // any other composition: one graph-captured CG per system, in turn
  cola_status worst = COLA_OK;
  int64_t off = 0;
  for (int s = 0; s < nsys; ++s) {
    cola_status st = cg_solve_impl(c, ops[s], B[s], X[s], nrhs[s], o, info ? info + off : nullptr);
    if (st != COLA_OK && worst == COLA_OK) worst = st;
    off += nrhs[s];
  }
  return worst;
}

}  // namespace cola

using namespace cola;

extern "C" {

cola_status cola_solve_backward(cola_ctx* ctx, const cola_linop* op, const void* X,
                                const void* gradX, void* gradB, int64_t nrhs,
                                void* const* grads, const cola_cg_opts* opts,
                                cola_cg_info* info, cola_stream stream) {
  cola_status result = COLA_OK;
  cola_status st = guard([&] {
    COLA_REQUIRE(ctx && op && X && gradX && gradB && opts, COLA_ERR_INVALID_ARG,
                 "NULL argument");
    check_cg_args(op, opts, nrhs);
    StreamJoin j(ctx, stream);
    cola_cg_opts o = *opts;
    o.x0_given = 0;
    result = cg_solve_impl(ctx, op, gradX, gradB, nrhs, o, info);
    if (grads) {
      // Leaf gradients are sums of large terms that cancel (a GP lengthscale
      // gradient is a difference of O(1e7) terms): contract in FP64 whenever
      // the solve returned FP64 vectors.
      const bool io64 = (o.precision == COLA_PREC_F64) || o.refine;
      const bool f64 = io64;
      const int64_t n = op->rows * nrhs;
      const void* U = as_working(ctx, gradB, n, io64, f64, "bw.U");
      const void* Xw = as_working(ctx, X, n, io64, f64, "bw.X");
      std::vector<double> w(nrhs, -1.0);
      int nl = 0;
      cola_linop_num_leaves(op, &nl);
      bilinear_entry(ctx, op, U, Xw, w.data(), nrhs, f64 ? COLA_PREC_F64 : COLA_PREC_F32, grads,
                     0, 0);
    }
  });
  return st != COLA_OK ? st : result;
}

cola_status cola_logdet_backward(cola_ctx* ctx, const cola_linop* op, const void* Z,
                                 const void* AinvZ, int64_t nprobes, double scale,
                                 void* const* grads, int32_t accumulate,
                                 const cola_cg_opts* opts, cola_stream stream) {
  cola_status result = COLA_OK;
  cola_status st = guard([&] {
    COLA_REQUIRE(ctx && op && Z && grads && opts, COLA_ERR_INVALID_ARG, "NULL argument");
    check_cg_args(op, opts, nprobes);
    StreamJoin j(ctx, stream);
    const bool io64 = (opts->precision == COLA_PREC_F64) || opts->refine;
    const bool f64 = io64;  // FP64 contractions for FP64 vectors (see solve backward)
    const size_t es = io64 ? 8 : 4;
    const int64_t n = op->rows * nprobes;
    const void* U = AinvZ;
    if (!U) {
      void* t = ctx->ws.get("ldb.U", es * n);
      cola_cg_opts o = *opts;
      o.x0_given = 0;
      result = cg_solve_impl(ctx, op, Z, t, nprobes, o, nullptr);
      U = t;
    }
    const void* Uw = as_working(ctx, U, n, io64, f64, "ldb.Uw");
    const void* Zw = as_working(ctx, Z, n, io64, f64, "ldb.Zw");
    std::vector<double> w(nprobes, scale / (double)nprobes);
    bilinear_entry(ctx, op, Uw, Zw, w.data(), nprobes, f64 ? COLA_PREC_F64 : COLA_PREC_F32, grads,
                   accumulate, 0);
  });
  return st != COLA_OK ? st : result;
}

}  // extern "C"
