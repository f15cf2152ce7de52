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

#include <algorithm>
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

template <typename T>
__global__ void k_scaled_copy(int64_t n, const T* src, double g, T* dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = (T)(g * (double)src[i]);
}

}  // namespace cola

using namespace cola;

extern "C" {

cola_status cola_gp_objective(cola_ctx* ctx, const cola_linop* op, const void* y, const void* Z,
                              int64_t nprobes, int32_t slq_steps, const cola_cg_opts* opts,
                              void* Sol, double* value, double* logdet, double* logdet_se,
                              cola_cg_info* info, cola_stream stream) {
  cola_status result = COLA_OK;
  cola_status st = guard([&] {
    COLA_REQUIRE(ctx && op && y && Z && opts && Sol && value, COLA_ERR_INVALID_ARG,
                 "NULL argument");
    COLA_REQUIRE(nprobes >= 1 && slq_steps >= 1, COLA_ERR_INVALID_ARG, "nprobes / slq_steps");
    check_cg_args(op, opts, 1 + nprobes);
    StreamJoin j(ctx, stream);
    const int64_t N = op->rows, R = 1 + nprobes;
    const bool io64 = (opts->precision == COLA_PREC_F64) || opts->refine;
    const size_t es = io64 ? 8 : 4;
    // the block [y, z_1 .. z_m]: one solve for the data term and the probes
    char* block = (char*)ctx->ws.get("gp.block", es * N * R);
    COLA_CUDA(cudaMemcpyAsync(block, y, es * N, cudaMemcpyDeviceToDevice, ctx->s));
    COLA_CUDA(cudaMemcpyAsync(block + es * N, Z, es * N * nprobes, cudaMemcpyDeviceToDevice,
                              ctx->s));
    cola_cg_opts o = *opts;
    o.x0_given = 0;
    result = cg_solve_impl(ctx, op, block, Sol, R, o, info);
    // y^T A^-1 y (deterministic FP64 reduction of the working-precision products)
    double* part = (double*)ctx->ws.get("gp.part", 8 * (size_t)dot_blocks(N));
    double* quad_d = (double*)ctx->ws.get("gp.quad", 8);
    if (io64)
      dots<double>(ctx, (const double*)y, (const double*)Sol, N, 1, part, quad_d);
    else
      dots<float>(ctx, (const float*)y, (const float*)Sol, N, 1, part, quad_d);
    double quad = 0.0;
    COLA_CUDA(cudaMemcpyAsync(&quad, quad_d, 8, cudaMemcpyDeviceToHost, ctx->s));
    COLA_CUDA(cudaStreamSynchronize(ctx->s));
    // log det A by SLQ on the same probes (FP32 probes for F32 / MIXED)
    const bool f64 = opts->precision == COLA_PREC_F64;
    const void* probes = as_working(ctx, Z, N * nprobes, io64, f64, "gp.Z");
    double ld = 0.0, se = 0.0;
    int clamped = 0;
    slq_impl(ctx, op, (int)nprobes, slq_steps, 0, probes, opts->precision, 0, &ld, &se, nullptr,
             &clamped);
    *value = 0.5 * quad + 0.5 * ld;
    if (logdet) *logdet = ld;
    if (logdet_se) *logdet_se = se;
  });
  return st != COLA_OK ? st : result;
}

cola_status cola_gp_objective_backward(cola_ctx* ctx, const cola_linop* op, const void* Sol,
                                       const void* Z, int64_t nprobes, double g,
                                       int32_t precision, void* const* grads, void* grad_y,
                                       cola_stream stream) {
  return guard([&] {
    COLA_REQUIRE(ctx && op && Sol && Z, COLA_ERR_INVALID_ARG, "NULL argument");
    COLA_REQUIRE(nprobes >= 1, COLA_ERR_INVALID_ARG, "nprobes = %lld", (long long)nprobes);
    COLA_REQUIRE(precision == COLA_PREC_F64 || precision == COLA_PREC_F32,
                 COLA_ERR_INVALID_ARG, "precision must be F64 or F32");
    StreamJoin j(ctx, stream);
    const int64_t N = op->rows, R = 1 + nprobes;
    const bool f64 = precision == COLA_PREC_F64;
    const size_t es = f64 ? 8 : 4;
    // X = [a, z_1 .. z_m] next to U = Sol = [a, u_1 .. u_m]
    char* X = (char*)ctx->ws.get("gpb.X", es * N * R);
    COLA_CUDA(cudaMemcpyAsync(X, Sol, es * N, cudaMemcpyDeviceToDevice, ctx->s));
    COLA_CUDA(cudaMemcpyAsync(X + es * N, Z, es * N * nprobes, cudaMemcpyDeviceToDevice,
                              ctx->s));
    if (grads) {
      std::vector<double> w(R, 0.5 * g / (double)nprobes);
      w[0] = -0.5 * g;
      bilinear_entry(ctx, op, Sol, X, w.data(), R, precision, grads, 0, 0);
    }
    if (grad_y) {
      const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 4096));
      if (f64)
        k_scaled_copy<double><<<grid, 256, 0, ctx->s>>>(N, (const double*)Sol, g,
                                                        (double*)grad_y);
      else
        k_scaled_copy<float><<<grid, 256, 0, ctx->s>>>(N, (const float*)Sol, g, (float*)grad_y);
      ctx->count_launch();
      COLA_CUDA(cudaGetLastError());
    }
  });
}

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
