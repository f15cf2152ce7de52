// Product splitting: A = A_1 A_2 ... A_m is solved as a sequence of solves,
// X = A_m^-1 ( ... (A_1^-1 B)), each factor by the rule its type allows
// (Sec. 3.2: the inverse of a product is the product of the inverses in
// reverse order; Table 3 dispatch).  A diagonal factor is divided out, an
// eigen-structured factor (Kron / KronSum [+ scalar * I]) takes the direct
// eigen solve, any other factor CG.  For a power A^n the split needs n solves
// of condition number kappa instead of one of kappa^n, the speed-up Sec. 3.2
// illustrates with the Bi-Poisson problem.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace cola {

namespace {

// X[r, i] = B[r, i] / (coeff * d[i * stride])  (stride 0: a scalar).
template <typename T>
__global__ void k_diag_solve(int64_t n, const T* B, T* X, const double* d, int64_t stride,
                             double coeff) {
  const int64_t v = blockIdx.y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    X[v * n + i] = (T)((double)B[v * n + i] / (coeff * d[i * stride]));
}

void flatten(const cola_linop* op, std::vector<const cola_linop*>& out) {
  if (op->kind == LK_PRODUCT) {
    for (auto* k : op->kids) flatten(k, out);
  } else {
    out.push_back(op);
  }
}

// Solve with one factor; accumulates CG iterations / replacements per RHS.
template <typename T>
void factor_solve(Ctx* c, const cola_linop* f, const T* B, T* X, int64_t R,
                  const cola_cg_opts& o, bool structure, std::vector<cola_cg_info>& acc,
                  cola_status& worst, int index) {
  const int64_t N = f->rows;
  if (f->kind == LK_DIAG) {
    prepare_leaves(c, const_cast<cola_linop*>(f), COLA_PREC_F64, 0);
    const int gx = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 2 * c->num_sms));
    k_diag_solve<T><<<dim3(gx, (unsigned)R), 256, 0, c->s>>>(N, B, X, leaf_ptr<double>(f),
                                                              f->stride, 1.0);
    c->count_launch();
    COLA_CUDA(cudaGetLastError());
    return;
  }
  if (structure && eig_solve_if_structured(c, f, B, X, R, sizeof(T) == 8)) return;
  COLA_REQUIRE(f->spd, COLA_ERR_UNSUPPORTED,
               "product factor %d is neither diagonal, eigen-structured nor annotated spd",
               index);
  std::vector<cola_cg_info> info(R);
  cola_cg_opts fo = o;
  fo.x0_given = 0;
  check_cg_args(f, &fo, R);
  const cola_status st = cg_solve_impl(c, f, B, X, R, fo, info.data());
  for (int64_t r = 0; r < R; ++r) {
    acc[r].iterations += info[r].iterations;
    acc[r].updates += info[r].updates;
    if (info[r].status != 0 && acc[r].status == 0) acc[r].status = info[r].status;
  }
  if (st != COLA_OK && worst == COLA_OK) worst = st;
}

template <typename T>
cola_status product_solve(Ctx* c, const cola_linop* op, const void* Bin, void* Xout, int64_t R,
                          const cola_cg_opts& o, bool structure, cola_cg_info* info) {
  std::vector<const cola_linop*> fs;
  flatten(op, fs);
  const int64_t N = op->rows;
  for (size_t k = 0; k < fs.size(); ++k)
    COLA_REQUIRE(fs[k]->rows == N && fs[k]->cols == N, COLA_ERR_SHAPE,
                 "product factor %zu is %lld x %lld, not %lld x %lld", k, (long long)fs[k]->rows,
                 (long long)fs[k]->cols, (long long)N, (long long)N);
  std::vector<cola_cg_info> acc(R);
  for (auto& a : acc) memset(&a, 0, sizeof a);
  cola_status worst = COLA_OK;
  T* y[2] = {(T*)c->ws.get("psolve.y0", sizeof(T) * N * R),
             (T*)c->ws.get("psolve.y1", sizeof(T) * N * R)};
  const T* cur = (const T*)Bin;
  for (size_t k = 0; k < fs.size(); ++k) {
    T* dst = (k + 1 == fs.size()) ? (T*)Xout : y[k & 1];
    factor_solve<T>(c, fs[k], cur, dst, R, o, structure, acc, worst, (int)k);
    cur = dst;
  }
  // true residual of the whole product, in the vectors' precision
  T* res = (T*)c->ws.get("psolve.r", sizeof(T) * N * R);
  COLA_CUDA(cudaMemcpyAsync(res, Bin, sizeof(T) * N * R, cudaMemcpyDeviceToDevice, c->s));
  const int prec = sizeof(T) == 8 ? COLA_PREC_F64 : COLA_PREC_F32;
  prepare_leaves(c, const_cast<cola_linop*>(op), prec, 0);
  apply<T>(c, op, (const T*)Xout, res, R, -1.0, 1.0, 1, false, prec);
  double* part = (double*)c->ws.get("psolve.part", 8 * (size_t)dot_blocks(N) * R);
  double* rr = (double*)c->ws.get("psolve.rr", 8 * R);
  double* bb = (double*)c->ws.get("psolve.bb", 8 * R);
  dots<T>(c, res, res, N, R, part, rr);
  dots<T>(c, (const T*)Bin, (const T*)Bin, N, R, part, bb);
  std::vector<double> hrr(R), hbb(R);
  COLA_CUDA(cudaMemcpyAsync(hrr.data(), rr, 8 * R, cudaMemcpyDeviceToHost, c->s));
  COLA_CUDA(cudaMemcpyAsync(hbb.data(), bb, 8 * R, cudaMemcpyDeviceToHost, c->s));
  COLA_CUDA(cudaStreamSynchronize(c->s));
  for (int64_t r = 0; r < R; ++r) {
    acc[r].rel_residual = hbb[r] > 0 ? sqrt(std::max(hrr[r], 0.0) / hbb[r]) : 0.0;
    if (info) info[r] = acc[r];
  }
  return worst;
}

}  // namespace
}  // namespace cola

using namespace cola;

extern "C" cola_status cola_product_solve(cola_ctx* ctx, const cola_linop* op, const void* B,
                                          void* X, int64_t nrhs, const cola_cg_opts* opts,
                                          int32_t use_structure, cola_cg_info* info,
                                          cola_stream stream) {
  cola_status result = COLA_OK;
  cola_status st = guard([&] {
    COLA_REQUIRE(ctx && op && B && X && opts, COLA_ERR_INVALID_ARG, "NULL argument");
    COLA_REQUIRE(nrhs >= 1, COLA_ERR_INVALID_ARG, "nrhs = %lld", (long long)nrhs);
    COLA_REQUIRE(op->rows == op->cols, COLA_ERR_SHAPE, "product solve needs a square operator");
    COLA_REQUIRE(opts->precision >= COLA_PREC_F64 && opts->precision <= COLA_PREC_MIXED,
                 COLA_ERR_INVALID_ARG, "precision %d", opts->precision);
    COLA_REQUIRE(B != X, COLA_ERR_INVALID_ARG, "B and X must not alias");
    StreamJoin j(ctx, stream);
    const bool io64 = opts->precision == COLA_PREC_F64 || opts->refine;
    result = io64 ? product_solve<double>(ctx, op, B, X, nrhs, *opts, use_structure != 0, info)
                  : product_solve<float>(ctx, op, B, X, nrhs, *opts, use_structure != 0, info);
    if (result != COLA_OK) set_error_message("a factor's CG solve did not reach tol");
  });
  return st != COLA_OK ? st : result;
}
