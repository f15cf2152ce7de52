// Stochastic estimates of Diag(A) and Tr(A) (Sec. 3.3; App. B.1).
//
// Hutchinson: Diag(A) ~ (1/n) sum_v z_v (.) A z_v over n Rademacher probes,
// Tr(A) ~ the sum of that vector.  Doubly stochastic, for A = sum_i c_i A_i
// (a Sum node): every term gets its own independent probes,
// Diag(A) ~ sum_i c_i (1/n) sum_v z_iv (.) A_i z_iv, which removes the cross
// terms between summands from the estimator's variance.
//
// Probes come from the counter-based SplitMix64 stream of cola_rademacher:
// term i, probe v, entry k is output (i n + v) N + k of the stream seeded with
// `seed` (the base estimator is term 0), so any probe can be regenerated from
// its index alone.  Each term's probes are applied in chunks through the
// ordinary MVM path (tensor cores for MIXED Kronecker terms) and folded into
// an FP64 accumulator by one memory-bound kernel.
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace cola {

namespace {

// acc[k] += scale * sum_v Z[v, k] * AZ[v, k]  (coalesced over k).
template <typename T>
__global__ void k_probe_diag(int64_t N, int np, const T* Z, const T* AZ, double scale,
                             double* acc) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int v = 0; v < np; ++v) s += (double)Z[(int64_t)v * N + k] * (double)AZ[(int64_t)v * N + k];
    acc[k] += scale * s;
  }
}

// Per-block partial sums of x (fixed order within a block).
__global__ void k_block_sum(int64_t N, const double* x, double* part) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x)
    s += x[k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

template <typename T>
void estimate(Ctx* c, const cola_linop* op, int nprobes, uint64_t seed, bool doubly, int prec,
              double* acc) {
  const int64_t N = op->rows;
  std::vector<const cola_linop*> terms;
  std::vector<double> coeffs;
  if (doubly && op->kind == LK_SUM) {
    for (size_t i = 0; i < op->kids.size(); ++i) {
      terms.push_back(op->kids[i]);
      coeffs.push_back(op->coeffs[i]);
    }
  } else {
    terms.push_back(op);
    coeffs.push_back(1.0);
  }
  // probe chunk: both blocks together at most ~1 GB
  const size_t es = sizeof(T);
  const int pc = (int)std::max<int64_t>(
      1, std::min<int64_t>(nprobes, (int64_t)((1ull << 30) / (2 * es * (size_t)N))));
  T* Z = (T*)c->ws.get("est.z", es * (size_t)N * pc);
  T* AZ = (T*)c->ws.get("est.az", es * (size_t)N * pc);
  COLA_CUDA(cudaMemsetAsync(acc, 0, 8 * (size_t)N, c->s));
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 4 * c->num_sms));
  for (size_t i = 0; i < terms.size(); ++i) {
    for (int v0 = 0; v0 < nprobes; v0 += pc) {
      const int np = std::min(pc, nprobes - v0);
      const int64_t offset = ((int64_t)i * nprobes + v0) * N;
      rademacher(c, seed, offset, (int64_t)np * N, Z, sizeof(T) == 8 ? COLA_F64 : COLA_F32);
      apply<T>(c, terms[i], Z, AZ, np, 1.0, 0.0, 1, false, prec);
      k_probe_diag<T><<<grid, 256, 0, c->s>>>(N, np, Z, AZ, coeffs[i] / nprobes, acc);
      c->count_launch();
      COLA_CUDA(cudaGetLastError());
    }
  }
}

}  // namespace
}  // namespace cola

using namespace cola;

extern "C" cola_status cola_diag_estimate(cola_ctx* ctx, const cola_linop* op, int32_t nprobes,
                                          uint64_t seed, int32_t doubly, int32_t precision,
                                          double* diag, double* trace, cola_stream stream) {
  return guard([&] {
    COLA_REQUIRE(ctx && op, COLA_ERR_INVALID_ARG, "NULL argument");
    COLA_REQUIRE(diag || trace, COLA_ERR_INVALID_ARG, "neither diag nor trace requested");
    COLA_REQUIRE(op->rows == op->cols, COLA_ERR_SHAPE, "diagonal estimate needs a square operator");
    COLA_REQUIRE(nprobes >= 1, COLA_ERR_INVALID_ARG, "nprobes = %d", nprobes);
    COLA_REQUIRE(precision >= COLA_PREC_F64 && precision <= COLA_PREC_MIXED, COLA_ERR_INVALID_ARG,
                 "precision %d", precision);
    StreamJoin j(ctx, stream);
    const int64_t N = op->rows;
    prepare_leaves(ctx, const_cast<cola_linop*>(op), precision, ctx->split_factor_terms);
    double* acc = diag ? diag : (double*)ctx->ws.get("est.acc", 8 * (size_t)N);
    if (precision == COLA_PREC_F64)
      estimate<double>(ctx, op, nprobes, seed, doubly != 0, precision, acc);
    else
      estimate<float>(ctx, op, nprobes, seed, doubly != 0, precision, acc);
    if (precision == COLA_PREC_MIXED) tc_check_error(ctx);
    if (trace) {
      const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 1024));
      double* part = (double*)ctx->ws.get("est.part", 8 * 1024);
      k_block_sum<<<nb, 256, 0, ctx->s>>>(N, acc, part);
      ctx->count_launch();
      COLA_CUDA(cudaGetLastError());
      std::vector<double> hp(nb);
      COLA_CUDA(cudaMemcpyAsync(hp.data(), part, 8 * nb, cudaMemcpyDeviceToHost, ctx->s));
      COLA_CUDA(cudaStreamSynchronize(ctx->s));
      double t = 0.0;
      for (double v : hp) t += v;
      *trace = t;
    }
  });
}
