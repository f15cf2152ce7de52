// Householder Arnoldi / Lanczos (Algorithm 2) for nvec starting vectors at
// once, each with its own Krylov space.
//
// Step j builds the reflector R_j = I - 2 u_j u_j^T that maps the tail
// nu_j[j:] onto a multiple of e_j, reads column j-1 of the Hessenberg matrix
// off R_j nu_j, forms q_j = R_0 ... R_j e_j and nu_{j+1} = R_j ... R_0 A q_j.
// The basis is orthogonal to working precision however many steps run, which
// is what makes the iteration usable in FP32 (App. C.3).  The products of
// reflectors use the compact WY form P_j = R_0 ... R_j = I + Y W Y^T (W upper
// triangular, Schreiber & Van Loan 1989), so each step is a handful of passes
// over the stored reflectors:
//   q_j      = e_j + Y (W y_j),          y_j = (u_0[j], .., u_j[j]),
//   nu_{j+1} = A q_j + Y (W^T (Y^T A q_j)).
// The reflector uses the sign that avoids cancellation, u_j[j] = nu_j + sign *
// ||tail|| (Golub & Van Loan 5.1.2): R_j nu_j then has -sign ||tail|| at j, so
// H differs from Algorithm 2's by a +-1 diagonal similarity (same diagonal,
// same eigenvalues, off-diagonal signs flipped).  Vectors and reflectors are
// stored in the working precision.  In FP64 every product runs in FP64; in
// FP32 the long sums (the dot products with the stored reflectors and their
// linear combinations) multiply in FP32 and accumulate runs of 16 products in
// FP32 before adding them in FP64 (GB300's FP64 rate would otherwise bound
// these passes), and the small W, H arithmetic stays FP64.
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "internal.h"

namespace cola {

namespace {

struct HhState {
  double amax;  // largest |H_ii| so far (breakdown scale)
  int stop;     // breakdown reached
  int meff;     // completed steps
};

// sum over k >= j of nu[k]^2, per (block, probe)
template <typename T>
__global__ void k_hh_tail(int64_t N, const T* nu, int j, double* part) {
  const int64_t p = blockIdx.y;
  const T* x = nu + p * N;
  double s = 0.0;
  for (int64_t k = j + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)x[k];
    s += v * v;
  }
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    part[p * gridDim.x + blockIdx.x] = t;
  }
}

// One thread per probe: the reflector's coefficients and H column j-1.
// coef[p] = (alpha, nu_j - alpha, 1/||u|| or 0 after a breakdown).
template <typename T>
__global__ void k_hh_reflector(int64_t N, int nv, const T* nu, int j, int m, const double* part,
                               int nb, double eps, HhState* st, double* coef, double* H) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nv) return;
  HhState& s = st[p];
  const T* x = nu + (int64_t)p * N;
  double tail2 = 0.0;
  for (int b = 0; b < nb; ++b) tail2 += part[(int64_t)p * nb + b];
  const double xj = (double)x[j];
  const double nrm = sqrt(tail2);
  const double alpha = xj >= 0.0 ? -nrm : nrm;
  if (j >= 1 && !s.stop) {
    double* Hp = H + (int64_t)p * (m + 1) * m;
    for (int i = 0; i < j; ++i) Hp[(int64_t)i * m + (j - 1)] = (double)x[i];
    Hp[(int64_t)j * m + (j - 1)] = alpha;
    s.amax = fmax(s.amax, fabs((double)x[j - 1]));
    if (nrm <= eps * s.amax) {
      s.stop = 1;
      s.meff = j;
    }
  }
  const double v0 = xj - alpha;
  const double un2 = tail2 - xj * xj + v0 * v0;
  const bool ok = !s.stop && un2 > 0.0 && j < N;
  coef[3 * p + 0] = alpha;
  coef[3 * p + 1] = v0;
  coef[3 * p + 2] = ok ? 1.0 / sqrt(un2) : 0.0;
}

// Y[p][j][k] = u_j[k]
template <typename T>
__global__ void k_hh_write_u(int64_t N, const T* nu, int j, int m, const double* coef, T* Y) {
  const int64_t p = blockIdx.y;
  const T* x = nu + p * N;
  T* u = Y + (p * (m + 1) + j) * N;
  const double v0 = coef[3 * p + 1], inv = coef[3 * p + 2];
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (k == j)
      v = v0 * inv;
    else if (k > j)
      v = (double)x[k] * inv;
    u[k] = (T)v;
  }
}

// part[p][i][b] = sum over block b's chunk of Y[p][i][k] x[p][k], i < cnt.
// Warp w of the block handles i = w, w + 8, ...
template <typename T>
__global__ void k_hh_multidot(int64_t N, const T* Y, int m, const T* X, int64_t xstride, int cnt,
                              double* part) {
  const int64_t p = blockIdx.y;
  const int nb = gridDim.x;
  const int64_t chunk = (N + nb - 1) / nb;
  const int64_t k0 = (int64_t)blockIdx.x * chunk;
  const int64_t k1 = min(N, k0 + chunk);
  const T* x = X + p * xstride;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i < cnt; i += (int)(blockDim.x >> 5)) {
    const T* y = Y + (p * (m + 1) + i) * N;
    double s = 0.0;
    if constexpr (std::is_same<T, float>::value) {
      int64_t k = k0 + lane;
      while (k < k1) {
        float f = 0.0f;
        for (int t = 0; t < 16 && k < k1; ++t, k += 32) f = fmaf(y[k], x[k], f);
        s += (double)f;
      }
    } else {
      for (int64_t k = k0 + lane; k < k1; k += 32) s += (double)y[k] * (double)x[k];
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) part[(p * (m + 1) + i) * nb + blockIdx.x] = s;
  }
}

// FP32 variant for N % 4 == 0: a block walks chunks of 2048 entries; every
// thread keeps its 8 entries of x in registers and, for each stored reflector
// i < cnt, multiplies them with 8 entries of Y[p][i] (two 16-byte loads per
// thread, 512 coalesced bytes per warp), reduces across the warp in FP32 and
// adds the warp's sum into an FP64 slot [i][warp] in shared memory.
__global__ void k_hh_multidot4(int64_t N, const float* Y, int m, const float* X, int64_t xstride,
                               int cnt, double* part) {
  const int64_t p = blockIdx.y;
  const int nb = gridDim.x;
  __shared__ double wsum[256][8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = lane; i < cnt; i += 32) wsum[i][warp] = 0.0;
  __syncwarp();
  const float* x = X + p * xstride;
  const float* Yp = Y + p * (int64_t)(m + 1) * N;
  const int64_t nchunks = (N + 2047) / 2048;
  const float4 zero = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += nb) {
    const int64_t k = ch * 2048 + (int64_t)threadIdx.x * 8;
    const bool in0 = k < N, in1 = k + 4 < N;
    const float4 x0 = in0 ? *reinterpret_cast<const float4*>(x + k) : zero;
    const float4 x1 = in1 ? *reinterpret_cast<const float4*>(x + k + 4) : zero;
    for (int i = 0; i < cnt; ++i) {
      const float* y = Yp + (int64_t)i * N;
      const float4 y0 = in0 ? *reinterpret_cast<const float4*>(y + k) : zero;
      const float4 y1 = in1 ? *reinterpret_cast<const float4*>(y + k + 4) : zero;
      float f = x0.x * y0.x;
      f = fmaf(x0.y, y0.y, f);
      f = fmaf(x0.z, y0.z, f);
      f = fmaf(x0.w, y0.w, f);
      f = fmaf(x1.x, y1.x, f);
      f = fmaf(x1.y, y1.y, f);
      f = fmaf(x1.z, y1.z, f);
      f = fmaf(x1.w, y1.w, f);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
      if (lane == 0) wsum[i][warp] += (double)f;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += wsum[i][w];
    part[(p * (m + 1) + i) * nb + blockIdx.x] = s;
  }
}

// out[p][i] = sum_b part[p][i][b] (fixed order), i < cnt.
__global__ void k_hh_multidot_final(const double* part, int m, int nb, int cnt, double* out) {
  const int64_t p = blockIdx.x;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(p * (m + 1) + i) * nb + b];
    out[p * (m + 1) + i] = s;
  }
}

// W gains column j: W[i][j] = -2 sum_{l=i..j-1} W[i][l] s[l], W[j][j] = -2
// (P_j = P_{j-1} R_j); then c = W y_j with y_j[i] = Y[p][i][j].
template <typename T>
__global__ void k_hh_w_and_c(int64_t N, const T* Y, int j, int m, const double* s, double* W,
                             double* c) {
  const int64_t p = blockIdx.x;
  const int M1 = m + 1;
  double* Wp = W + p * M1 * M1;
  const double* sp = s + p * M1;
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    double acc = 0.0;
    for (int l = i; l < j; ++l) acc += Wp[i * M1 + l] * sp[l];
    Wp[i * M1 + j] = -2.0 * acc;
  }
  if (threadIdx.x == 0) {
    Wp[j * M1 + j] = -2.0;
    for (int i = j + 1; i < M1; ++i) Wp[i * M1 + j] = 0.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    double acc = 0.0;
    for (int l = i; l <= j; ++l) acc += Wp[i * M1 + l] * (double)Y[(p * M1 + l) * N + j];
    c[p * M1 + i] = acc;
  }
}

// t = W^T s over the first cnt entries (W upper triangular).
__global__ void k_hh_wt(const double* W, int m, int cnt, const double* s, double* t) {
  const int64_t p = blockIdx.x;
  const int M1 = m + 1;
  const double* Wp = W + p * M1 * M1;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    double acc = 0.0;
    for (int l = 0; l <= i; ++l) acc += Wp[l * M1 + i] * s[p * M1 + l];
    t[p * M1 + i] = acc;
  }
}

// out[p][k] = base[p][k] (or e_j when base is null) + sum_{i<cnt} c[p][i] Y[p][i][k]
template <typename T>
__global__ void k_hh_lincomb(int64_t N, const T* base, int j, const T* Y, int m, int cnt,
                             const double* c, T* out) {
  const int64_t p = blockIdx.y;
  __shared__ double cs[256];
  __shared__ float cs32[256];
  const int M1 = m + 1;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    cs[i] = c[p * M1 + i];
    cs32[i] = (float)cs[i];
  }
  __syncthreads();
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x) {
    double acc = base ? (double)base[p * N + k] : (k == j ? 1.0 : 0.0);
    if constexpr (std::is_same<T, float>::value) {
      for (int i0 = 0; i0 < cnt; i0 += 16) {
        float f = 0.0f;
        const int i1 = min(cnt, i0 + 16);
        for (int i = i0; i < i1; ++i) f = fmaf(cs32[i], Y[(p * M1 + i) * N + k], f);
        acc += (double)f;
      }
    } else {
      for (int i = 0; i < cnt; ++i) acc += cs[i] * (double)Y[(p * M1 + i) * N + k];
    }
    out[p * N + k] = (T)acc;
  }
}

__global__ void k_hh_init(HhState* st, int nv, int m) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nv) return;
  st[p].amax = 0.0;
  st[p].stop = 0;
  st[p].meff = m;
}

// Lanczos coefficients from H: alpha_i = H[i][i], beta_i = |H[i+1][i]|.
__global__ void k_hh_extract(const double* H, const HhState* st, int nv, int m, double* alpha,
                             double* beta, int* m_eff) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nv) return;
  const double* Hp = H + (int64_t)p * (m + 1) * m;
  const int me = st[p].meff;
  for (int i = 0; i < m; ++i) {
    alpha[(int64_t)p * m + i] = i < me ? Hp[(int64_t)i * m + i] : 0.0;
    beta[(int64_t)p * m + i] = (i + 1 < me) ? fabs(Hp[(int64_t)(i + 1) * m + i]) : 0.0;
  }
  m_eff[p] = me;
}

template <typename T>
void hh_run(Ctx* c, const cola_linop* op, const T* Q0, int64_t nv, int m, int prec, double* H,
            int* m_eff_dev, double* alpha, double* beta) {
  const int64_t N = op->rows;
  COLA_REQUIRE(m >= 1 && m <= 255, COLA_ERR_UNSUPPORTED, "Householder Arnoldi: m = %d (1..255)",
               m);
  COLA_REQUIRE(m < N, COLA_ERR_INVALID_ARG, "Householder Arnoldi: m = %d >= N", m);
  auto& ws = c->ws;
  const int M1 = m + 1;
  prepare_leaves(c, const_cast<cola_linop*>(op), prec, c->split_factor_terms);
  T* Y = (T*)ws.get("hh.Y", sizeof(T) * (size_t)nv * M1 * N);
  T* q = (T*)ws.get("hh.q", sizeof(T) * (size_t)nv * N);
  T* w = (T*)ws.get("hh.w", sizeof(T) * (size_t)nv * N);
  T* nu = (T*)ws.get("hh.nu", sizeof(T) * (size_t)nv * N);
  const int nb = (int)std::max<int64_t>(
      1, std::min<int64_t>((N + 4095) / 4096, std::max<int64_t>(1, 4 * c->num_sms / nv)));
  // the FP32 multi-dot over 2048-entry chunks (N % 4 == 0; 16-byte rows)
  const bool md4 = std::is_same<T, float>::value && N % 4 == 0;
  const int nb4 = (int)std::max<int64_t>(
      1, std::min<int64_t>((N + 2047) / 2048, std::max<int64_t>(1, 8 * c->num_sms / nv)));
  double* part = (double*)ws.get("hh.part", 8 * (size_t)nv * M1 * std::max(nb, nb4));
  double* s = (double*)ws.get("hh.s", 8 * (size_t)nv * M1);
  double* cv = (double*)ws.get("hh.c", 8 * (size_t)nv * M1);
  double* W = (double*)ws.get("hh.W", 8 * (size_t)nv * M1 * M1);
  double* coef = (double*)ws.get("hh.coef", 24 * (size_t)nv);
  HhState* st = (HhState*)ws.get("hh.st", sizeof(HhState) * nv);
  COLA_CUDA(cudaMemsetAsync(H, 0, 8 * (size_t)nv * M1 * m, c->s));
  COLA_CUDA(cudaMemsetAsync(W, 0, 8 * (size_t)nv * M1 * M1, c->s));
  COLA_CUDA(cudaMemcpyAsync(nu, Q0, sizeof(T) * (size_t)nv * N, cudaMemcpyDeviceToDevice, c->s));
  const unsigned pb = (unsigned)((nv + 127) / 128);
  k_hh_init<<<pb, 128, 0, c->s>>>(st, (int)nv, m);
  c->count_launch();
  const double eps = (prec == COLA_PREC_F64) ? 1e-10 : 1e-6;
  const int gx = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 2 * c->num_sms));
  const dim3 g2(gx, (unsigned)nv), gnb(nb, (unsigned)nv), gnb4(nb4, (unsigned)nv);
  // s[p][0..cnt) = Y[p][0..cnt)^T x[p]
  auto multidot = [&](const T* x, int64_t xstride, int cnt) {
    if constexpr (std::is_same<T, float>::value) {
      if (md4) {
        k_hh_multidot4<<<gnb4, 256, 0, c->s>>>(N, Y, m, x, xstride, cnt, part);
        k_hh_multidot_final<<<(unsigned)nv, 128, 0, c->s>>>(part, m, nb4, cnt, s);
        return;
      }
    }
    k_hh_multidot<T><<<gnb, 256, 0, c->s>>>(N, Y, m, x, xstride, cnt, part);
    k_hh_multidot_final<<<(unsigned)nv, 128, 0, c->s>>>(part, m, nb, cnt, s);
  };
  for (int j = 0; j <= m; ++j) {
    k_hh_tail<T><<<gnb, 256, 0, c->s>>>(N, nu, j, part);
    k_hh_reflector<T><<<pb, 128, 0, c->s>>>(N, (int)nv, nu, j, m, part, nb, eps, st, coef, H);
    k_hh_write_u<T><<<g2, 256, 0, c->s>>>(N, nu, j, m, coef, Y);
    for (int i = 0; i < 3; ++i) c->count_launch();
    if (j == m) break;
    if (j >= 1) {
      // s = Y[0..j-1]^T u_j
      multidot(Y + (size_t)j * N, (int64_t)M1 * N, j);
      for (int i = 0; i < 2; ++i) c->count_launch();
    }
    k_hh_w_and_c<T><<<(unsigned)nv, 128, 0, c->s>>>(N, Y, j, m, s, W, cv);
    k_hh_lincomb<T><<<g2, 256, 0, c->s>>>(N, nullptr, j, Y, m, j + 1, cv, q);
    for (int i = 0; i < 2; ++i) c->count_launch();
    apply<T>(c, op, q, w, nv, 1.0, 0.0, 1, false, prec);
    multidot(w, N, j + 1);
    k_hh_wt<<<(unsigned)nv, 128, 0, c->s>>>(W, m, j + 1, s, cv);
    k_hh_lincomb<T><<<g2, 256, 0, c->s>>>(N, w, j, Y, m, j + 1, cv, nu);
    for (int i = 0; i < 4; ++i) c->count_launch();
    COLA_CUDA(cudaGetLastError());
  }
  if (alpha) {
    k_hh_extract<<<pb, 128, 0, c->s>>>(H, st, (int)nv, m, alpha, beta, m_eff_dev);
  } else {
    // m_eff only
    k_hh_extract<<<pb, 128, 0, c->s>>>(H, st, (int)nv, m,
                                       (double*)ws.get("hh.a", 8 * (size_t)nv * m),
                                       (double*)ws.get("hh.b", 8 * (size_t)nv * m), m_eff_dev);
  }
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
}

}  // namespace

void householder_lanczos(Ctx* c, const cola_linop* op, const void* Q0, int64_t nv, int m,
                         int prec, double* alpha, double* beta, int* m_eff) {
  double* H = (double*)c->ws.get("hh.H", 8 * (size_t)nv * (m + 1) * m);
  if (prec == COLA_PREC_F64)
    hh_run<double>(c, op, (const double*)Q0, nv, m, prec, H, m_eff, alpha, beta);
  else
    hh_run<float>(c, op, (const float*)Q0, nv, m, prec, H, m_eff, alpha, beta);
}

}  // namespace cola

using namespace cola;

extern "C" cola_status cola_arnoldi_householder(cola_ctx* ctx, const cola_linop* op,
                                                const void* Q0, int64_t nvec, int32_t m,
                                                int32_t precision, double* H, int32_t* m_eff,
                                                cola_stream stream) {
  return guard([&] {
    COLA_REQUIRE(ctx && op && Q0 && H && m_eff, COLA_ERR_INVALID_ARG, "NULL argument");
    COLA_REQUIRE(op->rows == op->cols, COLA_ERR_SHAPE, "Arnoldi needs a square operator");
    COLA_REQUIRE(nvec >= 1, COLA_ERR_INVALID_ARG, "nvec = %lld", (long long)nvec);
    COLA_REQUIRE(precision >= COLA_PREC_F64 && precision <= COLA_PREC_MIXED, COLA_ERR_INVALID_ARG,
                 "precision %d", precision);
    StreamJoin j(ctx, stream);
    if (precision == COLA_PREC_F64)
      hh_run<double>(ctx, op, (const double*)Q0, nvec, m, precision, H, m_eff, nullptr, nullptr);
    else
      hh_run<float>(ctx, op, (const float*)Q0, nvec, m, precision, H, m_eff, nullptr, nullptr);
  });
}
