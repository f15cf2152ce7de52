// SIMT kernels of the composed-operator MVM: strided-batched GEMM for the
// Kronecker mode products (Sec. 3.2, Table 3: MVM of K_A (x) K_B costs
// tau_A N_B + N_A tau_B), the Kronecker-sum tridiagonal stencil, diagonal and
// low-rank terms, deterministic per-vector reductions, leaf-gradient
// contractions (App. B.2) and the SplitMix64 probe generator.
#include <algorithm>
#include <type_traits>

#include "internal.h"

namespace cola {

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t n, int per_thread = 1, int cap = 152 * 16) {
  int64_t b = (n + (int64_t)kThreads * per_thread - 1) / ((int64_t)kThreads * per_thread);
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, cap));
}

template <typename T>
__device__ __forceinline__ void ld4(T* dst, const T* src);
template <>
__device__ __forceinline__ void ld4<float>(float* d, const float* s) {
  float4 v = *reinterpret_cast<const float4*>(s);
  d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
}
template <>
__device__ __forceinline__ void ld4<double>(double* d, const double* s) {
  double2 a = *reinterpret_cast<const double2*>(s);
  double2 b = *reinterpret_cast<const double2*>(s + 2);
  d[0] = a.x; d[1] = a.y; d[2] = b.x; d[3] = b.y;
}

template <typename T>
struct GemmP {
  int64_t M, N, K;
  const T* A;
  int64_t lam, lak, sA;
  const T* B;
  int64_t lbk, lbn, sB;
  T* C;
  int64_t lcm, lcn, sC;
  T alpha, beta;
};

// C[b](m, n) = alpha * sum_k A[b](m, k) B[b](k, n) + beta * C[b](m, n) with
// arbitrary element strides.  128 x 128 x 8 tiles, 256 threads, 8 x 8
// outputs per thread; tile loads run along whichever stride is unit.
template <typename T>
__device__ __forceinline__ void gemm_tile_body(const GemmP<T>& g, const T* A, const T* B, T* C) {
  constexpr int BM = 128, BN = 128, BK = 8;
  __shared__ __align__(16) T As[BK][BM];
  __shared__ __align__(16) T Bs[BK][BN];
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = T(0);
  const bool a_m_fast = (g.lam == 1);
  const bool b_n_fast = (g.lbn == 1);
  for (int64_t k0 = 0; k0 < g.K; k0 += BK) {
#pragma unroll
    for (int e0 = 0; e0 < BM * BK; e0 += 256) {
      const int e = e0 + tid;
      int mm, kk;
      if (a_m_fast) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
      const int64_t m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < g.M && k < g.K) ? A[m * g.lam + k * g.lak] : T(0);
    }
#pragma unroll
    for (int e0 = 0; e0 < BN * BK; e0 += 256) {
      const int e = e0 + tid;
      int nn, kk;
      if (b_n_fast) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
      const int64_t n = n0 + nn, k = k0 + kk;
      Bs[kk][nn] = (n < g.N && k < g.K) ? B[k * g.lbk + n * g.lbn] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[8], bb[8];
      ld4(a, &As[kk][ty * 4]);
      ld4(a + 4, &As[kk][64 + ty * 4]);
      ld4(bb, &Bs[kk][tx * 4]);
      ld4(bb + 4, &Bs[kk][64 + tx * 4]);
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t n = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
      if (n >= g.N) continue;
      T* p = C + m * g.lcm + n * g.lcn;
      T v = g.alpha * acc[i][j];
      if (g.beta != T(0)) v += g.beta * *p;
      *p = v;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_gemm(GemmP<T> g, int64_t batch0) {
  const int64_t b = batch0 + blockIdx.z;
  gemm_tile_body<T>(g, g.A + b * g.sA, g.B + b * g.sB, g.C + b * g.sC);
}


// FP32 mode product on the SIMT cores, for the layout of the Kronecker mode
// steps: A m-fast (lam = 1, the input vector viewed as [k][m]), B k-fast
// (lbk = 1, the row-major factor F[n][k]), C n-fast (lcn = 1).  128 x 128
// output tile per block, k in tiles of 16, 256 threads with 8 x 8 outputs
// each; float4 global loads of the next k tile are held in registers while
// the current one is multiplied out of the other shared-memory buffer, so one
// barrier per k tile separates the two.  Needs M, N, lak, lbn, lcm and sA,
// sB, sC multiples of 4 and 16-byte aligned bases (checked on the host).
constexpr int kMfBM = 128, kMfBN = 128, kMfBK = 16, kMfPadN = kMfBN + 4;

__global__ void __launch_bounds__(256, 2) k_gemm_mode_f32(GemmP<float> g, int64_t batch0) {
  __shared__ __align__(16) float As[2][kMfBK][kMfBM];
  __shared__ __align__(16) float Bs[2][kMfBK][kMfPadN];
  const int64_t b = batch0 + blockIdx.z;
  const float* A = g.A + b * g.sA;
  const float* B = g.B + b * g.sB;
  float* C = g.C + b * g.sC;
  const int64_t m0 = (int64_t)blockIdx.x * kMfBM, n0 = (int64_t)blockIdx.y * kMfBN;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // this thread's loads per k tile: A rows ka, ka + 8 at column ma (float4);
  // B rows nb, nb + 64 at k offset kb (float4 along k)
  const int ka = tid >> 5, ma = (tid & 31) * 4;
  const int nb = tid >> 2, kb = (tid & 3) * 4;
  const bool a_in = m0 + ma < g.M;
  const bool b_in0 = n0 + nb < g.N, b_in1 = n0 + nb + 64 < g.N;
  float4 ra[2], rb[2];
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t k = k0 + ka + 8 * h;
      ra[h] = (a_in && k < g.K)
                  ? __ldg(reinterpret_cast<const float4*>(A + k * g.lak + m0 + ma))
                  : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int64_t k = k0 + kb;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const bool in = (h ? b_in1 : b_in0);
      const float* src = B + (n0 + nb + 64 * h) * g.lbn + k;
      if (in && k + 4 <= g.K) {
        rb[h] = __ldg(reinterpret_cast<const float4*>(src));
      } else {
        rb[h].x = (in && k < g.K) ? src[0] : 0.f;
        rb[h].y = (in && k + 1 < g.K) ? src[1] : 0.f;
        rb[h].z = (in && k + 2 < g.K) ? src[2] : 0.f;
        rb[h].w = (in && k + 3 < g.K) ? src[3] : 0.f;
      }
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int h = 0; h < 2; ++h)
      *reinterpret_cast<float4*>(&As[buf][ka + 8 * h][ma]) = ra[h];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int n = nb + 64 * h;
      Bs[buf][kb + 0][n] = rb[h].x;
      Bs[buf][kb + 1][n] = rb[h].y;
      Bs[buf][kb + 2][n] = rb[h].z;
      Bs[buf][kb + 3][n] = rb[h].w;
    }
  };
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  const int ntk = (int)((g.K + kMfBK - 1) / kMfBK);
  load(0);
  store(0);
  __syncthreads();
  for (int t = 0; t < ntk; ++t) {
    const int cur = t & 1;
    if (t + 1 < ntk) load((int64_t)(t + 1) * kMfBK);
#pragma unroll
    for (int kk = 0; kk < kMfBK; ++kk) {
      float a[8], bb[8];
      ld4(a, &As[cur][kk][ty * 4]);
      ld4(a + 4, &As[cur][kk][64 + ty * 4]);
      ld4(bb, &Bs[cur][kk][tx * 4]);
      ld4(bb + 4, &Bs[cur][kk][64 + tx * 4]);
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
    }
    if (t + 1 < ntk) store(cur ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (m >= g.M) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t n = n0 + h * 64 + tx * 4;
      if (n >= g.N) continue;
      float4* p = reinterpret_cast<float4*>(C + m * g.lcm + n);
      float4 v = make_float4(g.alpha * acc[i][4 * h], g.alpha * acc[i][4 * h + 1],
                             g.alpha * acc[i][4 * h + 2], g.alpha * acc[i][4 * h + 3]);
      if (g.beta != 0.f) {
        const float4 o = *p;
        v.x += g.beta * o.x;
        v.y += g.beta * o.y;
        v.z += g.beta * o.z;
        v.w += g.beta * o.w;
      }
      *p = v;
    }
  }
}

// Small products (the whole C would fill only a few 128 x 128 tiles): one
// thread per output element, so that the work spreads over many SMs instead
// of sitting in one block; each thread runs its K-term dot product in order.
template <typename T>
__global__ void __launch_bounds__(256) k_gemm_small(GemmP<T> g, int64_t total) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t mn = g.M * g.N;
    const int64_t b = t / mn, rem = t - b * mn;
    // consecutive threads take consecutive m when A is m-fast, else consecutive n
    int64_t m, n;
    if (g.lam == 1) {
      n = rem / g.M;
      m = rem - n * g.M;
    } else {
      m = rem / g.N;
      n = rem - m * g.N;
    }
    const T* a = g.A + b * g.sA + m * g.lam;
    const T* bb = g.B + b * g.sB + n * g.lbn;
    T acc = T(0);
    for (int64_t k = 0; k < g.K; ++k) acc = fma(a[k * g.lak], bb[k * g.lbk], acc);
    T* p = g.C + b * g.sC + m * g.lcm + n * g.lcn;
    T v = g.alpha * acc;
    if (g.beta != T(0)) v += g.beta * *p;
    *p = v;
  }
}

// Grouped variant: problem blockIdx.z of a device table, same tiling.
template <typename T>
__global__ void __launch_bounds__(256) k_gemm_grouped(const GemmDesc<T>* probs) {
  const GemmDesc<T>& q = probs[blockIdx.z];
  if ((int64_t)blockIdx.x * 128 >= q.M || (int64_t)blockIdx.y * 128 >= q.N) return;
  GemmP<T> g{q.M, q.N, q.K, q.A, q.lam, q.lak, 0, q.B, q.lbk, q.lbn, 0, q.C, q.lcm, q.lcn, 0,
             q.alpha, q.beta};
  gemm_tile_body<T>(g, g.A, g.B, g.C);
}

// FP64 products in 32 x 32 output tiles (k in steps of 8, 256 threads with 4
// outputs each).  On this GPU the FP64 multiply-adds are the whole cost: small
// tiles keep the zero padding of small problems low (a 128 x 128 tile of a
// 40 x 60 problem is 85 % padding), and with 4 accumulators per thread many
// more warps stay resident than with 8 x 8 (measured: 1.40 TFLOP/s on the
// 512-system batch against 1.15 for 128 x 128 tiles on full 128^3 products).
template <typename T>
__device__ __forceinline__ void gemm32_tile(int64_t M, int64_t N, int64_t K, const T* A,
                                            int64_t lam, int64_t lak, const T* B, int64_t lbk,
                                            int64_t lbn, T* C, int64_t lcm, int64_t lcn, T alpha,
                                            T beta) {
  constexpr int BM = 32, BN = 32, BK = 8;
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  if (m0 >= M || n0 >= N) return;
  __shared__ T As[BK][BM];
  __shared__ T Bs[BK][BN];
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;  // n = tx, m = 4 ty + i
  const bool a_m_fast = (lam == 1), b_n_fast = (lbn == 1);
  T acc[4] = {T(0), T(0), T(0), T(0)};
  for (int64_t k0 = 0; k0 < K; k0 += BK) {
    {
      const int e = tid;  // BM * BK = 256 elements of A, 256 of B
      int mm, kk;
      if (a_m_fast) { mm = e % BM; kk = e / BM; } else { kk = e % BK; mm = e / BK; }
      const int64_t m = m0 + mm, k = k0 + kk;
      As[kk][mm] = (m < M && k < K) ? A[m * lam + k * lak] : T(0);
      int nn;
      if (b_n_fast) { nn = e % BN; kk = e / BN; } else { kk = e % BK; nn = e / BK; }
      const int64_t n = n0 + nn, kb = k0 + kk;
      Bs[kk][nn] = (n < N && kb < K) ? B[kb * lbk + n * lbn] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const T b = Bs[kk][tx];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[i] = fma(As[kk][4 * ty + i], b, acc[i]);
    }
    __syncthreads();
  }
  const int64_t n = n0 + tx;
  if (n >= N) return;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t m = m0 + 4 * ty + i;
    if (m >= M) continue;
    T* p = C + m * lcm + n * lcn;
    T v = alpha * acc[i];
    if (beta != T(0)) v += beta * *p;
    *p = v;
  }
}

// Grouped: problem blockIdx.z of a device table.
template <typename T>
__global__ void __launch_bounds__(256) k_gemm_grouped32(const GemmDesc<T>* probs) {
  const GemmDesc<T>& q = probs[blockIdx.z];
  gemm32_tile<T>(q.M, q.N, q.K, q.A, q.lam, q.lak, q.B, q.lbk, q.lbn, q.C, q.lcm, q.lcn,
                 q.alpha, q.beta);
}

// Strided batch: batch entry batch0 + blockIdx.z.
template <typename T>
__global__ void __launch_bounds__(256) k_gemm32(GemmP<T> g, int64_t batch0) {
  const int64_t b = batch0 + blockIdx.z;
  gemm32_tile<T>(g.M, g.N, g.K, g.A + b * g.sA, g.lam, g.lak, g.B + b * g.sB, g.lbk, g.lbn,
                 g.C + b * g.sC, g.lcm, g.lcn, g.alpha, g.beta);
}

// ------------------------------------------------------------- reductions
template <typename T>
__device__ __forceinline__ double block_sum(T v) {
  __shared__ double sh[32];
  double x = (double)v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = x;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

template <typename T>
__global__ void k_dot_partial(const T* a, const T* b, int64_t n, int nblk, double* part) {
  const int64_t r = blockIdx.y;
  const T* ar = a + r * n;
  const T* br = b + r * n;
  T s = T(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)nblk * blockDim.x)
    s = fma(ar[i], br[i], s);
  const double t = block_sum(s);
  if (threadIdx.x == 0) part[r * nblk + blockIdx.x] = t;
}

// One block per vector: a strided serial sum per thread, then the block's
// shuffle tree (fixed order, run-to-run deterministic).
__global__ void k_dot_final(const double* part, int nblk, int64_t R, double* out) {
  const int64_t r = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += part[r * nblk + i];
  const double t = block_sum(s);
  if (threadIdx.x == 0) out[r] = t;
}

// ------------------------------------------------------------ elementwise
template <typename TI, typename TO>
__global__ void k_convert(const TI* in, TO* out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (TO)in[i];
}

template <typename T>
__global__ void k_scale_rows(T* X, int64_t n, int64_t R, const double* w) {
  const int64_t tot = n * R;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x)
    X[i] = (T)((double)X[i] * w[i / n]);
}

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T>
__global__ void k_rademacher(uint64_t seed, int64_t offset, int64_t count, T* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (splitmix64_at(seed, (uint64_t)(offset + i)) >> 63) ? T(-1) : T(1);
}

template <typename T>
__global__ void k_diag(const T* d, int64_t stride, const T* X, T* Y, int64_t n, int64_t R,
                       T coeff, T beta) {
  const int64_t tot = n * R;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T dv = stride ? d[i % n] : d[0];
    T v = coeff * dv * X[i];
    if (beta != T(0)) v += beta * Y[i];
    Y[i] = v;
  }
}

struct StencilP {
  int nf;
  int64_t n[8];
  int64_t st[8];
  int64_t boff[8];
};

// Kronecker sum of tridiagonal factors: y = coeff * sum_k (A_k along mode k) x + beta y.
// Two-factor Kronecker sum of tridiagonal factors (n1 x n2 grid, rows of n2
// contiguous): four consecutive i2 of one row per thread, 32-bit indices within
// a vector; the same terms in the same order as k_stencil.  Optionally a
// diagonal term in the same pass: y += dcoeff d (.) x (d per element when
// dstride != 0, else d[0]).
template <typename T>
__global__ void k_stencil2(const T* bands, const T* X, T* Y, int n1, int n2, int64_t R, T coeff,
                           T beta, const T* dg, int64_t dstride, T dcoeff) {
  const int q4 = n2 / 4;
  const int64_t tot = (int64_t)n1 * q4 * R;
  const T* lo0 = bands;
  const T* di0 = bands + n1;
  const T* up0 = bands + 2 * n1;
  const T* lo1 = bands + 3 * n1;
  const T* di1 = lo1 + n2;
  const T* up1 = lo1 + 2 * n2;
  const int64_t N = (int64_t)n1 * n2;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / ((int64_t)n1 * q4);
    const int rem = (int)(t - r * (int64_t)n1 * q4);
    const int i1 = rem / q4, i2 = (rem - i1 * q4) * 4;
    const T* x = X + r * N + (int64_t)i1 * n2;
    T xc[4], xu[4], xd[4];
    ld4(xc, x + i2);
    if (i1 > 0) ld4(xu, x + i2 - n2);
    if (i1 < n1 - 1) ld4(xd, x + i2 + n2);
    const T xl = i2 > 0 ? x[i2 - 1] : T(0);
    const T xr = i2 + 4 < n2 ? x[i2 + 4] : T(0);
    T out[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int j = i2 + e;
      T v = T(0);
      v = fma(di0[i1], xc[e], v);
      if (i1 > 0) v = fma(lo0[i1], xu[e], v);
      if (i1 < n1 - 1) v = fma(up0[i1], xd[e], v);
      v = fma(di1[j], xc[e], v);
      if (j > 0) v = fma(lo1[j], e > 0 ? xc[e - 1] : xl, v);
      if (j < n2 - 1) v = fma(up1[j], e < 3 ? xc[e + 1] : xr, v);
      out[e] = v * coeff;
    }
    if (dg) {
      T dd[4];
      if (dstride)
        ld4(dd, dg + (int64_t)i1 * n2 + i2);
      else
        dd[0] = dd[1] = dd[2] = dd[3] = dg[0];
#pragma unroll
      for (int e = 0; e < 4; ++e) out[e] = fma(dcoeff * dd[e], xc[e], out[e]);
    }
    T* y = Y + r * N + (int64_t)i1 * n2 + i2;
    if (beta != T(0)) {
      T yo[4];
      ld4(yo, y);
#pragma unroll
      for (int e = 0; e < 4; ++e) out[e] += beta * yo[e];
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) y[e] = out[e];
  }
}

// k_stencil2 by strips: a thread walks S (<= kStencilStrip) rows of one column quad,
// keeping the rows above, at and below in registers (each row of x is loaded
// once per strip, plus one halo row at each end), and takes the left and right
// neighbours of its quad from the adjacent lanes.  The same terms in the same
// order as k_stencil2 (bit-identical results).  Work item t = (r, strip, quad),
// the quad fastest; a warp runs its items together (lanes past the end only
// take part in the exchanges).
constexpr int kStencilStrip = 16;
template <typename T>
__global__ void k_stencil2s(const T* bands, const T* X, T* Y, int n1, int n2, int64_t R, T coeff,
                            T beta, const T* dg, int64_t dstride, T dcoeff, int S) {
  const int q4 = n2 / 4;
  const int ns = (n1 + S - 1) / S;
  const int64_t tot = (int64_t)R * ns * q4;
  const T* lo0 = bands;
  const T* di0 = bands + n1;
  const T* up0 = bands + 2 * n1;
  const T* lo1 = bands + 3 * n1;
  const T* di1 = lo1 + n2;
  const T* up1 = lo1 + 2 * n2;
  const int64_t N = (int64_t)n1 * n2;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); t0 < tot;
       t0 += stride) {
    const int64_t t = t0 + lane;
    const bool on = t < tot;
    const int64_t tt = on ? t : tot - 1;
    const int cq = (int)(tt % q4);
    const int64_t rs = tt / q4;
    const int sidx = (int)(rs % ns);
    const int64_t r = rs / ns;
    const int i2 = cq * 4;
    const int i1a = sidx * S;  // < n1
    const int i1b = min(i1a + S, n1);
    const T* x = X + r * N + i2;
    T* y = Y + r * N + i2;
    // the left neighbour comes from lane - 1 when that lane holds quad cq - 1 of
    // the same rows, the right one from lane + 1 likewise
    const bool l_sh = lane > 0 && cq > 0;
    const bool r_sh = lane < 31 && cq < q4 - 1 && t + 1 < tot;
    T b_lo1[4], b_di1[4], b_up1[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      b_lo1[e] = lo1[i2 + e];
      b_di1[e] = di1[i2 + e];
      b_up1[e] = up1[i2 + e];
    }
    T xu[4], xc[4], xd[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) xu[e] = xd[e] = T(0);
    if (i1a > 0) ld4(xu, x + (int64_t)(i1a - 1) * n2);
    ld4(xc, x + (int64_t)i1a * n2);
    // every lane takes S steps (the exchanges need the whole warp); a step
    // past the lane's strip computes and stores nothing
    for (int k = 0; k < S; ++k) {
      const int i1 = i1a + k;
      const bool act = i1 < i1b;
      const T* xrow = x + (int64_t)(act ? i1 : i1a) * n2;
      if (act && i1 + 1 < n1) ld4(xd, xrow + n2);
      T xl = __shfl_up_sync(0xffffffffu, xc[3], 1);
      T xr = __shfl_down_sync(0xffffffffu, xc[0], 1);
      if (!act) continue;
      if (!l_sh) xl = cq > 0 ? xrow[-1] : T(0);
      if (!r_sh) xr = cq < q4 - 1 ? xrow[4] : T(0);
      const T a0 = di0[i1], l0 = lo0[i1], u0 = up0[i1];
      T out[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int j = i2 + e;
        T v = T(0);
        v = fma(a0, xc[e], v);
        if (i1 > 0) v = fma(l0, xu[e], v);
        if (i1 < n1 - 1) v = fma(u0, xd[e], v);
        v = fma(b_di1[e], xc[e], v);
        if (j > 0) v = fma(b_lo1[e], e > 0 ? xc[e - 1] : xl, v);
        if (j < n2 - 1) v = fma(b_up1[e], e < 3 ? xc[e + 1] : xr, v);
        out[e] = v * coeff;
      }
      if (dg) {
        T dd[4];
        if (dstride)
          ld4(dd, dg + (int64_t)i1 * n2 + i2);
        else
          dd[0] = dd[1] = dd[2] = dd[3] = dg[0];
#pragma unroll
        for (int e = 0; e < 4; ++e) out[e] = fma(dcoeff * dd[e], xc[e], out[e]);
      }
      T* yrow = y + (int64_t)i1 * n2;
      if (on) {
        if (beta != T(0)) {
          T yo[4];
          ld4(yo, yrow);
#pragma unroll
          for (int e = 0; e < 4; ++e) out[e] += beta * yo[e];
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) yrow[e] = out[e];
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        xu[e] = xc[e];
        xc[e] = xd[e];
      }
    }
  }
}

template <typename T>
__global__ void k_stencil(StencilP p, const T* bands, const T* X, T* Y, int64_t N, int64_t R,
                          T coeff, T beta) {
  const int64_t tot = N * R;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t loc = idx % N;
    const T xc = X[idx];
    T v = T(0);
#pragma unroll 1
    for (int k = 0; k < p.nf; ++k) {
      const int64_t nk = p.n[k], sk = p.st[k];
      const int64_t ik = (loc / sk) % nk;
      const T* bd = bands + p.boff[k];
      v = fma(bd[nk + ik], xc, v);
      if (ik > 0) v = fma(bd[ik], X[idx - sk], v);
      if (ik < nk - 1) v = fma(bd[2 * nk + ik], X[idx + sk], v);
    }
    v *= coeff;
    if (beta != T(0)) v += beta * Y[idx];
    Y[idx] = v;
  }
}

// W partials: part[blk][k][R] = sum over this block's rows of V[i,k] X[r,i].
// Lane = column of V within a 32-column group; X tiles are shared by shuffles.
template <typename T>
__global__ void k_lr_vtx(const T* V, const T* X, int64_t n, int64_t kdim, int64_t R,
                         int nblk, double* part) {
  // lane = column k of V; a warp walks 32-row tiles, the x entries of the
  // tile's rows travel by shuffle.  Full tiles load all 32 V rows before
  // using them (32 independent loads in flight per lane).
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t k0 = (int64_t)blockIdx.y * 32, r0 = (int64_t)blockIdx.z * 8;
  const int64_t col = k0 + lane;
  const bool col_ok = col < kdim;
  T acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = T(0);
  const int64_t ntiles = (n + 31) / 32;
  for (int64_t t = (int64_t)blockIdx.x * nw + warp; t < ntiles; t += (int64_t)nblk * nw) {
    const int64_t i0 = t * 32;
    T xr[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      xr[q] = (r0 + q < R && i0 + lane < n) ? __ldg(X + (r0 + q) * n + i0 + lane) : T(0);
    if (i0 + 32 <= n) {
      T v[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = col_ok ? __ldg(V + (i0 + j) * kdim + col) : T(0);
#pragma unroll
      for (int j = 0; j < 32; ++j)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = fma(v[j], __shfl_sync(0xffffffffu, xr[q], j), acc[q]);
    } else {
      const int jmax = (int)(n - i0);
      for (int j = 0; j < jmax; ++j) {
        const T v = col_ok ? V[(i0 + j) * kdim + col] : T(0);
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = fma(v, __shfl_sync(0xffffffffu, xr[q], j), acc[q]);
      }
    }
  }
  __shared__ double sh[8][8][32];
#pragma unroll
  for (int q = 0; q < 8; ++q) sh[warp][q][lane] = (double)acc[q];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += sh[w][q][lane];
      if (col_ok && r0 + q < R) part[((int64_t)blockIdx.x * kdim + col) * R + r0 + q] = s;
    }
  }
}

// 16-byte asynchronous global -> shared copy; src_bytes = 0 fills zeros and
// reads nothing.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// FP32 W partials through a ring of shared-memory stages.  A block owns the
// contiguous rows [rb0, rb1) (a multiple of 128 apart), one 32-column group
// of V and one group of 8 right-hand sides; stage = 128 rows: V tile
// [128][32] and X tile [8][128], copied 16 bytes at a time with cp.async
// (kVtxStages - 1 stages in flight while one is consumed).  Lane (c, g) of
// warp w, c = lane & 7, g = lane >> 3, multiplies the V block of rows
// 16 w + 4 g .. + 3 and columns 4 c .. + 3 with those rows' x entries of the
// 8 right-hand sides.  Needs n % 4 == 0, kdim % 4 == 0, 16-byte aligned V, X.
constexpr int kVtxStages = 4;
constexpr int kVtxStage = 128 * 32 + 8 * 128;  // floats per stage
constexpr size_t kVtxSmem = sizeof(float) * kVtxStages * kVtxStage;

__global__ void __launch_bounds__(256, 2) k_lr_vtx_cp(const float* V, const float* X, int64_t n,
                                                     int64_t kdim, int64_t R, int64_t rpb,
                                                     double* part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c = lane & 7, g = lane >> 3;
  const int64_t k0 = (int64_t)blockIdx.y * 32, r0 = (int64_t)blockIdx.z * 8;
  const int kw = (int)(kdim - k0 < 32 ? kdim - k0 : 32);
  const int64_t rb0 = (int64_t)blockIdx.x * rpb;
  const int64_t rb1 = rb0 + rpb < n ? rb0 + rpb : n;
  const int nst = rb0 < rb1 ? (int)((rb1 - rb0 + 127) / 128) : 0;
  auto issue = [&](int st) {
    float* vs = sm + (st % kVtxStages) * kVtxStage;
    float* xs = vs + 128 * 32;
    const int64_t i0 = rb0 + (int64_t)st * 128;
    const int rows = (int)(rb1 - i0 < 128 ? rb1 - i0 : 128);
#pragma unroll
    for (int m = 0; m < 4; ++m) {  // 1024 chunks of V: row e >> 3, columns 4 (e & 7) ..
      const int e = tid + 256 * m, row = e >> 3, j = e & 7;
      const bool ok = row < rows && 4 * j < kw;
      cp_async16(vs + row * 32 + 4 * j, ok ? V + (i0 + row) * kdim + k0 + 4 * j : V, ok ? 16 : 0);
    }
    {  // 256 chunks of X: right-hand side tid >> 5, rows 4 (tid & 31) ..
      const int q = tid >> 5, j = tid & 31;
      const bool ok = 4 * j < rows && r0 + q < R;
      cp_async16(xs + q * 128 + 4 * j, ok ? X + (r0 + q) * n + i0 + 4 * j : X, ok ? 16 : 0);
    }
  };
  float acc[4][8];
#pragma unroll
  for (int e = 0; e < 4; ++e)
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[e][q] = 0.f;
#pragma unroll
  for (int st = 0; st < kVtxStages - 1; ++st) {
    if (st < nst) issue(st);
    cp_async_commit();
  }
  const int rr = warp * 16 + 4 * g;
  for (int st = 0; st < nst; ++st) {
    cp_async_wait<kVtxStages - 2>();
    __syncthreads();  // stage st landed for every thread; stage st - 1's slot is free
    if (st + kVtxStages - 1 < nst) issue(st + kVtxStages - 1);
    cp_async_commit();
    const float* vs = sm + (st % kVtxStages) * kVtxStage;
    const float* xs = vs + 128 * 32;
    float4 v[4], x[8];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = *reinterpret_cast<const float4*>(vs + (rr + u) * 32 + 4 * c);
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = *reinterpret_cast<const float4*>(xs + q * 128 + rr);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float xq[4] = {x[q].x, x[q].y, x[q].z, x[q].w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        acc[0][q] = fmaf(v[u].x, xq[u], acc[0][q]);
        acc[1][q] = fmaf(v[u].y, xq[u], acc[1][q]);
        acc[2][q] = fmaf(v[u].z, xq[u], acc[2][q]);
        acc[3][q] = fmaf(v[u].w, xq[u], acc[3][q]);
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  // the 4 row quads of a warp (shuffles), then the 8 warps in a fixed order
  double* sh = reinterpret_cast<double*>(smem_raw);  // [8 warps][32 columns][8]
#pragma unroll
  for (int e = 0; e < 4; ++e)
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      double a = (double)acc[e][q];
      a += __shfl_xor_sync(0xffffffffu, a, 8);
      a += __shfl_xor_sync(0xffffffffu, a, 16);
      if (g == 0) sh[(warp * 32 + 4 * c + e) * 8 + q] = a;
    }
  __syncthreads();
  {
    const int kc = tid >> 3, q = tid & 7;
    double sum = 0.0;
#pragma unroll
    for (int w = 0; w < 8; ++w) sum += sh[(w * 32 + kc) * 8 + q];
    if (k0 + kc < kdim && r0 + q < R) part[((int64_t)blockIdx.x * kdim + k0 + kc) * R + r0 + q] = sum;
  }
}

template <typename T>
__global__ void k_lr_final(const double* part, int nblk, int64_t cnt, T* W) {
  // one warp per output: lane l sums blocks l, l + 32, ...; then a fixed
  // shuffle tree (run-to-run deterministic)
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= cnt) return;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += part[(int64_t)b * cnt + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) W[i] = (T)s;
}

// Y[r, i] = coeff sum_k Ut[k, i] W[k, r] + beta Y[r, i] from the transposed
// low-rank factor (k x n): thread i reads column i of Ut, so every load of a
// warp is one coalesced row segment; W in shared memory.
template <typename T>
__global__ void __launch_bounds__(256) k_lr_uw_t(const T* Ut, const T* W, T* Y, int64_t n,
                                                 int kdim, int64_t R, T coeff, T beta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ws = reinterpret_cast<T*>(smem_raw);
  for (int64_t e = threadIdx.x; e < kdim * R; e += blockDim.x) Ws[e] = W[e];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t r0 = 0; r0 < R; r0 += 8) {
      T acc[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = T(0);
#pragma unroll 8
      for (int k = 0; k < kdim; ++k) {
        const T u = __ldg(Ut + (int64_t)k * n + i);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (r0 + q < R) acc[q] = fma(u, Ws[k * R + r0 + q], acc[q]);
      }
      // every load of the group's old y before its stores
      T yo[8];
#pragma unroll
      for (int q = 0; q < 8; ++q)
        yo[q] = (beta != T(0) && r0 + q < R) ? Y[(r0 + q) * n + i] : T(0);
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (r0 + q < R) Y[(r0 + q) * n + i] = coeff * acc[q] + beta * yo[q];
    }
  }
}

// FP32 form of k_lr_uw_t with four consecutive outputs per thread: 16-byte
// loads of the rows of Ut and of Y, 16 rows of Ut in flight per thread, W in
// shared memory as
// [group of 8 right-hand sides][k][8] (zero-padded) for 16-byte broadcasts.
__global__ void __launch_bounds__(256, 2) k_lr_uw_t4(const float* Ut, const float* W, float* Y,
                                                    int64_t n, int kdim, int64_t R, float coeff,
                                                    float beta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Ws = reinterpret_cast<float*>(smem_raw);
  const int64_t ngr = (R + 7) / 8;
  for (int64_t e = threadIdx.x; e < ngr * kdim * 8; e += blockDim.x) {
    const int64_t q = e & 7, k = (e >> 3) % kdim, rg = (e >> 3) / kdim;
    Ws[e] = rg * 8 + q < R ? W[k * R + rg * 8 + q] : 0.f;
  }
  __syncthreads();
  const int64_t n4 = n / 4;
  for (int64_t i4 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i4 < n4;
       i4 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = 4 * i4;
    for (int64_t rg = 0; rg < ngr; ++rg) {
      const int64_t r0 = rg * 8;
      const float* wg = Ws + rg * kdim * 8;
      float4 acc[8], yo[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int kb = 0; kb < kdim; kb += 16) {
        float4 u[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)
          u[j] = kb + j < kdim ? __ldg(reinterpret_cast<const float4*>(Ut + (int64_t)(kb + j) * n + i))
                               : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          if (kb + j >= kdim) break;
          const float4 wa = *reinterpret_cast<const float4*>(wg + (kb + j) * 8);
          const float4 wb = *reinterpret_cast<const float4*>(wg + (kb + j) * 8 + 4);
          const float w[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            acc[q].x = fmaf(u[j].x, w[q], acc[q].x);
            acc[q].y = fmaf(u[j].y, w[q], acc[q].y);
            acc[q].z = fmaf(u[j].z, w[q], acc[q].z);
            acc[q].w = fmaf(u[j].w, w[q], acc[q].w);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q)
        yo[q] = (beta != 0.0f && r0 + q < R) ? *reinterpret_cast<const float4*>(Y + (r0 + q) * n + i)
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (r0 + q >= R) break;
        float4 v;
        v.x = fmaf(coeff, acc[q].x, beta * yo[q].x);
        v.y = fmaf(coeff, acc[q].y, beta * yo[q].y);
        v.z = fmaf(coeff, acc[q].z, beta * yo[q].z);
        v.w = fmaf(coeff, acc[q].w, beta * yo[q].w);
        *reinterpret_cast<float4*>(Y + (r0 + q) * n + i) = v;
      }
    }
  }
}

// Transpose of an n x k row-major matrix into k x n (32 x 32 shared tiles).
template <typename T>
__global__ void k_transpose_nk(const T* src, T* dst, int64_t n, int64_t k) {
  __shared__ T tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int r = ty; r < 32; r += 8) {
    const int64_t i = i0 + r, kk = k0 + tx;
    tile[r][tx] = (i < n && kk < k) ? src[i * k + kk] : T(0);
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t kk = k0 + r, i = i0 + tx;
    if (kk < k && i < n) dst[kk * n + i] = tile[tx][r];
  }
}

// k_lr_uw with the block's 256 rows of U staged in shared memory by
// coalesced loads (row stride kdim + 1 against bank conflicts): thread t then
// forms row t of Y from shared memory.
template <typename T>
__global__ void __launch_bounds__(256) k_lr_uw_staged(const T* U, const T* W, T* Y, int64_t n,
                                                      int kdim, int64_t R, T coeff, T beta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ws = reinterpret_cast<T*>(smem_raw);
  T* Us = Ws + (size_t)kdim * R;
  const int ld = kdim + 1;
  for (int64_t e = threadIdx.x; e < kdim * R; e += blockDim.x) Ws[e] = W[e];
  for (int64_t i0 = (int64_t)blockIdx.x * 256; i0 < n; i0 += (int64_t)gridDim.x * 256) {
    const int rows = (int)((n - i0 < 256) ? (n - i0) : 256);
    __syncthreads();
    const T* src = U + i0 * kdim;
    for (int e = threadIdx.x; e < rows * kdim; e += blockDim.x)
      Us[(e / kdim) * ld + (e % kdim)] = __ldg(src + e);
    __syncthreads();
    const int t = threadIdx.x;
    if (t < rows) {
      const T* ur = Us + t * ld;
      for (int64_t r0 = 0; r0 < R; r0 += 8) {
        T acc[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = T(0);
        for (int k = 0; k < kdim; ++k) {
          const T u = ur[k];
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (r0 + q < R) acc[q] = fma(u, Ws[k * R + r0 + q], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (r0 + q >= R) break;
          T* y = Y + (r0 + q) * n + i0 + t;
          T v = coeff * acc[q];
          if (beta != T(0)) v += beta * *y;
          *y = v;
        }
      }
    }
  }
}

// Y[r, i] = coeff * sum_k U[i, k] W[k, r] + beta Y[r, i]; W staged in shared memory.
template <typename T>
__global__ void k_lr_uw(const T* U, const T* W, T* Y, int64_t n, int64_t kdim, int64_t R,
                        T coeff, T beta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ws = reinterpret_cast<T*>(smem_raw);
  for (int64_t i = threadIdx.x; i < kdim * R; i += blockDim.x) Ws[i] = W[i];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t r0 = 0; r0 < R; r0 += 8) {
      T acc[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = T(0);
      for (int64_t k = 0; k < kdim; ++k) {
        const T u = U[i * kdim + k];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (r0 + q < R) acc[q] = fma(u, Ws[k * R + r0 + q], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (r0 + q >= R) break;
        T* y = Y + (r0 + q) * n + i;
        T v = coeff * acc[q];
        if (beta != T(0)) v += beta * *y;
        *y = v;
      }
    }
  }
}

template <typename T>
__global__ void k_lr_grad(const T* A, const T* W, T* G, int64_t n, int64_t kdim, int64_t R,
                          T scale) {
  const int64_t tot = n * kdim;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / kdim, k = e % kdim;
    T s = T(0);
    for (int64_t r = 0; r < R; ++r) s = fma(A[r * n + i], W[k * R + r], s);
    G[e] += scale * s;
  }
}

template <typename T>
__global__ void k_rowsum_prod(const T* U, const T* V, T* out, int64_t n, int64_t kdim, T coeff,
                              T beta) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T s = T(0);
    for (int64_t k = 0; k < kdim; ++k) s = fma(U[i * kdim + k], V[i * kdim + k], s);
    T v = coeff * s;
    if (beta != T(0)) v += beta * out[i];
    out[i] = v;
  }
}

template <typename T>
struct FacP {
  int nf;
  int64_t n[8];
  int64_t st[8];
  int64_t ld[8];
  const T* f[8];
};

template <typename T>
__global__ void k_kron_diag(FacP<T> p, T* out, int64_t N, T coeff, T beta, int sum_mode) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N;
       idx += (int64_t)gridDim.x * blockDim.x) {
    T v = sum_mode ? T(0) : T(1);
    for (int k = 0; k < p.nf; ++k) {
      const int64_t ik = (idx / p.st[k]) % p.n[k];
      const T d = p.f[k][ik * p.ld[k] + ik];
      v = sum_mode ? v + d : v * d;
    }
    v *= coeff;
    if (beta != T(0)) v += beta * out[idx];
    out[idx] = v;
  }
}

template <typename T>
__global__ void k_diag_grad_vec(const T* U, const T* X, T* G, int64_t n, int64_t R, T scale) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T s = T(0);
    for (int64_t r = 0; r < R; ++r) s = fma(U[r * n + i], X[r * n + i], s);
    G[i] += scale * s;
  }
}

template <typename T>
__global__ void k_add_scalar(T* G, const double* v, double scale) {
  if (threadIdx.x == 0 && blockIdx.x == 0) G[0] += (T)(scale * v[0]);
}

template <typename T>
__global__ void k_permute_front(const T* X, T* Y, int64_t RA, int64_t n, int64_t C) {
  const int64_t tot = RA * n * C;
  for (int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; o < tot;
       o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = o / (RA * C);
    const int64_t rem = o % (RA * C);
    const int64_t ra = rem / C, c = rem % C;
    Y[o] = X[(ra * n + j) * C + c];
  }
}

template <typename T>
__global__ void k_add_partials(const T* P, T* G, int64_t count, int64_t nparts, T scale) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    T s = T(0);
    for (int64_t p = 0; p < nparts; ++p) s += P[p * count + i];
    G[i] += scale * s;
  }
}

}  // namespace

// =================================================================== hosts

template <typename T>
void gemm(Ctx* c, int64_t M, int64_t N, int64_t K, double alpha, const T* A, int64_t lda_m,
          int64_t lda_k, int64_t sA, const T* B, int64_t ldb_k, int64_t ldb_n, int64_t sB,
          double beta, T* C, int64_t ldc_m, int64_t ldc_n, int64_t sC, int64_t batch) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  GemmP<T> g{M, N, K, A, lda_m, lda_k, sA, B, ldb_k, ldb_n, sB, C, ldc_m, ldc_n, sC,
             (T)alpha, (T)beta};
  const int64_t gy = (N + 127) / 128;
  COLA_REQUIRE(gy <= 65535, COLA_ERR_UNSUPPORTED, "gemm: N=%lld too large", (long long)N);
  auto a16 = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
  const bool mode_f32 = std::is_same<T, float>::value && lda_m == 1 && ldb_k == 1 &&
                        ldc_n == 1 && M % 4 == 0 && N % 4 == 0 && lda_k % 4 == 0 &&
                        ldb_n % 4 == 0 && ldc_m % 4 == 0 && sA % 4 == 0 && sB % 4 == 0 &&
                        sC % 4 == 0 && a16(A) && a16(B) && a16(C);
  // a product that fills fewer than a quarter of the SMs with 128 x 128 tiles
  // runs one output per thread instead
  const int64_t tiles = (M + 127) / 128 * gy * batch;
  const int64_t total = M * N * batch;
  if (tiles * 4 < c->num_sms && total <= ((int64_t)1 << 24)) {
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 65535);
    k_gemm_small<T><<<grid, 256, 0, c->s>>>(g, total);
    c->count_launch();
    COLA_CUDA(cudaGetLastError());
    return;
  }
  if (std::is_same<T, double>::value && (N + 31) / 32 <= 65535) {
    for (int64_t b0 = 0; b0 < batch; b0 += 65535) {
      const int64_t nb = std::min<int64_t>(65535, batch - b0);
      dim3 grid((unsigned)((M + 31) / 32), (unsigned)((N + 31) / 32), (unsigned)nb);
      k_gemm32<T><<<grid, 256, 0, c->s>>>(g, b0);
      c->count_launch();
    }
    COLA_CUDA(cudaGetLastError());
    return;
  }
  for (int64_t b0 = 0; b0 < batch; b0 += 65535) {
    const int64_t nb = std::min<int64_t>(65535, batch - b0);
    dim3 grid((unsigned)((M + 127) / 128), (unsigned)gy, (unsigned)nb);
    if constexpr (std::is_same<T, float>::value) {
      if (mode_f32) {
        k_gemm_mode_f32<<<grid, 256, 0, c->s>>>(g, b0);
        c->count_launch();
        continue;
      }
    }
    k_gemm<T><<<grid, 256, 0, c->s>>>(g, b0);
    c->count_launch();
  }
  COLA_CUDA(cudaGetLastError());
}

template <typename T>
void gemm_grouped(Ctx* c, const GemmDesc<T>* dev_probs, int nprob, int64_t max_m,
                  int64_t max_n) {
  if (nprob <= 0) return;
  COLA_REQUIRE(nprob <= 65535, COLA_ERR_UNSUPPORTED, "grouped gemm: %d problems", nprob);
  if (std::is_same<T, double>::value) {
    dim3 grid((unsigned)((max_m + 31) / 32), (unsigned)((max_n + 31) / 32), (unsigned)nprob);
    k_gemm_grouped32<T><<<grid, 256, 0, c->s>>>(dev_probs);
  } else {
    dim3 grid((unsigned)((max_m + 127) / 128), (unsigned)((max_n + 127) / 128),
              (unsigned)nprob);
    k_gemm_grouped<T><<<grid, 256, 0, c->s>>>(dev_probs);
  }
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
}
template void gemm_grouped<float>(Ctx*, const GemmDesc<float>*, int, int64_t, int64_t);
template void gemm_grouped<double>(Ctx*, const GemmDesc<double>*, int, int64_t, int64_t);

int dot_blocks(int64_t n) {
  const int64_t b = (n + 4095) / 4096;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 256));
}

template <typename T>
void dots(Ctx* c, const T* a, const T* b, int64_t n, int64_t R, double* partials, double* out) {
  const int nb = dot_blocks(n);
  k_dot_partial<T><<<dim3(nb, (unsigned)R), 256, 0, c->s>>>(a, b, n, nb, partials);
  c->count_launch();
  k_dot_final<<<(unsigned)R, 256, 0, c->s>>>(partials, nb, R, out);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
}

void dot_final(Ctx* c, const double* partials, int nblk, int64_t R, double* out) {
  k_dot_final<<<(unsigned)R, 256, 0, c->s>>>(partials, nblk, R, out);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
}

template <typename TI, typename TO>
void convert(Ctx* c, const TI* in, TO* out, int64_t n) {
  if (n <= 0) return;
  k_convert<TI, TO><<<grid_for(n, 4), kThreads, 0, c->s>>>(in, out, n);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
}

template <typename T>
void fill_zero(Ctx* c, T* p, int64_t n) {
  if (n > 0) COLA_CUDA(cudaMemsetAsync(p, 0, sizeof(T) * n, c->s));
}

template <typename T>
void scale_rows(Ctx* c, T* X, int64_t n, int64_t R, const double* w) {
  k_scale_rows<T><<<grid_for(n * R, 4), kThreads, 0, c->s>>>(X, n, R, w);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
}

void rademacher(Ctx* c, uint64_t seed, int64_t offset, int64_t count, void* out,
                cola_dtype dt) {
  if (count <= 0) return;
  if (dt == COLA_F64)
    k_rademacher<double><<<grid_for(count, 4), kThreads, 0, c->s>>>(seed, offset, count,
                                                                      (double*)out);
  else
    k_rademacher<float><<<grid_for(count, 4), kThreads, 0, c->s>>>(seed, offset, count,
                                                                    (float*)out);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
}

template <typename T>
void diag_apply(Ctx* c, const T* d, int64_t stride, const T* X, T* Y, int64_t n, int64_t R,
                double coeff, double beta) {
  k_diag<T><<<grid_for(n * R, 4), kThreads, 0, c->s>>>(d, stride, X, Y, n, R, (T)coeff,
                                                       (T)beta);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
}

template <typename T>
bool stencil_apply(Ctx* c, int nf, const int64_t* sizes, const T* bands, const T* X, T* Y,
                   int64_t R, double coeff, double beta, const T* dg, int64_t dstride,
                   double dcoeff) {
  bool fused = false;
  COLA_REQUIRE(nf >= 1 && nf <= 8, COLA_ERR_UNSUPPORTED, "stencil: %d factors", nf);
  StencilP p{};
  p.nf = nf;
  int64_t N = 1, off = 0;
  for (int k = 0; k < nf; ++k) N *= sizes[k];
  int64_t st = N;
  for (int k = 0; k < nf; ++k) {
    st /= sizes[k];
    p.n[k] = sizes[k];
    p.st[k] = st;
    p.boff[k] = off;
    off += 3 * sizes[k];
  }
  const uintptr_t al = (uintptr_t)X | (uintptr_t)Y | (dg && dstride ? (uintptr_t)dg : 0);
  if (nf == 2 && sizes[1] % 4 == 0 && sizes[0] < (1 << 30) && sizes[1] < (1 << 30) &&
      (al & (4 * sizeof(T) - 1)) == 0) {
    const int64_t tot = sizes[0] * (sizes[1] / 4) * R;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((tot + 255) / 256, 152 * 32));
    fused = dg != nullptr;
    // strips of up to 16 rows while they leave at least 512 threads per SM;
    // shorter strips than 8 rows do not pay for the halo rows and the lane
    // exchanges (a single right-hand side on a 1000^2 grid, 250 k row quads,
    // measured slower than one quad per thread)
    const int64_t quads = R * sizes[0] * (sizes[1] / 4);
    const int S = (int)std::min<int64_t>(kStencilStrip, quads / ((int64_t)c->num_sms * 512));
    if (S >= 8) {
      const int64_t items = R * ((sizes[0] + S - 1) / S) * (sizes[1] / 4);
      const int sgrid =
          (int)std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, 152 * 16));
      k_stencil2s<T><<<sgrid, kThreads, 0, c->s>>>(bands, X, Y, (int)sizes[0], (int)sizes[1],
                                                   R, (T)coeff, (T)beta, dg, dstride, (T)dcoeff,
                                                   S);
    } else {
      k_stencil2<T><<<grid, kThreads, 0, c->s>>>(bands, X, Y, (int)sizes[0], (int)sizes[1], R,
                                                 (T)coeff, (T)beta, dg, dstride, (T)dcoeff);
    }
  } else {
    k_stencil<T><<<grid_for(N * R, 4), kThreads, 0, c->s>>>(p, bands, X, Y, N, R, (T)coeff,
                                                            (T)beta);
  }
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
  return fused;
}

template <typename T>
void lowrank_vtx(Ctx* c, const T* V, const T* X, int64_t n, int64_t k, int64_t R, T* W,
                 double* partials) {
  const uintptr_t al = (uintptr_t)V | (uintptr_t)X;
  int nblk;
  if (sizeof(T) == 4 && n % 4 == 0 && k % 4 == 0 && (al & 15) == 0) {
    // one resident wave (2 blocks per SM), contiguous 128-row stages per block
    static bool attr = false;
    if (!attr) {
      COLA_CUDA(cudaFuncSetAttribute(k_lr_vtx_cp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kVtxSmem));
      attr = true;
    }
    const int64_t nstages = (n + 127) / 128;
    nblk = (int)std::max<int64_t>(1, std::min<int64_t>(nstages, 2 * 152));
    const int64_t rpb = (nstages + nblk - 1) / nblk * 128;
    dim3 grid(nblk, (unsigned)((k + 31) / 32), (unsigned)((R + 7) / 8));
    k_lr_vtx_cp<<<grid, 256, kVtxSmem, c->s>>>((const float*)V, (const float*)X, n, k, R, rpb,
                                              partials);
  } else {
    const int64_t ntiles = (n + 31) / 32;
    nblk = (int)std::max<int64_t>(1, std::min<int64_t>((ntiles + 7) / 8, kLowRankBlocks));
    dim3 grid(nblk, (unsigned)((k + 31) / 32), (unsigned)((R + 7) / 8));
    k_lr_vtx<T><<<grid, 256, 0, c->s>>>(V, X, n, k, R, nblk, partials);
  }
  c->count_launch();
  const int64_t cnt = k * R;
  k_lr_final<T><<<(unsigned)((cnt * 32 + 255) / 256), 256, 0, c->s>>>(partials, nblk, cnt, W);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
}

template <typename T>
void transpose_nk(Ctx* c, const T* src, T* dst, int64_t n, int64_t k) {
  dim3 grid((unsigned)((n + 31) / 32), (unsigned)((k + 31) / 32));
  k_transpose_nk<T><<<grid, 256, 0, c->s>>>(src, dst, n, k);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
}

template <typename T>
void lowrank_uw(Ctx* c, const T* U, const T* W, T* Y, int64_t n, int64_t k, int64_t R,
                double coeff, double beta, const T* Ut) {
  const size_t smem = sizeof(T) * k * R;
  COLA_REQUIRE(smem <= 48 * 1024, COLA_ERR_UNSUPPORTED, "low-rank: k*nrhs too large");
  const uintptr_t al = (uintptr_t)Ut | (uintptr_t)Y;
  const size_t smem4 = sizeof(float) * ((R + 7) / 8) * 8 * k;
  if (Ut && sizeof(T) == 4 && n % 4 == 0 && (al & 15) == 0 && smem4 <= 48 * 1024) {
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n / 4 + 255) / 256, 152 * 8));
    k_lr_uw_t4<<<grid, 256, smem4, c->s>>>((const float*)Ut, (const float*)W, (float*)Y, n,
                                          (int)k, R, (float)coeff, (float)beta);
    c->count_launch();
    COLA_CUDA(cudaGetLastError());
    return;
  }
  if (Ut) {
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
    k_lr_uw_t<T><<<grid, 256, smem, c->s>>>(Ut, W, Y, n, (int)k, R, (T)coeff, (T)beta);
    c->count_launch();
    COLA_CUDA(cudaGetLastError());
    return;
  }
  const size_t smem2 = smem + sizeof(T) * 256 * (k + 1);
  if (smem2 <= 48 * 1024) {
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8));
    k_lr_uw_staged<T><<<grid, 256, smem2, c->s>>>(U, W, Y, n, (int)k, R, (T)coeff, (T)beta);
  } else {
    k_lr_uw<T><<<grid_for(n, 1), kThreads, smem, c->s>>>(U, W, Y, n, k, R, (T)coeff, (T)beta);
  }
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
}

template <typename T>
void lowrank_grad(Ctx* c, const T* A, const T* W, T* G, int64_t n, int64_t k, int64_t R,
                  double scale) {
  k_lr_grad<T><<<grid_for(n * k, 1), kThreads, 0, c->s>>>(A, W, G, n, k, R, (T)scale);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
}

template <typename T>
void rowsum_products(Ctx* c, const T* U, const T* V, T* out, int64_t n, int64_t k,
                     double coeff, double beta) {
  k_rowsum_prod<T><<<grid_for(n, 1), kThreads, 0, c->s>>>(U, V, out, n, k, (T)coeff, (T)beta);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
}

template <typename T>
static void kron_like_diag(Ctx* c, int nf, const int64_t* sizes, const T* const* f,
                           const int64_t* lds, T* out, double coeff, double beta, int sum_mode) {
  COLA_REQUIRE(nf >= 1 && nf <= 8, COLA_ERR_UNSUPPORTED, "diag: %d factors", nf);
  FacP<T> p{};
  p.nf = nf;
  int64_t N = 1;
  for (int k = 0; k < nf; ++k) N *= sizes[k];
  int64_t st = N;
  for (int k = 0; k < nf; ++k) {
    st /= sizes[k];
    p.n[k] = sizes[k];
    p.st[k] = st;
    p.ld[k] = lds[k];
    p.f[k] = f[k];
  }
  k_kron_diag<T><<<grid_for(N, 4), kThreads, 0, c->s>>>(p, out, N, (T)coeff, (T)beta, sum_mode);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
}

template <typename T>
void kron_diag(Ctx* c, int nf, const int64_t* sizes, const T* const* f, const int64_t* lds,
               T* out, double coeff, double beta) {
  kron_like_diag(c, nf, sizes, f, lds, out, coeff, beta, 0);
}

template <typename T>
void kronsum_diag(Ctx* c, int nf, const int64_t* sizes, const T* const* f, const int64_t* lds,
                  T* out, double coeff, double beta) {
  kron_like_diag(c, nf, sizes, f, lds, out, coeff, beta, 1);
}

template <typename T>
void diag_grad(Ctx* c, const T* U, const T* X, T* G, int64_t n, int64_t R, double scale,
               bool scalar, double* partials) {
  if (scalar) {
    double* out = partials + (int64_t)dot_blocks(n * R);
    dots<T>(c, U, X, n * R, 1, partials, out);
    k_add_scalar<T><<<1, 32, 0, c->s>>>(G, out, scale);
    c->count_launch();
  } else {
    k_diag_grad_vec<T><<<grid_for(n, 1), kThreads, 0, c->s>>>(U, X, G, n, R, (T)scale);
    c->count_launch();
  }
  COLA_CUDA(cudaGetLastError());
}

template <typename T>
void permute_mode_front(Ctx* c, const T* X, T* Y, int64_t R, int64_t A, int64_t n, int64_t C) {
  k_permute_front<T><<<grid_for(R * A * n * C, 4), kThreads, 0, c->s>>>(X, Y, R * A, n, C);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
}

template <typename T>
void add_partials(Ctx* c, const T* P, T* G, int64_t count, int64_t nparts, double scale) {
  k_add_partials<T><<<grid_for(count, 1), kThreads, 0, c->s>>>(P, G, count, nparts, (T)scale);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
}

#define COLA_INST(T)                                                                        \
  template void gemm<T>(Ctx*, int64_t, int64_t, int64_t, double, const T*, int64_t, int64_t, \
                        int64_t, const T*, int64_t, int64_t, int64_t, double, T*, int64_t,   \
                        int64_t, int64_t, int64_t);                                         \
  template void dots<T>(Ctx*, const T*, const T*, int64_t, int64_t, double*, double*);      \
  template void fill_zero<T>(Ctx*, T*, int64_t);                                            \
  template void scale_rows<T>(Ctx*, T*, int64_t, int64_t, const double*);                   \
  template void diag_apply<T>(Ctx*, const T*, int64_t, const T*, T*, int64_t, int64_t,      \
                              double, double);                                              \
  template bool stencil_apply<T>(Ctx*, int, const int64_t*, const T*, const T*, T*, int64_t, \
                                 double, double, const T*, int64_t, double);                \
  template void lowrank_vtx<T>(Ctx*, const T*, const T*, int64_t, int64_t, int64_t, T*,     \
                               double*);                                                    \
  template void lowrank_uw<T>(Ctx*, const T*, const T*, T*, int64_t, int64_t, int64_t,      \
                              double, double, const T*);                                    \
  template void transpose_nk<T>(Ctx*, const T*, T*, int64_t, int64_t);                      \
  template void lowrank_grad<T>(Ctx*, const T*, const T*, T*, int64_t, int64_t, int64_t,    \
                                double);                                                    \
  template void rowsum_products<T>(Ctx*, const T*, const T*, T*, int64_t, int64_t, double,  \
                                   double);                                                 \
  template void kron_diag<T>(Ctx*, int, const int64_t*, const T* const*, const int64_t*, T*, \
                             double, double);                                               \
  template void kronsum_diag<T>(Ctx*, int, const int64_t*, const T* const*, const int64_t*, \
                                T*, double, double);                                        \
  template void diag_grad<T>(Ctx*, const T*, const T*, T*, int64_t, int64_t, double, bool,  \
                             double*);                                                      \
  template void permute_mode_front<T>(Ctx*, const T*, T*, int64_t, int64_t, int64_t,        \
                                      int64_t);                                             \
  template void add_partials<T>(Ctx*, const T*, T*, int64_t, int64_t, double);

COLA_INST(float)
COLA_INST(double)
template void convert<double, float>(Ctx*, const double*, float*, int64_t);
template void convert<float, double>(Ctx*, const float*, double*, int64_t);
template void convert<float, float>(Ctx*, const float*, float*, int64_t);
template void convert<double, double>(Ctx*, const double*, double*, int64_t);

}  // namespace cola
