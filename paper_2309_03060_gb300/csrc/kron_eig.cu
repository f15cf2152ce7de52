// Structured solve and log-determinant of shifted Kronecker products and
// Kronecker sums from the eigendecompositions of their factors (Table 3: the
// inverse and the eigendecomposition of a Kronecker product or sum are built
// from the factors'; Sec. 3.2 composition rules; App. A.1.2).  For
//     A = c_k (K_1 (x) ... (x) K_d) + c_d s I,   K_k = V_k diag(lambda_k) V_k^T,
// the eigenvectors of A are (x)_k V_k and its eigenvalues c_k prod_k lambda_k[i_k] + c_d s, so
//     A^-1 B     = ((x)_k V_k) diag(1 / (c_k prod lambda + c_d s)) ((x)_k V_k)^T B,
//     log det A  = sum over all index tuples of log(c_k prod lambda + c_d s).
// A Kronecker sum K_1 (+) ... (+) K_d has the same eigenvectors and the
// eigenvalues sum_k lambda_k[i_k]: the same code with a sum in place of the
// product.
// The factor eigendecompositions are computed once on the host in FP64 and
// cached on the factor (recomputed when its contents change); the solve is
// 2 d cyclic mode products plus one diagonal scaling on the GPU.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace cola {

namespace {

// Symmetric eigendecomposition on the host (FP64): Householder reduction to
// tridiagonal form, then implicit symmetric QR steps with Wilkinson shifts and
// deflation (Golub & Van Loan, Sec. 8.3), every reflection and rotation
// applied to the accumulated orthogonal factor.  a: n x n row-major,
// symmetric (destroyed).  Vt: n x n row-major, row j = the eigenvector of w[j].
// Returns false when the QR sweeps did not converge within 60 n iterations.
bool sym_eig(int n, double* a, double* Vt, double* w) {
  for (int i = 0; i < n * n; ++i) Vt[i] = 0.0;
  for (int i = 0; i < n; ++i) Vt[(size_t)i * n + i] = 1.0;
  std::vector<double> v(n), p(n), q(n), u(n);
  // T = H_{n-3} ... H_0 A H_0 ... H_{n-3}; Vt accumulates H_{n-3} ... H_0
  for (int k = 0; k + 2 < n; ++k) {
    double sig = 0.0;
    for (int i = k + 1; i < n; ++i) sig += a[(size_t)i * n + k] * a[(size_t)i * n + k];
    if (sig == 0.0) continue;
    const double x0 = a[(size_t)(k + 1) * n + k];
    const double alpha = x0 > 0.0 ? -sqrt(sig) : sqrt(sig);
    std::fill(v.begin(), v.end(), 0.0);
    v[k + 1] = x0 - alpha;
    for (int i = k + 2; i < n; ++i) v[i] = a[(size_t)i * n + k];
    double vv = 0.0;
    for (int i = k + 1; i < n; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    const double beta = 2.0 / vv;
    // H A H = A - v q^T - q v^T with p = beta A v, q = p - (beta p.v / 2) v
    for (int i = k; i < n; ++i) {
      double s = 0.0;
      for (int j = k + 1; j < n; ++j) s += a[(size_t)i * n + j] * v[j];
      p[i] = beta * s;
    }
    double pv = 0.0;
    for (int i = k + 1; i < n; ++i) pv += p[i] * v[i];
    const double half = 0.5 * beta * pv;
    for (int i = k; i < n; ++i) q[i] = p[i] - half * v[i];
    for (int i = k; i < n; ++i)
      for (int j = k; j < n; ++j) a[(size_t)i * n + j] -= v[i] * q[j] + q[i] * v[j];
    // Vt <- H Vt: rows k+1.. change by -beta v_i (v^T Vt)
    std::fill(u.begin(), u.end(), 0.0);
    for (int i = k + 1; i < n; ++i)
      for (int j = 0; j < n; ++j) u[j] += v[i] * Vt[(size_t)i * n + j];
    for (int i = k + 1; i < n; ++i) {
      const double f = beta * v[i];
      for (int j = 0; j < n; ++j) Vt[(size_t)i * n + j] -= f * u[j];
    }
  }
  // tridiagonal T: diagonal d, sub-diagonal e
  std::vector<double> d(n), e(n, 0.0);
  for (int i = 0; i < n; ++i) d[i] = a[(size_t)i * n + i];
  for (int i = 0; i + 1 < n; ++i) e[i] = a[(size_t)(i + 1) * n + i];
  const double eps = 2.220446049250313e-16;
  int hi = n - 1, it = 0;
  while (hi > 0 && it < 60 * n) {
    if (fabs(e[hi - 1]) <= eps * (fabs(d[hi - 1]) + fabs(d[hi]))) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && fabs(e[lo - 1]) > eps * (fabs(d[lo - 1]) + fabs(d[lo]))) --lo;
    ++it;
    // Wilkinson shift from the trailing 2 x 2 block, then chase the bulge down
    const double dd = 0.5 * (d[hi - 1] - d[hi]), bb = e[hi - 1];
    const double sg = dd >= 0.0 ? 1.0 : -1.0;
    const double mu = d[hi] - bb * bb / (dd + sg * hypot(dd, bb));
    double x = d[lo] - mu, z = e[lo];
    for (int k = lo; k < hi; ++k) {
      const double r = hypot(x, z);
      const double c = x / r, s = z / r;
      if (k > lo) e[k - 1] = r;
      const double ak = d[k], ak1 = d[k + 1], bk = e[k];
      d[k] = c * c * ak + 2.0 * c * s * bk + s * s * ak1;
      d[k + 1] = s * s * ak - 2.0 * c * s * bk + c * c * ak1;
      e[k] = c * s * (ak1 - ak) + (c * c - s * s) * bk;
      double* r0 = Vt + (size_t)k * n;
      double* r1 = Vt + (size_t)(k + 1) * n;
      for (int j = 0; j < n; ++j) {
        const double v0 = r0[j], v1 = r1[j];
        r0[j] = c * v0 + s * v1;
        r1[j] = -s * v0 + c * v1;
      }
      if (k < hi - 1) {
        x = e[k];
        z = s * e[k + 1];
        e[k + 1] = c * e[k + 1];
      }
    }
  }
  for (int i = 0; i < n; ++i) w[i] = d[i];
  return hi <= 0;
}

constexpr int kMaxFactors = 8;
constexpr int kKeyVt64 = 400, kKeyLam64 = 401, kKeyVt32 = 402;

struct EigDims {
  int d;
  int sum;  // 1: Kronecker sum (eigenvalues add), 0: Kronecker product (multiply)
  int64_t n[kMaxFactors];
  const double* lam[kMaxFactors];
};

// Eigenvalue of A at flat (row-major) index i.
__device__ __forceinline__ double eig_at(const EigDims& g, int64_t i, double ck, double shift) {
  double v = g.sum ? 0.0 : 1.0;
  for (int k = g.d - 1; k >= 0; --k) {
    const int64_t nk = g.n[k];
    const double l = g.lam[k][i % nk];
    v = g.sum ? v + l : v * l;
    i /= nk;
  }
  return ck * v + shift;
}

// Y[r, i] /= lambda_A(i).  The shift c_d s is read from the device scalar.
template <typename T>
__global__ void k_eig_scale(T* Y, int64_t N, int64_t R, EigDims g, double ck, const double* s,
                            double cd) {
  const double shift = s ? cd * s[0] : 0.0;
  const int64_t tot = N * R;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x)
    Y[e] = (T)((double)Y[e] / eig_at(g, e % N, ck, shift));
}

// out[i] = lambda_A(i) for every flat index (the eigenvalues of A in the
// order of the Kronecker eigenvectors (x)_k V_k).
__global__ void k_eig_values(int64_t N, EigDims g, double ck, const double* s, double cd,
                             double* out) {
  const double shift = s ? cd * s[0] : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = eig_at(g, i, ck, shift);
}

// V[i, j] = Vt[j, i] for an n x n row-major matrix.
__global__ void k_transpose64(int64_t n, const double* Vt, double* V) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / n, j = t % n;
    V[t] = Vt[j * n + i];
  }
}

// Per-block partial sums of log lambda_A(i); nonpos[b] counts lambda <= 0.
__global__ void k_eig_logdet(int64_t N, EigDims g, double ck, const double* s, double cd,
                             double* part, int* nonpos) {
  __shared__ double sh[32];
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  const double shift = s ? cd * s[0] : 0.0;
  double acc = 0.0;
  int nb = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double l = eig_at(g, i, ck, shift);
    if (l > 0.0)
      acc += log(l);
    else
      ++nb;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  if (nb) atomicAdd(&bad, nb);
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    part[blockIdx.x] = t;
    nonpos[blockIdx.x] = bad;
  }
}

// Contents fingerprint of an n x n factor (leading dimension ld) on the
// device: the sum mod 2^64 of a 64-bit mix (the SplitMix64 finaliser) of each
// entry's bits salted with its index.  The sum is order-independent, so the
// result is deterministic under any reduction order.
__device__ __forceinline__ unsigned long long fp_mix(unsigned long long z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T>
__global__ void k_fingerprint(const T* a, int64_t n, int64_t ld, unsigned long long* out) {
  unsigned long long acc = 0;
  const int64_t tot = n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x) {
    const T v = a[(e / n) * ld + e % n];
    unsigned long long bits;
    if (sizeof(T) == 8)
      bits = (unsigned long long)__double_as_longlong((double)v);
    else
      bits = (unsigned long long)__float_as_uint((float)v);
    acc += fp_mix(bits ^ ((unsigned long long)e * 0x9E3779B97F4A7C15ull));
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

uint64_t factor_fingerprint(Ctx* c, const cola_linop* f) {
  unsigned long long* d = (unsigned long long*)c->ws.get("keig.fp", 8);
  COLA_CUDA(cudaMemsetAsync(d, 0, 8, c->s));
  const int64_t n = f->rows;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n * n + 255) / 256, 2 * c->num_sms));
  if (f->dtype == COLA_F64)
    k_fingerprint<double><<<grid, 256, 0, c->s>>>((const double*)f->data, n, f->ld, d);
  else
    k_fingerprint<float><<<grid, 256, 0, c->s>>>((const float*)f->data, n, f->ld, d);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
  unsigned long long h = 0;
  COLA_CUDA(cudaMemcpyAsync(&h, d, 8, cudaMemcpyDeviceToHost, c->s));
  COLA_CUDA(cudaStreamSynchronize(c->s));
  return (uint64_t)h ^ ((uint64_t)n << 1) ^ (f->dtype == COLA_F64 ? 1u : 0u);
}

void* eig_buf(cola_linop* f, int key, size_t bytes) {
  auto it = f->derived.find(key);
  if (it != f->derived.end() && it->second.bytes >= bytes) return it->second.p;
  if (it != f->derived.end()) {
    cudaFree(it->second.p);
    f->derived.erase(it);
  }
  void* p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(bytes, 256)) != cudaSuccess) {
    cudaGetLastError();
    fail(COLA_ERR_OOM, "eigendecomposition buffer of %zu bytes", bytes);
  }
  f->derived[key] = Buf{p, bytes};
  return p;
}

// The operator's parts: the Kronecker product or sum node, c_k, and the
// optional scalar shift.
struct KronShift {
  const cola_linop* kron = nullptr;  // LK_KRON or LK_KRONSUM
  bool sum = false;
  double ck = 1.0, cd = 0.0;
  const cola_linop* diag = nullptr;
};

inline bool is_kron_node(const cola_linop* op) {
  return op->kind == LK_KRON || op->kind == LK_KRONSUM;
}

// Fills m when op is Kron/KronSum or Kron/KronSum + scalar Diag; false otherwise.
bool try_match(const cola_linop* op, KronShift& m) {
  m = KronShift{};
  if (is_kron_node(op)) {
    m.kron = op;
  } else if (op->kind == LK_SUM && op->kids.size() == 2) {
    for (int i = 0; i < 2; ++i) {
      const cola_linop* k = op->kids[i];
      if (is_kron_node(k)) {
        m.kron = k;
        m.ck = op->coeffs[i];
      } else if (k->kind == LK_DIAG && k->stride == 0) {
        m.diag = k;
        m.cd = op->coeffs[i];
      }
    }
    if (!m.kron || !m.diag) m.kron = nullptr;
  }
  if (!m.kron || (int)m.kron->kids.size() > kMaxFactors) return false;
  for (auto* f : m.kron->kids)
    if (f->kind != LK_DENSE || f->rows != f->cols) return false;
  m.sum = m.kron->kind == LK_KRONSUM;
  return true;
}

KronShift match(const cola_linop* op) {
  KronShift m;
  try_match(op, m);
  COLA_REQUIRE(m.kron, COLA_ERR_UNSUPPORTED,
               "the eigen-structured path takes Kron/KronSum(K_1..K_d) [+ scalar * I]");
  COLA_REQUIRE((int)m.kron->kids.size() <= kMaxFactors, COLA_ERR_UNSUPPORTED,
               "at most %d Kronecker factors", kMaxFactors);
  for (auto* f : m.kron->kids)
    COLA_REQUIRE(f->kind == LK_DENSE && f->rows == f->cols, COLA_ERR_UNSUPPORTED,
                 "the eigen-structured path takes square dense factors");
  return m;
}

// Factor eigendecompositions on the device (FP64 Vt and lambda, FP32 Vt),
// recomputed only when a factor's contents change: a device fingerprint of
// each distinct factor is compared with the one the cached decomposition was
// made from, and only a changed factor is read back and decomposed.
void prepare_eig(Ctx* c, const KronShift& m, bool want32) {
  std::vector<const cola_linop*> seen;
  for (auto* fc : m.kron->kids) {
    if (std::find(seen.begin(), seen.end(), fc) != seen.end()) continue;
    seen.push_back(fc);
    cola_linop* f = const_cast<cola_linop*>(fc);
    const int64_t n = f->rows;
    const uint64_t h = factor_fingerprint(c, f);
    if (f->eig_hash == h && f->derived.count(kKeyVt64) && f->derived.count(kKeyLam64) &&
        f->derived.count(kKeyVt32))
      continue;
    std::vector<double> A((size_t)n * n);
    if (f->dtype == COLA_F64) {
      COLA_CUDA(cudaMemcpy2DAsync(A.data(), n * 8, f->data, f->ld * 8, n * 8, n,
                                  cudaMemcpyDeviceToHost, c->s));
      COLA_CUDA(cudaStreamSynchronize(c->s));
    } else {
      std::vector<float> Af((size_t)n * n);
      COLA_CUDA(cudaMemcpy2DAsync(Af.data(), n * 4, f->data, f->ld * 4, n * 4, n,
                                  cudaMemcpyDeviceToHost, c->s));
      COLA_CUDA(cudaStreamSynchronize(c->s));
      for (size_t i = 0; i < A.size(); ++i) A[i] = Af[i];
    }
    double amax = 0.0, asym = 0.0;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) {
        amax = std::max(amax, fabs(A[(size_t)i * n + j]));
        asym = std::max(asym, fabs(A[(size_t)i * n + j] - A[(size_t)j * n + i]));
      }
    COLA_REQUIRE(asym <= 1e-12 * amax, COLA_ERR_INVALID_ARG,
                 "Kronecker factor is not symmetric (max |K - K^T| = %g)", asym);
    std::vector<double> Vt((size_t)n * n), lam(n);
    COLA_REQUIRE(sym_eig((int)n, A.data(), Vt.data(), lam.data()), COLA_ERR_NOT_CONVERGED,
                 "symmetric QR of a %lld x %lld Kronecker factor did not converge",
                 (long long)n, (long long)n);
    void* dv = eig_buf(f, kKeyVt64, (size_t)n * n * 8);
    void* dl = eig_buf(f, kKeyLam64, (size_t)n * 8);
    COLA_CUDA(cudaMemcpyAsync(dv, Vt.data(), (size_t)n * n * 8, cudaMemcpyHostToDevice, c->s));
    COLA_CUDA(cudaMemcpyAsync(dl, lam.data(), (size_t)n * 8, cudaMemcpyHostToDevice, c->s));
    std::vector<float> V32(Vt.begin(), Vt.end());
    void* d32 = eig_buf(f, kKeyVt32, (size_t)n * n * 4);
    COLA_CUDA(cudaMemcpyAsync(d32, V32.data(), (size_t)n * n * 4, cudaMemcpyHostToDevice, c->s));
    COLA_CUDA(cudaStreamSynchronize(c->s));  // host vectors go out of scope
    f->eig_hash = h;
  }
  (void)want32;
}

EigDims dims_of(const KronShift& m) {
  EigDims g{};
  g.d = (int)m.kron->kids.size();
  g.sum = m.sum ? 1 : 0;
  for (int k = 0; k < g.d; ++k) {
    const cola_linop* f = m.kron->kids[k];
    g.n[k] = f->rows;
    g.lam[k] = (const double*)f->derived.at(kKeyLam64).p;
  }
  return g;
}

// Y = ((x)_k F_k) X by cyclic mode products with F_k = Vt_k (tr = false) or
// Vt_k^T = V_k (tr = true); intermediates in two workspace buffers.
template <typename T>
void eig_modes(Ctx* c, const KronShift& m, bool tr, const T* X, T* Y, int64_t R) {
  const int d = (int)m.kron->kids.size();
  const int64_t N = m.kron->rows;
  const int key = sizeof(T) == 8 ? kKeyVt64 : kKeyVt32;
  T* t[2] = {(T*)c->ws.get("keig.t0", sizeof(T) * N * R),
             (T*)c->ws.get("keig.t1", sizeof(T) * N * R)};
  const T* cur = X;
  for (int k = 0; k < d; ++k) {
    const cola_linop* f = m.kron->kids[k];
    const int64_t n = f->rows, rest = N / n;
    const T* F = (const T*)f->derived.at(key).p;
    T* dst = (k == d - 1) ? Y : t[k & 1];
    // B[j][i] = F_op[i][j], F_op = tr ? F^T : F (F row-major n x n)
    gemm<T>(c, rest, n, n, 1.0, cur, 1, rest, N, F, tr ? n : 1, tr ? 1 : n, 0, 0.0, dst, n, 1, N,
            R);
    cur = dst;
  }
}

// X = (c_k Kron + cd s[0] I)^-1 B with s a device scalar (or none).
template <typename T>
void eig_solve(Ctx* c, const KronShift& m, const double* s, double cd, const T* B, T* X,
               int64_t R) {
  const int64_t N = m.kron->rows;
  T* mid = (T*)c->ws.get("keig.mid", sizeof(T) * N * R);
  eig_modes<T>(c, m, false, B, mid, R);  // (x) V^T B
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((N * R + 255) / 256, 8 * c->num_sms));
  k_eig_scale<T><<<grid, 256, 0, c->s>>>(mid, N, R, dims_of(m), m.ck, s, cd);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
  eig_modes<T>(c, m, true, mid, X, R);  // (x) V (...)
}

// 1 / (c_k prod_k lambda_k[i_k] + shift) per flat index, in FP32 and FP64.
__global__ void k_eig_inv(int64_t N, EigDims g, double ck, double shift, float* i32,
                          double* i64) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = 1.0 / eig_at(g, i, ck, shift);
    i32[i] = (float)v;
    i64[i] = v;
  }
}

// Per-block partial sums of x[0..n) (fixed order within a block).
__global__ void k_partial_sum(int64_t n, const double* x, double* part) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
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

// Y[r, i] *= inv[i]; grid.y runs over the right-hand sides.
template <typename T>
__global__ void k_scale_rows(T* Y, int64_t N, const T* inv) {
  T* y = Y + (int64_t)blockIdx.y * N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] *= inv[i];
}

}  // namespace

// Direct solve X = A^-1 B when A is eigen-structured (Kron or KronSum of
// square dense factors, optionally + scalar * I); false, with nothing
// launched, otherwise.  FP64 or FP32 vectors.
bool eig_solve_if_structured(Ctx* c, const cola_linop* op, const void* B, void* X, int64_t R,
                             bool f64) {
  KronShift m;
  if (!try_match(op, m)) return false;
  prepare_leaves(c, const_cast<cola_linop*>(op), COLA_PREC_F64, 0);
  prepare_eig(c, m, !f64);
  const double* s = m.diag ? leaf_ptr<double>(m.diag) : nullptr;
  if (f64)
    eig_solve<double>(c, m, s, m.cd, (const double*)B, (double*)X, R);
  else
    eig_solve<float>(c, m, s, m.cd, (const float*)B, (float*)X, R);
  return true;
}

// Preconditioner for A = c_k Kron + c_d Diag(d) (Kron a Kronecker product or
// sum): M = c_k Kron + c_d mean(d) I
// = Q diag(c_k lambda + c_d mean(d)) Q^T with Q = (x)_k V_k, applied exactly as
// Q^T, a diagonal scaling and Q.  The two Kronecker products run through the
// ordinary MVM path in the solve's precision (tensor cores for MIXED), with
// the factors' eigenvector matrices as the Kronecker factors.  False when A
// has another shape; COLA_ERR_INVALID_ARG when M is not positive definite.
// Sizes the workspace for R right-hand sides, so that a later graph capture
// allocates nothing.
bool kron_precond_setup(Ctx* c, cola_linop* op, KronPrecond* P, int64_t R, int prec,
                        int split_terms) {
  if (op->kind != LK_SUM || op->kids.size() != 2) return false;
  int ik = -1, id = -1;
  for (int i = 0; i < 2; ++i) {
    if (is_kron_node(op->kids[i])) ik = i;
    if (op->kids[i]->kind == LK_DIAG) id = i;
  }
  if (ik < 0 || id < 0) return false;
  cola_linop* kron = op->kids[ik];
  if ((int)kron->kids.size() > kMaxFactors) return false;
  for (auto* f : kron->kids)
    if (f->kind != LK_DENSE || f->rows != f->cols) return false;
  const cola_linop* dg = op->kids[id];
  prepare_leaves(c, op, COLA_PREC_F64, 0);
  // mean(d) on the device (block partials, summed here in a fixed order)
  const int64_t nd = dg->stride ? dg->rows : 1;
  const int nbs = (int)std::max<int64_t>(1, std::min<int64_t>((nd + 255) / 256, 1024));
  double* dpart = (double*)c->ws.get("keig.dpart", 8 * 1024);
  k_partial_sum<<<nbs, 256, 0, c->s>>>(nd, leaf_ptr<double>(dg), dpart);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
  std::vector<double> hp(nbs);
  COLA_CUDA(cudaMemcpyAsync(hp.data(), dpart, 8 * nbs, cudaMemcpyDeviceToHost, c->s));
  COLA_CUDA(cudaStreamSynchronize(c->s));
  double mean = 0.0;
  for (double v : hp) mean += v;
  mean /= (double)nd;
  const double shift = op->coeffs[id] * mean;
  KronShift m;
  m.kron = kron;
  m.sum = kron->kind == LK_KRONSUM;
  m.ck = op->coeffs[ik];
  prepare_eig(c, m, false);
  // smallest eigenvalue of M: the products (sums) of factor eigenvalues fill
  // an interval whose ends come from per-factor extreme eigenvalues
  double lo = m.sum ? 0.0 : 1.0, hi = lo;
  for (auto* f : kron->kids) {
    std::vector<double> lam(f->rows);
    COLA_CUDA(cudaMemcpyAsync(lam.data(), f->derived.at(kKeyLam64).p, 8 * f->rows,
                              cudaMemcpyDeviceToHost, c->s));
    COLA_CUDA(cudaStreamSynchronize(c->s));
    const double a = *std::min_element(lam.begin(), lam.end());
    const double b = *std::max_element(lam.begin(), lam.end());
    if (m.sum) {
      lo += a;
      hi += b;
    } else {
      const double q[4] = {lo * a, lo * b, hi * a, hi * b};
      lo = *std::min_element(q, q + 4);
      hi = *std::max_element(q, q + 4);
    }
  }
  const double mmin = (m.ck >= 0.0 ? m.ck * lo : m.ck * hi) + shift;
  COLA_REQUIRE(mmin > 0.0, COLA_ERR_INVALID_ARG,
               "kron_precond: M = c_k Kron + c_d mean(d) I is not positive definite (min "
               "eigenvalue %g)", mmin);
  // Q^T as a Kron node over the cached FP64 V_k^T (kept on the Kron node)
  if (!kron->eig_kron) {
    cola_ctx* cc = static_cast<cola_ctx*>(c);
    std::vector<cola_linop*> vt;
    cola_status st = COLA_OK;
    for (auto* f : kron->kids) {
      cola_linop* l = nullptr;
      if (st == COLA_OK)
        st = cola_linop_dense(cc, f->rows, f->rows, f->derived.at(kKeyVt64).p, f->rows, COLA_F64,
                              &l);
      if (l) vt.push_back(l);
    }
    cola_linop* q = nullptr;
    if (st == COLA_OK) st = cola_linop_kron(cc, (int)vt.size(), vt.data(), &q);
    for (auto* l : vt) cola_linop_release(l);
    COLA_REQUIRE(st == COLA_OK && q, COLA_ERR_CUDA, "kron_precond: building Q^T failed");
    kron->eig_kron = q;
  }
  // the factor splits are recomputed every time: V_k changes with K_k
  prepare_leaves(c, kron->eig_kron, prec, split_terms);
  const int64_t N = kron->rows;
  P->inv32 = (float*)c->ws.get("keig.inv32", 4 * N);
  P->inv64 = (double*)c->ws.get("keig.inv64", 8 * N);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 8 * c->num_sms));
  k_eig_inv<<<grid, 256, 0, c->s>>>(N, dims_of(m), m.ck, shift, P->inv32, P->inv64);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
  const size_t es = prec == COLA_PREC_F64 ? 8 : 4;
  c->ws.get("keig.pmid", es * N * R);
  P->qt = kron->eig_kron;
  P->prec = prec;
  return true;
}

// z = M^-1 r = Q (inv * (Q^T r)).  The mode products use workspace depth 4.
template <typename T>
void kron_precond_apply(Ctx* c, const KronPrecond& P, const T* r, T* z, int64_t R) {
  const int64_t N = P.qt->rows;
  T* mid = (T*)c->ws.get("keig.pmid", sizeof(T) * N * R);
  apply<T>(c, P.qt, r, mid, R, 1.0, 0.0, 4, false, P.prec);
  const T* inv = sizeof(T) == 8 ? (const T*)P.inv64 : (const T*)P.inv32;
  const int gx = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 2 * c->num_sms));
  k_scale_rows<T><<<dim3(gx, (unsigned)R), 256, 0, c->s>>>(mid, N, inv);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
  apply<T>(c, P.qt, mid, z, R, 1.0, 0.0, 4, true, P.prec);
}
template void kron_precond_apply<float>(Ctx*, const KronPrecond&, const float*, float*, int64_t);
template void kron_precond_apply<double>(Ctx*, const KronPrecond&, const double*, double*,
                                         int64_t);

}  // namespace cola

using namespace cola;

cola_status cola_sym_eig(int64_t n, const double* A, double* V, double* w) {
  return guard([&] {
    COLA_REQUIRE(A && V && w, COLA_ERR_INVALID_ARG, "NULL argument");
    COLA_REQUIRE(n >= 1 && n <= 8192, COLA_ERR_INVALID_ARG, "n = %lld", (long long)n);
    std::vector<double> a(A, A + n * n), Vt((size_t)(n * n));
    COLA_REQUIRE(sym_eig((int)n, a.data(), Vt.data(), w), COLA_ERR_NOT_CONVERGED,
                 "symmetric QR did not converge within %lld iterations", (long long)(60 * n));
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) V[i * n + j] = Vt[(size_t)(j * n + i)];
  });
}

cola_status cola_kron_eig_solve(cola_ctx* ctx, const cola_linop* op, const void* B, void* X,
                                int64_t nrhs, cola_precision prec, cola_stream stream) {
  return guard([&] {
    COLA_REQUIRE(ctx && op && B && X, COLA_ERR_INVALID_ARG, "NULL argument");
    COLA_REQUIRE(nrhs >= 1, COLA_ERR_INVALID_ARG, "nrhs = %lld", (long long)nrhs);
    COLA_REQUIRE(prec == COLA_PREC_F64 || prec == COLA_PREC_F32, COLA_ERR_INVALID_ARG,
                 "precision must be F64 or F32");
    COLA_REQUIRE(B != X, COLA_ERR_INVALID_ARG, "B and X must not alias");
    StreamJoin j(ctx, stream);
    const KronShift m = match(op);
    cola_linop* mop = const_cast<cola_linop*>(op);
    prepare_leaves(ctx, mop, COLA_PREC_F64, 0);  // the shift as an FP64 device scalar
    prepare_eig(ctx, m, prec == COLA_PREC_F32);
    const double* s = m.diag ? leaf_ptr<double>(m.diag) : nullptr;
    if (prec == COLA_PREC_F64)
      eig_solve<double>(ctx, m, s, m.cd, (const double*)B, (double*)X, nrhs);
    else
      eig_solve<float>(ctx, m, s, m.cd, (const float*)B, (float*)X, nrhs);
  });
}

cola_status cola_kron_eigs(cola_ctx* ctx, const cola_linop* op, double* factor_evals,
                           double* factor_evecs, double* evals, cola_stream stream) {
  return guard([&] {
    COLA_REQUIRE(ctx && op, COLA_ERR_INVALID_ARG, "NULL argument");
    COLA_REQUIRE(factor_evals || factor_evecs || evals, COLA_ERR_INVALID_ARG,
                 "no output requested");
    StreamJoin j(ctx, stream);
    const KronShift m = match(op);
    prepare_leaves(ctx, const_cast<cola_linop*>(op), COLA_PREC_F64, 0);
    prepare_eig(ctx, m, false);
    int64_t off_w = 0, off_v = 0;
    for (auto* f : m.kron->kids) {
      const int64_t n = f->rows;
      if (factor_evals)
        COLA_CUDA(cudaMemcpyAsync(factor_evals + off_w, f->derived.at(kKeyLam64).p, 8 * n,
                                  cudaMemcpyDeviceToDevice, ctx->s));
      if (factor_evecs) {
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n * n + 255) / 256, 1024));
        k_transpose64<<<grid, 256, 0, ctx->s>>>(n, (const double*)f->derived.at(kKeyVt64).p,
                                                factor_evecs + off_v);
        ctx->count_launch();
      }
      off_w += n;
      off_v += n * n;
    }
    if (evals) {
      const int64_t N = m.kron->rows;
      const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 4096));
      k_eig_values<<<grid, 256, 0, ctx->s>>>(N, dims_of(m), m.ck,
                                             m.diag ? leaf_ptr<double>(m.diag) : nullptr, m.cd,
                                             evals);
      ctx->count_launch();
    }
    COLA_CUDA(cudaGetLastError());
  });
}

cola_status cola_kron_eig_logdet(cola_ctx* ctx, const cola_linop* op, double* logdet,
                                 cola_stream stream) {
  return guard([&] {
    COLA_REQUIRE(ctx && op && logdet, COLA_ERR_INVALID_ARG, "NULL argument");
    StreamJoin j(ctx, stream);
    const KronShift m = match(op);
    prepare_leaves(ctx, const_cast<cola_linop*>(op), COLA_PREC_F64, 0);
    prepare_eig(ctx, m, false);
    const int64_t N = m.kron->rows;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, 1024));
    double* part = (double*)ctx->ws.get("keig.ldp", 8 * 1024);
    int* bad = (int*)ctx->ws.get("keig.ldb", 4 * 1024);
    k_eig_logdet<<<grid, 256, 0, ctx->s>>>(N, dims_of(m), m.ck,
                                           m.diag ? leaf_ptr<double>(m.diag) : nullptr, m.cd,
                                           part, bad);
    ctx->count_launch();
    COLA_CUDA(cudaGetLastError());
    std::vector<double> hp(grid);
    std::vector<int> hb(grid);
    COLA_CUDA(cudaMemcpyAsync(hp.data(), part, 8 * grid, cudaMemcpyDeviceToHost, ctx->s));
    COLA_CUDA(cudaMemcpyAsync(hb.data(), bad, 4 * grid, cudaMemcpyDeviceToHost, ctx->s));
    COLA_CUDA(cudaStreamSynchronize(ctx->s));
    double s = 0.0;
    int nb = 0;
    for (int b = 0; b < grid; ++b) {
      s += hp[b];
      nb += hb[b];
    }
    COLA_REQUIRE(nb == 0, COLA_ERR_BREAKDOWN, "%d eigenvalues of the operator are <= 0", nb);
    *logdet = s;
  });
}
