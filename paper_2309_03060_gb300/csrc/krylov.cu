// Krylov drivers on top of the operator MVM:
//  * conjugate gradients (Table 5: CG is the PSD solve base case), multi-RHS
//    with per-RHS step sizes and the all-solves stopping rule (App. D GP
//    training), optional Jacobi preconditioner (Diag rules, App. A.1.4), and
//    an FP64 iterative-refinement loop: the solution is accumulated in FP64
//    and the recursive FP32 residual is replaced by the FP64 true residual
//    b - A x whenever it has dropped by a set factor (reliable updates).  The
//    low-precision routines of Sec. 3.4 / App. C.3 motivate this; the paper
//    gives no algorithm for it.
//  * Lanczos (Table 5 self-adjoint base case) batched over starting vectors,
//    with the breakdown test of the Arnoldi iteration (Algorithm 1).
//  * stochastic Lanczos quadrature for log det A = Tr(log A) (App. A.2):
//    per probe ||z||^2 sum_k S_0k^2 log(theta_k), T_m = S diag(theta) S^T,
//    with an implicit-shift symmetric tridiagonal QR on the host (FP64).
//  * the adjoint rules of App. B.2 (solve VJP, log-det gradient).
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>

#include <thread>
#include <type_traits>

#include "internal.h"

namespace cola {

namespace {

template <typename T>
__device__ __forceinline__ double block_sum2(T v, double* out_other, T v2) {
  // Sums two values over the block; returns the first, writes the second.
  __shared__ double sh[2][32];
  double x = (double)v, y = (double)v2;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_xor_sync(0xffffffffu, x, o);
    y += __shfl_xor_sync(0xffffffffu, y, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) {
    sh[0][w] = x;
    sh[1][w] = y;
  }
  __syncthreads();
  double tx = 0.0, ty = 0.0;
  if (threadIdx.x < 32) {
    const bool ok = l < (int)(blockDim.x >> 5);
    tx = ok ? sh[0][l] : 0.0;
    ty = ok ? sh[1][l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      tx += __shfl_xor_sync(0xffffffffu, tx, o);
      ty += __shfl_xor_sync(0xffffffffu, ty, o);
    }
  }
  *out_other = ty;
  return tx;
}

// Refined solves: pause a right-hand side once its recursive residual norm fell
// by 1e6 since the last replacement; restart its search direction when a
// replacement finds the true residual norm more than 10x the recursive one.
constexpr double kPauseDrop2 = 1e-12;
// A replacement costing more than this many iterations waits for half of the
// right-hand sides (see cg_run).
constexpr double kDeferRatio = 100.0;
constexpr double kRestartGap2 = 100.0;

// alpha = r^T z / p^T A p, with p^T A p the ordered sum of nparts partials.
// One block per right-hand side: p^T A p from its partial sums, alpha = r^T z / p^T A p.
// alpha_out (optional): where this iteration's alpha is recorded (0 when inactive).
__global__ void k_cg_alpha(CgState* st, const double* parts, int nparts, double* alpha_out) {
  pdl_trigger();
  pdl_wait();
  const int64_t r = blockIdx.x;
  CgState& s = st[r];
  if (!s.active || s.paused) {
    if (threadIdx.x == 0) {
      s.alpha = 0.0;
      if (alpha_out) alpha_out[r] = 0.0;
    }
    return;
  }
  double v = 0.0;
  for (int j = threadIdx.x; j < nparts; j += blockDim.x) v += parts[r * nparts + j];
  double unused;
  v = block_sum2(v, &unused, 0.0);
  if (threadIdx.x != 0) return;
  s.pAp = v;
  if (!(v > 0.0) || !isfinite(v)) {
    s.status = COLA_ERR_BREAKDOWN;
    s.active = 0;
    s.alpha = 0.0;
    if (alpha_out) alpha_out[r] = 0.0;
    return;
  }
  s.alpha = s.rz / v;
  if (alpha_out) alpha_out[r] = s.alpha;
}

// x += alpha p; r -= alpha Ap; z = M^-1 r; partial sums of r^T z and r^T r.
template <typename T>
__global__ void k_cg_xr(int64_t n, T* x, T* r, const T* p, const T* Ap, const T* invd, T* z,
                        const CgState* st, int nblk, double* part_rz, double* part_rr) {
  const int64_t v = blockIdx.y;
  const T a = (T)st[v].alpha;
  T* xv = x + v * n;
  T* rv = r + v * n;
  const T* pv = p + v * n;
  const T* Av = Ap + v * n;
  T* zv = z ? z + v * n : nullptr;
  T s_rz = T(0), s_rr = T(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)nblk * blockDim.x) {
    T ri = rv[i];
    if (a != T(0)) {
      xv[i] = fma(a, pv[i], xv[i]);
      ri = fma(-a, Av[i], ri);
      rv[i] = ri;
    }
    T zi = ri;
    if (invd) {
      zi = ri * invd[i];
      zv[i] = zi;
    }
    s_rz = fma(ri, zi, s_rz);
    s_rr = fma(ri, ri, s_rr);
  }
  double rr;
  const double rz = block_sum2(s_rz, &rr, s_rr);
  if (threadIdx.x == 0) {
    part_rz[v * nblk + blockIdx.x] = rz;
    part_rr[v * nblk + blockIdx.x] = rr;
  }
}

// One block per right-hand side: the new r^T z and r^T r, beta, and the stopping rule.
// k_cg_xr for FP32 vectors of a length divisible by 4 (16-byte accesses keep
// enough bytes in flight for the HBM bandwidth); n4 = n / 4.
__global__ void k_cg_xr4(int64_t n4, float4* x, float4* r, const float4* p, const float4* Ap,
                         const float4* invd, float4* z, const CgState* st, int nblk,
                         double* part_rz, double* part_rr) {
  pdl_trigger();
  pdl_wait();
  const int64_t v = blockIdx.y;
  const float a = (float)st[v].alpha;
  float4* xv = x + v * n4;
  float4* rv = r + v * n4;
  const float4* pv = p + v * n4;
  const float4* Av = Ap + v * n4;
  float4* zv = z ? z + v * n4 : nullptr;
  float s_rz = 0.0f, s_rr = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)nblk * blockDim.x) {
    float4 ri = rv[i];
    if (a != 0.0f) {
      const float4 pi = pv[i], ai = Av[i];
      float4 xi = xv[i];
      xi.x = fmaf(a, pi.x, xi.x);
      xi.y = fmaf(a, pi.y, xi.y);
      xi.z = fmaf(a, pi.z, xi.z);
      xi.w = fmaf(a, pi.w, xi.w);
      ri.x = fmaf(-a, ai.x, ri.x);
      ri.y = fmaf(-a, ai.y, ri.y);
      ri.z = fmaf(-a, ai.z, ri.z);
      ri.w = fmaf(-a, ai.w, ri.w);
      xv[i] = xi;
      rv[i] = ri;
    }
    float4 zi = ri;
    if (invd) {
      const float4 d = invd[i];
      zi = make_float4(ri.x * d.x, ri.y * d.y, ri.z * d.z, ri.w * d.w);
      zv[i] = zi;
    }
    s_rz = fmaf(ri.x, zi.x, fmaf(ri.y, zi.y, fmaf(ri.z, zi.z, fmaf(ri.w, zi.w, s_rz))));
    s_rr = fmaf(ri.x, ri.x, fmaf(ri.y, ri.y, fmaf(ri.z, ri.z, fmaf(ri.w, ri.w, s_rr))));
  }
  double rr;
  const double rz = block_sum2(s_rz, &rr, s_rr);
  if (threadIdx.x == 0) {
    part_rz[v * nblk + blockIdx.x] = rz;
    part_rr[v * nblk + blockIdx.x] = rr;
  }
}

// k_cg_xr4 without the solution update: r -= alpha Ap, z = M^-1 r and the
// partial dots.  x is brought up to date every kPRing iterations by k_cg_xbatch.
// rev: right-hand sides and elements in reverse order.  The CG's kernels
// alternate their directions so that each starts on the part of its input the
// kernel before it wrote last (still in L2).
__global__ void k_cg_r4(int64_t n4, float4* r, const float4* Ap, const float4* invd, float4* z,
                        const CgState* st, int nblk, double* part_rz, double* part_rr,
                        int rev) {
  pdl_trigger();
  pdl_wait();
  const int64_t v = rev ? gridDim.y - 1 - blockIdx.y : blockIdx.y;
  const float a = (float)st[v].alpha;
  float4* rv = r + v * n4;
  const float4* Av = Ap + v * n4;
  float4* zv = z ? z + v * n4 : nullptr;
  float s_rz = 0.0f, s_rr = 0.0f;
  const int64_t stride = (int64_t)nblk * blockDim.x;
  // two elements per step, both loaded before either is stored: twice the
  // bytes in flight of a one-element loop
  for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n4; i0 += 2 * stride) {
    const int64_t j0 = i0 + stride;
    const bool two = j0 < n4;
    const int64_t i = rev ? n4 - 1 - i0 : i0, j = rev ? n4 - 1 - j0 : j0;
    float4 ri[2], ai[2];
    ri[0] = rv[i];
    ai[0] = a != 0.0f ? Av[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    ri[1] = two ? rv[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    ai[1] = (two && a != 0.0f) ? Av[j] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (u == 1 && !two) break;
      const int64_t k = u ? j : i;
      float4 r4 = ri[u];
      if (a != 0.0f) {
        r4.x = fmaf(-a, ai[u].x, r4.x);
        r4.y = fmaf(-a, ai[u].y, r4.y);
        r4.z = fmaf(-a, ai[u].z, r4.z);
        r4.w = fmaf(-a, ai[u].w, r4.w);
        rv[k] = r4;
      }
      float4 zi = r4;
      if (invd) {
        const float4 d = invd[k];
        zi = make_float4(r4.x * d.x, r4.y * d.y, r4.z * d.z, r4.w * d.w);
        zv[k] = zi;
      }
      s_rz = fmaf(r4.x, zi.x, fmaf(r4.y, zi.y, fmaf(r4.z, zi.z, fmaf(r4.w, zi.w, s_rz))));
      s_rr = fmaf(r4.x, r4.x, fmaf(r4.y, r4.y, fmaf(r4.z, r4.z, fmaf(r4.w, r4.w, s_rr))));
    }
  }
  double rr;
  const double rz = block_sum2(s_rz, &rr, s_rr);
  if (threadIdx.x == 0) {
    part_rz[v * nblk + blockIdx.x] = rz;
    part_rr[v * nblk + blockIdx.x] = rr;
  }
}

// The search directions of the last kPRing iterations (one ring slot each).
constexpr int kPRing = 8;
struct PRing {
  const float4* p[kPRing];
};

// x += sum_s alpha_s p_s over the ring (alpha_hist[s][r]; 0 for an inactive
// right-hand side): the x updates of kPRing CG iterations in one pass.
__global__ void k_cg_xbatch(int64_t n4, float4* x, PRing ring, const double* alpha_hist,
                            int64_t R, int nblk) {
  pdl_trigger();
  pdl_wait();
  const int64_t v = blockIdx.y;
  float a[kPRing];
  bool any = false;
#pragma unroll
  for (int s = 0; s < kPRing; ++s) {
    a[s] = (float)alpha_hist[s * R + v];
    any |= a[s] != 0.0f;
  }
  if (!any) return;
  float4* xv = x + v * n4;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)nblk * blockDim.x) {
    float4 acc = xv[i];
#pragma unroll
    for (int s = 0; s < kPRing; ++s) {
      const float4 ps = ring.p[s][v * n4 + i];
      acc.x = fmaf(a[s], ps.x, acc.x);
      acc.y = fmaf(a[s], ps.y, acc.y);
      acc.z = fmaf(a[s], ps.z, acc.z);
      acc.w = fmaf(a[s], ps.w, acc.w);
    }
    xv[i] = acc;
  }
}

__global__ void k_cg_beta(CgState* st, const double* part_rz, const double* part_rr, int nblk,
                          double delta2, int refine, double* beta_out) {
  pdl_trigger();
  pdl_wait();
  const int64_t r = blockIdx.x;
  CgState& s = st[r];
  if (!s.active || s.paused) {
    // a paused right-hand side keeps x and r and holds p = z until the next
    // residual replacement restarts it; its idle iterations are not counted
    if (threadIdx.x == 0) {
      s.beta = 0.0;
      if (beta_out) beta_out[r] = 0.0;
    }
    return;
  }
  double rz = 0.0, rr = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    rz += part_rz[r * nblk + b];
    rr += part_rr[r * nblk + b];
  }
  rz = block_sum2(rz, &rr, rr);
  if (threadIdx.x != 0) return;
  s.beta = rz / s.rz;
  s.rz = rz;
  s.rr = rr;
  s.iters += 1;
  if (!isfinite(rr) || !isfinite(rz)) {
    s.status = COLA_ERR_BREAKDOWN;
    s.active = 0;
    s.beta = 0.0;
    return;
  }
  if (refine) {
    if (rr <= s.tol2 || rr <= delta2 * s.rr_ref) s.flag = 1;
    // The recursive residual fell a million-fold since the last replacement
    // (or reached zero): FP32 cannot make the true residual follow it further,
    // and a fast recursion would underflow before the chunk ends.  Pause until
    // the replacement.
    if (rr <= kPauseDrop2 * s.rr_ref || rz == 0.0) {
      s.paused = 1;
      s.beta = 0.0;
    }
  } else if (rr <= s.tol2) {
    s.active = 0;
  }
  if (beta_out) beta_out[r] = s.active ? s.beta : 0.0;
}

template <typename T>
__global__ void k_cg_p(int64_t n, const T* z, T* p, const CgState* st) {
  const int64_t v = blockIdx.y;
  if (!st[v].active) return;
  const T b = (T)st[v].beta;
  const T* zv = z + v * n;
  T* pv = p + v * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    pv[i] = fma(b, pv[i], zv[i]);
}

// r = (T) r64 (refined) or r as is; z = M^-1 r; partial r^T z and r^T r.
template <typename T>
__global__ void k_refresh(int64_t n, const double* r64, T* r, const T* invd, T* z, int nblk,
                          double* part_rz, double* part_rr) {
  const int64_t v = blockIdx.y;
  T s_rz = T(0), s_rr = T(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)nblk * blockDim.x) {
    T ri = r64 ? (T)r64[v * n + i] : r[v * n + i];
    if (r64) r[v * n + i] = ri;
    T zi = ri;
    if (invd) {
      zi = ri * invd[i];
      z[v * n + i] = zi;
    }
    s_rz = fma(ri, zi, s_rz);
    s_rr = fma(ri, ri, s_rr);
  }
  double rr;
  const double rz = block_sum2(s_rz, &rr, s_rr);
  if (threadIdx.x == 0) {
    part_rz[v * nblk + blockIdx.x] = rz;
    part_rr[v * nblk + blockIdx.x] = rr;
  }
}

// p = z for the right-hand sides a replacement restarted.
template <typename T>
__global__ void k_cg_restart_p(int64_t n, const T* z, T* p, const CgState* st) {
  const int64_t v = blockIdx.y;
  if (!st[v].active || !st[v].restart) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[v * n + i] = z[v * n + i];
}

// Partial r^T z per block (same [R][nblk] layout as k_refresh), for a z that
// a separate preconditioner solve produced.
template <typename T>
__global__ void k_rz_parts(int64_t n, const T* r, const T* z, int nblk, double* part_rz) {
  const int64_t v = blockIdx.y;
  T s = T(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)nblk * blockDim.x)
    s = fma(r[v * n + i], z[v * n + i], s);
  double unused;
  const double rz = block_sum2(s, &unused, T(0));
  if (threadIdx.x == 0) part_rz[v * nblk + blockIdx.x] = rz;
}

// (Re)start state after a residual refresh.  first: initialise everything.
// Otherwise (a replacement of the recursive residual by the true one) the
// search direction is kept, as reliable updating does, unless the recursion
// had paused or the true residual came out more than 10x the recursive one:
// the old direction then no longer matches r, and the right-hand side restarts
// from p = z (restart = 1; beta_vec, when given, is zeroed for the fused update).
__global__ void k_cg_restate(CgState* st, const double* part_rz, const double* part_rr, int nblk,
                             int64_t R, const double* rr64, const double* bb, double tol,
                             int first, double* beta_vec) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  CgState& s = st[r];
  double rz = 0.0, rr = 0.0;
  for (int b = 0; b < nblk; ++b) {
    rz += part_rz[r * nblk + b];
    rr += part_rr[r * nblk + b];
  }
  s.restart = 0;
  if (first) {
    s.iters = 0;
    s.updates = 0;
    s.status = 0;
    s.bb = bb[r];
    s.tol2 = tol * tol * bb[r];
    s.active = 1;
    s.alpha = s.beta = 0.0;
    // a right-hand side with a NaN or Inf entry cannot be solved
    if (!isfinite(bb[r])) {
      s.status = COLA_ERR_BREAKDOWN;
      s.active = 0;
    }
  } else if (s.active) {
    s.updates += 1;
    if (s.paused || rr > kRestartGap2 * s.rr) {
      s.restart = 1;
      s.beta = 0.0;
      if (beta_vec) beta_vec[r] = 0.0;
    }
  }
  s.paused = 0;
  s.flag = 0;
  s.rz = rz;
  s.rr = rr;
  s.rr_ref = rr;
  if (rr64) s.rr64 = rr64[r];
  const double conv = rr64 ? rr64[r] : rr;
  if (s.active && conv <= s.tol2) s.active = 0;
}

// After the recursive residual met the tolerance: re-activate every
// right-hand side whose true residual (partials of the freshly computed r)
// still misses it, restarting its search direction.
__global__ void k_cg_verify(CgState* st, const double* part_rz, const double* part_rr, int nblk,
                            int64_t R, double* beta_vec) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  CgState& s = st[r];
  double rz = 0.0, rr = 0.0;
  for (int b = 0; b < nblk; ++b) {
    rz += part_rz[r * nblk + b];
    rr += part_rr[r * nblk + b];
  }
  s.rr64 = rr;
  if (s.status != 0 || s.active || !(rr > s.tol2)) return;
  s.active = 1;
  s.flag = 0;
  s.rz = rz;
  s.rr = rr;
  s.rr_ref = rr;
  s.beta = 0.0;
  s.updates += 1;
  if (beta_vec) beta_vec[r] = 0.0;
}

template <typename T>
__global__ void k_copy_active(int64_t n, const T* src, T* dst, const CgState* st) {
  const int64_t v = blockIdx.y;
  if (!st[v].active) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[v * n + i] = src[v * n + i];
}

template <typename T>
__global__ void k_accum_x(int64_t tot, double* x64, T* x) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot;
       i += (int64_t)gridDim.x * blockDim.x) {
    x64[i] += (double)x[i];
    x[i] = T(0);
  }
}

__global__ void k_invert(int64_t n, const double* d, float* out32, double* out64) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = 1.0 / d[i];
    if (out32) out32[i] = (float)v;
    if (out64) out64[i] = v;
  }
}

// ------------------------------------------- re-orthogonalised residuals
// CG with re-orthogonalised residuals (the low-precision CG variant of
// Maddox, Potapczynski & Wilson, UAI 2022, that Sec. 3.4 / App. C.3 cite):
// the stored residuals Q[r][i] (i < k[r]) of each right-hand side; every new
// residual is made orthogonal to them by classical Gram-Schmidt before it
// enters beta and the next search direction.

// c[r][i] = Q[r][i] . x_r / ||Q[r][i]||^2 for i < k[r] (0 beyond); one block
// per (i, r), FP64 block reduction in a fixed order.
template <typename T>
__global__ void k_ro_dots(int64_t n, const T* Q, const T* x, const int* k, const double* n2,
                          int cap, const CgState* st, double* coef) {
  const int i = blockIdx.x;
  const int64_t r = blockIdx.y;
  if (!st[r].active || i >= k[r]) {
    if (threadIdx.x == 0) coef[r * cap + i] = 0.0;
    return;
  }
  const T* q = Q + ((int64_t)r * cap + i) * n;
  const T* xr = x + r * n;
  double acc = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) acc += (double)q[e] * (double)xr[e];
  double unused;
  acc = block_sum2(acc, &unused, 0.0);
  if (threadIdx.x == 0) coef[r * cap + i] = acc / n2[r * cap + i];
}

// x_r -= sum_{i < k[r]} c[r][i] Q[r][i] (the sum in FP64).
template <typename T>
__global__ void k_ro_sub(int64_t n, T* x, const T* Q, const int* k, const double* coef,
                         int cap, const CgState* st) {
  const int64_t r = blockIdx.y;
  if (!st[r].active) return;
  const int kr = k[r];
  const T* Qr = Q + (int64_t)r * cap * n;
  const double* cr = coef + (int64_t)r * cap;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < kr; ++i) acc += cr[i] * (double)Qr[(int64_t)i * n + e];
    x[r * n + e] = (T)((double)x[r * n + e] - acc);
  }
}

// Stores x_r as Q[r][k[r]] (while k[r] < cap) and writes the partials of
// x_r . x_r as both r^T z and r^T r (unpreconditioned: z = r), in the layout
// the residual kernels use.
template <typename T>
__global__ void k_ro_store(int64_t n, const T* x, T* Q, const int* k, int cap,
                           const CgState* st, int nblk, double* part_rz, double* part_rr) {
  const int64_t r = blockIdx.y;
  if (!st[r].active) return;
  const int kr = k[r];
  T* dst = kr < cap ? Q + ((int64_t)r * cap + kr) * n : nullptr;
  double acc = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)nblk * blockDim.x) {
    const T v = x[r * n + e];
    if (dst) dst[e] = v;
    acc += (double)v * (double)v;
  }
  double unused;
  acc = block_sum2(acc, &unused, 0.0);
  if (threadIdx.x == 0) {
    part_rz[r * nblk + blockIdx.x] = acc;
    part_rr[r * nblk + blockIdx.x] = acc;
  }
}

// Records ||Q[r][k]||^2 = the r^T r the beta kernel (or the restate) just
// summed and counts the stored residual; reset = 1 empties the store first.
__global__ void k_ro_commit(int64_t R, const CgState* st, int* k, double* n2, int cap,
                            int reset) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= R) return;
  if (reset) k[r] = 0;
  if (!st[r].active || k[r] >= cap) return;
  n2[r * cap + k[r]] = st[r].rr;
  k[r] += 1;
}

// ------------------------------------------------------------------ Lanczos
struct LzState {
  double beta_prev, amax;
  int active, m_eff;
};

__global__ void k_lz_init(LzState* st, const double* nrm2, int64_t nv, int m) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  st[v].beta_prev = 0.0;
  st[v].amax = 0.0;
  st[v].active = nrm2[v] > 0.0 ? 1 : 0;
  st[v].m_eff = nrm2[v] > 0.0 ? m : 0;
}

template <typename T>
__global__ void k_lz_scale(int64_t n, const T* src, T* dst, const double* nrm2) {
  const int64_t v = blockIdx.y;
  const double s = nrm2[v] > 0.0 ? 1.0 / sqrt(nrm2[v]) : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[v * n + i] = (T)((double)src[v * n + i] * s);
}

// w -= beta_prev q_prev; partial q^T w
template <typename T>
__global__ void k_lz_a(int64_t n, T* w, const T* qprev, const T* q, const LzState* st, int nblk,
                       double* part) {
  const int64_t v = blockIdx.y;
  const T bp = (T)st[v].beta_prev;
  T s = T(0), dummy = T(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)nblk * blockDim.x) {
    T wi = w[v * n + i];
    if (bp != T(0)) {
      wi = fma(-bp, qprev[v * n + i], wi);
      w[v * n + i] = wi;
    }
    s = fma(q[v * n + i], wi, s);
  }
  double o;
  const double t = block_sum2(s, &o, dummy);
  if (threadIdx.x == 0) part[v * nblk + blockIdx.x] = t;
}

// One block per vector (fixed-order block reduction of the partials).
__global__ void k_lz_alpha(LzState* st, const double* part, int nblk, int64_t nv, int j, int m,
                           double* alpha, double* a_cur) {
  const int64_t v = blockIdx.x;
  double a = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) a += part[v * nblk + b];
  double unused;
  a = block_sum2(a, &unused, 0.0);
  if (threadIdx.x != 0) return;
  a_cur[v] = st[v].active ? a : 0.0;
  if (st[v].active) {
    alpha[v * m + j] = a;
    st[v].amax = fmax(st[v].amax, fabs(a));
  }
}

// w -= alpha q; partial ||w||^2
template <typename T>
__global__ void k_lz_b(int64_t n, T* w, const T* q, const double* a_cur, int nblk, double* part,
                       int want_norm) {
  const int64_t v = blockIdx.y;
  const T a = (T)a_cur[v];
  T s = T(0), dummy = T(0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)nblk * blockDim.x) {
    const T wi = fma(-a, q[v * n + i], w[v * n + i]);
    w[v * n + i] = wi;
    s = fma(wi, wi, s);
  }
  if (!want_norm) return;
  double o;
  const double t = block_sum2(s, &o, dummy);
  if (threadIdx.x == 0) part[v * nblk + blockIdx.x] = t;
}

__global__ void k_lz_beta(LzState* st, const double* nrm2, int64_t nv, int j, int m, double eps,
                          double* beta, double* b_cur) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  LzState& s = st[v];
  b_cur[v] = 0.0;
  if (!s.active) return;
  if (j == m - 1) {
    s.active = 0;
    s.m_eff = m;
    return;
  }
  const double b = sqrt(fmax(nrm2[v], 0.0));
  if (!(b > eps * s.amax)) {
    s.active = 0;
    s.m_eff = j + 1;
    return;
  }
  beta[v * m + j] = b;
  s.beta_prev = b;
  b_cur[v] = b;
}

template <typename T>
__global__ void k_lz_next(int64_t n, T* w, const double* b_cur) {
  const int64_t v = blockIdx.y;
  const double b = b_cur[v];
  if (b == 0.0) return;
  const T s = (T)(1.0 / b);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    w[v * n + i] *= s;
}

// dst[v] = 1 / sqrt(src[v]) (root = 1) or 1 / src[v] (root = 0); 0 when src[v] <= 0.
__global__ void k_lz_recip(int64_t nv, const double* src, double* dst, int root) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const double x = src[v];
  dst[v] = x > 0.0 ? 1.0 / (root ? sqrt(x) : x) : 0.0;
}

// Unnormalised Lanczos (v_j = beta_j q_j): coef = -alpha_{j-1} s_{j-1}, the
// coefficient of v_{j-1} in v_j = w + coef v_{j-1}.
__global__ void k_lz_coef(int64_t nv, const double* a_cur, const double* s_prev, double* coef) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < nv) coef[v] = -a_cur[v] * s_prev[v];
}

// s_j = 1 / beta_j (0 after a breakdown, beta_j = 0) and gamma = beta_j s_{j-1},
// the coefficient of v_{j-1} in w = A q_j - beta_j q_{j-1}.
__global__ void k_lz_scales(int64_t nv, const double* b_cur, const double* s_prev, double* s_new,
                            double* gamma) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const double b = b_cur[v];
  s_new[v] = b > 0.0 ? 1.0 / b : 0.0;
  gamma[v] = b * s_prev[v];
}

__global__ void k_lz_meff(const LzState* st, int64_t nv, int* m_eff) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < nv) m_eff[v] = st[v].m_eff;
}

// --------------------------------------------------------------- quadrature
// Implicit symmetric tridiagonal QR with Wilkinson shifts (Golub & Van Loan
// Sec. 8.3), tracking the first row of the accumulated rotations: at
// convergence a[k] are the Ritz values theta_k and w[k] = S_0k.  Host FP64:
// the bulge chase is a chain of dependent FP64 square roots and divisions,
// which one GPU thread runs tens of times slower than a CPU core.  Returns
// false when the QR sweeps did not converge within 60 n iterations.
static bool tridiag_eig_first_row(double* a, double* b, double* w, int n) {
  for (int k = 0; k < n; ++k) w[k] = (k == 0) ? 1.0 : 0.0;
  if (n > 0) b[n - 1] = 0.0;
  const double eps = 2.220446049250313e-16;
  int q = n - 1, it = 0;
  while (q > 0 && it < 60 * n) {
    if (std::fabs(b[q - 1]) <= eps * (std::fabs(a[q - 1]) + std::fabs(a[q]))) {
      b[q - 1] = 0.0;
      --q;
      continue;
    }
    int p = q - 1;
    while (p > 0 && std::fabs(b[p - 1]) > eps * (std::fabs(a[p - 1]) + std::fabs(a[p]))) --p;
    ++it;
    const double d = 0.5 * (a[q - 1] - a[q]), bb = b[q - 1];
    const double sg = d >= 0.0 ? 1.0 : -1.0;
    const double mu = a[q] - bb * bb / (d + sg * std::hypot(d, bb));
    double x = a[p] - mu, z = b[p];
    for (int k = p; k < q; ++k) {
      const double r = std::hypot(x, z);
      const double c = x / r, s = z / r;
      if (k > p) b[k - 1] = r;
      const double ak = a[k], ak1 = a[k + 1], bk = b[k];
      a[k] = c * c * ak + 2.0 * c * s * bk + s * s * ak1;
      a[k + 1] = s * s * ak - 2.0 * c * s * bk + c * c * ak1;
      b[k] = c * s * (ak1 - ak) + (c * c - s * s) * bk;
      const double wk = w[k], wk1 = w[k + 1];
      w[k] = c * wk + s * wk1;
      w[k + 1] = -s * wk + c * wk1;
      if (k < q - 1) {
        x = b[k];
        z = s * b[k + 1];
        b[k + 1] = c * b[k + 1];
      }
    }
  }
  return q <= 0;
}

// Gauss quadrature of one probe: ||z||^2 sum_k S_0k^2 log(theta_k) from the
// Lanczos coefficients (alpha_0..alpha_{n-1}, beta_0..beta_{n-2}); Ritz values
// <= 0 are replaced by the smallest positive one and counted in *clamped.
struct QuadResult {
  double value = 0.0;
  int clamped = 0;
  bool converged = true;
};

static QuadResult slq_quadrature(const double* alpha, const double* beta, int n, double znorm2) {
  std::vector<double> a(alpha, alpha + n), b(n, 0.0), w(n);
  for (int k = 0; k + 1 < n; ++k) b[k] = beta[k];
  QuadResult res;
  res.converged = tridiag_eig_first_row(a.data(), b.data(), w.data(), n);
  double tmin = 0.0;
  for (int k = 0; k < n; ++k)
    if (a[k] > 0.0 && (tmin == 0.0 || a[k] < tmin)) tmin = a[k];
  double s = 0.0;
  for (int k = 0; k < n; ++k) {
    double th = a[k];
    if (!(th > 0.0)) {
      th = tmin;
      ++res.clamped;
    }
    s += w[k] * w[k] * std::log(th);
  }
  res.value = znorm2 * s;
  return res;
}

inline dim3 rows_grid(int64_t n, int64_t R, int nblk) { return dim3(nblk, (unsigned)R); }

inline int ew_blocks(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 1023) / 1024, 1024));
}

}  // namespace

// ====================================================================== CG
template <typename T>
struct CgBufs {
  T *x, *r, *p, *Ap, *z;  // working precision; p is pp[cur]
  T* pp[kPRing];          // ring of search directions (fused MIXED path; 1 buffer else)
  int cur;
  bool defer_x;           // x updated every kPRing iterations from the ring (fused FP32)
  double* alpha_hist;     // [kPRing][R] alpha of each ring slot
  T* invd;
  KronPrecond kp;         // kron_precond: z = M^-1 r by the eigen-structured solve
  bool kprec;
  double *x64, *b64, *r64;
  double *part_rz, *part_rr, *dotp, *dotv;
  double* beta_vec;   // per-RHS beta for the fused p update (MIXED)
  double* tile_dot;   // per-(tile, warp) partials of p^T A p (MIXED)
  int64_t fused_tiles;  // > 0: the fused tensor-core CG MVM applies
  CgState* st;
  // re-orthogonalised residuals (ro_cap > 0): store [R][ro_cap][N], their
  // squared norms and the Gram-Schmidt coefficients [R][ro_cap], counts [R]
  int ro_cap;
  T* roQ;
  double *ro_n2, *ro_c;
  int* ro_k;
};

// Re-orthogonalises the residual just formed (two classical Gram-Schmidt
// passes against the stored residuals), stores it and rewrites the r^T z /
// r^T r partials the beta kernel reads.
template <typename T>
static void ro_project(Ctx* c, CgBufs<T>& B, int64_t N, int64_t R, int nblk) {
  for (int pass = 0; pass < 2; ++pass) {
    k_ro_dots<T><<<dim3((unsigned)B.ro_cap, (unsigned)R), 256, 0, c->s>>>(
        N, B.roQ, B.r, B.ro_k, B.ro_n2, B.ro_cap, B.st, B.ro_c);
    c->count_launch();
    k_ro_sub<T><<<dim3(ew_blocks(N), (unsigned)R), 256, 0, c->s>>>(N, B.r, B.roQ, B.ro_k,
                                                                    B.ro_c, B.ro_cap, B.st);
    c->count_launch();
  }
  k_ro_store<T><<<dim3((unsigned)nblk, (unsigned)R), 256, 0, c->s>>>(
      N, B.r, B.roQ, B.ro_k, B.ro_cap, B.st, nblk, B.part_rz, B.part_rr);
  c->count_launch();
}

// (Re)starts the store with the current residual, after a restate.
template <typename T>
static void ro_restart(Ctx* c, CgBufs<T>& B, int64_t N, int64_t R, int nblk) {
  k_ro_commit<<<(unsigned)((R + 127) / 128), 128, 0, c->s>>>(R, B.st, B.ro_k, B.ro_n2, 0, 1);
  c->count_launch();
  k_ro_store<T><<<dim3((unsigned)nblk, (unsigned)R), 256, 0, c->s>>>(
      N, B.r, B.roQ, B.ro_k, B.ro_cap, B.st, nblk, B.part_rz, B.part_rr);
  c->count_launch();
  k_ro_commit<<<(unsigned)((R + 127) / 128), 128, 0, c->s>>>(R, B.st, B.ro_k, B.ro_n2,
                                                             B.ro_cap, 0);
  c->count_launch();
}

static std::string key_of(const char* what, const cola_linop* op, int64_t R, int prec, int extra,
                          uint64_t gen) {
  char b[160];
  snprintf(b, sizeof b, "%s:%llu:%lld:%d:%d:%llu", what, (unsigned long long)op->uid,
           (long long)R, prec, extra, (unsigned long long)gen);
  return b;
}

// The vector the search direction is built from: z = M^-1 r when
// preconditioned, r otherwise.
template <typename T>
static T* z_of(const CgBufs<T>& B) {
  return (B.invd || B.kprec) ? B.z : B.r;
}

// kron_precond: z = M^-1 r and the r^T z partials (replacing the r^T r ones
// the residual kernel left in part_rz).
template <typename T>
static void precond_z(Ctx* c, CgBufs<T>& B, int64_t N, int64_t R, int nblk) {
  if (!B.kprec) return;
  kron_precond_apply<T>(c, B.kp, B.r, B.z, R);
  k_rz_parts<T><<<rows_grid(N, R, nblk), 256, 0, c->s>>>(N, B.r, B.z, nblk, B.part_rz);
  c->count_launch();
}

template <typename T>
static void cg_iteration(Ctx* c, const cola_linop* op, CgBufs<T>& B, int64_t N, int64_t R,
                         int nblk, int prec, double delta2, int refine, bool defer) {
  if (B.fused_tiles > 0) {
    // p_new = z + beta p_old (first mode step), Ap and p^T A p partials (last)
    const int nxt = (B.cur + 1) % kPRing;
    T* p_old = B.pp[B.cur];
    T* p_new = B.pp[nxt];
    // odd ring positions: the first mode step runs its tiles backwards, the
    // slab kernel forwards, the residual update backwards; even ones the
    // other way round (each kernel starts where the one before it ended)
    kron_tc_cg_mvm(c, op, (const float*)z_of(B), B.beta_vec, (const float*)p_old,
                   (float*)p_new, (float*)B.Ap, B.tile_dot, R, 1, B.cur & 1);
    B.cur = nxt;
    B.p = p_new;
    // the small CG kernels launch normally (an early launch measured slower);
    // their pdl_trigger lets the next tensor-core step start its set-up early
    k_cg_alpha<<<(unsigned)R, 256, 0, c->s>>>(B.st, B.tile_dot, (int)(8 * B.fused_tiles),
                                               defer ? B.alpha_hist + (int64_t)nxt * R : nullptr);
    c->count_launch();
  } else {
    apply<T>(c, op, B.p, B.Ap, R, 1.0, 0.0, 1, false, prec);
    dots<T>(c, B.p, B.Ap, N, R, B.dotp, B.dotv);
    k_cg_alpha<<<(unsigned)R, 32, 0, c->s>>>(B.st, B.dotv, 1, nullptr);
    c->count_launch();
  }
  bool vec4 = false;
  if constexpr (std::is_same<T, float>::value) {
    const uintptr_t al = (uintptr_t)B.x | (uintptr_t)B.r | (uintptr_t)B.p | (uintptr_t)B.Ap |
                         (uintptr_t)B.z | (uintptr_t)B.invd;
    vec4 = N % 4 == 0 && (al & 15u) == 0;
    if (vec4 && defer)
      k_cg_r4<<<rows_grid(N, R, nblk), 256, 0, c->s>>>(
          N / 4, (float4*)B.r, (const float4*)B.Ap, (const float4*)B.invd,
          B.invd ? (float4*)B.z : nullptr, B.st, nblk, B.part_rz, B.part_rr,
          (B.cur & 1) ? 0 : 1);
    else if (vec4)
      k_cg_xr4<<<rows_grid(N, R, nblk), 256, 0, c->s>>>(
          N / 4, (float4*)B.x, (float4*)B.r, (const float4*)B.p, (const float4*)B.Ap,
          (const float4*)B.invd, B.invd ? (float4*)B.z : nullptr, B.st, nblk, B.part_rz,
          B.part_rr);
  }
  if (!vec4)
    k_cg_xr<T><<<rows_grid(N, R, nblk), 256, 0, c->s>>>(N, B.x, B.r, B.p, B.Ap, B.invd,
                                                         B.invd ? B.z : nullptr, B.st, nblk,
                                                         B.part_rz, B.part_rr);
  c->count_launch();
  precond_z<T>(c, B, N, R, nblk);
  if (B.ro_cap > 0) ro_project<T>(c, B, N, R, nblk);
  k_cg_beta<<<(unsigned)R, 256, 0, c->s>>>(B.st, B.part_rz, B.part_rr, nblk, delta2, refine,
                                            B.beta_vec);
  c->count_launch();
  if (B.ro_cap > 0) {
    k_ro_commit<<<(unsigned)((R + 127) / 128), 128, 0, c->s>>>(R, B.st, B.ro_k, B.ro_n2,
                                                               B.ro_cap, 0);
    c->count_launch();
  }
  if (B.fused_tiles <= 0) {
    k_cg_p<T><<<dim3(ew_blocks(N), (unsigned)R), 256, 0, c->s>>>(N, z_of(B), B.p,
                                                                  B.st);
    c->count_launch();
  }
  COLA_CUDA(cudaGetLastError());
}

// x += the ring's kPRing updates (deferred-x mode).
template <typename T>
static void cg_flush_x(Ctx* c, CgBufs<T>& B, int64_t N, int64_t R, int nblk) {
  if constexpr (std::is_same<T, float>::value) {
    PRing ring;
    for (int s = 0; s < kPRing; ++s) ring.p[s] = (const float4*)B.pp[s];
    k_cg_xbatch<<<rows_grid(N, R, nblk), 256, 0, c->s>>>(N / 4, (float4*)B.x, ring, B.alpha_hist,
                                                          R, nblk);
    c->count_launch();
  }
}

// Runs `chunk` iterations as one CUDA graph (captured on first use).  In
// deferred-x mode the chunk is a multiple of kPRing and ends with x current.
template <typename T>
static void cg_chunk(Ctx* c, const cola_linop* op, CgBufs<T>& B, int64_t N, int64_t R, int nblk,
                     int prec, double delta2, int refine, int chunk, const std::string& key) {
  auto it = c->graphs.find(key);
  if (it == c->graphs.end() || it->second.generation != c->ws.generation) {
    if (it != c->graphs.end()) {
      cudaGraphExecDestroy(it->second.exec);
      c->graphs.erase(it);
    }
    cudaGraph_t g;
    COLA_CUDA(cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal));
    c->capturing = true;
    c->captured = 0;
    const uint64_t gen0 = c->ws.generation;
    try {
      for (int i = 0; i < chunk; ++i) {
        cg_iteration<T>(c, op, B, N, R, nblk, prec, delta2, refine, B.defer_x);
        if (B.defer_x && (i + 1) % kPRing == 0) cg_flush_x<T>(c, B, N, R, nblk);
      }
    } catch (...) {
      c->capturing = false;
      cudaStreamEndCapture(c->s, &g);
      throw;
    }
    c->capturing = false;
    COLA_CUDA(cudaStreamEndCapture(c->s, &g));
    COLA_REQUIRE(gen0 == c->ws.generation, COLA_ERR_CUDA,
                 "internal: workspace moved during graph capture");
    GraphEntry e;
    COLA_CUDA(cudaGraphInstantiate(&e.exec, g, 0));
    cudaGraphDestroy(g);
    e.kernels = c->captured;
    e.generation = c->ws.generation;
    it = c->graphs.emplace(key, e).first;
  }
  COLA_CUDA(cudaGraphLaunch(it->second.exec, c->s));
  c->launches += it->second.kernels;
}

template <typename T>
static cola_status cg_run(Ctx* c, cola_linop* op, const void* Bin, void* Xout, int64_t R,
                          const cola_cg_opts& o, cola_cg_info* info, bool transpose_unused) {
  (void)transpose_unused;
  const int64_t N = op->rows;
  const int prec = o.precision;
  const bool refine = (prec != COLA_PREC_F64) && o.refine;
  const int nblk = dot_blocks(N);
  auto& ws = c->ws;
  CgBufs<T> B{};
  B.x = (T*)ws.get("cg.x", sizeof(T) * N * R);
  B.r = (T*)ws.get("cg.r", sizeof(T) * N * R);
  for (int s = 0; s < kPRing; ++s) B.pp[s] = nullptr;
  B.pp[0] = (T*)ws.get("cg.p", sizeof(T) * N * R);
  B.cur = 0;
  B.p = B.pp[0];
  B.Ap = (T*)ws.get("cg.Ap", sizeof(T) * N * R);
  B.z = (o.jacobi || o.kron_precond) ? (T*)ws.get("cg.z", sizeof(T) * N * R) : nullptr;
  B.part_rz = (double*)ws.get("cg.prz", 8 * nblk * R);
  B.part_rr = (double*)ws.get("cg.prr", 8 * nblk * R);
  B.dotp = (double*)ws.get("cg.dotp", 8 * nblk * R);
  B.dotv = (double*)ws.get("cg.dotv", 8 * R);
  B.st = (CgState*)ws.get("cg.st", sizeof(CgState) * R);
  B.beta_vec = (double*)ws.get("cg.beta", 8 * R);
  B.fused_tiles = (prec == COLA_PREC_MIXED && sizeof(T) == 4) ? kron_tc_tiles_per_rhs(op) : 0;
  if (B.fused_tiles > 0) {
    for (int s = 1; s < kPRing; ++s) {
      char nm[16];
      snprintf(nm, sizeof nm, "cg.p%d", s + 1);
      B.pp[s] = (T*)ws.get(nm, sizeof(T) * N * R);
    }
    B.alpha_hist = (double*)ws.get("cg.ahist", 8 * kPRing * R);
    B.defer_x = sizeof(T) == 4 && N % 4 == 0;
  }
  B.tile_dot = B.fused_tiles > 0 ? (double*)ws.get("cg.tdot", 8 * 8 * B.fused_tiles * R) : nullptr;
  B.ro_cap = o.reorth_residuals;
  if (B.ro_cap > 0) {
    B.roQ = (T*)ws.get("cg.roQ", sizeof(T) * (size_t)N * R * B.ro_cap);
    B.ro_n2 = (double*)ws.get("cg.ron2", 8 * (size_t)R * B.ro_cap);
    B.ro_c = (double*)ws.get("cg.roc", 8 * (size_t)R * B.ro_cap);
    B.ro_k = (int*)ws.get("cg.rok", 4 * R);
  }
  COLA_CUDA(cudaMemsetAsync(B.beta_vec, 0, 8 * R, c->s));
  double* bb = (double*)ws.get("cg.bb", 8 * R);
  double* rr64 = (double*)ws.get("cg.rr64", 8 * R);
  double* dp64 = (double*)ws.get("cg.dp64", 8 * dot_blocks(N) * R);
  const bool io64 = (prec == COLA_PREC_F64) || refine;

  VectorTermsScope vterms(c, o.split_vector_terms);
  prepare_leaves(c, op, prec, o.split_factor_terms);
  if (refine) prepare_leaves(c, op, COLA_PREC_F64, o.split_factor_terms);

  // Jacobi preconditioner M = Diag(A) (Diag rules).
  if (o.jacobi) {
    double* d64 = (double*)ws.get("cg.diag64", 8 * N);
    prepare_leaves(c, op, COLA_PREC_F64, 0);
    diagonal<double>(c, op, d64, 0);
    B.invd = (T*)ws.get("cg.invd", sizeof(T) * N);
    if (sizeof(T) == 4)
      k_invert<<<ew_blocks(N), 256, 0, c->s>>>(N, d64, (float*)B.invd, nullptr);
    else
      k_invert<<<ew_blocks(N), 256, 0, c->s>>>(N, d64, nullptr, (double*)B.invd);
    c->count_launch();
  }
  // Kronecker preconditioner M = c_k Kron + c_d mean(d) I (Table 3 Inverse of Kron)
  if (o.kron_precond) {
    B.kprec = kron_precond_setup(c, op, &B.kp, R, prec, o.split_factor_terms);
    COLA_REQUIRE(B.kprec, COLA_ERR_UNSUPPORTED,
                 "kron_precond takes c_k Kron(K_1..K_d) + c_d Diag(d) with square dense factors");
  }

  if (refine) {
    B.x64 = (double*)ws.get("cg.x64", 8 * N * R);
    B.b64 = (double*)ws.get("cg.b64", 8 * N * R);
    B.r64 = (double*)ws.get("cg.r64", 8 * N * R);
    COLA_CUDA(cudaMemcpyAsync(B.b64, Bin, 8 * N * R, cudaMemcpyDeviceToDevice, c->s));
    if (o.x0_given)
      COLA_CUDA(cudaMemcpyAsync(B.x64, Xout, 8 * N * R, cudaMemcpyDeviceToDevice, c->s));
    else
      fill_zero<double>(c, B.x64, N * R);
    COLA_CUDA(cudaMemcpyAsync(B.r64, B.b64, 8 * N * R, cudaMemcpyDeviceToDevice, c->s));
    if (o.x0_given) apply<double>(c, op, B.x64, B.r64, R, -1.0, 1.0, 1, false, COLA_PREC_F64);
    dots<double>(c, B.b64, B.b64, N, R, dp64, bb);
    dots<double>(c, B.r64, B.r64, N, R, dp64, rr64);
    fill_zero<T>(c, B.x, N * R);
  } else {
    COLA_CUDA(cudaMemcpyAsync(B.r, Bin, sizeof(T) * N * R, cudaMemcpyDeviceToDevice, c->s));
    dots<T>(c, B.r, B.r, N, R, B.dotp, bb);
    if (o.x0_given) {
      COLA_CUDA(cudaMemcpyAsync(B.x, Xout, sizeof(T) * N * R, cudaMemcpyDeviceToDevice, c->s));
      apply<T>(c, op, B.x, B.r, R, -1.0, 1.0, 1, false, prec);
    } else {
      fill_zero<T>(c, B.x, N * R);
    }
  }
  k_refresh<T><<<rows_grid(N, R, nblk), 256, 0, c->s>>>(N, refine ? B.r64 : nullptr, B.r, B.invd,
                                                         B.z, nblk, B.part_rz, B.part_rr);
  c->count_launch();
  precond_z<T>(c, B, N, R, nblk);
  k_cg_restate<<<(unsigned)((R + 127) / 128), 128, 0, c->s>>>(
      B.st, B.part_rz, B.part_rr, nblk, R, refine ? rr64 : nullptr, bb, o.tol, 1, nullptr);
  c->count_launch();
  if (B.ro_cap > 0) ro_restart<T>(c, B, N, R, nblk);
  k_copy_active<T><<<dim3(ew_blocks(N), (unsigned)R), 256, 0, c->s>>>(N, z_of(B), B.p,
                                                                      B.st);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());

  CgState* hst = (CgState*)c->host_pinned(sizeof(CgState) * R);
  auto read_state = [&] {
    COLA_CUDA(cudaMemcpyAsync(hst, B.st, sizeof(CgState) * R, cudaMemcpyDeviceToHost, c->s));
    COLA_CUDA(cudaStreamSynchronize(c->s));
  };
  const double delta2 = o.reliable_delta * o.reliable_delta;
  // the fused path cycles through kPRing p buffers, so a graph chunk holds a
  // multiple of kPRing iterations: it starts and ends on the same buffer, and
  // in deferred-x mode x is current at its end
  int chunk = std::max(1, o.graph_chunk);
  // the preconditioned recursion converges within a few iterations: short
  // chunks keep the replacements (and restarts) close behind it
  if (B.kprec) chunk = std::min(chunk, kPRing);
  if (B.fused_tiles > 0) chunk = (chunk + kPRing - 1) / kPRing * kPRing;
  // everything a captured kernel bakes in is part of the graph key
  auto graph_key = [&] {
    char extra[128];
    snprintf(extra, sizeof extra, ":%c:d%.17g:s%d%d:p%d:o%d", sizeof(T) == 8 ? 'd' : 'f',
             delta2, o.split_factor_terms, o.split_vector_terms, B.cur, B.ro_cap);
    return key_of("cg", op, R, prec, (refine ? 1 : 0) | (o.jacobi ? 2 : 0) | (o.kron_precond ? 4 : 0) | (chunk << 3),
                  0) +
           extra;
  };
  int64_t iters = 0;
  int updates = 0;
  bool defer = false;   // replacements wait for half of the right-hand sides
  double iter_s = 0.0;  // host time per iteration of the fastest chunk so far
  // COLA_TRACE=1 prints the worst relative residual of the active right-hand
  // sides after every chunk and every FP64 replacement (stderr).
  const char* tr_env = getenv("COLA_TRACE");
  const bool trace = tr_env && tr_env[0] == '1';
  auto trace_line = [&](const char* what) {
    if (!trace) return;
    double worst = 0.0, worst64 = 0.0;
    int act = 0;
    for (int64_t r = 0; r < R; ++r) {
      if (!hst[r].active) continue;
      ++act;
      if (hst[r].bb > 0) {
        worst = std::max(worst, std::sqrt(std::max(hst[r].rr, 0.0) / hst[r].bb));
        worst64 = std::max(worst64, std::sqrt(std::max(hst[r].rr64, 0.0) / hst[r].bb));
      }
    }
    fprintf(stderr, "[cola cg] %s iter %lld active %d recursive %.3e true %.3e updates %d\n", what,
            (long long)iters, act, worst, worst64, updates);
  };
  read_state();
  bool any_active = false;
  for (int64_t r = 0; r < R; ++r) any_active |= hst[r].active != 0;
  // one eager iteration sizes every workspace buffer before capture
  if (any_active && o.maxiter > 0) {
    cg_iteration<T>(c, op, B, N, R, nblk, prec, delta2, refine ? 1 : 0, false);
    iters = 1;
  }
  for (int verify = 0;; ++verify) {
  while (any_active) {
    if (iters >= o.maxiter) break;
    const auto tc0 = std::chrono::steady_clock::now();
    cg_chunk<T>(c, op, B, N, R, nblk, prec, delta2, refine ? 1 : 0, chunk, graph_key());
    iters += chunk;
    read_state();
    {
      const double t = std::chrono::duration<double>(std::chrono::steady_clock::now() - tc0)
                           .count() / chunk;
      iter_s = iter_s > 0.0 ? std::min(iter_s, t) : t;
    }
    trace_line("chunk");
    // A replacement refreshes every right-hand side with one FP64 MVM of the
    // whole block.  Where that costs more than kDeferRatio iterations (large
    // factors: FP64 runs at a small fraction of the tensor rate on this GPU)
    // it waits until at least half of the active right-hand sides ask for
    // one, the others iterating meanwhile (a right-hand side whose recursion
    // ran 1e6-fold ahead pauses, and a pause triggers it); otherwise the first
    // request triggers it, which keeps the recursions closest to the true
    // residuals (fewest iterations).  Decided once per solve from the host
    // time of the first replacement and of the fastest chunk.
    int nact = 0, nflag = 0;
    bool paused = false;
    for (int64_t r = 0; r < R; ++r) {
      if (!hst[r].active) continue;
      ++nact;
      nflag += hst[r].flag ? 1 : 0;
      paused |= hst[r].paused != 0;
    }
    any_active = nact > 0;
    const bool flag = paused || (defer ? (nflag > 0 && 2 * nflag >= nact) : nflag > 0);
    if (refine && (flag || !any_active) && updates < o.max_updates) {
      const auto tr0 = std::chrono::steady_clock::now();
      // FP64 residual replacement: x64 += x; r64 = b - A x64; r = (T) r64.
      k_accum_x<T><<<ew_blocks(N * R), 256, 0, c->s>>>(N * R, B.x64, B.x);
      c->count_launch();
      COLA_CUDA(cudaMemcpyAsync(B.r64, B.b64, 8 * N * R, cudaMemcpyDeviceToDevice, c->s));
      apply<double>(c, op, B.x64, B.r64, R, -1.0, 1.0, 1, false, COLA_PREC_F64);
      dots<double>(c, B.r64, B.r64, N, R, dp64, rr64);
      k_refresh<T><<<rows_grid(N, R, nblk), 256, 0, c->s>>>(N, B.r64, B.r, B.invd, B.z, nblk,
                                                             B.part_rz, B.part_rr);
      c->count_launch();
      precond_z<T>(c, B, N, R, nblk);
      k_cg_restate<<<(unsigned)((R + 127) / 128), 128, 0, c->s>>>(
          B.st, B.part_rz, B.part_rr, nblk, R, rr64, bb, o.tol, 0, B.beta_vec);
      c->count_launch();
      k_cg_restart_p<T><<<dim3(ew_blocks(N), (unsigned)R), 256, 0, c->s>>>(N, z_of(B), B.p,
                                                                            B.st);
      c->count_launch();
      ++updates;
      read_state();
      if (updates == 1 && iter_s > 0.0) {
        const double t_repl =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - tr0).count();
        defer = t_repl > kDeferRatio * iter_s;
      }
      trace_line("update");
      any_active = false;
      for (int64_t r = 0; r < R; ++r) any_active |= hst[r].active != 0;
    }
    if (refine && updates >= o.max_updates) break;
  }
    // Without refinement the recursive residual decided convergence; check the
    // true residual b - A x and continue where it still misses the tolerance.
    if (refine || iters >= o.maxiter || verify >= o.max_updates) break;
    COLA_CUDA(cudaMemcpyAsync(B.r, Bin, sizeof(T) * N * R, cudaMemcpyDeviceToDevice, c->s));
    apply<T>(c, op, B.x, B.r, R, -1.0, 1.0, 1, false, prec);
    k_refresh<T><<<rows_grid(N, R, nblk), 256, 0, c->s>>>(N, nullptr, B.r, B.invd, B.z, nblk,
                                                           B.part_rz, B.part_rr);
    c->count_launch();
    precond_z<T>(c, B, N, R, nblk);
    k_cg_verify<<<(unsigned)((R + 127) / 128), 128, 0, c->s>>>(B.st, B.part_rz, B.part_rr, nblk,
                                                               R, B.beta_vec);
    c->count_launch();
    read_state();
    trace_line("verify");
    any_active = false;
    for (int64_t r = 0; r < R; ++r) any_active |= hst[r].active != 0;
    if (!any_active) break;
    // the true residual starts a new store of residuals
    if (B.ro_cap > 0) ro_restart<T>(c, B, N, R, nblk);
    k_copy_active<T><<<dim3(ew_blocks(N), (unsigned)R), 256, 0, c->s>>>(N, z_of(B),
                                                                        B.p, B.st);
    c->count_launch();
  }

  // Final solution and true residual.
  cola_status result = COLA_OK;
  if (refine) {
    k_accum_x<T><<<ew_blocks(N * R), 256, 0, c->s>>>(N * R, B.x64, B.x);
    c->count_launch();
    COLA_CUDA(cudaMemcpyAsync(Xout, B.x64, 8 * N * R, cudaMemcpyDeviceToDevice, c->s));
    COLA_CUDA(cudaMemcpyAsync(B.r64, B.b64, 8 * N * R, cudaMemcpyDeviceToDevice, c->s));
    apply<double>(c, op, B.x64, B.r64, R, -1.0, 1.0, 1, false, COLA_PREC_F64);
    dots<double>(c, B.r64, B.r64, N, R, dp64, rr64);
  } else {
    COLA_CUDA(cudaMemcpyAsync(Xout, B.x, sizeof(T) * N * R, cudaMemcpyDeviceToDevice, c->s));
    COLA_CUDA(cudaMemcpyAsync(B.r, Bin, sizeof(T) * N * R, cudaMemcpyDeviceToDevice, c->s));
    apply<T>(c, op, B.x, B.r, R, -1.0, 1.0, 1, false, prec);
    dots<T>(c, B.r, B.r, N, R, B.dotp, rr64);
  }
  if (prec == COLA_PREC_MIXED) tc_check_error(c);
  std::vector<double> hrr(R), hbb(R);
  COLA_CUDA(cudaMemcpyAsync(hrr.data(), rr64, 8 * R, cudaMemcpyDeviceToHost, c->s));
  COLA_CUDA(cudaMemcpyAsync(hbb.data(), bb, 8 * R, cudaMemcpyDeviceToHost, c->s));
  read_state();
  for (int64_t r = 0; r < R; ++r) {
    const double rel = hbb[r] > 0 ? std::sqrt(std::max(hrr[r], 0.0) / hbb[r]) : 0.0;
    int st = hst[r].status;
    if (st == 0 && !(rel <= o.tol * (refine || prec == COLA_PREC_F64 ? 1.0 : 10.0)))
      st = COLA_ERR_NOT_CONVERGED;
    if (st != 0 && result == COLA_OK) result = (cola_status)st;
    if (info) {
      info[r].iterations = hst[r].iters;
      info[r].rel_residual = rel;
      info[r].updates = hst[r].updates;
      info[r].status = st;
    }
  }
  (void)io64;
  return result;
}

cola_status cg_solve_impl(Ctx* c, const cola_linop* op, const void* B, void* X, int64_t R,
                          const cola_cg_opts& o, cola_cg_info* info) {
  cola_linop* m = const_cast<cola_linop*>(op);
  if (o.precision == COLA_PREC_F64) return cg_run<double>(c, m, B, X, R, o, info, false);
  return cg_run<float>(c, m, B, X, R, o, info, false);
}

void check_cg_args(const cola_linop* op, const cola_cg_opts* o, int64_t R) {
  COLA_REQUIRE(op->spd, COLA_ERR_INVALID_ARG, "CG needs an operator annotated spd (set_spd)");
  COLA_REQUIRE(op->rows == op->cols, COLA_ERR_SHAPE, "CG needs a square operator");
  COLA_REQUIRE(R >= 1, COLA_ERR_INVALID_ARG, "nrhs = %lld", (long long)R);
  COLA_REQUIRE(o->precision >= COLA_PREC_F64 && o->precision <= COLA_PREC_MIXED,
               COLA_ERR_INVALID_ARG, "precision %d", o->precision);
  COLA_REQUIRE(o->tol >= 0.0 && o->maxiter >= 0, COLA_ERR_INVALID_ARG, "tol/maxiter");
  COLA_REQUIRE(o->reorth_residuals >= 0 && o->reorth_residuals <= 4096, COLA_ERR_INVALID_ARG,
               "reorth_residuals = %d (0 .. 4096)", o->reorth_residuals);
  COLA_REQUIRE(o->reorth_residuals == 0 ||
                   (!o->jacobi && !o->kron_precond &&
                    (o->precision == COLA_PREC_F64 || !o->refine)),
               COLA_ERR_INVALID_ARG,
               "reorth_residuals takes an unpreconditioned solve without FP64 refinement");
  COLA_REQUIRE(o->split_factor_terms >= 1 && o->split_factor_terms <= 3 &&
                   o->split_vector_terms >= 1 && o->split_vector_terms <= 3,
               COLA_ERR_INVALID_ARG, "split terms must be 1..3");
  COLA_REQUIRE(!(o->jacobi && o->kron_precond), COLA_ERR_INVALID_ARG,
               "jacobi and kron_precond are exclusive");
}

// ------------------------------------------------------------- bilinear
void bilinear_entry(Ctx* c, const cola_linop* op, const void* U, const void* X,
                    const double* weights, int64_t R, int prec, void* const* grads,
                    int accumulate, int depth) {
  cola_linop* m = const_cast<cola_linop*>(op);
  std::vector<const cola_linop*> leaves;
  collect_leaves(op, leaves);
  const bool f64 = prec == COLA_PREC_F64;
  prepare_leaves(c, m, f64 ? COLA_PREC_F64 : COLA_PREC_F32, 0);
  const size_t es = f64 ? 8 : 4;
  const int64_t n_in = op->cols, n_out = op->rows;
  // weighted copy of U
  void* Uw = c->ws.get("bl.Uw", es * n_out * R);
  COLA_CUDA(cudaMemcpyAsync(Uw, U, es * n_out * R, cudaMemcpyDeviceToDevice, c->s));
  if (weights) {
    double* wd = (double*)c->ws.get("bl.w", 8 * R);
    COLA_CUDA(cudaMemcpyAsync(wd, weights, 8 * R, cudaMemcpyHostToDevice, c->s));
    if (f64)
      scale_rows<double>(c, (double*)Uw, n_out, R, wd);
    else
      scale_rows<float>(c, (float*)Uw, n_out, R, wd);
  }
  // per-leaf accumulators in working type
  std::vector<void*> acc(leaves.size(), nullptr);
  std::vector<int64_t> cnt(leaves.size(), 0);
  for (size_t l = 0; l < leaves.size(); ++l) {
    if (!grads[l]) continue;
    const cola_linop* f = leaves[l];
    int64_t elems = f->kind == LK_DENSE ? f->rows * f->cols
                    : f->kind == LK_DIAG ? (f->stride ? f->rows : 1)
                                         : f->rows * f->rank;
    cnt[l] = elems;
    char nm[32];
    snprintf(nm, sizeof nm, "bl.g%zu", l);
    acc[l] = c->ws.get(nm, es * elems);
    COLA_CUDA(cudaMemsetAsync(acc[l], 0, es * elems, c->s));
  }
  int li = 0;
  if (f64)
    bilinear<double>(c, op, (const double*)Uw, (const double*)X, R, 1.0, acc, li, depth + 1);
  else
    bilinear<float>(c, op, (const float*)Uw, (const float*)X, R, 1.0, acc, li, depth + 1);
  (void)n_in;
  // write / accumulate into the caller's buffers in the leaf dtype
  for (size_t l = 0; l < leaves.size(); ++l) {
    if (!grads[l]) continue;
    const cola_dtype dt = leaves[l]->dtype;
    if (!accumulate) COLA_CUDA(cudaMemsetAsync(grads[l], 0, (dt == COLA_F64 ? 8 : 4) * cnt[l], c->s));
    if (f64 && dt == COLA_F64)
      add_partials<double>(c, (const double*)acc[l], (double*)grads[l], cnt[l], 1, 1.0);
    else if (!f64 && dt == COLA_F32)
      add_partials<float>(c, (const float*)acc[l], (float*)grads[l], cnt[l], 1, 1.0);
    else if (f64) {
      float* t = (float*)c->ws.get("bl.cvt", 4 * cnt[l]);
      convert<double, float>(c, (const double*)acc[l], t, cnt[l]);
      add_partials<float>(c, t, (float*)grads[l], cnt[l], 1, 1.0);
    } else {
      double* t = (double*)c->ws.get("bl.cvt", 8 * cnt[l]);
      convert<float, double>(c, (const float*)acc[l], t, cnt[l]);
      add_partials<double>(c, t, (double*)grads[l], cnt[l], 1, 1.0);
    }
  }
}

}  // namespace cola

using namespace cola;

extern "C" {

void cola_cg_opts_default(cola_cg_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->tol = 1e-8;
  o->maxiter = 100000;
  o->precision = COLA_PREC_MIXED;
  o->refine = 1;
  o->reliable_delta = 0.1;
  o->max_updates = 200;
  o->split_factor_terms = 3;
  o->split_vector_terms = 3;
  o->graph_chunk = 64;
  o->jacobi = 0;
  o->x0_given = 0;
  o->kron_precond = 0;
  o->reorth_residuals = 0;
}

cola_status cola_cg_solve(cola_ctx* ctx, const cola_linop* op, const void* B, void* X,
                          int64_t nrhs, const cola_cg_opts* opts, cola_cg_info* info,
                          cola_stream stream) {
  cola_status result = COLA_OK;
  cola_status st = guard([&] {
    COLA_REQUIRE(ctx && op && B && X && opts, COLA_ERR_INVALID_ARG, "NULL argument");
    check_cg_args(op, opts, nrhs);
    StreamJoin j(ctx, stream);
    result = cg_solve_impl(ctx, op, B, X, nrhs, *opts, info);
    if (result != COLA_OK) set_error_message(result == COLA_ERR_NOT_CONVERGED
                                                 ? "CG did not reach tol for every RHS"
                                                 : "CG breakdown (p^T A p <= 0 or non-finite)");
  });
  return st != COLA_OK ? st : result;
}

cola_status cola_cg_solve_batched(cola_ctx* ctx, int32_t nsys, const cola_linop* const* ops,
                                  const void* const* B, void* const* X, const int64_t* nrhs,
                                  const cola_cg_opts* opts, cola_cg_info* info,
                                  cola_stream stream) {
  cola_status result = COLA_OK;
  cola_status st = guard([&] {
    COLA_REQUIRE(ctx && ops && B && X && nrhs && opts, COLA_ERR_INVALID_ARG, "NULL argument");
    COLA_REQUIRE(nsys >= 1, COLA_ERR_INVALID_ARG, "nsys = %d", nsys);
    for (int s = 0; s < nsys; ++s) {
      COLA_REQUIRE(ops[s] && B[s] && X[s], COLA_ERR_INVALID_ARG, "system %d: NULL argument", s);
      check_cg_args(ops[s], opts, nrhs[s]);
    }
    StreamJoin j(ctx, stream);
    result = batched_cg_impl(ctx, nsys, ops, B, X, nrhs, *opts, info);
  });
  return st != COLA_OK ? st : result;
}

cola_status cola_lanczos(cola_ctx* ctx, const cola_linop* op, const void* Q0, int64_t nvec,
                         int32_t m, int32_t prec, int32_t reorth, double* alpha, double* beta,
                         int32_t* m_eff, cola_stream stream) {
  return guard([&] {
    COLA_REQUIRE(ctx && op && Q0 && alpha && beta && m_eff, COLA_ERR_INVALID_ARG,
                 "NULL argument");
    COLA_REQUIRE(op->spd, COLA_ERR_INVALID_ARG, "Lanczos needs an operator annotated spd");
    COLA_REQUIRE(nvec >= 1 && m >= 1, COLA_ERR_INVALID_ARG, "nvec/m");
    COLA_REQUIRE(prec >= COLA_PREC_F64 && prec <= COLA_PREC_MIXED, COLA_ERR_INVALID_ARG,
                 "precision");
    COLA_REQUIRE(reorth >= 0 && reorth <= 2, COLA_ERR_INVALID_ARG, "reorth = %d (0, 1, 2)",
                 reorth);
    StreamJoin j(ctx, stream);
    lanczos_impl(ctx, op, Q0, nvec, m, prec, reorth, alpha, beta, m_eff);
  });
}

}  // extern "C"

namespace cola {

// MIXED Lanczos for A = c_k Kron + c_d s I with the recurrence fused into the
// tensor-core MVM: step j's first mode step forms q_j = w / beta_{j-1} (w =
// Q0 and the scale 1 / ||z|| at j = 0), its last mode step writes
// w = A q_j - beta_{j-1} q_{j-1} with the partials of alpha_j = q_j . w; one
// vector pass then forms w -= alpha_j q_j and ||w||^2, the same recurrence
// and breakdown test as the unfused loop.  false when the operator does not
// have this shape.
// The fused Lanczos step with unnormalised basis vectors v_j = beta_j q_j
// (slab-shaped operators): the first mode step forms v_j = w - alpha_{j-1}
// s_{j-1} v_{j-1} from the two streams and the partials of ||v_j||^2, so no
// separate pass subtracts alpha q and normalises; the slab kernel's epilogue
// applies s_j = 1 / beta_j.  The same recurrence as Algorithm 1 (Table 5)
// with the division by beta_j moved after the Kronecker product.
static void lanczos_unnormalised(Ctx* c, cola_linop* op, const float* Q0, int64_t nv, int m,
                                 double* alpha, double* beta, int* m_eff) {
  const int64_t N = op->rows;
  const int nblk = dot_blocks(N);
  auto& ws = c->ws;
  const int64_t tiles = kron_tc_tiles_per_rhs(op);  // slabs per right-hand side
  float* w = (float*)ws.get("lz.0", sizeof(float) * N * nv);
  float* vb[2] = {(float*)ws.get("lz.1", sizeof(float) * N * nv),
                  (float*)ws.get("lz.2", sizeof(float) * N * nv)};
  double* tdot = (double*)ws.get("lz.tdot", 8 * 8 * (size_t)tiles * nv);
  double* part = (double*)ws.get("lz.part", 8 * nblk * nv);
  double* nrm2 = (double*)ws.get("lz.nrm2", 8 * nv);
  double* a_cur = (double*)ws.get("lz.a", 8 * nv);
  double* b_cur = (double*)ws.get("lz.b", 8 * nv);
  double* coef = (double*)ws.get("lz.coef", 8 * nv);
  double* gam = (double*)ws.get("lz.gam", 8 * nv);
  double* sc[2] = {(double*)ws.get("lz.s0", 8 * nv), (double*)ws.get("lz.s1", 8 * nv)};
  LzState* st = (LzState*)ws.get("lz.st", sizeof(LzState) * nv);
  const unsigned vb_ = (unsigned)((nv + 127) / 128);
  COLA_CUDA(cudaMemsetAsync(alpha, 0, 8 * nv * m, c->s));
  COLA_CUDA(cudaMemsetAsync(beta, 0, 8 * nv * m, c->s));
  COLA_CUDA(cudaMemsetAsync(b_cur, 0, 8 * nv, c->s));
  COLA_CUDA(cudaMemsetAsync(gam, 0, 8 * nv, c->s));
  dots<float>(c, Q0, Q0, N, nv, part, nrm2);
  k_lz_init<<<vb_, 128, 0, c->s>>>(st, nrm2, nv, m);
  c->count_launch();
  k_lz_recip<<<vb_, 128, 0, c->s>>>(nv, nrm2, sc[0], 1);  // s_0 = 1 / ||z||
  c->count_launch();
  const double eps = 1e-6;
  // step 0: v_0 = z
  kron_tc_lanczos_step1(c, op, Q0, nullptr, nullptr, nullptr, nullptr, nv, 1);
  double* npart = nullptr;
  int64_t tiles1 = 0;
  int64_t t = kron_tc_lanczos_slab(c, op, Q0, Q0, gam, sc[0], w, tdot, nv, 1, 1);
  COLA_REQUIRE(t == tiles, COLA_ERR_UNSUPPORTED, "internal: fused Lanczos tile count");
  k_lz_alpha<<<(unsigned)nv, 256, 0, c->s>>>(st, tdot, (int)(8 * tiles), nv, 0, m, alpha, a_cur);
  c->count_launch();
  for (int j = 1; j < m; ++j) {
    const float* vprev = (j == 1) ? Q0 : vb[(j - 1) & 1];
    float* vj = vb[j & 1];
    double* s_prev = sc[(j - 1) & 1];
    double* s_new = sc[j & 1];
    k_lz_coef<<<vb_, 128, 0, c->s>>>(nv, a_cur, s_prev, coef);
    c->count_launch();
    if (!npart) {
      const cola_linop* kr = op->kids[0]->kind == LK_KRON ? op->kids[0] : op->kids[1];
      tiles1 = (kr->cols / kr->kids[0]->cols + 127) / 128;
      npart = (double*)ws.get("lz.npart", 8 * 8 * (size_t)tiles1 * nv);
    }
    const int64_t t1 = kron_tc_lanczos_step1(c, op, vprev, w, coef, vj, npart, nv, 1);
    COLA_REQUIRE(t1 == tiles1, COLA_ERR_UNSUPPORTED, "internal: fused Lanczos step-1 tiles");
    dot_final(c, npart, (int)(8 * tiles1), nv, nrm2);
    k_lz_beta<<<vb_, 128, 0, c->s>>>(st, nrm2, nv, j - 1, m, eps, beta, b_cur);
    c->count_launch();
    k_lz_scales<<<vb_, 128, 0, c->s>>>(nv, b_cur, s_prev, s_new, gam);
    c->count_launch();
    // the slab kernel walks its slabs backwards and the first mode step its
    // tiles forwards, so each starts on what the launch before it wrote last
    t = kron_tc_lanczos_slab(c, op, vj, vprev, gam, s_new, w, tdot, nv, 1, 1);
    COLA_REQUIRE(t == tiles, COLA_ERR_UNSUPPORTED, "internal: fused Lanczos tile count");
    k_lz_alpha<<<(unsigned)nv, 256, 0, c->s>>>(st, tdot, (int)(8 * tiles), nv, j, m, alpha,
                                               a_cur);
    c->count_launch();
  }
  // the last step: every right-hand side still running took all m steps
  k_lz_beta<<<vb_, 128, 0, c->s>>>(st, nrm2, nv, m - 1, m, eps, beta, b_cur);
  c->count_launch();
  k_lz_meff<<<vb_, 128, 0, c->s>>>(st, nv, m_eff);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
}

static bool lanczos_fused(Ctx* c, cola_linop* op, const float* Q0, int64_t nv, int m,
                          double* alpha, double* beta, int* m_eff) {
  const int64_t tiles = kron_tc_tiles_per_rhs(op);
  if (tiles <= 0) return false;
  if (kron_tc_lanczos_unnormalised(op)) {
    lanczos_unnormalised(c, op, Q0, nv, m, alpha, beta, m_eff);
    return true;
  }
  const int64_t N = op->rows;
  const int nblk = dot_blocks(N);
  auto& ws = c->ws;
  float* w = (float*)ws.get("lz.0", sizeof(float) * N * nv);
  float* q[2] = {(float*)ws.get("lz.1", sizeof(float) * N * nv),
                 (float*)ws.get("lz.2", sizeof(float) * N * nv)};
  double* tdot = (double*)ws.get("lz.tdot", 8 * 8 * (size_t)tiles * nv);
  double* part = (double*)ws.get("lz.part", 8 * nblk * nv);
  double* nrm2 = (double*)ws.get("lz.nrm2", 8 * nv);
  double* a_cur = (double*)ws.get("lz.a", 8 * nv);
  double* b_cur = (double*)ws.get("lz.b", 8 * nv);
  double* scale = (double*)ws.get("lz.scale", 8 * nv);
  LzState* st = (LzState*)ws.get("lz.st", sizeof(LzState) * nv);
  const unsigned vb = (unsigned)((nv + 127) / 128);
  COLA_CUDA(cudaMemsetAsync(alpha, 0, 8 * nv * m, c->s));
  COLA_CUDA(cudaMemsetAsync(beta, 0, 8 * nv * m, c->s));
  COLA_CUDA(cudaMemsetAsync(b_cur, 0, 8 * nv, c->s));
  dots<float>(c, Q0, Q0, N, nv, part, nrm2);
  k_lz_init<<<vb, 128, 0, c->s>>>(st, nrm2, nv, m);
  c->count_launch();
  k_lz_recip<<<vb, 128, 0, c->s>>>(nv, nrm2, scale, 1);
  c->count_launch();
  const double eps = 1e-6;
  for (int j = 0; j < m; ++j) {
    float* qj = q[j & 1];
    const float* qprev = q[(j + 1) & 1];
    const int64_t t = kron_tc_lanczos_mvm(c, op, j == 0 ? Q0 : w, scale, qj, qprev, b_cur, w,
                                          tdot, nv, 1);
    COLA_REQUIRE(t == tiles, COLA_ERR_UNSUPPORTED, "internal: fused Lanczos tile count");
    k_lz_alpha<<<(unsigned)nv, 256, 0, c->s>>>(st, tdot, (int)(8 * tiles), nv, j, m, alpha,
                                               a_cur);
    c->count_launch();
    k_lz_b<float><<<rows_grid(N, nv, nblk), 256, 0, c->s>>>(N, w, qj, a_cur, nblk, part, 1);
    c->count_launch();
    dot_final(c, part, nblk, nv, nrm2);
    k_lz_beta<<<vb, 128, 0, c->s>>>(st, nrm2, nv, j, m, eps, beta, b_cur);
    c->count_launch();
    k_lz_recip<<<vb, 128, 0, c->s>>>(nv, b_cur, scale, 0);
    c->count_launch();
  }
  k_lz_meff<<<vb, 128, 0, c->s>>>(st, nv, m_eff);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
  return true;
}

template <typename T>
static void lanczos_run(Ctx* c, cola_linop* op, const T* Q0, int64_t nv, int m, int prec,
                        int reorth, double* alpha, double* beta, int* m_eff) {
  const int64_t N = op->rows;
  const int nblk = dot_blocks(N);
  auto& ws = c->ws;
  // MIXED: the context's split terms (cola_set_split_terms), as cola_matvec
  prepare_leaves(c, op, prec, c->split_factor_terms);
  if constexpr (sizeof(T) == 4) {
    if (prec == COLA_PREC_MIXED && !reorth &&
        lanczos_fused(c, op, (const float*)Q0, nv, m, alpha, beta, m_eff))
      return;
  }
  T* bufs[3];
  bufs[0] = (T*)ws.get("lz.0", sizeof(T) * N * nv);
  bufs[1] = (T*)ws.get("lz.1", sizeof(T) * N * nv);
  bufs[2] = (T*)ws.get("lz.2", sizeof(T) * N * nv);
  T* Qall = reorth ? (T*)ws.get("lz.Q", sizeof(T) * N * nv * m) : nullptr;
  T* H = reorth ? (T*)ws.get("lz.H", sizeof(T) * nv * m) : nullptr;
  double* part = (double*)ws.get("lz.part", 8 * nblk * nv);
  double* nrm2 = (double*)ws.get("lz.nrm2", 8 * nv);
  double* a_cur = (double*)ws.get("lz.a", 8 * nv);
  double* b_cur = (double*)ws.get("lz.b", 8 * nv);
  LzState* st = (LzState*)ws.get("lz.st", sizeof(LzState) * nv);
  COLA_CUDA(cudaMemsetAsync(alpha, 0, 8 * nv * m, c->s));
  COLA_CUDA(cudaMemsetAsync(beta, 0, 8 * nv * m, c->s));
  T *qprev = bufs[0], *q = bufs[1], *w = bufs[2];
  fill_zero<T>(c, qprev, N * nv);
  dots<T>(c, Q0, Q0, N, nv, part, nrm2);
  k_lz_init<<<(unsigned)((nv + 127) / 128), 128, 0, c->s>>>(st, nrm2, nv, m);
  c->count_launch();
  k_lz_scale<T><<<dim3(ew_blocks(N), (unsigned)nv), 256, 0, c->s>>>(N, Q0, q, nrm2);
  c->count_launch();
  const double eps = (prec == COLA_PREC_F64) ? 1e-10 : 1e-6;
  for (int j = 0; j < m; ++j) {
    apply<T>(c, op, q, w, nv, 1.0, 0.0, 1, false, prec);
    k_lz_a<T><<<rows_grid(N, nv, nblk), 256, 0, c->s>>>(N, w, qprev, q, st, nblk, part);
    c->count_launch();
    k_lz_alpha<<<(unsigned)nv, 256, 0, c->s>>>(st, part, nblk, nv, j, m, alpha, a_cur);
    c->count_launch();
    k_lz_b<T><<<rows_grid(N, nv, nblk), 256, 0, c->s>>>(N, w, q, a_cur, nblk, part,
                                                         reorth ? 0 : 1);
    c->count_launch();
    if (reorth) {
      COLA_CUDA(cudaMemcpy2DAsync(Qall + (int64_t)j * N, sizeof(T) * N * m, q, sizeof(T) * N,
                                  sizeof(T) * N, nv, cudaMemcpyDeviceToDevice, c->s));
      for (int pass = 0; pass < 2; ++pass) {
        // H[v][0..j] = Q_v[0..j] w_v ; w_v -= H[v] Q_v
        gemm<T>(c, 1, j + 1, N, 1.0, w, N, 1, N, Qall, 1, N, N * m, 0.0, H, j + 1, 1, m, nv);
        gemm<T>(c, 1, N, j + 1, -1.0, H, j + 1, 1, m, Qall, N, 1, N * m, 1.0, w, N, 1, N, nv);
      }
      dots<T>(c, w, w, N, nv, part, nrm2);
    } else {
      dot_final(c, part, nblk, nv, nrm2);
    }
    k_lz_beta<<<(unsigned)((nv + 127) / 128), 128, 0, c->s>>>(st, nrm2, nv, j, m, eps, beta,
                                                             b_cur);
    c->count_launch();
    k_lz_next<T><<<dim3(ew_blocks(N), (unsigned)nv), 256, 0, c->s>>>(N, w, b_cur);
    c->count_launch();
    T* old = qprev;
    qprev = q;
    q = w;
    w = old;
  }
  k_lz_meff<<<(unsigned)((nv + 127) / 128), 128, 0, c->s>>>(st, nv, m_eff);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
}

void lanczos_impl(Ctx* c, const cola_linop* op, const void* Q0, int64_t nv, int m, int prec,
                  int reorth, double* alpha, double* beta, int* m_eff) {
  cola_linop* mo = const_cast<cola_linop*>(op);
  if (reorth == 2) {  // Householder basis (Algorithm 2)
    householder_lanczos(c, op, Q0, nv, m, prec, alpha, beta, m_eff);
    return;
  }
  if (prec == COLA_PREC_F64)
    lanczos_run<double>(c, mo, (const double*)Q0, nv, m, prec, reorth, alpha, beta, m_eff);
  else
    lanczos_run<float>(c, mo, (const float*)Q0, nv, m, prec, reorth, alpha, beta, m_eff);
}

}  // namespace cola

// ===================================================================== SLQ
namespace cola {

void slq_impl(Ctx* c, const cola_linop* op, int nprobes, int m, uint64_t seed,
              const void* probes, int prec, int reorth, double* logdet, double* std_err,
              double* per_probe, int* clamped) {
  const int64_t N = op->rows;
  const bool f64 = prec == COLA_PREC_F64;
  const size_t es = f64 ? 8 : 4;
  auto& ws = c->ws;
  void* Z = (void*)probes;
  if (!probes) {
    Z = ws.get("slq.Z", es * N * nprobes);
    rademacher(c, seed, 0, N * nprobes, Z, f64 ? COLA_F64 : COLA_F32);
  }
  double* alpha = (double*)ws.get("slq.alpha", 8 * (size_t)nprobes * m);
  double* beta = (double*)ws.get("slq.beta", 8 * (size_t)nprobes * m);
  int* meff = (int*)ws.get("slq.meff", 4 * nprobes);
  double* zn = (double*)ws.get("slq.zn", 8 * nprobes);
  double* part = (double*)ws.get("slq.part", 8 * (size_t)dot_blocks(N) * nprobes);
  lanczos_impl(c, op, Z, nprobes, m, prec, reorth, alpha, beta, meff);
  if (f64)
    dots<double>(c, (const double*)Z, (const double*)Z, N, nprobes, part, zn);
  else
    dots<float>(c, (const float*)Z, (const float*)Z, N, nprobes, part, zn);
  // the tridiagonal matrices T_m (a few KB) come back to the host, where the
  // quadrature runs in FP64, probes spread over the host's cores
  std::vector<double> ha((size_t)nprobes * m), hb((size_t)nprobes * m), hz(nprobes);
  std::vector<int> hm(nprobes);
  COLA_CUDA(cudaMemcpyAsync(ha.data(), alpha, 8 * ha.size(), cudaMemcpyDeviceToHost, c->s));
  COLA_CUDA(cudaMemcpyAsync(hb.data(), beta, 8 * hb.size(), cudaMemcpyDeviceToHost, c->s));
  COLA_CUDA(cudaMemcpyAsync(hz.data(), zn, 8 * hz.size(), cudaMemcpyDeviceToHost, c->s));
  COLA_CUDA(cudaMemcpyAsync(hm.data(), meff, 4 * hm.size(), cudaMemcpyDeviceToHost, c->s));
  COLA_CUDA(cudaStreamSynchronize(c->s));
  std::vector<QuadResult> qr(nprobes);
  const int nthreads = (int)std::max<int64_t>(
      1, std::min<int64_t>(nprobes, std::max(1u, std::thread::hardware_concurrency())));
  auto work = [&](int t0) {
    for (int v = t0; v < nprobes; v += nthreads)
      qr[v] = slq_quadrature(ha.data() + (size_t)v * m, hb.data() + (size_t)v * m, hm[v], hz[v]);
  };
  if (nthreads == 1) {
    work(0);
  } else {
    std::vector<std::thread> pool;
    for (int t = 0; t < nthreads; ++t) pool.emplace_back(work, t);
    for (auto& th : pool) th.join();
  }
  std::vector<double> vals(nprobes);
  int ncl = 0;
  for (int v = 0; v < nprobes; ++v) {
    COLA_REQUIRE(qr[v].converged, COLA_ERR_NOT_CONVERGED,
                 "SLQ: the QR iteration of probe %d's tridiagonal matrix did not converge", v);
    vals[v] = qr[v].value;
    ncl += qr[v].clamped;
  }
  // mean and sample standard error over the probes, summed in probe order
  double mean = 0.0;
  for (int v = 0; v < nprobes; ++v) mean += vals[v];
  mean /= nprobes;
  double var = 0.0;
  for (int v = 0; v < nprobes; ++v) var += (vals[v] - mean) * (vals[v] - mean);
  if (per_probe) {
    COLA_CUDA(cudaMemcpyAsync(per_probe, vals.data(), 8 * vals.size(), cudaMemcpyHostToDevice,
                              c->s));
    COLA_CUDA(cudaStreamSynchronize(c->s));
  }
  if (logdet) *logdet = mean;
  if (std_err) *std_err = nprobes > 1 ? std::sqrt(var / (nprobes - 1) / nprobes) : 0.0;
  if (clamped) *clamped = ncl;
}

}  // namespace cola

extern "C" cola_status cola_slq_logdet(cola_ctx* ctx, const cola_linop* op, int32_t nprobes,
                                       int32_t m, uint64_t seed, const void* probes,
                                       int32_t prec, int32_t reorth, double* logdet,
                                       double* std_err, double* per_probe, int32_t* clamped,
                                       cola_stream stream) {
  return cola::guard([&] {
    COLA_REQUIRE(ctx && op && logdet && std_err, COLA_ERR_INVALID_ARG, "NULL argument");
    COLA_REQUIRE(op->spd, COLA_ERR_INVALID_ARG, "SLQ needs an operator annotated spd");
    COLA_REQUIRE(nprobes >= 1 && m >= 1, COLA_ERR_INVALID_ARG, "nprobes/m");
    COLA_REQUIRE(prec >= COLA_PREC_F64 && prec <= COLA_PREC_MIXED, COLA_ERR_INVALID_ARG,
                 "precision");
    COLA_REQUIRE(reorth >= 0 && reorth <= 2, COLA_ERR_INVALID_ARG, "reorth = %d (0, 1, 2)",
                 reorth);
    cola::StreamJoin j(ctx, stream);
    cola::slq_impl(ctx, op, nprobes, m, seed, probes, prec, reorth, logdet, std_err, per_probe,
                   clamped);
  });
}
