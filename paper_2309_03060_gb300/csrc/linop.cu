// Operator tree and its MVM (CoLA Sec. 3.1-3.2), Diag rules (App. A.1.4),
// transpose rules (App. A.1.5) and leaf gradients of bilinear forms
// (App. B.2), plus the context, workspace and error plumbing of the C ABI.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>

#include "internal.h"

namespace cola {

// ------------------------------------------------------------------ errors
static thread_local std::string g_last_error;

void set_error_message(const char* msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }

void fail(cola_status st, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  throw Failure{st};
}

// --------------------------------------------------------------- workspace
void* Workspace::get(const std::string& name, size_t bytes) {
  bytes = std::max<size_t>(bytes, 256);
  auto it = bufs.find(name);
  if (it != bufs.end() && it->second.bytes >= bytes) return it->second.p;
  if (it != bufs.end()) {
    COLA_CUDA(cudaFree(it->second.p));
    bufs.erase(it);
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(COLA_ERR_OOM, "workspace '%s': cudaMalloc(%zu) failed: %s", name.c_str(), bytes,
         cudaGetErrorString(e));
  }
  bufs[name] = Buf{p, bytes};
  ++generation;
  return p;
}

void Workspace::release_all() {
  for (auto& kv : bufs) cudaFree(kv.second.p);
  bufs.clear();
  ++generation;
}

void* Ctx::host_pinned(size_t bytes) {
  if (bytes > pinned_bytes) {
    if (pinned) cudaFreeHost(pinned);
    pinned = nullptr;
    COLA_CUDA(cudaHostAlloc(&pinned, bytes, cudaHostAllocDefault));
    pinned_bytes = bytes;
  }
  return pinned;
}

// A caller that already works on the context's own stream needs no join.
StreamJoin::StreamJoin(Ctx* c_, cola_stream s) : c(c_), user((cudaStream_t)s) {
  COLA_CUDA(cudaSetDevice(c->device));
  if (user == c->s) return;
  COLA_CUDA(cudaEventRecord(c->ev_a, user));
  COLA_CUDA(cudaStreamWaitEvent(c->s, c->ev_a, 0));
}

StreamJoin::~StreamJoin() {
  if (user == c->s) return;
  cudaEventRecord(c->ev_b, c->s);
  cudaStreamWaitEvent(user, c->ev_b, 0);
}

// ------------------------------------------------------------ leaf helpers
static size_t dtype_size(cola_dtype d) { return d == COLA_F64 ? 8 : 4; }

template <typename T>
static cola_dtype dtype_of();
template <>
cola_dtype dtype_of<float>() { return COLA_F32; }
template <>
cola_dtype dtype_of<double>() { return COLA_F64; }

template <typename T>
const T* leaf_ptr(const cola_linop* op, bool second) {
  const void* src = second ? op->data2 : op->data;
  if (op->dtype == dtype_of<T>() && (op->kind != LK_DENSE || op->ld == op->cols))
    return (const T*)src;
  const int key = second ? (dtype_of<T>() == COLA_F64 ? DK_V_F64 : DK_V_F32)
                         : (dtype_of<T>() == COLA_F64 ? DK_F64 : DK_F32);
  auto it = op->derived.find(key);
  if (it == op->derived.end())
    fail(COLA_ERR_INVALID_ARG, "internal: leaf not prepared for this precision");
  return (const T*)it->second.p;
}
template const float* leaf_ptr<float>(const cola_linop*, bool);
template const double* leaf_ptr<double>(const cola_linop*, bool);

static int64_t leaf_ld(const cola_linop* op) { return op->cols; }  // working copies are packed

__global__ void k_pack_convert_f64_f32(const double* in, int64_t ld, float* out, int64_t rows,
                                       int64_t cols) {
  const int64_t tot = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (float)in[(e / cols) * ld + e % cols];
}
__global__ void k_pack_convert_f32_f64(const float* in, int64_t ld, double* out, int64_t rows,
                                       int64_t cols) {
  const int64_t tot = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (double)in[(e / cols) * ld + e % cols];
}
template <typename T>
__global__ void k_pack_copy(const T* in, int64_t ld, T* out, int64_t rows, int64_t cols) {
  const int64_t tot = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = in[(e / cols) * ld + e % cols];
}

static void* derived_buf(cola_linop* op, int key, size_t bytes) {
  auto it = op->derived.find(key);
  if (it != op->derived.end() && it->second.bytes >= bytes) return it->second.p;
  if (it != op->derived.end()) {
    cudaFree(it->second.p);
    op->derived.erase(it);
  }
  void* p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(bytes, 256)) != cudaSuccess) {
    cudaGetLastError();
    fail(COLA_ERR_OOM, "leaf copy of %zu bytes", bytes);
  }
  op->derived[key] = Buf{p, bytes};
  return p;
}

// Working copy of a leaf array in dtype `want` (packed rows x cols).
static void make_copy(Ctx* c, cola_linop* op, const void* src, int64_t rows, int64_t cols,
                      int64_t ld, cola_dtype want, int key) {
  const int64_t n = rows * cols;
  void* dst = derived_buf(op, key, n * dtype_size(want));
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 1023) / 1024, 4096));
  if (op->dtype == COLA_F64 && want == COLA_F32)
    k_pack_convert_f64_f32<<<grid, 256, 0, c->s>>>((const double*)src, ld, (float*)dst, rows,
                                                    cols);
  else if (op->dtype == COLA_F32 && want == COLA_F64)
    k_pack_convert_f32_f64<<<grid, 256, 0, c->s>>>((const float*)src, ld, (double*)dst, rows,
                                                    cols);
  else if (want == COLA_F64)
    k_pack_copy<double><<<grid, 256, 0, c->s>>>((const double*)src, ld, (double*)dst, rows,
                                                 cols);
  else
    k_pack_copy<float><<<grid, 256, 0, c->s>>>((const float*)src, ld, (float*)dst, rows, cols);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
}

void kron_tc_prepare(Ctx* c, cola_linop* op, int split_terms);  // kron_tc.cu

// make_copy unless a reusable copy under `key` exists (prep_fresh).
static void copy_once(Ctx* c, cola_linop* op, const void* src, int64_t rows, int64_t cols,
                      int64_t ld, cola_dtype want, int key) {
  if (prep_fresh(op, key)) return;
  make_copy(c, op, src, rows, cols, ld, want, key);
  prep_mark(op, key);
}

static void prepare_rec(Ctx* c, cola_linop* op, cola_dtype want, int prec, int split) {
  switch (op->kind) {
    case LK_DENSE:
      if (op->dtype != want || op->ld != op->cols)
        copy_once(c, op, op->data, op->rows, op->cols, op->ld, want,
                  want == COLA_F64 ? DK_F64 : DK_F32);
      break;
    case LK_DIAG:
      if (op->dtype != want)
        copy_once(c, op, op->data, op->stride ? op->rows : 1, 1, 1, want,
                  want == COLA_F64 ? DK_F64 : DK_F32);
      break;
    case LK_LOWRANK:
      if (op->dtype != want) {
        copy_once(c, op, op->data, op->rows, op->rank, op->rank, want,
                  want == COLA_F64 ? DK_F64 : DK_F32);
        if (op->data2)
          copy_once(c, op, op->data2, op->rows, op->rank, op->rank, want,
                    want == COLA_F64 ? DK_V_F64 : DK_V_F32);
      }
      // k x n transposes of U (and V) for the coalesced U W product
      for (int second = 0; second < (op->data2 ? 2 : 1); ++second) {
        const int key = want == COLA_F64 ? (second ? DK_VT_F64 : DK_UT_F64)
                                         : (second ? DK_VT_F32 : DK_UT_F32);
        if (prep_fresh(op, key)) continue;
        void* dst = derived_buf(op, key, op->rows * op->rank * dtype_size(want));
        if (want == COLA_F64)
          transpose_nk<double>(c, leaf_ptr<double>(op, second), (double*)dst, op->rows, op->rank);
        else
          transpose_nk<float>(c, leaf_ptr<float>(op, second), (float*)dst, op->rows, op->rank);
        prep_mark(op, key);
      }
      break;
    default:
      for (auto* k : op->kids) prepare_rec(c, k, want, prec, split);
      if (op->kind == LK_KRON && prec == COLA_PREC_MIXED) kron_tc_prepare(c, op, split);
      break;
  }
}

void prepare_leaves(Ctx* c, cola_linop* op, int prec, int split_terms) {
  prepare_rec(c, op, prec == COLA_PREC_F64 ? COLA_F64 : COLA_F32, prec, split_terms);
}

void collect_leaves(const cola_linop* op, std::vector<const cola_linop*>& out) {
  if (op->kind == LK_DENSE || op->kind == LK_DIAG || op->kind == LK_LOWRANK) {
    out.push_back(op);
    return;
  }
  for (auto* k : op->kids) collect_leaves(k, out);
}

static std::string tmpname(const char* what, int depth, int slot) {
  char b[64];
  snprintf(b, sizeof b, "%s.d%d.%d", what, depth, slot);
  return b;
}

template <typename T>
static T* tmp(Ctx* c, const char* what, int depth, int slot, int64_t elems) {
  return (T*)c->ws.get(tmpname(what, depth, slot), sizeof(T) * (size_t)elems);
}

// In-place-layout mode product: Y[r, a, i, c] = coeff sum_j F[i, j] X[r, a, j, c] + beta Y.
// dims: current mode sizes; F is rows x cols (or its transpose) with leading dim ld.
template <typename T>
static void mode_product(Ctx* c, const T* F, int64_t ld, int64_t frows, int64_t fcols, bool tr,
                         const std::vector<int64_t>& dims, int mode, const T* X, T* Y,
                         int64_t R, double coeff, double beta) {
  const int64_t rows = tr ? fcols : frows, cols = tr ? frows : fcols;
  int64_t A = 1, C = 1;
  for (int m = 0; m < mode; ++m) A *= dims[m];
  for (size_t m = mode + 1; m < dims.size(); ++m) C *= dims[m];
  // F_op[i, j] = tr ? F[j, i] : F[i, j]
  const int64_t f_i = tr ? 1 : ld, f_j = tr ? ld : 1;
  if (C > 1) {
    gemm<T>(c, rows, C, cols, coeff, F, f_i, f_j, 0, X, C, 1, cols * C, beta, Y, C, 1, rows * C,
            R * A);
  } else {
    gemm<T>(c, R * A, rows, cols, coeff, X, cols, 1, 0, F, f_j, f_i, 0, beta, Y, rows, 1, 0, 1);
  }
}

template <typename T>
const T* band_ptr(const cola_linop* op, bool tr) {
  const bool f64 = dtype_of<T>() == COLA_F64;
  const int key = f64 ? (tr ? 7 : DK_BAND64) : (tr ? 8 : DK_BAND32);
  return (const T*)op->derived.at(key).p;
}

template <typename T>
void kron_tc_apply(Ctx* c, const cola_linop* op, const T* X, T* Y, int64_t R, double coeff,
                   double beta, int depth, bool tr);  // kron_tc.cu

template <typename T>
void apply(Ctx* c, const cola_linop* op, const T* X, T* Y, int64_t R, double coeff, double beta,
           int depth, bool tr, int prec) {
  switch (op->kind) {
    case LK_DENSE: {
      const T* M = leaf_ptr<T>(op);
      const int64_t ld = leaf_ld(op);
      const int64_t rows = tr ? op->cols : op->rows, cols = tr ? op->rows : op->cols;
      // C[r, i] = sum_j X[r, j] Mop[i, j]
      gemm<T>(c, R, rows, cols, coeff, X, cols, 1, 0, M, tr ? ld : 1, tr ? 1 : ld, 0, beta, Y,
              rows, 1, 0, 1);
      break;
    }
    case LK_DIAG:
      diag_apply<T>(c, leaf_ptr<T>(op), op->stride, X, Y, op->rows, R, coeff, beta);
      break;
    case LK_LOWRANK: {
      const T* U = leaf_ptr<T>(op);
      const T* V = op->data2 ? leaf_ptr<T>(op, true) : U;
      if (tr) std::swap(U, V);
      T* W = tmp<T>(c, "lrW", depth, 0, op->rank * R);
      double* part = tmp<double>(c, "lrP", depth, 0, (int64_t)kLowRankBlocks * op->rank * R);
      lowrank_vtx<T>(c, V, X, op->rows, op->rank, R, W, part);
      // the transposed copy of whichever factor multiplies W
      const bool f64 = dtype_of<T>() == COLA_F64;
      const bool use_v = tr && op->data2;
      const int tkey = f64 ? (use_v ? DK_VT_F64 : DK_UT_F64) : (use_v ? DK_VT_F32 : DK_UT_F32);
      auto it = op->derived.find(tkey);
      const T* Ut = it != op->derived.end() ? (const T*)it->second.p : nullptr;
      lowrank_uw<T>(c, U, W, Y, op->rows, op->rank, R, coeff, beta, Ut);
      break;
    }
    case LK_SUM: {
      size_t i0 = 0;
      // a tridiagonal Kronecker sum followed by a diagonal term: one pass
      const cola_linop* k0 = op->kids[0];
      if (op->kids.size() >= 2 && k0->kind == LK_KRONSUM && k0->tridiag &&
          op->kids[1]->kind == LK_DIAG) {
        std::vector<int64_t> dims;
        for (auto* f : k0->kids) dims.push_back(f->rows);
        const cola_linop* dg = op->kids[1];
        i0 = stencil_apply<T>(c, (int)dims.size(), dims.data(), band_ptr<T>(k0, tr), X, Y, R,
                              coeff * op->coeffs[0], beta, leaf_ptr<T>(dg), dg->stride,
                              coeff * op->coeffs[1])
                 ? 2
                 : 1;
      }
      for (size_t i = i0; i < op->kids.size(); ++i)
        apply<T>(c, op->kids[i], X, Y, R, coeff * op->coeffs[i], i == 0 ? beta : 1.0, depth + 1,
                 tr, prec);
      break;
    }
    case LK_PRODUCT: {
      const int m = (int)op->kids.size();
      const T* cur = X;
      for (int s = 0; s < m; ++s) {
        const cola_linop* t = tr ? op->kids[s] : op->kids[m - 1 - s];
        if (s == m - 1) {
          apply<T>(c, t, cur, Y, R, coeff, beta, depth + 1, tr, prec);
        } else {
          const int64_t out_rows = tr ? t->cols : t->rows;
          T* dst = tmp<T>(c, "prod", depth, s & 1, out_rows * R);
          apply<T>(c, t, cur, dst, R, 1.0, 0.0, depth + 1, tr, prec);
          cur = dst;
        }
      }
      break;
    }
    case LK_KRON: {
      if (prec == COLA_PREC_MIXED && dtype_of<T>() == COLA_F32) {
        kron_tc_apply<T>(c, op, X, Y, R, coeff, beta, depth, tr);
        break;
      }
      // Cyclic mode products: step k contracts the leading index of the
      // current layout [j_k, rest] into [rest, i_k]; after d steps the layout
      // is back in (i_1, ..., i_d) order.
      const int d = (int)op->kids.size();
      int64_t cur_size = tr ? op->rows : op->cols;
      int64_t maxsz = cur_size;
      for (int k = 0; k < d; ++k) {
        const cola_linop* f = op->kids[k];
        const int64_t n_in = tr ? f->rows : f->cols, n_out = tr ? f->cols : f->rows;
        cur_size = cur_size / n_in * n_out;
        maxsz = std::max(maxsz, cur_size);
      }
      cur_size = tr ? op->rows : op->cols;
      const T* cur = X;
      for (int k = 0; k < d; ++k) {
        const cola_linop* f = op->kids[k];
        const T* F = leaf_ptr<T>(f);
        const int64_t ld = leaf_ld(f);
        const int64_t n_in = tr ? f->rows : f->cols, n_out = tr ? f->cols : f->rows;
        const int64_t rest = cur_size / n_in, out_size = rest * n_out;
        const bool last = (k == d - 1);
        T* dst = last ? Y : tmp<T>(c, "kron", depth, k & 1, maxsz * R);
        // B[k=j, n=i] = F_op[i, j]
        const int64_t lbk = tr ? ld : 1, lbn = tr ? 1 : ld;
        gemm<T>(c, rest, n_out, n_in, last ? coeff : 1.0, cur, 1, rest, cur_size, F, lbk, lbn, 0,
                last ? beta : 0.0, dst, n_out, 1, out_size, R);
        cur = dst;
        cur_size = out_size;
      }
      break;
    }
    case LK_KRONSUM: {
      const int d = (int)op->kids.size();
      std::vector<int64_t> dims;
      for (auto* f : op->kids) dims.push_back(f->rows);
      if (op->tridiag) {
        stencil_apply<T>(c, d, dims.data(), band_ptr<T>(op, tr), X, Y, R, coeff, beta);
      } else {
        for (int k = 0; k < d; ++k) {
          const cola_linop* f = op->kids[k];
          mode_product<T>(c, leaf_ptr<T>(f), leaf_ld(f), f->rows, f->cols, tr, dims, k, X, Y, R,
                          coeff, k == 0 ? beta : 1.0);
        }
      }
      break;
    }
  }
}

template void apply<float>(Ctx*, const cola_linop*, const float*, float*, int64_t, double,
                           double, int, bool, int);
template void apply<double>(Ctx*, const cola_linop*, const double*, double*, int64_t, double,
                            double, int, bool, int);

// ---------------------------------------------------------------- Diag rules
template <typename T>
__global__ void k_diag_of_diag(const T* d, int64_t stride, T* out, int64_t n, T coeff, T beta) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    T v = coeff * (stride ? d[i] : d[0]);
    if (beta != T(0)) v += beta * out[i];
    out[i] = v;
  }
}

template <typename T>
static void diag_rec(Ctx* c, const cola_linop* op, T* out, double coeff, double beta) {
  switch (op->kind) {
    case LK_DENSE: {
      COLA_REQUIRE(op->rows == op->cols, COLA_ERR_SHAPE, "Diag of a non-square dense leaf");
      const T* f = leaf_ptr<T>(op);
      int64_t n = op->rows, ld = leaf_ld(op);
      kron_diag<T>(c, 1, &n, &f, &ld, out, coeff, beta);
      break;
    }
    case LK_DIAG: {
      const int64_t n = op->rows;
      const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096));
      k_diag_of_diag<T><<<grid, 256, 0, c->s>>>(leaf_ptr<T>(op), op->stride, out, n, (T)coeff,
                                                 (T)beta);
      c->count_launch();
      COLA_CUDA(cudaGetLastError());
      break;
    }
    case LK_LOWRANK: {
      const T* U = leaf_ptr<T>(op);
      const T* V = op->data2 ? leaf_ptr<T>(op, true) : U;
      rowsum_products<T>(c, U, V, out, op->rows, op->rank, coeff, beta);
      break;
    }
    case LK_SUM:
      for (size_t i = 0; i < op->kids.size(); ++i)
        diag_rec<T>(c, op->kids[i], out, coeff * op->coeffs[i], i == 0 ? beta : 1.0);
      break;
    case LK_KRON:
    case LK_KRONSUM: {
      std::vector<int64_t> sizes, lds;
      std::vector<const T*> f;
      for (auto* k : op->kids) {
        COLA_REQUIRE(k->rows == k->cols, COLA_ERR_SHAPE, "Diag of a non-square Kronecker factor");
        sizes.push_back(k->rows);
        lds.push_back(leaf_ld(k));
        f.push_back(leaf_ptr<T>(k));
      }
      if (op->kind == LK_KRON)
        kron_diag<T>(c, (int)sizes.size(), sizes.data(), f.data(), lds.data(), out, coeff, beta);
      else
        kronsum_diag<T>(c, (int)sizes.size(), sizes.data(), f.data(), lds.data(), out, coeff,
                        beta);
      break;
    }
    case LK_PRODUCT:
      fail(COLA_ERR_UNSUPPORTED, "Diag of a Product has no composition rule");
  }
}

template <typename T>
void diagonal(Ctx* c, const cola_linop* op, T* out, int depth) {
  (void)depth;
  diag_rec<T>(c, op, out, 1.0, 0.0);
}
template void diagonal<float>(Ctx*, const cola_linop*, float*, int);
template void diagonal<double>(Ctx*, const cola_linop*, double*, int);

// ---------------------------------------------------------- leaf gradients
// Gradient of sum_r Uw_r^T (scale * op) X_r with respect to every leaf, in
// tree order, accumulated (in working type T) into grads[leaf].
template <typename T>
static void grad_of_unfolded(Ctx* c, const T* Up, const T* Zp, int64_t rows, int64_t cols,
                             int64_t L, T* G, double scale, int depth) {
  // G[i, j] += scale * sum_m Up[i, m] Zp[j, m]; split-K over S chunks for parallelism.
  const int64_t tiles = ((rows + 127) / 128) * ((cols + 127) / 128);
  int64_t S = std::max<int64_t>(1, std::min<int64_t>(64, (2 * c->num_sms + tiles - 1) / tiles));
  S = std::min<int64_t>(S, std::max<int64_t>(1, L / 256));
  const int64_t chunk = L / S;
  T* P = tmp<T>(c, "gpart", depth, 0, (S + 1) * rows * cols);
  gemm<T>(c, rows, cols, chunk, 1.0, Up, L, 1, chunk, Zp, 1, L, chunk, 0.0, P, cols, 1,
          rows * cols, S);
  int64_t parts = S;
  if (chunk * S < L) {
    gemm<T>(c, rows, cols, L - chunk * S, 1.0, Up + chunk * S, L, 1, 0, Zp + chunk * S, 1, L, 0,
            0.0, P + S * rows * cols, cols, 1, 0, 1);
    parts = S + 1;
  }
  add_partials<T>(c, P, G, rows * cols, parts, scale);
}

template <typename T>
static T* grad_target(Ctx* c, std::vector<T*>& acc, int leaf) {
  return acc[leaf];
}

template <typename T>
static void bil_rec(Ctx* c, const cola_linop* op, const T* Uw, const T* X, int64_t R,
                    double scale, std::vector<T*>& acc, int& li, int depth) {
  switch (op->kind) {
    case LK_DENSE: {
      T* G = acc[li++];
      if (G)
        gemm<T>(c, op->rows, op->cols, R, scale, Uw, 1, op->rows, 0, X, op->cols, 1, 0, 1.0, G,
                op->cols, 1, 0, 1);
      break;
    }
    case LK_DIAG: {
      T* G = acc[li++];
      if (G) {
        double* part = tmp<double>(c, "dgp", depth, 0, 2 * 256 + 8);
        diag_grad<T>(c, Uw, X, G, op->rows, R, scale, op->stride == 0, part);
      }
      break;
    }
    case LK_LOWRANK: {
      T* G = acc[li++];
      if (!G) break;
      const T* U = leaf_ptr<T>(op);
      const T* V = op->data2 ? leaf_ptr<T>(op, true) : U;
      T* W = tmp<T>(c, "blW", depth, 0, op->rank * R);
      double* part = tmp<double>(c, "blP", depth, 0, (int64_t)kLowRankBlocks * op->rank * R);
      lowrank_vtx<T>(c, V, X, op->rows, op->rank, R, W, part);  // W[k][r] = (V^T x_r)_k
      lowrank_grad<T>(c, Uw, W, G, op->rows, op->rank, R, scale);
      if (!op->data2) {
        lowrank_vtx<T>(c, U, Uw, op->rows, op->rank, R, W, part);  // (U^T u_r)_k
        lowrank_grad<T>(c, X, W, G, op->rows, op->rank, R, scale);
      }
      break;
    }
    case LK_SUM:
      for (size_t i = 0; i < op->kids.size(); ++i)
        bil_rec<T>(c, op->kids[i], Uw, X, R, scale * op->coeffs[i], acc, li, depth + 1);
      break;
    case LK_PRODUCT: {
      // u^T A_1 .. A_m x: leaf in A_i sees left (A_1..A_{i-1})^T u and right A_{i+1}..A_m x.
      const int m = (int)op->kids.size();
      std::vector<const T*> rights(m);
      const T* v = X;
      for (int i = m - 1; i >= 0; --i) {
        rights[i] = v;
        if (i > 0) {
          T* dst = tmp<T>(c, "bright", depth, i, op->kids[i]->rows * R);
          apply<T>(c, op->kids[i], v, dst, R, 1.0, 0.0, depth + 1, false, COLA_PREC_F32);
          v = dst;
        }
      }
      const T* left = Uw;
      for (int i = 0; i < m; ++i) {
        bil_rec<T>(c, op->kids[i], left, rights[i], R, scale, acc, li, depth + 1);
        if (i < m - 1) {
          T* dst = tmp<T>(c, "bleft", depth, i & 1, op->kids[i]->cols * R);
          apply<T>(c, op->kids[i], left, dst, R, 1.0, 0.0, depth + 1, true, COLA_PREC_F32);
          left = dst;
        }
      }
      break;
    }
    case LK_KRON:
    case LK_KRONSUM: {
      const int d = (int)op->kids.size();
      const int64_t L_total = op->rows * R;
      for (int k = 0; k < d; ++k) {
        const cola_linop* f = op->kids[k];
        T* G = acc[li++];
        if (!G) continue;
        // Z = every other factor applied to X (Kronecker); X itself (Kronecker sum).
        const T* Z = X;
        std::vector<int64_t> dims;
        for (auto* g : op->kids) dims.push_back(g->cols);
        if (op->kind == LK_KRON) {
          int slot = 0;
          for (int m = 0; m < d; ++m) {
            if (m == k) continue;
            const cola_linop* g = op->kids[m];
            int64_t out_size = R;
            for (int q = 0; q < d; ++q) out_size *= (q == m ? g->rows : dims[q]);
            T* dst = tmp<T>(c, "bkz", depth, slot, out_size);
            mode_product<T>(c, leaf_ptr<T>(g), leaf_ld(g), g->rows, g->cols, false, dims, m, Z,
                            dst, R, 1.0, 0.0);
            dims[m] = g->rows;
            Z = dst;
            slot ^= 1;
          }
        }
        int64_t A = 1, C = 1;
        for (int m = 0; m < k; ++m) A *= op->kids[m]->rows;
        for (int m = k + 1; m < d; ++m) C *= op->kids[m]->rows;
        const int64_t L = R * A * C;
        T* Up = tmp<T>(c, "bku", depth, 0, f->rows * L);
        T* Zp = tmp<T>(c, "bkzp", depth, 0, f->cols * L);
        permute_mode_front<T>(c, Uw, Up, R, A, f->rows, C);
        permute_mode_front<T>(c, Z, Zp, R, A, f->cols, C);
        (void)L_total;
        grad_of_unfolded<T>(c, Up, Zp, f->rows, f->cols, L, G, scale, depth);
      }
      break;
    }
  }
}

template <typename T>
void bilinear(Ctx* c, const cola_linop* op, const T* Uw, const T* X, int64_t R, double scale,
              const std::vector<void*>& grads, int& leaf_index, int depth) {
  std::vector<T*> acc;
  for (void* g : grads) acc.push_back((T*)g);
  bil_rec<T>(c, op, Uw, X, R, scale, acc, leaf_index, depth);
}
template void bilinear<float>(Ctx*, const cola_linop*, const float*, const float*, int64_t,
                              double, const std::vector<void*>&, int&, int);
template void bilinear<double>(Ctx*, const cola_linop*, const double*, const double*, int64_t,
                               double, const std::vector<void*>&, int&, int);

}  // namespace cola

// ============================================================== linop nodes
cola_linop::~cola_linop() {
  if (eig_kron) cola_linop_release(eig_kron);
  for (auto& kv : derived) cudaFree(kv.second.p);
  for (auto* k : kids) cola_linop_release(k);
}

using namespace cola;

static uint64_t next_uid() {
  static std::atomic<uint64_t> counter{1};
  return counter.fetch_add(1);
}

static cola_linop* new_node(cola_ctx* ctx, LinKind kind) {
  auto* op = new cola_linop();
  op->uid = next_uid();
  op->ctx = ctx;
  op->kind = kind;
  return op;
}

static void check_dtype(cola_dtype d) {
  COLA_REQUIRE(d == COLA_F64 || d == COLA_F32, COLA_ERR_DTYPE, "dtype %d is not F64/F32", (int)d);
}

extern "C" {

const char* cola_last_error(void) { return g_last_error.c_str(); }

cola_status cola_create(int device, cola_ctx** out) {
  return guard([&] {
    COLA_REQUIRE(out, COLA_ERR_INVALID_ARG, "out is NULL");
    int ndev = 0;
    COLA_CUDA(cudaGetDeviceCount(&ndev));
    COLA_REQUIRE(device >= 0 && device < ndev, COLA_ERR_INVALID_ARG, "device %d of %d", device,
                 ndev);
    auto* c = new cola_ctx();
    c->device = device;
    COLA_CUDA(cudaSetDevice(device));
    COLA_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
    COLA_CUDA(cudaStreamCreateWithFlags(&c->s, cudaStreamNonBlocking));
    COLA_CUDA(cudaEventCreateWithFlags(&c->ev_a, cudaEventDisableTiming));
    COLA_CUDA(cudaEventCreateWithFlags(&c->ev_b, cudaEventDisableTiming));
    *out = c;
  });
}

cola_status cola_destroy(cola_ctx* c) {
  return guard([&] {
    COLA_REQUIRE(c, COLA_ERR_INVALID_ARG, "ctx is NULL");
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->s);
    for (auto& kv : c->graphs)
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    c->ws.release_all();
    if (c->pinned) cudaFreeHost(c->pinned);
    if (c->tc_err_host) cudaFreeHost(c->tc_err_host);
    if (c->tc_err_ev) cudaEventDestroy(c->tc_err_ev);
    cudaEventDestroy(c->ev_a);
    cudaEventDestroy(c->ev_b);
    cudaStreamDestroy(c->s);
    delete c;
  });
}

cola_status cola_linop_dense(cola_ctx* ctx, int64_t rows, int64_t cols, const void* data,
                             int64_t ld, cola_dtype dtype, cola_linop** out) {
  return guard([&] {
    COLA_REQUIRE(ctx && out, COLA_ERR_INVALID_ARG, "ctx/out is NULL");
    COLA_REQUIRE(rows > 0 && cols > 0, COLA_ERR_SHAPE, "dense: %lld x %lld", (long long)rows,
                 (long long)cols);
    COLA_REQUIRE(data, COLA_ERR_INVALID_ARG, "dense: data is NULL");
    COLA_REQUIRE(ld >= cols, COLA_ERR_SHAPE, "dense: ld %lld < cols %lld", (long long)ld,
                 (long long)cols);
    check_dtype(dtype);
    auto* op = new_node(ctx, LK_DENSE);
    op->rows = rows;
    op->cols = cols;
    op->data = data;
    op->ld = ld;
    op->dtype = dtype;
    *out = op;
  });
}

cola_status cola_linop_diag(cola_ctx* ctx, int64_t n, const void* d, int64_t stride,
                            cola_dtype dtype, cola_linop** out) {
  return guard([&] {
    COLA_REQUIRE(ctx && out, COLA_ERR_INVALID_ARG, "ctx/out is NULL");
    COLA_REQUIRE(n > 0, COLA_ERR_SHAPE, "diag: n = %lld", (long long)n);
    COLA_REQUIRE(d, COLA_ERR_INVALID_ARG, "diag: d is NULL");
    COLA_REQUIRE(stride == 0 || stride == 1, COLA_ERR_INVALID_ARG, "diag: stride must be 0 or 1");
    check_dtype(dtype);
    auto* op = new_node(ctx, LK_DIAG);
    op->rows = op->cols = n;
    op->data = d;
    op->stride = stride;
    op->dtype = dtype;
    *out = op;
  });
}

cola_status cola_linop_lowrank(cola_ctx* ctx, int64_t n, int64_t k, const void* U, const void* V,
                               cola_dtype dtype, cola_linop** out) {
  return guard([&] {
    COLA_REQUIRE(ctx && out, COLA_ERR_INVALID_ARG, "ctx/out is NULL");
    COLA_REQUIRE(n > 0 && k > 0, COLA_ERR_SHAPE, "lowrank: n=%lld k=%lld", (long long)n,
                 (long long)k);
    COLA_REQUIRE(U, COLA_ERR_INVALID_ARG, "lowrank: U is NULL");
    check_dtype(dtype);
    auto* op = new_node(ctx, LK_LOWRANK);
    op->rows = op->cols = n;
    op->rank = k;
    op->data = U;
    op->data2 = V;
    op->dtype = dtype;
    *out = op;
  });
}

static cola_linop* composite(cola_ctx* ctx, LinKind kind, int n, cola_linop* const* kids) {
  COLA_REQUIRE(ctx, COLA_ERR_INVALID_ARG, "ctx is NULL");
  COLA_REQUIRE(n >= 1 && kids, COLA_ERR_INVALID_ARG, "need at least one child");
  for (int i = 0; i < n; ++i) {
    COLA_REQUIRE(kids[i], COLA_ERR_INVALID_ARG, "child %d is NULL", i);
    COLA_REQUIRE(kids[i]->ctx == ctx, COLA_ERR_INVALID_ARG, "child %d belongs to another context",
                 i);
  }
  auto* op = new_node(ctx, kind);
  for (int i = 0; i < n; ++i) {
    op->kids.push_back(kids[i]);
    kids[i]->refs++;
  }
  return op;
}

cola_status cola_linop_kron(cola_ctx* ctx, int nf, cola_linop* const* factors,
                            cola_linop** out) {
  return guard([&] {
    COLA_REQUIRE(out, COLA_ERR_INVALID_ARG, "out is NULL");
    COLA_REQUIRE(nf >= 1 && nf <= 8, COLA_ERR_UNSUPPORTED, "kron: %d factors (1..8)", nf);
    for (int i = 0; i < nf; ++i)
      COLA_REQUIRE(factors && factors[i] && factors[i]->kind == LK_DENSE, COLA_ERR_UNSUPPORTED,
                   "kron: factor %d must be a dense leaf", i);
    cola_linop* op = composite(ctx, LK_KRON, nf, factors);
    op->rows = op->cols = 1;
    for (int i = 0; i < nf; ++i) {
      op->rows *= factors[i]->rows;
      op->cols *= factors[i]->cols;
    }
    *out = op;
  });
}

cola_status cola_linop_kronsum(cola_ctx* ctx, int nf, cola_linop* const* factors,
                               cola_linop** out) {
  return guard([&] {
    COLA_REQUIRE(out, COLA_ERR_INVALID_ARG, "out is NULL");
    COLA_REQUIRE(nf >= 1 && nf <= 8, COLA_ERR_UNSUPPORTED, "kronsum: %d factors (1..8)", nf);
    for (int i = 0; i < nf; ++i) {
      COLA_REQUIRE(factors && factors[i] && factors[i]->kind == LK_DENSE, COLA_ERR_UNSUPPORTED,
                   "kronsum: factor %d must be a dense leaf", i);
      COLA_REQUIRE(factors[i]->rows == factors[i]->cols, COLA_ERR_SHAPE,
                   "kronsum: factor %d is not square", i);
    }
    cola_linop* op = composite(ctx, LK_KRONSUM, nf, factors);
    op->rows = 1;
    for (int i = 0; i < nf; ++i) op->rows *= factors[i]->rows;
    op->cols = op->rows;
    // Band check: read each factor once.
    COLA_CUDA(cudaSetDevice(ctx->device));
    COLA_CUDA(cudaDeviceSynchronize());
    bool tri = true;
    std::vector<double> bands, bandsT;
    for (int i = 0; i < nf && tri; ++i) {
      const cola_linop* f = factors[i];
      const int64_t n = f->rows;
      std::vector<double> h(n * n);
      if (f->dtype == COLA_F64) {
        COLA_CUDA(cudaMemcpy2D(h.data(), n * 8, f->data, f->ld * 8, n * 8, n,
                               cudaMemcpyDeviceToHost));
      } else {
        std::vector<float> hf(n * n);
        COLA_CUDA(cudaMemcpy2D(hf.data(), n * 4, f->data, f->ld * 4, n * 4, n,
                               cudaMemcpyDeviceToHost));
        for (int64_t e = 0; e < n * n; ++e) h[e] = hf[e];
      }
      for (int64_t r = 0; r < n && tri; ++r)
        for (int64_t q = 0; q < n; ++q)
          if ((q < r - 1 || q > r + 1) && h[r * n + q] != 0.0) {
            tri = false;
            break;
          }
      if (!tri) break;
      std::vector<double> lo(n, 0.0), di(n), up(n, 0.0);
      for (int64_t r = 0; r < n; ++r) {
        di[r] = h[r * n + r];
        if (r > 0) lo[r] = h[r * n + r - 1];
        if (r < n - 1) up[r] = h[r * n + r + 1];
      }
      bands.insert(bands.end(), lo.begin(), lo.end());
      bands.insert(bands.end(), di.begin(), di.end());
      bands.insert(bands.end(), up.begin(), up.end());
      // transpose: lo'[r] = A[r-1, r] = up[r-1], up'[r] = A[r+1, r] = lo[r+1]
      std::vector<double> loT(n, 0.0), upT(n, 0.0);
      for (int64_t r = 0; r < n; ++r) {
        if (r > 0) loT[r] = up[r - 1];
        if (r < n - 1) upT[r] = lo[r + 1];
      }
      bandsT.insert(bandsT.end(), loT.begin(), loT.end());
      bandsT.insert(bandsT.end(), di.begin(), di.end());
      bandsT.insert(bandsT.end(), upT.begin(), upT.end());
    }
    if (tri) {
      op->tridiag = true;
      op->band_host = bands;
      const size_t nb = bands.size();
      std::vector<float> bf(nb), bfT(nb);
      for (size_t e = 0; e < nb; ++e) {
        bf[e] = (float)bands[e];
        bfT[e] = (float)bandsT[e];
      }
      void* p64 = derived_buf(op, DK_BAND64, nb * 8);
      void* p32 = derived_buf(op, DK_BAND32, nb * 4);
      void* p64T = derived_buf(op, 7, nb * 8);
      void* p32T = derived_buf(op, 8, nb * 4);
      COLA_CUDA(cudaMemcpy(p64, bands.data(), nb * 8, cudaMemcpyHostToDevice));
      COLA_CUDA(cudaMemcpy(p32, bf.data(), nb * 4, cudaMemcpyHostToDevice));
      COLA_CUDA(cudaMemcpy(p64T, bandsT.data(), nb * 8, cudaMemcpyHostToDevice));
      COLA_CUDA(cudaMemcpy(p32T, bfT.data(), nb * 4, cudaMemcpyHostToDevice));
    }
    *out = op;
  });
}

cola_status cola_linop_sum(cola_ctx* ctx, int n, cola_linop* const* terms, const double* coeffs,
                           cola_linop** out) {
  return guard([&] {
    COLA_REQUIRE(out, COLA_ERR_INVALID_ARG, "out is NULL");
    for (int i = 0; i < n; ++i)
      COLA_REQUIRE(terms && terms[i] && terms[i]->rows == terms[0]->rows &&
                       terms[i]->cols == terms[0]->cols,
                   COLA_ERR_SHAPE, "sum: term %d shape differs", i);
    cola_linop* op = composite(ctx, LK_SUM, n, terms);
    op->rows = terms[0]->rows;
    op->cols = terms[0]->cols;
    for (int i = 0; i < n; ++i) op->coeffs.push_back(coeffs ? coeffs[i] : 1.0);
    *out = op;
  });
}

cola_status cola_linop_product(cola_ctx* ctx, int n, cola_linop* const* terms, cola_linop** out) {
  return guard([&] {
    COLA_REQUIRE(out, COLA_ERR_INVALID_ARG, "out is NULL");
    for (int i = 0; i + 1 < n; ++i)
      COLA_REQUIRE(terms && terms[i] && terms[i + 1] && terms[i]->cols == terms[i + 1]->rows,
                   COLA_ERR_SHAPE, "product: term %d cols != term %d rows", i, i + 1);
    cola_linop* op = composite(ctx, LK_PRODUCT, n, terms);
    op->rows = terms[0]->rows;
    op->cols = terms[n - 1]->cols;
    *out = op;
  });
}

cola_status cola_linop_cache_prepared(cola_linop* op, int32_t on) {
  return guard([&] {
    COLA_REQUIRE(op, COLA_ERR_INVALID_ARG, "op is NULL");
    op->cache_prepared = on != 0;
  });
}

static void touch_rec(cola_linop* op) {
  ++op->version;
  for (auto* k : op->kids) touch_rec(k);
}

cola_status cola_linop_touch(cola_linop* op) {
  return guard([&] {
    COLA_REQUIRE(op, COLA_ERR_INVALID_ARG, "op is NULL");
    touch_rec(op);
  });
}

cola_status cola_linop_set_spd(cola_linop* op, int spd) {
  return guard([&] {
    COLA_REQUIRE(op, COLA_ERR_INVALID_ARG, "op is NULL");
    COLA_REQUIRE(!spd || op->rows == op->cols, COLA_ERR_SHAPE, "spd needs a square operator");
    op->spd = spd ? 1 : 0;
  });
}

cola_status cola_linop_shape(const cola_linop* op, int64_t* rows, int64_t* cols) {
  return guard([&] {
    COLA_REQUIRE(op && rows && cols, COLA_ERR_INVALID_ARG, "NULL argument");
    *rows = op->rows;
    *cols = op->cols;
  });
}

cola_status cola_linop_num_leaves(const cola_linop* op, int* n) {
  return guard([&] {
    COLA_REQUIRE(op && n, COLA_ERR_INVALID_ARG, "NULL argument");
    std::vector<const cola_linop*> l;
    collect_leaves(op, l);
    *n = (int)l.size();
  });
}

cola_status cola_linop_leaf_info(const cola_linop* op, int index, int* kind, int64_t* rows,
                                 int64_t* cols) {
  return guard([&] {
    COLA_REQUIRE(op && kind && rows && cols, COLA_ERR_INVALID_ARG, "NULL argument");
    std::vector<const cola_linop*> l;
    collect_leaves(op, l);
    COLA_REQUIRE(index >= 0 && index < (int)l.size(), COLA_ERR_INVALID_ARG, "leaf %d of %d",
                 index, (int)l.size());
    const cola_linop* f = l[index];
    if (f->kind == LK_DENSE) {
      *kind = COLA_LEAF_DENSE;
      *rows = f->rows;
      *cols = f->cols;
    } else if (f->kind == LK_DIAG) {
      *kind = f->stride ? COLA_LEAF_DIAG : COLA_LEAF_SCALAR;
      *rows = f->stride ? f->rows : 1;
      *cols = 1;
    } else {
      *kind = COLA_LEAF_LOWRANK;
      *rows = f->rows;
      *cols = f->rank;
    }
  });
}

cola_status cola_linop_release(cola_linop* op) {
  return guard([&] {
    COLA_REQUIRE(op, COLA_ERR_INVALID_ARG, "op is NULL");
    if (--op->refs <= 0) delete op;
  });
}

cola_status cola_set_split_terms(cola_ctx* ctx, int32_t factor_terms, int32_t vector_terms) {
  return guard([&] {
    COLA_REQUIRE(ctx, COLA_ERR_INVALID_ARG, "ctx is NULL");
    COLA_REQUIRE(factor_terms >= 1 && factor_terms <= 3 && vector_terms >= 1 && vector_terms <= 3,
                 COLA_ERR_INVALID_ARG, "split terms must be 1..3");
    ctx->split_factor_terms = factor_terms;
    ctx->split_vector_terms = vector_terms;
  });
}

cola_status cola_test_stall_next_launch(cola_ctx* ctx, int64_t wait_ns) {
  return guard([&] {
    COLA_REQUIRE(ctx, COLA_ERR_INVALID_ARG, "ctx is NULL");
    COLA_REQUIRE(wait_ns >= 0 && wait_ns <= 2000000000LL, COLA_ERR_INVALID_ARG,
                 "wait_ns = %lld (0 .. 2e9)", (long long)wait_ns);
    ctx->tc_stall_ns = wait_ns;
  });
}

cola_status cola_kernel_launches(const cola_ctx* ctx, int64_t* count) {
  return guard([&] {
    COLA_REQUIRE(ctx && count, COLA_ERR_INVALID_ARG, "NULL argument");
    *count = ctx->launches;
  });
}

cola_status cola_get_stream(const cola_ctx* ctx, cola_stream* stream) {
  return guard([&] {
    COLA_REQUIRE(ctx && stream, COLA_ERR_INVALID_ARG, "NULL argument");
    *stream = (cola_stream)ctx->s;
  });
}

cola_status cola_matvec(cola_ctx* ctx, const cola_linop* op, const void* X, void* Y,
                        int64_t nrhs, cola_precision prec, cola_stream stream) {
  return guard([&] {
    COLA_REQUIRE(ctx && op && X && Y, COLA_ERR_INVALID_ARG, "NULL argument");
    COLA_REQUIRE(nrhs >= 1, COLA_ERR_INVALID_ARG, "nrhs = %lld", (long long)nrhs);
    COLA_REQUIRE(prec >= COLA_PREC_F64 && prec <= COLA_PREC_MIXED, COLA_ERR_INVALID_ARG,
                 "precision %d", (int)prec);
    COLA_REQUIRE(X != Y, COLA_ERR_INVALID_ARG, "X and Y must not alias");
    StreamJoin j(ctx, stream);
    cola_linop* m = const_cast<cola_linop*>(op);
    prepare_leaves(ctx, m, prec, ctx->split_factor_terms);
    if (prec == COLA_PREC_F64)
      apply<double>(ctx, op, (const double*)X, (double*)Y, nrhs, 1.0, 0.0, 0, false, prec);
    else
      apply<float>(ctx, op, (const float*)X, (float*)Y, nrhs, 1.0, 0.0, 0, false, prec);
    if (prec == COLA_PREC_MIXED) tc_check_error_async(ctx);
  });
}

cola_status cola_rademacher(cola_ctx* ctx, uint64_t seed, int64_t offset, int64_t count,
                            void* out, cola_dtype dtype, cola_stream stream) {
  return guard([&] {
    COLA_REQUIRE(ctx && out, COLA_ERR_INVALID_ARG, "NULL argument");
    COLA_REQUIRE(offset >= 0 && count >= 0, COLA_ERR_INVALID_ARG, "negative offset/count");
    check_dtype(dtype);
    StreamJoin j(ctx, stream);
    rademacher(ctx, seed, offset, count, out, dtype);
  });
}

cola_status cola_bilinear_grad(cola_ctx* ctx, const cola_linop* op, const void* U, const void* X,
                               const double* weights, int64_t nrhs, int32_t prec,
                               void* const* grads, int32_t accumulate, cola_stream stream) {
  return guard([&] {
    COLA_REQUIRE(ctx && op && U && X && grads, COLA_ERR_INVALID_ARG, "NULL argument");
    COLA_REQUIRE(nrhs >= 1, COLA_ERR_INVALID_ARG, "nrhs = %lld", (long long)nrhs);
    StreamJoin j(ctx, stream);
    bilinear_entry(ctx, op, U, X, weights, nrhs, prec, grads, accumulate, 0);
  });
}

}  // extern "C"
