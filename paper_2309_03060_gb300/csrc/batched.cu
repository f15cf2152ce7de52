// Many independent SPD systems A_s = c_k K1_s (x) K2_s + c_d Diag(d_s) (uneven
// factor sizes and right-hand-side counts) solved together by mixed-precision
// CG with FP64 reliable updates (the same iteration as krylov.cu).
//
// All right-hand sides of all systems live in packed buffers; one right-hand
// side of one system is a "segment".  The host builds integer work tables once
// (bit-exact, deterministic order):
//   * tensor-core problem and tile tables for the two Kronecker mode steps of
//     every live system (k_kron_tc<ProbTable>, one persistent launch per step),
//   * a block table cutting every live segment into chunks for the
//     segmented vector kernels, with each segment's block range,
//   * each segment's range of p^T A p partials written by the mode-step epilogue.
// A CG iteration is five launches over all systems (mode step 1 with the
// fused p update, mode step 2 with the fused shift and p^T A p partials,
// alpha, x/r update, beta), and a chunk of iterations is one CUDA-graph replay.
// Systems whose right-hand sides have all converged retire: the host rewrites
// the tables (and their live counts) between replays, so the captured graph
// stays valid.  FP64 residual replacements run only for the systems that ask.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"

namespace cola {

namespace {

struct SegBlock {
  int32_t seg;
  int32_t pad;
  int64_t start;
  int64_t len;
};

struct SegShift {  // shift term of a segment's system: coeff * d (stride 0: d[0])
  const double* d;
  int64_t stride;
  int64_t off;     // element offset of the segment within the packed vectors
  double coeff;
};

constexpr int kChunkElems = 8192;

__device__ __forceinline__ void block_sum_pair(double& x, double& y) {
  __shared__ double sh[2][32];
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
  if (threadIdx.x < 32) {
    const bool ok = l < (int)(blockDim.x >> 5);
    x = ok ? sh[0][l] : 0.0;
    y = ok ? sh[1][l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, o);
      y += __shfl_xor_sync(0xffffffffu, y, o);
    }
  }
}

// x += alpha p; r -= alpha Ap; partials of r^T r (twice: rz = rr without a preconditioner)
// Segment blocks in reverse order: the MVM before ends with the last systems'
// Ap (still in L2) and the pre-split pass after starts with the first systems'
// r (left in L2 by this pass).  Each block's result is the same in any order.
__global__ void k_seg_xr(const SegBlock* blk, const int* nblk, float* x, float* r, const float* p,
                         const float* Ap, const CgState* st, double* part_rz, double* part_rr) {
  const int nb = *nblk;
  for (int bb = blockIdx.x; bb < nb; bb += gridDim.x) {
    const int b = nb - 1 - bb;
    const SegBlock B = blk[b];
    const float a = (float)st[B.seg].alpha;
    float s = 0.0f;
    const int64_t end = B.start + B.len;
    // four elements per thread per pass, every load issued before the stores
    for (int64_t i0 = B.start + threadIdx.x; i0 < end; i0 += 4 * (int64_t)blockDim.x) {
      float ri[4], xi[4], pi[4], ai[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t i = i0 + (int64_t)u * blockDim.x;
        const bool in = i < end;
        ri[u] = in ? r[i] : 0.0f;
        xi[u] = (in && a != 0.0f) ? x[i] : 0.0f;
        pi[u] = (in && a != 0.0f) ? p[i] : 0.0f;
        ai[u] = (in && a != 0.0f) ? Ap[i] : 0.0f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t i = i0 + (int64_t)u * blockDim.x;
        if (i < end && a != 0.0f) {
          x[i] = fmaf(a, pi[u], xi[u]);
          ri[u] = fmaf(-a, ai[u], ri[u]);
          r[i] = ri[u];
        }
        s = fmaf(ri[u], ri[u], s);
      }
    }
    double t = s, u = 0.0;
    block_sum_pair(t, u);
    if (threadIdx.x == 0) {
      part_rz[b] = t;
      part_rr[b] = t;
    }
  }
}

// r = (float) r64; partials of r^T r
__global__ void k_seg_refresh(const SegBlock* blk, const int* nblk, const double* r64, float* r,
                              double* part_rz, double* part_rr) {
  const int nb = *nblk;
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    const SegBlock B = blk[b];
    float s = 0.0f;
    for (int64_t i = B.start + threadIdx.x; i < B.start + B.len; i += blockDim.x) {
      const float ri = (float)r64[i];
      r[i] = ri;
      s = fmaf(ri, ri, s);
    }
    double t = s, u = 0.0;
    block_sum_pair(t, u);
    if (threadIdx.x == 0) {
      part_rz[b] = t;
      part_rr[b] = t;
    }
  }
}

// partials of a^T b in FP64 per block
__global__ void k_seg_dot64(const SegBlock* blk, const int* nblk, const double* a, const double* bb,
                            double* part) {
  const int nb = *nblk;
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    const SegBlock B = blk[b];
    double s = 0.0;
    for (int64_t i = B.start + threadIdx.x; i < B.start + B.len; i += blockDim.x)
      s = fma(a[i], bb[i], s);
    double u = 0.0;
    block_sum_pair(s, u);
    if (threadIdx.x == 0) part[b] = s;
  }
}

__global__ void k_seg_sum(const int* seg_list, const int* nseg, const int* seg_b0,
                          const int* seg_nb, const double* part, double* out) {
  const int n = *nseg;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int g = seg_list[k];
    double s = 0.0;
    for (int j = 0; j < seg_nb[g]; ++j) s += part[seg_b0[g] + j];
    out[g] = s;
  }
}

__global__ void k_seg_restate(CgState* st, const int* seg_list, const int* nseg,
                              const int* seg_b0, const int* seg_nb, const double* part_rr,
                              const double* rr64, const double* bb, double tol, int first) {
  const int n = *nseg;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int g = seg_list[k];
    CgState& s = st[g];
    double rr = 0.0;
    for (int j = 0; j < seg_nb[g]; ++j) rr += part_rr[seg_b0[g] + j];
    if (first) {
      s.iters = 0;
      s.updates = 0;
      s.status = 0;
      s.bb = bb[g];
      s.tol2 = tol * tol * bb[g];
      s.active = 1;
      s.alpha = s.beta = 0.0;
    } else if (s.active) {
      s.updates += 1;
    }
    s.flag = 0;
    s.rz = rr;
    s.rr = rr;
    s.rr_ref = rr;
    s.rr64 = rr64[g];
    if (s.active && rr64[g] <= s.tol2) s.active = 0;
  }
}

__global__ void k_seg_alpha(CgState* st, const int* seg_list, const int* nseg,
                            const int64_t* seg_p0, const int* seg_pn, const double* tdot) {
  const int n = *nseg;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int g = seg_list[k];
    CgState& s = st[g];
    if (!s.active) {
      s.alpha = 0.0;
      continue;
    }
    double v = 0.0;
    for (int j = 0; j < seg_pn[g]; ++j) v += tdot[seg_p0[g] + j];
    s.pAp = v;
    if (!(v > 0.0) || !isfinite(v)) {
      s.status = COLA_ERR_BREAKDOWN;
      s.active = 0;
      s.alpha = 0.0;
      continue;
    }
    s.alpha = s.rz / v;
  }
}

__global__ void k_seg_beta(CgState* st, const int* seg_list, const int* nseg, const int* seg_b0,
                           const int* seg_nb, const double* part_rr, double delta2,
                           double* beta_vec) {
  const int n = *nseg;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int g = seg_list[k];
    CgState& s = st[g];
    if (!s.active) {
      s.beta = 0.0;
      beta_vec[g] = 0.0;
      continue;
    }
    double rr = 0.0;
    for (int j = 0; j < seg_nb[g]; ++j) rr += part_rr[seg_b0[g] + j];
    s.beta = rr / s.rz;
    s.rz = rr;
    s.rr = rr;
    s.iters += 1;
    if (!isfinite(rr)) {
      s.status = COLA_ERR_BREAKDOWN;
      s.active = 0;
      s.beta = 0.0;
    } else if (rr <= s.tol2 || rr <= delta2 * s.rr_ref) {
      s.flag = 1;
    }
    beta_vec[g] = s.active ? s.beta : 0.0;
  }
}

__global__ void k_seg_copy_active(const SegBlock* blk, const int* nblk, const float* src,
                                  float* dst, const CgState* st) {
  const int nb = *nblk;
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    const SegBlock B = blk[b];
    if (!st[B.seg].active) continue;
    for (int64_t i = B.start + threadIdx.x; i < B.start + B.len; i += blockDim.x) dst[i] = src[i];
  }
}

__global__ void k_seg_accum(const SegBlock* blk, const int* nblk, double* x64, float* x) {
  const int nb = *nblk;
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    const SegBlock B = blk[b];
    for (int64_t i = B.start + threadIdx.x; i < B.start + B.len; i += blockDim.x) {
      x64[i] += (double)x[i];
      x[i] = 0.0f;
    }
  }
}

// r64 = b64 - shift * x64 (the Kronecker part is subtracted by the grouped GEMM)
__global__ void k_seg_resid_init(const SegBlock* blk, const int* nblk, const SegShift* sh,
                                 const double* b64, const double* x64, double* r64) {
  const int nb = *nblk;
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    const SegBlock B = blk[b];
    const SegShift S = sh[B.seg];
    for (int64_t i = B.start + threadIdx.x; i < B.start + B.len; i += blockDim.x) {
      const double d = S.stride ? S.d[i - S.off] : S.d[0];
      r64[i] = b64[i] - S.coeff * d * x64[i];
    }
  }
}

}  // namespace

// Host tables of one set of segments.
struct SegTables {
  std::vector<SegBlock> blocks;
  std::vector<int> seg_list, seg_b0, seg_nb;
};

struct BatchSys {
  const cola_linop* op;
  const cola_linop* kron;
  const cola_linop* diag;
  const cola_linop* f1;
  const cola_linop* f2;
  double ck, cd;
  int64_t n1, n2, N, R, off, g0;
};

static bool batch_shape_ok(const cola_linop* op, BatchSys& s) {
  if (op->kind != LK_SUM || op->kids.size() != 2) return false;
  int ik = -1, id = -1;
  for (int i = 0; i < 2; ++i) {
    if (op->kids[i]->kind == LK_KRON) ik = i;
    if (op->kids[i]->kind == LK_DIAG) id = i;
  }
  if (ik < 0 || id < 0) return false;
  const cola_linop* k = op->kids[ik];
  if (k->kids.size() != 2) return false;
  for (auto* f : k->kids)
    if (f->kind != LK_DENSE || f->rows != f->cols) return false;
  s.op = op;
  s.kron = k;
  s.diag = op->kids[id];
  s.f1 = k->kids[0];
  s.f2 = k->kids[1];
  s.ck = op->coeffs[ik];
  s.cd = op->coeffs[id];
  s.n1 = s.f1->rows;
  s.n2 = s.f2->rows;
  s.N = s.n1 * s.n2;
  return true;
}

static SegTables seg_tables(const std::vector<BatchSys>& sys, const std::vector<char>& live) {
  SegTables t;
  for (size_t s = 0; s < sys.size(); ++s) {
    if (!live[s]) continue;
    for (int64_t r = 0; r < sys[s].R; ++r) {
      const int g = (int)(sys[s].g0 + r);
      t.seg_list.push_back(g);
      const int64_t start = sys[s].off + r * sys[s].N;
      const int b0 = (int)t.blocks.size();
      for (int64_t c = 0; c < sys[s].N; c += kChunkElems)
        t.blocks.push_back(SegBlock{g, 0, start + c, std::min<int64_t>(kChunkElems, sys[s].N - c)});
      (void)b0;
    }
  }
  return t;
}

struct DevSeg {
  SegBlock* blocks;
  int* nblk;
  int* seg_list;
  int* nseg;
  int* seg_b0;
  int* seg_nb;
  int grid;
};

// Upload tables (fixed capacity, so replays of captured graphs stay valid).
static DevSeg upload_seg(Ctx* c, const char* tag, const SegTables& t, int64_t cap_blocks,
                         int64_t G) {
  DevSeg d;
  const std::string p(tag);
  d.blocks = (SegBlock*)c->ws.get(p + ".blk", sizeof(SegBlock) * cap_blocks);
  d.nblk = (int*)c->ws.get(p + ".nblk", 8);
  d.seg_list = (int*)c->ws.get(p + ".segs", 4 * G);
  d.nseg = (int*)c->ws.get(p + ".nseg", 8);
  d.seg_b0 = (int*)c->ws.get(p + ".b0", 4 * G);
  d.seg_nb = (int*)c->ws.get(p + ".nb", 4 * G);
  std::vector<int> b0(G, 0), nb(G, 0);
  for (size_t b = 0; b < t.blocks.size(); ++b) {
    const int g = t.blocks[b].seg;
    if (nb[g] == 0) b0[g] = (int)b;
    nb[g] += 1;
  }
  const int nblk = (int)t.blocks.size(), nseg = (int)t.seg_list.size();
  if (nblk)
    COLA_CUDA(cudaMemcpyAsync(d.blocks, t.blocks.data(), sizeof(SegBlock) * nblk,
                              cudaMemcpyHostToDevice, c->s));
  if (nseg)
    COLA_CUDA(cudaMemcpyAsync(d.seg_list, t.seg_list.data(), 4 * nseg, cudaMemcpyHostToDevice,
                              c->s));
  COLA_CUDA(cudaMemcpyAsync(d.seg_b0, b0.data(), 4 * G, cudaMemcpyHostToDevice, c->s));
  COLA_CUDA(cudaMemcpyAsync(d.seg_nb, nb.data(), 4 * G, cudaMemcpyHostToDevice, c->s));
  COLA_CUDA(cudaMemcpyAsync(d.nblk, &nblk, 4, cudaMemcpyHostToDevice, c->s));
  COLA_CUDA(cudaMemcpyAsync(d.nseg, &nseg, 4, cudaMemcpyHostToDevice, c->s));
  COLA_CUDA(cudaStreamSynchronize(c->s));
  d.grid = (int)std::max<int64_t>(1, std::min<int64_t>(cap_blocks, (int64_t)c->num_sms * 8));
  return d;
}

// output-chunk cap of the batched tensor-core launch before tuning
constexpr int kBatchChunkCap = 128;

static unsigned small_grid(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + 127) / 128); }

cola_status batched_cg_fast(Ctx* c, int32_t nsys, const cola_linop* const* ops,
                            const void* const* Bin, void* const* Xout, const int64_t* nrhs,
                            const cola_cg_opts& o, cola_cg_info* info, bool* handled) {
  *handled = false;
  if (o.precision != COLA_PREC_MIXED || !o.refine || o.jacobi || o.kron_precond) return COLA_OK;
  std::vector<BatchSys> sys(nsys);
  int64_t tot = 0, G = 0, maxn = 0, max_m = 0;
  for (int s = 0; s < nsys; ++s) {
    if (!batch_shape_ok(ops[s], sys[s])) return COLA_OK;
    sys[s].R = nrhs[s];
    sys[s].off = tot;
    sys[s].g0 = G;
    tot += (sys[s].N * nrhs[s] + 31) / 32 * 32;  // each system starts on a 128-byte boundary
    G += nrhs[s];
    maxn = std::max({maxn, sys[s].n1, sys[s].n2});
    max_m = std::max({max_m, sys[s].n1, sys[s].n2});
  }
  *handled = true;
  const int tf = o.split_factor_terms, tv = o.split_vector_terms;
  VectorTermsScope vterms(c, tv);
  for (int s = 0; s < nsys; ++s) {
    cola_linop* m = const_cast<cola_linop*>(ops[s]);
    prepare_leaves(c, m, COLA_PREC_MIXED, tf);
    prepare_leaves(c, m, COLA_PREC_F64, tf);
  }
  auto& ws = c->ws;
  float* x = (float*)ws.get("bcg.x", 4 * tot);
  float* r = (float*)ws.get("bcg.r", 4 * tot);
  float* pbuf[2] = {(float*)ws.get("bcg.p", 4 * tot), (float*)ws.get("bcg.p2", 4 * tot)};
  float* p = pbuf[0];  // search direction at parity 0 (set-up writes here)
  float* Ap = (float*)ws.get("bcg.Ap", 4 * tot);
  float* T1 = (float*)ws.get("bcg.T1", 4 * tot);
  double* x64 = (double*)ws.get("bcg.x64", 8 * tot);
  double* b64 = (double*)ws.get("bcg.b64", 8 * tot);
  double* r64 = (double*)ws.get("bcg.r64", 8 * tot);
  double* T64 = (double*)ws.get("bcg.T64", 8 * tot);
  CgState* st = (CgState*)ws.get("bcg.st", sizeof(CgState) * G);
  double* beta_vec = (double*)ws.get("bcg.beta", 8 * G);
  double* bb = (double*)ws.get("bcg.bb", 8 * G);
  double* rr64 = (double*)ws.get("bcg.rr64", 8 * G);
  SegShift* shift = (SegShift*)ws.get("bcg.shift", sizeof(SegShift) * G);
  int64_t cap_blocks = 0;
  for (auto& s : sys) cap_blocks += s.R * ((s.N + kChunkElems - 1) / kChunkElems);
  double* part_rz = (double*)ws.get("bcg.prz", 8 * cap_blocks);
  double* part_rr = (double*)ws.get("bcg.prr", 8 * cap_blocks);

  // p^T A p partial slots: fixed per system (8 per tile of mode step 2); the
  // tile count depends on the output-chunk width (the tuned N tile)
  std::vector<int64_t> tiles2(nsys), tdot_off(nsys);
  auto tdot_layout = [&](int cap) {
    int64_t tot2 = 0;
    for (int s = 0; s < nsys; ++s) {
      // step 2 contracts n2: rest = n1, output chunks over n2 (see make_plan)
      int chunks = 1;
      kron_tc_chunk_width((int)sys[s].n2, cap, &chunks);
      tiles2[s] = (sys[s].n1 + 127) / 128 * chunks;  // per right-hand side
      tdot_off[s] = tot2;
      tot2 += 8 * tiles2[s] * sys[s].R;
    }
    return tot2;
  };
  int64_t tdot_cap = 1;
  for (int cap : {64, 128}) tdot_cap = std::max(tdot_cap, tdot_layout(cap));
  double* tdot = (double*)ws.get("bcg.tdot", 8 * tdot_cap);
  // widest output chunk over the batch under a chunk cap (sizes the stages)
  auto max_chunk_for = [&](int cap) {
    int mc = 16;
    for (auto& s : sys) {
      int nc = 1;
      mc = std::max({mc, kron_tc_chunk_width((int)s.n1, cap, &nc),
                     kron_tc_chunk_width((int)s.n2, cap, &nc)});
    }
    return mc;
  };
  int64_t* seg_p0 = (int64_t*)ws.get("bcg.sp0", 8 * G);
  int* seg_pn = (int*)ws.get("bcg.spn", 4 * G);
  auto upload_slot_tables = [&] {
    std::vector<int64_t> hp0(G);
    std::vector<int> hpn(G);
    std::vector<SegShift> hs(G);
    for (int s = 0; s < nsys; ++s)
      for (int64_t q = 0; q < sys[s].R; ++q) {
        const int64_t g = sys[s].g0 + q;
        hp0[g] = tdot_off[s] + 8 * tiles2[s] * q;
        hpn[g] = (int)(8 * tiles2[s]);
        hs[g] = SegShift{leaf_ptr<double>(sys[s].diag), sys[s].diag->stride,
                         sys[s].off + q * sys[s].N, sys[s].cd};
      }
    COLA_CUDA(cudaMemcpyAsync(seg_p0, hp0.data(), 8 * G, cudaMemcpyHostToDevice, c->s));
    COLA_CUDA(cudaMemcpyAsync(seg_pn, hpn.data(), 4 * G, cudaMemcpyHostToDevice, c->s));
    COLA_CUDA(cudaMemcpyAsync(shift, hs.data(), sizeof(SegShift) * G, cudaMemcpyHostToDevice,
                              c->s));
    COLA_CUDA(cudaStreamSynchronize(c->s));
  };
  constexpr int kChunkGemm = 128;  // output chunk of the split GEMM form
  int tile_cap = kBatchChunkCap, tile_stages = 0;  // set by the tuner below
  bool use_gemm = false;  // split GEMM form of the mode steps (tuner's choice)
  tdot_layout(tile_cap);
  upload_slot_tables();

  // inputs into the packed FP64 right-hand side
  for (int s = 0; s < nsys; ++s)
    COLA_CUDA(cudaMemcpyAsync(b64 + sys[s].off, Bin[s], 8 * sys[s].N * sys[s].R,
                              cudaMemcpyDeviceToDevice, c->s));
  fill_zero<double>(c, x64, tot);
  fill_zero<float>(c, x, tot);
  COLA_CUDA(cudaMemsetAsync(beta_vec, 0, 8 * G, c->s));

  std::vector<char> live(nsys, 1);
  // live-set tables used inside the graph
  // Two table sets: parity q reads p from pbuf[q] and writes p_new to pbuf[q ^ 1]
  // (re-reads of the same X rows by several output chunks stay idempotent).
  static const char* kTc1[2] = {"bcg.tc1a", "bcg.tc1b"};
  static const char* kTc2[2] = {"bcg.tc2a", "bcg.tc2b"};
  static const char* kGm1[2] = {"bcg.gm1a", "bcg.gm1b"};
  static const char* kGm2[2] = {"bcg.gm2a", "bcg.gm2b"};
  auto tc_tables = [&](const std::vector<char>& lv) {
    tdot_layout(tile_cap);
    for (int q = 0; q < 2; ++q) {
      std::vector<TcBatchProblem> s1, s2;
      for (int s = 0; s < nsys; ++s) {
        if (!lv[s]) continue;
        const BatchSys& b = sys[s];
        TcBatchProblem q1{};
        q1.X = pbuf[q] + b.off;
        q1.Y = T1 + b.off;
        q1.factor = b.f1;
        q1.rest = b.n2;
        q1.size_in = b.N;
        q1.size_out = b.N;
        q1.R = b.R;
        q1.coeff = 1.0f;
        q1.pro_z = r + b.off;
        q1.pro_beta = beta_vec + b.g0;
        q1.pro_out = pbuf[q ^ 1] + b.off;
        s1.push_back(q1);
        TcBatchProblem q2{};
        q2.X = T1 + b.off;
        q2.Y = Ap + b.off;
        q2.factor = b.f2;
        q2.rest = b.n1;
        q2.size_in = b.N;
        q2.size_out = b.N;
        q2.R = b.R;
        q2.coeff = (float)b.ck;
        q2.epi_x = pbuf[q ^ 1] + b.off;
        q2.epi_d = leaf_ptr<float>(b.diag);
        q2.epi_dstride = b.diag->stride;
        q2.epi_coeff = (float)b.cd;
        q2.epi_dot = tdot + tdot_off[s];
        s2.push_back(q2);
      }
      if (use_gemm) {
        // step 1's epilogue writes step 2's image (two-factor systems)
        kron_tc_gemm_batch_upload_pair(c, s1, s2, tf, tv, kGm1[q], kGm2[q], "bcg.gimg1",
                                       "bcg.gimg2");
      } else {
        kron_tc_batch_upload(c, s1, tf, tv, kTc1[q], tile_cap);
        kron_tc_batch_upload(c, s2, tf, tv, kTc2[q], tile_cap);
      }
    }
  };

  // FP64 true residual r64 = b64 - A x64 for the systems in `which`
  auto residual64 = [&](const std::vector<char>& which, const DevSeg& dseg) {
    k_seg_resid_init<<<dseg.grid, 256, 0, c->s>>>(dseg.blocks, dseg.nblk, shift, b64, x64, r64);
    c->count_launch();
    std::vector<GemmDesc<double>> g1, g2;
    int64_t mm = 1, nn = 1;
    for (int s = 0; s < nsys; ++s) {
      if (!which[s]) continue;
      const BatchSys& b = sys[s];
      const double* F1 = leaf_ptr<double>(b.f1);
      const double* F2 = leaf_ptr<double>(b.f2);
      for (int64_t q = 0; q < b.R; ++q) {
        const int64_t o = b.off + q * b.N;
        // step 1: T[rest = n2][i1] = sum_j X[j1][rest] K1[i1][j1]
        g1.push_back(GemmDesc<double>{b.n2, b.n1, b.n1, x64 + o, 1, b.n2, F1, 1, b.n1, T64 + o,
                                      b.n1, 1, 1.0, 0.0});
        // step 2: r[rest = n1][i2] -= ck sum_j T[j2][rest] K2[i2][j2]
        g2.push_back(GemmDesc<double>{b.n1, b.n2, b.n2, T64 + o, 1, b.n1, F2, 1, b.n2, r64 + o,
                                      b.n2, 1, -b.ck, 1.0});
        mm = std::max({mm, b.n1, b.n2});
        nn = std::max({nn, b.n1, b.n2});
      }
    }
    const int ng = (int)g1.size();
    for (int base = 0; base < ng; base += 65535) {
      const int cnt = std::min(65535, ng - base);
      auto* d1 = (GemmDesc<double>*)ws.get("bcg.g1", sizeof(GemmDesc<double>) * 65535);
      auto* d2 = (GemmDesc<double>*)ws.get("bcg.g2", sizeof(GemmDesc<double>) * 65535);
      COLA_CUDA(cudaMemcpyAsync(d1, g1.data() + base, sizeof(GemmDesc<double>) * cnt,
                                cudaMemcpyHostToDevice, c->s));
      COLA_CUDA(cudaMemcpyAsync(d2, g2.data() + base, sizeof(GemmDesc<double>) * cnt,
                                cudaMemcpyHostToDevice, c->s));
      gemm_grouped<double>(c, d1, cnt, mm, nn);
      gemm_grouped<double>(c, d2, cnt, mm, nn);
      COLA_CUDA(cudaStreamSynchronize(c->s));  // host descriptor vectors go out of scope
    }
    k_seg_dot64<<<dseg.grid, 256, 0, c->s>>>(dseg.blocks, dseg.nblk, r64, r64, part_rr);
    c->count_launch();
    k_seg_sum<<<small_grid(G), 128, 0, c->s>>>(dseg.seg_list, dseg.nseg, dseg.seg_b0,
                                               dseg.seg_nb, part_rr, rr64);
    c->count_launch();
  };

  // ---------------------------------------------------------------- set-up
  DevSeg live_seg = upload_seg(c, "bcg.live", seg_tables(sys, live), cap_blocks, G);
  {
    k_seg_dot64<<<live_seg.grid, 256, 0, c->s>>>(live_seg.blocks, live_seg.nblk, b64, b64,
                                                 part_rr);
    c->count_launch();
    k_seg_sum<<<small_grid(G), 128, 0, c->s>>>(live_seg.seg_list, live_seg.nseg, live_seg.seg_b0,
                                               live_seg.seg_nb, part_rr, bb);
    c->count_launch();
    residual64(live, live_seg);  // r64 = b (x64 = 0)
    k_seg_refresh<<<live_seg.grid, 256, 0, c->s>>>(live_seg.blocks, live_seg.nblk, r64, r,
                                                   part_rz, part_rr);
    c->count_launch();
    k_seg_restate<<<small_grid(G), 128, 0, c->s>>>(st, live_seg.seg_list, live_seg.nseg,
                                                   live_seg.seg_b0, live_seg.seg_nb, part_rr,
                                                   rr64, bb, o.tol, 1);
    c->count_launch();
    k_seg_copy_active<<<live_seg.grid, 256, 0, c->s>>>(live_seg.blocks, live_seg.nblk, r, p, st);
    c->count_launch();
    COLA_CUDA(cudaGetLastError());
  }
  // Autotuner: the output-chunk width (N tile, 64 or 128 columns) and the
  // pipeline depth of the streaming table kernel, and the split GEMM form
  // (pre-split pass + table-driven GEMM, 128-output chunks), are timed on this
  // batch's own mode steps (CUDA events, parity-0 tables; outputs go to
  // scratch buffers the first iteration rewrites), and the fastest is cached
  // per (terms, histogram of factor sizes and RHS counts).
  {
    std::map<std::tuple<int, int, int64_t>, int> hist;
    for (auto& s : sys)
      ++hist[std::make_tuple((int)((s.n1 + 31) / 32), (int)((s.n2 + 31) / 32), s.R)];
    std::string tkey = "bt:" + std::to_string(tf) + std::to_string(tv);
    for (auto& kv : hist)
      tkey += ":" + std::to_string(std::get<0>(kv.first)) + "," +
              std::to_string(std::get<1>(kv.first)) + "," + std::to_string(std::get<2>(kv.first)) +
              "x" + std::to_string(kv.second);
    auto hit = c->tuned.find(tkey);
    if (hit != c->tuned.end()) {
      tile_cap = hit->second.first;
      tile_stages = hit->second.second;
      use_gemm = tile_stages < 0;
    } else {
      cudaEvent_t e0, e1;
      COLA_CUDA(cudaEventCreate(&e0));
      COLA_CUDA(cudaEventCreate(&e1));
      float best = 1e30f;
      int best_cap = kBatchChunkCap, best_st = 0;
      for (int cap : {64, 128}) {
        if (cap == 128 && max_chunk_for(64) == max_chunk_for(128)) continue;  // same tiles
        tile_cap = cap;
        tc_tables(live);
        const int mc = max_chunk_for(cap);
        for (int stg = 2; stg <= kron_tc_batch_max_stages(tf, tv, mc); ++stg) {
          kron_tc_batch_launch(c, kTc1[0], tf, tv, mc, stg);  // warm-up
          kron_tc_batch_launch(c, kTc2[0], tf, tv, mc, stg);
          COLA_CUDA(cudaEventRecord(e0, c->s));
          for (int rep = 0; rep < 2; ++rep) {
            kron_tc_batch_launch(c, kTc1[0], tf, tv, mc, stg);
            kron_tc_batch_launch(c, kTc2[0], tf, tv, mc, stg);
          }
          COLA_CUDA(cudaEventRecord(e1, c->s));
          COLA_CUDA(cudaEventSynchronize(e1));
          float ms = 0.0f;
          COLA_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          if (ms < best) {
            best = ms;
            best_cap = cap;
            best_st = stg;
          }
        }
      }
      {
        use_gemm = true;
        tile_cap = kChunkGemm;
        tc_tables(live);
        kron_tc_gemm_batch_launch(c, kGm1[0], tf, tv);  // warm-up
        kron_tc_gemm_batch_launch(c, kGm2[0], tf, tv, false);
        COLA_CUDA(cudaEventRecord(e0, c->s));
        for (int rep = 0; rep < 2; ++rep) {
          kron_tc_gemm_batch_launch(c, kGm1[0], tf, tv);
          kron_tc_gemm_batch_launch(c, kGm2[0], tf, tv, false);
        }
        COLA_CUDA(cudaEventRecord(e1, c->s));
        COLA_CUDA(cudaEventSynchronize(e1));
        float ms = 0.0f;
        COLA_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
          best = ms;
          best_cap = kChunkGemm;
          best_st = -1;  // the split GEMM form
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      tc_check_error(c);
      tile_cap = best_cap;
      tile_stages = best_st;
      use_gemm = tile_stages < 0;
      c->tuned[tkey] = std::make_pair(tile_cap, tile_stages);
    }
    const char* tr = getenv("COLA_TRACE");
    if (tr && tr[0] == '1') {
      if (use_gemm)
        fprintf(stderr, "[cola batched] split GEMM form\n");
      else
        fprintf(stderr, "[cola batched] N tile <= %d columns, %d stages\n", tile_cap,
                tile_stages);
    }
  }
  tc_tables(live);
  upload_slot_tables();
  const double delta2 = o.reliable_delta * o.reliable_delta;
  const int max_chunk = max_chunk_for(tile_cap);
  int cur = 0;  // parity: the current search direction is pbuf[cur]
  auto iteration = [&] {
    if (use_gemm) {
      kron_tc_gemm_batch_launch(c, kGm1[cur], tf, tv);
      kron_tc_gemm_batch_launch(c, kGm2[cur], tf, tv, false);
    } else {
      kron_tc_batch_launch(c, kTc1[cur], tf, tv, max_chunk, tile_stages);
      kron_tc_batch_launch(c, kTc2[cur], tf, tv, max_chunk, tile_stages);
    }
    float* p_new = pbuf[cur ^ 1];
    cur ^= 1;
    k_seg_alpha<<<small_grid(G), 128, 0, c->s>>>(st, live_seg.seg_list, live_seg.nseg, seg_p0,
                                                 seg_pn, tdot);
    c->count_launch();
    k_seg_xr<<<live_seg.grid, 256, 0, c->s>>>(live_seg.blocks, live_seg.nblk, x, r, p_new, Ap,
                                              st, part_rz, part_rr);
    c->count_launch();
    k_seg_beta<<<small_grid(G), 128, 0, c->s>>>(st, live_seg.seg_list, live_seg.nseg,
                                                live_seg.seg_b0, live_seg.seg_nb, part_rr, delta2,
                                                beta_vec);
    c->count_launch();
    COLA_CUDA(cudaGetLastError());
  };

  CgState* hst = (CgState*)c->host_pinned(sizeof(CgState) * G);
  auto read_state = [&] {
    COLA_CUDA(cudaMemcpyAsync(hst, st, sizeof(CgState) * G, cudaMemcpyDeviceToHost, c->s));
    COLA_CUDA(cudaStreamSynchronize(c->s));
  };
  read_state();
  int chunk = std::max(2, o.graph_chunk);
  chunk += chunk & 1;  // even: every replay starts and ends on the same p buffer
  int64_t iters = 0;
  bool any = false;
  for (int64_t g = 0; g < G; ++g) any |= hst[g].active != 0;
  if (any && o.maxiter > 0) {
    iteration();  // sizes every buffer before capture
    iters = 1;
  }
  char key[160];
  snprintf(key, sizeof key, "bcg:%llu:%d:%lld:%d:%d%d:%.17g:%llu:p%d",
           (unsigned long long)ops[0]->uid, nsys, (long long)G, chunk, tf, tv, delta2,
           (unsigned long long)ws.generation, cur);
  cudaGraphExec_t exec = nullptr;
  int64_t graph_kernels = 0;
  int updates = 0;
  const char* tr_env = getenv("COLA_TRACE");
  const bool trace = tr_env && tr_env[0] == '1';
  while (any && iters < o.maxiter) {
    if (!exec) {
      auto it = c->graphs.find(key);
      if (it != c->graphs.end() && it->second.generation == ws.generation) {
        exec = it->second.exec;
        graph_kernels = it->second.kernels;
      } else {
        cudaGraph_t gph;
        const uint64_t gen0 = ws.generation;
        COLA_CUDA(cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal));
        c->capturing = true;
        c->captured = 0;
        try {
          for (int i = 0; i < chunk; ++i) iteration();
        } catch (...) {
          c->capturing = false;
          cudaStreamEndCapture(c->s, &gph);
          throw;
        }
        c->capturing = false;
        COLA_CUDA(cudaStreamEndCapture(c->s, &gph));
        COLA_REQUIRE(gen0 == ws.generation, COLA_ERR_CUDA,
                     "internal: workspace moved during graph capture");
        GraphEntry e;
        COLA_CUDA(cudaGraphInstantiate(&e.exec, gph, 0));
        cudaGraphDestroy(gph);
        e.kernels = c->captured;
        e.generation = ws.generation;
        c->graphs[key] = e;
        exec = e.exec;
        graph_kernels = e.kernels;
      }
    }
    COLA_CUDA(cudaGraphLaunch(exec, c->s));
    c->launches += graph_kernels;
    iters += chunk;
    read_state();
    // systems asking for a residual replacement, and systems still live
    std::vector<char> want(nsys, 0), still(nsys, 0);
    bool anyw = false;
    any = false;
    for (int s = 0; s < nsys; ++s)
      for (int64_t q = 0; q < sys[s].R; ++q) {
        const CgState& h = hst[sys[s].g0 + q];
        if (h.active) {
          still[s] = 1;
          any = true;
          if (h.flag) {
            want[s] = 1;
            anyw = true;
          }
        }
      }
    if (anyw && updates < o.max_updates) {
      DevSeg ws_seg = upload_seg(c, "bcg.upd", seg_tables(sys, want), cap_blocks, G);
      k_seg_accum<<<ws_seg.grid, 256, 0, c->s>>>(ws_seg.blocks, ws_seg.nblk, x64, x);
      c->count_launch();
      residual64(want, ws_seg);
      k_seg_refresh<<<ws_seg.grid, 256, 0, c->s>>>(ws_seg.blocks, ws_seg.nblk, r64, r, part_rz,
                                                   part_rr);
      c->count_launch();
      k_seg_restate<<<small_grid(G), 128, 0, c->s>>>(st, ws_seg.seg_list, ws_seg.nseg,
                                                     ws_seg.seg_b0, ws_seg.seg_nb, part_rr, rr64,
                                                     bb, o.tol, 0);
      c->count_launch();
      ++updates;
      read_state();
      any = false;
      std::fill(still.begin(), still.end(), 0);
      for (int s = 0; s < nsys; ++s)
        for (int64_t q = 0; q < sys[s].R; ++q)
          if (hst[sys[s].g0 + q].active) {
            still[s] = 1;
            any = true;
          }
    }
    if (still != live) {
      // retire converged systems: rewrite the tables the graph reads
      live = still;
      live_seg = upload_seg(c, "bcg.live", seg_tables(sys, live), cap_blocks, G);
      tc_tables(live);
    }
    if (trace) {
      int nl = 0;
      for (char v : live) nl += v;
      fprintf(stderr, "[cola batched] iter %lld live systems %d updates %d\n", (long long)iters,
              nl, updates);
    }
    if (updates >= o.max_updates) break;
  }

  // final FP64 solution and true residuals for every system
  std::vector<char> all(nsys, 1);
  DevSeg all_seg = upload_seg(c, "bcg.all", seg_tables(sys, all), cap_blocks, G);
  k_seg_accum<<<all_seg.grid, 256, 0, c->s>>>(all_seg.blocks, all_seg.nblk, x64, x);
  c->count_launch();
  residual64(all, all_seg);
  tc_check_error(c);
  for (int s = 0; s < nsys; ++s)
    COLA_CUDA(cudaMemcpyAsync(Xout[s], x64 + sys[s].off, 8 * sys[s].N * sys[s].R,
                              cudaMemcpyDeviceToDevice, c->s));
  std::vector<double> hrr(G), hbb(G);
  COLA_CUDA(cudaMemcpyAsync(hrr.data(), rr64, 8 * G, cudaMemcpyDeviceToHost, c->s));
  COLA_CUDA(cudaMemcpyAsync(hbb.data(), bb, 8 * G, cudaMemcpyDeviceToHost, c->s));
  read_state();
  cola_status result = COLA_OK;
  for (int64_t g = 0; g < G; ++g) {
    const double rel = hbb[g] > 0 ? std::sqrt(std::max(hrr[g], 0.0) / hbb[g]) : 0.0;
    int stt = hst[g].status;
    if (stt == 0 && !(rel <= o.tol)) stt = COLA_ERR_NOT_CONVERGED;
    if (stt != 0 && result == COLA_OK) result = (cola_status)stt;
    if (info) {
      info[g].iterations = hst[g].iters;
      info[g].rel_residual = rel;
      info[g].updates = hst[g].updates;
      info[g].status = stt;
    }
  }
  return result;
}

}  // namespace cola
