// Kronecker mode products on the tcgen05 tensor cores (sm_103a).
//
// One mode step of the Kronecker MVM (Sec. 3.2, Table 3) contracts the leading
// index of the current layout [j, rest] with a factor K (n_out x n_in):
//     D[rest, i] = sum_j X[j, rest] * K[i, j]
// which is a GEMM with M = rest, N = n_out, K = n_in per right-hand side.
// Operands are split into BF16 terms (x = x_0 + x_1 [+ x_2], each the
// round-to-nearest BF16 of the remainder) and the cross products whose term
// indices sum to less than max(T_f, T_v) accumulate in FP32 in tensor memory.
//
// Kernel layout (persistent, one 288-thread CTA per SM):
//   warps 0-3  producers: load FP32 X, split to BF16 terms, write the A tile
//              (128 rows x 64 k, K-major, 128-byte swizzle) into a pipeline
//              stage; thread 0 also bulk-copies the pre-split factor tile
//              (cp.async.bulk, completes on the stage's mbarrier).
//   warp 8     MMA issuer: waits for a full stage, issues tcgen05.mma for
//              every 16-wide k step and term pair, commits to the stage's
//              empty barrier; after the tile, commits to the accumulator's
//              full barrier.  Also allocates / frees TMEM.
//   warps 4-7  epilogue: tcgen05.ld the FP32 accumulator (warp w reads TMEM
//              lanes 32(w-4)..), Y = coeff * D + beta * Y, store.
// Accumulators are double-buffered in TMEM so the epilogue of one tile
// overlaps the MMAs of the next.  Every mbarrier wait gives up after ~2 s,
// raises an error flag and lets the CTA drain and free its TMEM.
#include <cuda.h>  // CUtensorMap (types only; the encoder comes from the runtime's entry point)
#include <cuda_bf16.h>

#include <stdio.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>

#include "internal.h"

namespace cola {

namespace {

constexpr int kTileM = 128;
constexpr int kBlockK = 64;               // bf16 elements per 128-byte swizzled row
constexpr int kProducerThreads = 128;
constexpr int kThreadsTc = 288;
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s per wait
constexpr int kDotSlots = 8;  // p . Ap partials per tile (one per epilogue warp slot)

struct TcParams {
  const float* X;
  float* Y;
  const uint16_t* Bimg;  // [tf][kblocks][n_pad rows][64] bf16, 128-byte swizzled rows
  int64_t rest, size_in, size_out, batch, tiles_m, ntiles;
  int n_in, n_out, n_pad, kblocks, ksteps_last, tf, tv, stages, nbuf;
  int img_rows;          // rows per (term, k block) of the split factor image (>= n_pad)
  int n_chunk, nchunks;  // output columns per tile (<= 256) and chunks per row tile
  uint32_t stage_bytes, a_term_bytes, b_term_bytes, tmem_cols;
  float coeff, beta;
  int* err;
  uint64_t stall_ns;  // > 0: the MMA role first waits on a barrier that nothing
                      // completes, with this limit (test of the time-out path)
  // optional prologue (first mode step of a CG iteration): the input is
  // p = z + beta_r * p_old, computed here and written back to X in place
  const float* pro_z;
  const double* pro_beta;
  float* pro_out;  // where p is written (never the input X: tiles of several
                   // output chunks re-read the same X rows)
  // pro_out without pro_z: the input is pro_beta[r] * X (a per-vector scale,
  // the Lanczos normalisation q = w / beta), written to pro_out
  // optional Lanczos term of the epilogue: Y -= epi_gamma[r] * epi_q2 (the
  // previous basis vector), before the partial sums of epi_x . Y
  const float* epi_q2;
  const double* epi_gamma;
  int out_trans;  // 1: store Y[r][i][m] (output index major) instead of Y[r][m][i]
  double* pro_nrm;  // with pro_z: per (tile, warp) partials of the formed input's ||p||^2
  int rev;          // factor-stationary kernel: tiles in reverse order (same results)
                    // (factor-stationary kernel)
  // optional epilogue (last mode step, output in the input's layout):
  // Y += epi_coeff * d * epi_x (d = epi_d[0] when epi_dstride == 0), and the
  // per-(tile, epilogue warp) partial sums of epi_x . Y go to epi_dot[4 tile + warp]
  const float* epi_x;
  const float* epi_d;
  int64_t epi_dstride;
  float epi_coeff;
  double* epi_dot;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Arrive once and add `bytes` to the phase's expected transaction count.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(
                   smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false when the phase did not complete within limit_ns (the
// role then raises the CTA's abort flag and the device error flag) or another
// role of the CTA already gave up.
__device__ __noinline__ bool mbar_wait_slow(uint64_t* bar, uint32_t parity,
                                            volatile int* abort_flag, int* err,
                                            uint64_t limit_ns) {
  const uint64_t t0 = now_ns();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63) == 0) {
      if (*abort_flag) return false;
      if (now_ns() - t0 > limit_ns) {
        *abort_flag = 1;
        atomicExch(err, COLA_ERR_TIMEOUT);
        return false;
      }
    }
  }
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          int* err) {
  if (mbar_try_wait(bar, parity)) return true;
  return mbar_wait_slow(bar, parity, abort_flag, err, kWaitNs);
}

// Wait for this CTA's own bulk copies or MMAs to complete before it frees
// tensor memory and exits: it does not give up when another role raised the
// abort flag (the copies are in flight whatever the other roles do), only
// after its own limit of kWaitNs.
__device__ __noinline__ bool mbar_wait_own(uint64_t* bar, uint32_t parity, int* err) {
  const uint64_t t0 = now_ns();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63) == 0 && now_ns() - t0 > kWaitNs) {
      atomicExch(err, COLA_ERR_TIMEOUT);
      return false;
    }
  }
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// SMEM matrix descriptor: K-major operand, 128-byte swizzle, 8-row atoms of
// 1024 bytes (stride-dimension offset 1024), version 1 (bits 46-47).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;                // leading-dimension offset (unused for this layout)
  d |= (uint64_t)(1024u >> 4) << 32;      // stride-dimension offset
  d |= (uint64_t)1u << 46;                // descriptor version
  d |= (uint64_t)2u << 61;                // SWIZZLE_128B
  return d;
}

// Instruction descriptor, kind::f16: BF16 x BF16 -> FP32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4)                          // D format F32
         | (1u << 7)                        // A format BF16
         | (1u << 10)                       // B format BF16
         | ((uint32_t)(N >> 3) << 17)       // N / 8
         | ((uint32_t)(M >> 4) << 24);      // M / 16
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Split two FP32 values into up to three BF16x2 terms (round to nearest even).
__device__ __forceinline__ void split2(float a, float b, int terms, uint32_t* out) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  out[0] = *reinterpret_cast<uint32_t*>(&h);
  if (terms > 1) {
    const float ra = a - __low2float(h), rb = b - __high2float(h);
    __nv_bfloat162 l = __floats2bfloat162_rn(ra, rb);
    out[1] = *reinterpret_cast<uint32_t*>(&l);
    if (terms > 2) {
      __nv_bfloat162 l2 = __floats2bfloat162_rn(ra - __low2float(l), rb - __high2float(l));
      out[2] = *reinterpret_cast<uint32_t*>(&l2);
    }
  }
}

// Per-tile parameter sources of k_kron_tc: one problem passed by value, or a
// device table of problems (many independent systems in one launch).
struct OneProb {
  TcParams p;
  __device__ __forceinline__ int64_t count() const { return p.ntiles; }
  __device__ __forceinline__ const TcParams& get(int64_t t, int64_t& lt) const {
    lt = t;
    return p;
  }
};

struct ProbTable {
  const TcParams* probs;   // one entry per problem
  const int* tile_prob;    // problem of every global tile
  const int64_t* first;    // first global tile of every problem
  const int64_t* count_dev;  // number of live tiles (read at kernel start)
  __device__ __forceinline__ int64_t count() const { return *count_dev; }
  __device__ __forceinline__ const TcParams& get(int64_t t, int64_t& lt) const {
    const int pid = tile_prob[t];
    lt = t - first[pid];
    return probs[pid];
  }
};

template <class Src>
__global__ void __launch_bounds__(kThreadsTc, 1) k_kron_tc(Src src, TcParams K) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned stage area
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(base + (size_t)K.stages * K.stage_bytes);
  uint64_t* full = bars;
  uint64_t* empty = bars + K.stages;
  uint64_t* acc_full = bars + 2 * K.stages;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  uint64_t* cbar = drain + 1;        // [stages] factor copies of each stage
  uint64_t* stall = cbar + K.stages;  // never completed (time-out test)
  uint32_t* tmem_slot = (uint32_t*)(stall + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < K.stages; ++s) {
      mbar_init(&full[s], kProducerThreads);
      mbar_init(&empty[s], 1);
      mbar_init(&cbar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 128);
    }
    mbar_init(drain, 1);
    mbar_init(stall, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(K.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp < 4) {
    // ------------------------------------------------------------ producers
    int s = 0;
    uint32_t ph = 0;
    uint32_t issued = 0, issued_ph = 0;  // bit s: a copy went to stage s / its parity
    bool ok = true;
    const int64_t ntiles = src.count();
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      int64_t lt;
      const TcParams p = src.get(t, lt);  // by value: one read of the table entry per tile
      const int64_t tm = lt / p.nchunks;
      const int nc = (int)(lt % p.nchunks);
      const int64_t r = tm / p.tiles_m, m0 = (tm % p.tiles_m) * kTileM;
      const float* Xb = p.X + r * p.size_in;
      const float* Pb = Xb;
      float* Pw = p.pro_out ? p.pro_out + r * p.size_in : nullptr;
      const float* Zb = p.pro_z ? p.pro_z + r * p.size_in : nullptr;
      const float beta_r = p.pro_z ? (float)p.pro_beta[r] : 0.0f;
      const int64_t m = m0 + tid;
      (void)r;
      const bool row_ok = m < p.rest;
      for (int kb = 0; kb < p.kblocks; ++kb) {
        if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, K.err)) {
          ok = false;
          break;
        }
        unsigned char* st = base + (size_t)s * K.stage_bytes;
        if (tid == 0) {
          // the factor block lands on its own barrier, so its completion can
          // be awaited whatever the other producers do
          mbar_arrive_expect_tx(&cbar[s], p.b_term_bytes * K.tf);
          for (int ti = 0; ti < K.tf; ++ti)
            bulk_g2s(st + K.tv * K.a_term_bytes + ti * p.b_term_bytes,
                     p.Bimg + (((size_t)ti * p.kblocks + kb) * (size_t)p.img_rows +
                               (size_t)nc * p.n_chunk) * kBlockK,
                     p.b_term_bytes, &cbar[s]);
          issued |= 1u << s;
          issued_ph = (issued_ph & ~(1u << s)) | (ph << s);
        }
        const int k0 = kb * kBlockK;
        float v[kBlockK];
        if (Zb) {
#pragma unroll
          for (int g = 0; g < kBlockK; g += 16) {
            float zz[16], pp[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              const int kk = k0 + g + k;
              const bool in = row_ok && kk < p.n_in;
              const int64_t idx = (int64_t)kk * p.rest + m;
              zz[k] = in ? Zb[idx] : 0.0f;
              pp[k] = in ? Pb[idx] : 0.0f;
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              const int kk = k0 + g + k;
              v[g + k] = fmaf(beta_r, pp[k], zz[k]);
              if (row_ok && kk < p.n_in) Pw[(int64_t)kk * p.rest + m] = v[g + k];
            }
          }
        } else if (Pw) {
          // scaled input, written back: q = beta_r x
          const float sc = (float)p.pro_beta[r];
#pragma unroll
          for (int k = 0; k < kBlockK; ++k) {
            const int kk = k0 + k;
            const bool in = row_ok && kk < p.n_in;
            v[k] = in ? sc * Pb[(int64_t)kk * p.rest + m] : 0.0f;
            if (in) Pw[(int64_t)kk * p.rest + m] = v[k];
          }
        } else {
#pragma unroll
          for (int k = 0; k < kBlockK; ++k) {
            const int kk = k0 + k;
            v[k] = (row_ok && kk < p.n_in) ? __ldg(Xb + (int64_t)kk * p.rest + m) : 0.0f;
          }
        }
        const uint32_t row_off = (uint32_t)tid * 128u;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          uint32_t w[3][4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            uint32_t o[3];
            split2(v[8 * c + 2 * e], v[8 * c + 2 * e + 1], K.tv, o);
            w[0][e] = o[0];
            w[1][e] = o[1];
            w[2][e] = o[2];
          }
          const uint32_t off = row_off + ((uint32_t)(c ^ (tid & 7)) << 4);
#pragma unroll
          for (int tv = 0; tv < 3; ++tv) {
            if (tv < K.tv)
              *reinterpret_cast<uint4*>(st + tv * K.a_term_bytes + off) =
                  make_uint4(w[tv][0], w[tv][1], w[tv][2], w[tv][3]);
          }
        }
        fence_proxy_async();
        mbar_arrive(&full[s]);
        if (++s == K.stages) {
          s = 0;
          ph ^= 1u;
        }
      }
    }
    // no bulk copy may still be landing in this CTA's shared memory when it
    // exits: earlier copies into a stage were consumed before the stage was
    // refilled, so only the latest copy of each stage can be in flight
    if (tid == 0)
      for (int st = 0; st < K.stages; ++st)
        if (issued & (1u << st)) mbar_wait_own(&cbar[st], (issued_ph >> st) & 1u, K.err);
  } else if (warp == 8) {
    // ----------------------------------------------------------------- MMA
    if (lane == 0) {
      const int maxt = K.tf > K.tv ? K.tf : K.tv;
      int s = 0;
      uint32_t ph = 0;
      int64_t it = 0;
      bool ok = true;
      if (K.stall_ns) ok = mbar_wait_slow(stall, 0, abort_flag, K.err, K.stall_ns);
      const int64_t ntiles = src.count();
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++it) {
        int64_t lt;
        const TcParams p = src.get(t, lt);  // by value: one read of the table entry per tile
        const uint32_t idesc = idesc_bf16(kTileM, p.n_chunk);
        const int b = (int)(it % K.nbuf);
        const uint32_t use = (uint32_t)((it / K.nbuf) & 1);
        if (!mbar_wait(&acc_empty[b], use ^ 1u, abort_flag, K.err)) break;
        tc_fence_after();
        // hi x hi products accumulate in d_big; every smaller cross term in
        // d_small, so the rounding of each MMA's accumulate step on the
        // dominant sum happens once per k step only.
        // buffer stride from the launch-wide widest chunk (K.n_chunk), so
        // problems of different widths never share accumulator columns
        const uint32_t d_big = tmem_base + (uint32_t)(b * 2 * K.n_chunk);
        const uint32_t d_small = d_big + (uint32_t)p.n_chunk;
        uint32_t acc_big = 0, acc_small = 0;
        for (int kb = 0; kb < p.kblocks; ++kb) {
          if (!mbar_wait(&full[s], ph, abort_flag, K.err) ||
              !mbar_wait(&cbar[s], ph, abort_flag, K.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(base + (size_t)s * K.stage_bytes);
          const int steps = (kb == p.kblocks - 1) ? p.ksteps_last : 4;
          for (int kk = 0; kk < steps; ++kk) {
            for (int ti = 0; ti < K.tf; ++ti)
              for (int tv = 0; tv < K.tv; ++tv) {
                if (ti + tv >= maxt) continue;
                const uint64_t ad = sw128_desc(st + tv * K.a_term_bytes + kk * 32);
                const uint64_t bd =
                    sw128_desc(st + K.tv * K.a_term_bytes + ti * p.b_term_bytes + kk * 32);
                if (ti == 0 && tv == 0) {
                  mma_bf16(d_big, ad, bd, idesc, acc_big);
                  acc_big = 1;
                } else {
                  mma_bf16(d_small, ad, bd, idesc, acc_small);
                  acc_small = 1;
                }
              }
          }
          mma_commit(&empty[s]);
          if (++s == K.stages) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (!ok) break;
        mma_commit(&acc_full[b]);
      }
      // drain: all MMAs issued by this thread have completed
      mma_commit(drain);
      mbar_wait_own(drain, 0, K.err);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp - 4;
    const int row = q * 32 + lane;
    int64_t it = 0;
    const bool has_small = (K.tf > 1 || K.tv > 1);
    const int64_t ntiles = src.count();
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      const int b = (int)(it % K.nbuf);
      if (!mbar_wait(&acc_full[b], (uint32_t)((it / K.nbuf) & 1), abort_flag, K.err)) break;
      tc_fence_after();
      int64_t lt;
      const TcParams p = src.get(t, lt);  // by value: one read of the table entry per tile
      const int64_t tm = lt / p.nchunks;
      const int nc = (int)(lt % p.nchunks);
      const int64_t r = tm / p.tiles_m, m0 = (tm % p.tiles_m) * kTileM;
      const int64_t m = m0 + row;
      const int ncol0 = nc * p.n_chunk;   // first output column of this tile
      const int ncols = min(p.n_chunk, p.n_out - ncol0);
      float* yrow = p.Y + r * p.size_out + m * p.n_out + ncol0;
      // 16-byte stores only where the row really is 16-byte aligned
      const bool vec_ok = ((reinterpret_cast<uintptr_t>(yrow) & 15u) == 0);
      const float* xrow = p.epi_x ? p.epi_x + r * p.size_out + m * p.n_out + ncol0 : nullptr;
      const int64_t dbase = m * p.n_out + ncol0;
      const float gam = p.epi_q2 ? (float)p.epi_gamma[r] : 0.0f;
      const float* q2row = p.epi_q2 ? p.epi_q2 + r * p.size_out + m * p.n_out + ncol0 : nullptr;
      double dot = 0.0;
      const uint32_t taddr =
          tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * 2 * K.n_chunk);
      for (int c0 = 0; c0 < p.n_chunk; c0 += 16) {
        uint32_t v[16], w[16];
        tmem_ld16(taddr + (uint32_t)c0, v);
        if (has_small) {
          tmem_ld16(taddr + (uint32_t)(p.n_chunk + c0), w);
        } else {
#pragma unroll
          for (int e = 0; e < 16; ++e) w[e] = 0u;
        }
        float a[16];
#pragma unroll
        for (int e = 0; e < 16; ++e)
          a[e] = p.coeff * (__uint_as_float(v[e]) + __uint_as_float(w[e]));
        if (xrow && m < p.rest) {
          float xd[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int i = c0 + e;
            xd[e] = (i < ncols) ? xrow[i] : 0.0f;
          }
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int i = c0 + e;
            const float dv = p.epi_dstride ? (i < ncols ? p.epi_d[dbase + i] : 0.0f) : p.epi_d[0];
            a[e] = fmaf(p.epi_coeff * dv, xd[e], a[e]);
            if (gam != 0.0f && i < ncols) a[e] = fmaf(-gam, __ldg(q2row + i), a[e]);
            if (p.beta == 0.0f && i < ncols) dot += (double)(a[e] * xd[e]);
          }
        }
        if (m < p.rest) {
          if (c0 + 16 <= ncols && vec_ok) {
#pragma unroll
            for (int e = 0; e < 16; e += 4) {
              float4 o = make_float4(a[e], a[e + 1], a[e + 2], a[e + 3]);
              float4* dst = reinterpret_cast<float4*>(yrow + c0 + e);
              if (p.beta != 0.0f) {
                const float4 old = *dst;
                o.x += p.beta * old.x;
                o.y += p.beta * old.y;
                o.z += p.beta * old.z;
                o.w += p.beta * old.w;
              }
              *dst = o;
            }
          } else {
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const int i = c0 + e;
              if (i < ncols) {
                float o = a[e];
                if (p.beta != 0.0f) o += p.beta * yrow[i];
                yrow[i] = o;
              }
            }
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&acc_empty[b]);
      if (p.epi_dot) {
        // one partial per (tile, epilogue warp); summed in fixed order later
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        if (lane == 0) {
          p.epi_dot[lt * kDotSlots + q] = dot;
          p.epi_dot[lt * kDotSlots + 4 + q] = 0.0;  // this kernel fills 4 of the 8 slots
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 8) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(K.tmem_cols)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Factor-stationary variant (factor sides <= 128, rows of X 16-byte aligned).
// The mode step runs transposed, D^T[i, m] = sum_j K[i, j] X[j, m]: the split
// factor is the MMA's A operand and stays in tensor memory for the whole
// launch, the split X tile is the B operand in shared memory, and accumulator
// lane i holds output i of every row m of the tile, so the 32 lanes of an
// epilogue warp store 32 consecutive outputs of one row (128-byte stores).
//   warp 17     loader: per 64-wide k block of a tile, one 2-D TMA copy of the
//               64 x 128 FP32 block of X (and one of z for the fused p update)
//               into a multi-stage staging ring.
//   warps 0-7   converters: thread (row m, k half) reads its 32 staged values,
//               forms p = z + beta p when fused (writing p back), splits them
//               into BF16 terms and stores the B stage (K-major rows of 64
//               BF16, 128-byte swizzle), then fences it for the tensor core.
//   warp 16     MMA: tcgen05.mma, A = factor term (tensor memory), B = X term
//               (shared memory); dominant / cross terms in separate
//               accumulators; allocates / frees tensor memory.
//   warps 8-15  epilogue: first copy the split factor into tensor memory; per
//               tile drain both accumulators into registers, release them,
//               then store (with the fused shift term and p . Ap partials).
//   warp 18     when the shift term is fused: the tile's rows of p (contiguous
//               in the output layout) with one cp.async.bulk into shared
//               memory, so the epilogue reads them without global latency.
// TMEM columns: [0, 128) dominant accumulator, [128, 256) cross terms,
// [256 + 64 t, ...) factor term t (32 columns per 64-wide k block).
constexpr int kFsConvWarps = 8;
constexpr int kFsEpiWarps = 8;
constexpr int kFsMmaWarp = kFsConvWarps + kFsEpiWarps;  // 16
constexpr int kFsLoaderWarp = kFsMmaWarp + 1;           // 17
constexpr int kFsEpiLoaderWarp = kFsLoaderWarp + 1;     // 18
constexpr int kThreadsFs = 32 * (kFsEpiLoaderWarp + 1); // 608
constexpr int kFsConvThreads = 32 * kFsConvWarps;
constexpr int kFsEpiThreads = 32 * kFsEpiWarps;
constexpr uint32_t kFsSmallCol = 128;
constexpr uint32_t kFsFactorCol0 = 256;
constexpr uint32_t kFsBTermBytes = kTileM * 128;  // 128 rows x 64 BF16

struct TcFsParams {
  CUtensorMap tm_x;  // X as [R * n_in rows][rest], box 64 rows x 128
  CUtensorMap tm_z;  // z, same shape (fused p update only)
  const uint16_t* Bimg;  // split factor [tf][kblocks][n_pad][64] BF16, swizzled rows
  float* Y;
  int64_t rest, size_in, size_out, tiles_m, ntiles;
  int n_in, n_out, n_pad, kblocks, ksteps_last, xstages, nsrc;
  int img_rows;  // rows per (term, k block) of the split factor image
  int e_mode;  // epilogue: 0 store; 1 fused shift term and p . Ap partials; 2 add beta Y;
               // 5 store transposed, Y[r][i][m] (output index major: slab-major layout)
               // 3 as 1 with a per-element diagonal

  uint32_t x_src_bytes, e_bytes;  // e_bytes: rows staged per tile for e_mode 1 and 2
  const float* e_src;             // staged rows: p (e_mode 1) or the old Y (e_mode 2)
  float coeff, beta, e_coeff;     // e_coeff: coefficient of the shift term (e_mode 1)
  const float* e_d;               // its diagonal: d[0] (e_mode 1) or d[N] (e_mode 3), device
  int* err;
  uint64_t stall_ns;              // > 0: time-out test (see TcParams)
  const double* pro_beta;
  float* pro_out;
  double* epi_dot;
  int pro_scale;          // 1: the input is pro_beta[r] * X, written to pro_out
  const float* e_q2;      // e_mode 4: previous Lanczos vector (output layout)
  const double* e_gamma;  // e_mode 4: its coefficient per right-hand side
  double* pro_nrm;        // two-source input: per (tile, converter warp) partials of ||p||^2
  int rev;                // tiles in reverse order (same results; L2 reuse between kernels)
};

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
      "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15])
      : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7])
      : "r"(taddr));
}

__device__ __forceinline__ void mma_bf16_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// 2-D tiled TMA load of the box at (x, y) of a tensor map into shared memory.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Converts this thread's 32 values of one staged 64-wide k block (row `row`,
// k half `khalf`) into TV BF16 terms: logical 16-byte chunk c of the row goes
// to chunk position c ^ (row & 7) of each term's B stage.  NSRC == 2 first
// forms p = z + beta_r p and writes it to Pout (row m of p, k stride `rest`).
// FULL: the row and the whole block are in range, nothing is masked.
// NSRC == 2 also adds the squares of the formed values to nrm.
// NSRC == 0: the staged values times beta_r, written to Pout (the Lanczos
// normalisation q = w / beta).
template <int TV, int NSRC, bool FULL>
__device__ __forceinline__ void fs_convert(const float* st, const float* stz, unsigned char* brow,
                                           int row, int khalf, int kbase, int n_in, bool row_ok,
                                           float beta_r, float* Pout, int64_t rest, float& nrm) {
  const uint32_t swz = (uint32_t)(row & 7);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int kl = khalf * 32 + j * 8 + e;
      const bool in = FULL || (row_ok && kbase + kl < n_in);
      float x = in ? st[kl * kTileM + row] : 0.0f;
      if (NSRC > 1 && in) {
        x = fmaf(beta_r, x, stz[kl * kTileM + row]);
        Pout[(int64_t)(kbase + kl) * rest] = x;
        nrm = fmaf(x, x, nrm);
      } else if (NSRC == 0 && in) {
        x = beta_r * x;
        Pout[(int64_t)(kbase + kl) * rest] = x;
      }
      v[e] = x;
    }
    uint32_t w[TV][4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      uint32_t o[3];
      split2(v[2 * e], v[2 * e + 1], TV, o);
#pragma unroll
      for (int tv = 0; tv < TV; ++tv) w[tv][e] = o[tv];
    }
    const uint32_t chunk = ((uint32_t)(khalf * 4 + j) ^ swz) * 16u;
#pragma unroll
    for (int tv = 0; tv < TV; ++tv)
      *reinterpret_cast<uint4*>(brow + (size_t)tv * kFsBTermBytes + chunk) =
          make_uint4(w[tv][0], w[tv][1], w[tv][2], w[tv][3]);
  }
}

// Stores this thread's 64 outputs (rows c < nrows of its column half, output
// i): y = a (MODE 0), y = a + sc x with the partial sum of y x (MODE 1, x the
// staged p), y = a + sc y_old (MODE 2, y_old staged), y = a + sc d x with d
// read per element from dp (MODE 3, otherwise as MODE 1).
// MODE 4: as MODE 1, then y -= gam q2 (q2 read per element from dp).
template <int MODE>
__device__ __forceinline__ float fs_store(const float (&a)[64], float* yp, const float* es,
                                          int64_t ld, int nrows, float sc,
                                          const float* dp = nullptr, float gam = 0.0f) {
  float part = 0.0f;
#pragma unroll
  for (int c = 0; c < 64; ++c) {
    if (c < nrows) {
      float v = a[c];
      if (MODE == 1 || MODE == 3 || MODE == 4) {
        const float xd = es[c * ld];
        const float s = MODE == 3 ? sc * __ldg(dp + c * ld) : sc;
        v = fmaf(s, xd, v);
        if (MODE == 4 && gam != 0.0f) v = fmaf(-gam, __ldg(dp + c * ld), v);
        part = fmaf(v, xd, part);
      } else if (MODE == 2) {
        v = fmaf(sc, es[c * ld], v);
      }
      yp[c * ld] = v;
    }
  }
  return part;
}

template <int TF, int TV>
__global__ void __launch_bounds__(kThreadsFs, 1) k_kron_tc_fs(const __grid_constant__ TcFsParams p) {
  constexpr int kMaxT = TF > TV ? TF : TV;
  constexpr bool kSmall = TF > 1 || TV > 1;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned base for the swizzle atoms, still a shared-space pointer
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* bsm = base;                           // 2 B stages x TV terms
  unsigned char* xsm = base + 2 * TV * kFsBTermBytes;  // FP32 staging ring
  unsigned char* esm = xsm + (size_t)p.xstages * p.nsrc * p.x_src_bytes;  // epilogue rows
  uint64_t* bars = (uint64_t*)(esm + p.e_bytes);
  uint64_t* xfull = bars;
  uint64_t* xempty = xfull + p.xstages;
  uint64_t* bfull = xempty + p.xstages;
  uint64_t* bempty = bfull + 2;
  uint64_t* afac = bempty + 2;
  uint64_t* dfull = afac + 1;
  uint64_t* dempty = dfull + 1;
  uint64_t* drain = dempty + 1;
  uint64_t* efull = drain + 1;
  uint64_t* eempty = efull + 1;
  uint64_t* stall = eempty + 1;  // never completed (time-out test)
  uint32_t* tmem_slot = (uint32_t*)(stall + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < p.xstages; ++s) {
      mbar_init(&xfull[s], 1);
      mbar_init(&xempty[s], kFsConvThreads);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&bfull[s], kFsConvThreads);
      mbar_init(&bempty[s], 1);
    }
    mbar_init(afac, kFsEpiThreads);
    mbar_init(dfull, 1);
    mbar_init(dempty, kFsEpiThreads);
    mbar_init(drain, 1);
    mbar_init(efull, 1);
    mbar_init(eempty, kFsEpiThreads);
    mbar_init(stall, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kFsMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  // the next kernel may start its own set-up; every role below that touches
  // memory written or read by earlier kernels first waits for them (pdl_wait)
  pdl_trigger();

  if (warp == kFsLoaderWarp) {
    // ---------------------------------------------------------------- loader
    pdl_wait();
    if (lane == 0) {  // one thread waits, issues and tracks every copy
      bool ok = true;
      int s = 0;
      uint32_t ph = 0;
      uint32_t issued = 0, issued_ph = 0;  // bit s: a copy went to stage s / its parity
      for (int64_t t0 = blockIdx.x; t0 < p.ntiles && ok; t0 += gridDim.x) {
        const int64_t t = p.rev ? p.ntiles - 1 - t0 : t0;  // tile (order of rev)
        const int64_t r = t / p.tiles_m, m0 = (t % p.tiles_m) * kTileM;
        for (int kb = 0; kb < p.kblocks; ++kb) {
          if (!mbar_wait(&xempty[s], ph ^ 1u, abort_flag, p.err)) {
            ok = false;
            break;
          }
          // rows past n_in or columns past rest arrive as zeros or as another
          // right-hand side's rows; the converters mask both
          unsigned char* st = xsm + (size_t)s * p.nsrc * p.x_src_bytes;
          const int y = (int)(r * p.n_in) + kb * kBlockK;
          mbar_arrive_expect_tx(&xfull[s], p.x_src_bytes * (uint32_t)p.nsrc);
          tma_load_2d(st, &p.tm_x, (int)m0, y, &xfull[s]);
          if (p.nsrc > 1) tma_load_2d(st + p.x_src_bytes, &p.tm_z, (int)m0, y, &xfull[s]);
          issued |= 1u << s;
          issued_ph = (issued_ph & ~(1u << s)) | (ph << s);
          if (++s == p.xstages) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
      // no bulk copy may still be landing when the CTA exits: earlier copies
      // into a stage were consumed before the stage was refilled, so only the
      // latest copy of each stage can be in flight
      for (int st = 0; st < p.xstages; ++st)
        if (issued & (1u << st)) mbar_wait_own(&xfull[st], (issued_ph >> st) & 1u, p.err);
    }
    __syncwarp();
  } else if (warp == kFsEpiLoaderWarp) {
    // ------------------------------------------------ rows for the epilogue
    pdl_wait();
    if (lane == 0 && p.e_bytes) {
      int64_t it = 0;
      for (int64_t t0 = blockIdx.x; t0 < p.ntiles; t0 += gridDim.x, ++it) {
        const int64_t t = p.rev ? p.ntiles - 1 - t0 : t0;  // tile (order of rev)
        if (!mbar_wait(eempty, (uint32_t)(it & 1) ^ 1u, abort_flag, p.err)) break;
        const int64_t r = t / p.tiles_m, m0 = (t % p.tiles_m) * kTileM;
        const int64_t rows = (p.rest - m0 < kTileM) ? (p.rest - m0) : kTileM;
        const uint32_t bytes = (uint32_t)(rows * p.n_out) * 4u;
        mbar_arrive_expect_tx(efull, bytes);
        bulk_g2s(esm, p.e_src + r * p.size_out + m0 * p.n_out, bytes, efull);
      }
      // the last copy (the only one that can be in flight: each waited for
      // the epilogue to free the buffer) has landed before the CTA exits
      if (it > 0) mbar_wait_own(efull, (uint32_t)((it - 1) & 1), p.err);
    }
    __syncwarp();
  } else if (warp < kFsConvWarps) {
    // ------------------------------------------------------------ converters
    pdl_wait();
    bool ok = true;
    int s = 0, sb = 0;
    uint32_t ph = 0, phb = 0;
    const int quarter = warp & 3, khalf = warp >> 2;
    const int row = quarter * 32 + lane;
    for (int64_t t0 = blockIdx.x; t0 < p.ntiles && ok; t0 += gridDim.x) {
        const int64_t t = p.rev ? p.ntiles - 1 - t0 : t0;  // tile (order of rev)
      const int64_t r = t / p.tiles_m, m0 = (t % p.tiles_m) * kTileM;
      const int64_t m = m0 + row;
      const bool row_ok = m < p.rest;
      const bool pro = p.nsrc > 1 || p.pro_scale;
      const float beta_r = pro ? (float)p.pro_beta[r] : 0.0f;
      float* Pout = pro ? p.pro_out + r * p.size_in + m : nullptr;
      float nrm = 0.0f;  // squares of the formed values (two-source mode)
      for (int kb = 0; kb < p.kblocks; ++kb) {
        if (!mbar_wait(&bempty[sb], phb ^ 1u, abort_flag, p.err) ||
            !mbar_wait(&xfull[s], ph, abort_flag, p.err)) {
          ok = false;
          break;
        }
        const float* st = reinterpret_cast<const float*>(xsm + (size_t)s * p.nsrc * p.x_src_bytes);
        const float* stz = st + p.x_src_bytes / 4;
        unsigned char* brow = bsm + (size_t)sb * TV * kFsBTermBytes + (size_t)row * 128;
        const int kbase = kb * kBlockK;
        const bool full = row_ok && kbase + kBlockK <= p.n_in;
        if (p.nsrc > 1) {
          if (full)
            fs_convert<TV, 2, true>(st, stz, brow, row, khalf, kbase, p.n_in, row_ok, beta_r,
                                    Pout, p.rest, nrm);
          else
            fs_convert<TV, 2, false>(st, stz, brow, row, khalf, kbase, p.n_in, row_ok, beta_r,
                                     Pout, p.rest, nrm);
        } else if (p.pro_scale) {
          if (full)
            fs_convert<TV, 0, true>(st, stz, brow, row, khalf, kbase, p.n_in, row_ok, beta_r,
                                    Pout, p.rest, nrm);
          else
            fs_convert<TV, 0, false>(st, stz, brow, row, khalf, kbase, p.n_in, row_ok, beta_r,
                                     Pout, p.rest, nrm);
        } else {
          if (full)
            fs_convert<TV, 1, true>(st, stz, brow, row, khalf, kbase, p.n_in, row_ok, beta_r,
                                    Pout, p.rest, nrm);
          else
            fs_convert<TV, 1, false>(st, stz, brow, row, khalf, kbase, p.n_in, row_ok, beta_r,
                                     Pout, p.rest, nrm);
        }
        fence_proxy_async();
        mbar_arrive(&xempty[s]);
        mbar_arrive(&bfull[sb]);
        if (++s == p.xstages) {
          s = 0;
          ph ^= 1u;
        }
        if (++sb == 2) {
          sb = 0;
          phb ^= 1u;
        }
      }
      if (p.pro_nrm && ok) {
        // per (tile, converter warp) partial of the formed input's squared norm
        double dn = (double)nrm;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dn += __shfl_xor_sync(0xffffffffu, dn, o);
        if (lane == 0) p.pro_nrm[t * kDotSlots + warp] = dn;
      }
    }
  } else if (warp == kFsMmaWarp) {
    // ------------------------------------------------------------------- MMA
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(kTileM, kTileM);  // M = outputs, N = rows
      bool ok = mbar_wait(afac, 0, abort_flag, p.err);
      if (ok && p.stall_ns) ok = mbar_wait_slow(stall, 0, abort_flag, p.err, p.stall_ns);
      tc_fence_after();
      const uint32_t bbase = smem_u32(bsm);
      int sb = 0;
      uint32_t phb = 0;
      int64_t it = 0;
      for (int64_t t0 = blockIdx.x; t0 < p.ntiles && ok; t0 += gridDim.x, ++it) {
        if (!mbar_wait(dempty, (uint32_t)(it & 1) ^ 1u, abort_flag, p.err)) break;
        tc_fence_after();
        uint32_t acc_small = 0;
        for (int kb = 0; kb < p.kblocks; ++kb) {
          if (!mbar_wait(&bfull[sb], phb, abort_flag, p.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const int steps = (kb == p.kblocks - 1) ? p.ksteps_last : 4;
          const uint32_t bst = bbase + (uint32_t)sb * (uint32_t)TV * kFsBTermBytes;
          const uint32_t fa = tmem_base + kFsFactorCol0 + (uint32_t)kb * 32u;
          for (int kk = 0; kk < steps; ++kk) {
#pragma unroll
            for (int ti = 0; ti < TF; ++ti)
#pragma unroll
              for (int tv = 0; tv < TV; ++tv) {
                if (ti + tv >= kMaxT) continue;
                const uint32_t a = fa + (uint32_t)(ti * 64 + kk * 8);
                const uint64_t bd =
                    sw128_desc(bst + (uint32_t)tv * kFsBTermBytes + (uint32_t)kk * 32u);
                if (ti == 0 && tv == 0) {
                  mma_bf16_ta(tmem_base, a, bd, idesc, (kb | kk) ? 1u : 0u);
                } else {
                  mma_bf16_ta(tmem_base + kFsSmallCol, a, bd, idesc, acc_small);
                  acc_small = 1;
                }
              }
          }
          mma_commit(&bempty[sb]);
          if (++sb == 2) {
            sb = 0;
            phb ^= 1u;
          }
        }
        if (!ok) break;
        mma_commit(dfull);
      }
      mma_commit(drain);
      mbar_wait_own(drain, 0, p.err);
    }
    __syncwarp();
  } else {
    // -------------------------------------------------------------- epilogue
    const int ew = warp - kFsConvWarps;
    const int quarter = warp & 3, chalf = ew >> 2;
    const int i = quarter * 32 + lane;  // output index = TMEM lane
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    // the split factor: k block `chalf` of every term, row i (unswizzled)
    if (chalf < p.kblocks) {
#pragma unroll
      for (int ti = 0; ti < TF; ++ti) {
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          uint32_t u[16];
          if (i < p.n_pad) {
            const uint4* src = reinterpret_cast<const uint4*>(
                p.Bimg + ((size_t)(ti * p.kblocks + chalf) * p.img_rows + i) * kBlockK);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const uint4 q = __ldg(src + ((hh * 4 + c) ^ (i & 7)));
              u[4 * c] = q.x;
              u[4 * c + 1] = q.y;
              u[4 * c + 2] = q.z;
              u[4 * c + 3] = q.w;
            }
          } else {
#pragma unroll
            for (int c = 0; c < 16; ++c) u[c] = 0u;
          }
          tmem_st16(tmem_base + lane_off + kFsFactorCol0 +
                        (uint32_t)(ti * 64 + chalf * 32 + hh * 16),
                    u);
        }
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    mbar_arrive(afac);
    pdl_wait();  // the factor copy above overlaps the previous kernel's tail
    const bool staged = p.e_mode != 0 && p.e_mode != 5;
    const float sc = (p.e_mode == 1 || p.e_mode == 4) ? p.e_coeff * p.e_d[0]
                                                      : (p.e_mode == 3 ? p.e_coeff : p.beta);
    int64_t it = 0;
    for (int64_t t0 = blockIdx.x; t0 < p.ntiles; t0 += gridDim.x, ++it) {
        const int64_t t = p.rev ? p.ntiles - 1 - t0 : t0;  // tile (order of rev)
      if (staged && !mbar_wait(efull, (uint32_t)(it & 1), abort_flag, p.err)) break;
      if (!mbar_wait(dfull, (uint32_t)(it & 1), abort_flag, p.err)) break;
      tc_fence_after();
      const int64_t r = t / p.tiles_m, m0 = (t % p.tiles_m) * kTileM;
      const uint32_t taddr = tmem_base + lane_off + (uint32_t)(chalf * 64);
      float a[64];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        uint32_t v[8], w[8];
        tmem_ld8(taddr + (uint32_t)(q * 8), v);
        if (kSmall) tmem_ld8(taddr + kFsSmallCol + (uint32_t)(q * 8), w);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int e = 0; e < 8; ++e)
          a[q * 8 + e] =
              p.coeff * (__uint_as_float(v[e]) + (kSmall ? __uint_as_float(w[e]) : 0.0f));
      }
      tc_fence_before();
      mbar_arrive(dempty);
      // row m = mbase + c of the tile, output i: 32 lanes write 128 contiguous bytes
      const int64_t mbase = m0 + chalf * 64;
      const int nrows = (int)((p.rest - mbase < 64) ? (p.rest - mbase) : 64);
      float part = 0.0f;  // this thread's <= 64 products of p . Ap
      if (p.e_mode == 5) {
        // output index i major: this thread's rows m are contiguous.  Lanes
        // 2k and 2k + 1 (outputs i, i + 1) swap half of every 8-value group,
        // so that each pair of 16-byte stores fills a whole 32-byte sector of
        // one output row: the even lane stores the first halves, the odd lane
        // the second halves, of row i and then of row i + 1.
        const bool full = nrows == 64 && p.n_out % 2 == 0 && i < p.n_out;
        if (__all_sync(0xffffffffu, full)) {
          const bool odd = lane & 1;
          float* y0 = p.Y + r * p.size_out + (int64_t)(i & ~1) * p.rest + mbase;
#pragma unroll
          for (int g = 0; g < 8; ++g) {
            float recv[4];
#pragma unroll
            for (int e = 0; e < 4; ++e)
              recv[e] = __shfl_xor_sync(0xffffffffu, odd ? a[8 * g + e] : a[8 * g + 4 + e], 1);
            const int c0 = 8 * g + (odd ? 4 : 0);
            const float4 lo = make_float4(a[8 * g], a[8 * g + 1], a[8 * g + 2], a[8 * g + 3]);
            const float4 hi =
                make_float4(a[8 * g + 4], a[8 * g + 5], a[8 * g + 6], a[8 * g + 7]);
            const float4 rv = make_float4(recv[0], recv[1], recv[2], recv[3]);
            const float4 first = odd ? rv : lo;
            const float4 second = odd ? hi : rv;
            *reinterpret_cast<float4*>(y0 + c0) = first;
            *reinterpret_cast<float4*>(y0 + p.rest + c0) = second;
          }
        } else if (i < p.n_out && nrows > 0) {
          float* yt = p.Y + r * p.size_out + (int64_t)i * p.rest + mbase;
          if (nrows == 64) {
#pragma unroll
            for (int c = 0; c < 64; c += 4)
              *reinterpret_cast<float4*>(yt + c) = make_float4(a[c], a[c + 1], a[c + 2], a[c + 3]);
          } else {
#pragma unroll
            for (int c = 0; c < 64; ++c)
              if (c < nrows) yt[c] = a[c];
          }
        }
      } else if (i < p.n_out && nrows > 0) {
        const int64_t ld = p.n_out;
        float* yp = p.Y + r * p.size_out + mbase * ld + i;
        const float* es = reinterpret_cast<const float*>(esm) + chalf * 64 * ld + i;
        if (p.e_mode == 0)
          fs_store<0>(a, yp, es, ld, nrows, 0.0f);
        else if (p.e_mode == 1)
          part = fs_store<1>(a, yp, es, ld, nrows, sc);
        else if (p.e_mode == 3)
          part = fs_store<3>(a, yp, es, ld, nrows, sc, p.e_d + mbase * ld + i);
        else if (p.e_mode == 4)
          part = fs_store<4>(a, yp, es, ld, nrows, sc, p.e_q2 + r * p.size_out + mbase * ld + i,
                             (float)p.e_gamma[r]);
        else
          fs_store<2>(a, yp, es, ld, nrows, sc);
      }
      if (staged) mbar_arrive(eempty);
      if (p.epi_dot) {
        double dsum = (double)part;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
        if (lane == 0) p.epi_dot[t * kDotSlots + ew] = dsum;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kFsMmaWarp) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(512)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Split GEMM mode step for factors with a side above 128 (no factor in tensor
// memory).  A pre-split pass writes the mode step's input as K-major BF16
// term images (and forms the fused first-step input p = z + beta p or
// beta x on the way); the GEMM then moves both operands with copy engines
// only:
//   D[i, m] = sum_k K[i, k] X[m, k]   A = factor block (128 outputs x 64 k per
//   term, pre-split image, one cp.async.bulk each), B = X image block (128
//   rows x 64 k per term, 2-D TMA with the 128-byte swizzle); accumulator
//   lane i holds output i of the tile's rows, so the 32 lanes of an epilogue
//   warp store 32 consecutive outputs of one row.  With the whole of tensor
//   memory free for accumulators, the dominant / cross-term pair is
//   double-buffered (2 x 256 columns): the epilogue drains one tile while the
//   MMAs of the next run.
//   warp 0      loader (one lane)
//   warp 1      MMA (one lane), tensor-memory allocation
//   warps 2-9   epilogue: warp w drains TMEM lanes 32 (w mod 4) .. + 31 of
//               column half (w - 2) / 4 (rows 0-63 or 64-127 of the tile)
// Tiles (right-hand side r, 128-row tile of rest, 128-output chunk nc) run
// with the chunk fastest, so CTAs working at the same time share X blocks in
// L2.
constexpr int kGemmThreads = 320;
constexpr uint32_t kGemmTermBytes = (uint32_t)kTileM * 128u;  // 128 rows x 64 BF16

// One problem of the split GEMM (a mode step of one operator, all its
// right-hand sides).
struct TcGemmParams {
  CUtensorMap tm_x;      // one problem: X image [TV * xrows][kpad] BF16, box 64 x 128,
                         // 128-byte swizzle (TMA)
  const uint16_t* ximg;  // batched: X image [TV][kblocks][rows_pad][64] BF16, rows pre-swizzled
                         // (bulk copies); rows_pad = R tiles_m 128 (128-row aligned per RHS)
  const uint16_t* Bimg;  // factor image [tf][kblocks][img_rows][64] BF16, swizzled rows
  float* Y;
  int64_t rest, size_out, tiles_m, ntiles, xrows, rows_pad;  // xrows = R * rest
  int n_out, nchunks, kblocks, img_rows;
  float coeff, beta;
  const float* epi_x;  // epilogue terms as in TcParams
  const float* epi_d;
  int64_t epi_dstride;
  float epi_coeff;
  double* epi_dot;
  const float* epi_q2;
  const double* epi_gamma;
  // batched pre-split pass: the step's input and its fused first-step terms
  const float* X;
  const float* pro_z;
  const double* pro_beta;
  float* pro_out;
  int n_in, kpad, mode;  // mode as k_presplit's
  int64_t R;
  // image output (a two-factor product's first step): instead of Y the
  // epilogue writes the second step's pre-split image, whose contraction
  // index is this step's row index and whose rows are this step's outputs
  uint16_t* oimg;
  int64_t o_rstride;  // image rows per right-hand side
  int64_t o_rows;     // rows per term (TMA layout) or per (term, k block) (swizzled)
  int o_kpad, o_swz;  // the second step's padded k; 1: pre-swizzled layout
};

// Launch-wide settings of the split GEMM.
struct TcGemmLaunch {
  int stages;
  int* err;
  uint64_t stall_ns;  // > 0: time-out test (see TcParams)
  int rev = 0;        // tiles in reverse order (same results; L2 reuse between kernels)
};

// Tile sources of the split GEMM: one problem by value (X by TMA), or a
// device table of problems (X by bulk copies of pre-swizzled images).
struct GemmOne {
  static constexpr bool kTma = true;
  TcGemmParams p;
  __device__ __forceinline__ int64_t count() const { return p.ntiles; }
  __device__ __forceinline__ const TcGemmParams& get(int64_t t, int64_t& lt) const {
    lt = t;
    return p;
  }
};
struct GemmTab {
  static constexpr bool kTma = false;
  const TcGemmParams* probs;
  const int* tile_prob;      // problem of every global tile
  const int64_t* first;      // first global tile of every problem
  const int64_t* count_dev;  // number of live tiles (read at kernel start)
  __device__ __forceinline__ int64_t count() const { return *count_dev; }
  __device__ __forceinline__ const TcGemmParams& get(int64_t t, int64_t& lt) const {
    const int i = tile_prob[t];
    lt = t - first[i];
    return probs[i];
  }
};

// One 64 (k) x 64 (m) tile of the pre-split pass: X [R][n_in][rest] FP32
// (mode 0), or beta_r X + z (mode 2) or beta_r X (mode 1), both also written
// to pro_out, into TV K-major BF16 terms (zero for k >= n_in), through shared
// memory: reads along m, writes 16-byte runs of 8 k along each row.  SWZ
// false: img[t][xrows][kpad], rows r rest + m (the TMA-loaded layout); SWZ
// true: img[t][kblocks][rows_pad][64], rows r rest128 + m with rest128 =
// rest rounded up to 128 (every 128-row tile starts on an 8-row boundary, and
// a tile's rows past rest are zero padding), the 16-byte runs of row j at
// position c ^ (j mod 8) (the bulk-copied layout of a 128-byte swizzled
// K-major operand).
constexpr int kPresplitThreads = 256;  // block size of the pre-split passes

template <int TV, bool SWZ>
__device__ __forceinline__ void presplit_tile(float (*tile)[65], const float* X, int n_in,
                                              int64_t rest, int kpad, int64_t xrows,
                                              int64_t rows_pad, int mode, const float* pro_z,
                                              const double* pro_beta, float* pro_out,
                                              uint16_t* img, int64_t r, int64_t m0, int k0) {
  const int64_t off = r * (int64_t)n_in * rest;
  const float beta_r = mode != 0 ? (float)pro_beta[r] : 0.0f;
  // this thread's 16 entries: every load issued before the first store (a
  // store to pro_out, which the compiler cannot prove distinct from X and z,
  // would otherwise hold back the next load)
  constexpr int kPer = 64 * 64 / kPresplitThreads;
  const int ml = threadIdx.x & 63, kl0 = threadIdx.x >> 6;
  const int64_t m = m0 + ml;
  float v[kPer], zv[kPer];
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int k = k0 + kl0 + j * (kPresplitThreads / 64);
    const bool in = k < n_in && m < rest;
    const int64_t idx = off + (int64_t)k * rest + m;
    v[j] = in ? X[idx] : 0.0f;
    zv[j] = (in && mode == 2) ? pro_z[idx] : 0.0f;
  }
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int kl = kl0 + j * (kPresplitThreads / 64);
    const int k = k0 + kl;
    float x = v[j];
    if (mode == 2)
      x = fmaf(beta_r, x, zv[j]);
    else if (mode == 1)
      x = beta_r * x;
    if (mode != 0 && k < n_in && m < rest) pro_out[off + (int64_t)k * rest + m] = x;
    tile[kl][ml] = x;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < 64 * 8; e += kPresplitThreads) {
    const int ml = e >> 3, ch = e & 7;
    const int64_t m = m0 + ml;
    if (m >= rest) continue;
    uint32_t w[3][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      uint32_t o[3];
      split2(tile[ch * 8 + 2 * j][ml], tile[ch * 8 + 2 * j + 1][ml], TV, o);
      w[0][j] = o[0];
      w[1][j] = o[1];
      w[2][j] = o[2];
    }
    const int64_t row = SWZ ? r * ((rest + kTileM - 1) / kTileM * kTileM) + m : r * rest + m;
#pragma unroll
    for (int t = 0; t < TV; ++t) {
      size_t pos;
      if (SWZ) {
        const int kblocks = kpad / kBlockK;
        pos = (((size_t)t * kblocks + k0 / kBlockK) * rows_pad + row) * kBlockK +
              (size_t)((ch ^ (int)(row & 7)) * 8);
      } else {
        pos = ((size_t)t * xrows + row) * kpad + k0 + ch * 8;
      }
      *reinterpret_cast<uint4*>(img + pos) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
    }
  }
  __syncthreads();  // the tile is reused by the block's next tile
}

// Pre-split pass of one mode step: block (m tile, k tile, right-hand side).
template <int TV>
__global__ void __launch_bounds__(kPresplitThreads) k_presplit(const float* X, int n_in, int64_t rest,
                                                  int kpad, int64_t xrows, int mode,
                                                  const float* pro_z, const double* pro_beta,
                                                  float* pro_out, uint16_t* img) {
  __shared__ float tile[64][65];
  pdl_wait();
  presplit_tile<TV, false>(tile, X, n_in, rest, kpad, xrows, 0, mode, pro_z, pro_beta, pro_out,
                           img, blockIdx.z, (int64_t)blockIdx.x * 64, blockIdx.y * 64);
}

// Pre-split pass of a batched mode step: persistent blocks over a table of
// tiles (tile -> problem; a problem's tiles run over right-hand side, m tile,
// k tile with the k tile fastest).
template <int TV>
__global__ void __launch_bounds__(kPresplitThreads) k_presplit_tab(const TcGemmParams* probs,
                                                      const int* tile_prob, const int64_t* first,
                                                      const int64_t* count_dev) {
  __shared__ float tile[64][65];
  pdl_wait();
  const int64_t n = *count_dev;
  for (int64_t t = blockIdx.x; t < n; t += gridDim.x) {
    const int i = tile_prob[t];
    const TcGemmParams& q = probs[i];
    const int64_t lt = t - first[i];
    const int nk = q.kpad / 64;
    const int64_t nm = (q.rest + 63) / 64;
    const int kt = (int)(lt % nk);
    const int64_t mt = (lt / nk) % nm, r = lt / nk / nm;
    presplit_tile<TV, true>(tile, q.X, q.n_in, q.rest, q.kpad, q.xrows, q.rows_pad, q.mode,
                            q.pro_z, q.pro_beta, q.pro_out, const_cast<uint16_t*>(q.ximg), r,
                            mt * 64, kt * 64);
  }
}

template <int TF, int TV, class Src>
__global__ void __launch_bounds__(kGemmThreads, 1)
    k_kron_tc_gemm(const __grid_constant__ Src src, const TcGemmLaunch L) {
  constexpr int kMaxT = TF > TV ? TF : TV;
  constexpr bool kSmall = TF > 1 || TV > 1;
  constexpr uint32_t kStageBytes = (uint32_t)(TF + TV) * kGemmTermBytes;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  uint64_t* full = (uint64_t*)(base + (size_t)L.stages * kStageBytes);  // [stages]
  uint64_t* empty = full + L.stages;                                   // [stages]
  uint64_t* afull = empty + L.stages;                                  // [2]
  uint64_t* aempty = afull + 2;                                        // [2]
  uint64_t* drain = aempty + 2;
  uint64_t* stall = drain + 1;  // never completed (time-out test)
  uint32_t* tmem_slot = (uint32_t*)(stall + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < L.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&afull[b], 1);
      mbar_init(&aempty[b], kGemmThreads - 64);
    }
    mbar_init(drain, 1);
    mbar_init(stall, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  pdl_trigger();

  if (warp == 0) {
    // ---------------------------------------------------------------- loader
    pdl_wait();
    if (lane == 0) {
      bool ok = true;
      int s = 0;
      uint32_t ph = 0;
      uint32_t issued = 0, issued_ph = 0;  // bit s: a copy went to stage s / its parity
      const int64_t ntiles = src.count();
      for (int64_t t0 = blockIdx.x; t0 < ntiles && ok; t0 += gridDim.x) {
        const int64_t t = L.rev ? ntiles - 1 - t0 : t0;
        int64_t lt;
        const TcGemmParams& p = src.get(t, lt);
        const int nc = (int)(lt % p.nchunks);
        const int64_t tm = lt / p.nchunks;
        const int64_t r = tm / p.tiles_m, m0 = (tm % p.tiles_m) * kTileM;
        // the tile's fields in registers (a problem table in global memory
        // would be re-read after every asm statement of the loop below)
        const int kblocks = p.kblocks, img_rows = p.img_rows;
        const uint16_t* bimg = p.Bimg;
        const uint16_t* ximg = p.ximg;
        const int64_t rows_pad = p.rows_pad, xrows = p.xrows, xrow0 = r * p.tiles_m * kTileM + m0;
        // rows past rest arrive as the next right-hand side's rows (or zeros
        // past the image); the epilogue masks them
        const int y0 = (int)(r * p.rest + m0);
        for (int kb = 0; kb < kblocks; ++kb) {
          if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, L.err)) {
            ok = false;
            break;
          }
          unsigned char* st = base + (size_t)s * kStageBytes;
          mbar_arrive_expect_tx(&full[s], kStageBytes);
#pragma unroll
          for (int tv = 0; tv < TV; ++tv) {
            if constexpr (Src::kTma)
              tma_load_2d(st + tv * kGemmTermBytes, &p.tm_x, kb * kBlockK,
                          (int)(tv * xrows) + y0, &full[s]);
            else
              bulk_g2s(st + tv * kGemmTermBytes,
                       ximg + (((size_t)tv * kblocks + kb) * (size_t)rows_pad + (size_t)xrow0) *
                                  kBlockK,
                       kGemmTermBytes, &full[s]);
          }
#pragma unroll
          for (int ti = 0; ti < TF; ++ti)
            bulk_g2s(st + (TV + ti) * kGemmTermBytes,
                     bimg + (((size_t)ti * kblocks + kb) * (size_t)img_rows +
                               (size_t)nc * kTileM) * kBlockK,
                     kGemmTermBytes, &full[s]);
          issued |= 1u << s;
          issued_ph = (issued_ph & ~(1u << s)) | (ph << s);
          if (++s == L.stages) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
      // only the latest copy of each stage can still be in flight
      for (int st = 0; st < L.stages; ++st)
        if (issued & (1u << st)) mbar_wait_own(&full[st], (issued_ph >> st) & 1u, L.err);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------------- MMA
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(kTileM, kTileM);  // M = outputs, N = rows
      bool ok = true;
      if (L.stall_ns) ok = mbar_wait_slow(stall, 0, abort_flag, L.err, L.stall_ns);
      int s = 0;
      uint32_t ph = 0;
      int64_t it = 0;
      const int64_t ntiles = src.count();
      for (int64_t t0 = blockIdx.x; t0 < ntiles && ok; t0 += gridDim.x, ++it) {
        const int64_t t = L.rev ? ntiles - 1 - t0 : t0;
        int64_t lt;
        const int kblocks = src.get(t, lt).kblocks;
        const int b = (int)(it & 1);
        if (!mbar_wait(&aempty[b], (uint32_t)((it >> 1) & 1) ^ 1u, abort_flag, L.err)) break;
        tc_fence_after();
        const uint32_t d_big = tmem_base + (uint32_t)b * 256u, d_small = d_big + 128u;
        uint32_t acc_big = 0, acc_small = 0;
        for (int kb = 0; kb < kblocks; ++kb) {
          if (!mbar_wait(&full[s], ph, abort_flag, L.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_u32(base + (size_t)s * kStageBytes);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
            for (int ti = 0; ti < TF; ++ti)
#pragma unroll
              for (int tv = 0; tv < TV; ++tv) {
                if (ti + tv >= kMaxT) continue;
                const uint64_t ad =
                    sw128_desc(st + (uint32_t)(TV + ti) * kGemmTermBytes + (uint32_t)kk * 32u);
                const uint64_t bd =
                    sw128_desc(st + (uint32_t)tv * kGemmTermBytes + (uint32_t)kk * 32u);
                if (ti == 0 && tv == 0) {
                  mma_bf16(d_big, ad, bd, idesc, acc_big);
                  acc_big = 1;
                } else {
                  mma_bf16(d_small, ad, bd, idesc, acc_small);
                  acc_small = 1;
                }
              }
          }
          mma_commit(&empty[s]);
          if (++s == L.stages) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (!ok) break;
        mma_commit(&afull[b]);
      }
      mma_commit(drain);
      mbar_wait_own(drain, 0, L.err);
    }
    __syncwarp();
  } else {
    // -------------------------------------------------------------- epilogue
    pdl_wait();
    const int ew = warp - 2;
    const int quarter = warp & 3, chalf = ew >> 2;
    const int il = quarter * 32 + lane;  // output within the chunk = TMEM lane
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    int64_t it = 0;
    const int64_t ntiles = src.count();
    for (int64_t t0 = blockIdx.x; t0 < ntiles; t0 += gridDim.x, ++it) {
      const int64_t t = L.rev ? ntiles - 1 - t0 : t0;
      const int b = (int)(it & 1);
      if (!mbar_wait(&afull[b], (uint32_t)((it >> 1) & 1), abort_flag, L.err)) break;
      tc_fence_after();
      int64_t lt;
      const TcGemmParams& p = src.get(t, lt);
      const float d0 = (p.epi_x && p.epi_dstride == 0) ? p.epi_d[0] : 0.0f;
      const int nc = (int)(lt % p.nchunks);
      const int64_t tm = lt / p.nchunks;
      const int64_t r = tm / p.tiles_m, m0 = (tm % p.tiles_m) * kTileM;
      const uint32_t taddr = tmem_base + lane_off + (uint32_t)b * 256u + (uint32_t)chalf * 64u;
      const int i = nc * kTileM + il;
      const int64_t mbase = m0 + chalf * 64;
      const int nrows = (int)((p.rest - mbase < 64) ? (p.rest - mbase) : 64);
      const bool live = i < p.n_out && nrows > 0;
      const int64_t ld = p.n_out;
      float* yp = p.Y + r * p.size_out + mbase * ld + i;
      const float* ex = p.epi_x ? p.epi_x + r * p.size_out + mbase * ld + i : nullptr;
      const float* ed = (p.epi_x && p.epi_dstride) ? p.epi_d + mbase * ld + i : nullptr;
      const float* eq = p.epi_q2 ? p.epi_q2 + r * p.size_out + mbase * ld + i : nullptr;
      const float gam = p.epi_q2 ? (float)p.epi_gamma[r] : 0.0f;
      const float sc = p.epi_coeff * d0;
      // the tile's scalars in registers: with a problem table in global memory
      // the compiler would reload them after every store of the loops below
      const float coeff = p.coeff, beta = p.beta, ecoef = p.epi_coeff;
      double* const edot = p.epi_dot;
      uint16_t* const oimg = p.oimg;
      const int64_t o_rstride = p.o_rstride, o_rows = p.o_rows;
      const int o_kpad = p.o_kpad, o_swz = p.o_swz;
      float part = 0.0f;  // this thread's <= 64 products of x . y
      if (!ex && beta == 0.0f) {
        // plain step: the whole accumulator into registers, released, stored
        float a[64];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          uint32_t v[8], w[8];
          tmem_ld8(taddr + (uint32_t)(q * 8), v);
          if (kSmall) tmem_ld8(taddr + 128u + (uint32_t)(q * 8), w);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int e = 0; e < 8; ++e)
            a[q * 8 + e] =
                coeff * (__uint_as_float(v[e]) + (kSmall ? __uint_as_float(w[e]) : 0.0f));
        }
        tc_fence_before();
        mbar_arrive(&aempty[b]);
        if (live && oimg) {
          // row i (this step's output) of the next step's image, its 64 k
          // (this step's rows mbase ..) in TV split terms, zero past rest
          const int64_t row = r * o_rstride + i;
          const int kb = (int)(mbase / kBlockK);
#pragma unroll
          for (int ch = 0; ch < 8; ++ch) {
            uint32_t w[3][4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int c = ch * 8 + 2 * j;
              uint32_t o[3];
              split2(c < nrows ? a[c] : 0.0f, c + 1 < nrows ? a[c + 1] : 0.0f, TV, o);
              w[0][j] = o[0];
              w[1][j] = o[1];
              w[2][j] = o[2];
            }
#pragma unroll
            for (int tv = 0; tv < TV; ++tv) {
              const size_t pos =
                  o_swz ? (((size_t)tv * (o_kpad / kBlockK) + kb) * (size_t)o_rows + row) * kBlockK +
                              (size_t)((ch ^ (int)(row & 7)) * 8)
                        : ((size_t)tv * o_rows + row) * o_kpad + mbase + ch * 8;
              *reinterpret_cast<uint4*>(oimg + pos) = make_uint4(w[tv][0], w[tv][1], w[tv][2], w[tv][3]);
            }
          }
        } else if (live) {
#pragma unroll
          for (int c = 0; c < 64; ++c)
            if (c < nrows) yp[c * ld] = a[c];
        }
        continue;
      }
      if (ex && !ed && !eq && beta == 0.0f) {
        // the CG step: x for all 64 rows first (one global latency; loads
        // issued after a store to a buffer the compiler cannot prove distinct
        // would wait for it), then 16 rows at a time from the accumulator
        float xa[64];
#pragma unroll
        for (int c = 0; c < 64; ++c) xa[c] = (live && c < nrows) ? __ldg(ex + c * ld) : 0.0f;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          uint32_t v[16], w[16];
          tmem_ld8(taddr + (uint32_t)(h * 16), v);
          tmem_ld8(taddr + (uint32_t)(h * 16 + 8), v + 8);
          if (kSmall) {
            tmem_ld8(taddr + 128u + (uint32_t)(h * 16), w);
            tmem_ld8(taddr + 128u + (uint32_t)(h * 16 + 8), w + 8);
          }
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int c = h * 16 + e;
            float y = coeff * (__uint_as_float(v[e]) + (kSmall ? __uint_as_float(w[e]) : 0.0f));
            y = fmaf(sc, xa[c], y);
            if (live && c < nrows) {
              part = fmaf(y, xa[c], part);
              yp[c * ld] = y;
            }
          }
        }
      } else {
        // 16 rows at a time: accumulator columns, every load of the group, then
        // its stores (loads interleaved with the stores would wait for them)
#pragma unroll 1
        for (int h = 0; h < 4; ++h) {
          uint32_t v[16], w[16];
          tmem_ld8(taddr + (uint32_t)(h * 16), v);
          tmem_ld8(taddr + (uint32_t)(h * 16 + 8), v + 8);
          if (kSmall) {
            tmem_ld8(taddr + 128u + (uint32_t)(h * 16), w);
            tmem_ld8(taddr + 128u + (uint32_t)(h * 16 + 8), w + 8);
          }
          float xd[16], dd[16], qd[16], yo[16];
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const bool in = live && h * 16 + e < nrows;
            xd[e] = (ex && in) ? __ldg(ex + (h * 16 + e) * ld) : 0.0f;
            dd[e] = (ed && in) ? __ldg(ed + (h * 16 + e) * ld) : 0.0f;
            qd[e] = (eq && in) ? __ldg(eq + (h * 16 + e) * ld) : 0.0f;
            yo[e] = (beta != 0.0f && in) ? yp[(h * 16 + e) * ld] : 0.0f;
          }
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            float y =
                coeff * (__uint_as_float(v[e]) + (kSmall ? __uint_as_float(w[e]) : 0.0f));
            const bool in = live && h * 16 + e < nrows;
            if (ex) {
              y = fmaf(ed ? ecoef * dd[e] : sc, xd[e], y);
              if (eq) y = fmaf(-gam, qd[e], y);
              if (in) part = fmaf(y, xd[e], part);
            }
            y = fmaf(beta, yo[e], y);
            if (in) yp[(h * 16 + e) * ld] = y;
          }
        }
      }
      tc_fence_before();
      mbar_arrive(&aempty[b]);
      if (edot) {
        double dsum = (double)part;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
        if (lane == 0) edot[lt * kDotSlots + ew] = dsum;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(512)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Fused last two mode steps of a three-factor Kronecker MVM with 128 x 128
// second and third factors (the slab kernel).  The first mode step writes its
// output slab-major, T[r][i1][j2][j3] (e_mode 5), so every (right-hand side,
// i1) slab S[j2][j3] is one contiguous 128 x 128 block; this kernel applies
// K2 S K3^T to a slab with the intermediate kept on chip:
//   GEMM 1  U^T[i2, j3] = sum_j2 K2[i2, j2] S[j2, j3]   (A = K2 in tensor memory,
//           B = the split S tile in shared memory, accumulator lane i2)
//   GEMM 2  Y^T[i3, i2] = sum_j3 K3[i3, j3] U[j3, i2]   (A = K3 in tensor memory,
//           B = U re-split into BF16 terms by the epilogue, read from lane i2's
//           accumulator row into a K-major shared-memory operand)
// and writes Y[r][i1][i2][i3] = c_k Y + c_d s x (x the vector the MVM acts on,
// in the output's layout) with the per-(slab, epilogue warp) partials of x . Y
// (Lanczos' q . w after subtracting gamma q_prev; the Q2 = false variant, the
// CG step's p . Ap, is kept in the code but the CG uses the three-step path,
// which measured faster for it).
// Both factors' split images live in tensor memory (2 x 192 columns) and the
// accumulator (dominant and cross terms, 64 columns each) takes the other 128:
// each GEMM runs as two N = 64 half tiles, drained by the epilogue in turn.
//   warps 0-7   converters: read S (global, coalesced), split into BF16 terms,
//               store the GEMM 1 B operand (K-major, 128-byte swizzle)
//   warps 8-15  epilogue: factor copies into tensor memory; GEMM 1 drains into
//               the GEMM 2 B operand; GEMM 2 drains to Y
//   warp 16     MMA issue, tensor-memory allocation
constexpr int kSlabN = 128;                       // n2 = n3
constexpr int kSlabThreads = 32 * (kFsEpiWarps + kFsConvWarps + 1);  // 544

struct TcSlabParams {
  const float* S;        // [nslab][128][128] slab-major first-step output
  const uint16_t* img2;  // split K2 image [tf][2][img_rows2][64]
  const uint16_t* img3;  // split K3 image [tf][2][img_rows3][64]
  int img_rows2, img_rows3;
  float* Y;              // [nslab][128][128] output, natural layout
  const float* x;        // vector the MVM acts on (shift term and dot), Y's layout;
                         // nullptr: Y = c_k K S only (no shift term, no partials)
  const float* q2;       // optional: Y -= gamma[r] q2 (Lanczos), Y's layout
  const double* gamma;
  const double* scale;   // optional per right-hand side: Y = scale[r] (c_k K x + c_d d[0] x)
                         // - gamma q2, partials of scale[r] x . Y (x unnormalised)
  const float* d;        // shift scalar (device), term c_d d[0] x
  float coeff, dcoeff;
  int64_t nslab, slabs_per_rhs;
  double* dot;           // [nslab][8] partials of x . Y
  int* err;
  uint64_t stall_ns;
  int rev;  // slabs in reverse order (same results; L2 reuse between kernels)
};

// Splits 16 FP32 values into TV BF16 terms and stores them as 16 consecutive
// k positions (two 16-byte chunks, starting at chunk c0) of K-major row `row`
// of a 128-row B operand with 128-byte swizzle.
template <int TV>
__device__ __forceinline__ void slab_put16(unsigned char* bst, int row, int c0, const float* v) {
  uint32_t w[TV][8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    uint32_t o[3];
    split2(v[2 * e], v[2 * e + 1], TV, o);
#pragma unroll
    for (int tv = 0; tv < TV; ++tv) w[tv][e] = o[tv];
  }
  unsigned char* rowp = bst + (size_t)row * 128;
  const uint32_t swz = (uint32_t)(row & 7);
#pragma unroll
  for (int tv = 0; tv < TV; ++tv)
#pragma unroll
    for (int h = 0; h < 2; ++h)
      *reinterpret_cast<uint4*>(rowp + (size_t)tv * kFsBTermBytes +
                                (((uint32_t)(c0 + h) ^ swz) << 4)) =
          make_uint4(w[tv][4 * h], w[tv][4 * h + 1], w[tv][4 * h + 2], w[tv][4 * h + 3]);
}

// Slab kernel, full-width form.  Both GEMMs of a slab run as N = 128 tiles
// (48 MMAs each at 3 x 3 split terms) into one dominant / cross accumulator
// pair (256 tensor-memory columns):
//   GEMM 1  U^T = K2 S     A = K2's split image in tensor memory (192 columns)
//   GEMM 2  Y^T = K3 U^T   A = K3's split image in shared memory (one bulk
//                          copy per term and k block at the start)
// One B operand buffer holds the slab's split (GEMM 1) and then the re-split
// intermediate U (GEMM 2), tracked per 64-wide k block: GEMM 2 starts on a k
// block of U as soon as the epilogue warps of that column half have written
// it, and the converters write a k block of the next slab's split as soon as
// GEMM 2 has finished reading it.  The two accumulator uses are drained by
// different warps, so that the re-split feeding GEMM 2 never waits behind the
// global loads and stores of the output:
//   warps 0-7   converters: thread (row j3, k half) loads its 64 values of the
//               next slab's S (j2 = its k half of both k blocks) and splits
//               them into B; then drains GEMM 2 of the previous slab (lane i3,
//               columns i2 of its half) into Y with the shift term, the
//               Lanczos term and the partials of x . Y
//   warp 16     MMA (one lane), tensor-memory allocation, K3 image copies
//   warps 8-15  epilogue: K2 image into tensor memory; per slab drains GEMM 1
//               (lane i2, columns j3 of its half) into the U split
constexpr uint32_t kSlabAccCol = 256;  // dominant accumulator; cross term at +128

// Issues the loads of 16 columns of the dominant and of the cross accumulator
// (no wait).
template <bool kSmall>
__device__ __forceinline__ void slab_ld16(uint32_t taddr, uint32_t* v, uint32_t* w) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  if (kSmall)
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]),
          "=r"(w[7]), "=r"(w[8]), "=r"(w[9]), "=r"(w[10]), "=r"(w[11]), "=r"(w[12]),
          "=r"(w[13]), "=r"(w[14]), "=r"(w[15])
        : "r"(taddr + 128u));
}

// Waits for the tensor-memory loads in flight; v (and w) are tied to the wait
// so that no use of them moves above it.
template <bool kSmall>
__device__ __forceinline__ void slab_ld_wait(uint32_t* v, uint32_t* w) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]),
                 "+r"(v[6]), "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]),
                 "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15])
               :
               : "memory");
  if (kSmall)
    asm volatile(""
                 : "+r"(w[0]), "+r"(w[1]), "+r"(w[2]), "+r"(w[3]), "+r"(w[4]), "+r"(w[5]),
                   "+r"(w[6]), "+r"(w[7]), "+r"(w[8]), "+r"(w[9]), "+r"(w[10]), "+r"(w[11]),
                   "+r"(w[12]), "+r"(w[13]), "+r"(w[14]), "+r"(w[15])
                 :
                 : "memory");
}

// Loads 16 columns of the dominant and of the cross accumulator (one wait)
// and returns their sums.
template <bool kSmall>
__device__ __forceinline__ void slab_drain16(uint32_t taddr, float* a) {
  uint32_t v[16], w[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  if (kSmall)
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(w[0]), "=r"(w[1]), "=r"(w[2]), "=r"(w[3]), "=r"(w[4]), "=r"(w[5]), "=r"(w[6]),
          "=r"(w[7]), "=r"(w[8]), "=r"(w[9]), "=r"(w[10]), "=r"(w[11]), "=r"(w[12]),
          "=r"(w[13]), "=r"(w[14]), "=r"(w[15])
        : "r"(taddr + 128u));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int e = 0; e < 16; ++e)
    a[e] = __uint_as_float(v[e]) + (kSmall ? __uint_as_float(w[e]) : 0.0f);
}

// EM: 0 Y = c_k K S; 1 adds the shift term c_d d[0] x and writes the partials
// of x . Y; 2 as 1 with the Lanczos term (- gamma q2) and the scale.
template <int TF, int TV, int EM>
__global__ void __launch_bounds__(kSlabThreads, 1)
    k_kron_tc_slab(const __grid_constant__ TcSlabParams p) {
  constexpr bool Q2 = EM == 2, HX = EM >= 1;
  constexpr int kMaxT = TF > TV ? TF : TV;
  constexpr bool kSmall = TF > 1 || TV > 1;
  constexpr uint32_t kKbBytes = (uint32_t)TV * kFsBTermBytes;  // one 64-wide k block, TV terms
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char* bbuf = base;                  // B operand: 2 k blocks x TV terms
  unsigned char* a3 = base + 2 * kKbBytes;     // K3 image: TF terms x 2 k blocks
  uint64_t* bars = (uint64_t*)(a3 + (size_t)TF * 2 * kFsBTermBytes);
  uint64_t* bfull = bars;           // [2] S k block split (converters)
  uint64_t* bfree = bfull + 2;      // [2] GEMM 2 done reading a k block (MMA commit)
  uint64_t* ufull = bfree + 2;      // [2] U k block split (epilogue column half)
  uint64_t* a1full = ufull + 2;     // GEMM 1 accumulated (MMA commit)
  uint64_t* a1empty = a1full + 1;   // GEMM 1 drained (epilogue)
  uint64_t* a2full = a1empty + 1;   // GEMM 2 accumulated (MMA commit)
  uint64_t* a2empty = a2full + 1;   // GEMM 2 drained (converters)
  uint64_t* afac = a2empty + 1;     // K2 image in tensor memory (epilogue)
  uint64_t* a3full = afac + 1;      // K3 image in shared memory (bulk copies)
  uint64_t* drain = a3full + 1;
  uint64_t* stall = drain + 1;
  uint32_t* tmem_slot = (uint32_t*)(stall + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&bfull[s], kFsConvThreads);
      mbar_init(&bfree[s], 1);
      mbar_init(&ufull[s], kFsEpiThreads / 2);
    }
    mbar_init(a1full, 1);
    mbar_init(a1empty, kFsEpiThreads);
    mbar_init(a2full, 1);
    mbar_init(a2empty, kFsConvThreads);
    mbar_init(afac, kFsEpiThreads);
    mbar_init(a3full, 1);
    mbar_init(drain, 1);
    mbar_init(stall, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kFsMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  pdl_trigger();

  if (warp < kFsConvWarps) {
    // ---------------------------------------- converters and GEMM 2 drains
    pdl_wait();
    const int row = (warp & 3) * 32 + lane;  // j3: row of the B operand; i3: TMEM lane
    const int khalf = warp >> 2;             // 32 of the 64 k (= j2) of a block; i2 half
    const uint32_t taddr =
        tmem_base + ((uint32_t)((warp & 3) * 32) << 16) + kSlabAccCol + (uint32_t)khalf * 64u;
    const float sc = HX ? p.dcoeff * p.d[0] : 0.0f;
    float v[2][32];
    auto load_s = [&](int64_t sl) {
      const float* src = p.S + sl * (int64_t)(kSlabN * kSlabN) + row;
#pragma unroll
      for (int kb = 0; kb < 2; ++kb)
#pragma unroll
        for (int e = 0; e < 32; ++e)
          v[kb][e] = __ldg(src + (int64_t)(kb * 64 + khalf * 32 + e) * kSlabN);
    };
    // GEMM 2 of slab sl (its it-th): Y[i2][i3], i3 = row, i2 = 64 khalf + c
    auto drain_y = [&](int64_t sl, int64_t it) -> bool {
      if (!mbar_wait(a2full, (uint32_t)(it & 1), abort_flag, p.err)) return false;
      tc_fence_after();
      float a[64];
#pragma unroll
      for (int q = 0; q < 4; ++q) slab_drain16<kSmall>(taddr + (uint32_t)q * 16u, a + 16 * q);
      tc_fence_before();
      mbar_arrive(a2empty);
      const int64_t r = sl / p.slabs_per_rhs;
      const float gam = Q2 ? (float)p.gamma[r] : 0.0f;
      const float srr = (HX && p.scale) ? (float)p.scale[r] : 1.0f;
      const int64_t i0 = sl * (int64_t)(kSlabN * kSlabN) + (int64_t)(khalf * 64) * kSlabN + row;
      constexpr int kBlk = 16;
      float part = 0.0f;
#pragma unroll
      for (int blk = 0; blk < 64 / kBlk; ++blk) {
        float xv[kBlk], qv[Q2 ? kBlk : 1];
#pragma unroll
        for (int c = 0; c < kBlk; ++c) {
          const int64_t o = i0 + (int64_t)(blk * kBlk + c) * kSlabN;
          xv[c] = HX ? __ldg(p.x + o) : 0.0f;
          if (Q2) qv[c] = gam != 0.0f ? __ldg(p.q2 + o) : 0.0f;
        }
#pragma unroll
        for (int c = 0; c < kBlk; ++c) {
          const int cc = blk * kBlk + c;
          float y = HX ? srr * fmaf(sc, xv[c], p.coeff * a[cc]) : p.coeff * a[cc];
          if (Q2) y = fmaf(-gam, qv[c], y);
          if (HX) part = fmaf(y, xv[c], part);
          p.Y[i0 + (int64_t)cc * kSlabN] = y;
        }
      }
      if (HX && p.dot) {
        double dsum = (double)part;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
        if (lane == 0) p.dot[sl * kDotSlots + warp] = dsum * (double)srr;
      }
      return true;
    };
    // Iteration `it` loads slab sl's values (issued right after the previous
    // iteration's output stores, they land while the GEMMs of the previous
    // slab run), writes its split into each k block of B once GEMM 2 of the
    // previous slab has finished reading it, then stores the previous slab's
    // output.
    int64_t it = 0;
    bool ok = true;
    auto slab_at = [&](int64_t k) { return p.rev ? p.nslab - 1 - k : k; };
    for (int64_t sl = blockIdx.x; sl < p.nslab; sl += gridDim.x, ++it) {
      load_s(slab_at(sl));
#pragma unroll
      for (int kb = 0; kb < 2; ++kb) {
        if (!mbar_wait(&bfree[kb], (uint32_t)(it & 1) ^ 1u, abort_flag, p.err)) {
          ok = false;
          break;
        }
        unsigned char* bst = bbuf + (size_t)kb * kKbBytes;
        slab_put16<TV>(bst, row, khalf * 4, v[kb]);
        slab_put16<TV>(bst, row, khalf * 4 + 2, v[kb] + 16);
        fence_proxy_async();
        mbar_arrive(&bfull[kb]);
      }
      if (!ok) break;
      if (it > 0 && !drain_y(slab_at(sl - gridDim.x), it - 1)) {
        ok = false;
        break;
      }
    }
    if (ok && it > 0) drain_y(slab_at(blockIdx.x + (it - 1) * (int64_t)gridDim.x), it - 1);
  } else if (warp == kFsMmaWarp) {
    // ------------------------------------------------------------------- MMA
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(kTileM, kSlabN);  // M = outputs, N = 128 rows
      // K3's split image: TF terms x 2 k blocks of 128 swizzled rows
      mbar_arrive_expect_tx(a3full, (uint32_t)(TF * 2) * kFsBTermBytes);
#pragma unroll
      for (int b = 0; b < TF * 2; ++b)
        bulk_g2s(a3 + (size_t)b * kFsBTermBytes, p.img3 + (size_t)b * p.img_rows3 * kBlockK,
                 kFsBTermBytes, a3full);
      bool ok = mbar_wait_own(a3full, 0, p.err) && mbar_wait(afac, 0, abort_flag, p.err);
      if (ok && p.stall_ns) ok = mbar_wait_slow(stall, 0, abort_flag, p.err, p.stall_ns);
      tc_fence_after();
      // operand descriptors: base descriptor plus (offset >> 4), the 14-bit
      // address field holding any shared-memory address below 256 KB
      const uint64_t bdesc0 = sw128_desc(smem_u32(bbuf)), adesc0 = sw128_desc(smem_u32(a3));
      const uint32_t d_dom = tmem_base + kSlabAccCol, d_small = d_dom + 128u;
      int64_t it = 0;
      for (int64_t sl = blockIdx.x; sl < p.nslab && ok; sl += gridDim.x, ++it) {
        const uint32_t ph = (uint32_t)(it & 1);
        // GEMM 1: A = K2 (tensor memory), B = S split; the accumulator is free
        // once the converters drained GEMM 2 of the previous slab
        if (!mbar_wait(a2empty, ph ^ 1u, abort_flag, p.err)) break;
        uint32_t acc_small = 0;
        for (int kb = 0; kb < 2 && ok; ++kb) {
          if (!mbar_wait(&bfull[kb], ph, abort_flag, p.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
#pragma unroll
            for (int ti = 0; ti < TF; ++ti)
#pragma unroll
              for (int tv = 0; tv < TV; ++tv) {
                if (ti + tv >= kMaxT) continue;
                const uint32_t a = tmem_base + (uint32_t)(ti * 64 + kb * 32 + kk * 8);
                const uint64_t bd =
                    bdesc0 + (((uint32_t)kb * kKbBytes + (uint32_t)tv * kFsBTermBytes +
                               (uint32_t)kk * 32u) >> 4);
                if (ti == 0 && tv == 0) {
                  mma_bf16_ta(d_dom, a, bd, idesc, (kb | kk) ? 1u : 0u);
                } else {
                  mma_bf16_ta(d_small, a, bd, idesc, acc_small);
                  acc_small = 1;
                }
              }
        }
        if (!ok) break;
        mma_commit(a1full);
        // GEMM 2: A = K3 (shared memory), B = U split, one k block at a time
        if (!mbar_wait(a1empty, ph, abort_flag, p.err)) break;
        acc_small = 0;
        for (int kb = 0; kb < 2 && ok; ++kb) {
          if (!mbar_wait(&ufull[kb], ph, abort_flag, p.err)) {
            ok = false;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
#pragma unroll
            for (int ti = 0; ti < TF; ++ti)
#pragma unroll
              for (int tv = 0; tv < TV; ++tv) {
                if (ti + tv >= kMaxT) continue;
                const uint64_t ad =
                    adesc0 + (((uint32_t)(ti * 2 + kb) * kFsBTermBytes + (uint32_t)kk * 32u) >> 4);
                const uint64_t bd =
                    bdesc0 + (((uint32_t)kb * kKbBytes + (uint32_t)tv * kFsBTermBytes +
                               (uint32_t)kk * 32u) >> 4);
                if (ti == 0 && tv == 0) {
                  mma_bf16(d_dom, ad, bd, idesc, (kb | kk) ? 1u : 0u);
                } else {
                  mma_bf16(d_small, ad, bd, idesc, acc_small);
                  acc_small = 1;
                }
              }
          mma_commit(&bfree[kb]);
        }
        if (!ok) break;
        mma_commit(a2full);
      }
      mma_commit(drain);
      mbar_wait_own(drain, 0, p.err);
    }
    __syncwarp();
  } else {
    // -------------------------------------------------------------- epilogue
    const int ew = warp - kFsConvWarps;  // 0..7
    const int quarter_l = warp & 3, chalf = ew >> 2;
    const int i = quarter_l * 32 + lane;  // TMEM lane: i2
    const uint32_t lane_off = (uint32_t)(quarter_l * 32) << 16;
    // K2's split image into tensor memory: k block `chalf` of every term, row i
#pragma unroll
    for (int ti = 0; ti < TF; ++ti) {
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        uint32_t u[16];
        const uint4* src = reinterpret_cast<const uint4*>(
            p.img2 + ((size_t)(ti * 2 + chalf) * p.img_rows2 + i) * kBlockK);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const uint4 qv = __ldg(src + ((hh * 4 + c) ^ (i & 7)));
          u[4 * c] = qv.x;
          u[4 * c + 1] = qv.y;
          u[4 * c + 2] = qv.z;
          u[4 * c + 3] = qv.w;
        }
        tmem_st16(tmem_base + lane_off + (uint32_t)(ti * 64 + chalf * 32 + hh * 16), u);
      }
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    tc_fence_before();
    mbar_arrive(afac);
    const uint32_t taddr = tmem_base + lane_off + kSlabAccCol + (uint32_t)chalf * 64u;
    int64_t it = 0;
    for (int64_t sl = blockIdx.x; sl < p.nslab; sl += gridDim.x, ++it) {
      // GEMM 1 -> U split: row i2 = i of the B operand, k = j3 = 64 chalf + c
      if (!mbar_wait(a1full, (uint32_t)(it & 1), abort_flag, p.err)) break;
      tc_fence_after();
      // the loads of the next 16 columns are in flight while this thread
      // splits and stores the current ones
      uint32_t v[2][16], w[2][16];
      slab_ld16<kSmall>(taddr, v[0], w[0]);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        slab_ld_wait<kSmall>(v[q & 1], w[q & 1]);
        if (q < 3) slab_ld16<kSmall>(taddr + (uint32_t)(q + 1) * 16u, v[(q + 1) & 1], w[(q + 1) & 1]);
        float a[16];
#pragma unroll
        for (int e = 0; e < 16; ++e)
          a[e] = __uint_as_float(v[q & 1][e]) + (kSmall ? __uint_as_float(w[q & 1][e]) : 0.0f);
        slab_put16<TV>(bbuf + (size_t)chalf * kKbBytes, i, 2 * q, a);
      }
      tc_fence_before();
      mbar_arrive(a1empty);
      fence_proxy_async();
      mbar_arrive(&ufull[chalf]);
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kFsMmaWarp) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(512)
                 : "memory");
  }
}

// Pre-split factor image: Fop (n_out x n_in, row-major, Fop = F or F^T) into
// [tf][kblocks][n_pad][64] BF16 terms with 128-byte swizzled rows.
template <typename TF>
__global__ void k_split_factor(const TF* F, int64_t ld, int tr, int n_out, int n_in, int n_pad,
                               int kblocks, int tf, uint16_t* img) {
  const int64_t per_term = (int64_t)kblocks * n_pad * kBlockK;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < per_term;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int kb = (int)(e / ((int64_t)n_pad * kBlockK));
    const int rem = (int)(e % ((int64_t)n_pad * kBlockK));
    const int i = rem / kBlockK, kk = rem % kBlockK;
    const int j = kb * kBlockK + kk;
    double v = 0.0;
    if (i < n_out && j < n_in) v = (double)(tr ? F[(int64_t)j * ld + i] : F[(int64_t)i * ld + j]);
    const size_t pos = (size_t)kb * n_pad * kBlockK + (size_t)i * kBlockK +
                       (size_t)((((kk >> 3) ^ (i & 7)) << 3) | (kk & 7));
    for (int t = 0; t < tf; ++t) {
      const __nv_bfloat16 h = __double2bfloat16(v);
      img[(size_t)t * per_term + pos] = *reinterpret_cast<const uint16_t*>(&h);
      v -= (double)__bfloat162float(h);
    }
  }
}

constexpr int kChunkMax = 128;
// output-chunk widths (N tile) the batched launch can be tuned over
constexpr int kChunkCaps[2] = {64, 128};

struct TcPlan {
  int n_in, n_out, n_pad, kblocks, ksteps_last, tf, tv, stages, nbuf, n_chunk, nchunks;
  int img_rows;
  uint32_t stage_bytes, a_term_bytes, b_term_bytes, tmem_cols;
  size_t smem;
};

// Output columns padded to 16 and split into equal chunks of at most `cap`.
static int chunk_layout(int n_out, int cap, int* nchunks) {
  const int n16 = (n_out + 15) / 16 * 16;
  *nchunks = (n16 + cap - 1) / cap;
  return ((n16 + *nchunks - 1) / *nchunks + 15) / 16 * 16;
}

TcPlan make_plan(int n_in, int n_out, int tf, int tv, int chunk_cap = kChunkMax) {
  TcPlan q{};
  q.n_in = n_in;
  q.n_out = n_out;
  // output columns in chunks of at most chunk_cap (128 keeps two pipeline
  // stages of A and B terms in shared memory); a plan covers a whole number
  // of equal chunks
  q.n_chunk = chunk_layout(n_out, chunk_cap, &q.nchunks);
  q.n_pad = q.nchunks * q.n_chunk;
  // the split factor image holds enough (zero) rows for every chunk width
  q.img_rows = q.n_pad;
  for (int cap : kChunkCaps) {
    int nc = 0;
    const int w = chunk_layout(n_out, cap, &nc);
    q.img_rows = std::max(q.img_rows, nc * w);
  }
  const int kpad = (n_in + 15) / 16 * 16;
  q.kblocks = (kpad + kBlockK - 1) / kBlockK;
  q.ksteps_last = (kpad - (q.kblocks - 1) * kBlockK) / 16;
  q.tf = tf;
  q.tv = tv;
  q.a_term_bytes = kTileM * 128;
  q.b_term_bytes = (uint32_t)q.n_chunk * 128;
  q.stage_bytes = (uint32_t)(tv * q.a_term_bytes + tf * q.b_term_bytes);
  q.stage_bytes = (q.stage_bytes + 1023) / 1024 * 1024;
  const size_t budget = 200 * 1024;
  q.stages = (int)std::min<size_t>(4, budget / q.stage_bytes);
  q.smem = (size_t)q.stages * q.stage_bytes + 1024 + 256;
  // two accumulators (dominant and cross terms) per buffer; double-buffer when it fits
  q.nbuf = (4 * q.n_chunk <= 512) ? 2 : 1;
  uint32_t cols = 32;
  while (cols < (uint32_t)(2 * q.nbuf * q.n_chunk)) cols <<= 1;
  q.tmem_cols = cols;
  return q;
}

}  // namespace

// Largest factor side the tensor-core path takes (N in chunks of <= 256,
// K streamed in 64-wide blocks).
constexpr int kTcMaxN = 8192;

static bool tc_supported(const cola_linop* op) {
  for (auto* f : op->kids)
    if (f->rows > kTcMaxN || f->cols > kTcMaxN) return false;
  return true;
}

static std::string depth_name(const char* what, int depth, int slot) {
  char b[64];
  snprintf(b, sizeof b, "%s.d%d.%d", what, depth, slot);
  return b;
}

static int* tc_errflag(Ctx* c) {
  const bool fresh = c->ws.bufs.find("tc.err") == c->ws.bufs.end();
  int* p = (int*)c->ws.get("tc.err", 256);
  if (fresh) COLA_CUDA(cudaMemsetAsync(p, 0, 256, c->s));
  return p;
}

void tc_check_error(Ctx* c) {
  if (c->ws.bufs.find("tc.err") == c->ws.bufs.end()) return;
  int* p = (int*)c->ws.bufs["tc.err"].p;
  int h = 0;
  COLA_CUDA(cudaMemcpyAsync(&h, p, 4, cudaMemcpyDeviceToHost, c->s));
  COLA_CUDA(cudaStreamSynchronize(c->s));
  c->tc_err_pending = false;  // the device flag read here covers any queued copy
  if (h != 0) {
    COLA_CUDA(cudaMemsetAsync(p, 0, 4, c->s));
    fail(COLA_ERR_TIMEOUT, "tensor-core Kronecker kernel timed out waiting on an mbarrier");
  }
}

// The device flag is only cleared when a timeout is reported, so a copy taken
// at any later point still shows it.  One copy is in flight at a time.
void tc_check_error_async(Ctx* c) {
  if (c->ws.bufs.find("tc.err") == c->ws.bufs.end()) return;
  int* p = (int*)c->ws.bufs["tc.err"].p;
  if (!c->tc_err_host) {
    COLA_CUDA(cudaHostAlloc((void**)&c->tc_err_host, sizeof(int), cudaHostAllocDefault));
    *c->tc_err_host = 0;
    COLA_CUDA(cudaEventCreateWithFlags(&c->tc_err_ev, cudaEventDisableTiming));
  }
  if (c->tc_err_pending && cudaEventQuery(c->tc_err_ev) == cudaSuccess) {
    c->tc_err_pending = false;
    if (*c->tc_err_host != 0) {
      *c->tc_err_host = 0;
      COLA_CUDA(cudaMemsetAsync(p, 0, 4, c->s));
      fail(COLA_ERR_TIMEOUT,
           "tensor-core Kronecker kernel of an earlier call timed out waiting on an mbarrier");
    }
  }
  if (!c->tc_err_pending) {
    COLA_CUDA(cudaMemcpyAsync(c->tc_err_host, p, sizeof(int), cudaMemcpyDeviceToHost, c->s));
    COLA_CUDA(cudaEventRecord(c->tc_err_ev, c->s));
    c->tc_err_pending = true;
  }
}

void kron_tc_prepare(Ctx* c, cola_linop* op, int split_terms) {
  if (!tc_supported(op)) return;
  const int tf = std::max(1, std::min(3, split_terms));
  for (auto* f : op->kids) {
    for (int tr = 0; tr < 2; ++tr) {
      const int n_out = (int)(tr ? f->cols : f->rows), n_in = (int)(tr ? f->rows : f->cols);
      const TcPlan q = make_plan(n_in, n_out, tf, 2);
      const size_t per_term = (size_t)q.kblocks * q.img_rows * kBlockK;
      const int key = 100 + tr * 10 + tf;
      if (prep_fresh(f, key)) continue;
      auto it = f->derived.find(key);
      void* img;
      if (it == f->derived.end() || it->second.bytes < per_term * tf * 2) {
        if (it != f->derived.end()) {
          cudaFree(it->second.p);
          f->derived.erase(it);
        }
        COLA_CUDA(cudaMalloc(&img, per_term * tf * 2));
        f->derived[key] = Buf{img, per_term * tf * 2};
      } else {
        img = it->second.p;
      }
      const int grid = (int)std::min<size_t>(1024, (per_term + 255) / 256);
      if (f->dtype == COLA_F64)
        k_split_factor<double><<<grid, 256, 0, c->s>>>((const double*)f->data, f->ld, tr, n_out,
                                                        n_in, q.img_rows, q.kblocks, tf,
                                                        (uint16_t*)img);
      else
        k_split_factor<float><<<grid, 256, 0, c->s>>>((const float*)f->data, f->ld, tr, n_out,
                                                      n_in, q.img_rows, q.kblocks, tf,
                                                      (uint16_t*)img);
      c->count_launch();
      COLA_CUDA(cudaGetLastError());
      prep_mark(const_cast<cola_linop*>(f), key);
    }
  }
  op->derived[200] = Buf{nullptr, (size_t)tf};  // remembers the factor split terms
}

template <typename T>
void kron_tc_apply(Ctx* c, const cola_linop* op, const T* X, T* Y, int64_t R, double coeff,
                   double beta, int depth, bool tr);

template <>
void kron_tc_apply<double>(Ctx*, const cola_linop*, const double*, double*, int64_t, double,
                           double, int, bool) {
  fail(COLA_ERR_UNSUPPORTED, "tensor-core Kronecker contraction takes FP32 vectors");
}

constexpr size_t kSmemMax = 232448;  // 227 KB opt-in dynamic shared memory per CTA

// cuTensorMapEncodeTiled from the driver through the runtime (no libcuda link).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
  });
  return fn;
}

// FP32 matrix [rows][cols] (row stride cols), box 64 rows x 128 columns; reads
// outside the matrix return zeros.
static bool tmap_rows(CUtensorMap* m, const float* base, int64_t rows, int64_t cols) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 4};
  const cuuint32_t box[2] = {(cuuint32_t)kTileM, (cuuint32_t)kBlockK};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static size_t fs_smem(const TcFsParams& r, int tv) {
  return 1024 + 2 * (size_t)tv * kFsBTermBytes + (size_t)r.xstages * r.nsrc * r.x_src_bytes +
         r.e_bytes + 256;
}

// Factor-stationary plan: factor sides <= 128 (two 64-wide k blocks, one
// output chunk) and X rows 16-byte aligned for cp.async.bulk.
static bool fs_plan(const TcParams& p, TcFsParams& r) {
  if (p.nchunks != 1 || p.n_pad > kTileM || p.kblocks > 2) return false;
  if (p.rest % 4 != 0 || p.size_in % 4 != 0) return false;
  r.e_mode = p.epi_x ? (p.epi_dstride != 0 ? 3 : 1) : (p.beta != 0.0f ? 2 : 0);
  if (p.epi_q2) {
    if (r.e_mode != 1) return false;  // the Lanczos term takes the scalar-shift epilogue
    r.e_mode = 4;
  }
  if (p.out_trans) {
    if (r.e_mode != 0 || p.rest % 4 != 0) return false;
    r.e_mode = 5;
  }
  // a fused shift with a nonzero beta takes the streaming kernel
  if (p.epi_x && p.beta != 0.0f) return false;
  r.e_src = (r.e_mode == 1 || r.e_mode == 3 || r.e_mode == 4) ? p.epi_x
                                                             : (r.e_mode == 2 ? p.Y : nullptr);
  if (r.e_src && (((uintptr_t)r.e_src & 15u) != 0 || p.size_out % 4 != 0)) return false;
  const int64_t xrows = p.batch * p.n_in;
  if (!tmap_rows(&r.tm_x, p.X, xrows, p.rest)) return false;
  if (p.pro_z && !tmap_rows(&r.tm_z, p.pro_z, xrows, p.rest)) return false;
  r.Bimg = p.Bimg;
  r.Y = p.Y;
  r.rest = p.rest;
  r.size_in = p.size_in;
  r.size_out = p.size_out;
  r.tiles_m = p.tiles_m;
  r.ntiles = p.ntiles;
  r.n_in = p.n_in;
  r.n_out = p.n_out;
  r.n_pad = p.n_pad;
  r.img_rows = p.img_rows;
  r.kblocks = p.kblocks;
  r.ksteps_last = p.ksteps_last;
  r.nsrc = p.pro_z ? 2 : 1;
  r.rev = p.rev;
  r.x_src_bytes = (uint32_t)kBlockK * kTileM * 4u;
  r.e_bytes = (r.e_mode && r.e_mode != 5)
                  ? (((uint32_t)kTileM * (uint32_t)p.n_out * 4u + 1023u) & ~1023u)
                  : 0u;
  const size_t avail = kSmemMax - 1024 - 256 - 2 * (size_t)p.tv * kFsBTermBytes - r.e_bytes;
  r.xstages = (int)std::min<size_t>(4, avail / ((size_t)r.nsrc * r.x_src_bytes));
  if (r.xstages < 2) return false;
  r.coeff = p.coeff;
  r.beta = p.beta;
  r.e_coeff = p.epi_coeff;
  r.e_d = p.epi_d;
  r.err = p.err;
  r.stall_ns = p.stall_ns;
  r.pro_beta = p.pro_beta;
  r.pro_out = p.pro_out;
  r.epi_dot = p.epi_dot;
  r.pro_scale = (p.pro_out && !p.pro_z) ? 1 : 0;
  r.e_q2 = p.epi_q2;
  r.e_gamma = p.epi_gamma;
  r.pro_nrm = p.pro_nrm;
  return true;
}

// BF16 image [rows][cols] of the GEMM path's X image, box 64 columns x 128
// rows, 128-byte swizzle (the UMMA K-major layout); reads past the rows
// return zeros.
static bool tmap_image(CUtensorMap* m, const uint16_t* base, int64_t rows, int64_t cols) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBlockK, (cuuint32_t)kTileM};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t*>(base), dims, strides,
             box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <class Src>
using GemmKernel = void (*)(Src, TcGemmLaunch);
template <class Src>
static GemmKernel<Src> gemm_kernel(int tf, int tv) {
  static const GemmKernel<Src> tab[3][3] = {
      {k_kron_tc_gemm<1, 1, Src>, k_kron_tc_gemm<1, 2, Src>, k_kron_tc_gemm<1, 3, Src>},
      {k_kron_tc_gemm<2, 1, Src>, k_kron_tc_gemm<2, 2, Src>, k_kron_tc_gemm<2, 3, Src>},
      {k_kron_tc_gemm<3, 1, Src>, k_kron_tc_gemm<3, 2, Src>, k_kron_tc_gemm<3, 3, Src>}};
  return tab[tf - 1][tv - 1];
}
using PresplitKernel = void (*)(const float*, int, int64_t, int, int64_t, int, const float*,
                                const double*, float*, uint16_t*);
static PresplitKernel presplit_kernel(int tv) {
  static const PresplitKernel tab[3] = {k_presplit<1>, k_presplit<2>, k_presplit<3>};
  return tab[tv - 1];
}
constexpr int kGemmStages = 2;
static size_t gemm_smem(int tf, int tv) {
  return 1024 + (size_t)kGemmStages * (tf + tv) * kGemmTermBytes + 256;
}

// The split GEMM mode step (factor sides above 128): pre-split pass, then the
// GEMM.  The factor's GEMM image (128-row output chunks) is made on first use
// outside graph capture; false (the caller takes the streaming kernel) while
// it does not exist yet, or when the step has a form the GEMM does not take.
// The split GEMM's image of a factor: [tf][kblocks][nch * 128][64] BF16 with
// swizzled rows (128-row output chunks, zero past the factor), made on first
// use; nullptr while it does not exist and the stream is being captured.
static const uint16_t* gemm_factor_image(Ctx* c, const cola_linop* f, bool tr, int tf) {
  const int n_out = (int)(tr ? f->cols : f->rows), n_in = (int)(tr ? f->rows : f->cols);
  const int kblocks = (n_in + kBlockK - 1) / kBlockK;
  const int img_rows = (n_out + kTileM - 1) / kTileM * kTileM;
  cola_linop* fm = const_cast<cola_linop*>(f);
  const int key = 120 + (tr ? 10 : 0) + tf;
  if (!prep_fresh(f, key)) {
    if (c->capturing) return nullptr;
    const size_t per_term = (size_t)kblocks * img_rows * kBlockK;
    auto it = fm->derived.find(key);
    if (it != fm->derived.end() && it->second.bytes < per_term * tf * 2) {
      cudaFree(it->second.p);
      fm->derived.erase(it);
      it = fm->derived.end();
    }
    void* img = nullptr;
    if (it == fm->derived.end()) {
      COLA_CUDA(cudaMalloc(&img, per_term * tf * 2));
      fm->derived[key] = Buf{img, per_term * (size_t)tf * 2};
    } else {
      img = it->second.p;
    }
    const int grid = (int)std::min<size_t>(1024, (per_term + 255) / 256);
    if (f->dtype == COLA_F64)
      k_split_factor<double><<<grid, 256, 0, c->s>>>((const double*)f->data, f->ld, tr ? 1 : 0,
                                                      n_out, n_in, img_rows, kblocks, tf,
                                                      (uint16_t*)img);
    else
      k_split_factor<float><<<grid, 256, 0, c->s>>>((const float*)f->data, f->ld, tr ? 1 : 0,
                                                    n_out, n_in, img_rows, kblocks, tf,
                                                    (uint16_t*)img);
    c->count_launch();
    COLA_CUDA(cudaGetLastError());
    prep_mark(fm, key);
  }
  return (const uint16_t*)f->derived.at(key).p;
}

// True when a mode step with these sizes takes the split GEMM (the factor's
// GEMM image is made here when missing, outside graph capture).
static bool gemm_ok(Ctx* c, const TcParams& p, const cola_linop* f, bool tr) {
  if (p.n_in <= kTileM && p.n_out <= kTileM) return false;  // the factor-stationary kernel's
  if (p.out_trans || p.tf < 1 || p.tf > 3 || p.tv < 1 || p.tv > 3) return false;
  const int64_t xrows = p.batch * p.rest;
  if ((int64_t)p.tv * xrows > INT32_MAX || p.rest > INT32_MAX) return false;
  return gemm_factor_image(c, f, tr, p.tf) != nullptr;
}

// The X image of a split GEMM step: TMA layout [tv][R rest][kpad].
static uint16_t* gemm_ximage(Ctx* c, const TcParams& p, int depth, int k) {
  const int kpad = (p.n_in + kBlockK - 1) / kBlockK * kBlockK;
  return (uint16_t*)c->ws.get(depth_name("kgemm", depth, k & 1),
                              (size_t)p.tv * p.batch * p.rest * kpad * 2);
}

// One split GEMM mode step.  `next` (a two-factor product's first step): the
// epilogue writes the second step's X image instead of Y.  `have_img`: this
// step's X image was written by the previous step's epilogue (no pre-split).
static bool gemm_launch(Ctx* c, const cola_linop* f, bool tr, const TcParams& p, int depth,
                        int k, const TcParams* next = nullptr, bool have_img = false) {
  if (!gemm_ok(c, p, f, tr)) return false;
  const int kblocks = (p.n_in + kBlockK - 1) / kBlockK, kpad = kblocks * kBlockK;
  const int nch = (p.n_out + kTileM - 1) / kTileM, img_rows = nch * kTileM;
  const int64_t xrows = p.batch * p.rest;
  const uint16_t* fimg = gemm_factor_image(c, f, tr, p.tf);
  uint16_t* ximg = gemm_ximage(c, p, depth, k);
  TcGemmParams g{};
  if (!tmap_image(&g.tm_x, ximg, (int64_t)p.tv * xrows, kpad)) return false;
  if (!have_img) {
    const int mode = p.pro_z ? 2 : (p.pro_out ? 1 : 0);
    const dim3 pgrid((unsigned)((p.rest + 63) / 64), (unsigned)(kpad / 64), (unsigned)p.batch);
    presplit_kernel(p.tv)<<<pgrid, kPresplitThreads, 0, c->s>>>(
        p.X, p.n_in, p.rest, kpad, xrows, mode, p.pro_z, p.pro_beta, p.pro_out, ximg);
    c->count_launch();
    COLA_CUDA(cudaGetLastError());
  }
  if (next) {
    g.oimg = gemm_ximage(c, *next, depth, k + 1);
    g.o_rstride = next->rest;  // = this step's n_out
    g.o_rows = next->batch * next->rest;
    g.o_kpad = (next->n_in + kBlockK - 1) / kBlockK * kBlockK;
    g.o_swz = 0;
  }
  g.Bimg = fimg;
  g.Y = p.Y;
  g.rest = p.rest;
  g.size_out = p.size_out;
  g.tiles_m = p.tiles_m;
  g.nchunks = nch;
  g.ntiles = p.tiles_m * p.batch * nch;
  g.xrows = xrows;
  g.n_out = p.n_out;
  g.kblocks = kblocks;
  g.img_rows = img_rows;
  g.coeff = p.coeff;
  g.beta = p.beta;
  g.epi_x = p.epi_x;
  g.epi_d = p.epi_d;
  g.epi_dstride = p.epi_dstride;
  g.epi_coeff = p.epi_coeff;
  g.epi_dot = p.epi_dot;
  g.epi_q2 = p.epi_q2;
  g.epi_gamma = p.epi_gamma;
  TcGemmLaunch L{kGemmStages, p.err, p.stall_ns};
  const int grid = (int)std::min<int64_t>(g.ntiles, c->num_sms);
  launch_pdl(gemm_kernel<GemmOne>(p.tf, p.tv), dim3(grid), dim3(kGemmThreads),
             gemm_smem(p.tf, p.tv), c->s, GemmOne{g}, L);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
  return true;
}

using FsKernel = void (*)(TcFsParams);
static FsKernel fs_kernel(int tf, int tv) {
  static const FsKernel tab[3][3] = {
      {k_kron_tc_fs<1, 1>, k_kron_tc_fs<1, 2>, k_kron_tc_fs<1, 3>},
      {k_kron_tc_fs<2, 1>, k_kron_tc_fs<2, 2>, k_kron_tc_fs<2, 3>},
      {k_kron_tc_fs<3, 1>, k_kron_tc_fs<3, 2>, k_kron_tc_fs<3, 3>}};
  return tab[tf - 1][tv - 1];
}

using SlabKernel = void (*)(TcSlabParams);
static SlabKernel slab_kernel(int tf, int tv, int em) {
#define COLA_SLAB_ROW(a, e) \
  {k_kron_tc_slab<a, 1, e>, k_kron_tc_slab<a, 2, e>, k_kron_tc_slab<a, 3, e>}
#define COLA_SLAB_EM(e) {COLA_SLAB_ROW(1, e), COLA_SLAB_ROW(2, e), COLA_SLAB_ROW(3, e)}
  static const SlabKernel tab[3][3][3] = {COLA_SLAB_EM(0), COLA_SLAB_EM(1), COLA_SLAB_EM(2)};
#undef COLA_SLAB_EM
#undef COLA_SLAB_ROW
  return tab[em][tf - 1][tv - 1];
}

static size_t slab_smem(int tf, int tv) {
  return 1024 + 2 * (size_t)(tf + tv) * kFsBTermBytes + 256;
}

struct TcFusion {
  const float* pro_z = nullptr;
  const double* pro_beta = nullptr;
  float* pro_out = nullptr;
  const float* epi_x = nullptr;
  const float* epi_d = nullptr;
  int64_t epi_dstride = 0;
  float epi_coeff = 0.0f;
  double* epi_dot = nullptr;
  const float* epi_q2 = nullptr;
  const double* epi_gamma = nullptr;
  int out_trans = 0;  // first mode step stores slab-major (the slab kernel's input)
  int nsteps = -1;    // mode steps to run (-1: all)
  double* pro_nrm = nullptr;
  int rev = 0;        // first mode step: tiles in reverse order
};

// Runs the d mode steps of a Kronecker MVM on the tensor cores; returns the
// number of row tiles per right-hand side of the last step.
static int64_t kron_tc_run(Ctx* c, const cola_linop* op, const float* X, float* Y, int64_t R,
                           double coeff, double beta, int depth, bool tr, const TcFusion& fu) {
  COLA_REQUIRE(tc_supported(op), COLA_ERR_UNSUPPORTED,
               "tensor-core path takes factors with at most %d rows", kTcMaxN);
  auto tfit = op->derived.find(200);
  COLA_REQUIRE(tfit != op->derived.end(), COLA_ERR_INVALID_ARG,
               "internal: Kronecker factors not split for MIXED precision");
  const int tf = (int)tfit->second.bytes;
  const int tv = std::max(1, std::min(3, c->split_vector_terms));
  int* err = tc_errflag(c);
  static bool attr_set[64] = {false};
  const int d = (int)op->kids.size();
  int64_t cur_size = tr ? op->rows : op->cols, maxsz = cur_size;
  for (int k = 0; k < d; ++k) {
    const cola_linop* f = op->kids[k];
    cur_size = cur_size / (tr ? f->rows : f->cols) * (tr ? f->cols : f->rows);
    maxsz = std::max(maxsz, cur_size);
  }
  cur_size = tr ? op->rows : op->cols;
  const float* cur = X;
  int64_t last_tiles = 0;
  const int nsteps = fu.nsteps < 0 ? d : fu.nsteps;
  // A two-factor product whose both steps take the split GEMM: the first
  // step's epilogue writes the second step's X image (no FP32 intermediate,
  // no second pre-split pass)
  bool chain = false;
  TcParams p1{};
  if (d == 2 && nsteps == 2 && !fu.out_trans) {
    const cola_linop* f0 = op->kids[0];
    const cola_linop* f1 = op->kids[1];
    TcParams p0{};
    p0.n_in = (int)(tr ? f0->rows : f0->cols);
    p0.n_out = (int)(tr ? f0->cols : f0->rows);
    p0.rest = cur_size / p0.n_in;
    p0.batch = R;
    p0.tf = tf;
    p0.tv = tv;
    p1.n_in = (int)(tr ? f1->rows : f1->cols);
    p1.n_out = (int)(tr ? f1->cols : f1->rows);
    p1.rest = p0.rest * p0.n_out / p1.n_in;
    p1.batch = R;
    p1.tf = tf;
    p1.tv = tv;
    chain = gemm_ok(c, p0, f0, tr) && gemm_ok(c, p1, f1, tr);
  }
  for (int k = 0; k < nsteps; ++k) {
    const cola_linop* f = op->kids[k];
    const int n_in = (int)(tr ? f->rows : f->cols), n_out = (int)(tr ? f->cols : f->rows);
    const TcPlan q = make_plan(n_in, n_out, tf, tv);
    const int64_t rest = cur_size / n_in, out_size = rest * n_out;
    const bool last = (k == nsteps - 1);
    float* dst = last ? Y : (float*)c->ws.get(depth_name("kron", depth, k & 1), 4 * maxsz * R);
    TcParams p{};
    p.X = cur;
    p.Y = dst;
    p.Bimg = (const uint16_t*)f->derived.at(100 + (tr ? 10 : 0) + tf).p;
    p.rest = rest;
    p.size_in = cur_size;
    p.size_out = out_size;
    p.batch = R;
    p.tiles_m = (rest + kTileM - 1) / kTileM;
    p.n_chunk = q.n_chunk;
    p.nchunks = q.nchunks;
    p.ntiles = p.tiles_m * R * q.nchunks;
    p.n_in = n_in;
    p.n_out = n_out;
    p.n_pad = q.n_pad;
    p.img_rows = q.img_rows;
    p.kblocks = q.kblocks;
    p.ksteps_last = q.ksteps_last;
    p.tf = tf;
    p.tv = tv;
    p.stages = q.stages;
    p.nbuf = q.nbuf;
    p.stage_bytes = q.stage_bytes;
    p.a_term_bytes = q.a_term_bytes;
    p.b_term_bytes = q.b_term_bytes;
    p.tmem_cols = q.tmem_cols;
    p.coeff = (float)(last ? coeff : 1.0);
    p.beta = (float)(last ? beta : 0.0);
    p.err = err;
    if (k == 0 && c->tc_stall_ns > 0 && !c->capturing) {
      p.stall_ns = (uint64_t)c->tc_stall_ns;  // armed once by cola_test_stall_next_launch
      c->tc_stall_ns = 0;
    }
    if (k == 0) {
      p.pro_z = fu.pro_z;
      p.pro_beta = fu.pro_beta;
      p.pro_out = fu.pro_out;
      p.out_trans = fu.out_trans;
      p.pro_nrm = fu.pro_nrm;
      p.rev = fu.rev;
    }
    if (last && nsteps == d) {
      p.epi_x = fu.epi_x;
      p.epi_d = fu.epi_d;
      p.epi_dstride = fu.epi_dstride;
      p.epi_coeff = fu.epi_coeff;
      p.epi_dot = fu.epi_dot;
      p.epi_q2 = fu.epi_q2;
      p.epi_gamma = fu.epi_gamma;
      last_tiles = p.tiles_m * q.nchunks;
    }
    if (c->device < 64 && !attr_set[c->device]) {
      COLA_CUDA(cudaFuncSetAttribute(k_kron_tc<OneProb>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
      COLA_CUDA(cudaFuncSetAttribute(k_kron_tc<ProbTable>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
      for (int a = 1; a <= 3; ++a)
        for (int b = 1; b <= 3; ++b) {
          COLA_CUDA(cudaFuncSetAttribute(fs_kernel(a, b),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemMax));
          for (int em = 0; em < 3; ++em)
            COLA_CUDA(cudaFuncSetAttribute(slab_kernel(a, b, em),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)slab_smem(a, b)));
          COLA_CUDA(cudaFuncSetAttribute(gemm_kernel<GemmOne>(a, b),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)gemm_smem(a, b)));
          COLA_CUDA(cudaFuncSetAttribute(gemm_kernel<GemmTab>(a, b),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)gemm_smem(a, b)));
        }
      attr_set[c->device] = true;
    }
    const int grid = (int)std::min<int64_t>(p.ntiles, c->num_sms);
    TcFsParams rp{};
    if (fs_plan(p, rp)) {
      launch_pdl(fs_kernel(tf, tv), dim3(grid), dim3(kThreadsFs), fs_smem(rp, tv), c->s, rp);
      c->count_launch();
      COLA_CUDA(cudaGetLastError());
    } else if (!gemm_launch(c, f, tr, p, depth, k, chain && k == 0 ? &p1 : nullptr,
                            chain && k == 1)) {
      COLA_REQUIRE(!chain, COLA_ERR_CUDA, "internal: chained split GEMM step not launched");
      COLA_REQUIRE(!p.out_trans, COLA_ERR_UNSUPPORTED,
                   "internal: slab-major output needs the factor-stationary kernel");
      k_kron_tc<OneProb><<<grid, kThreadsTc, q.smem, c->s>>>(OneProb{p}, p);
      c->count_launch();
      COLA_CUDA(cudaGetLastError());
    }
    cur = dst;
    cur_size = out_size;
  }
  return last_tiles;
}


// The slab kernel takes K_1 (x) K_2 (x) K_3 with K_2, K_3 square 128 x 128 and
// K_1 square of side <= 128 (the first step on the factor-stationary kernel).
static bool slab_ok(const cola_linop* kron) {
  if (kron->kind != LK_KRON || kron->kids.size() != 3) return false;
  const cola_linop* f1 = kron->kids[0];
  for (int k = 1; k < 3; ++k)
    if (kron->kids[k]->rows != kSlabN || kron->kids[k]->cols != kSlabN) return false;
  return f1->rows == f1->cols && f1->rows <= kTileM;
}

// Steps 2 and 3 of the MVM of c_k Kron + c_d d[0] I from the slab-major first
// step output T1: Y = c_k (K_2 (x) K_3 per slab) + c_d d[0] x [- gamma q2] and
// the partials of x . Y.  Returns the slabs per right-hand side (K_1's side).
static int64_t slab_launch(Ctx* c, const cola_linop* kron, const float* T1, float* Y,
                           const float* x, const float* q2, const double* gamma, const float* d,
                           float coeff, float dcoeff, double* dot, int64_t R,
                           const double* scale = nullptr, int rev = 0) {
  const int tf = (int)kron->derived.at(200).bytes;
  const int tv = std::max(1, std::min(3, c->split_vector_terms));
  TcSlabParams sp{};
  sp.rev = rev;
  sp.S = T1;
  sp.img2 = (const uint16_t*)kron->kids[1]->derived.at(100 + tf).p;
  sp.img3 = (const uint16_t*)kron->kids[2]->derived.at(100 + tf).p;
  sp.img_rows2 = make_plan(kSlabN, kSlabN, tf, tv).img_rows;
  sp.img_rows3 = sp.img_rows2;
  sp.Y = Y;
  sp.x = x;
  sp.q2 = q2;
  sp.gamma = gamma;
  sp.scale = scale;
  sp.d = d;
  sp.coeff = coeff;
  sp.dcoeff = dcoeff;
  const int64_t n1 = kron->kids[0]->rows;
  sp.nslab = R * n1;
  sp.slabs_per_rhs = n1;
  sp.dot = dot;
  sp.err = tc_errflag(c);
  const int grid = (int)std::min<int64_t>(sp.nslab, c->num_sms);
  const int em = q2 ? 2 : (x ? 1 : 0);
  launch_pdl(slab_kernel(tf, tv, em), dim3(grid), dim3(kSlabThreads),
             slab_smem(tf, tv), c->s, sp);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
  return n1;
}

// A Kronecker product of the slab shape (see slab_ok) runs as the first mode
// step (slab-major output) and the slab kernel (steps 2 and 3 on chip); other
// shapes, Y = coeff K X + beta Y with beta != 0 and transposes take the d mode
// steps.
template <>
void kron_tc_apply<float>(Ctx* c, const cola_linop* op, const float* X, float* Y, int64_t R,
                          double coeff, double beta, int depth, bool tr) {
  if (!tr && beta == 0.0 && slab_ok(op) && op->derived.count(200)) {
    float* T1 = (float*)c->ws.get(depth_name("kslab", depth, 0), 4 * (size_t)op->cols * R);
    TcFusion f1;
    f1.out_trans = 1;
    f1.nsteps = 1;
    kron_tc_run(c, op, X, T1, R, 1.0, 0.0, depth, false, f1);
    slab_launch(c, op, T1, Y, nullptr, nullptr, nullptr, nullptr, (float)coeff, 0.0f, nullptr,
                R);
    return;
  }
  kron_tc_run(c, op, X, Y, R, coeff, beta, depth, tr, TcFusion{});
}

// One CG MVM for A = c_k * Kron(...) + c_d * Diag(d): the first mode step forms
// p = z + beta p in place, the last step adds c_d * d * p and writes the
// per-(tile, warp) partials of p . Ap.  Returns the last step's row tiles per
// right-hand side (partials per RHS = 4 x that), or 0 when the operator does
// not have this shape (the caller then takes the generic path).
int64_t kron_tc_cg_mvm(Ctx* c, const cola_linop* op, const float* z, const double* beta_vec,
                       const float* p_old, float* p_new, float* Ap, double* tile_dot, int64_t R,
                       int depth, int rev) {
  if (op->kind != LK_SUM || op->kids.size() != 2) return 0;
  int ik = -1, id = -1;
  for (int i = 0; i < 2; ++i) {
    if (op->kids[i]->kind == LK_KRON) ik = i;
    if (op->kids[i]->kind == LK_DIAG) id = i;
  }
  if (ik < 0 || id < 0) return 0;
  const cola_linop* kron = op->kids[ik];
  const cola_linop* dg = op->kids[id];
  if (kron->kids.size() < 2 || !tc_supported(kron)) return 0;
  if (kron->derived.find(200) == kron->derived.end()) return 0;
  if (slab_ok(kron) && dg->stride == 0) {
    // first mode step: p = z + beta p, written, and the slab-major T1; then
    // steps 2 and 3 on chip with the shift term and the p . Ap partials
    float* T1 = (float*)c->ws.get(depth_name("kslab", depth, 0), 4 * (size_t)kron->cols * R);
    TcFusion f1;
    f1.pro_z = z;
    f1.pro_beta = beta_vec;
    f1.pro_out = p_new;
    f1.out_trans = 1;
    f1.nsteps = 1;
    // the two launches run in opposite orders, so that the slab kernel starts
    // on the part of T1 and p the first step wrote last (still in L2)
    f1.rev = rev;
    kron_tc_run(c, kron, p_old, T1, R, 1.0, 0.0, depth, false, f1);
    return slab_launch(c, kron, T1, Ap, p_new, nullptr, nullptr, leaf_ptr<float>(dg),
                       (float)op->coeffs[ik], (float)op->coeffs[id], tile_dot, R, nullptr,
                       !rev);
  }
  TcFusion fu;
  fu.pro_z = z;
  fu.pro_beta = beta_vec;
  fu.pro_out = p_new;
  fu.epi_x = p_new;
  fu.epi_d = leaf_ptr<float>(dg);
  fu.epi_dstride = dg->stride;
  fu.epi_coeff = (float)op->coeffs[id];
  fu.epi_dot = tile_dot;
  return kron_tc_run(c, kron, p_old, Ap, R, op->coeffs[ik], 0.0, depth, false, fu);
}

// One Lanczos MVM for A = c_k * Kron(...) + c_d * s I (s a device scalar): the
// first mode step forms q = scale[r] * w_in and writes it to q_out, the last
// writes w_out = A q - gamma[r] * q_prev and the per-(tile, warp) partials of
// q . w_out.  w_in and w_out may be the same buffer (the first step has
// finished reading before the last one writes).  Returns the last step's row
// tiles per right-hand side, or 0 when the operator does not have this shape.
int64_t kron_tc_lanczos_mvm(Ctx* c, const cola_linop* op, const float* w_in,
                            const double* scale, float* q_out, const float* q_prev,
                            const double* gamma, float* w_out, double* tile_dot, int64_t R,
                            int depth) {
  if (op->kind != LK_SUM || op->kids.size() != 2) return 0;
  int ik = -1, id = -1;
  for (int i = 0; i < 2; ++i) {
    if (op->kids[i]->kind == LK_KRON) ik = i;
    if (op->kids[i]->kind == LK_DIAG && op->kids[i]->stride == 0) id = i;
  }
  if (ik < 0 || id < 0) return 0;
  const cola_linop* kron = op->kids[ik];
  const cola_linop* dg = op->kids[id];
  if (kron->kids.size() < 2 || !tc_supported(kron)) return 0;
  if (kron->derived.find(200) == kron->derived.end()) return 0;
  if (slab_ok(kron)) {
    float* T1 = (float*)c->ws.get(depth_name("kslab", depth, 0), 4 * (size_t)kron->cols * R);
    TcFusion f1;
    f1.pro_beta = scale;
    f1.pro_out = q_out;
    f1.out_trans = 1;
    f1.nsteps = 1;
    kron_tc_run(c, kron, w_in, T1, R, 1.0, 0.0, depth, false, f1);
    return slab_launch(c, kron, T1, w_out, q_out, q_prev, gamma, leaf_ptr<float>(dg),
                       (float)op->coeffs[ik], (float)op->coeffs[id], tile_dot, R);
  }
  TcFusion fu;
  fu.pro_beta = scale;
  fu.pro_out = q_out;
  fu.epi_x = q_out;
  fu.epi_d = leaf_ptr<float>(dg);
  fu.epi_dstride = 0;
  fu.epi_coeff = (float)op->coeffs[id];
  fu.epi_dot = tile_dot;
  fu.epi_q2 = q_prev;
  fu.epi_gamma = gamma;
  return kron_tc_run(c, kron, w_in, w_out, R, op->coeffs[ik], 0.0, depth, false, fu);
}

// Lanczos with unnormalised vectors on a slab-shaped operator (see
// kron_tc_lanczos_unnormalised): the kron node and diagonal of Sum(Kron, Diag).
static bool lanczos_parts(const cola_linop* op, const cola_linop** kron, const cola_linop** dg,
                          int* ik, int* id) {
  if (op->kind != LK_SUM || op->kids.size() != 2) return false;
  *ik = -1;
  *id = -1;
  for (int i = 0; i < 2; ++i) {
    if (op->kids[i]->kind == LK_KRON) *ik = i;
    if (op->kids[i]->kind == LK_DIAG && op->kids[i]->stride == 0) *id = i;
  }
  if (*ik < 0 || *id < 0) return false;
  *kron = op->kids[*ik];
  *dg = op->kids[*id];
  return (*kron)->derived.count(200) && slab_ok(*kron);
}

bool kron_tc_lanczos_unnormalised(const cola_linop* op) {
  const cola_linop *kron, *dg;
  int ik, id;
  return lanczos_parts(op, &kron, &dg, &ik, &id);
}

int64_t kron_tc_lanczos_step1(Ctx* c, const cola_linop* op, const float* v_prev, const float* w,
                              const double* coef, float* v_out, double* nrm, int64_t R,
                              int depth, int rev) {
  const cola_linop *kron, *dg;
  int ik, id;
  COLA_REQUIRE(lanczos_parts(op, &kron, &dg, &ik, &id), COLA_ERR_UNSUPPORTED,
               "internal: unnormalised Lanczos needs a slab-shaped operator");
  float* T1 = (float*)c->ws.get(depth_name("kslab", depth, 0), 4 * (size_t)kron->cols * R);
  TcFusion f1;
  f1.out_trans = 1;
  f1.nsteps = 1;
  f1.rev = rev;
  if (w) {
    f1.pro_z = w;
    f1.pro_beta = coef;
    f1.pro_out = v_out;
    f1.pro_nrm = nrm;
  }
  kron_tc_run(c, kron, v_prev, T1, R, 1.0, 0.0, depth, false, f1);
  return (kron->cols / kron->kids[0]->cols + kTileM - 1) / kTileM;
}

int64_t kron_tc_lanczos_slab(Ctx* c, const cola_linop* op, const float* v, const float* v_prev,
                             const double* gamma, const double* scale, float* w_out,
                             double* tile_dot, int64_t R, int depth, int rev) {
  const cola_linop *kron, *dg;
  int ik, id;
  COLA_REQUIRE(lanczos_parts(op, &kron, &dg, &ik, &id), COLA_ERR_UNSUPPORTED,
               "internal: unnormalised Lanczos needs a slab-shaped operator");
  const float* T1 = (const float*)c->ws.get(depth_name("kslab", depth, 0),
                                            4 * (size_t)kron->cols * R);
  return slab_launch(c, kron, T1, w_out, v, v_prev, gamma, leaf_ptr<float>(dg),
                     (float)op->coeffs[ik], (float)op->coeffs[id], tile_dot, R, scale, rev);
}

int64_t kron_tc_tiles_per_rhs(const cola_linop* op) {
  // row tiles of the last mode step when the operator is Sum(Kron, Diag)
  if (op->kind != LK_SUM || op->kids.size() != 2) return 0;
  for (auto* k : op->kids)
    if (k->kind == LK_KRON && k->kids.size() >= 2 && tc_supported(k)) {
      const cola_linop* last = k->kids.back();
      const int64_t rest = k->rows / last->rows;  // rows produced by the earlier steps
      const int n16 = (int)((last->rows + 15) / 16 * 16);
      return (rest + kTileM - 1) / kTileM * ((n16 + kChunkMax - 1) / kChunkMax);
    }
  return 0;
}

}  // namespace cola

// ------------------------------------------------------------------ batches
namespace cola {

static std::string tagged(const char* tag, const char* what) {
  return std::string(tag) + "." + what;
}

// Tiles of one problem of a batched mode step: 128-row tiles of each
// right-hand side times the output chunks of the factor (host, integer).
static int64_t batch_problem_tiles(int n_out, int64_t rest, int64_t R, int chunk_cap) {
  int nchunks = 0;
  chunk_layout(n_out, chunk_cap, &nchunks);
  return (rest + kTileM - 1) / kTileM * R * nchunks;
}

// Global tile -> problem table of a batched launch (host, integer): problem i
// owns tiles [first[i], first[i] + ntiles[i]) in problem order.
static int64_t batch_tile_table(const std::vector<int64_t>& ntiles, std::vector<int64_t>& first,
                                std::vector<int>& tile_prob) {
  first.assign(ntiles.size(), 0);
  tile_prob.clear();
  int64_t tot = 0;
  for (size_t i = 0; i < ntiles.size(); ++i) {
    first[i] = tot;
    tile_prob.insert(tile_prob.end(), (size_t)ntiles[i], (int)i);
    tot += ntiles[i];
  }
  return tot;
}

std::vector<int64_t> kron_tc_batch_upload(Ctx* c, const std::vector<TcBatchProblem>& probs,
                                          int tf, int tv, const char* tag, int chunk_cap) {
  std::vector<TcParams> hp(probs.size());
  std::vector<int64_t> first(probs.size()), counts(probs.size());
  std::vector<int> tile_prob;
  int64_t tot = 0;
  for (size_t i = 0; i < probs.size(); ++i) {
    const TcBatchProblem& b = probs[i];
    const cola_linop* f = b.factor;
    const int n_in = (int)(b.transpose ? f->rows : f->cols);
    const int n_out = (int)(b.transpose ? f->cols : f->rows);
    const TcPlan q = make_plan(n_in, n_out, tf, tv, chunk_cap);
    TcParams& p = hp[i];
    p = TcParams{};
    p.X = b.X;
    p.Y = b.Y;
    auto it = f->derived.find(100 + (b.transpose ? 10 : 0) + tf);
    COLA_REQUIRE(it != f->derived.end(), COLA_ERR_INVALID_ARG,
                 "internal: batch factor not split for MIXED precision");
    p.Bimg = (const uint16_t*)it->second.p;
    p.rest = b.rest;
    p.size_in = b.size_in;
    p.size_out = b.size_out;
    p.batch = b.R;
    p.tiles_m = (b.rest + kTileM - 1) / kTileM;
    p.n_chunk = q.n_chunk;
    p.nchunks = q.nchunks;
    p.ntiles = batch_problem_tiles(n_out, b.rest, b.R, chunk_cap);
    p.n_in = n_in;
    p.n_out = n_out;
    p.n_pad = q.n_pad;
    p.img_rows = q.img_rows;
    p.kblocks = q.kblocks;
    p.ksteps_last = q.ksteps_last;
    p.b_term_bytes = q.b_term_bytes;
    p.coeff = b.coeff;
    p.beta = b.beta;
    p.pro_z = b.pro_z;
    p.pro_beta = b.pro_beta;
    p.pro_out = b.pro_out;
    p.epi_x = b.epi_x;
    p.epi_d = b.epi_d;
    p.epi_dstride = b.epi_dstride;
    p.epi_coeff = b.epi_coeff;
    p.epi_dot = b.epi_dot;
    counts[i] = p.ntiles;
  }
  tot = batch_tile_table(counts, first, tile_prob);
  // fixed-capacity device tables so replays of a captured graph stay valid
  const size_t cap_p = std::max<size_t>(1, hp.size());
  void* dp = c->ws.get(tagged(tag, "probs"), sizeof(TcParams) * cap_p);
  void* dt = c->ws.get(tagged(tag, "tile"), sizeof(int) * std::max<size_t>(1, tile_prob.size()));
  void* df = c->ws.get(tagged(tag, "first"), sizeof(int64_t) * cap_p);
  void* dc = c->ws.get(tagged(tag, "count"), sizeof(int64_t));
  if (!hp.empty()) {
    COLA_CUDA(cudaMemcpyAsync(dp, hp.data(), sizeof(TcParams) * hp.size(),
                              cudaMemcpyHostToDevice, c->s));
    COLA_CUDA(cudaMemcpyAsync(df, first.data(), sizeof(int64_t) * first.size(),
                              cudaMemcpyHostToDevice, c->s));
  }
  if (!tile_prob.empty())
    COLA_CUDA(cudaMemcpyAsync(dt, tile_prob.data(), sizeof(int) * tile_prob.size(),
                              cudaMemcpyHostToDevice, c->s));
  COLA_CUDA(cudaMemcpyAsync(dc, &tot, sizeof(int64_t), cudaMemcpyHostToDevice, c->s));
  // pageable sources: the copies above are staged before returning, but make
  // the host vectors' lifetime irrelevant by waiting here (tables are small)
  COLA_CUDA(cudaStreamSynchronize(c->s));
  return counts;
}

// Host tables of a batched split GEMM step.
struct GemmBatchTables {
  std::vector<TcGemmParams> hp;
  std::vector<int64_t> counts, pcounts;
};

// Split GEMM form of a batched mode step: per problem the pre-split image of
// its input (inside the shared buffer `image`, zeroed here), its factor's
// GEMM image, and the tile counts of the pre-split pass (64 x 64 tiles) and
// the GEMM (128-row tiles x 128-output chunks, chunk fastest).
static GemmBatchTables gemm_batch_build(Ctx* c, const std::vector<TcBatchProblem>& probs, int tf,
                                        int tv, const char* image) {
  const size_t n = probs.size();
  GemmBatchTables T;
  T.hp.resize(n);
  T.counts.resize(n);
  T.pcounts.resize(n);
  size_t img_elems = 0;
  std::vector<size_t> img_off(n);
  for (size_t i = 0; i < n; ++i) {
    const TcBatchProblem& b = probs[i];
    const cola_linop* f = b.factor;
    const int n_in = (int)(b.transpose ? f->rows : f->cols);
    const int n_out = (int)(b.transpose ? f->cols : f->rows);
    const int kblocks = (n_in + kBlockK - 1) / kBlockK;
    TcGemmParams& g = T.hp[i];
    g = TcGemmParams{};
    g.Bimg = gemm_factor_image(c, f, b.transpose, tf);
    COLA_REQUIRE(g.Bimg, COLA_ERR_INVALID_ARG, "internal: batch factor image during capture");
    g.Y = b.Y;
    g.rest = b.rest;
    g.size_out = b.size_out;
    g.tiles_m = (b.rest + kTileM - 1) / kTileM;
    g.nchunks = (n_out + kTileM - 1) / kTileM;
    g.ntiles = b.R * g.tiles_m * g.nchunks;
    g.xrows = b.R * b.rest;
    g.rows_pad = b.R * g.tiles_m * kTileM;  // each RHS's rows start on a tile boundary
    g.n_out = n_out;
    g.kblocks = kblocks;
    g.img_rows = (int)(g.nchunks * kTileM);
    g.coeff = b.coeff;
    g.beta = b.beta;
    g.epi_x = b.epi_x;
    g.epi_d = b.epi_d;
    g.epi_dstride = b.epi_dstride;
    g.epi_coeff = b.epi_coeff;
    g.epi_dot = b.epi_dot;
    g.X = b.X;
    g.pro_z = b.pro_z;
    g.pro_beta = b.pro_beta;
    g.pro_out = b.pro_out;
    g.n_in = n_in;
    g.kpad = kblocks * kBlockK;
    g.mode = b.pro_z ? 2 : (b.pro_out ? 1 : 0);
    g.R = b.R;
    img_off[i] = img_elems;
    img_elems += (size_t)tv * kblocks * (size_t)g.rows_pad * kBlockK;
    T.counts[i] = g.ntiles;
    T.pcounts[i] = b.R * ((b.rest + 63) / 64) * (g.kpad / 64);
  }
  uint16_t* img = (uint16_t*)c->ws.get(image, std::max<size_t>(1, img_elems) * 2);
  COLA_CUDA(cudaMemsetAsync(img, 0, img_elems * 2, c->s));
  for (size_t i = 0; i < n; ++i) T.hp[i].ximg = img + img_off[i];
  return T;
}

// Uploads the tables under `tag` (fixed-capacity device buffers, so replays of
// a captured graph stay valid).
static void gemm_batch_put(Ctx* c, const GemmBatchTables& T, const char* tag) {
  const size_t n = T.hp.size();
  std::vector<int64_t> first, pfirst;
  std::vector<int> tile_prob, ptile_prob;
  const int64_t tot = batch_tile_table(T.counts, first, tile_prob);
  const int64_t ptot = batch_tile_table(T.pcounts, pfirst, ptile_prob);
  const size_t cap_p = std::max<size_t>(1, n);
  void* dp = c->ws.get(tagged(tag, "gprobs"), sizeof(TcGemmParams) * cap_p);
  void* dt = c->ws.get(tagged(tag, "gtile"), sizeof(int) * std::max<size_t>(1, tile_prob.size()));
  void* df = c->ws.get(tagged(tag, "gfirst"), sizeof(int64_t) * cap_p);
  void* dc = c->ws.get(tagged(tag, "gcount"), 2 * sizeof(int64_t));
  void* pt = c->ws.get(tagged(tag, "ptile"), sizeof(int) * std::max<size_t>(1, ptile_prob.size()));
  void* pf = c->ws.get(tagged(tag, "pfirst"), sizeof(int64_t) * cap_p);
  if (n) {
    COLA_CUDA(cudaMemcpyAsync(dp, T.hp.data(), sizeof(TcGemmParams) * n, cudaMemcpyHostToDevice,
                              c->s));
    COLA_CUDA(cudaMemcpyAsync(df, first.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice,
                              c->s));
    COLA_CUDA(cudaMemcpyAsync(pf, pfirst.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice,
                              c->s));
  }
  if (!tile_prob.empty())
    COLA_CUDA(cudaMemcpyAsync(dt, tile_prob.data(), sizeof(int) * tile_prob.size(),
                              cudaMemcpyHostToDevice, c->s));
  if (!ptile_prob.empty())
    COLA_CUDA(cudaMemcpyAsync(pt, ptile_prob.data(), sizeof(int) * ptile_prob.size(),
                              cudaMemcpyHostToDevice, c->s));
  const int64_t cnt[2] = {tot, ptot};
  COLA_CUDA(cudaMemcpyAsync(dc, cnt, 2 * sizeof(int64_t), cudaMemcpyHostToDevice, c->s));
  COLA_CUDA(cudaStreamSynchronize(c->s));  // host vectors go out of scope
}

std::vector<int64_t> kron_tc_gemm_batch_upload(Ctx* c, const std::vector<TcBatchProblem>& probs,
                                               int tf, int tv, const char* tag,
                                               const char* image) {
  const GemmBatchTables T = gemm_batch_build(c, probs, tf, tv, image);
  gemm_batch_put(c, T, tag);
  return T.counts;
}

void kron_tc_gemm_batch_upload_pair(Ctx* c, const std::vector<TcBatchProblem>& s1,
                                    const std::vector<TcBatchProblem>& s2, int tf, int tv,
                                    const char* tag1, const char* tag2, const char* image1,
                                    const char* image2) {
  COLA_REQUIRE(s1.size() == s2.size(), COLA_ERR_INVALID_ARG, "internal: unpaired batch steps");
  GemmBatchTables T1 = gemm_batch_build(c, s1, tf, tv, image1);
  GemmBatchTables T2 = gemm_batch_build(c, s2, tf, tv, image2);
  for (size_t i = 0; i < s1.size(); ++i) {
    TcGemmParams& a = T1.hp[i];
    const TcGemmParams& b = T2.hp[i];
    COLA_REQUIRE(b.n_in == a.rest && b.rest == a.n_out && b.R == a.R, COLA_ERR_INVALID_ARG,
                 "internal: batch steps do not chain");
    a.oimg = const_cast<uint16_t*>(b.ximg);
    a.o_rstride = b.tiles_m * kTileM;
    a.o_rows = b.rows_pad;
    a.o_kpad = b.kpad;
    a.o_swz = 1;
    T2.pcounts[i] = 0;  // step 2's image comes from step 1's epilogue
  }
  gemm_batch_put(c, T1, tag1);
  gemm_batch_put(c, T2, tag2);
}

void kron_tc_gemm_batch_launch(Ctx* c, const char* tag, int tf, int tv, bool presplit) {
  const TcGemmParams* probs = (const TcGemmParams*)c->ws.bufs.at(tagged(tag, "gprobs")).p;
  const int64_t* cnt = (const int64_t*)c->ws.bufs.at(tagged(tag, "gcount")).p;
  const int* pt = (const int*)c->ws.bufs.at(tagged(tag, "ptile")).p;
  const int64_t* pf = (const int64_t*)c->ws.bufs.at(tagged(tag, "pfirst")).p;
  // persistent: as many blocks as are resident at once (3 x 256 threads x 80
  // registers per SM), so that no block starts its share of tiles late
  const dim3 pgrid((unsigned)(3 * c->num_sms));
  if (presplit) {
    if (tv == 1)
      k_presplit_tab<1><<<pgrid, kPresplitThreads, 0, c->s>>>(probs, pt, pf, cnt + 1);
    else if (tv == 2)
      k_presplit_tab<2><<<pgrid, kPresplitThreads, 0, c->s>>>(probs, pt, pf, cnt + 1);
    else
      k_presplit_tab<3><<<pgrid, kPresplitThreads, 0, c->s>>>(probs, pt, pf, cnt + 1);
    c->count_launch();
    COLA_CUDA(cudaGetLastError());
  }
  TcGemmLaunch L{kGemmStages, tc_errflag(c), 0};
  if (c->tc_stall_ns > 0 && !c->capturing) {
    L.stall_ns = (uint64_t)c->tc_stall_ns;  // armed once by cola_test_stall_next_launch
    c->tc_stall_ns = 0;
  }
  // the first step of a CG iteration runs its tiles backwards: it starts on
  // the images the pre-split pass wrote last, and leaves the first problems'
  // output in L2 for the second step, which runs forwards
  L.rev = presplit ? 1 : 0;
  GemmTab src{probs, (const int*)c->ws.bufs.at(tagged(tag, "gtile")).p,
              (const int64_t*)c->ws.bufs.at(tagged(tag, "gfirst")).p, cnt};
  COLA_CUDA(cudaFuncSetAttribute(gemm_kernel<GemmTab>(tf, tv),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gemm_smem(tf, tv)));
  launch_pdl(gemm_kernel<GemmTab>(tf, tv), dim3(c->num_sms), dim3(kGemmThreads),
             gemm_smem(tf, tv), c->s, src, L);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
}

int kron_tc_batch_max_stages(int tf, int tv, int max_n_chunk) {
  uint32_t sb = (uint32_t)(tv * kTileM * 128 + tf * (uint32_t)max_n_chunk * 128u);
  sb = (sb + 1023) / 1024 * 1024;
  return (int)std::min<size_t>(4, (size_t)(200 * 1024) / sb);
}

int kron_tc_chunk_width(int n_out, int chunk_cap, int* nchunks) {
  return chunk_layout(n_out, chunk_cap, nchunks);
}

void kron_tc_batch_launch(Ctx* c, const char* tag, int tf, int tv, int max_n_chunk, int stages) {
  TcParams K{};
  K.tf = tf;
  K.tv = tv;
  K.a_term_bytes = kTileM * 128;
  K.stage_bytes = (uint32_t)(tv * K.a_term_bytes + tf * (uint32_t)max_n_chunk * 128u);
  K.stage_bytes = (K.stage_bytes + 1023) / 1024 * 1024;
  const int max_stages = kron_tc_batch_max_stages(tf, tv, max_n_chunk);
  K.stages = stages > 0 ? std::min(stages, max_stages) : max_stages;
  K.n_chunk = max_n_chunk;
  K.nbuf = (4 * max_n_chunk <= 512) ? 2 : 1;
  uint32_t cols = 32;
  while (cols < (uint32_t)(2 * K.nbuf * max_n_chunk)) cols <<= 1;
  K.tmem_cols = cols;
  K.err = tc_errflag(c);
  if (c->tc_stall_ns > 0 && !c->capturing) {
    K.stall_ns = (uint64_t)c->tc_stall_ns;  // armed once by cola_test_stall_next_launch
    c->tc_stall_ns = 0;
  }
  const size_t smem = (size_t)K.stages * K.stage_bytes + 1024 + 256;
  ProbTable src;
  src.probs = (const TcParams*)c->ws.bufs.at(tagged(tag, "probs")).p;
  src.tile_prob = (const int*)c->ws.bufs.at(tagged(tag, "tile")).p;
  src.first = (const int64_t*)c->ws.bufs.at(tagged(tag, "first")).p;
  src.count_dev = (const int64_t*)c->ws.bufs.at(tagged(tag, "count")).p;
  COLA_CUDA(cudaFuncSetAttribute(k_kron_tc<ProbTable>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  k_kron_tc<ProbTable><<<c->num_sms, kThreadsTc, smem, c->s>>>(src, K);
  c->count_launch();
  COLA_CUDA(cudaGetLastError());
}

}  // namespace cola

// ------------------------------------------------------------------ plans
using namespace cola;

extern "C" cola_status cola_batch_tile_table(int32_t nprob, const int32_t* n_out,
                                             const int64_t* rest, const int64_t* nrhs,
                                             int32_t chunk_cap, int64_t* first,
                                             int32_t* tile_prob, int64_t capacity,
                                             int64_t* total) {
  return guard([&] {
    COLA_REQUIRE(nprob >= 0 && (nprob == 0 || (n_out && rest && nrhs && first)) && total,
                 COLA_ERR_INVALID_ARG, "NULL argument");
    COLA_REQUIRE(chunk_cap == 64 || chunk_cap == 128, COLA_ERR_INVALID_ARG,
                 "chunk_cap %d (64 or 128)", chunk_cap);
    std::vector<int64_t> nt(nprob), f;
    std::vector<int> tp;
    for (int32_t i = 0; i < nprob; ++i) {
      COLA_REQUIRE(n_out[i] >= 1 && n_out[i] <= 8192 && rest[i] >= 1 && nrhs[i] >= 1,
                   COLA_ERR_INVALID_ARG, "problem %d: n_out %d rest %lld nrhs %lld", i,
                   n_out[i], (long long)rest[i], (long long)nrhs[i]);
      nt[i] = batch_problem_tiles(n_out[i], rest[i], nrhs[i], chunk_cap);
    }
    const int64_t tot = batch_tile_table(nt, f, tp);
    *total = tot;
    for (int32_t i = 0; i < nprob; ++i) first[i] = f[i];
    COLA_REQUIRE(tot <= capacity && (tot == 0 || tile_prob), COLA_ERR_INVALID_ARG,
                 "tile table of %lld entries, capacity %lld", (long long)tot,
                 (long long)capacity);
    for (int64_t t = 0; t < tot; ++t) tile_prob[t] = tp[(size_t)t];
  });
}
