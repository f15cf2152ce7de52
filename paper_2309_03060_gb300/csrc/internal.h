// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <utility>
#include <string>
#include <vector>

#include "../../include/cola.h"

namespace cola {

// ---------------------------------------------------------------- errors
struct Failure {
  cola_status status;
};
[[noreturn]] void fail(cola_status st, const char* fmt, ...);
void set_error_message(const char* msg);
void clear_error();

#define COLA_CUDA(x)                                                                     \
  do {                                                                                   \
    cudaError_t e_ = (x);                                                                \
    if (e_ != cudaSuccess)                                                               \
      ::cola::fail(COLA_ERR_CUDA, "%s:%d: %s: %s", __FILE__, __LINE__, #x,               \
                   cudaGetErrorString(e_));                                              \
  } while (0)

#define COLA_REQUIRE(cond, st, ...)                                                      \
  do {                                                                                   \
    if (!(cond)) ::cola::fail(st, __VA_ARGS__);                                          \
  } while (0)

// Runs `body` and converts internal failures into a status code.
template <typename F>
cola_status guard(F&& body) {
  try {
    clear_error();
    body();
    return COLA_OK;
  } catch (const Failure& f) {
    return f.status;
  }
}

// -------------------------------------------------------------- workspace
struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Workspace {
  std::map<std::string, Buf> bufs;
  uint64_t generation = 0;  // bumps whenever any buffer moves (graphs key on it)
  void* get(const std::string& name, size_t bytes);
  void release_all();
};

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  int64_t kernels = 0;  // kernel nodes per replay
  uint64_t generation = 0;
};

struct Ctx {
  int device = 0;
  int num_sms = 0;
  cudaStream_t s = nullptr;   // internal stream; all work runs here
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;
  Workspace ws;
  int64_t launches = 0;
  int split_vector_terms = 2;  // BF16 terms per vector entry of the MIXED contraction
  int split_factor_terms = 2;  // BF16 terms per factor entry (cola_matvec)
  bool capturing = false;
  int64_t captured = 0;
  std::map<std::string, GraphEntry> graphs;
  // tile shapes picked by timing for batched solves: key -> (chunk cap, stages)
  std::map<std::string, std::pair<int, int>> tuned;
  void* pinned = nullptr;     // small host staging area (pinned)
  size_t pinned_bytes = 0;
  int* tc_err_host = nullptr;  // pinned copy of the tensor-core timeout flag
  cudaEvent_t tc_err_ev = nullptr;
  bool tc_err_pending = false;  // a copy of the flag is in flight
  int64_t tc_stall_ns = 0;      // armed by cola_test_stall_next_launch, consumed once
  void* host_pinned(size_t bytes);
  void count_launch() {
    if (capturing)
      ++captured;
    else
      ++launches;
  }
};

// Sets the context's BF16 vector split terms for the duration of one call
// (a solve with its own option) and restores the caller's setting after it.
struct VectorTermsScope {
  Ctx* c;
  int saved;
  VectorTermsScope(Ctx* c_, int terms) : c(c_), saved(c_->split_vector_terms) {
    c->split_vector_terms = terms;
  }
  ~VectorTermsScope() { c->split_vector_terms = saved; }
};

// Orders the internal stream after the caller's stream on entry and the
// caller's stream after the internal one on exit.
struct StreamJoin {
  Ctx* c;
  cudaStream_t user;
  StreamJoin(Ctx* c_, cola_stream s);
  ~StreamJoin();
};

}  // namespace cola

struct cola_ctx : cola::Ctx {};

// ----------------------------------------------------------------- linops
enum LinKind { LK_DENSE, LK_DIAG, LK_LOWRANK, LK_KRON, LK_KRONSUM, LK_SUM, LK_PRODUCT };

struct cola_linop {
  cola_ctx* ctx = nullptr;
  uint64_t uid = 0;             // unique per node for the life of the process
  uint64_t eig_hash = 0;        // contents hash of the factor its cached eigendecomposition is of
  cola_linop* eig_kron = nullptr;  // Kron node: the eigenvector matrices (x)_k V_k^T of
                                   // this Kron node's factors (owned; kron_precond)
  LinKind kind = LK_DENSE;
  int64_t rows = 0, cols = 0;
  int refs = 1;
  int spd = 0;
  // leaves
  const void* data = nullptr;   // dense matrix / diagonal / U
  const void* data2 = nullptr;  // V of a low-rank leaf (nullptr: U U^T)
  int64_t ld = 0;               // dense leading dimension
  int64_t stride = 1;           // diag: 1 vector, 0 scalar
  int64_t rank = 0;             // low-rank k
  cola_dtype dtype = COLA_F64;
  // compositions
  std::vector<cola_linop*> kids;
  std::vector<double> coeffs;
  // tridiagonal band of a Kronecker-sum factor: lo[i]=A[i,i-1], di[i]=A[i,i], up[i]=A[i,i+1]
  bool tridiag = false;
  std::vector<double> band_host;  // 3*n
  // converted copies of borrowed leaf data, owned here
  std::map<int, cola::Buf> derived;
  // reuse of derived copies across calls (cola_linop_cache_prepared): a copy
  // made while `version` was v is recorded as v + 1 and reused while the
  // version is unchanged; cola_linop_touch bumps the version
  bool cache_prepared = false;
  uint64_t version = 0;
  std::map<int, uint64_t> prep_version;
  ~cola_linop();
};

namespace cola {
// True when derived copy `key` of leaf op may be reused as it is.
inline bool prep_fresh(const cola_linop* op, int key) {
  if (!op->cache_prepared || !op->derived.count(key)) return false;
  auto it = op->prep_version.find(key);
  return it != op->prep_version.end() && it->second == op->version + 1;
}
inline void prep_mark(cola_linop* op, int key) { op->prep_version[key] = op->version + 1; }
}  // namespace cola

namespace cola {

enum DerivedKey {
  DK_F64 = 0, DK_F32 = 1, DK_BAND64 = 2, DK_BAND32 = 3,
  DK_V_F64 = 4, DK_V_F32 = 5, DK_SPLIT_BF16 = 6,
  // transposed (k x n) low-rank factors in the working type: U, V for FP64 / FP32
  DK_UT_F64 = 20, DK_UT_F32 = 21, DK_VT_F64 = 22, DK_VT_F32 = 23
};

// dtype used for vectors at a precision
inline bool prec_is_f64(int prec) { return prec == COLA_PREC_F64; }

// Leaf data in the working type T, converting the borrowed array on the
// context stream when its dtype differs (prepare_leaves must have run).
template <typename T>
const T* leaf_ptr(const cola_linop* op, bool second = false);

// Convert every leaf of the tree to the working type of `prec` (and the BF16
// splits for MIXED).  Enqueued on c->s.
void prepare_leaves(Ctx* c, cola_linop* op, int prec, int split_terms);

// Y = coeff * op(X) + beta * Y for R vectors (op^T when transpose).
// X and Y must not alias.  depth selects the temp buffers of this level.
template <typename T>
void apply(Ctx* c, const cola_linop* op, const T* X, T* Y, int64_t R, double coeff, double beta,
           int depth, bool transpose, int prec);

// Diag(A) (App. A.1.4 rules) into out[n] (type T).
template <typename T>
void diagonal(Ctx* c, const cola_linop* op, T* out, int depth);

// grads[l] += scale * sum_r Uw_r^T (dA/dtheta_l) X_r   (Uw already weighted)
template <typename T>
void bilinear(Ctx* c, const cola_linop* op, const T* Uw, const T* X, int64_t R, double scale,
              const std::vector<void*>& grads, int& leaf_index, int depth);

void collect_leaves(const cola_linop* op, std::vector<const cola_linop*>& out);

// ------------------------------------------------------------- kernels API
template <typename T>
void gemm(Ctx* c, int64_t M, int64_t N, int64_t K, double alpha, const T* A, int64_t lda_m,
          int64_t lda_k, int64_t sA, const T* B, int64_t ldb_k, int64_t ldb_n, int64_t sB,
          double beta, T* C, int64_t ldc_m, int64_t ldc_n, int64_t sC, int64_t batch);

// One problem of a grouped GEMM: C = alpha A B + beta C with element strides.
template <typename T>
struct GemmDesc {
  int64_t M, N, K;
  const T* A;
  int64_t lam, lak;
  const T* B;
  int64_t lbk, lbn;
  T* C;
  int64_t lcm, lcn;
  T alpha, beta;
};
// Grouped GEMM over a device table of nprob problems (one per blockIdx.z);
// max_m / max_n bound the problems' M and N.
template <typename T>
void gemm_grouped(Ctx* c, const GemmDesc<T>* dev_probs, int nprob, int64_t max_m, int64_t max_n);

// Deterministic per-vector dot products: out[r] = sum_i a[r*lda+i] b[r*ldb+i].
// partials: workspace of dot_blocks(n)*R doubles.  Two launches.
int dot_blocks(int64_t n);
template <typename T>
void dots(Ctx* c, const T* a, const T* b, int64_t n, int64_t R, double* partials, double* out);

template <typename TI, typename TO>
void convert(Ctx* c, const TI* in, TO* out, int64_t n);
template <typename T>
void fill_zero(Ctx* c, T* p, int64_t n);
template <typename T>
void scale_rows(Ctx* c, T* X, int64_t n, int64_t R, const double* w_dev);  // X[r] *= w[r]

void rademacher(Ctx* c, uint64_t seed, int64_t offset, int64_t count, void* out, cola_dtype dt);

template <typename T>
void diag_apply(Ctx* c, const T* d, int64_t stride, const T* X, T* Y, int64_t n, int64_t R,
                double coeff, double beta);
// Kronecker sum of tridiagonal factors; with dg, also the diagonal term
// dcoeff Diag(d) X in the same pass where the two-factor kernel runs (returns
// true then; false: the caller applies the diagonal itself).
template <typename T>
bool stencil_apply(Ctx* c, int nf, const int64_t* sizes, const T* bands, const T* X, T* Y,
                   int64_t R, double coeff, double beta, const T* dg = nullptr,
                   int64_t dstride = 0, double dcoeff = 0.0);
// Blocks of the low-rank V^T X reduction: partials hold kLowRankBlocks * k * R doubles.
constexpr int kLowRankBlocks = 608;
template <typename T>
void lowrank_vtx(Ctx* c, const T* V, const T* X, int64_t n, int64_t k, int64_t R, T* W,
                 double* partials);  // W[k][R] = V^T X^T
template <typename T>
void lowrank_uw(Ctx* c, const T* U, const T* W, T* Y, int64_t n, int64_t k, int64_t R,
                double coeff, double beta,
                const T* Ut = nullptr);  // Y[r,i] = coeff sum_k U[i,k] W[k,r] + beta Y
                                          // (Ut: U transposed, k x n, when prepared)
template <typename T>
void transpose_nk(Ctx* c, const T* src, T* dst, int64_t n, int64_t k);  // n x k -> k x n
template <typename T>
void lowrank_grad(Ctx* c, const T* A, const T* W, T* G, int64_t n, int64_t k, int64_t R,
                  double scale);  // G[i,k] += scale sum_r A[r,i] W[k,r]
template <typename T>
void rowsum_products(Ctx* c, const T* U, const T* V, T* out, int64_t n, int64_t k,
                     double coeff, double beta);  // out[i] = coeff sum_k U[i,k]V[i,k] + beta out
template <typename T>
void kron_diag(Ctx* c, int nf, const int64_t* sizes, const T* const* fdiag_src,
               const int64_t* lds, T* out, double coeff, double beta);
template <typename T>
void kronsum_diag(Ctx* c, int nf, const int64_t* sizes, const T* const* f, const int64_t* lds,
                  T* out, double coeff, double beta);
template <typename T>
void diag_grad(Ctx* c, const T* U, const T* X, T* G, int64_t n, int64_t R, double scale,
               bool scalar, double* partials);
template <typename T>
void permute_mode_front(Ctx* c, const T* X, T* Y, int64_t R, int64_t A, int64_t n, int64_t C);
template <typename T>
void add_partials(Ctx* c, const T* P, T* G, int64_t count, int64_t nparts, double scale);
// out[r] = sum of partials[r*nblk .. r*nblk+nblk-1] in order
void dot_final(Ctx* c, const double* partials, int nblk, int64_t R, double* out);

// Per right-hand-side CG state in device memory.
struct CgState {
  double rz, pAp, alpha, beta;
  double rr, rr_ref, bb, tol2;
  double rr64;
  long long iters;
  int active, flag, status, updates;
  int paused;   // refined solves: the recursion has run ahead of what FP32 can resolve
  int restart;  // set by a residual replacement that restarts the search direction
};

// ------------------------------------------------------------ solver entries
cola_status cg_solve_impl(Ctx* c, const cola_linop* op, const void* B, void* X, int64_t R,
                          const cola_cg_opts& o, cola_cg_info* info);
cola_status batched_cg_impl(Ctx* c, int32_t nsys, const cola_linop* const* ops,
                            const void* const* B, void* const* X, const int64_t* nrhs,
                            const cola_cg_opts& o, cola_cg_info* info);
void lanczos_impl(Ctx* c, const cola_linop* op, const void* Q0, int64_t nv, int m, int prec,
                  int reorth, double* alpha, double* beta, int* m_eff);
void householder_lanczos(Ctx* c, const cola_linop* op, const void* Q0, int64_t nv, int m,
                         int prec, double* alpha, double* beta, int* m_eff);
// SLQ log-det estimate (cola_slq_logdet without the argument checks); synchronous.
void slq_impl(Ctx* c, const cola_linop* op, int nprobes, int m, uint64_t seed,
              const void* probes, int prec, int reorth, double* logdet, double* std_err,
              double* per_probe, int* clamped);
void bilinear_entry(Ctx* c, const cola_linop* op, const void* U, const void* X,
                    const double* weights, int64_t R, int prec, void* const* grads,
                    int accumulate, int depth);
void check_cg_args(const cola_linop* op, const cola_cg_opts* o, int64_t R);
// Raises COLA_ERR_TIMEOUT when a tensor-core kernel gave up waiting (and clears the flag).
void tc_check_error(Ctx* c);        // synchronises the stream
void tc_check_error_async(Ctx* c);  // reports an earlier call's timeout, queues a check
// Fused MIXED CG MVM for Sum(Kron, Diag); see kron_tc.cu.  0 = not applicable.
// p_new = z + beta p_old is formed in the first mode step (p_new != p_old).
// rev: the first mode step walks its tiles in reverse order (and the slab
// kernel, where used, the other way); results do not depend on it.
int64_t kron_tc_cg_mvm(Ctx* c, const cola_linop* op, const float* z, const double* beta_vec,
                       const float* p_old, float* p_new, float* Ap, double* tile_dot, int64_t R,
                       int depth, int rev = 0);
int64_t kron_tc_tiles_per_rhs(const cola_linop* op);
// Fused Lanczos MIXED MVM for Sum(Kron, scalar Diag); see kron_tc.cu.  0 = not applicable.
int64_t kron_tc_lanczos_mvm(Ctx* c, const cola_linop* op, const float* w_in,
                            const double* scale, float* q_out, const float* q_prev,
                            const double* gamma, float* w_out, double* tile_dot, int64_t R,
                            int depth);
// Lanczos with unnormalised basis vectors v_j (q_j = s_j v_j, s_j = 1 / beta_j)
// for Sum(c_k K_1 (x) K_2 (x) K_3, c_d s I) with 128 x 128 K_2, K_3 (kron_tc.cu):
//   step 1: v_out = w + coef[r] v_prev (coef = -alpha_{j-1} s_{j-1}), written,
//           its K_1 mode product slab-major, per (tile, warp) partials of
//           ||v_out||^2 in nrm (8 per tile; returns the tiles per right-hand
//           side); w == nullptr: v_prev itself, nothing written
//   slab:   w_out = s (c_k K v + c_d s v) - gamma v_prev and the per-(slab,
//           warp) partials of (s v) . w_out (returns the slabs per RHS)
bool kron_tc_lanczos_unnormalised(const cola_linop* op);
// rev: tiles (slabs) in reverse order; results do not depend on it.
int64_t kron_tc_lanczos_step1(Ctx* c, const cola_linop* op, const float* v_prev, const float* w,
                              const double* coef, float* v_out, double* nrm, int64_t R,
                              int depth, int rev = 0);
int64_t kron_tc_lanczos_slab(Ctx* c, const cola_linop* op, const float* v, const float* v_prev,
                             const double* gamma, const double* scale, float* w_out,
                             double* tile_dot, int64_t R, int depth, int rev = 0);

// One tensor-core mode-step problem of a batch (host mirror of the kernel's
// per-problem parameters) and the launch over a device problem table.
struct TcBatchProblem {
  const float* X;
  float* Y;
  const cola_linop* factor;  // dense leaf, already split (kron_tc_prepare)
  bool transpose;
  int64_t rest, size_in, size_out, R;
  float coeff, beta;
  const float* pro_z;
  const double* pro_beta;
  float* pro_out;
  const float* epi_x;
  const float* epi_d;
  int64_t epi_dstride;
  float epi_coeff;
  double* epi_dot;
};
// Uploads the problem and tile tables into workspace buffers named after
// `tag` and returns the number of tiles per problem (in table order).
// Every problem's output columns go in chunks of at most chunk_cap (64 or 128).
std::vector<int64_t> kron_tc_batch_upload(Ctx* c, const std::vector<TcBatchProblem>& probs,
                                          int tf, int tv, const char* tag, int chunk_cap);
// Launches one persistent k_kron_tc over the table uploaded under `tag` with
// `stages` pipeline stages (0: as many as fit, at most 4).
void kron_tc_batch_launch(Ctx* c, const char* tag, int tf, int tv, int max_n_chunk, int stages);
int kron_tc_batch_max_stages(int tf, int tv, int max_n_chunk);
// Split GEMM form of a batched mode step (kron_tc.cu): uploads its tables under
// `tag`, the pre-split images in the workspace buffer `image` (one buffer may
// serve the table sets of steps that never run at the same time), and returns
// the tiles per problem (128-row tiles x 128-output chunks, chunk fastest:
// the p . Ap slots follow this tile order).
std::vector<int64_t> kron_tc_gemm_batch_upload(Ctx* c, const std::vector<TcBatchProblem>& probs,
                                               int tf, int tv, const char* tag,
                                               const char* image);
// Both steps of two-factor problems (s2[i] is the second mode step of
// s1[i]'s operator): step 1's epilogue writes step 2's pre-split image, so
// step 2 runs without a pre-split pass.
void kron_tc_gemm_batch_upload_pair(Ctx* c, const std::vector<TcBatchProblem>& s1,
                                    const std::vector<TcBatchProblem>& s2, int tf, int tv,
                                    const char* tag1, const char* tag2, const char* image1,
                                    const char* image2);
// Launches the pre-split pass (unless `presplit` is false: the image was
// written by the previous step) and the persistent split GEMM over the tables
// uploaded under `tag`.
void kron_tc_gemm_batch_launch(Ctx* c, const char* tag, int tf, int tv, bool presplit = true);
// Chunk width (and count) of n_out output columns under a chunk cap.
int kron_tc_chunk_width(int n_out, int chunk_cap, int* nchunks);

// Preconditioner M = c_k (K_1 (x) ... (x) K_d) + c_d mean(d) I for A = c_k Kron
// + c_d Diag(d), applied exactly from the factor eigendecompositions (kron_eig.cu).
struct KronPrecond {
  const cola_linop* qt = nullptr;  // Q^T = (x)_k V_k^T as a Kron node
  int prec = 0;                    // precision the mode products run in
  float* inv32 = nullptr;          // 1 / eigenvalue of M per flat index (device)
  double* inv64 = nullptr;
};
bool eig_solve_if_structured(Ctx* c, const cola_linop* op, const void* B, void* X, int64_t R,
                             bool f64);
bool kron_precond_setup(Ctx* c, cola_linop* op, KronPrecond* P, int64_t R, int prec,
                        int split_terms);
template <typename T>
void kron_precond_apply(Ctx* c, const KronPrecond& P, const T* r, T* z, int64_t R);

// Programmatic dependent launch: a kernel launched with launch_pdl may start
// while the previous kernel on the stream is still running.  It must call
// pdl_wait() before it touches memory that earlier kernels write or read;
// pdl_trigger() lets the next kernel start early.  Both are no-ops for a
// kernel launched without the attribute.
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
void launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  COLA_CUDA(cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...));
}
#endif

}  // namespace cola
