/*
 * cola.h - C ABI of the GB300 (sm_103a) compositional linear-algebra library.
 *
 * Operators are trees of linear maps defined by their MVM (CoLA Sec. 3.1):
 * Dense, Diagonal and LowRank leaves composed by Sum, Product, Kronecker and
 * Kronecker sum (Sec. 3.2).  On top of the MVM the library runs conjugate
 * gradients (Table 5, PSD base case), Lanczos and stochastic Lanczos
 * quadrature for log det A = Tr(log A) (App. A.2, Table 5), and the adjoint
 * rules of App. B.2 for gradients with respect to the operator's leaves.
 *
 * Conventions shared by every call:
 *  - All array arguments are DEVICE pointers unless the comment says host.
 *    Leaf data is BORROWED: the library keeps the pointer, never copies or
 *    frees it; the caller keeps it alive (and unchanged in structure) until
 *    the linop and every linop built from it are released.
 *  - Matrices are row-major; `ld` is the distance between rows in elements.
 *  - Vectors are row-major (C order) over the Kronecker index:
 *    (K_1 (x) ... (x) K_d) vec(X) = vec(K_1 X ... ) with entry (i_1..i_d) at
 *    ((i_1 n_2 + i_2) n_3 + ...).  A block of R vectors is [R][N], contiguous.
 *  - Every call returns cola_status; COLA_OK is 0.  On error the message of
 *    the calling thread's last failure is available from cola_last_error().
 *    Results of a failed call are unspecified unless its comment says so.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    are ordered after prior work on `stream`; calls documented as
 *    synchronous return after their results are complete, the others only
 *    enqueue work.
 *  - A context owns device workspace, cached launch plans and CUDA graphs.
 *    A context must not be used by two host threads at the same time.
 */
#ifndef COLA_GB300_H
#define COLA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cola_ctx cola_ctx;
typedef struct cola_linop cola_linop;
typedef void* cola_stream;

typedef enum {
  COLA_OK = 0,
  COLA_ERR_INVALID_ARG = 1,
  COLA_ERR_SHAPE = 2,
  COLA_ERR_DTYPE = 3,
  COLA_ERR_BREAKDOWN = 4,      /* CG: p^T A p <= 0 or NaN (operator not SPD in working
                                  precision), or a right-hand side with a NaN / Inf entry */
  COLA_ERR_NOT_CONVERGED = 5,  /* tolerance not reached in maxiter; results still written */
  COLA_ERR_TIMEOUT = 6,
  COLA_ERR_CUDA = 7,
  COLA_ERR_OOM = 8,
  COLA_ERR_UNSUPPORTED = 9     /* composition the GPU path does not implement */
} cola_status;

typedef enum { COLA_F64 = 0, COLA_F32 = 1 } cola_dtype;

/* Arithmetic of the MVM and Krylov recurrences.
 *  F64   : FP64 everywhere (vectors FP64).
 *  F32   : FP32 SIMT MVM and FP32 recurrences (vectors FP32).
 *  MIXED : Kronecker contractions on tcgen05 tensor cores with BF16 split
 *          operands (hi + lo [+ lo2] terms) and FP32 accumulation in TMEM,
 *          FP32 recurrences (vectors FP32).  Non-Kronecker terms as F32. */
typedef enum { COLA_PREC_F64 = 0, COLA_PREC_F32 = 1, COLA_PREC_MIXED = 2 } cola_precision;

typedef enum {
  COLA_LEAF_DENSE = 0, COLA_LEAF_DIAG = 1, COLA_LEAF_SCALAR = 2, COLA_LEAF_LOWRANK = 3
} cola_leaf_kind;

/* Message of the calling thread's most recent failure ("" if none). */
const char* cola_last_error(void);

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  *out receives the handle. */
cola_status cola_create(int device, cola_ctx** out);
/* Free the context's workspace, plans and graphs.  Linops built on it must
 * be released first. */
cola_status cola_destroy(cola_ctx* ctx);

/* --------------------------------------------------------------- operators */

/* Dense leaf (Sec. 3.1): rows x cols, row-major with leading dimension ld,
 * element type dtype.  Borrowed. */
cola_status cola_linop_dense(cola_ctx* ctx, int64_t rows, int64_t cols, const void* data,
                             int64_t ld, cola_dtype dtype, cola_linop** out);

/* Diagonal leaf (Sec. 3.1): [Diag(d) v]_i = d_i v_i, n x n.
 * stride 1: d holds n entries.  stride 0: d holds ONE entry s, read on the
 * device at every use, and the operator is s * I (a differentiable scalar,
 * e.g. a noise variance).  Borrowed. */
cola_status cola_linop_diag(cola_ctx* ctx, int64_t n, const void* d, int64_t stride,
                            cola_dtype dtype, cola_linop** out);

/* Low-rank leaf U V^T (the low-rank term of the Woodbury rule, App. A.1.1):
 * U is n x k row-major, V is n x k row-major or NULL for U U^T.  Borrowed. */
cola_status cola_linop_lowrank(cola_ctx* ctx, int64_t n, int64_t k, const void* U,
                               const void* V, cola_dtype dtype, cola_linop** out);

/* Kronecker product K_1 (x) ... (x) K_d (Sec. 3.2, Table 3: MVM cost
 * tau_A N_B + N_A tau_B).  Factors must be Dense leaves (any shape).
 * The node takes a reference on each factor. */
cola_status cola_linop_kron(cola_ctx* ctx, int nfactors, cola_linop* const* factors,
                            cola_linop** out);

/* Kronecker sum A_1 (+) ... (+) A_d = sum_k I (x) .. A_k .. (x) I (Sec. 3.2,
 * App. A.1.2).  Factors must be square Dense leaves.  A factor whose entries
 * are zero outside the three central diagonals is applied as a tridiagonal
 * stencil; that check reads the factor once, at this call, so its data must
 * be valid here. */
cola_status cola_linop_kronsum(cola_ctx* ctx, int nfactors, cola_linop* const* factors,
                               cola_linop** out);

/* Sum  sum_i c_i A_i (Sec. 3.2); coeffs is a HOST array of nterms doubles or
 * NULL for all ones.  All terms must have the same shape. */
cola_status cola_linop_sum(cola_ctx* ctx, int nterms, cola_linop* const* terms,
                           const double* coeffs, cola_linop** out);

/* Product A_1 A_2 ... A_m (Sec. 3.2), applied right to left. */
cola_status cola_linop_product(cola_ctx* ctx, int nterms, cola_linop* const* terms,
                               cola_linop** out);

/* PSD / self-adjoint annotation (Sec. 3.2 decorators).  CG, Lanczos and the
 * adjoint solve require spd = 1 (they return COLA_ERR_INVALID_ARG otherwise). */
cola_status cola_linop_set_spd(cola_linop* op, int spd);

/* Reuse of prepared copies.  Every call converts the leaves it uses into the
 * working precision (FP32 / FP64 copies, BF16 split images of Kronecker
 * factors for MIXED), by default anew on each call, so that changes to the
 * borrowed data are always seen.  cola_linop_cache_prepared(op, 1) lets the
 * leaf op keep those copies across calls; the caller then reports a change
 * of its data with cola_linop_touch (on the leaf, or on any node: every leaf
 * below it counts as changed).  The Python binding sets the cache on the
 * leaves it creates and touches a leaf whenever its tensor's version counter
 * moved.  No counterpart in the paper. */
cola_status cola_linop_cache_prepared(cola_linop* op, int32_t on);
cola_status cola_linop_touch(cola_linop* op);

cola_status cola_linop_shape(const cola_linop* op, int64_t* rows, int64_t* cols);

/* Leaves in tree order (depth first, left to right; App. B.2 flatten).
 * kind is a cola_leaf_kind; rows x cols is the shape of the leaf's
 * parameter array (SCALAR: 1 x 1, DIAG: n x 1, LOWRANK: n x k for U). */
cola_status cola_linop_num_leaves(const cola_linop* op, int* n);
cola_status cola_linop_leaf_info(const cola_linop* op, int index, int* kind, int64_t* rows,
                                 int64_t* cols);

/* Drop the caller's reference; the node is freed when no parent holds it. */
cola_status cola_linop_release(cola_linop* op);

/* --------------------------------------------------------------------- MVM */

/* Y = A X for nrhs vectors (Sec. 3.1).  X is [nrhs][cols], Y is [nrhs][rows],
 * both FP64 for COLA_PREC_F64 and FP32 otherwise.  Asynchronous on stream.
 * A tensor-core kernel that gave up waiting (COLA_ERR_TIMEOUT, MIXED only) is
 * reported by a later call on the same context: the next cola_matvec once the
 * device has passed this one, or any call that synchronises (solves). */
cola_status cola_matvec(cola_ctx* ctx, const cola_linop* op, const void* X, void* Y,
                        int64_t nrhs, cola_precision precision, cola_stream stream);

/* -------------------------------------------------------------- CG solves */

typedef struct {
  double tol;                   /* target ||b - A x||_2 / ||b||_2 for EVERY right-hand side */
  int64_t maxiter;              /* cap on CG iterations (all chunks together) */
  int32_t precision;            /* cola_precision of MVM + recurrence */
  int32_t refine;               /* F32/MIXED: 1 = FP64 solution and FP64 true residual
                                   b - A x replacing the recursive one (reliable updates) */
  double reliable_delta;        /* replace the residual once the recursive residual norm fell
                                   by this factor since the last replacement (e.g. 0.1) */
  int32_t max_updates;          /* cap on FP64 residual replacements */
  int32_t split_factor_terms;   /* MIXED: BF16 terms per Kronecker-factor entry, 1..3 */
  int32_t split_vector_terms;   /* MIXED: BF16 terms per vector entry, 1..3 */
  int32_t graph_chunk;          /* iterations per CUDA-graph replay between host checks */
  int32_t jacobi;               /* 1 = Jacobi preconditioner M = Diag(A) from the Diag rules */
  int32_t x0_given;             /* 1 = X holds the initial guess, 0 = start from x = 0 */
  int32_t kron_precond;         /* 1 = for A = c_k K + c_d Diag(d), K a Kronecker product
                                   K_1 (x) ... (x) K_d or sum K_1 (+) ... (+) K_d of
                                   symmetric dense factors, precondition with
                                   M = c_k K + c_d mean(d) I, applied exactly from the
                                   factors' eigendecompositions (Table 3 Inverse / Eigs of
                                   Kron and KronSum; Sec. 3.2 composition).  Needs M
                                   positive definite; exclusive with jacobi; another operator
                                   shape is COLA_ERR_UNSUPPORTED.  Graph chunks are capped at
                                   8 iterations. */
  int32_t reorth_residuals;     /* > 0: CG with re-orthogonalised residuals, the
                                   low-precision CG variant Sec. 3.4 / App. C.3 cite
                                   (Maddox, Potapczynski & Wilson 2022): every new residual
                                   is made orthogonal, by two classical Gram-Schmidt passes,
                                   to the residuals stored so far (up to this many per
                                   right-hand side, 1 .. 4096; later ones are projected but
                                   not stored) before it enters beta and the next direction.
                                   Workspace reorth_residuals x nrhs x N vector elements.
                                   Unpreconditioned, without FP64 refinement (refine = 0 for
                                   F32 / MIXED); COLA_ERR_INVALID_ARG otherwise.  0 = off. */
} cola_cg_opts;

typedef struct {
  int64_t iterations;           /* CG iterations this right-hand side took (iterations it sat
                                   paused, waiting at the end of a graph chunk for an FP64
                                   residual replacement, are not counted) */
  double rel_residual;          /* final relative residual (FP64 true residual when refined
                                   or precision F64; recursive one otherwise) */
  int32_t updates;              /* FP64 residual replacements performed */
  int32_t status;               /* cola_status of this right-hand side */
} cola_cg_info;

/* Fill opts with defaults: tol 1e-8, maxiter 100000, MIXED, refine 1,
 * reliable_delta 0.1, max_updates 200, split terms 3 (factor) / 3 (vector),
 * graph_chunk 64,
 * jacobi 0, x0_given 0, kron_precond 0, reorth_residuals 0. */
void cola_cg_opts_default(cola_cg_opts* opts);

/* Solve A X = B for nrhs right-hand sides by (preconditioned) conjugate
 * gradients (Table 5 PSD base case), stopping when every right-hand side
 * reaches opts->tol (the all-solves rule of App. D GP training).
 * B, X are [nrhs][N]: FP64 when precision is F64 or refine = 1, FP32 else.
 * info (HOST, nrhs entries, may be NULL) receives per-RHS results.
 * Synchronous.  Returns COLA_ERR_NOT_CONVERGED / COLA_ERR_BREAKDOWN with X
 * written as far as it got. */
cola_status cola_cg_solve(cola_ctx* ctx, const cola_linop* op, const void* B, void* X,
                          int64_t nrhs, const cola_cg_opts* opts, cola_cg_info* info,
                          cola_stream stream);

/* Many independent SPD systems in one call: system s is ops[s] with
 * nrhs[s] right-hand sides B[s], X[s] (HOST arrays of device pointers, same
 * dtype rule as cola_cg_solve).  The systems advance together through
 * batched kernels driven by integer work tables (system, tile) that the
 * host builds once; converged systems retire from the tables.  info is HOST,
 * sum(nrhs) entries in system order.  Synchronous. */
cola_status cola_cg_solve_batched(cola_ctx* ctx, int32_t nsys, const cola_linop* const* ops,
                                  const void* const* B, void* const* X, const int64_t* nrhs,
                                  const cola_cg_opts* opts, cola_cg_info* info,
                                  cola_stream stream);

/* ------------------------------------------- Kronecker eigen-structured path */

/* X = A^-1 B directly, for A = c_k (K_1 (x) ... (x) K_d) [+ c_d s I] with
 * square symmetric dense factors and a scalar shift (the operator as built by
 * cola_linop_kron, optionally summed with cola_linop_diag of a scalar): the
 * eigenvectors of a Kronecker product are the Kronecker product of the factor
 * eigenvectors and its eigenvalues the products of the factor eigenvalues
 * (Table 3, Inverse and Eigs rules), so
 *   X = ((x)_k V_k) diag(1 / (c_k prod_k lambda_k + c_d s)) ((x)_k V_k)^T B.
 * A Kronecker sum K_1 (+) ... (+) K_d (cola_linop_kronsum) in place of the
 * product is accepted too: same eigenvectors, eigenvalues sum_k lambda_k.
 * Each factor's eigendecomposition is computed on the host in FP64
 * (cola_sym_eig) on first use and cached on the factor; it is recomputed when
 * the factor's contents change (the factor is read back to compare).
 * B, X: [nrhs][N], FP64 for COLA_PREC_F64 (FP64 mode products) and FP32 for
 * COLA_PREC_F32 (FP32 mode products, eigenvalue scaling in FP64).
 * COLA_ERR_UNSUPPORTED for any other operator shape (a per-element diagonal
 * is not diagonalised by the factor eigenvectors); COLA_ERR_INVALID_ARG for
 * a factor that is not symmetric.  Synchronous on first use of a factor,
 * asynchronous on stream afterwards. */
cola_status cola_kron_eig_solve(cola_ctx* ctx, const cola_linop* op, const void* B, void* X,
                                int64_t nrhs, cola_precision prec, cola_stream stream);

/* Exact log det A for the same operator class: the sum over all N index
 * tuples of log(c_k prod_k lambda_k[i_k] + c_d s) (sum_k for a Kronecker sum)
 * (Table 3 LogDet rule with the
 * Eigs rule; App. A.1.2), reduced in FP64 in a fixed order.
 * COLA_ERR_BREAKDOWN if any eigenvalue of A is <= 0.  Synchronous. */
cola_status cola_kron_eig_logdet(cola_ctx* ctx, const cola_linop* op, double* logdet,
                                 cola_stream stream);

/* Eigendecomposition of A = c_k (K_1 (x) ... (x) K_d) [+ c_d s I] (or of a
 * Kronecker sum of the K_k) in Kronecker form, without forming A (Table 3
 * Eigs rule; App. A.1.2): A = Q diag(lambda) Q^T with Q = V_1 (x) ... (x) V_d,
 * K_k = V_k diag(w_k) V_k^T, and lambda at flat index (i_1..i_d) equal to
 * c_k prod_k w_k[i_k] + c_d s (c_k sum_k w_k[i_k] + c_d s for a Kronecker sum),
 * so column (i_1..i_d) of Q is the Kronecker product of the columns i_k of
 * the V_k.  Same operator class and factor decompositions (cached, FP64) as
 * cola_kron_eig_solve.  Outputs, each a DEVICE FP64 array or NULL (at least
 * one given): factor_evals, the w_k concatenated (sum_k n_k entries);
 * factor_evecs, the V_k concatenated (sum_k n_k^2 entries, each n_k x n_k
 * row-major with column j the unit eigenvector of w_k[j]); evals, the N
 * eigenvalues lambda of A in flat index order.  COLA_ERR_UNSUPPORTED for
 * another operator shape, COLA_ERR_INVALID_ARG for a non-symmetric factor,
 * COLA_ERR_NOT_CONVERGED if a factor's QR iteration did not converge.
 * Synchronous on first use of a factor, asynchronous on stream afterwards. */
cola_status cola_kron_eigs(cola_ctx* ctx, const cola_linop* op, double* factor_evals,
                           double* factor_evecs, double* evals, cola_stream stream);

/* Solve A X = B for A = A_1 A_2 ... A_m (cola_linop_product; nested products
 * are flattened) by splitting the product: X = A_m^-1 ( ... (A_1^-1 B)), one
 * factor at a time (Sec. 3.2: the inverse of a product is the product of the
 * inverses in reverse order; Table 3 dispatch).  Each factor is solved by the
 * rule its type allows: a diagonal factor is divided out; with use_structure
 * = 1 a Kron / KronSum [+ scalar * I] factor takes the eigen-structured direct
 * solve of cola_kron_eig_solve; every other factor must be annotated spd and
 * is solved by cola_cg_solve's CG with opts (x0_given ignored).  An operator
 * that is not a product is one factor.  opts->tol applies to each factor's CG:
 * the product's own residual can exceed it by up to the condition number of
 * the leading factors, while the forward error stays of the order a single
 * CG on the product at tol would reach.  B, X are [nrhs][N], FP64 when
 * precision is F64 or refine = 1, FP32 else.  info (HOST, nrhs entries, may
 * be NULL): iterations and updates summed over the factors' CG solves,
 * rel_residual = ||B - A X|| / ||B|| of the whole product computed through
 * the product's MVM in the vectors' precision, status the first factor
 * failure.  COLA_ERR_UNSUPPORTED for a factor no rule covers, COLA_ERR_SHAPE
 * for a non-square factor.  Synchronous.  The paper's illustration is the
 * Bi-Poisson operator (L (+) L)^2 as a product of two Kronecker sums. */
cola_status cola_product_solve(cola_ctx* ctx, const cola_linop* op, const void* B, void* X,
                               int64_t nrhs, const cola_cg_opts* opts, int32_t use_structure,
                               cola_cg_info* info, cola_stream stream);

/* The global tile table of one table-driven batched mode step, as
 * cola_cg_solve_batched builds it (HOST arrays, no device work; the
 * integer launch plan of the batched solve, no counterpart in the paper).
 * Problem i has output width n_out[i], rest[i] rows per right-hand side and
 * nrhs[i] right-hand sides; a tile is 128 consecutive rows of one right-hand
 * side times one output chunk, the output width being padded to a multiple of
 * 16 and split into the fewest equal chunks of at most chunk_cap (64 or 128)
 * columns.  first[i] (nprob entries) receives the first global tile of
 * problem i, tile_prob[t] (capacity entries) the problem of tile t, *total
 * the number of tiles (written even when capacity is too small, which is
 * COLA_ERR_INVALID_ARG). */
cola_status cola_batch_tile_table(int32_t nprob, const int32_t* n_out, const int64_t* rest,
                                  const int64_t* nrhs, int32_t chunk_cap, int64_t* first,
                                  int32_t* tile_prob, int64_t capacity, int64_t* total);

/* Symmetric eigendecomposition of an n x n matrix in HOST memory, the routine
 * the two calls above apply to each factor: A = V diag(w) V^T with V's
 * column j the unit eigenvector of w[j].  Householder tridiagonalisation and
 * implicit symmetric QR with Wilkinson shifts, FP64 (Golub & Van Loan 8.3).
 * A (row-major, symmetric) is read only; V (n x n row-major) and w (n) are
 * written.  COLA_ERR_NOT_CONVERGED if the QR sweeps did not converge within
 * 60 n iterations.  Needs no GPU. */
cola_status cola_sym_eig(int64_t n, const double* A, double* V, double* w);

/* --------------------------------------------------------- Lanczos / SLQ */

/* m steps of symmetric Lanczos from q_0 = Q0[v] / ||Q0[v]|| for nvec starting
 * vectors at once (Table 5 self-adjoint base case; stop rule as the Arnoldi
 * breakdown test of Algorithm 1).  Q0 is [nvec][N] (FP64 for F64 precision,
 * FP32 else).  alpha [nvec][m] and beta [nvec][m] are FP64 device arrays;
 * row v holds alpha_0..alpha_{m_eff-1} and beta_0..beta_{m_eff-2}.  m_eff
 * [nvec] (int32, device) is where vector v stopped: breakdown at
 * beta_j <= 1e-10 (F64) / 1e-6 (F32) times max|alpha| truncates it (not an
 * error).  reorth = 1 adds full reorthogonalisation (stores all q: nvec*m*N
 * elements of workspace); reorth = 2 builds the basis from Householder
 * reflectors instead (cola_arnoldi_householder; alpha_j = H_jj, beta_j =
 * |H_j+1,j|; nvec*(m+1)*N elements of workspace, m <= 255).  With
 * COLA_PREC_MIXED the Kronecker contractions use the BF16 split terms set by
 * cola_set_split_terms (factor and vector terms), as cola_matvec does.
 * Asynchronous. */
cola_status cola_lanczos(cola_ctx* ctx, const cola_linop* op, const void* Q0, int64_t nvec,
                         int32_t m, int32_t precision, int32_t reorth, double* alpha,
                         double* beta, int32_t* m_eff, cola_stream stream);

/* Householder Arnoldi iteration (Algorithm 2) for nvec starting vectors Q0
 * ([nvec][N], FP64 for F64 precision, FP32 else) at once, m steps each (1 <=
 * m <= 255, m < N): reflectors R_j = I - 2 u_j u_j^T with u_j zero above
 * index j map the tail of nu_j onto e_j, q_j = R_0 ... R_j e_j and
 * nu_{j+1} = R_j ... R_0 A q_j, so the basis is orthogonal to working
 * precision (the low-precision-robust variant of App. C.3).  H (device FP64,
 * [nvec][m+1][m] row-major) receives the Hessenberg matrix with
 * A Q[:, :m] = Q H.  The reflector takes the cancellation-free sign (Golub &
 * Van Loan 5.1.2), so H equals Algorithm 2's up to a +-1 diagonal similarity
 * (diagonal and eigenvalues identical, off-diagonal signs may differ).
 * m_eff (device int32 [nvec]): columns computed before the new sub-diagonal
 * fell to 1e-10 (F64) / 1e-6 (else) times max|H_ii|.  Any square operator
 * (the symmetric case is Lanczos: cola_lanczos with reorth = 2).  Workspace
 * nvec*(m+1)*N vector elements.  Asynchronous. */
cola_status cola_arnoldi_householder(cola_ctx* ctx, const cola_linop* op, const void* Q0,
                                     int64_t nvec, int32_t m, int32_t precision, double* H,
                                     int32_t* m_eff, cola_stream stream);

/* Stochastic estimate of Diag(A) and Tr(A) (Sec. 3.3; App. B.1).  Base
 * (doubly = 0, or op not a Sum node): Hutchinson's estimator
 *   Diag(A) ~ (1/n) sum_v z_v (.) A z_v  over n = nprobes Rademacher probes.
 * Doubly stochastic (doubly = 1 and op a Sum node A = sum_i c_i A_i): each
 * term draws its own probes,
 *   Diag(A) ~ sum_i c_i (1/n) sum_v z_iv (.) A_i z_iv,
 * which drops the cross terms between summands from the variance.  Probe
 * entry (term i, probe v, index k) = sign of the top bit of SplitMix64 output
 * (i n + v) N + k of the stream seeded with `seed` (term 0 for the base
 * estimator), as cola_rademacher draws it.  MVMs run in `precision` (MIXED:
 * the tensor-core path for Kronecker terms, with the context's split terms);
 * the estimate accumulates in FP64.  diag: device FP64 [N] or NULL; trace:
 * HOST double (the sum of the diagonal estimate) or NULL; at least one must
 * be given.  Synchronous when trace is requested, asynchronous otherwise. */
cola_status cola_diag_estimate(cola_ctx* ctx, const cola_linop* op, int32_t nprobes,
                               uint64_t seed, int32_t doubly, int32_t precision, double* diag,
                               double* trace, cola_stream stream);

/* Stochastic Lanczos quadrature for log det A = Tr(log A) (App. A.2):
 * nprobes Rademacher probes z_v drawn on the device from `seed` (entry
 * (v, i) = sign of the top bit of SplitMix64 output v*N + i), or taken from
 * `probes` ([nprobes][N], same dtype as cola_lanczos's Q0) when it is not
 * NULL; m Lanczos steps each (cola_lanczos, MIXED with the context's split
 * terms); per probe ||z||^2 sum_k S_0k^2 log(theta_k) from the
 * eigendecomposition of T_m (implicit symmetric tridiagonal QR, FP64, on the
 * host's cores: a few KB come back from the device).
 * logdet, std_err are HOST doubles (mean over probes, sample standard error);
 * per_probe (device FP64 [nprobes]) may be NULL.  A Ritz value <= 0 (low
 * precision) is clamped to the smallest positive one; the count of clamps is
 * written to *clamped (HOST, may be NULL).  COLA_ERR_NOT_CONVERGED if the QR
 * iteration of a tridiagonal matrix did not converge.  Synchronous. */
cola_status cola_slq_logdet(cola_ctx* ctx, const cola_linop* op, int32_t nprobes, int32_t m,
                            uint64_t seed, const void* probes, int32_t precision,
                            int32_t reorth, double* logdet, double* std_err,
                            double* per_probe, int32_t* clamped, cola_stream stream);

/* ------------------------------------------------------------- gradients */

/* Leaf gradients of the weighted bilinear form sum_r w_r u_r^T A x_r
 * (App. B.2): for every leaf theta, grads[l] (+)= sum_r w_r u_r^T (dA/dtheta) x_r
 * in the leaf's shape and dtype (DENSE rows x cols, DIAG n, SCALAR 1,
 * LOWRANK n x k for U).  U is [nrhs][rows], X is [nrhs][cols] (FP64 for F64
 * precision, FP32 else); weights is a HOST array (NULL = ones).  grads is a
 * HOST array of num_leaves device pointers; a NULL entry skips that leaf.
 * accumulate = 0 overwrites.  Asynchronous. */
cola_status cola_bilinear_grad(cola_ctx* ctx, const cola_linop* op, const void* U,
                               const void* X, const double* weights, int64_t nrhs,
                               int32_t precision, void* const* grads, int32_t accumulate,
                               cola_stream stream);

/* Backward of X = A^-1 B (App. B.2 rule 1):  gradB = A^-T gradX (a second CG
 * solve with the same kernels; A is SPD so A^T = A) and, per leaf,
 * grads[l] = - sum_r (A^-T gradX_r)^T (dA/dtheta) X_r.  X, gradX, gradB follow
 * the dtype rule of cola_cg_solve; no Krylov iterate of the forward solve is
 * needed.  info as in cola_cg_solve for the adjoint solve.  Synchronous. */
cola_status cola_solve_backward(cola_ctx* ctx, const cola_linop* op, const void* X,
                                const void* gradX, void* gradB, int64_t nrhs,
                                void* const* grads, const cola_cg_opts* opts,
                                cola_cg_info* info, cola_stream stream);

/* Log-det gradient d log det A / dtheta = Tr(A^-1 dA/dtheta) (App. B.2 rule 4)
 * by Hutchinson probes (App. B.1):
 * grads[l] (+)= scale / nprobes * sum_k (A^-1 z_k)^T (dA/dtheta) z_k.
 * Z is [nprobes][N]; AinvZ holds A^-1 Z from an earlier block solve or is
 * NULL to solve here with opts.  Same dtype rule as cola_cg_solve.
 * accumulate = 0 overwrites.  Synchronous. */
cola_status cola_logdet_backward(cola_ctx* ctx, const cola_linop* op, const void* Z,
                                 const void* AinvZ, int64_t nprobes, double scale,
                                 void* const* grads, int32_t accumulate,
                                 const cola_cg_opts* opts, cola_stream stream);

/* GP training objective (Sec. 4 GP application; App. D GP training):
 *   L = 1/2 y^T A^-1 y + 1/2 log det A.
 * Solves the block [y, z_1 .. z_m] (1 + nprobes right-hand sides) with opts
 * in one CG call (the probes share the solve, App. D), takes y^T A^-1 y from
 * the first solution (FP64 reduction) and log det A by SLQ (App. A.2) on the
 * same probes Z with slq_steps Lanczos steps, and returns L in *value.
 * y [N], Z [nprobes][N] and Sol [1 + nprobes][N] (written: A^-1 [y, Z]) follow
 * the dtype rule of cola_cg_solve (FP64 when precision is F64 or refine = 1,
 * FP32 else).  value, logdet, logdet_se: HOST doubles (the last two may be
 * NULL); info: HOST, 1 + nprobes entries, may be NULL.  Returns the solve's
 * status (COLA_ERR_NOT_CONVERGED with everything still written).  Synchronous. */
cola_status cola_gp_objective(cola_ctx* ctx, const cola_linop* op, const void* y, const void* Z,
                              int64_t nprobes, int32_t slq_steps, const cola_cg_opts* opts,
                              void* Sol, double* value, double* logdet, double* logdet_se,
                              cola_cg_info* info, cola_stream stream);

/* Backward of cola_gp_objective scaled by g = dLoss/dL (App. B.2 rules 1 and
 * 4 with the Hutchinson trace of App. B.1): for every leaf theta,
 *   grads[l] = g (-1/2 a^T (dA/dtheta) a + 1/2 (1/m) sum_k u_k^T (dA/dtheta) z_k),
 * a = Sol[0], u_k = Sol[k] (m = nprobes), in the leaf's shape and dtype, and
 * grad_y = g a.  Sol and Z are FP64 for precision F64 and FP32 for F32 (the
 * contraction precision; FP64 keeps the cancelling lengthscale terms exact).
 * grads: HOST array of num_leaves device pointers (NULL entries, or grads
 * NULL, skip leaves); grad_y: device [N] or NULL.  Asynchronous. */
cola_status cola_gp_objective_backward(cola_ctx* ctx, const cola_linop* op, const void* Sol,
                                       const void* Z, int64_t nprobes, double g,
                                       int32_t precision, void* const* grads, void* grad_y,
                                       cola_stream stream);

/* ------------------------------------------------------------- utilities */

/* Fill out [count] (device, FP64 or FP32 by dtype) with Rademacher signs of
 * SplitMix64 outputs offset .. offset+count-1 of `seed` (the probe
 * generator of cola_slq_logdet).  Asynchronous. */
cola_status cola_rademacher(cola_ctx* ctx, uint64_t seed, int64_t offset, int64_t count,
                            void* out, cola_dtype dtype, cola_stream stream);

/* BF16 terms per Kronecker-factor entry and per vector entry (1..3) used by
 * cola_matvec, cola_lanczos, cola_slq_logdet, cola_diag_estimate and
 * cola_arnoldi_householder with COLA_PREC_MIXED (the CG solvers take theirs
 * from cola_cg_opts and leave this setting unchanged).  Default 2 / 2. */
cola_status cola_set_split_terms(cola_ctx* ctx, int32_t factor_terms, int32_t vector_terms);

/* Allocation-free Kronecker MVM (no counterpart in the paper; it exists for
 * callers that cannot let a library allocate device memory: a framework that
 * owns every byte of the device through its own pool, code running where an
 * allocation would implicitly synchronise the device, or a caller that has no
 * cola_ctx).  Computes Y = (K_1 (x) ... (x) K_d) X in FP32 exactly like
 * cola_matvec with COLA_PREC_F32 on a Kronecker node.
 *   rows[k], cols[k] (HOST): shape of factor k; factors[k] (HOST array of
 *   device pointers): factor k, FP32, row-major, packed (ld = cols[k]).
 *   X [nrhs][prod cols], Y [nrhs][prod rows]: FP32 device, must not alias.
 * The intermediate mode products live in one fixed device array inside the
 * library, 2 x 4 Mi floats (32 MiB), which every GPU that loads the library
 * holds until the process exits; nrhs times the largest intermediate must not
 * exceed 4 Mi floats, else COLA_ERR_INVALID_ARG.  The call allocates nothing:
 * no cudaMalloc, cudaFree or allocating library routine.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with the
 * current device; make that first call before any stream capture.  Every call
 * shares the array, so calls that overlap on the GPU (other streams, other
 * host threads) race; order them on one stream.  Asynchronous on stream. */
cola_status cola_kron_matvec_noalloc(int nfactors, const int64_t* rows, const int64_t* cols,
                                     const float* const* factors, const float* X, float* Y,
                                     int64_t nrhs, cola_stream stream);

/* Test hook of the failure path (no counterpart in the paper).  The next
 * tensor-core Kronecker launch of this context (a mode step of an MVM or of
 * a batched solve) that is not being captured into a CUDA graph has its MMA
 * role first wait on a barrier that nothing
 * completes, with a limit of wait_ns nanoseconds (1 .. 2e9; 0 disarms) in
 * place of the usual 2 s.  When the limit runs out the launch takes the
 * ordinary time-out path: every role of every CTA stops, each CTA waits for
 * its own bulk copies and MMAs, frees its tensor memory and exits, and the
 * device error flag reports COLA_ERR_TIMEOUT to the host (for cola_matvec on
 * a later call of the context, as documented there).  Nothing faults or
 * hangs; the context stays usable.  Used by the tests to exercise the path. */
cola_status cola_test_stall_next_launch(cola_ctx* ctx, int64_t wait_ns);

/* Number of kernels this library launched (or recorded into replayed graphs,
 * counted per replay) since the context was created. */
cola_status cola_kernel_launches(const cola_ctx* ctx, int64_t* count);

/* The context's internal launch stream (every kernel of this library runs on
 * it; calls join the caller's stream before and after, or not at all when the
 * caller passes this stream itself).  Exposed so that a caller can time
 * kernels with events on the stream they run on, or queue its own work on it.
 * No counterpart in the paper.  The stream is owned by the context and stays
 * valid until cola_destroy. */
cola_status cola_get_stream(const cola_ctx* ctx, cola_stream* stream);

#ifdef __cplusplus
}
#endif
#endif /* COLA_GB300_H */
