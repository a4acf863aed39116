/*
 * rqlp.h - C ABI of the GB300 (sm_103a) randomized QLP library.
 *
 * The library computes the randomized QLP factorization A ~= Q L P^T of
 * Wu & Xiang, "Randomized QLP algorithm and error analysis" (arXiv
 * 1811.09334): RQLP (Algorithm 2.1), the enhanced ERQLP with d inner QR
 * iterations (Algorithm 2.2) and the blocked BRQLP (Algorithm 4.1), plus
 * q power steps Y = (A A^T)^q A Omega in the range finder.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrices are dense, row-major, with an explicit leading dimension
 *   (ld >= number of columns), FP64 unless stated.
 * - l = k + p is the sketch width; 1 <= l <= min(m, n) and l <= 256.
 * - All pointers are DEVICE pointers except in rqlp_host() and
 *   rqlp_host_async().  The caller owns every buffer, including the
 *   workspace; the library never allocates device memory.  Buffers must not
 *   overlap unless stated.
 * - Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL is
 *   the legacy default stream); rqlp_host(), rqlp_read_status() and
 *   rqlp_brqlp_tol() synchronize it.  Argument errors are returned at once
 *   and enqueue nothing.  Errors found on the device (non-finite data, a
 *   device-side wait that ran out of time) are written to a status word in
 *   the workspace; read it with rqlp_read_status() after the work is done.
 * - Every QR inside returns R with a non-negative diagonal, so Q, L and P
 *   are unique for full-rank inputs.  Column pivoting compares exact
 *   trailing column norms; exact ties go to the lowest original column
 *   index; columns never chosen as pivots keep their original order.
 * - Workspaces may be reused between calls on the same stream; two calls
 *   that run concurrently need two workspaces.
 */
#ifndef RQLP_H
#define RQLP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *rqlp_stream_t; /* a cudaStream_t */

/* Status codes.  Negative: error (outputs are invalid).  Positive: warning
 * (outputs are valid). */
typedef enum {
  RQLP_OK = 0,
  RQLP_WARN_SHIFTED_CHOLQR = 1,  /* a Gram matrix was numerically singular; a shifted CholeskyQR pass was added */
  RQLP_ERR_INVALID_ARG = -1,     /* bad size, pointer, leading dimension or option */
  RQLP_ERR_NONFINITE = -2,       /* NaN or Inf met in A, Omega or an intermediate */
  RQLP_ERR_RANK_DEFICIENT = -3,  /* a Gram matrix stayed singular after the shift */
  RQLP_ERR_TIMEOUT = -4,         /* a device-side wait gave up (see spin_limit_ns) */
  RQLP_ERR_CUDA = -5,            /* a CUDA runtime call failed */
  RQLP_ERR_WORKSPACE = -6,       /* workspace too small or misaligned (needs 256-byte alignment) */
  RQLP_ERR_UNSUPPORTED = -7      /* option combination not supported */
} rqlp_status;

/* Precision of the products with A (sketch, power steps, projection).
 * The QR factorizations and the QLP of B always run in FP64. */
typedef enum {
  RQLP_PREC_FP64 = 0,   /* FP64 CUDA-core products (A in FP64 or FP32) */
  RQLP_PREC_BF16X3 = 1, /* tcgen05 BF16 tensor cores, split A = Ah + Al and W = Wh + Wl,
                           three products Ah Wh + Ah Wl + Al Wh accumulated in FP32 */
  RQLP_PREC_BF16 = 2,   /* tcgen05 BF16 tensor cores, one product, FP32 accumulation */
  RQLP_PREC_FP8 = 3,    /* tcgen05 E4M3 tensor cores, one product, FP32 accumulation; A scaled
                           by a power of two per row (per column for the A^T products) and the
                           skinny operand per column, the scales divided out in FP64 */
  RQLP_PREC_TF32X3 = 4, /* tcgen05 TF32 tensor cores (10-bit significands), split A = Ah + Al
                           and W = Wh + Wl into TF32 values (round to nearest), three products
                           Ah Wh + Ah Wl + Al Wh accumulated in FP32 over four rotating
                           accumulators: the pairs hold about 2^-22, the tensor cores'
                           accumulation (about 2^-24 per 8 values of K per accumulator)
                           dominates at large K (7e-6 normwise at K = 8192, BF16X3 1.5e-5);
                           twice the bytes of BF16X3 per pass over A */
  RQLP_PREC_TF32 = 5,   /* tcgen05 TF32 tensor cores, one product, FP32 accumulation */
  RQLP_PREC_FP64TC = 6  /* FP64 accuracy on the BF16 tensor cores: A and the skinny operand are
                           cut into six signed 8-bit digits per element against a power-of-two
                           scale per row (Ozaki-style exact splitting), the 21 digit products
                           of weight down to 2^-40 of the leading one are formed with tcgen05
                           (the three leading weight groups summed exactly), so a product is
                           FP64-accurate to about 2^-47 relative to the row scales; needs
                           k + p <= 128 */
} rqlp_prec;

/* Element type of A. */
typedef enum { RQLP_F64 = 0, RQLP_F32 = 1 } rqlp_dtype;

typedef struct {
  int32_t q;            /* power steps, q >= 0 (Y = (A A^T)^q A Omega, QR after every product) */
  int32_t d;            /* inner QR iterations of Algorithm 2.2, d >= 1 (used when pivot2 == 0) */
  int32_t pivot2;       /* 1: Algorithm 2.1, second QR column-pivoted; 0: Algorithm 2.2 */
  int32_t prec;         /* rqlp_prec */
  int32_t block_b;      /* 0: unblocked; b > 0: Algorithm 4.1 with blocks of b columns (b divides l) */
  int32_t debug_flags;  /* 0 in normal use; bit 0: the first grid-wide exchange of the pivoted QR
                           waits for an exchange number that never comes, so that it runs out of
                           time (tests of the timeout path) */
  int64_t spin_limit_ns;/* bound on every device-side wait in ns; 0 selects 2 s */
  int32_t fixed_pivots; /* 0: the column pivots are chosen (and written to piv0 / piv1);
                           1: piv0 (its first l entries) and, for Algorithm 2.1 (pivot2 = 1),
                           piv1 are INPUTS, and the two QRs take these columns in this order
                           (the unpivoted QR of B Pi0 and of R0^T Pi1): the factorization
                           at fixed pivots, on which the adjoint and finite differences at a
                           pivot change rely.  An index out of range or repeated gives the
                           device status RQLP_ERR_INVALID_ARG.  Not with block_b > 0. */
  int32_t truncate_k;   /* 0: outputs l wide; 1: the rank-k truncation (the abstract's rank-k
                           L): Q m x k, L k x k, P n x k and k L-values, each with ld k
                           (Q[:, :k], L[:k, :k], P[:, :k] of the l-wide factorization) */
  int32_t in_flight;    /* how many factorizations the caller keeps running at once, each on its
                           own stream with its own workspace (0 or 1: one at a time; read by
                           rqlp(), rqlp_host*(), rqlp_brqlp_tol() and rqlp_graph_create()).  With 2 or
                           more, the column-pivoted QR of B, whose CTAs spend most of each
                           pivot step waiting on the grid-wide exchange, runs on half of the
                           SMs and leaves the others to the kernels of the other
                           factorizations, and the FP64 Cholesky factorizations run on
                           clusters of 8 CTAs instead of 16 (easier to place beside other
                           kernels): a longer single factorization, more of them per second
                           overall.  The results are identical bit for bit. */
} rqlp_opts;

/* Human-readable name of a status code. */
const char *rqlp_status_string(int status);

/* Library ABI version (major * 100 + minor); 200 added fixed_pivots, truncate_k,
 * rqlp_rvalues() and the pivot arguments of rqlp_backward(); 201 added in_flight and
 * rqlp_graph_*. */
int rqlp_version(void);

/* Bytes of device workspace rqlp() needs for these sizes and options
 * (0 if the arguments are invalid). */
size_t rqlp_workspace_size(int64_t m, int64_t n, int32_t k, int32_t p, const rqlp_opts *opts);

/*
 * Randomized QLP of A (Algorithms 2.1, 2.2 and 4.1; the problem statement of
 * Section 1, eq. 1.1).
 *
 *  A       [in]  m x n, element type a_dtype, leading dimension lda.
 *  Omega   [in]  n x l Gaussian sketch (FP64, ld ldo); the caller draws it so
 *                that other implementations can be fed the same sketch.
 *  Q       [out] m x l, column-orthonormal (ld l).
 *  L       [out] l x l middle factor (ld l): lower triangular, except for
 *                ERQLP with even d, where the exact middle factor of
 *                B = Q_B R(d) P_B^T is upper triangular.  BRQLP: blkdiag(L_j).
 *  P       [out] n x l (ld l); column-orthonormal (within each block for BRQLP).
 *  Lvalues [out] l values diag(L) (>= 0); may be NULL.
 *  piv0    [out] n int32 column pivots of the CPQR of B (position i holds the
 *                original column index); may be NULL.  BRQLP: first block.
 *                [in] with opts->fixed_pivots: l entries, required.
 *  piv1    [out] l int32 pivots of the second CPQR (identity for ERQLP); may be NULL.
 *                [in] with opts->fixed_pivots and pivot2 = 1: l entries, required.
 *  ws      [in]  device workspace of ws_bytes >= rqlp_workspace_size(), 256-byte aligned.
 * With opts->truncate_k, Q, L, P and Lvalues are k wide (ld k).
 * Returns RQLP_OK once the work is enqueued, or an argument error.
 */
int rqlp(const void *A, int32_t a_dtype, int64_t m, int64_t n, int64_t lda, int32_t k, int32_t p,
         const double *Omega, int64_t ldo, const rqlp_opts *opts, double *Q, double *L, double *P,
         double *Lvalues, int32_t *piv0, int32_t *piv1, void *ws, size_t ws_bytes,
         rqlp_stream_t stream);

/*
 * Fixed-accuracy BRQLP: the blocks of Algorithm 4.1 (b columns each) are
 * added until the relative residual ||A - V V^T A||_F / ||A||_F is at most
 * `tol`, evaluated through eq. 2.1 as ||A||_F^2 - ||B||_F^2 with B = V^T A
 * the stacked B_j, or until l_max columns (the blocked scheme's use for an
 * unknown rank, which the paper's conclusion names).  Omega is n x l_max
 * (ldo >= l_max); the workspace is rqlp_workspace_size(m, n, l_max, 0, opts)
 * with opts->block_b = b; opts->q must be 0 (no power steps in Algorithm
 * 4.1).  *l_used gets the number of columns used, a multiple of b; Q (m x
 * l_max), P (n x l_max) and L (l_max x l_max, zero outside the used blocks)
 * hold the factorization in their first *l_used columns (of L: its leading
 * *l_used x *l_used block), Lvalues (may be NULL) its first *l_used
 * L-values, piv0 (n) the first block's column pivots and piv1 (l_max) the
 * per-block second-stage pivots.  The stopping test is taken on the host
 * after every block, so this call synchronizes `stream` once per block and
 * returns the final status (argument, CUDA or device status).
 */
int rqlp_brqlp_tol(const void *A, int32_t a_dtype, int64_t m, int64_t n, int64_t lda, int32_t b,
                   int32_t l_max, double tol, const double *Omega, int64_t ldo,
                   const rqlp_opts *opts, double *Q, double *L, double *P, double *Lvalues,
                   int32_t *piv0, int32_t *piv1, int32_t *l_used, void *ws, size_t ws_bytes,
                   rqlp_stream_t stream);

/* The R-values of the last rqlp() call that used `ws` with these sizes and
 * options: diag R0 (>= 0) of the column-pivoted QR of B (Algorithm 2.1 step 5),
 * which Section 5 (Figures 1-2) sets beside the L-values as the cruder
 * estimate of the singular values; for BRQLP the R-values of each block's
 * B_j in block order.  Copies l values (k with truncate_k) to the device
 * array Rvalues, enqueued on `stream` after that call. */
int rqlp_rvalues(const void *ws, int64_t m, int64_t n, int32_t k, int32_t p, const rqlp_opts *opts,
                 double *Rvalues, rqlp_stream_t stream);

/* Synchronizes `stream` and returns the device status word of the last call
 * that used `ws` (RQLP_OK, a warning or an error). */
int rqlp_read_status(const void *ws, rqlp_stream_t stream);

/* Bytes of device workspace rqlp_host() needs (inputs and outputs are staged in it). */
size_t rqlp_host_workspace_size(int64_t m, int64_t n, int32_t k, int32_t p, const rqlp_opts *opts,
                                int32_t a_dtype);

/*
 * rqlp() on HOST buffers: copies A (m x n, dense, lda = n) and Omega (n x l)
 * to the device workspace, factors, copies Q, L, P, Lvalues, piv0, piv1 back
 * and synchronizes the stream.  Host buffers should be page-locked for full
 * copy speed.  With opts->fixed_pivots piv0 / piv1 are host inputs (copied in,
 * not back); with opts->truncate_k the outputs are k wide.  Returns the final
 * status (argument, CUDA or device status).
 */
int rqlp_host(const void *A_host, int32_t a_dtype, int64_t m, int64_t n, int32_t k, int32_t p,
              const double *Omega_host, const rqlp_opts *opts, double *Q_host, double *L_host,
              double *P_host, double *Lvalues_host, int32_t *piv0_host, int32_t *piv1_host,
              void *ws, size_t ws_bytes, rqlp_stream_t stream);

/*
 * rqlp_host() without the final synchronization: enqueues the copies in,
 * the factorization and the copies out on `stream` and returns at once
 * (RQLP_OK, or an argument or CUDA error found while enqueueing).  The host
 * buffers must stay valid and untouched until the stream has finished;
 * rqlp_read_status(ws, stream) then gives the device status.  Calls with
 * their own workspaces and streams overlap one problem's copies with
 * another's factorization (double buffering across a sequence of problems).
 */
int rqlp_host_async(const void *A_host, int32_t a_dtype, int64_t m, int64_t n, int32_t k,
                    int32_t p, const double *Omega_host, const rqlp_opts *opts, double *Q_host,
                    double *L_host, double *P_host, double *Lvalues_host, int32_t *piv0_host,
                    int32_t *piv1_host, void *ws, size_t ws_bytes, rqlp_stream_t stream);

/* ------------------------------------------------------------------------
 * Stage entry points (each one a step of Algorithm 2.1 / 2.2).  They use the
 * same workspace rules; rqlp_stage_workspace_size() covers all of them.
 * ---------------------------------------------------------------------- */
size_t rqlp_stage_workspace_size(int64_t rows, int64_t cols, int32_t l, int32_t prec);

/* Y = A W (Algorithm 2.1, step 2 with W = Omega; also the second half of a
 * power step).  A m x n (a_dtype, lda), W n x l (ldw), Y m x l (ldy). */
int rqlp_sketch(const void *A, int32_t a_dtype, int64_t m, int64_t n, int64_t lda, const double *W,
                int64_t ldw, int32_t l, int32_t prec, double *Y, int64_t ldy, void *ws,
                size_t ws_bytes, rqlp_stream_t stream);

/* Z = A^T V (n x l, ldz), i.e. B^T for B = V^T A (Algorithm 2.1, step 4;
 * also the first half of a power step).  A m x n, V m x l (ldv). */
int rqlp_project(const void *A, int32_t a_dtype, int64_t m, int64_t n, int64_t lda, const double *V,
                 int64_t ldv, int32_t l, int32_t prec, double *Z, int64_t ldz, void *ws,
                 size_t ws_bytes, rqlp_stream_t stream);

/* Thin QR X = Qx R of a rows x l matrix (Algorithm 2.1, step 3) by
 * CholeskyQR2 in FP64, with a shifted first pass and a third pass when a
 * Gram matrix is numerically singular.  X is read (ldx); Qx (rows x l, ldq)
 * and, if R != NULL, R (l x l upper, ld l, non-negative diagonal) are written. */
int rqlp_orth(const double *X, int64_t rows, int32_t l, int64_t ldx, double *Qx, int64_t ldq,
              double *R, void *ws, size_t ws_bytes, rqlp_stream_t stream);

/* Column-pivoted Householder QR of the l x n matrix B (Algorithm 2.1, step 5),
 * B given as Bt = B^T (n x l row-major, ld ldb; each row one column of B).
 * Writes R0t = R0^T (n x l, ld l; row i is column i of R0 in pivot order),
 * piv0 (n) and Q0 (l x l, ld l) with B[:, piv0] = Q0 R0. */
int rqlp_cpqr(const double *Bt, int64_t n, int32_t l, int64_t ldb, double *R0t, int32_t *piv0,
              double *Q0, void *ws, size_t ws_bytes, rqlp_stream_t stream);

/* ------------------------------------------------------------------------
 * Deterministic truncated pivoted QLP (the comparison method of Section 5).
 * ---------------------------------------------------------------------- */
/* Workspace of rqlp_qlp() (0 if invalid: needs 1 <= t <= min(m, n, 256),
 * m <= 16384). */
size_t rqlp_qlp_workspace_size(int64_t m, int64_t n, int32_t t, const rqlp_opts *opts);

/*
 * Stewart's pivoted QLP (Section 1, eq. 1.2) truncated at t steps, the
 * deterministic "QLP" of Section 5 and Tables 1-4: the first t steps of the
 * column-pivoted Householder QR of A, A Pi0 ~= Q0 R0 with R0 the first t rows
 * of R, then the QR of R0^T = Q1 R1 (unpivoted for opts->pivot2 = 0; with
 * opts->pivot2 = 1 pivoted on its t x t R factor as in Algorithm 2.1), so that
 * A ~= Q L P^T with L = R1^T lower triangular.  The column norms of A are
 * exact at every step like rqlp()'s; ties go to the lowest column index.
 *  A       [in]  m x n FP64 (a_dtype RQLP_F64), lda >= n; m <= 16384.
 *  Q       [out] m x t (ld t); L t x t (ld t); P n x t (ld t); Lvalues t (may
 *                be NULL); piv0 n and piv1 t (may be NULL).
 *  ws      [in]  device workspace of rqlp_qlp_workspace_size() bytes (holds a
 *                transposed copy of A).
 * Every step rewrites the trailing columns of A (a BLAS-2 sweep: t passes over
 * A), so it costs far more than rqlp() at the same t; it is the reference the
 * randomized methods are measured against.  Only opts->pivot2 and
 * opts->spin_limit_ns are read.  Returns RQLP_OK once enqueued, or an argument
 * error; device errors go to the status word (rqlp_read_status()).
 */
int rqlp_qlp(const void *A, int32_t a_dtype, int64_t m, int64_t n, int64_t lda, int32_t t,
             const rqlp_opts *opts, double *Q, double *L, double *P, double *Lvalues,
             int32_t *piv0, int32_t *piv1, void *ws, size_t ws_bytes, rqlp_stream_t stream);

/* ------------------------------------------------------------------------
 * Adjoint (reverse-mode derivative) of RQLP.  The paper has no derivative;
 * this differentiates Algorithm 2.1 (pivot2 = 1) with the column pivots held
 * fixed (they are piecewise constant in A).
 * ---------------------------------------------------------------------- */
/* Workspace of rqlp_backward() (0 if invalid; needs pivot2 = 1, block_b = 0,
 * truncate_k = 0). */
size_t rqlp_backward_workspace_size(int64_t m, int64_t n, int32_t k, int32_t p,
                                    const rqlp_opts *opts);

/* dA = J^T (dQ, dL, dP): the vector-Jacobian product of A -> (Q, L, P) of
 * rqlp() at A with the same Omega and options.  dQ (m x l), dL (l x l), dP
 * (n x l) are FP64 device cotangents with ld l (NULL = zero); dA (m x n, FP64,
 * ld ldda) is written.  piv0 / piv1 (device, l int32 each, both or neither):
 * the pivots of the forward call, held fixed in the recomputed forward (the
 * derivative of the factorization at those pivots even where another column
 * order is as good); NULL recomputes them from A.  The forward is recomputed
 * inside (no other state is kept between rqlp() and this call); the sweep
 * runs in FP64. */
int rqlp_backward(const void *A, int32_t a_dtype, int64_t m, int64_t n, int64_t lda, int32_t k,
                  int32_t p, const double *Omega, int64_t ldo, const rqlp_opts *opts,
                  const int32_t *piv0, const int32_t *piv1, const double *dQ, const double *dL,
                  const double *dP, double *dA, int64_t ldda, void *ws, size_t ws_bytes,
                  rqlp_stream_t stream);

/* ------------------------------------------------------------------------
 * Batched factorizations: many independent problems in one graph launch.
 * ---------------------------------------------------------------------- */
/* One problem of a batch: the arguments of rqlp() (device pointers). */
typedef struct {
  const void *A;
  int32_t a_dtype;
  int32_t k;
  int64_t m, n, lda;
  int32_t p;
  int32_t reserved;
  const double *Omega;
  int64_t ldo;
  double *Q, *L, *P, *Lvalues;
  int32_t *piv0, *piv1;
} rqlp_problem;

/* How a batch runs (0 selects a default) and its launch shapes.
 *
 * engine: RQLP_BATCH_PERSISTENT (one persistent kernel: one CTA per SM takes
 * (problem, stage, tile) work items from an ordered device list, waiting for
 * each item's previous stage on per-problem counters with a bounded poll),
 * RQLP_BATCH_GRAPH (every problem's kernels recorded into one CUDA graph over
 * parallel branches), or RQLP_BATCH_AUTO (0: the persistent kernel where it
 * supports the batch, else the graph).  The persistent kernel supports the
 * FP64 and BF16x3 forms with l = k + p <= 128, n <= 6000, d <= 4 (d = 1 with
 * pivot2), no given pivots and no truncation.
 * For the graph engine: parallel branches (problems in flight), CTAs the FP64
 * products aim for, K splits of the tensor-core products.  The autotuner of
 * the Python package picks the engine and the shapes per batch shape. */
enum { RQLP_BATCH_AUTO = 0, RQLP_BATCH_GRAPH = 1, RQLP_BATCH_PERSISTENT = 2 };
typedef struct {
  int32_t branches;
  int32_t gemm_target_ctas;
  int32_t mma_max_splits;
  int32_t engine;
} rqlp_batch_tuning;

typedef struct rqlp_batch *rqlp_batch_t;

/* Device workspace of a batch: the graph engine needs one rqlp() workspace
 * per branch, the persistent engine every problem's buffers at once (plus its
 * work-item tables), both a per-problem status array; 0 if a problem or the
 * options are invalid (block_b must be 0: BRQLP is not batched) or the
 * requested engine does not support them. */
size_t rqlp_batched_workspace_size(const rqlp_problem *probs, int32_t count, const rqlp_opts *opts,
                                   const rqlp_batch_tuning *tune);

/* Prepares the factorizations of all `count` problems (Algorithms 2.1 / 2.2
 * with the options in `opts`) as one CUDA graph and instantiates it.  Graph
 * engine: every problem's kernels over tune->branches parallel streams, with
 * small launch shapes so that many fit on the GPU at once.  Persistent
 * engine: one zeroing node and one kernel node; the work-item list, the
 * problem and stage tables and the tensor maps are written into the
 * workspace here (synchronous copies).  Results are those of rqlp() on each
 * problem (the persistent engine's l x l QRs are Householder QRs, equal to
 * rqlp()'s up to rounding).  Not thread-safe with other calls of this library
 * on the same host thread while it records.  The problem table is read during
 * this call only. */
int rqlp_batched_create(const rqlp_problem *probs, int32_t count, const rqlp_opts *opts,
                        const rqlp_batch_tuning *tune, void *ws, size_t ws_bytes,
                        rqlp_batch_t *plan);

/* Runs the whole batch: one cudaGraphLaunch on `stream`. */
int rqlp_batched_launch(rqlp_batch_t plan, rqlp_stream_t stream);

/* Synchronizes `stream`, writes each problem's status to statuses[count] (may
 * be NULL) and returns the first error, else the first warning, else RQLP_OK. */
int rqlp_batched_status(rqlp_batch_t plan, rqlp_stream_t stream, int32_t *statuses);

/* Number of kernel nodes in the batch's graph (kernels per launch). */
int rqlp_batched_kernel_nodes(rqlp_batch_t plan);

/* The engine the batch runs on (RQLP_BATCH_GRAPH or RQLP_BATCH_PERSISTENT)
 * and, for the persistent engine, its work items per launch (else 0). */
int rqlp_batched_engine(rqlp_batch_t plan, int64_t *items);

/* Persistent engine only: where the last launch's CTA time went, per stage
 * kind (16 slots; 1 preparation of A, 2 split of Omega, 3 products with A,
 * 4 Gram tiles, 5 Cholesky, 6 solve tiles, 7 CPQR of B, 8 the l x l QLP
 * part, 9 assembly, 10 status): busy_us[k], the microseconds CTAs spent
 * running items of kind k, wait_us[k], the microseconds they spent taking
 * such items (the queue and the wait for the previous stage), both summed
 * over CTAs, and items[k], the items that ran (skipped conditional passes
 * not counted).  Any pointer may be NULL.  Synchronizes `stream`;
 * RQLP_ERR_INVALID_ARG for a graph-engine batch. */
int rqlp_batched_stage_times(rqlp_batch_t plan, rqlp_stream_t stream, double *busy_us,
                             double *wait_us, int64_t *items);

/* Frees the graph (not the workspace, which the caller owns). */
void rqlp_batched_destroy(rqlp_batch_t plan);

/* ------------------------------------------------------------------------
 * One factorization recorded once and replayed (a deployment feature the
 * paper has no counterpart for).  rqlp() enqueues about 110 kernels; a
 * replay of the recording is one CUDA graph launch.
 * ---------------------------------------------------------------------- */
typedef struct rqlp_graph *rqlp_graph_t;

/* Arguments as for rqlp(), plus *graph [out].  The call first runs rqlp()
 * once on `stream` (argument checks and one-time set-up; the outputs then
 * hold that factorization) and synchronizes `stream`, then records the same
 * call on a private stream into a graph.  The graph reads A, Omega (and the
 * given pivots) and writes the outputs and the workspace at the addresses
 * given here: to factor new data, write it to A (and Omega) in place and
 * launch again.  The workspace belongs to the graph while it exists (one
 * graph, or rqlp() call, at a time per workspace).  Returns rqlp()'s codes,
 * or RQLP_ERR_CUDA if the recording fails (*graph is then NULL). */
int rqlp_graph_create(const void *A, int32_t a_dtype, int64_t m, int64_t n, int64_t lda,
                      int32_t k, int32_t p, const double *Omega, int64_t ldo,
                      const rqlp_opts *opts, double *Q, double *L, double *P, double *Lvalues,
                      int32_t *piv0, int32_t *piv1, void *ws, size_t ws_bytes,
                      rqlp_stream_t stream, rqlp_graph_t *graph);

/* Enqueues one replay on `stream` (any stream; replays of one graph must not
 * overlap).  The device status is read with rqlp_read_status(ws, stream). */
int rqlp_graph_launch(rqlp_graph_t graph, rqlp_stream_t stream);

/* Library kernels one replay runs (what rqlp_launch_count() adds per launch). */
int rqlp_graph_kernels(rqlp_graph_t graph);

/* Frees the graph (not the workspace or the outputs). */
void rqlp_graph_destroy(rqlp_graph_t graph);

/*
 * rqlp_cpqr() for callers that cannot allocate device memory.  The paper has
 * no counterpart.
 *
 * Who needs it: code that runs under another runtime's memory manager which
 * owns all of the device memory, or a latency-critical loop that must not call
 * cudaMalloc (it can synchronize the whole device), so it cannot pass a
 * workspace.  This entry point allocates nothing and calls no allocating
 * routine; its scratch (control block, reflectors, pivot tables) lives in one
 * fixed 2 MiB __device__ array inside the library, which every GPU that loads
 * the library holds until the process exits.
 *
 * Arguments as for rqlp_cpqr() (Bt n x l device input, R0t n x l, piv0 n and,
 * if not NULL, Q0 l x l device outputs).  With sync != 0 the call synchronizes
 * `stream` and returns the device status; with sync == 0 it returns after
 * enqueueing, and a device-side error (a timeout, non-finite data) is NOT
 * reported to the caller: the status word stays in the library's array and
 * the next call clears it.  Callers that need the status pass sync != 0.
 * Limits: the pivot tables plus l x l reflectors must fit the 2 MiB array and
 * each CTA's slab of columns must fit in shared memory (about
 * n * l * 8 bytes <= 152 * 190 KiB on GB300); larger sizes return
 * RQLP_ERR_WORKSPACE without touching the GPU.
 * The first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  Every call
 * shares the one array and clears its control block at the start, so calls
 * whose work overlaps on the GPU (other streams or threads) race: serialize them.
 */
int rqlp_cpqr_static(const double *Bt, int64_t n, int32_t l, int64_t ldb, double *R0t,
                     int32_t *piv0, double *Q0, int32_t sync, rqlp_stream_t stream);

/* ------------------------------------------------------------------------
 * Instrumentation.
 * ---------------------------------------------------------------------- */
/* Number of CUDA kernels this library has launched in this process. */
long long rqlp_launch_count(void);

/* Starts timing kernel classes: from now on rqlp() records a CUDA event pair
 * on its stream around (0) every product with A, (1) every column-pivoted QR
 * of B, and, inside every CholeskyQR pass, (2) the Gram matrix, (3) the
 * Cholesky factor, (4) the triangular inverse, (5) X R^{-1} with the R
 * update; (6) the explicit Q0 of the first CPQR; (7) the precision
 * preparation of A; (8) the final products Q = V Q_B and P. */
int rqlp_profile_begin(void);

/* Stops timing; waits for the recorded events and writes, per class c <
 * nclass, the summed device time in ms (ms[c]) and the number of timed
 * regions (count[c]).  Either array may be NULL. */
int rqlp_profile_end(double *ms, long long *count, int nclass);

/* ------------------------------------------------------------------------
 * Self-test of the device arithmetic helpers (a diagnostic; the paper has no
 * counterpart).  The kernels round FP64 to FP32 and back with integer
 * operations (a conversion instruction would occupy the scarce FP64 unit)
 * and take reciprocals and reciprocal square roots from an FP32 estimate
 * refined in FP64.  This entry point checks them on the device against
 * CUDA's own operations over `count` pseudo-random inputs each:
 *   fails[0]: FP64 -> FP32 round-to-nearest-even, bit-exact (inputs in the
 *             FP32 normal range);
 *   fails[1]: FP32 -> FP64, bit-exact (normal floats);
 *   fails[2]: reciprocal, relative error above 2^-51 (4 units of roundoff);
 *   fails[3]: reciprocal square root, relative error above 2^-51.
 * fails: host array of 4 ints, written on return (the call synchronizes the
 * stream).  count in [1, 2^24].  Returns RQLP_OK, RQLP_ERR_INVALID_ARG or
 * RQLP_ERR_CUDA.  Uses a 16-byte static device counter, so concurrent calls
 * race; serialize them.
 */
int rqlp_selftest(int32_t count, int32_t *fails, rqlp_stream_t stream);

/*
 * FP64 throughput probe (a diagnostic; the paper has no counterpart): enqueues
 * one kernel on `stream` whose threads (four 256-thread CTAs per SM) run eight
 * independent FP64 FMA chains of `iters` steps each, so that it is bound by
 * the FP64 units alone.  *flops (host) gets the flop count of the launch
 * (2 per FMA); time the launch with CUDA events on `stream` to measure the
 * GPU's FP64 rate, the denominator of the FP64 kernels' rooflines.  sink: one
 * device double, written only in a case that never arises.  Returns at once.
 */
int rqlp_fp64_probe(int32_t iters, double *sink, double *flops, rqlp_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* RQLP_H */
