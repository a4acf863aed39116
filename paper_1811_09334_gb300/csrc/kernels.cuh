// Host-side launchers shared by the translation units of the library.
#pragma once

#include <algorithm>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace rqk {

int num_sms();

// Launch-shape knobs.  The defaults fill the whole GPU with one problem; the
// batched driver lowers them so that many problems run side by side (the
// autotuner picks its values).  Workspace sizes are computed with the
// defaults, which are upper bounds of every tuned value.
struct Tuning {
  int gemm_target_ctas;  // FP64 GEMM: split K until about this many CTAs (0: 3 x SMs)
  int cpqr_max_ctas;     // CPQR of B: at most this many CTAs (0: one per SM; 1: one CTA, no waits on others)
  int mma_max_splits;    // tcgen05 products: at most this many K splits (0: fill the SMs)
  int chol_ctas;         // Cholesky of the Gram matrix: cluster of 16 or 8 CTAs, or 1 CTA
                         // (0: 16 where such a cluster fits, else 8)
  int no_digit_products; // 1: the FP64 Gram matrices and the assembly stay on the FP64 units
                         // (batches: a digit product takes a whole SM per CTA)
};
Tuning &tuning();

// Launch counter (every launcher adds its launches) and event timing of
// kernel classes (see prof.cu).
void count_launch(int n = 1);
long long launch_count();
enum ProfClass {
  kProfProducts = 0,  // products with A (sketch, power steps, projection)
  kProfCpqr = 1,      // column-pivoted QR of B
  kProfGram = 2,      // CholeskyQR: Gram matrices X^T X
  kProfChol = 3,      // CholeskyQR: Cholesky factors
  kProfTrinv = 4,     // CholeskyQR: triangular inverses
  kProfApply = 5,     // CholeskyQR: X R^{-1} and R products
  kProfSmall = 6,     // explicit Q0 from the reflectors
  kProfPrep = 7,      // precision preparation of A (mixed forms)
  kProfAssembly = 8,  // Q = V Q_B and P = Pi0 (Q1 ...), the final products
  kProfClasses = 9
};
int prof_start(int cls, cudaStream_t st);
void prof_stop(int cls, int idx, cudaStream_t st);

// Carves a workspace in 256-byte aligned pieces; with a null base it only
// measures.
struct Arena {
  char *base;
  size_t off = 0;
  explicit Arena(void *b) : base(reinterpret_cast<char *>(b)) {}
  template <class T>
  T *take(size_t count) {
    const size_t bytes = (count * sizeof(T) + 255) / 256 * 256;
    T *r = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += bytes;
    return r;
  }
};

// ---- api.cu: the side stream that runs Q0 beside the QR of R0^T ----------
// For recording one factorization into a graph: create the side stream of
// `st` now (outside a capture), and let rqlp() fork to it while `st` is
// being recorded (the fork and the join become branches of the graph).
void side_stream_prepare(cudaStream_t st);
void side_stream_in_capture(bool on);

// ---- gemm_f64.cu ---------------------------------------------------------
int64_t gemm_f64_splits(int64_t M, int64_t N, int64_t K);
size_t gemm_f64_part_bytes(int64_t M, int64_t N, int64_t K);
// C = alpha op(A) B + beta C; op(A) = A (M x K) or A^T (A is K x M).
// With rowmap, row i of the result goes to row rowmap[i] of C.  `part` is
// split-K scratch of gemm_f64_part_bytes(M, N, K) bytes (M * N doubles at
// least when rowmap is used).  skip_unless: the kernels return at once when
// *skip_unless == 0 (device-side conditional passes); may be null.
// C = alpha op(A) op(B) + beta C for small products (one thread per entry of C;
// meant for M N <= 16384), FP64
cudaError_t gemm_small(bool transA, bool transB, const double *A, int64_t lda, const double *B,
                       int64_t ldb, double *C, int64_t ldc, int64_t M, int64_t N, int64_t K,
                       double alpha, double beta, const int *skip_unless, cudaStream_t st);
cudaError_t gemm_f64(bool transA, int a_dtype, const void *A, int64_t lda, const double *B,
                     int64_t ldb, double *C, int64_t ldc, int64_t M, int64_t N, int64_t K,
                     double alpha, double beta, double *part, const int32_t *rowmap,
                     const int *skip_unless, cudaStream_t st);

// ---- dense_small.cu ------------------------------------------------------
// kernel attributes of the CholeskyQR kernels (call before any stream capture)
cudaError_t chol_init();
// Rinv = R^{-1} for upper triangular R (l x l, ld l).
cudaError_t trinv_upper(const double *R, int l, double *Rinv, const int *skip_unless,
                        cudaStream_t st);
// Y = X^T for an r x c matrix (ld ldx) into c x r (ld ldy).
cudaError_t transpose(const double *X, int64_t r, int64_t c, int64_t ldx, double *Y, int64_t ldy,
                      cudaStream_t st);
// Copy an r x c block (optionally only when *skip_unless != 0).
cudaError_t copy2d(const double *X, int64_t r, int64_t c, int64_t ldx, double *Y, int64_t ldy,
                   const int *skip_unless, cudaStream_t st);
// Fill an r x c block with the identity pattern (1 on the diagonal).
cudaError_t set_identity(double *X, int64_t r, int64_t c, int64_t ld, cudaStream_t st);
// Y[:, j] = X[:, perm[j]] for an r x c matrix.
cudaError_t gather_cols(const double *X, int64_t r, int64_t c, int64_t ldx, const int32_t *perm,
                        double *Y, int64_t ldy, cudaStream_t st);
// p[i] = i (a valid permutation, written before a pivoting kernel that may abort)
cudaError_t iota(int32_t *p, int64_t n, cudaStream_t st);
// S = tril(M) + tril(M, -1)^T for an l x l M (ld l)
cudaError_t copyltu(const double *M, int l, double *S, cudaStream_t st);
// Y[:, perm[j]] = X[:, j]
cudaError_t scatter_cols(const double *X, int64_t r, int64_t c, int64_t ldx, const int32_t *perm,
                         double *Y, int64_t ldy, cudaStream_t st);
// rows: Y[i] = X[perm[i]] (gather) or Y[perm[i]] = X[i] (scatter)
cudaError_t permute_rows(const double *X, int64_t r, int64_t c, int64_t ldx, const int32_t *perm,
                         double *Y, int64_t ldy, bool scatter, cudaStream_t st);
// X[i][j] = 0 for j > i (i < min(r, c))
cudaError_t mask_lower_trapezoid(double *X, int64_t r, int64_t c, int64_t ld, cudaStream_t st);
// Lvalues[i] = T[i][i]
cudaError_t diag_of(const double *T, int l, int64_t ldt, double *out, cudaStream_t st);
// Zero the strict lower (lower_zero = 1) or strict upper part of an l x l matrix.
cudaError_t zero_triangle(double *T, int l, int64_t ld, bool strict_lower, cudaStream_t st);
// Form Q = H_0 H_1 ... H_{t-1} [I; 0] (rows x t, ld ldq) from reflectors stored
// as columns of Vh (rows x t, ld ldv; v_s[s] = 1 implicit, zeros above) and tau.
cudaError_t form_q(const double *Vh, int64_t ldv, const double *tau, int64_t rows, int t,
                   double *Q, int64_t ldq, cudaStream_t st, double *scratch = nullptr);
// Row-vector triangular solves (one warp per vector, n <= kMaxL): y U = x, or
// with backward U y = x using only U's strictly upper part and U symmetric in
// storage; 1 / U_jj from dinv (length n) when given, else from U.
cudaError_t tri_rows(const double *U, int64_t ldu, const double *dinv, int n, const double *X,
                     int64_t ldx, double *Y, int64_t ldy, int nvec, bool backward,
                     cudaStream_t st);

// ---- cholqr.cu: one CholeskyQR pass on a rows x l panel -------------------
int64_t gram_chunks(int64_t rows);
int64_t gram_chunks_max(int64_t rows_max);  // >= gram_chunks(r) for every r <= rows_max
cudaError_t cholqr_init();  // kernel attributes, set before any stream capture
// unit roundoffs of the two CholeskyQR pass precisions
constexpr double kEpsF64 = 1.1102230246251565e-16;  // 2^-53
constexpr double kEpsF32 = 5.9604644775390625e-08;  // 2^-24
// G = X^T X (symmetric, l x l, ld l); part: gram_chunks(rows) * l * l doubles (at most
// gram_chunks_max of the largest rows).  lowp: X rounded to FP32, products in FP32
// over chunks of <= 32 rows, chunks summed in FP64 (error about kEpsF32 |X|^T |X|).
cudaError_t gram_sym(const double *X, int64_t rows, int l, int64_t ldx, double *part, double *G,
                     const int *skip_unless, cudaStream_t st, bool lowp = false);
// G = R^T R (R upper, ld l) with shifted retry; Dinv: inverses of R's 16 x 16
// diagonal blocks (block-diagonal, ld l).  eps: unit roundoff of the pass that
// formed G (breakdown threshold l 2 eps G_jj, shift of shifted CholeskyQR).
// again_tol >= 0: set ctrl->again_flag[site] (and done_flag = 1 - it) when
// eps cond(R)^2 > again_tol, i.e. when one pass leaves Q less orthonormal
// lowp: factor in FP32 on one CTA (the FP32 CholeskyQR pass; l <= 226)
// pack (may be null; f32_pack_floats(l) floats): written by the FP32
// factorization (lowp, l <= 128, again_tol < 0): R and the block inverses
// also in FP32, laid out as the FP32 solve stages them
cudaError_t chol_blocked(const double *G, int l, int64_t rows, double *R, double *Dinv, Ctrl *ctrl,
                         int site, const int *skip_unless, cudaStream_t st,
                         double again_tol = -1.0, double eps = kEpsF64, bool lowp = false,
                         float *pack = nullptr);
size_t f32_pack_floats(int l);
// Q = X R^{-1} by a blocked triangular solve (X and Q must not alias); lowp:
// the solve runs in FP32 (Q stored in FP64), staging R and the block
// inverses from `pack` (written by the FP32 Cholesky) when it is given
cudaError_t apply_trsm(const double *X, int64_t rows, int l, int64_t ldx, const double *R,
                       const double *Dinv, double *Q, int64_t ldq, const int *skip_unless,
                       cudaStream_t st, bool lowp = false, const float *pack = nullptr);

// ---- cpqr.cu ---------------------------------------------------------------
size_t cpqr_ws_bytes(int64_t n, int l);
// Scratch bytes cpqr_wide() touches when the column slabs fit in shared
// memory (*fits tells whether they do; otherwise a global slab is needed too).
size_t cpqr_scratch_bytes_smem_only(int64_t n, int l, bool *fits);
// Column-pivoted Householder QR of the l x n matrix whose columns are the
// rows of Bt (n x l, ld ldb).  Writes R0t (n x l, ld ldr), piv (n), the
// reflectors Vh (l x l, ld l) and tau (l).  Cooperative launch.  With
// fixed_piv (device, l entries) step s takes column fixed_piv[s] instead of
// the largest trailing norm: the unpivoted Householder QR of the permuted
// matrix; an index out of range or repeated sets RQLP_ERR_INVALID_ARG.
// max_ctas > 0: at most this many CTAs (one per SM otherwise), as long as
// the column slabs still fit in shared memory; the results do not depend on
// the grid.
cudaError_t cpqr_wide(const double *Bt, int64_t n, int l, int64_t ldb, double *R0t, int64_t ldr,
                      int32_t *piv, double *Vh, double *tau, void *scratch, Ctrl *ctrl,
                      unsigned long long limit_ns, unsigned debug_extra, cudaStream_t st,
                      const int32_t *fixed_piv = nullptr, int max_ctas = 0);
// The first `steps` pivot steps of the column-pivoted Householder QR of an
// L x n matrix (L <= 16384, steps <= 256) given as At = its transpose (n x L,
// ld ldat): R0t (n x steps, ld ldr) holds the first `steps` rows of R as
// columns (pivot order), piv (n) the column order, Vh (L x steps, ld ldv) and
// tau (steps) the reflectors.  Scratch: cpqr_tall_ws_bytes(n, L).
size_t cpqr_tall_ws_bytes(int64_t n, int64_t L);
cudaError_t cpqr_tall(const double *At, int64_t n, int64_t L, int steps, int64_t ldat, double *R0t,
                      int64_t ldr, int32_t *piv, double *Vh, int64_t ldv, double *tau,
                      void *scratch, Ctrl *ctrl, unsigned long long limit_ns, cudaStream_t st);

}  // namespace rqk
