// Mixed-precision products with A on the tcgen05 tensor cores.
#pragma once

#include "kernels.cuh"
#include "ozaki.cuh"

namespace rqk {

// Device buffers of the mixed-precision path (all null for RQLP_PREC_FP64).
struct MixedBufs {
  void *Ahi, *Alo;    // m x n BF16 split of A (row-major)
  void *Athi, *Atlo;  // n x m BF16 split of A^T (row-major)
  void *Whi, *Wlo;    // l_pad x max(m, n) BF16 split of a transposed skinny operand
  float *part;        // split-K FP32 partial sums
  int64_t part_floats;
  // E4M3 form: A row-scaled, A^T column-scaled, skinny operand column-scaled
  float *sA, *sAt, *sW, *rmax;
  unsigned *cmax;
  // FP64TC form: digits of A's rows and columns, of the skinny operand, and
  // the partial sums of the digit products
  OzOperand oA, oAt, oW;
  float *opart;
  int64_t opart_floats;
  int64_t m, n;
  int l;
};

// One-time set-up (driver entry point, kernel attributes) done before any
// stream capture.
int mixed_init();
void carve_mixed(Arena &a, int64_t m, int64_t n, int l, int prec, MixedBufs &mx);
// Splits A (and A^T) into BF16 pairs once per factorization.
int mixed_prepare_A(const MixedBufs &mx, int prec, const void *A, int a_dtype, int64_t m, int64_t n,
                    int64_t lda, Ctrl *ctrl, cudaStream_t st);
// Y (m x l, ld l, FP64) = A W with W n x l (ld ldw, FP64).
int mixed_nn(const MixedBufs &mx, int prec, int64_t m, int64_t n, const double *W, int64_t ldw,
             int l, double *Y, Ctrl *ctrl, int64_t spin_ns, cudaStream_t st);
// Z (n x l, ld l, FP64) = A^T V with V m x l (ld ldv, FP64).
int mixed_tn(const MixedBufs &mx, int prec, int64_t m, int64_t n, const double *V, int64_t ldv,
             int l, double *Z, Ctrl *ctrl, int64_t spin_ns, cudaStream_t st);

}  // namespace rqk
