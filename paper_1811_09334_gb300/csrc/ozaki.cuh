// FP64-accurate products on the BF16 tensor cores (ozaki.cu).
#pragma once

#include "kernels.cuh"

namespace rqk {

// An FP64 operand row of K values is written as kOzDigits BF16 "digits" of
// at most 8 significant bits relative to a power-of-two row scale 2^e
// (|x| < 2^e):  x = 2^e (d_0 2^-7 + d_1 2^-15 + ... + d_5 2^-47) + r with
// |d_i| <= 128 and |r| <= 2^(e - 48).  A product of two digits is an integer
// of at most 2^14, so up to 1024 of them add up exactly in the tensor
// cores' FP32 accumulator.
constexpr int kOzDigits = 6;
constexpr int kOzCopies = 2;  // Y operands also hold digit j times 2^-8

// Digits of one operand: [kOzDigits x copies][rows][ld] BF16 (plane
// i * copies + m holds digit i times 2^(-8m)), and the row exponents e
// (int32, rows).  An X operand needs copies = 1 (or reads the unscaled
// planes of a Y operand's arrays), a Y operand copies = kOzCopies.
struct OzOperand {
  void *digits;
  int32_t *exps;
  int64_t rows, K, ld;
  int copies;
};

// Bytes of the digit arrays of a rows x K operand.
size_t oz_operand_bytes(int64_t rows, int64_t K, int copies);
// Carves an operand's arrays from a workspace (ld = K rounded up to 8).
OzOperand oz_carve(Arena &a, int64_t rows, int64_t K, int copies);
// FP32 partial sums oz_gemm needs for C of M x N with K terms.
size_t oz_part_floats(int64_t M, int N, int64_t K);

// Digits of an FP64 (dtype RQLP_F64) or FP32 (RQLP_F32) matrix S stored
// r x c with leading dimension ld: trans = false makes the operand rows the
// rows of S (K = c), trans = true the columns of S (K = r).  Writes
// op.digits / op.exps with op.copies planes per digit.  Non-finite data
// records RQLP_ERR_NONFINITE.  skip: as in the other kernels (the launches
// return at once when *skip == 0); may be null.
int oz_split(const void *S, int dtype, int64_t r, int64_t c, int64_t ld, bool trans,
             const OzOperand &op, Ctrl *ctrl, const int *skip, cudaStream_t st);

// The digits of the rows and of the columns of S (r x c, ld) at once (two
// reads of S: exponents, then digits): rows.rows = r, rows.K = c, cols.rows =
// c, cols.K = r, copies 1.
int oz_split_both(const void *S, int dtype, int64_t r, int64_t c, int64_t ld,
                  const OzOperand &rows, const OzOperand &cols, Ctrl *ctrl, cudaStream_t st);

// C (M x N, FP64, ldc) = X Y^T with X (M x K) and Y (N x K) given as digits,
// to about 2^-47 relative to the row scales (every digit pair of weight
// 2^-40 or more of the leading pair; the four leading weight groups are
// summed exactly).  With rowmap, row i goes to row rowmap[i] of C.  part:
// oz_part_floats(M, N, K) floats.  N <= 128.
int oz_gemm(const OzOperand &X, const OzOperand &Y, int64_t M, int N, int64_t K, double *C,
            int64_t ldc, const int32_t *rowmap, float *part, int64_t part_floats, Ctrl *ctrl,
            int64_t spin_ns, const int *skip, cudaStream_t st);

int ozaki_init();

}  // namespace rqk
