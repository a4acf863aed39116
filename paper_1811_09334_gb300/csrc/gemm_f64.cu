// FP64 products on the CUDA cores: C = alpha op(A) B (+ beta C).
//
// The FP64 form of the method's products (Algorithm 2.1 steps 2 and 4, the
// power steps, the Gram matrices and triangular solves of CholeskyQR and the
// assembly Q = V Q_B of step 7) all have one small dimension l <= 256.  On
// GB300 the FP64 pipe is the bound (about 1.25 TFLOP/s for the whole GPU),
// so the kernel is a plain register-tiled DFMA loop: a 64 x 64 output tile
// per CTA, 16-deep K slabs staged in shared memory, a 4 x 4 register tile
// per thread, and split-K over gridDim.z when the M x N tiles alone cannot
// fill the 152 SMs.  Split-K partial tiles go to a workspace and a second
// kernel sums them in a fixed order, so results are deterministic.
#include "kernels.cuh"

namespace rqk {

namespace {
constexpr int BM = 64, BK = 16, NT = 256, kMaxNC = 8;

template <typename TA>
__device__ __forceinline__ double ld_as_f64(const TA *p) { return static_cast<double>(*p); }

// op(A) is A (M x K, row-major, lda) or, with TRANS_A, A^T where A is K x M.
// B is K x N row-major (ldb).  The CTA tile is 64 x (16 NC): NC is picked per
// call so that the N-tiles cover N with little padding (l = 110 -> NC = 7,
// one 112-wide tile).  With part != nullptr the raw sums of K-slice z go to
// part + z * part_stride (M x N, ld N); otherwise C = alpha acc + beta C.
template <bool TRANS_A, typename TA, int NC>
__global__ void __launch_bounds__(NT)
k_gemm_f64(const TA *__restrict__ A, int64_t lda, const double *__restrict__ B, int64_t ldb,
           double *__restrict__ C, int64_t ldc, int64_t M, int64_t N, int64_t K, int64_t kchunk,
           double alpha, double beta, double *__restrict__ part, int64_t part_stride,
           const int *skip_unless) {
  constexpr int BN = 16 * NC;
  if (skip_unless && *reinterpret_cast<const volatile int *>(skip_unless) == 0) return;
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.x * BM, j0 = (int64_t)blockIdx.y * BN;
  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = min(K, kbeg + kchunk);
  double acc[4][NC];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[r][c] = 0.0;

  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    if (!TRANS_A) {
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        const int r = ty + 16 * rr;
        const int64_t i = i0 + r, k = k0 + tx;
        As[tx][r] = (i < M && k < kend) ? ld_as_f64(A + i * lda + k) : 0.0;
      }
    } else {
#pragma unroll
      for (int rr = 0; rr < 4; ++rr) {
        const int r = tid & 63, c = (tid >> 6) + 4 * rr;
        const int64_t i = i0 + r, k = k0 + c;
        As[c][r] = (i < M && k < kend) ? ld_as_f64(A + k * lda + i) : 0.0;
      }
    }
#pragma unroll
    for (int e = tid; e < BK * BN; e += NT) {
      const int kk = e / BN, jj = e - kk * BN;
      const int64_t j = j0 + jj, k = k0 + kk;
      Bs[kk][jj] = (j < N && k < kend) ? B[k * ldb + j] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double a[4], b[NC];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < NC; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t i = i0 + ty + 16 * r;
    if (i >= M) continue;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int64_t j = j0 + tx + 16 * c;
      if (j >= N) continue;
      if (part) {
        part[(int64_t)blockIdx.z * part_stride + i * N + j] = acc[r][c];
      } else {
        double v = alpha * acc[r][c];
        if (beta != 0.0) v = fma(beta, C[i * ldc + j], v);
        C[i * ldc + j] = v;
      }
    }
  }
}

// N-tiling: the fewest tiles of at most 128 columns, each 16 NC wide.
inline void n_tiling(int64_t N, int *nc, int64_t *ntiles) {
  int64_t t = (N + 16 * kMaxNC - 1) / (16 * kMaxNC);
  if (t < 1) t = 1;
  int64_t per = (N + t - 1) / t;
  int c = (int)((per + 15) / 16);
  if (c < 1) c = 1;
  if (c > kMaxNC) c = kMaxNC;
  *nc = c;
  *ntiles = (N + 16 * c - 1) / (16 * c);
}

// C[rowmap(i), j] = alpha * sum_z part[z][i][j] + beta * C[rowmap(i), j]
__global__ void k_reduce_parts(const double *__restrict__ part, int S, int64_t part_stride,
                               int64_t M, int64_t N, double *__restrict__ C, int64_t ldc,
                               double alpha, double beta, const int32_t *__restrict__ rowmap,
                               const int *skip_unless) {
  if (skip_unless && *reinterpret_cast<const volatile int *>(skip_unless) == 0) return;
  const int64_t total = M * N;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N, j = e - i * N;
    double s = 0.0;
    for (int z = 0; z < S; ++z) s += part[(int64_t)z * part_stride + e];
    const int64_t oi = rowmap ? (int64_t)rowmap[i] : i;
    if (oi < 0 || oi >= M) continue;  // an aborted pivoting kernel must not send writes astray
    double v = alpha * s;
    if (beta != 0.0) v = fma(beta, C[oi * ldc + j], v);
    C[oi * ldc + j] = v;
  }
}
// Small products (M N <= kSmallMN): four consecutive threads per entry of C
// split K among themselves (k = g, g + 4, ...) and combine with two shuffles.
// Every FP64 warp instruction costs ~64 clocks of an SM sub-partition here,
// so the work per warp, not the thread count, sets the time: an l x l x l
// product (l ~ 100) runs ~K/4 dependent FMAs per thread over ~200 CTAs.
// op(A)(i, k) = A[i lda + k] or, with TA, A[k lda + i]; op(B)(k, j) =
// B[k ldb + j] or, with TB, B[j ldb + k].
constexpr int64_t kSmallMN = 128 * 128;
template <bool TA, bool TB>
__global__ void __launch_bounds__(256)
k_gemm_small(const double *__restrict__ A, int64_t lda, const double *__restrict__ B, int64_t ldb,
             double *__restrict__ C, int64_t ldc, int64_t M, int64_t N, int64_t K, double alpha,
             double beta, const int *skip_unless) {
  if (skip_unless && *reinterpret_cast<const volatile int *>(skip_unless) == 0) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int g = (int)(t & 3);
  const int64_t e = t >> 2;
  const bool valid = e < M * N;
  const int64_t i = valid ? e / N : 0, j = valid ? e - i * N : 0;
  double s0 = 0.0, s1 = 0.0;
  if (valid) {
    int64_t k = g;
    for (; k + 4 < K; k += 8) {
      s0 = fma(TA ? A[k * lda + i] : A[i * lda + k], TB ? B[j * ldb + k] : B[k * ldb + j], s0);
      const int64_t k1 = k + 4;
      s1 = fma(TA ? A[k1 * lda + i] : A[i * lda + k1], TB ? B[j * ldb + k1] : B[k1 * ldb + j], s1);
    }
    if (k < K) s0 = fma(TA ? A[k * lda + i] : A[i * lda + k], TB ? B[j * ldb + k] : B[k * ldb + j], s0);
  }
  double s = s0 + s1;
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  if (valid && g == 0) {
    double v = alpha * s;
    if (beta != 0.0) v = fma(beta, C[i * ldc + j], v);
    C[i * ldc + j] = v;
  }
}
}  // namespace

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

int64_t gemm_f64_splits(int64_t M, int64_t N, int64_t K) {
  int nc;
  int64_t nt;
  n_tiling(N, &nc, &nt);
  const int64_t tiles = ((M + BM - 1) / BM) * nt;
  const int tt = tuning().gemm_target_ctas;
  const int64_t target = (tt > 0 && tt < 3 * num_sms()) ? tt : 3LL * num_sms();
  int64_t s = (target + tiles - 1) / tiles;
  const int64_t kmax = (K + 4 * BK - 1) / (4 * BK);  // keep >= 4 slabs per split
  if (s > kmax) s = kmax;
  if (s < 1) s = 1;
  if (s > 256) s = 256;
  return s;
}

size_t gemm_f64_part_bytes(int64_t M, int64_t N, int64_t K) {
  const int64_t s = gemm_f64_splits(M, N, K);
  return s > 1 ? (size_t)s * M * N * sizeof(double) : 0;
}

cudaError_t gemm_small(bool transA, bool transB, const double *A, int64_t lda, const double *B,
                       int64_t ldb, double *C, int64_t ldc, int64_t M, int64_t N, int64_t K,
                       double alpha, double beta, const int *skip_unless, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((4 * M * N + 255) / 256);
#define LAUNCH_SMALL(TA, TB)                                                                      \
  k_gemm_small<TA, TB><<<blocks, 256, 0, st>>>(A, lda, B, ldb, C, ldc, M, N, K, alpha, beta,     \
                                               skip_unless)
  if (transA) {
    if (transB) LAUNCH_SMALL(true, true); else LAUNCH_SMALL(true, false);
  } else {
    if (transB) LAUNCH_SMALL(false, true); else LAUNCH_SMALL(false, false);
  }
#undef LAUNCH_SMALL
  count_launch();
  return cudaGetLastError();
}

cudaError_t gemm_f64(bool transA, int a_dtype, const void *A, int64_t lda, const double *B,
                     int64_t ldb, double *C, int64_t ldc, int64_t M, int64_t N, int64_t K,
                     double alpha, double beta, double *part, const int32_t *rowmap,
                     const int *skip_unless, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (a_dtype == RQLP_F64 && rowmap == nullptr && M * N <= kSmallMN)
    return gemm_small(transA, false, reinterpret_cast<const double *>(A), lda, B, ldb, C, ldc, M,
                      N, K, alpha, beta, skip_unless, st);
  int64_t S = part ? gemm_f64_splits(M, N, K) : 1;
  const bool use_part = (S > 1) || (rowmap != nullptr);
  if (use_part && !part) return cudaErrorInvalidValue;
  int64_t kchunk = (K + S - 1) / S;
  kchunk = (kchunk + BK - 1) / BK * BK;
  if (kchunk <= 0) kchunk = BK;
  S = (K + kchunk - 1) / kchunk;
  if (S < 1) S = 1;
  int nc;
  int64_t ntiles;
  n_tiling(N, &nc, &ntiles);
  dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)ntiles, (unsigned)S);
  const int64_t pstride = M * N;
  double *p = use_part ? part : nullptr;
#define LAUNCH_NC(TR, T, NCV)                                                                    \
  k_gemm_f64<TR, T, NCV><<<grid, NT, 0, st>>>(reinterpret_cast<const T *>(A), lda, B, ldb, C,    \
                                              ldc, M, N, K, kchunk, alpha, beta, p, pstride,    \
                                              skip_unless)
#define LAUNCH(TR, T)                          \
  switch (nc) {                                \
    case 1: LAUNCH_NC(TR, T, 1); break;        \
    case 2: LAUNCH_NC(TR, T, 2); break;        \
    case 3: LAUNCH_NC(TR, T, 3); break;        \
    case 4: LAUNCH_NC(TR, T, 4); break;        \
    case 5: LAUNCH_NC(TR, T, 5); break;        \
    case 6: LAUNCH_NC(TR, T, 6); break;        \
    case 7: LAUNCH_NC(TR, T, 7); break;        \
    default: LAUNCH_NC(TR, T, 8); break;       \
  }
  if (a_dtype == RQLP_F32) {
    if (transA) { LAUNCH(true, float); } else { LAUNCH(false, float); }
  } else {
    if (transA) { LAUNCH(true, double); } else { LAUNCH(false, double); }
  }
#undef LAUNCH_NC
#undef LAUNCH
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (use_part) {
    const int64_t total = M * N;
    int blocks = (int)std::min<int64_t>((total + 255) / 256, 8LL * num_sms());
    if (blocks < 1) blocks = 1;
    k_reduce_parts<<<blocks, 256, 0, st>>>(part, (int)S, pstride, M, N, C, ldc, alpha, beta,
                                            rowmap, skip_unless);
    count_launch();
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace rqk
