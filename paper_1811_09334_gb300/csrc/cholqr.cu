// CholeskyQR pass kernels for a tall-skinny X (rows x l, l <= 256), FP64.
//
// One pass of CholeskyQR (Algorithm 2.1 step 3 and every re-orthonormalization)
// is   G = X^T X,   G = R^T R,   Q = X R^{-1}.
// On GB300 FP64 runs at about 2 FMAs per clock per SM, so each piece is shaped
// for FP64 work and few barriers:
//   k_gram_sym      each CTA forms the upper triangle of X_c^T X_c for a chunk
//                   of 32 rows (4 x 4 register tiles of the triangle); a second
//                   kernel sums the chunks in a fixed order (deterministic) and
//                   mirrors the triangle.  Half the FMAs of a full product.
//   k_chol_blocked  one CTA, right-looking over columns with the work of each
//                   column spread over every warp (a warp-wide FP64
//                   instruction holds an SMSP's FP64 pipe for many cycles, so
//                   single-warp FP64 work is slow here); warp 0 updates the
//                   next diagonal entry first and takes its reciprocal square
//                   root while the others update the trailing triangle.  It
//                   also writes the inverses of R's 16 x 16 diagonal blocks.
//   k_apply_trsm    Q = X R^{-1} as a blocked triangular solve on 32-row tiles:
//                   Q[:, b] = (X[:, b] - Q[:, <b] R[<b, b]) inv(R[b, b]); half
//                   the FMAs of multiplying by a full inverse, and no separate
//                   triangular inversion.
#include <cmath>

#include "kernels.cuh"

namespace rqk {

namespace {

constexpr double kEps = 1.1102230246251565e-16;
constexpr int kB = 16;       // block size of the Cholesky and the solve
constexpr int kGramRows = 32;
constexpr int kGramThreads = 256;

// Upper triangle of X_c^T X_c for the rows of chunk c = blockIdx.x, into
// part[c] (l x l, only j >= i written).  Tiles of 4 x 4 over the triangle.
__global__ void __launch_bounds__(kGramThreads)
k_gram_sym(const double *__restrict__ X, int64_t rows, int l, int64_t ldx,
           double *__restrict__ part, const int *skip_unless) {
  if (skip_unless && *reinterpret_cast<const volatile int *>(skip_unless) == 0) return;
  extern __shared__ double xs[];  // [kGramRows][lp]
  const int lp = ((l + 3) / 4) * 4 + 1;
  const int64_t r0 = (int64_t)blockIdx.x * kGramRows;
  const int nr = (int)min((int64_t)kGramRows, rows - r0);
  for (int e = threadIdx.x; e < kGramRows * lp; e += blockDim.x) {
    const int r = e / lp, c = e - r * lp;
    xs[e] = (r < nr && c < l) ? X[(r0 + r) * ldx + c] : 0.0;
  }
  __syncthreads();
  const int nb = (l + 3) / 4;
  const int ntiles = nb * (nb + 1) / 2;
  double *out = part + (int64_t)blockIdx.x * l * l;
  for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
    // tile t -> (bi, bj), bi <= bj, row-major over the upper triangle
    int bi = 0, rem = t;
    while (rem >= nb - bi) {
      rem -= nb - bi;
      ++bi;
    }
    const int bj = bi + rem;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int r = 0; r < kGramRows; ++r) {
      const double *row = xs + r * lp;
      double x[4], y[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) x[a] = row[4 * bi + a];
#pragma unroll
      for (int b = 0; b < 4; ++b) y[b] = row[4 * bj + b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(x[a], y[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = 4 * bi + a;
      if (i >= l) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int j = 4 * bj + b;
        if (j < l && j >= i) out[(int64_t)i * l + j] = acc[a][b];
      }
    }
  }
}

// G[i][j] = G[j][i] = sum_c part[c][i][j] for i <= j
__global__ void k_gram_reduce(const double *__restrict__ part, int chunks, int l,
                              double *__restrict__ G, const int *skip_unless) {
  if (skip_unless && *reinterpret_cast<const volatile int *>(skip_unless) == 0) return;
  const int64_t ll = (int64_t)l * l;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ll;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / l), j = (int)(e - (int64_t)i * l);
    if (j < i) continue;
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += part[(int64_t)c * ll + e];
    G[(int64_t)i * l + j] = s;
    G[(int64_t)j * l + i] = s;
  }
}

// Upper Cholesky G = R^T R with 16-column blocks, breakdown detection and one
// shifted retry (shifted CholeskyQR, Fukaya et al. 2020), as k_chol_upper in
// dense_small.cu.  Also writes Dinv: the inverses of R's 16 x 16 diagonal
// blocks (block-diagonal l x l, ld l).
__global__ void __launch_bounds__(512)
k_chol_blocked(const double *__restrict__ G, int l, double rows, double *__restrict__ R,
               double *__restrict__ Dinv, Ctrl *ctrl, int site, const int *skip_unless,
               int use_smem, double again_tol) {
  if (skip_unless && *reinterpret_cast<const volatile int *>(skip_unless) == 0) return;
  extern __shared__ double sm[];
  __shared__ double red[32];
  __shared__ double s_gdiag[kMaxL];
  __shared__ double s_next;
  __shared__ int s_fail;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  double *W = use_smem ? sm : R;
  double tr = 0.0;
  for (int i = tid; i < l; i += blockDim.x) tr += G[(int64_t)i * l + i];
  tr = block_sum(tr, red);
  int fail = 0;
  for (int attempt = 0; attempt < 2; ++attempt) {
    const double shift = attempt ? 11.0 * (rows * l + (double)l * (l + 1)) * kEps * tr : 0.0;
    for (int e = tid; e < l * l; e += blockDim.x) {
      const int i = e / l, j = e - i * l;
      W[e] = G[e] + (i == j ? shift : 0.0);
    }
    for (int i = tid; i < l; i += blockDim.x) s_gdiag[i] = G[(int64_t)i * l + i] + shift;
    if (tid == 0) s_fail = 0;
    __syncthreads();
    // right-looking, one column per step, spread over every warp; warp 0
    // updates the next diagonal entry first and takes its reciprocal square
    // root while the other warps update the rest of the trailing triangle
    if (tid == 0) {
      const double d = W[0];
      const double g0 = s_gdiag[0];
      int f = 0;
      if (!isfinite(d) || !isfinite(g0)) f = 2;
      else if (!(d > (double)l * 2.0 * kEps * g0) || !(d > 0.0)) f = 1;
      s_fail = f;
      s_next = f ? 1.0 : rsqrt(d);
    }
    __syncthreads();
    for (int j = 0; j < l && !s_fail; ++j) {
      const double rs = s_next;
      double *Wj = W + j * l;  // l <= 256: 32-bit offsets
      const double d = Wj[j];
      __syncthreads();
      for (int c = j + 1 + tid; c < l; c += blockDim.x) Wj[c] *= rs;
      if (tid == 0) Wj[j] = d * rs;
      __syncthreads();
      if (warp == 0) {
        if (j + 1 < l) {
          double *W1 = W + (j + 1) * l;
          const double r1 = Wj[j + 1];
          if (lane == 0) {
            const double dn = W1[j + 1] - r1 * r1;
            W1[j + 1] = dn;
            const double g0 = s_gdiag[j + 1];
            int f = 0;
            if (!isfinite(dn) || !isfinite(g0)) f = 2;
            else if (!(dn > (double)l * 2.0 * kEps * g0) || !(dn > 0.0)) f = 1;
            if (f) s_fail = f;
            s_next = f ? 1.0 : rsqrt(dn);
          }
          // the rest of row j + 1 of the trailing triangle
          for (int c = j + 2 + lane; c < l; c += 32) W1[c] = fma(-r1, Wj[c], W1[c]);
        }
      } else {
        for (int a = j + 2 + (warp - 1); a < l; a += nw - 1) {
          const double ra = Wj[a];
          double *Wa = W + a * l;
          int c = a + lane;
          for (; c + 32 < l; c += 64) {
            const double x0 = fma(-ra, Wj[c], Wa[c]);
            const double x1 = fma(-ra, Wj[c + 32], Wa[c + 32]);
            Wa[c] = x0;
            Wa[c + 32] = x1;
          }
          if (c < l) Wa[c] = fma(-ra, Wj[c], Wa[c]);
        }
      }
      __syncthreads();
    }
    __syncthreads();
    fail = s_fail;
    __syncthreads();
    if (fail == 0 || fail == 2) break;
    if (attempt == 0 && tid == 0) {
      ctrl->shift_flag[site] = 1;
      set_status(ctrl, RQLP_WARN_SHIFTED_CHOLQR);
    }
  }
  if (fail == 2) {
    if (tid == 0) set_status(ctrl, RQLP_ERR_NONFINITE);
  } else if (fail == 1) {
    if (tid == 0) set_status(ctrl, RQLP_ERR_RANK_DEFICIENT);
  }
  __syncthreads();
  for (int e = tid; e < l * l; e += blockDim.x) {
    const int i = e / l, j = e - i * l;
    R[e] = (j >= i) ? W[e] : 0.0;
  }
  __syncthreads();
  // a second pass is needed when eps * cond(R)^2, the loss of orthogonality
  // of one CholeskyQR pass, exceeds again_tol (cond estimated from diag(R))
  if (again_tol >= 0.0 && warp == 0) {
    double mx = 0.0, mn = 1e300;
    for (int i = lane; i < l; i += 32) {
      const double d = R[(int64_t)i * l + i];
      mx = fmax(mx, d);
      mn = fmin(mn, d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    }
    if (lane == 0) {
      const double c = (mn > 0.0) ? mx / mn : 1e300;
      const int again = (fail != 0) || !(2.0 * kEps * c * c <= again_tol);
      ctrl->again_flag[site] = again;
      ctrl->done_flag[site] = 1 - again;
    }
  }
  // inverses of the diagonal blocks: one warp per block, lane = column
  const int nblk = (l + kB - 1) / kB;
  for (int bk = warp; bk < nblk; bk += nw) {
    const int c0 = bk * kB, bs = min(kB, l - c0);
    const int c = lane;  // column of the block inverse
    if (c < kB) {
      double x[kB];
#pragma unroll
      for (int i = 0; i < kB; ++i) x[i] = 0.0;
      if (c < bs) {
        const double *Rb = R + (int64_t)c0 * l + c0;
        // upper triangular U x = e_c, rows c .. 0
        for (int i = bs - 1; i >= 0; --i) {
          if (i > c) continue;
          double s = (i == c) ? 1.0 : 0.0;
          for (int t = i + 1; t <= c; ++t) s = fma(-Rb[(int64_t)i * l + t], x[t], s);
          x[i] = s / Rb[(int64_t)i * l + i];
        }
      }
      for (int i = 0; i < kB; ++i) {
        if (i < bs && c < bs) Dinv[(int64_t)(c0 + i) * l + c0 + c] = x[i];
      }
    }
  }
}

constexpr int kApplyRows = 32;
constexpr int kApplyThreads = 128;

// Q (rows x l, ldq) = X R^{-1}, blocked over 16 columns; X and Q may not alias.
__global__ void __launch_bounds__(kApplyThreads)
k_apply_trsm(const double *__restrict__ X, int64_t rows, int l, int64_t ldx,
             const double *__restrict__ R, const double *__restrict__ Dinv, double *__restrict__ Q,
             int64_t ldq, const int *skip_unless) {
  if (skip_unless && *reinterpret_cast<const volatile int *>(skip_unless) == 0) return;
  extern __shared__ double sm[];
  const int lp = l + 1;
  double *qs = sm;                                  // [kApplyRows][lp]
  double *rc = sm + kApplyRows * lp;                // [l][kB] block column of R
  double *dv = rc + (int64_t)l * kB;                // [kB][kB] inverse diagonal block
  const int64_t r0 = (int64_t)blockIdx.x * kApplyRows;
  const int nr = (int)min((int64_t)kApplyRows, rows - r0);
  for (int e = threadIdx.x; e < kApplyRows * l; e += blockDim.x) {
    const int r = e / l, c = e - r * l;
    qs[r * lp + c] = (r < nr) ? X[(r0 + r) * ldx + c] : 0.0;
  }
  // thread -> (row r, 4 columns j0..j0+3 of the block)
  const int r = threadIdx.x >> 2, j0 = (threadIdx.x & 3) * 4;
  for (int c0 = 0; c0 < l; c0 += kB) {
    const int bs = min(kB, l - c0);
    __syncthreads();
    for (int e = threadIdx.x; e < c0 * kB; e += blockDim.x) {
      const int t = e / kB, j = e - t * kB;
      rc[e] = (j < bs) ? R[(int64_t)t * l + c0 + j] : 0.0;
    }
    for (int e = threadIdx.x; e < kB * kB; e += blockDim.x) {
      const int i = e / kB, j = e - i * kB;
      dv[e] = (i < bs && j < bs) ? Dinv[(int64_t)(c0 + i) * l + c0 + j] : 0.0;
    }
    __syncthreads();
    double acc[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) acc[a] = (j0 + a < bs) ? qs[r * lp + c0 + j0 + a] : 0.0;
    for (int t = 0; t < c0; ++t) {
      const double qv = qs[r * lp + t];
#pragma unroll
      for (int a = 0; a < 4; ++a) acc[a] = fma(-qv, rc[t * kB + j0 + a], acc[a]);
    }
    // share the 16 residuals of row r, then multiply by the inverse block
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a)
      if (j0 + a < bs) qs[r * lp + c0 + j0 + a] = acc[a];
    __syncthreads();
    double out[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = 0; i < bs; ++i) {
      const double v = qs[r * lp + c0 + i];
#pragma unroll
      for (int a = 0; a < 4; ++a) out[a] = fma(v, dv[i * kB + j0 + a], out[a]);
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a)
      if (j0 + a < bs) qs[r * lp + c0 + j0 + a] = out[a];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nr * l; e += blockDim.x) {
    const int rr = e / l, c = e - rr * l;
    Q[(r0 + rr) * ldq + c] = qs[rr * lp + c];
  }
}

inline int grid_for(int64_t total, int threads) {
  int64_t b = (total + threads - 1) / threads;
  if (b > 4LL * num_sms()) b = 4LL * num_sms();
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t cholqr_init() {
  cudaError_t e = cudaFuncSetAttribute(k_gram_sym, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       100 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_chol_blocked, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_apply_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  return e;
}

int64_t gram_chunks(int64_t rows) { return (rows + kGramRows - 1) / kGramRows; }

cudaError_t gram_sym(const double *X, int64_t rows, int l, int64_t ldx, double *part, double *G,
                     const int *skip_unless, cudaStream_t st) {
  const int64_t chunks = gram_chunks(rows);
  const int lp = ((l + 3) / 4) * 4 + 1;
  const size_t smem = (size_t)kGramRows * lp * sizeof(double);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_gram_sym, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         100 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_gram_sym<<<(unsigned)chunks, kGramThreads, smem, st>>>(X, rows, l, ldx, part, skip_unless);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_gram_reduce<<<grid_for((int64_t)l * l, 256), 256, 0, st>>>(part, (int)chunks, l, G,
                                                                skip_unless);
  count_launch();
  return cudaGetLastError();
}

cudaError_t chol_blocked(const double *G, int l, int64_t rows, double *R, double *Dinv, Ctrl *ctrl,
                         int site, const int *skip_unless, cudaStream_t st, double again_tol) {
  const size_t smem = (size_t)l * l * sizeof(double);
  const bool use_smem = smem <= 200 * 1024;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_chol_blocked, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int threads = ((l * l / 24) + 31) / 32 * 32;
  threads = std::max(128, std::min(512, threads));
  k_chol_blocked<<<1, threads, use_smem ? smem : 0, st>>>(G, l, (double)rows, R, Dinv, ctrl, site,
                                                          skip_unless, use_smem ? 1 : 0,
                                                          again_tol);
  count_launch();
  return cudaGetLastError();
}

cudaError_t apply_trsm(const double *X, int64_t rows, int l, int64_t ldx, const double *R,
                       const double *Dinv, double *Q, int64_t ldq, const int *skip_unless,
                       cudaStream_t st) {
  const size_t smem = ((size_t)kApplyRows * (l + 1) + (size_t)l * kB + kB * kB) * sizeof(double);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_apply_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int64_t tiles = (rows + kApplyRows - 1) / kApplyRows;
  k_apply_trsm<<<(unsigned)tiles, kApplyThreads, smem, st>>>(X, rows, l, ldx, R, Dinv, Q, ldq,
                                                              skip_unless);
  count_launch();
  return cudaGetLastError();
}

}  // namespace rqk
