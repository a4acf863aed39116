// Small dense FP64 kernels around the l x l matrices of the method: the
// triangular inverse used by the adjoint, explicit Q from Householder
// reflectors, transposes, gathers and diagonals.
#include <cmath>

#include "kernels.cuh"

namespace rqk {

namespace {

// Rinv = R^{-1}, R upper triangular l x l.  One warp per column c: row i of
// the column solves R(i, i:c) x(i:c) = e_c(i) from the bottom up.
__global__ void __launch_bounds__(256)
k_trinv_upper(const double *__restrict__ R, int l, double *__restrict__ Rinv,
              const int *skip_unless) {
  if (skip_unless && *reinterpret_cast<const volatile int *>(skip_unless) == 0) return;
  __shared__ double xs[8][kMaxL];
  __shared__ double dinv[kMaxL];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < l; i += blockDim.x) dinv[i] = 1.0 / R[(int64_t)i * l + i];
  __syncthreads();
  const int c = blockIdx.x * 8 + warp;
  if (c >= l) return;
  double *x = xs[warp];
  for (int i = lane; i < l; i += 32) x[i] = 0.0;
  __syncwarp();
  if (lane == 0) x[c] = dinv[c];
  __syncwarp();
  for (int i = c - 1; i >= 0; --i) {
    double s = 0.0;
    for (int t = i + 1 + lane; t <= c; t += 32) s = fma(R[(int64_t)i * l + t], x[t], s);
    s = warp_sum(s);
    if (lane == 0) x[i] = -s * dinv[i];
    __syncwarp();
  }
  for (int i = lane; i < l; i += 32) Rinv[(int64_t)i * l + c] = x[i];
}

__global__ void k_transpose(const double *__restrict__ X, int64_t r, int64_t c, int64_t ldx,
                            double *__restrict__ Y, int64_t ldy) {
  __shared__ double t[32][33];
  const int64_t bi = (int64_t)blockIdx.y * 32, bj = (int64_t)blockIdx.x * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t i = bi + k, j = bj + threadIdx.x;
    if (i < r && j < c) t[k][threadIdx.x] = X[i * ldx + j];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t j = bj + k, i = bi + threadIdx.x;
    if (i < r && j < c) Y[j * ldy + i] = t[threadIdx.x][k];
  }
}

// Row-major elementwise kernels run on (32, 8) blocks: lanes along a row
// (coalesced), warps over rows, no index division per element.
__global__ void k_copy2d(const double *__restrict__ X, int64_t r, int64_t c, int64_t ldx,
                         double *__restrict__ Y, int64_t ldy, const int *skip_unless) {
  if (skip_unless && *reinterpret_cast<const volatile int *>(skip_unless) == 0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; i < r;
       i += (int64_t)gridDim.x * blockDim.y)
    for (int64_t j = threadIdx.x; j < c; j += blockDim.x) Y[i * ldy + j] = X[i * ldx + j];
}

__global__ void k_set_identity(double *X, int64_t r, int64_t c, int64_t ld) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; i < r;
       i += (int64_t)gridDim.x * blockDim.y)
    for (int64_t j = threadIdx.x; j < c; j += blockDim.x) X[i * ld + j] = (i == j) ? 1.0 : 0.0;
}

__global__ void k_gather_cols(const double *__restrict__ X, int64_t r, int64_t c, int64_t ldx,
                              const int32_t *__restrict__ perm, double *__restrict__ Y,
                              int64_t ldy) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < r * c;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / c, j = e - i * c;
    const int32_t pj = perm[j];
    Y[i * ldy + j] = (pj >= 0 && pj < c) ? X[i * ldx + pj] : 0.0;
  }
}

__global__ void k_iota(int32_t *p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (int32_t)i;
}

__global__ void k_diag_of(const double *__restrict__ T, int l, int64_t ldt, double *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < l) out[i] = T[(int64_t)i * ldt + i];
}

__global__ void k_zero_triangle(double *T, int l, int64_t ld, int strict_lower) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < l * l; e += gridDim.x * blockDim.x) {
    const int i = e / l, j = e - i * l;
    if (strict_lower ? (i > j) : (j > i)) T[(int64_t)i * ld + j] = 0.0;
  }
}

// Column c of Q = H_0 ... H_{t-1} e_c, applying H_s for s = min(c, t-1) .. 0
// (H_s e_c = e_c for s > c).  One warp per column, rows <= kMaxL.
__global__ void __launch_bounds__(256)
k_form_q(const double *__restrict__ Vh, int64_t ldv, const double *__restrict__ tau, int rows,
         int t, double *__restrict__ Q, int64_t ldq) {
  __shared__ double xs[8][kMaxL];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.x * (blockDim.x >> 5) + warp;
  if (c >= t) return;
  double *x = xs[warp];
  for (int i = lane; i < rows; i += 32) x[i] = (i == c) ? 1.0 : 0.0;
  __syncwarp();
  for (int s = min(c, t - 1); s >= 0; --s) {
    const double ts = tau[s];
    if (ts == 0.0) continue;
    double w = 0.0;
    for (int i = s + lane; i < rows; i += 32) w = fma(Vh[(int64_t)i * ldv + s], x[i], w);
    w = warp_sum(w) * ts;
    for (int i = s + lane; i < rows; i += 32) x[i] -= w * Vh[(int64_t)i * ldv + s];
    __syncwarp();
  }
  for (int i = lane; i < rows; i += 32) Q[(int64_t)i * ldq + c] = x[i];
}

// Triangular solves for a batch of row vectors, one warp per vector x of
// length n <= kMaxL (lane k holds entries k, k + 32, ...), right-looking so
// that each step is one multiply and a few lane-parallel FMAs:
//   backward = false: y U = x  (y_j = s_j / U_jj, then s_k -= y_j U_jk, k > j)
//   backward = true:  U y = x  with U symmetric in storage, only its strictly
//                     upper part used (y_t = s_t / U_tt, s_i -= U_ti y_t, i < t)
// 1 / U_jj comes from `dinv` when given, else from U's diagonal.
// U is staged in shared memory (n x n, ld n) when the launch gives it room
// (dynamic smem >= n^2 doubles): every step then reads its row at shared-
// memory latency instead of an L2 round trip.
// STAGED is a template argument so that the compiler addresses the staged
// copy as shared memory (a run-time choice would make every access generic).
template <bool STAGED>
__global__ void __launch_bounds__(128)
k_tri_rows(const double *__restrict__ Ug, int64_t ldug, const double *__restrict__ dinv, int n,
           const double *__restrict__ X, int64_t ldx, double *__restrict__ Y, int64_t ldy,
           int nvec, int backward) {
  extern __shared__ double us[];
  __shared__ double di[kMaxL];
  const double *U = Ug;
  int64_t ldu = ldug;
  if (STAGED) {
    stage_smem<double>(
        n * n, Ug,
        [&](int e) -> const double * {
          const int i = e / n, j = e - i * n;
          return Ug + (int64_t)i * ldug + j;
        },
        [&](int e) { return us + e; });
    U = us;
    ldu = n;
  }
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    di[j] = dinv ? dinv[j] : rcp_fast(Ug[(int64_t)j * ldug + j]);
  if (STAGED) cp_async_wait_all();
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int vec = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (vec >= nvec) return;
  constexpr int kSlots = kMaxL / 32;
  double sv[kSlots];
#pragma unroll
  for (int q = 0; q < kSlots; ++q) {
    const int k = 32 * q + lane;
    sv[q] = k < n ? X[(int64_t)vec * ldx + k] : 0.0;
  }
  if (!backward) {
#pragma unroll
    for (int jb = 0; jb < kSlots; ++jb) {
      if (32 * jb >= n) break;
      for (int jj = 0; jj < 32; ++jj) {
        const int j = 32 * jb + jj;
        if (j >= n) break;
        const double yj = __shfl_sync(0xffffffffu, sv[jb], jj) * di[j];
        if (lane == jj) sv[jb] = yj;
        const double *Uj = U + (int64_t)j * ldu;
#pragma unroll
        for (int q = jb; q < kSlots; ++q) {
          if (32 * q >= n) break;  // warp-uniform: no FP64 issue for empty slots
          const int k = 32 * q + lane;
          if (k > j && k < n) sv[q] = fma(-yj, Uj[k], sv[q]);
        }
      }
    }
  } else {
#pragma unroll
    for (int tb = kSlots - 1; tb >= 0; --tb) {
      if (32 * tb >= n) continue;
      for (int tt = 31; tt >= 0; --tt) {
        const int t = 32 * tb + tt;
        if (t >= n) continue;
        const double yt = __shfl_sync(0xffffffffu, sv[tb], tt) * di[t];
        if (lane == tt) sv[tb] = yt;
        const double *Ut = U + (int64_t)t * ldu;  // U_ti = U_it (symmetric storage)
#pragma unroll
        for (int q = 0; q <= tb; ++q) {
          if (32 * q >= t) break;  // warp-uniform
          const int i = 32 * q + lane;
          if (i < t) sv[q] = fma(-Ut[i], yt, sv[q]);
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < kSlots; ++q) {
    const int k = 32 * q + lane;
    if (k < n) Y[(int64_t)vec * ldy + k] = sv[q];
  }
}

// S = tril(M) + tril(M, -1)^T
__global__ void k_copyltu(const double *__restrict__ M, int l, double *__restrict__ S) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < l * l; e += gridDim.x * blockDim.x) {
    const int i = e / l, j = e - i * l;
    S[e] = (i >= j) ? M[e] : M[(int64_t)j * l + i];
  }
}

// Y[:, perm[j]] = X[:, j] (rows x c)
__global__ void k_scatter_cols(const double *__restrict__ X, int64_t r, int64_t c, int64_t ldx,
                               const int32_t *__restrict__ perm, double *__restrict__ Y,
                               int64_t ldy) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < r * c;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / c, j = e - i * c;
    const int32_t pj = perm[j];
    if (pj >= 0 && pj < c) Y[i * ldy + pj] = X[i * ldx + j];
  }
}

// gather (Y[i] = X[perm[i]]) or scatter (Y[perm[i]] = X[i]) of rows
__global__ void k_permute_rows(const double *__restrict__ X, int64_t r, int64_t c, int64_t ldx,
                               const int32_t *__restrict__ perm, double *__restrict__ Y,
                               int64_t ldy, int scatter) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < r * c;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / c, j = e - i * c;
    const int64_t pi = perm[i];
    if (pi < 0 || pi >= r) continue;
    if (scatter) Y[pi * ldy + j] = X[i * ldx + j];
    else Y[i * ldy + j] = X[pi * ldx + j];
  }
}

// zero X[i][j] for j > i in the first min(r, c) rows (the transposed
// structure of an upper-trapezoidal factor)
__global__ void k_mask_lower_trapezoid(double *X, int64_t r, int64_t c, int64_t ld) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < r * c;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / c, j = e - i * c;
    if (j > i) X[i * ld + j] = 0.0;
  }
}

// blocks for a (32, 8)-block row kernel: 8 rows per block, at most 4 waves
inline int rows_grid(int64_t rows) {
  int64_t b = (rows + 7) / 8;
  if (b > 4LL * num_sms()) b = 4LL * num_sms();
  return (int)std::max<int64_t>(b, 1);
}

inline int grid_for(int64_t total, int threads) {
  int64_t b = (total + threads - 1) / threads;
  if (b > 4LL * num_sms()) b = 4LL * num_sms();
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t chol_init() {
  const cudaError_t e = cudaFuncSetAttribute(
      k_tri_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
  return e == cudaSuccess ? cholqr_init() : e;
}

cudaError_t trinv_upper(const double *R, int l, double *Rinv, const int *skip_unless,
                        cudaStream_t st) {
  k_trinv_upper<<<(l + 7) / 8, 256, 0, st>>>(R, l, Rinv, skip_unless);
  count_launch();
  return cudaGetLastError();
}

cudaError_t transpose(const double *X, int64_t r, int64_t c, int64_t ldx, double *Y, int64_t ldy,
                      cudaStream_t st) {
  if (r <= 0 || c <= 0) return cudaSuccess;
  dim3 grid((unsigned)((c + 31) / 32), (unsigned)((r + 31) / 32));
  k_transpose<<<grid, dim3(32, 8), 0, st>>>(X, r, c, ldx, Y, ldy);
  count_launch();
  return cudaGetLastError();
}

cudaError_t copy2d(const double *X, int64_t r, int64_t c, int64_t ldx, double *Y, int64_t ldy,
                   const int *skip_unless, cudaStream_t st) {
  if (r <= 0 || c <= 0) return cudaSuccess;
  k_copy2d<<<rows_grid(r), dim3(32, 8), 0, st>>>(X, r, c, ldx, Y, ldy, skip_unless);
  count_launch();
  return cudaGetLastError();
}

cudaError_t set_identity(double *X, int64_t r, int64_t c, int64_t ld, cudaStream_t st) {
  if (r <= 0 || c <= 0) return cudaSuccess;
  k_set_identity<<<rows_grid(r), dim3(32, 8), 0, st>>>(X, r, c, ld);
  count_launch();
  return cudaGetLastError();
}

cudaError_t gather_cols(const double *X, int64_t r, int64_t c, int64_t ldx, const int32_t *perm,
                        double *Y, int64_t ldy, cudaStream_t st) {
  if (r <= 0 || c <= 0) return cudaSuccess;
  k_gather_cols<<<grid_for(r * c, 256), 256, 0, st>>>(X, r, c, ldx, perm, Y, ldy);
  count_launch();
  return cudaGetLastError();
}

cudaError_t iota(int32_t *p, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_iota<<<grid_for(n, 256), 256, 0, st>>>(p, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t copyltu(const double *M, int l, double *S, cudaStream_t st) {
  k_copyltu<<<grid_for((int64_t)l * l, 256), 256, 0, st>>>(M, l, S);
  count_launch();
  return cudaGetLastError();
}

cudaError_t scatter_cols(const double *X, int64_t r, int64_t c, int64_t ldx, const int32_t *perm,
                         double *Y, int64_t ldy, cudaStream_t st) {
  if (r <= 0 || c <= 0) return cudaSuccess;
  k_scatter_cols<<<grid_for(r * c, 256), 256, 0, st>>>(X, r, c, ldx, perm, Y, ldy);
  count_launch();
  return cudaGetLastError();
}

cudaError_t permute_rows(const double *X, int64_t r, int64_t c, int64_t ldx, const int32_t *perm,
                         double *Y, int64_t ldy, bool scatter, cudaStream_t st) {
  if (r <= 0 || c <= 0) return cudaSuccess;
  k_permute_rows<<<grid_for(r * c, 256), 256, 0, st>>>(X, r, c, ldx, perm, Y, ldy,
                                                       scatter ? 1 : 0);
  count_launch();
  return cudaGetLastError();
}

cudaError_t mask_lower_trapezoid(double *X, int64_t r, int64_t c, int64_t ld, cudaStream_t st) {
  if (r <= 0 || c <= 0) return cudaSuccess;
  k_mask_lower_trapezoid<<<grid_for(std::min(r, c) * c, 256), 256, 0, st>>>(X, std::min(r, c),
                                                                             c, ld);
  count_launch();
  return cudaGetLastError();
}

cudaError_t diag_of(const double *T, int l, int64_t ldt, double *out, cudaStream_t st) {
  k_diag_of<<<(l + 255) / 256, 256, 0, st>>>(T, l, ldt, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t zero_triangle(double *T, int l, int64_t ld, bool strict_lower, cudaStream_t st) {
  k_zero_triangle<<<grid_for((int64_t)l * l, 256), 256, 0, st>>>(T, l, ld, strict_lower ? 1 : 0);
  count_launch();
  return cudaGetLastError();
}

cudaError_t tri_rows(const double *U, int64_t ldu, const double *dinv, int n, const double *X,
                     int64_t ldx, double *Y, int64_t ldy, int nvec, bool backward,
                     cudaStream_t st) {
  if (n > kMaxL || n <= 0 || nvec <= 0) return cudaErrorInvalidValue;
  const size_t smem = (size_t)n * n * sizeof(double);
  const bool staged = smem <= 160 * 1024;
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k_tri_rows<true>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               160 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const unsigned grid = (unsigned)((nvec + 3) / 4);
  if (staged)
    k_tri_rows<true><<<grid, 128, smem, st>>>(U, ldu, dinv, n, X, ldx, Y, ldy, nvec,
                                              backward ? 1 : 0);
  else
    k_tri_rows<false><<<grid, 128, 0, st>>>(U, ldu, dinv, n, X, ldx, Y, ldy, nvec,
                                            backward ? 1 : 0);
  count_launch();
  return cudaGetLastError();
}

cudaError_t form_q(const double *Vh, int64_t ldv, const double *tau, int64_t rows, int t,
                   double *Q, int64_t ldq, cudaStream_t st, double *scratch) {
  if (rows > kMaxL || t <= 0) return cudaErrorInvalidValue;
  if (scratch && rows == t) {
    // compact WY (UT transform): H_0 ... H_{t-1} = I - V T V^T with
    // T^{-1} = diag(1 / tau) + striu(V^T V), so Q = I - V W, W = T V^T:
    // S = V^T V, row c of W^T solves T^{-1} w = (row c of V)^T, then one
    // small product.  A handful of short launches instead of t dependent
    // reflector applications per column.
    double *S = scratch, *Wt = scratch + (int64_t)t * t;
    cudaError_t e = gemm_small(true, false, Vh, ldv, Vh, ldv, S, t, t, t, rows, 1.0, 0.0, nullptr,
                               st);
    if (e == cudaSuccess) e = tri_rows(S, t, tau, t, Vh, ldv, Wt, t, t, true, st);
    if (e == cudaSuccess) e = set_identity(Q, rows, t, ldq, st);
    if (e == cudaSuccess)
      e = gemm_small(false, true, Vh, ldv, Wt, t, Q, ldq, rows, t, t, -1.0, 1.0, nullptr, st);
    return e;
  }
  // one warp per CTA: each column is a chain of t reflector applications,
  // so the columns are spread over as many SMs as possible
  k_form_q<<<t, 32, 0, st>>>(Vh, ldv, tau, (int)rows, t, Q, ldq);
  count_launch();
  return cudaGetLastError();
}

}  // namespace rqk
