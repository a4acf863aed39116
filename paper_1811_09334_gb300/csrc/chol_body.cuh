// Single-CTA Cholesky of a Gram matrix (cholqr.cu): the body of the one-CTA
// kernel, also run inside a work item of the persistent batch kernel.  Any
// block size that is a multiple of 32 (at most 1024).
#pragma once

#include "kernels.cuh"

namespace rqk {
namespace cholk {

constexpr int kB = 16;  // block size of the Cholesky and the solve

// Upper Cholesky G = R^T R with 16-column blocks, breakdown detection and one
// shifted retry: a pivot d_j <= l 2 eps G_jj means the Gram matrix is
// numerically singular, and the factorization is redone once on G + s I with
// the shift s = 11 (rows l + l (l + 1)) eps tr(G) of shifted CholeskyQR
// (Fukaya et al. 2020).  Also writes Dinv: the inverses of R's 16 x 16 diagonal
// blocks (block-diagonal l x l, ld l).  T = float (use_smem only): the FP32
// factorization of the FP32 CholeskyQR pass, ~20x faster per column than the
// FP64 one on this GPU; R and Dinv are still written in FP64.
template <typename T>
__device__ __forceinline__ T fmaT(T a, T b, T c);
template <>
__device__ __forceinline__ float fmaT(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <>
__device__ __forceinline__ double fmaT(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rsqrtT(float x) {
  const float y = rsqrtf(x);
  return y * fmaf(-0.5f * x * y, y, 1.5f);  // one Newton step: FP32 accuracy
}
__device__ __forceinline__ double rsqrtT(double x) { return rsqrt(x); }

template <typename T>
__device__ __forceinline__ void chol_body(const double *G, int l, double rows, double *R,
                                          double *Dinv, Ctrl *ctrl, int site, int use_smem,
                                          double again_tol, double eps, double *sm) {
  __shared__ double red[32];
  __shared__ T s_gdiag[kMaxL];
  __shared__ T s_next;
  __shared__ int s_fail;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  T *W = use_smem ? reinterpret_cast<T *>(sm) : reinterpret_cast<T *>(R);
  const T thr_scale = (T)((double)l * 2.0 * eps);
  double tr = 0.0;
  for (int i = tid; i < l; i += blockDim.x) tr += G[(int64_t)i * l + i];
  tr = block_sum(tr, red);
  int fail = 0;
  for (int attempt = 0; attempt < 2; ++attempt) {
    const double shift = attempt ? 11.0 * (rows * l + (double)l * (l + 1)) * eps * tr : 0.0;
    for (int e = tid; e < l * l; e += blockDim.x) {
      const int i = e / l, j = e - i * l;
      W[e] = (T)(G[e] + (i == j ? shift : 0.0));
    }
    for (int i = tid; i < l; i += blockDim.x) s_gdiag[i] = (T)(G[(int64_t)i * l + i] + shift);
    if (tid == 0) s_fail = 0;
    __syncthreads();
    // right-looking, one column per step, spread over every warp; warp 0
    // updates the next diagonal entry first and takes its reciprocal square
    // root while the other warps update the rest of the trailing triangle
    if (tid == 0) {
      const T d = W[0];
      const T g0 = s_gdiag[0];
      int f = 0;
      if (!isfinite(d) || !isfinite(g0)) f = 2;
      else if (!(d > thr_scale * g0) || !(d > (T)0)) f = 1;
      s_fail = f;
      s_next = f ? (T)1 : rsqrtT(d);
    }
    __syncthreads();
    for (int j = 0; j < l && !s_fail; ++j) {
      const T rs = s_next;
      T *Wj = W + j * l;  // l <= 256: 32-bit offsets
      // only thread 0 reads and rewrites the pivot; s_next and row j were
      // written before the previous barrier
      for (int c = j + 1 + tid; c < l; c += blockDim.x) Wj[c] *= rs;
      if (tid == 0) Wj[j] = Wj[j] * rs;
      __syncthreads();
      if (warp == 0) {
        if (j + 1 < l) {
          T *W1 = W + (j + 1) * l;
          const T r1 = Wj[j + 1];
          if (lane == 0) {
            const T dn = fmaT(-r1, r1, W1[j + 1]);
            W1[j + 1] = dn;
            const T g0 = s_gdiag[j + 1];
            int f = 0;
            if (!isfinite(dn) || !isfinite(g0)) f = 2;
            else if (!(dn > thr_scale * g0) || !(dn > (T)0)) f = 1;
            if (f) s_fail = f;
            s_next = f ? (T)1 : rsqrtT(dn);
          }
          // the rest of row j + 1 of the trailing triangle
          for (int c = j + 2 + lane; c < l; c += 32) W1[c] = fmaT(-r1, Wj[c], W1[c]);
        }
      } else {
        for (int a = j + 2 + (warp - 1); a < l; a += nw - 1) {
          const T ra = Wj[a];
          T *Wa = W + a * l;
          int c = a + lane;
          for (; c + 32 < l; c += 64) {
            const T x0 = fmaT(-ra, Wj[c], Wa[c]);
            const T x1 = fmaT(-ra, Wj[c + 32], Wa[c + 32]);
            Wa[c] = x0;
            Wa[c + 32] = x1;
          }
          if (c < l) Wa[c] = fmaT(-ra, Wj[c], Wa[c]);
        }
      }
      __syncthreads();
    }
    __syncthreads();
    fail = s_fail;
    __syncthreads();
    if (fail == 0 || fail == 2) break;
    // the FP32 pass (power steps: only the span of the basis matters) shifts
    // silently; an FP64 pass that needs the shift is reported
    if (attempt == 0 && tid == 0 && sizeof(T) == sizeof(double)) {
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
    R[e] = (j >= i) ? (double)W[e] : 0.0;
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
      const int again = (fail != 0) || !(2.0 * eps * c * c <= again_tol);
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
      T x[kB];
#pragma unroll
      for (int i = 0; i < kB; ++i) x[i] = (T)0;
      if (c < bs) {
        const T *Rb = W + (int64_t)c0 * l + c0;  // the factor, in the working precision
        // upper triangular U x = e_c, rows c .. 0
        for (int i = bs - 1; i >= 0; --i) {
          if (i > c) continue;
          T s = (i == c) ? (T)1 : (T)0;
          for (int t = i + 1; t <= c; ++t) s = fmaT(-Rb[(int64_t)i * l + t], x[t], s);
          x[i] = s / Rb[(int64_t)i * l + i];
        }
      }
      for (int i = 0; i < kB; ++i) {
        if (i < bs && c < bs) Dinv[(int64_t)(c0 + i) * l + c0 + c] = (double)x[i];
      }
    }
  }
}

}  // namespace cholk
}  // namespace rqk
