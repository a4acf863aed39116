// Column-pivoted Householder QR of the wide l x n matrix B
// (Algorithm 2.1 step 5 / Algorithm 2.2 step 5, "cpqr(B)").
//
// One persistent cooperative kernel.  CTA b owns a contiguous slab of
// columns of B (each column l doubles), kept in shared memory when it fits
// and in a global scratch copy otherwise.  Per pivot step s there is exactly
// one grid barrier:
//   1. every CTA reads the candidate table (one (norm^2, index) pair and one
//      column per CTA, written before the barrier) and picks the same winner:
//      the largest trailing norm, ties to the lowest original column index;
//   2. every CTA builds the same Householder reflector from the winner's
//      column, mapping it to +alpha e_s (non-negative R(s, s));
//   3. every CTA applies the reflector to its own unpivoted columns (one warp
//      per column: a shuffle-reduced dot product, an axpy, and the exact new
//      trailing norm^2 over rows s+1..l-1), the owner of the winner writes its
//      final R column, and each CTA publishes its best candidate for s + 1.
// Candidate tables are double-buffered by step parity, so one barrier per
// step suffices.  After l steps the unchosen columns are written in their
// original order behind the pivots.
#include <cmath>

#include "kernels.cuh"

namespace rqk {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxGrid = 1024;

struct CpqrParams {
  const double *Bt;
  int64_t n;
  int l;
  int64_t ldb;
  double *R0t;
  int64_t ldr;
  int32_t *piv;
  double *Vh;
  double *tau;
  double *cand_norm;  // [2][G]
  int32_t *cand_idx;  // [2][G]
  double *pcol;       // [2][G][l]
  int32_t *counts;    // [G]
  double *gcols;      // G * cpb * l when the slab does not fit in shared memory
  Ctrl *ctrl;
  unsigned long long limit_ns;
  unsigned extra;
  int cpb;
  int use_smem;
};

__device__ __forceinline__ bool better(double na, int ia, double nb, int ib) {
  // (na, ia) beats (nb, ib): larger norm, ties to the lower index; ia < 0 is
  // empty.  Norms are >= 0 (empty slots hold -1), so their bit patterns order
  // like the values and the comparison stays on the integer pipe.
  if (ia < 0) return false;
  if (ib < 0) return true;
  const long long ka = __double_as_longlong(na), kb = __double_as_longlong(nb);
  if (ka != kb) return ka > kb;
  return ia < ib;
}

__global__ void __launch_bounds__(kThreads) k_cpqr_wide(CpqrParams P) {
  extern __shared__ double sm[];
  __shared__ double red[32];
  __shared__ double s_v[kMaxL];
  __shared__ double s_bn[kWarps];
  __shared__ int s_bi[kWarps];
  __shared__ int s_win_cta, s_win_idx;
  __shared__ double s_tau, s_beta, s_rv0;

  const int G = gridDim.x, b = blockIdx.x, l = P.l;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t c0 = (int64_t)b * P.cpb;
  const int nc = (int)max((int64_t)0, min(P.n, c0 + P.cpb) - c0);
  double *cols = P.use_smem ? sm : P.gcols + (int64_t)b * P.cpb * l;
  double *nrm = P.use_smem ? sm + (int64_t)P.cpb * l : reinterpret_cast<double *>(sm);
  double *nrm0 = nrm + P.cpb;  // norm^2 when last computed exactly
  int *pivoted = reinterpret_cast<int *>(nrm0 + P.cpb);

  // ---- load the slab, exact initial norms ------------------------------
  for (int jj = warp; jj < nc; jj += kWarps) {
    const double *src = P.Bt + (c0 + jj) * P.ldb;
    double s = 0.0;
    for (int r = lane; r < l; r += 32) {
      const double v = src[r];
      cols[(int64_t)jj * l + r] = v;
      s = fma(v, v, s);
    }
    s = warp_sum(s);
    if (lane == 0) {
      nrm[jj] = s;
      nrm0[jj] = s;
      pivoted[jj] = 0;
      if (!isfinite(s)) set_status(P.ctrl, RQLP_ERR_NONFINITE);
    }
  }
  __syncthreads();

  // local best candidate -> table slot `buf`
  auto publish = [&](int buf, int from_row) {
    double bn = -1.0;
    int bi = -1;
    for (int jj = tid; jj < nc; jj += kThreads) {
      if (pivoted[jj]) continue;
      const int idx = (int)(c0 + jj);
      if (better(nrm[jj], idx, bn, bi)) { bn = nrm[jj]; bi = idx; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double on = __shfl_xor_sync(0xffffffffu, bn, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (better(on, oi, bn, bi)) { bn = on; bi = oi; }
    }
    if (lane == 0) { s_bn[warp] = bn; s_bi[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double cn = -1.0;
      int ci = -1;
      for (int w = 0; w < kWarps; ++w)
        if (better(s_bn[w], s_bi[w], cn, ci)) { cn = s_bn[w]; ci = s_bi[w]; }
      s_win_idx = ci;
      P.cand_norm[buf * G + b] = cn;
      P.cand_idx[buf * G + b] = ci;
    }
    __syncthreads();
    const int ci = s_win_idx;
    if (ci >= 0) {
      const double *col = cols + (int64_t)(ci - c0) * l;
      double *dst = P.pcol + ((int64_t)buf * G + b) * l;
      for (int r = from_row + tid; r < l; r += kThreads) dst[r] = col[r];
    }
  };

  publish(0, 0);
  if (!grid_barrier(P.ctrl, G, P.limit_ns, P.extra, 1)) return;

  for (int s = 0; s < l; ++s) {
    const int buf = s & 1;
    // ---- 1. winner ----
    if (warp == 0) {
      double bn = -1.0;
      int bi = -1, bc = -1;
      for (int c = lane; c < G; c += 32) {
        const double cn = __ldcg(P.cand_norm + buf * G + c);
        const int ci = __ldcg(P.cand_idx + buf * G + c);
        if (better(cn, ci, bn, bi)) { bn = cn; bi = ci; bc = c; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double on = __shfl_xor_sync(0xffffffffu, bn, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
        if (better(on, oi, bn, bi)) { bn = on; bi = oi; bc = oc; }
      }
      if (lane == 0) { s_win_cta = bc; s_win_idx = bi; }
    }
    __syncthreads();
    const int wc = s_win_cta, wi = s_win_idx;
    if (wi < 0) { if (tid == 0) set_status(P.ctrl, RQLP_ERR_INVALID_ARG); return; }
    // ---- 2. reflector from the winner's column, rows s..l-1 ----
    const double *xc = P.pcol + ((int64_t)buf * G + wc) * l;
    double part = 0.0;
    for (int r = s + tid; r < l; r += kThreads) {
      const double v = __ldcg(xc + r);
      s_v[r - s] = v;
      if (r > s) part = fma(v, v, part);
    }
    const double sigma = block_sum(part, red);  // includes a __syncthreads
    // one thread forms the reflector (FP64 sqrt and divisions are costly here)
    if (tid == 0) {
      const double x0 = s_v[0];
      double tau, beta, rv0;
      if (sigma == 0.0) {
        if (x0 >= 0.0) { tau = 0.0; beta = x0; }
        else { tau = 2.0; beta = -x0; }
        rv0 = 0.0;
      } else {
        const double alpha = sqrt(fma(x0, x0, sigma));
        const double v0 = (x0 <= 0.0) ? (x0 - alpha) : (-sigma / (x0 + alpha));
        tau = 2.0 * v0 * v0 / (sigma + v0 * v0);
        beta = alpha;
        rv0 = 1.0 / v0;
      }
      s_tau = tau;
      s_beta = beta;
      s_rv0 = rv0;
    }
    __syncthreads();
    const double tau = s_tau, beta = s_beta, rv0 = s_rv0;
    for (int r = 1 + tid; r < l - s; r += kThreads) s_v[r] *= rv0;
    __syncthreads();
    if (tid == 0) s_v[0] = 1.0;
    __syncthreads();
    if (b == 0) {
      for (int r = tid; r < l; r += kThreads) P.Vh[(int64_t)r * l + s] = (r < s) ? 0.0 : s_v[r - s];
      if (tid == 0) { P.tau[s] = tau; P.piv[s] = wi; }
    }
    // ---- 3. apply to the slab ----
    // the winner's column is final: rows < s from the slab, beta at s, zeros below
    if ((int)(wi - c0) >= 0 && (int)(wi - c0) < nc && warp == 0) {
      const int jw = (int)(wi - c0);
      const double *col = cols + (int64_t)jw * l;
      double *out = P.R0t + (int64_t)s * P.ldr;
      for (int r = lane; r < l; r += 32) out[r] = (r < s) ? col[r] : (r == s ? beta : 0.0);
      if (lane == 0) { pivoted[jw] = 1; nrm[jw] = -1.0; }
    }
    // groups of 8 lanes per column, four columns per warp: the dot product
    // needs a 3-level reduction, and each FP64 warp instruction works on four
    // columns at once
    {
      const int sub = lane >> 3, gl = lane & 7;
      for (int jb = warp * 4; jb < nc; jb += kWarps * 4) {
        const int jj = jb + sub;
        const bool act = jj < nc && !pivoted[jj] && (int)(c0 + jj) != wi;
        double *col = cols + (int64_t)(act ? jj : 0) * l;
        double w = 0.0;
        if (act && tau != 0.0)
          for (int r = s + gl; r < l; r += 8) w = fma(s_v[r - s], col[r], w);
        w += __shfl_xor_sync(0xffffffffu, w, 4);
        w += __shfl_xor_sync(0xffffffffu, w, 2);
        w += __shfl_xor_sync(0xffffffffu, w, 1);
        if (act && tau != 0.0) {
          w *= tau;
          for (int r = s + gl; r < l; r += 8) col[r] = fma(-w, s_v[r - s], col[r]);
        }
        __syncwarp();
        // norm downdating: ||col(s+1:)||^2 = ||col(s:)||^2 - col(s)^2 (the
        // reflector preserves ||col(s:)||); recomputed exactly when more than
        // 99% of the norm has cancelled since the last exact value
        int need = 0;
        double nd = 0.0;
        if (act && gl == 0) {
          const double rsv = col[s];
          nd = nrm[jj] - rsv * rsv;
          need = !(nd > 0.01 * nrm0[jj]);
        }
        need = __shfl_sync(0xffffffffu, need, lane & ~7);
        double t = 0.0;
        if (need)
          for (int r = s + 1 + gl; r < l; r += 8) t = fma(col[r], col[r], t);
        t += __shfl_xor_sync(0xffffffffu, t, 4);
        t += __shfl_xor_sync(0xffffffffu, t, 2);
        t += __shfl_xor_sync(0xffffffffu, t, 1);
        if (act && gl == 0) {
          if (need) {
            nrm[jj] = t;
            nrm0[jj] = t;
          } else {
            nrm[jj] = nd;
          }
        }
      }
    }
    __syncthreads();
    if (s + 1 < l) {
      publish(buf ^ 1, s + 1);
      if (!grid_barrier(P.ctrl, G, P.limit_ns, 0, 2)) return;
    }
  }

  // ---- unchosen columns keep their order behind the l pivots ----
  int mine = 0;
  if (tid == 0) {
    for (int jj = 0; jj < nc; ++jj) mine += pivoted[jj] ? 0 : 1;
    P.counts[b] = mine;
  }
  if (!grid_barrier(P.ctrl, G, P.limit_ns, 0, 3)) return;
  __shared__ int s_prefix;
  if (tid == 0) {
    int pre = 0;
    for (int c = 0; c < b; ++c) pre += __ldcg(P.counts + c);
    s_prefix = pre;
  }
  __syncthreads();
  if (warp == 0) {
    // rank of each unpivoted column within the slab, in index order
    int pos = l + s_prefix;
    for (int jj0 = 0; jj0 < nc; jj0 += 32) {
      const int jj = jj0 + lane;
      const int un = (jj < nc && !pivoted[jj]) ? 1 : 0;
      const unsigned mask = __ballot_sync(0xffffffffu, un);
      const int rank = __popc(mask & ((1u << lane) - 1u));
      if (un) {
        P.piv[pos + rank] = (int32_t)(c0 + jj);
        pivoted[jj] = -(pos + rank) - 1;  // remember the destination row
      }
      pos += __popc(mask);
    }
  }
  __syncthreads();
  for (int jj = warp; jj < nc; jj += kWarps) {
    const int code = pivoted[jj];
    if (code >= 0) continue;
    const int64_t dst = -(int64_t)code - 1;
    const double *col = cols + (int64_t)jj * l;
    for (int r = lane; r < l; r += 32) P.R0t[dst * P.ldr + r] = col[r];
  }
}

struct Plan {
  int G, cpb, use_smem;
  size_t smem;
};

Plan plan_for(int64_t n, int l) {
  Plan p;
  const int sms = num_sms();
  const int cap = tuning().cpqr_max_ctas;
  int G = (int)std::min<int64_t>(n, (int64_t)((cap > 0 && cap < sms) ? cap : sms));
  if (G < 1) G = 1;
  int cpb = (int)((n + G - 1) / G);
  G = (int)((n + cpb - 1) / cpb);
  const size_t state = (size_t)cpb * (2 * sizeof(double) + sizeof(int));
  const size_t slab = (size_t)cpb * l * sizeof(double);
  p.use_smem = (slab + state <= 190 * 1024) ? 1 : 0;
  p.smem = (p.use_smem ? slab : 0) + state;
  p.G = G;
  p.cpb = cpb;
  return p;
}

}  // namespace

size_t cpqr_ws_bytes(int64_t n, int l) {
  const size_t G = kMaxGrid;
  size_t b = 0;
  b += 2 * G * sizeof(double);
  b += 2 * G * sizeof(int32_t);
  b += 2 * G * (size_t)l * sizeof(double);
  b += G * sizeof(int32_t);
  b += (size_t)(n + kMaxGrid) * l * sizeof(double);  // global slabs (fallback)
  return b + 8192;
}

size_t cpqr_scratch_bytes_smem_only(int64_t n, int l, bool *fits) {
  const Plan pl = plan_for(n, l);
  *fits = pl.use_smem != 0 && pl.G <= kMaxGrid;
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  return up(2 * (size_t)pl.G * sizeof(double)) + up(2 * (size_t)pl.G * sizeof(int32_t)) +
         up(2 * (size_t)pl.G * l * sizeof(double)) + up((size_t)pl.G * sizeof(int32_t));
}

cudaError_t cpqr_wide(const double *Bt, int64_t n, int l, int64_t ldb, double *R0t, int64_t ldr,
                      int32_t *piv, double *Vh, double *tau, void *scratch, Ctrl *ctrl,
                      unsigned long long limit_ns, unsigned debug_extra, cudaStream_t st) {
  if (n <= 0 || l <= 0 || l > kMaxL || l > n) return cudaErrorInvalidValue;
  Plan pl = plan_for(n, l);
  if (pl.G > kMaxGrid) return cudaErrorInvalidValue;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaError_t e = cudaFuncSetAttribute(k_cpqr_wide, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)std::max<size_t>(pl.smem, 1));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cpqr_wide, kThreads, pl.smem);
  if (e != cudaSuccess) return e;
  if ((int64_t)per_sm * num_sms() < pl.G) return cudaErrorCooperativeLaunchTooLarge;

  char *p = reinterpret_cast<char *>(scratch);
  auto take = [&](size_t bytes) { char *r = p; p += (bytes + 255) / 256 * 256; return r; };
  CpqrParams P;
  P.Bt = Bt; P.n = n; P.l = l; P.ldb = ldb; P.R0t = R0t; P.ldr = ldr; P.piv = piv;
  P.Vh = Vh; P.tau = tau;
  P.cand_norm = reinterpret_cast<double *>(take(2 * (size_t)pl.G * sizeof(double)));
  P.cand_idx = reinterpret_cast<int32_t *>(take(2 * (size_t)pl.G * sizeof(int32_t)));
  P.pcol = reinterpret_cast<double *>(take(2 * (size_t)pl.G * l * sizeof(double)));
  P.counts = reinterpret_cast<int32_t *>(take((size_t)pl.G * sizeof(int32_t)));
  P.gcols = reinterpret_cast<double *>(take((size_t)pl.G * pl.cpb * l * sizeof(double)));
  P.ctrl = ctrl;
  P.limit_ns = limit_ns ? limit_ns : kDefaultSpinNs;
  P.extra = debug_extra;
  P.cpb = pl.cpb;
  P.use_smem = pl.use_smem;
  // the permutation stays valid even if the kernel stops early on an error
  e = iota(piv, n, st);
  if (e != cudaSuccess) return e;
  if (pl.G == 1) {
    // one CTA: its grid barrier never waits, no co-residency is needed
    k_cpqr_wide<<<1, kThreads, pl.smem, st>>>(P);
    count_launch();
    return cudaGetLastError();
  }
  void *args[] = {&P};
  e = cudaLaunchCooperativeKernel((const void *)k_cpqr_wide, dim3(pl.G), dim3(kThreads), args,
                                  pl.smem, st);
  count_launch();
  return e;
}

}  // namespace rqk
