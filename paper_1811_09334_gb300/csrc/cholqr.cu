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
//   k_chol_cluster  upper Cholesky of G on a cluster of 16 (or 8) CTAs (l <= 224):
//                   rows dealt round-robin, finished rows pushed to every CTA
//                   through distributed shared memory, look-ahead on the next
//                   row; breakdown detection and the shifted retry.
//   k_chol_blocked  the same for l > 224 on one CTA, right-looking over
//                   columns with the work of each
//                   column spread over every warp (a warp-wide FP64
//                   instruction holds an SMSP's FP64 pipe for many cycles, so
//                   single-warp FP64 work is slow here); warp 0 updates the
//                   next diagonal entry first and takes its reciprocal square
//                   root while the others update the trailing triangle.  It
//                   also writes the inverses of R's 16 x 16 diagonal blocks.
//   k_chol_f32      the FP32 Cholesky of the power steps' FP32 passes
//                   (l <= 128, one CTA, registers); it also leaves R and the
//                   block inverses in FP32 for the FP32 solve.
//   k_apply_trsm    Q = X R^{-1} as a blocked triangular solve on 32-row tiles:
//                   Q[:, b] = (X[:, b] - Q[:, <b] R[<b, b]) inv(R[b, b]); half
//                   the FMAs of multiplying by a full inverse, and no separate
//                   triangular inversion.
#include <cmath>

#include "chol_body.cuh"

namespace rqk {

namespace {

using namespace cholk;
constexpr int kGramMaxRows = 32;  // rows of X per Gram chunk, at most
constexpr int kGramThreads = 256;

// Upper triangle of X_c^T X_c for the rc rows of chunk c = blockIdx.x, into
// part[c] (l x l, only j >= i written).  Tiles of 4 x 4 over the triangle.
// T = float: the chunk is rounded to FP32 and its products accumulate in FP32
// over at most 32 rows (the chunks are summed in FP64).
template <typename T>
__global__ void __launch_bounds__(kGramThreads)
k_gram_sym(const double *__restrict__ X, int64_t rows, int l, int64_t ldx, int rc,
           double *__restrict__ part, const int *skip_unless) {
  if (skip_unless && *reinterpret_cast<const volatile int *>(skip_unless) == 0) return;
  extern __shared__ double xs_raw[];
  T *xs = reinterpret_cast<T *>(xs_raw);  // [rc][lp]
  const int lp = ((l + 3) / 4) * 4 + 1;
  const int64_t r0 = (int64_t)blockIdx.x * rc;
  const int nr = (int)min((int64_t)rc, rows - r0);
  for (int e = threadIdx.x; e < nr * lp; e += blockDim.x) {
    const int r = e / lp, c = e - r * lp;
    xs[e] = (c < l) ? from_f64<T>(X[(r0 + r) * ldx + c]) : (T)0;
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
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
    for (int r = 0; r < nr; ++r) {
      const T *row = xs + r * lp;
      T x[4], y[4];
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
        if (j < l && j >= i) out[(int64_t)i * l + j] = to_f64(acc[a][b]);
      }
    }
  }
}

// G[i][j] = G[j][i] = sum_c part[c][i][j] for i <= j.  Block (32, 8): 32
// consecutive entries, the chunks split over threadIdx.y (two accumulators
// each), then a fixed-order sum over y, so the result is deterministic and
// no thread runs a long chain of dependent FP64 additions.
constexpr int kReduceY = 8;
__global__ void __launch_bounds__(32 * kReduceY)
k_gram_reduce(const double *__restrict__ part, int chunks, int l, double *__restrict__ G,
              const int *skip_unless) {
  if (skip_unless && *reinterpret_cast<const volatile int *>(skip_unless) == 0) return;
  __shared__ double red[kReduceY][33];
  const int64_t ll = (int64_t)l * l;
  const int64_t e = (int64_t)blockIdx.x * 32 + threadIdx.x;
  const int y = threadIdx.y;
  int i = 0, j = 0;
  bool want = false;
  if (e < ll) {
    i = (int)(e / l);
    j = (int)(e - (int64_t)i * l);
    want = j >= i;
  }
  double a0 = 0.0, a1 = 0.0;
  if (want) {
    int c = y;
    for (; c + kReduceY < chunks; c += 2 * kReduceY) {
      a0 += part[(int64_t)c * ll + e];
      a1 += part[(int64_t)(c + kReduceY) * ll + e];
    }
    if (c < chunks) a0 += part[(int64_t)c * ll + e];
  }
  red[y][threadIdx.x] = a0 + a1;
  __syncthreads();
  if (y == 0 && want) {
    double s = red[0][threadIdx.x];
#pragma unroll
    for (int k = 1; k < kReduceY; ++k) s += red[k][threadIdx.x];
    G[(int64_t)i * l + j] = s;
    G[(int64_t)j * l + i] = s;
  }
}

template <typename T>
__global__ void __launch_bounds__(512)
k_chol_blocked(const double *__restrict__ G, int l, double rows, double *__restrict__ R,
               double *__restrict__ Dinv, Ctrl *ctrl, int site, const int *skip_unless,
               int use_smem, double again_tol, double eps) {
  if (skip_unless && *reinterpret_cast<const volatile int *>(skip_unless) == 0) return;
  extern __shared__ double sm[];
  chol_body<T>(G, l, rows, R, Dinv, ctrl, site, use_smem, again_tol, eps, sm);
}

// ---------------------------------------------------------------------------
// Cluster Cholesky.  One SM does the l^3/6 FP64 FMAs of an l x l Cholesky at
// about 2 FMA per clock, and every column adds a chain of dependent FP64
// operations; here a cluster of C = 16 (or 8) CTAs shares the work.  Row a of
// the trailing matrix belongs to CTA a % C (round-robin: while one CTA forms
// row j + 1, the owner of row j + 2 has already applied row j to it, so the
// other updates stay off the column chain; contiguous row blocks measured
// slower); thread c of that CTA keeps column c of its rows in registers.
// Every finished row is also kept packed in each CTA's shared memory (row j
// at off(j), entries j .. l-1): the owner pushes it to the other CTAs with
// st.async stores that complete bytes on the receiver's mbarrier for that
// row.  Every row is written once per attempt, so no buffer is reused and
// nothing has to be acknowledged.  The owner of row j + 1 applies row j to it
// first, scales it and sends it (look-ahead), then updates its other rows.  A
// breakdown is sent in place of the diagonal entry (-1: not positive enough,
// -2: not finite), so every CTA stops at the same row; the shifted retry (as
// in the single-CTA kernel) uses a second set of mbarriers.  The critical
// path per column (pivot test, reciprocal square root, scaling) uses integer
// tests on the bit patterns and an FP32 estimate refined in FP64, so few
// dependent FP64 operations sit on it.
constexpr int kClusterMaxL = 224;

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned map_shared(unsigned addr, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void bar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_expect(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool bar_try(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// false when the phase did not complete within limit_ns
__device__ __forceinline__ bool bar_wait_bounded(unsigned bar, unsigned parity,
                                                 unsigned long long limit_ns) {
  if (bar_try(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  while (!bar_try(bar, parity))
    if (globaltimer_ns() - t0 > limit_ns) return false;
  return true;
}
__device__ __forceinline__ void st_async_f64(unsigned raddr, double v, unsigned rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];" ::"r"(
                   raddr),
               "d"(v), "r"(rbar)
               : "memory");
}

// pivot test on bit patterns: 0 accepted, 1 not above thr (or not positive),
// 2 not finite; thr >= 0
__device__ __forceinline__ int pivot_code(double x, double thr) {
  const long long b = __double_as_longlong(x);
  if (((b >> 52) & 0x7ff) == 0x7ff) return 2;
  return (b > __double_as_longlong(thr)) ? 0 : 1;  // negative x: b < 0 <= thr bits
}

// blockDim.x = 32 NW with NW = 4 (l <= 128) or 8 (l <= 256); l <= kClusterMaxL;
// ceil(l / C) <= RMAX.  Thread (warp w, lane) holds, of own row i (a_i =
// rank + i C), the entry in column a_i + 32 ((w - i) mod NW) + lane: each row's
// 32-wide chunks rotate over the warps, so the FP64 work of a column (one warp
// instruction per chunk, about 64 clocks of an SMSP's FP64 unit each) is
// spread evenly over the SM's four schedulers.
template <int C, int RMAX>
__global__ void __launch_bounds__(256)
k_chol_cluster(const double *__restrict__ G, int l, double rows, double *__restrict__ R,
               double *__restrict__ Dinv, Ctrl *ctrl, int site, const int *skip_unless,
               double again_tol, double eps, unsigned long long limit_ns) {
  if (skip_unless && *reinterpret_cast<const volatile int *>(skip_unless) == 0) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int ntri = l * (l + 1) / 2;
  double *tri = reinterpret_cast<double *>(smraw);  // packed upper triangle
  unsigned long long *bars = reinterpret_cast<unsigned long long *>(tri + ntri);  // [2][l]
  double *thr = reinterpret_cast<double *>(bars + 2 * l);  // [l] pivot thresholds
  __shared__ double red[32];
  __shared__ double s_rs;
  __shared__ int s_f, s_code;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const unsigned me = cluster_rank();
  auto off = [l](int j) { return j * l - (j * (j - 1)) / 2; };
  // column of own row i held by this thread
  auto col = [&](int i) { return (int)me + i * C + ((((warp - i) & (nw - 1))) << 5) + lane; };
  const unsigned tri0 = smem_u32(tri), bar0 = smem_u32(bars);
  unsigned rtri[C], rbar[C];  // this layout in every CTA of the cluster
#pragma unroll
  for (int d = 0; d < C; ++d) {
    rtri[d] = map_shared(tri0, d);
    rbar[d] = map_shared(bar0, d);
  }

  for (int i = tid; i < 2 * l; i += blockDim.x) bar_init(bar0 + 8u * i, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  for (int i = tid; i < 2 * l; i += blockDim.x) {
    const int j = i % l;
    if ((unsigned)(j % C) != me) bar_expect(bar0 + 8u * i, (unsigned)(l - j) * 8u);
  }
  double tr = 0.0;
  for (int i = tid; i < l; i += blockDim.x) tr += G[(int64_t)i * l + i];
  tr = block_sum(tr, red);
  // no CTA sends before every CTA's barriers are initialised and armed
  cluster_sync_all();

  double v[RMAX];  // v[i] = working entry (a_i, col(i))
  int fail = 0;
  for (int att = 0; att < 2; ++att) {
    const double shift = att ? 11.0 * (rows * l + (double)l * (l + 1)) * eps * tr : 0.0;
#pragma unroll
    for (int i = 0; i < RMAX; ++i) {
      const int a = (int)me + i * C, c = col(i);
      v[i] = (a < l && c < l) ? G[(int64_t)a * l + c] + (c == a ? shift : 0.0) : 0.0;
    }
    for (int a = (int)me + tid * C; a < l; a += (int)blockDim.x * C)
      thr[a] = (double)l * 2.0 * eps * (G[(int64_t)a * l + a] + shift);
    if (tid == 0) s_code = 0;
    __syncthreads();
    const unsigned barA = bar0 + 8u * (unsigned)(att * l);
    // row r of R from its fully updated entries: this thread holds x = (r, cx)
    auto produce = [&](int r, double x, int cx) {
      if (cx == r) {
        int f = pivot_code(x, thr[r]);
        if (f == 0 && pivot_code(thr[r], 0.0) == 2) f = 2;  // threshold from a non-finite G
        s_f = f;
        s_rs = f ? 1.0 : rsqrt_fast(x);
      }
      __syncthreads();
      if (cx < l) {
        const int f = s_f;
        double y = x * s_rs;
        if (cx == r && f) y = -(double)f;
        const unsigned e8 = 8u * (unsigned)(off(r) + (cx - r)), b8 = 8u * (unsigned)(att * l + r);
        tri[e8 >> 3] = y;
#pragma unroll
        for (int d = 0; d < C; ++d)
          if ((unsigned)d != me) st_async_f64(rtri[d] + e8, y, rbar[d] + b8);
      }
    };
    if (me == 0) produce(0, v[0], col(0));
    int j = 0;
    for (; j < l; ++j) {
      int code;
      if ((unsigned)(j % C) != me) {
        if (!bar_wait_bounded(barA + 8u * j, 0, limit_ns)) {
          code = 3;
        } else {
          const long long bv = __double_as_longlong(tri[off(j)]);
          code = bv > 0 ? 0 : (bv == __double_as_longlong(-1.0) ? 1 : 2);
        }
      } else {
        code = s_f;
      }
      if (code) atomicMax(&s_code, code);
      if (__syncthreads_or(code != 0)) break;
      const double *Rj = tri + off(j) - j;  // Rj[t] = R(j, t), t >= j
      if (j + 1 < l && (unsigned)((j + 1) % C) == me) {
        const int i1 = (j + 1 - (int)me) / C;
        double w = 0.0;
#pragma unroll
        for (int i = 0; i < RMAX; ++i)
          if (i == i1) w = v[i];
        const int c1 = col(i1);
        produce(j + 1, c1 < l ? fma(-Rj[j + 1], Rj[c1], w) : 0.0, c1);
      }
      // own rows a >= j + 2; a warp skips rows where its chunk is empty
#pragma unroll
      for (int i = 0; i < RMAX; ++i) {
        const int a = (int)me + i * C;
        if (a >= j + 2 && a < l && ((((warp - i) & (nw - 1))) << 5) < l - a) {
          const int c = col(i);
          if (c < l) v[i] = fma(-Rj[a], Rj[c], v[i]);
        }
      }
    }
    fail = (j < l) ? s_code : 0;
    if (fail == 1 && att == 0) {
      if (me == 0 && tid == 0) {
        ctrl->shift_flag[site] = 1;
        set_status(ctrl, RQLP_WARN_SHIFTED_CHOLQR);
      }
      cluster_sync_all();  // every CTA has left the first attempt
      continue;
    }
    break;
  }
  if (me == 0 && tid == 0) {
    if (fail == 2) set_status(ctrl, RQLP_ERR_NONFINITE);
    else if (fail == 1) set_status(ctrl, RQLP_ERR_RANK_DEFICIENT);
  }
  if (fail == 3 && tid == 0) {
    set_status(ctrl, RQLP_ERR_TIMEOUT);
    atomicExch(&ctrl->timeout_site, 200 + site);
  }
  __syncthreads();
  // own rows of R, zeros below the diagonal
  for (int a = (int)me; a < l; a += C)
    for (int t = tid; t < l; t += blockDim.x)
      R[(int64_t)a * l + t] = t >= a ? tri[off(a) + t - a] : 0.0;
  // a second pass is needed when eps * cond(R)^2 exceeds again_tol (cond
  // estimated from diag(R)), as in the single-CTA kernel
  if (again_tol >= 0.0 && me == 0 && warp == 0) {
    double mx = 0.0, mn = 1e300;
    for (int i = lane; i < l; i += 32) {
      const double d = tri[off(i)];
      mx = fmax(mx, d);
      mn = fmin(mn, d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    }
    if (lane == 0) {
      const double cn = (mn > 0.0) ? mx / mn : 1e300;
      const int again = (fail != 0) || !(2.0 * eps * cn * cn <= again_tol);
      ctrl->again_flag[site] = again;
      ctrl->done_flag[site] = 1 - again;
    }
  }
  // inverses of the 16 x 16 diagonal blocks, block bk on CTA bk % C: lane
  // cc solves U x = e_cc by back substitution with the reciprocals of U's
  // diagonal taken once
  const int nblk = (l + kB - 1) / kB;
  for (int bk = (int)me + C * warp; bk < nblk; bk += C * nw) {
    const int c0 = bk * kB, bs = min(kB, l - c0);
    const int cc = lane;
    auto U = [&](int i, int t) { return tri[off(c0 + i) + (t - i)]; };  // t >= i
    const double dl = (lane < bs) ? 1.0 / U(lane, lane) : 0.0;
    double x[kB];
#pragma unroll
    for (int i = 0; i < kB; ++i) x[i] = 0.0;
#pragma unroll
    for (int i = kB - 1; i >= 0; --i) {
      const double di = __shfl_sync(0xffffffffu, dl, i);
      if (i < bs && cc < bs && i <= cc) {
        double s = (i == cc) ? 1.0 : 0.0;
#pragma unroll
        for (int t = i + 1; t < kB; ++t)
          if (t <= cc && t < bs) s = fma(-U(i, t), x[t], s);
        x[i] = s * di;
      }
    }
    if (cc < bs)
#pragma unroll
      for (int i = 0; i < kB; ++i)
        if (i < bs) Dinv[(int64_t)(c0 + i) * l + c0 + cc] = x[i];
  }
  // no CTA leaves while another may still send to it
  cluster_sync_all();
}

// FP32 Cholesky for the FP32 CholeskyQR pass, l <= 128, one CTA of 1024
// threads: thread t holds column c = t % 128 of rows 16 g .. 16 g + 15 of
// the trailing matrix (g = t / 128) in registers.  Per column j: the pivot's
// thread takes the reciprocal square root (FP32 MUFU estimate and one Newton
// step), row j is scaled by its group and published in shared memory
// (double-buffered by parity), and every thread applies it to its rows with
// one broadcast row load per 4 rows.  Two barriers per column, no FP64 on
// the chain.  The column loop is bound by instruction issue (32 warps share
// four schedulers), so the updates carry no per-entry tests: a warp with
// nothing left (rows finished, columns finished or below the diagonal) skips
// them, and the entries below the diagonal or beyond column l take updates
// that are never read.  Conversions to and from FP64 use the integer pipe,
// the diagonal blocks stay in shared memory for their inverses, and R and
// the block inverses are written in FP64 (and in FP32 to `pack`).
constexpr int kChol32MaxL = 128;
__global__ void __launch_bounds__(1024)
k_chol_f32(const double *__restrict__ G, int l, double rows, double *__restrict__ R,
           double *__restrict__ Dinv, Ctrl *ctrl, int site, const int *skip_unless, double eps,
           float *__restrict__ pack) {
  if (skip_unless && *reinterpret_cast<const volatile int *>(skip_unless) == 0) return;
  __shared__ __align__(16) float rowbuf[2][kChol32MaxL];
  __shared__ float s_thr[kChol32MaxL];
  __shared__ float s_blk[kChol32MaxL / kB][kB][kB + 1];  // diagonal blocks of R
  __shared__ double red[32];
  __shared__ float s_rs;
  __shared__ int s_f;
  const int tid = threadIdx.x, c = tid & 127, g = tid >> 7;
  const int lane = tid & 31, warp = tid >> 5;
  float v[16];
  int fail = 0;
  for (int att = 0; att < 2; ++att) {
    double shift = 0.0;
    if (att) {
      double tr = 0.0;
      for (int i = tid; i < l; i += blockDim.x) tr += G[(int64_t)i * l + i];
      tr = block_sum(tr, red);
      shift = 11.0 * (rows * l + (double)l * (l + 1)) * eps * tr;
    }
    // eight loads in flight at a time (clamped indices, masked after)
#pragma unroll
    for (int h = 0; h < 16; h += 8) {
      double gv[8];
      const int cl = min(c, l - 1);
#pragma unroll
      for (int i = 0; i < 8; ++i) gv[i] = G[(int64_t)min(16 * g + h + i, l - 1) * l + cl];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int a = 16 * g + h + i;
        double x = gv[i];
        if (att && c == a) x += shift;
        v[h + i] = (a < l && c >= a && c < l) ? d2f_rn(x) : 0.0f;
      }
    }
    for (int a = tid; a < l; a += blockDim.x)
      s_thr[a] = d2f_rn((double)l * 2.0 * eps * (G[(int64_t)a * l + a] + shift));
    if (tid == 0) s_f = 0;
    __syncthreads();
    for (int jb = 0; jb * 16 < l; ++jb) {
      bool stop = false;
#pragma unroll
      for (int ii = 0; ii < 16; ++ii) {
        const int j = 16 * jb + ii;
        if (j >= l) break;
        const int buf = j & 1;
        if (g == jb && c == j) {
          const float d = v[ii], th = s_thr[j];
          int f = 0;
          if (!isfinite(d) || !isfinite(th)) f = 2;
          else if (!(d > th) || !(d > 0.0f)) f = 1;
          s_f = f;
          s_rs = f ? 1.0f : rsqrtT(d);
        }
        __syncthreads();
        if (s_f) { stop = true; break; }
        if (g == jb) {
          // row j of R (zeros left of the diagonal)
          const float y = (c >= j && c < l) ? v[ii] * s_rs : 0.0f;
          if (c >= j && c < l) rowbuf[buf][c] = y;
          if (c < l) R[(int64_t)j * l + c] = f2d(y);
          if (c >= j && c < 16 * jb + 16) s_blk[jb][ii][c - 16 * jb] = y;
          if (pack && c < (l + kB - 1) / kB * kB) pack[(size_t)j * ((l + kB - 1) / kB * kB) + c] = y;  // padded to lpad columns
        }
        __syncthreads();
        // this warp's columns are (c & ~31) .. (c | 31)
        if (g >= jb && (c | 31) > j && (c | 31) >= 16 * g && (c & ~31) < l) {
          const float rjc = rowbuf[buf][c];
          const float4 *rb4 = reinterpret_cast<const float4 *>(&rowbuf[buf][16 * g]);
          if (g > jb) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float4 r4 = rb4[q];
              v[4 * q] = fmaf(-r4.x, rjc, v[4 * q]);
              v[4 * q + 1] = fmaf(-r4.y, rjc, v[4 * q + 1]);
              v[4 * q + 2] = fmaf(-r4.z, rjc, v[4 * q + 2]);
              v[4 * q + 3] = fmaf(-r4.w, rjc, v[4 * q + 3]);
            }
          } else {
            // the group's own rows below row j (ii is known at compile time)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              if (4 * q + 3 <= ii) continue;
              const float4 r4 = rb4[q];
              const float ra[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
              for (int k = 0; k < 4; ++k)
                if (4 * q + k > ii) v[4 * q + k] = fmaf(-ra[k], rjc, v[4 * q + k]);
            }
          }
        }
      }
      if (stop) break;
    }
    fail = s_f;
    __syncthreads();
    if (fail == 1 && att == 0) continue;  // the FP32 pass shifts silently
    break;
  }
  if (tid == 0) {
    if (fail == 2) set_status(ctrl, RQLP_ERR_NONFINITE);
    else if (fail == 1) set_status(ctrl, RQLP_ERR_RANK_DEFICIENT);
  }
  // inverses of the 16 x 16 diagonal blocks in FP32, one warp per block
  const int nblk = (l + kB - 1) / kB;
  for (int bk = warp; bk < nblk; bk += (int)(blockDim.x >> 5)) {
    const int c0 = bk * kB, bs = min(kB, l - c0);
    const int cc = lane;
    auto U = [&](int i, int t) { return s_blk[bk][i][t]; };
    const float dl = (lane < bs) ? 1.0f / U(lane, lane) : 0.0f;
    float x[kB];
#pragma unroll
    for (int i = 0; i < kB; ++i) x[i] = 0.0f;
#pragma unroll
    for (int i = kB - 1; i >= 0; --i) {
      const float di = __shfl_sync(0xffffffffu, dl, i);
      if (i < bs && cc < bs && i <= cc) {
        float sacc = (i == cc) ? 1.0f : 0.0f;
#pragma unroll
        for (int t = i + 1; t < kB; ++t)
          if (t <= cc && t < bs) sacc = fmaf(-U(i, t), x[t], sacc);
        x[i] = sacc * di;
      }
    }
    if (cc < bs)
#pragma unroll
      for (int i = 0; i < kB; ++i)
        if (i < bs) Dinv[(int64_t)(c0 + i) * l + c0 + cc] = f2d(x[i]);
    if (pack && cc < kB) {
      // the block inverse in FP32: rows c0 .. c0 + 15 of the [lpad][16] panel
      float *dp = pack + (size_t)l * ((l + kB - 1) / kB * kB) + (size_t)c0 * kB;
#pragma unroll
      for (int i = 0; i < kB; ++i) dp[i * kB + cc] = (i < bs && cc < bs) ? x[i] : 0.0f;
    }
  }
}

size_t chol_cluster_smem(int l) {
  return (size_t)l * (l + 1) / 2 * sizeof(double) + 2 * (size_t)l * 8 + (size_t)l * sizeof(double);
}

template <int C, int RMAX>
cudaError_t launch_chol_cluster(const double *G, int l, int64_t rows, double *R, double *Dinv,
                                Ctrl *ctrl, int site, const int *skip_unless, cudaStream_t st,
                                double again_tol, double eps) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(l <= 128 ? 128 : 256);
  cfg.dynamicSmemBytes = chol_cluster_smem(l);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_chol_cluster<C, RMAX>, G, l, (double)rows, R,
                                           Dinv, ctrl, site, skip_unless, again_tol, eps,
                                           (unsigned long long)kDefaultSpinNs);
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

template <int C, int RMAX>
cudaError_t chol_cluster_attr() {
  cudaError_t e = cudaFuncSetAttribute(k_chol_cluster<C, RMAX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)chol_cluster_smem(kClusterMaxL));
  if (e == cudaSuccess && C > 8)
    e = cudaFuncSetAttribute(k_chol_cluster<C, RMAX>,
                             cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

// kernel attributes of the cluster Cholesky (once) and the cluster size it
// uses by default: 16 CTAs where a 16-CTA cluster of it fits, else 8
int chol_cluster_init() {
  static int best = 0;
  if (best == 0) {
    if (chol_cluster_attr<8, 16>() != cudaSuccess || chol_cluster_attr<8, 28>() != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    best = 8;
    if (chol_cluster_attr<16, 8>() == cudaSuccess && chol_cluster_attr<16, 14>() == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(16);
      cfg.blockDim = dim3(256);
      cfg.dynamicSmemBytes = chol_cluster_smem(kClusterMaxL);
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 16;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, k_chol_cluster<16, 14>, &cfg) == cudaSuccess && n > 0)
        best = 16;
    }
    cudaGetLastError();
  }
  return best;
}

constexpr int kApplyRows = 32;
constexpr int kApplyThreads = 128;

// Q (rows x l, ldq) = X R^{-1}, blocked over 16 columns; X and Q may not alias.
// T = float: X, R and the block inverses are rounded to FP32 and the solve
// runs in FP32 (Q is written in FP64).  PRE: R (padded to lpad = a multiple of
// 16 columns) and the diagonal block inverses are staged in shared memory
// once, instead of one block column per step (FP32 is latency-bound on those
// loads, FP64 on its FMAs).
template <typename T, bool PRE>
__global__ void __launch_bounds__(kApplyThreads)
k_apply_trsm(const double *__restrict__ X, int64_t rows, int l, int64_t ldx,
             const double *__restrict__ R, const double *__restrict__ Dinv, double *__restrict__ Q,
             int64_t ldq, const int *skip_unless, const float *__restrict__ pack) {
  if (skip_unless && *reinterpret_cast<const volatile int *>(skip_unless) == 0) return;
  extern __shared__ double sm_raw[];
  T *sm = reinterpret_cast<T *>(sm_raw);
  const int lp = l + 1;
  const int lpad = (l + kB - 1) / kB * kB;
  T *qs = sm;                                  // [kApplyRows][lp]
  T *rc = sm + kApplyRows * lp;                // [l][kB] block column of R, or PRE: R [l][lpad]
  T *dv = PRE ? rc + (int64_t)l * lpad : rc + (int64_t)l * kB;  // [kB][kB], or PRE: [lpad][kB]
  if (PRE && sizeof(T) == 4 && pack) {
    // R and the block inverses, already FP32 in this layout: 16-byte copies,
    // all in flight at once (rc and dv are contiguous, 16-byte aligned)
    const int n4 = (l * lpad + lpad * kB) / 4;
    const unsigned s0 = (unsigned)__cvta_generic_to_shared(rc);
    for (int e = threadIdx.x; e < n4; e += blockDim.x)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s0 + 16u * (unsigned)e),
                   "l"(pack + 4 * (int64_t)e)
                   : "memory");
  } else if (PRE) {
    stage_smem<T>(
        l * lpad, R,
        [&](int e) -> const double * {
          const int t = e / lpad, j = e - t * lpad;
          return j < l ? R + (int64_t)t * l + j : nullptr;
        },
        [&](int e) { return rc + e; });
    stage_smem<T>(
        lpad * kB, R,
        [&](int e) -> const double * {
          const int i = e / kB, j = e - i * kB, c0 = i / kB * kB;
          return (i < l && c0 + j < l) ? Dinv + (int64_t)i * l + c0 + j : nullptr;
        },
        [&](int e) { return dv + e; });
  }
  const int64_t r0 = (int64_t)blockIdx.x * kApplyRows;
  const int nr = (int)min((int64_t)kApplyRows, rows - r0);
  stage_smem<T>(
      kApplyRows * l, X,
      [&](int e) -> const double * {
        const int r = e / l, c = e - r * l;
        return r < nr ? X + (r0 + r) * ldx + c : nullptr;
      },
      [&](int e) {
        const int r = e / l, c = e - r * l;
        return qs + r * lp + c;
      });
  if (PRE && (sizeof(T) == 8 || pack)) cp_async_wait_all();  // the loop's first barrier follows
  // lane -> row r, warp -> columns j0..j0+3 of the block: every lane of a
  // warp needs the same rows of inv(R[b, b]), so the triangular product
  // stops at row j0 + 3 for the whole warp
  const int r = threadIdx.x & 31, j0 = (threadIdx.x >> 5) * 4;
  for (int c0 = 0; c0 < l; c0 += kB) {
    const int bs = min(kB, l - c0);
    __syncthreads();
    if (!PRE) {
      stage_smem<T>(
          c0 * kB, R,
          [&](int e) -> const double * {
            const int t = e / kB, j = e - t * kB;
            return j < bs ? R + (int64_t)t * l + c0 + j : nullptr;
          },
          [&](int e) { return rc + e; });
      stage_smem<T>(
          kB * kB, R,
          [&](int e) -> const double * {
            const int i = e / kB, j = e - i * kB;
            return (i < bs && j < bs) ? Dinv + (int64_t)(c0 + i) * l + c0 + j : nullptr;
          },
          [&](int e) { return dv + e; });
      // (the FP64 copies of this block and, at c0 = 0, of the X tile)
      if (sizeof(T) == 8) cp_async_wait_all();
      __syncthreads();
    }
    const T *rcb = PRE ? rc + c0 : rc;           // rcb[t * rstride + j] = R(t, c0 + j)
    const int rstride = PRE ? lpad : kB;
    const T *dvb = PRE ? dv + (int64_t)c0 * kB : dv;  // dvb[i * kB + j] = inv(R_bb)(i, j)
    T acc[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) acc[a] = (j0 + a < bs) ? qs[r * lp + c0 + j0 + a] : (T)0;
    for (int t = 0; t < c0; ++t) {
      const T qv = qs[r * lp + t];
#pragma unroll
      for (int a = 0; a < 4; ++a) acc[a] = fma(-qv, rcb[t * rstride + j0 + a], acc[a]);
    }
    // share the 16 residuals of row r, then multiply by the inverse block
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a)
      if (j0 + a < bs) qs[r * lp + c0 + j0 + a] = acc[a];
    __syncthreads();
    T out[4] = {(T)0, (T)0, (T)0, (T)0};
    const int iend = min(bs, j0 + 4);  // inv(R[b, b]) is upper triangular
    for (int i = 0; i < iend; ++i) {
      const T v = qs[r * lp + c0 + i];
#pragma unroll
      for (int a = 0; a < 4; ++a) out[a] = fma(v, dvb[i * kB + j0 + a], out[a]);
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a)
      if (j0 + a < bs) qs[r * lp + c0 + j0 + a] = out[a];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nr * l; e += blockDim.x) {
    const int rr = e / l, c = e - rr * l;
    Q[(r0 + rr) * ldq + c] = (double)qs[rr * lp + c];
  }
}

}  // namespace

size_t f32_pack_floats(int l) {
  const size_t lpad = (size_t)(l + kB - 1) / kB * kB;
  return (size_t)l * lpad + lpad * kB;
}

cudaError_t cholqr_init() {
  cudaError_t e = cudaFuncSetAttribute(k_gram_sym<double>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_gram_sym<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             100 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_chol_blocked<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_chol_blocked<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_apply_trsm<double, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_apply_trsm<float, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_apply_trsm<float, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e == cudaSuccess && chol_cluster_init() < 0) e = cudaErrorInvalidValue;
  return e;
}

// Rows per Gram chunk: two chunks per SM where that gives 8..32 rows, so
// that every SM gets the same number of rows (no partial second wave).
int gram_rows_per_chunk(int64_t rows) {
  const int64_t target = 2LL * num_sms();
  const int64_t r = (rows + target - 1) / target;
  return (int)std::max<int64_t>(8, std::min<int64_t>(kGramMaxRows, r));
}

int64_t gram_chunks(int64_t rows) {
  const int rc = gram_rows_per_chunk(rows);
  return (rows + rc - 1) / rc;
}

// bound on gram_chunks(r) for every r <= rows_max
int64_t gram_chunks_max(int64_t rows_max) {
  return std::max<int64_t>(2LL * num_sms(), (rows_max + kGramMaxRows - 1) / kGramMaxRows);
}

cudaError_t gram_sym(const double *X, int64_t rows, int l, int64_t ldx, double *part, double *G,
                     const int *skip_unless, cudaStream_t st, bool lowp) {
  const int rc = gram_rows_per_chunk(rows);
  const int64_t chunks = gram_chunks(rows);
  const int lp = ((l + 3) / 4) * 4 + 1;
  const size_t smem = (size_t)rc * lp * (lowp ? sizeof(float) : sizeof(double));
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_gram_sym<double>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_gram_sym<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               100 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (lowp)
    k_gram_sym<float><<<(unsigned)chunks, kGramThreads, smem, st>>>(X, rows, l, ldx, rc, part,
                                                                    skip_unless);
  else
    k_gram_sym<double><<<(unsigned)chunks, kGramThreads, smem, st>>>(X, rows, l, ldx, rc, part,
                                                                     skip_unless);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_gram_reduce<<<(unsigned)(((int64_t)l * l + 31) / 32), dim3(32, kReduceY), 0, st>>>(
      part, (int)chunks, l, G, skip_unless);
  count_launch();
  return cudaGetLastError();
}

cudaError_t chol_blocked(const double *G, int l, int64_t rows, double *R, double *Dinv, Ctrl *ctrl,
                         int site, const int *skip_unless, cudaStream_t st, double again_tol,
                         double eps, bool lowp, float *pack) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_chol_blocked<double>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_chol_blocked<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               200 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int threads = ((l * l / 24) + 31) / 32 * 32;
  threads = std::max(128, std::min(512, threads));
  // FP32 pass: one CTA, registers and FP32 only (its column chain is a few
  // FP32 operations and two barriers)
  if (lowp && l <= kChol32MaxL && again_tol < 0.0) {
    k_chol_f32<<<1, 1024, 0, st>>>(G, l, (double)rows, R, Dinv, ctrl, site, skip_unless, eps,
                                   pack);
    count_launch();
    return cudaGetLastError();
  }
  const int best = chol_cluster_init();
  if (best < 0) return cudaErrorInvalidValue;
  const int cc = l > kClusterMaxL ? 1 : (tuning().chol_ctas > 0 ? tuning().chol_ctas : best);
  if (cc == 16)
    return l <= 128 ? launch_chol_cluster<16, 8>(G, l, rows, R, Dinv, ctrl, site, skip_unless, st,
                                                 again_tol, eps)
                    : launch_chol_cluster<16, 14>(G, l, rows, R, Dinv, ctrl, site, skip_unless, st,
                                                  again_tol, eps);
  if (cc == 8)
    return l <= 128 ? launch_chol_cluster<8, 16>(G, l, rows, R, Dinv, ctrl, site, skip_unless, st,
                                                 again_tol, eps)
                    : launch_chol_cluster<8, 28>(G, l, rows, R, Dinv, ctrl, site, skip_unless, st,
                                                 again_tol, eps);
  const size_t smem = (size_t)l * l * sizeof(double);
  const bool use_smem = smem <= 200 * 1024;
  k_chol_blocked<double><<<1, threads, use_smem ? smem : 0, st>>>(
      G, l, (double)rows, R, Dinv, ctrl, site, skip_unless, use_smem ? 1 : 0, again_tol, eps);
  count_launch();
  return cudaGetLastError();
}

cudaError_t apply_trsm(const double *X, int64_t rows, int l, int64_t ldx, const double *R,
                       const double *Dinv, double *Q, int64_t ldq, const int *skip_unless,
                       cudaStream_t st, bool lowp, const float *pack) {
  const int lpad = (l + kB - 1) / kB * kB;
  const size_t base = (size_t)kApplyRows * (l + 1);
  const size_t smem_pre = (base + (size_t)l * lpad + (size_t)lpad * kB) * sizeof(float);
  const bool pre = lowp && smem_pre <= 150 * 1024;
  const size_t smem = pre ? smem_pre
                          : (base + (size_t)l * kB + kB * kB) * (lowp ? sizeof(float)
                                                                       : sizeof(double));
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_apply_trsm<double, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_apply_trsm<float, false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_apply_trsm<float, true>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int64_t tiles = (rows + kApplyRows - 1) / kApplyRows;
  // the pack exists only where the FP32 Cholesky of chol_blocked wrote it
  if (l > kChol32MaxL) pack = nullptr;
  if (pre)
    k_apply_trsm<float, true><<<(unsigned)tiles, kApplyThreads, smem, st>>>(
        X, rows, l, ldx, R, Dinv, Q, ldq, skip_unless, pack);
  else if (lowp)
    k_apply_trsm<float, false><<<(unsigned)tiles, kApplyThreads, smem, st>>>(
        X, rows, l, ldx, R, Dinv, Q, ldq, skip_unless, nullptr);
  else
    k_apply_trsm<double, false><<<(unsigned)tiles, kApplyThreads, smem, st>>>(
        X, rows, l, ldx, R, Dinv, Q, ldq, skip_unless, nullptr);
  count_launch();
  return cudaGetLastError();
}

}  // namespace rqk
