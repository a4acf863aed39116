// Column-pivoted Householder QR of the wide l x n matrix B
// (Algorithm 2.1 step 5 / Algorithm 2.2 step 5, "cpqr(B)").
//
// One persistent cooperative kernel.  CTA b owns a contiguous slab of
// columns of B (each column l doubles), kept in shared memory when it fits
// and in a global scratch copy otherwise.  Per pivot step s there is exactly
// one grid barrier:
//   1. the winner of step s (largest trailing norm, ties to the lowest
//      original column index) was picked by the last CTA to arrive at the
//      barrier; every CTA polls its two tagged records: the CTA that holds
//      it, x0 and the exact ||x(s+1:)||^2 of its column;
//   2. every CTA builds the same Householder reflector from the winner's
//      column, mapping it to +alpha e_s (non-negative R(s, s)), while it
//      loads that column;
//   3. every CTA forms v^T col for its unpivoted columns (4 lanes per column)
//      from the unscaled column, v^T col = col(s) + (x(s+1:)^T col(s+1:)) /
//      (x0 - alpha), and the downdated norms ||col(s+1:)||^2 =
//      ||col(s:)||^2 - col'(s)^2 (recomputed exactly after more than 99 %
//      cancellation);
//   4. it updates its best column for step s + 1, publishes it (norm, index,
//      exact trailing sigma, the column from row s + 1) and arrives at the
//      barrier;
//   5. the rest of its axpys col -= (v^T col) tau v run while the barrier
//      completes.
// Candidate tables and columns are double-buffered by step parity, so one
// barrier per step suffices.  The winner records need one copy: the record
// of barrier k + 1 is written only after every CTA has read that of k.  After l steps the unchosen columns are written in their
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
  double2 *cand;      // [2][G][2]: (norm^2, index as a 64-bit integer), (sigma, x0)
  unsigned *arrive;   // barrier counter, alone in its 128-byte line
  unsigned long long *rec;  // [G][16]: CTA c's winner records in line c
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

// (norm, index) of the better of this lane's pair and its xor partners'
__device__ __forceinline__ void warp_best(double &bn, int &bi) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double on = __shfl_xor_sync(0xffffffffu, bn, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (better(on, oi, bn, bi)) { bn = on; bi = oi; }
  }
}

// Grid barriers count arrivals on one counter that the host zeroes, with the
// winner records, before every launch.  At step barrier k (k = 1, 2, ...)
// the k G-th arriver reads the whole candidate table, picks the winner and
// writes it to every CTA as two 128-bit records tagged with k, one with sigma
// and one with x0, in a 128-byte line of that CTA's own.  Each CTA polls its
// records (a 128-bit access is a single access, so a record whose tag
// matches carries that barrier's data): no second round trip after polling a
// counter, and no line that all CTAs poll while the arrivals' atomics hit it.
// Every wait is bounded by limit_ns; an error recorded by another CTA ends
// it.  `extra` (only the timeout test sets it) makes the first wait need a
// tag or arrivals that never come.
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned *p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void red_add_release(unsigned *p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// (a fence.acq_rel.gpu before these stores makes them releases)
__device__ __forceinline__ void st_relaxed_b128(unsigned long long *p, unsigned long long lo,
                                                unsigned long long hi) {
  asm volatile("{\n .reg .b128 t;\n mov.b128 t, {%1, %2};\n st.relaxed.gpu.global.b128 [%0], t;\n}"
               ::"l"(p), "l"(lo), "l"(hi) : "memory");
}
__device__ __forceinline__ void ld_acquire_b128(const unsigned long long *p, unsigned long long &lo,
                                                unsigned long long &hi) {
  asm volatile("{\n .reg .b128 t;\n ld.acquire.gpu.global.b128 t, [%2];\n mov.b128 {%0, %1}, t;\n}"
               : "=l"(lo), "=l"(hi) : "l"(p) : "memory");
}
__device__ __forceinline__ void ld_relaxed_b128(const unsigned long long *p, unsigned long long &lo,
                                                unsigned long long &hi) {
  asm volatile("{\n .reg .b128 t;\n ld.relaxed.gpu.global.b128 t, [%2];\n mov.b128 {%0, %1}, t;\n}"
               : "=l"(lo), "=l"(hi) : "l"(p) : "memory");
}
// one thread: wait until both records at rec (A at rec, B at rec + 2) carry
// tag (bits 48..63 of their first words).  B is loaded (relaxed) beside each
// acquire load of A, so both are in flight at once; its tag vouches for its
// data, A's acquire for everything the winner's column needs.  False on
// timeout or error.
__device__ __forceinline__ bool wait_records(Ctrl *c, const unsigned long long *rec, unsigned tag,
                                             unsigned long long &a0, unsigned long long &a1,
                                             unsigned long long &b1, unsigned long long limit_ns,
                                             int site) {
  unsigned long long t0 = 0, b0 = 0;
  bool have_a = false;
  for (unsigned it = 0;; ++it) {
    ld_relaxed_b128(rec + 2, b0, b1);
    if (!have_a) {
      ld_acquire_b128(rec, a0, a1);
      have_a = (unsigned)(a0 >> 48) == tag;
    }
    if (have_a && (unsigned)(b0 >> 48) == tag) return true;
    if ((it & 15) == 15) {
      if (ld_volatile_i32(&c->status) < 0) return false;
      const unsigned long long t = globaltimer_ns();
      if (t0 == 0) {
        t0 = t;
      } else if (t - t0 > limit_ns) {
        set_status(c, RQLP_ERR_TIMEOUT);
        atomicExch(&c->timeout_site, site);
        return false;
      }
    }
  }
}
// lane-0 wait until the counter reaches target; false on timeout or error
__device__ __forceinline__ bool wait_count(Ctrl *c, const unsigned *counter, unsigned target,
                                           unsigned long long limit_ns, int site) {
  unsigned long long t0 = 0;
  for (unsigned it = 0; (int)(ld_acquire_u32(counter) - target) < 0; ++it) {
    if ((it & 15) == 15) {
      if (ld_volatile_i32(&c->status) < 0) return false;
      const unsigned long long t = globaltimer_ns();
      if (t0 == 0) {
        t0 = t;
      } else if (t - t0 > limit_ns) {
        set_status(c, RQLP_ERR_TIMEOUT);
        atomicExch(&c->timeout_site, site);
        return false;
      }
    }
  }
  return true;
}

// USE_SMEM (the slab in shared memory) is a template argument so that the
// compiler addresses the columns as shared memory, not through generic loads.
template <bool USE_SMEM>
__global__ void __launch_bounds__(kThreads) k_cpqr_wide(CpqrParams P) {
  extern __shared__ double sm[];
  __shared__ double s_v[kMaxL];
  __shared__ double s_bn[kWarps];
  __shared__ int s_bi[kWarps];
  __shared__ int s_win_cta, s_win_idx;
  __shared__ double s_sigma, s_x0;
  __shared__ double s_tau, s_beta, s_rv0, s_trv;
  __shared__ int s_ok;

  const int G = gridDim.x, b = blockIdx.x, l = P.l;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t c0 = (int64_t)b * P.cpb;
  const int nc = (int)max((int64_t)0, min(P.n, c0 + P.cpb) - c0);
  double *cols = USE_SMEM ? sm : P.gcols + (int64_t)b * P.cpb * l;
  double *nrm = USE_SMEM ? sm + (int64_t)P.cpb * l : sm;
  // 1% of the norm^2 when it was last computed exactly: below that the
  // downdated value has lost too many digits and is recomputed
  double *thr = nrm + P.cpb;
  double *wdot = thr + P.cpb;  // this step's axpy multiple of x(s+1:) per column
  int *pivoted = reinterpret_cast<int *>(wdot + P.cpb);
  int *axdone = pivoted + P.cpb;                       // column updated early this step

  // Step barrier k (k = 1, 2, ...): G increments.  arrive(): after this
  // CTA's candidate is published; the k G-th arriver reads the whole table
  // and writes the winner records.  Called by warp 0.
  unsigned nsteps = 0;
  // the last arriver of barrier `won` keeps the winner it wrote (lane 0)
  unsigned won = 0;
  unsigned long long won_w0 = 0;
  double won_sigma = 0.0, won_x0 = 0.0;
  auto arrive = [&](int buf) {
    ++nsteps;
    const unsigned done = nsteps * (unsigned)G;
    unsigned old = 0;
    __syncwarp();
    if (lane == 0) old = atom_add_acq_rel(P.arrive, 1u);
    old = __shfl_sync(0xffffffffu, old, 0);
    __syncwarp();
    if (old != done - 1u) return;
    // both halves of every record in one round of loads; the reduction
    // carries (norm, index, CTA), and sigma and x0 come from the lane that
    // holds the winning entry
    double bn = -1.0, bs = 0.0, bx = 0.0;
    int bi = -1, bc = -1;
    if (G <= 160) {
      double2 e[5], f[5];
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const int c = lane + 32 * k;
        e[k] = c < G ? __ldcg(P.cand + 2 * (buf * G + c))
                     : make_double2(-1.0, __longlong_as_double(-1LL));
        f[k] = c < G ? __ldcg(P.cand + 2 * (buf * G + c) + 1) : make_double2(0.0, 0.0);
      }
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        const int ci = (int)__double_as_longlong(e[k].y);
        if (better(e[k].x, ci, bn, bi)) {
          bn = e[k].x; bi = ci; bc = lane + 32 * k; bs = f[k].x; bx = f[k].y;
        }
      }
    } else {
      for (int c = lane; c < G; c += 32) {
        const double2 e = __ldcg(P.cand + 2 * (buf * G + c));
        const double2 f = __ldcg(P.cand + 2 * (buf * G + c) + 1);
        const int ci = (int)__double_as_longlong(e.y);
        if (better(e.x, ci, bn, bi)) { bn = e.x; bi = ci; bc = c; bs = f.x; bx = f.y; }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double on = __shfl_xor_sync(0xffffffffu, bn, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
      if (better(on, oi, bn, bi)) { bn = on; bi = oi; bc = oc; }
    }
    // entry c sits in lane c mod 32, whose own best it is
    bs = __shfl_sync(0xffffffffu, bs, bc & 31);
    bx = __shfl_sync(0xffffffffu, bx, bc & 31);
    const unsigned long long w0 = (unsigned long long)(unsigned)bi |
                                  ((unsigned long long)((unsigned)bc & 0xffffu) << 32) |
                                  ((unsigned long long)(nsteps & 0xffffu) << 48);
    // every lane is ordered after lane 0's acquire (the warp barrier above),
    // so its fence releases what that acquire made visible
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    for (int c = lane; c < G; c += 32) {
      if (c == b) continue;  // this CTA takes the winner from registers
      st_relaxed_b128(P.rec + 16 * (int64_t)c + 2, w0, (unsigned long long)__double_as_longlong(bx));
      st_relaxed_b128(P.rec + 16 * (int64_t)c, w0, (unsigned long long)__double_as_longlong(bs));
    }
    won = nsteps;
    won_w0 = w0;
    won_sigma = bs;
    won_x0 = bx;
  };
  // thread 0: the winner of step barrier k (given here: nsteps counts only
  // in warp 0), from its own registers when this CTA arrived last, else
  // from this CTA's records
  auto wait_winner = [&](int site, unsigned k) {
    if (tid == 0) {
      unsigned long long a0 = won_w0, a1 = (unsigned long long)__double_as_longlong(won_sigma),
                         b1 = (unsigned long long)__double_as_longlong(won_x0);
      bool ok = true;
      if (won != k || P.extra != 0)
        ok = wait_records(P.ctrl, P.rec + 16 * (int64_t)b, (k + P.extra) & 0xffffu, a0, a1, b1,
                          P.limit_ns, site);
      s_ok = ok;
      s_win_idx = (int)(unsigned)(a0 & 0xffffffffULL);
      s_win_cta = (int)((a0 >> 32) & 0xffffULL);
      s_sigma = __longlong_as_double((long long)a1);
      s_x0 = __longlong_as_double((long long)b1);
    }
    __syncthreads();
    return s_ok != 0;
  };
  // plain barrier after the l step barriers
  auto final_sync = [&](int site) {
    __syncthreads();
    if (tid == 0) {
      red_add_release(P.arrive, 1u);
      s_ok = wait_count(P.ctrl, P.arrive, (unsigned)(l + 1) * (unsigned)G + P.extra, P.limit_ns,
                        site);
    }
    __syncthreads();
    return s_ok != 0;
  };
  // warp 0: publish candidate jc (local index, key cn) of the next step,
  // whose column is final through row r0 - 1 once cj x(r0:) (cj != 0: the
  // step's axpy, applied here) is subtracted: the record (cn, index), sigma =
  // ||col(r0 + 1:)||^2 exactly and x0 = col(r0), and the column from row r0 on
  auto publish = [&](int buf, int jc, double cn, int r0, double cj) {
    double sg = 0.0, x0 = 0.0;
    if (jc >= 0) {
      double *col = cols + (int64_t)jc * l;
      double *dst = P.pcol + ((int64_t)buf * G + b) * l;
      for (int r = r0 + lane; r < l; r += 32) {
        double x = col[r];
        if (cj != 0.0) {
          x = fma(-cj, s_v[r - r0 + 1], x);
          col[r] = x;
        }
        dst[r] = x;
        if (r > r0) sg = fma(x, x, sg);
        else x0 = x;  // lane 0
      }
      sg = warp_sum(sg);
    }
    if (lane == 0) {
      P.cand[2 * (buf * G + b)] =
          make_double2(jc >= 0 ? cn : -1.0, __longlong_as_double(jc >= 0 ? (long long)(c0 + jc) : -1LL));
      P.cand[2 * (buf * G + b) + 1] = make_double2(sg, x0);
    }
  };

  // nothing to do after an earlier error (its data may be garbage)
  if (ld_volatile_i32(&P.ctrl->status) < 0) return;

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
      thr[jj] = 0.01 * s;
      pivoted[jj] = 0;
      axdone[jj] = 0;
      if (!isfinite(s)) set_status(P.ctrl, RQLP_ERR_NONFINITE);
    }
  }
  __syncthreads();
  // ---- candidate for step 0 -----------------------------------------------
  {
    double bn = -1.0;
    int bi = -1;
    for (int jj = tid; jj < nc; jj += kThreads)
      if (better(nrm[jj], (int)(c0 + jj), bn, bi)) { bn = nrm[jj]; bi = (int)(c0 + jj); }
    warp_best(bn, bi);
    if (lane == 0) { s_bn[warp] = bn; s_bi[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      double cn = s_bn[0];
      int ci = s_bi[0];
      for (int w = 1; w < kWarps; ++w)
        if (better(s_bn[w], s_bi[w], cn, ci)) { cn = s_bn[w]; ci = s_bi[w]; }
      publish(0, ci >= 0 ? (int)(ci - c0) : -1, cn, 0, 0.0);
      arrive(0);
    }
  }
  if (!wait_winner(1, 1u)) return;

  const int sub = lane >> 2, gl = lane & 3;
  for (int s = 0; s < l; ++s) {
    const int buf = s & 1;
    // ---- 1. winner (picked by the last CTA to arrive) and its sigma ----
    const int wc = s_win_cta, wi = s_win_idx;
    if (wi < 0 || wc < 0 || wc >= G) {
      if (tid == 0) set_status(P.ctrl, RQLP_ERR_INVALID_ARG);
      return;
    }
    // ---- 2. reflector from the winner's column, rows s..l-1 ----
    // one thread forms H = I - tau v v^T with v(0) = 1 and H x = alpha e_1,
    // alpha = ||x|| >= 0: tau = 1 - x0/alpha, v(1:) = x(1:) / (x0 - alpha),
    // where x0 > 0 uses x0 - alpha = -sigma / (x0 + alpha) (no cancellation);
    // x0 and sigma = ||x(1:)||^2 came with the winner's record, so this runs
    // while the other threads load the column
    if (tid == 0) {
      const double x0 = s_x0, sigma = s_sigma;
      double tau, beta, rv0;
      if (sigma == 0.0) {
        if (x0 >= 0.0) { tau = 0.0; beta = x0; }
        else { tau = 2.0; beta = -x0; }
        rv0 = 0.0;
      } else {
        const double isig = rcp_fast(sigma);
        const double n2 = fma(x0, x0, sigma);
        const double ra = rsqrt_fast(n2);  // 1 / alpha
        const double alpha = n2 * ra;
        if (x0 <= 0.0) {
          rv0 = rcp_fast(x0 - alpha);
          tau = fma(-x0, ra, 1.0);
        } else {
          const double t = x0 + alpha;
          rv0 = -t * isig;
          tau = (sigma * ra) * rcp_fast(t);
        }
        beta = alpha;
      }
      s_tau = tau;
      s_beta = beta;
      s_rv0 = rv0;
      s_trv = tau * rv0;
    }
    // warps 1.. load the column meanwhile
    const double *xc = P.pcol + ((int64_t)buf * G + wc) * l;
    if (warp > 0)
      for (int r = s + tid - 32; r < l; r += kThreads - 32) s_v[r - s] = __ldcg(xc + r);
    __syncthreads();
    // s_v holds the winner's column x(s:) unscaled; v = (1, x(s+1:) rv0)
    const double tau = s_tau, beta = s_beta, rv0 = s_rv0, trv = s_trv;
    // the winner's column is final: rows < s from the slab, beta at s, zeros below
    if ((int)(wi - c0) >= 0 && (int)(wi - c0) < nc && warp == 0) {
      const int jw = (int)(wi - c0);
      const double *col = cols + (int64_t)jw * l;
      double *out = P.R0t + (int64_t)s * P.ldr;
      for (int r = lane; r < l; r += 32) out[r] = (r < s) ? col[r] : (r == s ? beta : 0.0);
      if (lane == 0) { pivoted[jw] = 1; nrm[jw] = -1.0; }
    }
    // ---- 3. dot products v^T col and downdated norms (the axpys wait) ----
    // groups of 4 lanes per column, eight columns per warp: every FP64 warp
    // instruction costs the same issue slots whatever its active lanes, so
    // the reductions are kept short (two levels).  v^T col = col(s) +
    // rv0 x(s+1:)^T col(s+1:); the new col(s) is stored at once, and the
    // axpy of rows s+1.. is col -= ((v^T col) tau rv0) x, with that multiple
    // kept in wdot.  A column whose norm has cancelled by more than 99 % since
    // its last exact value is updated now and its norm recomputed.
    double bn = -1.0;
    int bi = -1;
    for (int jb = warp * 8; jb < nc; jb += kWarps * 8) {
      const int jj = jb + sub;
      const bool act = jj < nc && !pivoted[jj] && (int)(c0 + jj) != wi;
      double *col = cols + (int64_t)(act ? jj : 0) * l;
      double d = 0.0;
      if (act)
        for (int r = s + 1 + gl; r < l; r += 4) d = fma(s_v[r - s], col[r], d);
      d += __shfl_xor_sync(0xffffffffu, d, 2);
      d += __shfl_xor_sync(0xffffffffu, d, 1);
      int need = 0;
      double nd = 0.0, cf = 0.0;
      if (act && gl == 0) {
        const double cs = col[s];
        const double w = fma(rv0, d, cs);     // v^T col
        const double rsv = fma(-w, tau, cs);  // new col(s)
        col[s] = rsv;
        cf = w * trv;
        wdot[jj] = cf;
        axdone[jj] = 0;
        nd = fma(-rsv, rsv, nrm[jj]);
        need = __double_as_longlong(nd) <= __double_as_longlong(thr[jj]);
      }
      need = __shfl_sync(0xffffffffu, need, lane & ~3);
      // warp-uniform branch: the shuffles inside need every lane
      if (__any_sync(0xffffffffu, need)) {
        cf = __shfl_sync(0xffffffffu, cf, lane & ~3);
        if (need)
          for (int r = s + 1 + gl; r < l; r += 4) col[r] = fma(-cf, s_v[r - s], col[r]);
        __syncwarp();
        double t = 0.0;
        if (need)
          for (int r = s + 1 + gl; r < l; r += 4) t = fma(col[r], col[r], t);
        t += __shfl_xor_sync(0xffffffffu, t, 2);
        t += __shfl_xor_sync(0xffffffffu, t, 1);
        if (need) nd = t;
      }
      if (act && gl == 0) {
        nrm[jj] = nd;
        if (need) {
          thr[jj] = 0.01 * nd;
          axdone[jj] = 1;
        }
        if (better(nd, (int)(c0 + jj), bn, bi)) { bn = nd; bi = (int)(c0 + jj); }
      }
    }
    warp_best(bn, bi);
    if (lane == 0) { s_bn[warp] = bn; s_bi[warp] = bi; }
    __syncthreads();
    // this CTA's candidate for step s + 1 (every thread reads the same table)
    int jc = -1;
    double cn = -1.0;
    if (s + 1 < l) {
      int ci = -1;
      for (int w = 0; w < kWarps; ++w)
        if (better(s_bn[w], s_bi[w], cn, ci)) { cn = s_bn[w]; ci = s_bi[w]; }
      jc = ci >= 0 ? (int)(ci - c0) : -1;
    }
    // ---- 4. warp 0: update the candidate, publish it, arrive ----
    if (warp == 0 && s + 1 < l) {
      publish(buf ^ 1, jc, cn, s + 1, (jc >= 0 && !axdone[jc]) ? wdot[jc] : 0.0);
      arrive(buf ^ 1);
    }
    // ---- 5. the remaining axpys, while the barrier completes ----
    // (warps 1..: warp 0 goes from its arrival, and the last arriver's
    // scan, straight to the next wait)
    if (b == 0 && warp == kWarps - 1) {
      // this step's reflector, off the path to the barrier
      for (int r = lane; r < l; r += 32)
        P.Vh[(int64_t)r * l + s] = (r < s) ? 0.0 : (r == s ? 1.0 : s_v[r - s] * rv0);
      if (lane == 0) { P.tau[s] = tau; P.piv[s] = wi; }
    }
    for (int jb = (warp - 1) * 8; warp > 0 && jb < nc; jb += (kWarps - 1) * 8) {
      const int jj = jb + sub;
      if (jj < nc && !pivoted[jj] && (int)(c0 + jj) != wi && jj != jc && !axdone[jj]) {
        double *col = cols + (int64_t)jj * l;
        const double cf = wdot[jj];
        for (int r = s + 1 + gl; r < l; r += 4) col[r] = fma(-cf, s_v[r - s], col[r]);
      }
    }
    // (the wait's own barrier orders these axpys before the next column load)
    if (s + 1 < l && !wait_winner(2, (unsigned)(s + 2))) return;
  }

  // ---- unchosen columns keep their order behind the l pivots ----
  int mine = 0;
  if (tid == 0) {
    for (int jj = 0; jj < nc; ++jj) mine += pivoted[jj] ? 0 : 1;
    P.counts[b] = mine;
  }
  __syncthreads();
  if (!final_sync(3)) return;
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
      if (un && pos + rank < P.n) {
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
    if (dst >= P.n) continue;
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
  const size_t state = (size_t)cpb * (3 * sizeof(double) + 2 * sizeof(int));
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
  b += 128 + 128 * G;  // counter line, one record line per CTA
  b += 4 * G * sizeof(double2);
  b += 2 * G * (size_t)l * sizeof(double);
  b += G * sizeof(int32_t);
  b += (size_t)(n + kMaxGrid) * l * sizeof(double);  // global slabs (fallback)
  return b + 8192;
}

size_t cpqr_scratch_bytes_smem_only(int64_t n, int l, bool *fits) {
  const Plan pl = plan_for(n, l);
  *fits = pl.use_smem != 0 && pl.G <= kMaxGrid;
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  return up(128 + 128 * (size_t)pl.G) + up(4 * (size_t)pl.G * sizeof(double2)) +
         up(2 * (size_t)pl.G * l * sizeof(double)) + up((size_t)pl.G * sizeof(int32_t));
}

cudaError_t cpqr_wide(const double *Bt, int64_t n, int l, int64_t ldb, double *R0t, int64_t ldr,
                      int32_t *piv, double *Vh, double *tau, void *scratch, Ctrl *ctrl,
                      unsigned long long limit_ns, unsigned debug_extra, cudaStream_t st) {
  if (n <= 0 || l <= 0 || l > kMaxL || l > n) return cudaErrorInvalidValue;
  Plan pl = plan_for(n, l);
  if (pl.G > kMaxGrid) return cudaErrorInvalidValue;
  void *kfn = pl.use_smem ? (void *)k_cpqr_wide<true> : (void *)k_cpqr_wide<false>;
  cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)std::max<size_t>(pl.smem, 1));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kThreads, pl.smem);
  if (e != cudaSuccess) return e;
  if ((int64_t)per_sm * num_sms() < pl.G) return cudaErrorCooperativeLaunchTooLarge;

  char *p = reinterpret_cast<char *>(scratch);
  auto take = [&](size_t bytes) { char *r = p; p += (bytes + 255) / 256 * 256; return r; };
  CpqrParams P;
  P.Bt = Bt; P.n = n; P.l = l; P.ldb = ldb; P.R0t = R0t; P.ldr = ldr; P.piv = piv;
  P.Vh = Vh; P.tau = tau;
  const size_t sync_bytes = 128 + 128 * (size_t)pl.G;
  char *sync = take(sync_bytes);
  P.arrive = reinterpret_cast<unsigned *>(sync);
  P.rec = reinterpret_cast<unsigned long long *>(sync + 128);
  P.cand = reinterpret_cast<double2 *>(take(4 * (size_t)pl.G * sizeof(double2)));
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
  // barrier counter and winner records of this launch
  e = cudaMemsetAsync(sync, 0, sync_bytes, st);
  if (e != cudaSuccess) return e;
  if (pl.G == 1) {
    // one CTA: its grid barrier never waits, no co-residency is needed
    if (pl.use_smem)
      k_cpqr_wide<true><<<1, kThreads, pl.smem, st>>>(P);
    else
      k_cpqr_wide<false><<<1, kThreads, pl.smem, st>>>(P);
    count_launch();
    return cudaGetLastError();
  }
  void *args[] = {&P};
  e = cudaLaunchCooperativeKernel((const void *)kfn, dim3(pl.G), dim3(kThreads), args, pl.smem,
                                  st);
  count_launch();
  return e;
}

}  // namespace rqk
