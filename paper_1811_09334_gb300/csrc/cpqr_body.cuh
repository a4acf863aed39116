// The pivot-step loop of the column-pivoted Householder QR of B (cpqr.cu):
// one CTA of kThreads threads, CTA b of G.  The kernel of cpqr.cu runs it on
// a grid of G CTAs; the persistent batch kernel runs it with G = 1 inside one
// work item.  The algorithm and the exchange are described in cpqr.cu.
#pragma once

#include "kernels.cuh"

namespace rqk {
namespace cpqrk {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxGrid = 1024;
// 16-byte words per CTA record: (norm, index | k << 32), (sigma, k << 32),
// (x0, k << 32), unused
constexpr int kRecWords = 4;

struct CpqrParams {
  const double *Bt;
  int64_t n;
  int l;              // column length (rows of the matrix whose columns are the rows of Bt)
  int steps;          // pivot steps, <= l (l for the full QR; fewer for a truncated one)
  int ldv;            // leading dimension of Vh (l x steps)
  int64_t ldb;
  double *R0t;
  int64_t ldr;
  int32_t *piv;
  double *Vh;
  double *tau;
  unsigned *arrive;   // arrivals since the launch began, alone in its 128-byte line
  ulonglong2 *win;    // [G][8]: CTA c's winner words in line c
  ulonglong2 *rec;    // [2][G][kRecWords] tagged candidate records
  ulonglong2 *pcol;   // [2][G][l] tagged words (value, k << 32)
  double *gcols;      // G * cpb * l when the slab does not fit in shared memory
  Ctrl *ctrl;
  unsigned long long limit_ns;
  unsigned extra;
  int cpb;
  int use_smem;
  const int32_t *fpiv;  // given pivots (original column indices of steps 0..l-1), or null
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

// Selection key of column `idx` for step s: its trailing norm^2, or with
// given pivots 1 for the step's given column and 0 for every other one (the
// exchange then elects the given column; ties among the others go to the
// lowest index as usual and never win).
__device__ __forceinline__ double pick_key(const int32_t *fpiv, int s, int idx, double nrm2) {
  if (!fpiv) return nrm2;
  return (idx == __ldg(fpiv + s)) ? 1.0 : 0.0;
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

// tagged words: relaxed 128-bit stores and loads at GPU scope
__device__ __forceinline__ void st_word(ulonglong2 *p, unsigned long long v, unsigned long long t) {
  asm volatile("{\n .reg .b128 q;\n mov.b128 q, {%1, %2};\n st.relaxed.gpu.global.b128 [%0], q;\n}"
               ::"l"(p), "l"(v), "l"(t) : "memory");
}
__device__ __forceinline__ ulonglong2 ld_word(const ulonglong2 *p) {
  ulonglong2 w;
  asm volatile("{\n .reg .b128 q;\n ld.relaxed.gpu.global.b128 q, [%2];\n mov.b128 {%0, %1}, q;\n}"
               : "=l"(w.x), "=l"(w.y) : "l"(p) : "memory");
  return w;
}
__device__ __forceinline__ unsigned tag_of(const ulonglong2 &w) { return (unsigned)(w.y >> 32); }
__device__ __forceinline__ unsigned long long dbits(double x) {
  return (unsigned long long)__double_as_longlong(x);
}
__device__ __forceinline__ double dval(unsigned long long b) {
  return __longlong_as_double((long long)b);
}

// A bounded wait, checked by one thread every 16th round: true once an error
// is recorded (here or by another CTA) or limit_ns has passed since the first
// check; a timeout is recorded with its site.
struct Deadline {
  unsigned long long t0 = 0;
  unsigned it = 0;
};
__device__ __forceinline__ bool expired(Ctrl *c, Deadline &d, unsigned long long limit_ns,
                                        int site) {
  if ((++d.it & 15u) != 0) return false;
  if (ld_volatile_i32(&c->status) < 0) return true;
  const unsigned long long t = globaltimer_ns();
  if (d.t0 == 0) {
    d.t0 = t;
    return false;
  }
  if (t - d.t0 > limit_ns) {
    set_status(c, RQLP_ERR_TIMEOUT);
    atomicExch(&c->timeout_site, site);
    return true;
  }
  return false;
}

// USE_SMEM (the slab in shared memory) is a template argument so that the
// compiler addresses the columns as shared memory, not through generic loads.

template <bool USE_SMEM>
__device__ __forceinline__ void cpqr_body(const CpqrParams &P, const int G, const int b, double *sm) {
  __shared__ double s_bn[kWarps];
  __shared__ int s_bi[kWarps];
  __shared__ int s_win_cta, s_win_idx;
  __shared__ double s_sigma, s_x0;
  __shared__ double s_tau, s_beta, s_rv0, s_trv;
  __shared__ int s_ok, s_err, s_prefix;

  const int l = P.l;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t c0 = (int64_t)b * P.cpb;
  const int nc = (int)max((int64_t)0, min(P.n, c0 + P.cpb) - c0);
  const int steps = P.steps;
  // the winner's column x(s:), unscaled (l doubles, 16-byte rounded), then
  // the slab when it sits in shared memory, then the per-column state
  double *s_v = sm;
  double *sm1 = sm + ((l + 1) & ~1);
  double *cols = USE_SMEM ? sm1 : P.gcols + (int64_t)b * P.cpb * l;
  double *nrm = USE_SMEM ? sm1 + (int64_t)P.cpb * l : sm1;
  // 1% of the norm^2 when it was last computed exactly: below that the
  // downdated value has lost too many digits and is recomputed
  double *thr = nrm + P.cpb;
  double *wdot = thr + P.cpb;  // this step's axpy multiple of x(s+1:) per column
  int *pivoted = reinterpret_cast<int *>(wdot + P.cpb);
  int *axdone = pivoted + P.cpb;                       // column updated early this step

  // warp 0: publish candidate jc (local index, key cn) for exchange k into
  // buffer buf; its column is final through row r0 - 1 once cj x(r0:)
  // (cj != 0: the step's axpy, applied here) is subtracted.  The record is
  // (cn, index), sigma = ||col(r0 + 1:)||^2 exactly and x0 = col(r0) (also
  // returned, sigma to every lane, x0 to lane 0); the column goes out from
  // row r0 on.
  // One CTA (G = 1) exchanges nothing: it keeps sigma and x0 (lane 0) and
  // takes the winner, its own candidate, straight from shared memory.
  auto publish = [&](int buf, unsigned k, int jc, double cn, int r0, double cj, double &sg,
                     double &x0) {
    const unsigned long long t = (unsigned long long)k << 32;
    sg = 0.0;
    x0 = 0.0;
    if (jc >= 0) {
      double *col = cols + (int64_t)jc * l;
      ulonglong2 *dst = P.pcol + ((int64_t)buf * G + b) * l;
      for (int r = r0 + lane; r < l; r += 32) {
        double x = col[r];
        if (cj != 0.0) {
          x = fma(-cj, s_v[r - r0 + 1], x);
          col[r] = x;
        }
        if (G > 1) st_word(dst + r, dbits(x), t);
        if (r > r0) sg = fma(x, x, sg);
        else x0 = x;  // lane 0
      }
      sg = warp_sum(sg);
    }
    if (lane == 0 && G > 1) {
      ulonglong2 *rc = P.rec + ((int64_t)buf * G + b) * kRecWords;
      st_word(rc + 1, dbits(sg), t);
      st_word(rc + 2, dbits(x0), t);
      st_word(rc, dbits(jc >= 0 ? cn : -1.0),
              (unsigned long long)(unsigned)(jc >= 0 ? (int)(c0 + jc) : -1) | t);
    }
  };
  // Exchange k: warp 0 publishes, then counts itself in (a relaxed atomic:
  // everything it published is tagged); the k G-th arrival reads all G
  // records (re-reading any whose words do not carry k yet), picks the
  // winner and writes it to every other CTA's line as two words tagged in
  // bits 48..63 of their first halves: (index | CTA << 32 | k << 48, sigma)
  // and (same, x0).  It keeps the winner in registers itself.
  unsigned won = 0;
  unsigned long long won_w0 = 0;
  double won_sigma = 0.0, won_x0 = 0.0;
  auto arrive = [&](int buf, unsigned k, int site) -> bool {
    unsigned old = 0;
    if (lane == 0) old = atomicAdd(P.arrive, 1u);
    old = __shfl_sync(0xffffffffu, old, 0);
    if (old != k * (unsigned)G - 1u) return true;
    const ulonglong2 *rb = P.rec + (int64_t)buf * G * kRecWords;
    double bn = -1.0, bs = 0.0, bx = 0.0;
    int bi = -1, bc = -1;
    Deadline dl;
    for (int cb = 0; cb < G; cb += 32 * 5) {
      ulonglong2 w0[5], w1[5], w2[5];
      unsigned pend = 0;
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        w0[j] = w1[j] = w2[j] = make_ulonglong2(0ull, 0ull);
        if (cb + lane + 32 * j < G) pend |= 1u << j;
      }
      while (true) {
#pragma unroll
        for (int j = 0; j < 5; ++j)
          if (pend & (1u << j)) {
            const ulonglong2 *rc = rb + (int64_t)(cb + lane + 32 * j) * kRecWords;
            w0[j] = ld_word(rc);
            w1[j] = ld_word(rc + 1);
            w2[j] = ld_word(rc + 2);
          }
#pragma unroll
        for (int j = 0; j < 5; ++j)
          if ((pend & (1u << j)) && tag_of(w0[j]) == k && tag_of(w1[j]) == k && tag_of(w2[j]) == k)
            pend &= ~(1u << j);
        if (!__any_sync(0xffffffffu, pend != 0)) break;
        int give_up = 0;
        if (lane == 0) give_up = expired(P.ctrl, dl, P.limit_ns, site) ? 1 : 0;
        if (__shfl_sync(0xffffffffu, give_up, 0)) return false;
      }
#pragma unroll
      for (int j = 0; j < 5; ++j) {
        const int c = cb + lane + 32 * j;
        const double nv = dval(w0[j].x);
        const int iv = (int)(unsigned)(w0[j].y & 0xffffffffull);
        if (c < G && better(nv, iv, bn, bi)) {
          bn = nv; bi = iv; bc = c; bs = dval(w1[j].x); bx = dval(w2[j].x);
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double on = __shfl_xor_sync(0xffffffffu, bn, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      const int oc = __shfl_xor_sync(0xffffffffu, bc, o);
      if (better(on, oi, bn, bi)) { bn = on; bi = oi; bc = oc; }
    }
    // record c was read by lane c mod 32, whose own best it is
    bs = __shfl_sync(0xffffffffu, bs, bc & 31);
    bx = __shfl_sync(0xffffffffu, bx, bc & 31);
    const unsigned long long w = (unsigned long long)(unsigned)bi |
                                 ((unsigned long long)((unsigned)bc & 0xffffu) << 32) |
                                 ((unsigned long long)(k & 0xffffu) << 48);
    for (int c = lane; c < G; c += 32) {
      if (c == b) continue;
      st_word(P.win + 8 * (int64_t)c + 1, w, dbits(bx));
      st_word(P.win + 8 * (int64_t)c, w, dbits(bs));
    }
    won = k;
    won_w0 = w;
    won_sigma = bs;
    won_x0 = bx;
    return true;
  };
  // G = 1: lane 0 of warp 0 records its own candidate as exchange k's winner
  auto keep_own = [&](unsigned k, int jc, double sg, double x0) {
    won = k;
    won_w0 = (unsigned long long)(unsigned)(jc >= 0 ? (int)(c0 + jc) : -1) |
             ((unsigned long long)(k & 0xffffu) << 48);
    won_sigma = sg;
    won_x0 = x0;
  };
  // thread 0: the winner of exchange k, from registers when this CTA
  // arrived last, else from the two words in its line; all threads return
  // whether it succeeded.  `extra` > 0 (the timeout test) asks for a tag
  // that never comes.
  auto wait_winner = [&](unsigned k, int site) {
    if (tid == 0) {
      unsigned long long a0 = won_w0, a1 = dbits(won_sigma), b0 = won_w0, b1 = dbits(won_x0);
      bool ok = true;
      if (won != k || P.extra != 0) {
        const unsigned want = (k + P.extra) & 0xffffu;
        const ulonglong2 *wa = P.win + 8 * (int64_t)b;
        Deadline dl;
        bool ha = false, hb = false;
        while (true) {
          if (!ha) {
            const ulonglong2 w = ld_word(wa);
            a0 = w.x;
            a1 = w.y;
            ha = (unsigned)(a0 >> 48) == want;
          }
          if (!hb) {
            const ulonglong2 w = ld_word(wa + 1);
            b0 = w.x;
            b1 = w.y;
            hb = (unsigned)(b0 >> 48) == want;
          }
          if (ha && hb) break;
          if (expired(P.ctrl, dl, P.limit_ns, site)) {
            ok = false;
            break;
          }
        }
      }
      s_ok = ok ? 1 : 0;
      s_win_idx = (int)(unsigned)(a0 & 0xffffffffull);
      s_win_cta = (int)((a0 >> 32) & 0xffffull);
      s_sigma = dval(a1);
      s_x0 = dval(b1);
    }
    __syncthreads();
    return s_ok != 0;
  };

  // nothing to do after an earlier error (its data may be garbage)
  if (ld_volatile_i32(&P.ctrl->status) < 0) return;
  if (tid == 0) s_err = 0;

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
    for (int jj = tid; jj < nc; jj += kThreads) {
      const double key = pick_key(P.fpiv, 0, (int)(c0 + jj), nrm[jj]);
      if (better(key, (int)(c0 + jj), bn, bi)) { bn = key; bi = (int)(c0 + jj); }
    }
    warp_best(bn, bi);
    if (lane == 0) { s_bn[warp] = bn; s_bi[warp] = bi; }
    __syncthreads();
    if (warp == 0) {
      double cn = s_bn[0];
      int ci = s_bi[0];
      for (int w = 1; w < kWarps; ++w)
        if (better(s_bn[w], s_bi[w], cn, ci)) { cn = s_bn[w]; ci = s_bi[w]; }
      const int jc0 = ci >= 0 ? (int)(ci - c0) : -1;
      double sg, x0;
      publish(0, 1u, jc0, cn, 0, 0.0, sg, x0);
      if (G == 1) keep_own(1u, jc0, sg, x0);
      else if (!arrive(0, 1u, 1)) s_err = 1;
    }
  }
  if (!wait_winner(1u, 1) || s_err) return;

  const int sub = lane >> 2, gl = lane & 3;
  for (int s = 0; s < steps; ++s) {
    const int buf = s & 1;
    // ---- 1. winner (every CTA picked the same one) and its sigma ----
    const int wc = s_win_cta, wi = s_win_idx;
    // with given pivots the elected column must be the given one: a given
    // index out of range or repeated leaves no column with key 1
    if (wi < 0 || wc < 0 || wc >= G || (P.fpiv && wi != __ldg(P.fpiv + s))) {
      if (tid == 0) set_status(P.ctrl, RQLP_ERR_INVALID_ARG);
      return;
    }
    // ---- 2. reflector from the winner's column, rows s..l-1 ----
    // one thread forms H = I - tau v v^T with v(0) = 1 and H x = alpha e_1,
    // alpha = ||x|| >= 0: tau = 1 - x0/alpha, v(1:) = x(1:) / (x0 - alpha),
    // where x0 > 0 uses x0 - alpha = -sigma / (x0 + alpha) (no cancellation);
    // x0 and sigma = ||x(1:)||^2 came with the winner's record, so this runs
    // while warps 1.. load the column
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
    // warps 1.. load the column (published for exchange s + 1) meanwhile
    const ulonglong2 *xc = P.pcol + ((int64_t)buf * G + wc) * l;
    if (G == 1) {
      // the winner is this CTA's own column, updated in the slab
      const double *own = cols + (int64_t)(wi - c0) * l;
      if (warp > 0)
        for (int r = s + tid - 32; r < l; r += kThreads - 32) s_v[r - s] = own[r];
    } else if (warp > 0)
      for (int r = s + tid - 32; r < l; r += kThreads - 32) {
        ulonglong2 w = ld_word(xc + r);
        Deadline dl;
        while (tag_of(w) != (unsigned)(s + 1)) {
          if (expired(P.ctrl, dl, P.limit_ns, 4)) {
            s_err = 1;
            break;
          }
          w = ld_word(xc + r);
        }
        s_v[r - s] = dval(w.x);
      }
    __syncthreads();
    if (s_err) return;
    // s_v holds the winner's column x(s:) unscaled; v = (1, x(s+1:) rv0)
    const double tau = s_tau, beta = s_beta, rv0 = s_rv0, trv = s_trv;
    // the winner's column is final: rows < s from the slab, beta at s, zeros below
    if ((int)(wi - c0) >= 0 && (int)(wi - c0) < nc && warp == 0) {
      const int jw = (int)(wi - c0);
      const double *col = cols + (int64_t)jw * l;
      double *out = P.R0t + (int64_t)s * P.ldr;
      for (int r = lane; r < steps; r += 32) out[r] = (r < s) ? col[r] : (r == s ? beta : 0.0);
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
        const double key = s + 1 < steps ? pick_key(P.fpiv, s + 1, (int)(c0 + jj), nd) : nd;
        if (better(key, (int)(c0 + jj), bn, bi)) { bn = key; bi = (int)(c0 + jj); }
      }
    }
    warp_best(bn, bi);
    if (lane == 0) { s_bn[warp] = bn; s_bi[warp] = bi; }
    __syncthreads();
    // this CTA's candidate for step s + 1 (every thread reads the same table)
    int jc = -1;
    double cn = -1.0;
    if (s + 1 < steps) {
      int ci = -1;
      for (int w = 0; w < kWarps; ++w)
        if (better(s_bn[w], s_bi[w], cn, ci)) { cn = s_bn[w]; ci = s_bi[w]; }
      jc = ci >= 0 ? (int)(ci - c0) : -1;
    }
    // ---- 4. warp 0: update the candidate and publish it ----
    if (warp == 0 && s + 1 < steps) {
      const unsigned k = (unsigned)(s + 2);
      double sg, x0;
      publish(buf ^ 1, k, jc, cn, s + 1, (jc >= 0 && !axdone[jc]) ? wdot[jc] : 0.0, sg, x0);
      if (G == 1) keep_own(k, jc, sg, x0);
      else if (!arrive(buf ^ 1, k, 5) && lane == 0) s_err = 1;
    }
    // ---- 5. the remaining axpys, while warp 0 arrives (and, if last, picks
    // the winner) ----
    if (b == 0 && warp == kWarps - 1) {
      // this step's reflector, off the path to the exchange
      for (int r = lane; r < l; r += 32)
        P.Vh[(int64_t)r * P.ldv + s] = (r < s) ? 0.0 : (r == s ? 1.0 : s_v[r - s] * rv0);
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
    // (the wait's block barrier orders these axpys before the next column load)
    if (s + 1 < steps && (!wait_winner((unsigned)(s + 2), 2) || s_err)) return;
  }

  // ---- unchosen columns keep their order behind the pivots ----
  // one more exchange (steps + 1, record word 0): the number of unchosen
  // columns of every CTA; CTA b needs those of CTAs 0..b-1
  if (warp == 0) {
    const unsigned kf = (unsigned)(steps + 1);
    const int fb = steps & 1;
    int mine = 0;
    for (int jj = lane; jj < nc; jj += 32) mine += pivoted[jj] ? 0 : 1;
    mine = __reduce_add_sync(0xffffffffu, mine);
    if (lane == 0)
      st_word(P.rec + ((int64_t)fb * G + b) * kRecWords, (unsigned long long)mine,
              (unsigned long long)kf << 32);
    int pre = 0;
    bool ok = true;
    Deadline dl;
    for (int cb = 0; cb < b && ok; cb += 32) {
      const int c = cb + lane;
      bool pend = c < b;
      while (true) {
        if (pend) {
          const ulonglong2 w = ld_word(P.rec + ((int64_t)fb * G + c) * kRecWords);
          if (tag_of(w) == kf) {
            pend = false;
            pre += (int)w.x;
          }
        }
        if (!__any_sync(0xffffffffu, pend)) break;
        int give_up = 0;
        if (lane == 0) give_up = expired(P.ctrl, dl, P.limit_ns, 3) ? 1 : 0;
        if (__shfl_sync(0xffffffffu, give_up, 0)) {
          ok = false;
          break;
        }
      }
    }
    pre = __reduce_add_sync(0xffffffffu, pre);
    if (lane == 0) {
      s_prefix = pre;
      s_ok = ok ? 1 : 0;
    }
  }
  __syncthreads();
  if (!s_ok) return;
  if (warp == 0) {
    // rank of each unpivoted column within the slab, in index order
    int pos = steps + s_prefix;
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
    for (int r = lane; r < steps; r += 32) P.R0t[dst * P.ldr + r] = col[r];
  }
}

}  // namespace cpqrk
}  // namespace rqk
