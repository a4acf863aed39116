// Column-pivoted Householder QR of the wide l x n matrix B
// (Algorithm 2.1 step 5 / Algorithm 2.2 step 5, "cpqr(B)").
//
// One persistent cooperative kernel.  CTA b owns a contiguous slab of
// columns of B (each column l doubles), kept in shared memory when it fits
// and in a global scratch copy otherwise.  Per pivot step s there is exactly
// one grid-wide exchange:
//   1. every CTA has published its best column for step s: a record (norm,
//      index), the exact ||x(s+1:)||^2 of that column (sigma), x0 = x(s) and
//      the column itself; the last CTA to arrive picked the winner (largest
//      trailing norm, ties to the lowest original index) and sent it to all;
//   2. every CTA builds the same Householder reflector from the winner's
//      x0 and sigma, mapping its column to +alpha e_s (non-negative
//      R(s, s)), while it loads that column;
//   3. every CTA forms v^T col for its unpivoted columns (4 lanes per column)
//      from the unscaled column, v^T col = col(s) + (x(s+1:)^T col(s+1:)) /
//      (x0 - alpha), and the downdated norms ||col(s+1:)||^2 =
//      ||col(s:)||^2 - col'(s)^2 (recomputed exactly after more than 99 %
//      cancellation);
//   4. warp 0 updates the CTA's best column for step s + 1, publishes it and
//      arrives (the last arrival picks the winner);
//   5. meanwhile the other warps apply the rest of the axpys
//      col -= (v^T col) tau v.
// After l steps the unchosen columns are written in their original order
// behind the pivots.
//
// The exchange needs no fences: every value a CTA publishes is stored as one
// 128-bit word together with the number k of the exchange it belongs to, and
// readers re-read a word until it carries k.  A 128-bit access is a single
// memory access, so a word that carries k holds exchange k's value, whatever
// order the stores arrive in.  Each CTA then counts itself in with a relaxed
// atomic; the last of the G reads the G candidate records, picks the winner
// and writes it into one 128-byte line per CTA, which that CTA polls alone.
// Candidate records and columns are double-buffered by exchange parity: a CTA
// overwrites exchange k's buffers (for k + 2) only after exchange k + 1's
// winner exists, which needed every CTA's exchange k + 1 arrival, made after
// it had read exchange k.  The host zeroes the exchange state before every
// launch, so no word of an earlier launch matches.
#include <cmath>

#include "cpqr_body.cuh"

namespace rqk {

namespace {

using namespace cpqrk;

template <bool USE_SMEM>
__global__ void __launch_bounds__(kThreads) k_cpqr_wide(CpqrParams P) {
  extern __shared__ double sm[];
  cpqr_body<USE_SMEM>(P, (int)gridDim.x, (int)blockIdx.x, sm);
}

struct Plan {
  int G, cpb, use_smem;
  size_t smem;
};

Plan plan_for(int64_t n, int l, int max_ctas) {
  Plan p;
  const int sms = num_sms();
  const int cap = max_ctas > 0 ? max_ctas : tuning().cpqr_max_ctas;
  int G = (int)std::min<int64_t>(n, (int64_t)((cap > 0 && cap < sms) ? cap : sms));
  if (G < 1) G = 1;
  int cpb = (int)((n + G - 1) / G);
  G = (int)((n + cpb - 1) / cpb);
  const size_t sv = (size_t)((l + 1) & ~1) * sizeof(double);  // the winner's column
  const size_t state = (size_t)cpb * (3 * sizeof(double) + 2 * sizeof(int));
  const size_t slab = (size_t)cpb * l * sizeof(double);
  p.use_smem = (sv + slab + state <= 190 * 1024) ? 1 : 0;
  p.smem = sv + (p.use_smem ? slab : 0) + state;
  p.G = G;
  p.cpb = cpb;
  // a smaller grid asked for keeps the slabs in shared memory, or is not taken
  if (max_ctas > 0 && !p.use_smem) return plan_for(n, l, 0);
  return p;
}

}  // namespace

// per-launch exchange state, zeroed before every launch: the arrival
// counter (one 128-byte line), the winner lines (one per CTA), the tagged
// candidate records and the tagged published columns (both double-buffered)
static size_t tagged_bytes(int G, int64_t l) {
  return 128 + 128 * (size_t)G + 2 * (size_t)G * kRecWords * sizeof(ulonglong2) +
         2 * (size_t)G * l * sizeof(ulonglong2);
}

size_t cpqr_ws_bytes(int64_t n, int l) {
  size_t b = (tagged_bytes(kMaxGrid, l) + 255) / 256 * 256;
  b += (size_t)(n + kMaxGrid) * l * sizeof(double);  // global slabs (fallback)
  return b + 8192;
}

size_t cpqr_scratch_bytes_smem_only(int64_t n, int l, bool *fits) {
  const Plan pl = plan_for(n, l, 0);
  *fits = pl.use_smem != 0 && pl.G <= kMaxGrid;
  return (tagged_bytes(pl.G, l) + 255) / 256 * 256;
}

size_t cpqr_tall_ws_bytes(int64_t n, int64_t L) {
  const int G = (int)std::max<int64_t>(1, std::min<int64_t>(n, num_sms()));
  const int64_t cpb = (n + G - 1) / G;
  size_t b = (tagged_bytes(G, L) + 255) / 256 * 256;
  b += ((size_t)G * cpb * L * sizeof(double) + 255) / 256 * 256;
  return b + 8192;
}

// The launch shared by the wide CPQR of B (l = column length = steps) and the
// truncated CPQR of a tall matrix (column length L, `steps` pivots).
static cudaError_t cpqr_launch(const double *Bt, int64_t n, int64_t L, int steps, int64_t ldb,
                               double *R0t, int64_t ldr, int32_t *piv, double *Vh, int64_t ldv,
                               double *tau, void *scratch, Ctrl *ctrl,
                               unsigned long long limit_ns, unsigned debug_extra, cudaStream_t st,
                               const int32_t *fixed_piv, int max_ctas) {
  Plan pl = plan_for(n, (int)L, max_ctas);
  if (pl.G > kMaxGrid || pl.smem > 220 * 1024) return cudaErrorInvalidValue;
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
  P.Bt = Bt; P.n = n; P.l = (int)L; P.steps = steps; P.ldv = (int)ldv; P.ldb = ldb;
  P.R0t = R0t; P.ldr = ldr; P.piv = piv;
  P.Vh = Vh; P.tau = tau;
  const size_t tb = tagged_bytes(pl.G, L);
  char *tagged = take(tb);
  P.arrive = reinterpret_cast<unsigned *>(tagged);
  P.win = reinterpret_cast<ulonglong2 *>(tagged + 128);
  P.rec = reinterpret_cast<ulonglong2 *>(tagged + 128 + 128 * (size_t)pl.G);
  P.pcol = P.rec + 2 * (size_t)pl.G * kRecWords;
  P.gcols = reinterpret_cast<double *>(take((size_t)pl.G * pl.cpb * L * sizeof(double)));
  P.ctrl = ctrl;
  P.limit_ns = limit_ns ? limit_ns : kDefaultSpinNs;
  P.extra = debug_extra;
  P.cpb = pl.cpb;
  P.use_smem = pl.use_smem;
  P.fpiv = fixed_piv;
  // the permutation stays valid even if the kernel stops early on an error
  e = iota(piv, n, st);
  if (e != cudaSuccess) return e;
  // no tagged word of an earlier launch may match this launch's exchanges
  e = cudaMemsetAsync(tagged, 0, tb, st);
  if (e != cudaSuccess) return e;
  if (pl.G == 1) {
    // one CTA: it exchanges nothing, no co-residency is needed
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

cudaError_t cpqr_wide(const double *Bt, int64_t n, int l, int64_t ldb, double *R0t, int64_t ldr,
                      int32_t *piv, double *Vh, double *tau, void *scratch, Ctrl *ctrl,
                      unsigned long long limit_ns, unsigned debug_extra, cudaStream_t st,
                      const int32_t *fixed_piv, int max_ctas) {
  if (n <= 0 || l <= 0 || l > kMaxL || l > n) return cudaErrorInvalidValue;
  return cpqr_launch(Bt, n, l, l, ldb, R0t, ldr, piv, Vh, l, tau, scratch, ctrl, limit_ns,
                     debug_extra, st, fixed_piv, max_ctas);
}

cudaError_t cpqr_tall(const double *At, int64_t n, int64_t L, int steps, int64_t ldat, double *R0t,
                      int64_t ldr, int32_t *piv, double *Vh, int64_t ldv, double *tau,
                      void *scratch, Ctrl *ctrl, unsigned long long limit_ns, cudaStream_t st) {
  if (n <= 0 || L <= 0 || steps < 1 || steps > kMaxL || steps > n || steps > L || ldr < steps ||
      ldv < steps || L > 16384)
    return cudaErrorInvalidValue;
  return cpqr_launch(At, n, L, steps, ldat, R0t, ldr, piv, Vh, ldv, tau, scratch, ctrl, limit_ns,
                     0, st, nullptr, 0);
}

}  // namespace rqk
