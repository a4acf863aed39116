// C ABI driver: enqueues the stages of RQLP / ERQLP / BRQLP on one stream.
//
// Algorithm 2.1 / 2.2 (Section 2) as launched here:
//   range finder   Y = A Omega; q times { V = qr(Y); Z = A^T V; W = qr(Z); Y = A W }; V = qr(Y)
//   projection     B^T = A^T V                     (n x l; column-major B)
//   first CPQR     B Pi0 = Q0 R0                    (cooperative kernel)
//   second stage   X = R0^T:  RQLP  X = Qa Ra, Ra Pi1 = Qc R1   => L = R1^T, P = Pi0 Qa Qc
//                             ERQLP X = Q(1) R(1), R(i-1)^T = Q(i) R(i), i = 2..d
//   assembly       Q = V Q_B,  P = Pi0 (Q(1) Q(3) ...),  L-values = diag(L)
// Every thin QR is CholeskyQR2 in FP64; with column pivoting compared on
// exact norms the CPQR of the tall X equals the CPQR of its R factor Ra,
// which is why the second CPQR runs on the l x l matrix Ra.
#include <cstring>
#include <vector>

#include "kernels.cuh"
#include "mixed.cuh"

using namespace rqk;

namespace {

#define CK(x)                                     \
  do {                                            \
    cudaError_t e_ = (x);                         \
    if (e_ != cudaSuccess) return RQLP_ERR_CUDA;  \
  } while (0)

#define RET_IF(x)                 \
  do {                            \
    int r_ = (x);                 \
    if (r_ != RQLP_OK) return r_; \
  } while (0)

// Scratch for CholeskyQR2 on rows x l data.
struct OrthBufs {
  double *part;   // split-K partials
  double *gpart;  // Gram chunk partials
  double *G, *Rp, *Rinv, *Racc, *Rtmp, *Dinv;
  double *tmp;    // rows x l ping-pong
  float *rf;      // FP32 R and block inverses of an FP32 pass (f32_pack_floats(l))
  // FP64-accurate digit products on the tensor cores for the Gram matrix, X R^-1
  // and the final assembly (the forms other than FP64, l <= 128)
  bool oz;
  OzOperand oz_xt;  // columns of X (Gram: both operands), with the scaled copies
  OzOperand oz_x;   // rows of X (X R^-1, the assembly)
  OzOperand oz_ri;  // columns of an l x l right factor (R^-1, Q_B, ...)
  double *eye;      // l x l identity
  float *oz_part;
  int64_t oz_part_floats;
};

// unit roundoff of a Gram matrix formed from digit products (2^-47 relative
// to the column scales, with a factor 2 of margin)
constexpr double kEpsOz = 1.4210854715202004e-14;  // 2^-46
// which parts of a tall FP64 CholeskyQR pass use digit products (the final
// assembly always does when the buffers exist): the Gram matrix (one
// product with K = rows), and X R^-1 (needs R^-1 first: measured slower than
// the FP64 blocked solve, whose triangular structure halves the work)
constexpr bool kOzGram = true;
constexpr bool kOzApply = false;

size_t part_doubles(int64_t m, int64_t n, int l) {
  const int64_t big = std::max(m, n);
  size_t b = 0;
  auto upd = [&](int64_t M, int64_t N, int64_t K) {
    b = std::max(b, gemm_f64_part_bytes(M, N, K) / sizeof(double));
  };
  upd(m, l, n);
  upd(n, l, m);
  upd(l, l, m);
  upd(l, l, n);
  upd(l, l, l);
  upd(big, l, l);
  b = std::max(b, (size_t)4 * big * l);  // products with K = l (<= 4 splits) and the scatter
  return b;
}

// The digit-product buffers of the orthonormalizations and the assembly,
// carved last so that every other piece of a workspace keeps its offset.
void carve_orth_oz(Arena &a, int64_t rows_max, int l, OrthBufs &o, bool oz) {
  o.oz = oz && l <= 128 && !tuning().no_digit_products;
  if (!o.oz) return;
  o.oz_xt = oz_carve(a, l, rows_max, kOzCopies);
  o.oz_x = oz_carve(a, rows_max, l, 1);
  o.oz_ri = oz_carve(a, l, l, kOzCopies);
  o.eye = a.take<double>((size_t)l * l);
  o.oz_part_floats = (int64_t)std::max(oz_part_floats(l, l, rows_max),
                                       oz_part_floats(rows_max, l, l));
  o.oz_part = a.take<float>((size_t)o.oz_part_floats);
}

void carve_orth(Arena &a, int64_t rows_max, int l, int64_t m, int64_t n, OrthBufs &o,
                double *shared_part) {
  o.oz = false;
  o.part = shared_part ? shared_part : a.take<double>(part_doubles(m, n, l));
  o.gpart = a.take<double>((size_t)gram_chunks_max(std::max<int64_t>(rows_max, l)) * l * l);
  o.Dinv = a.take<double>((size_t)l * l);
  o.G = a.take<double>((size_t)l * l);
  o.Rp = a.take<double>((size_t)l * l);
  o.Rinv = a.take<double>((size_t)l * l);
  o.Racc = a.take<double>((size_t)l * l);
  o.Rtmp = a.take<double>((size_t)l * l);
  o.tmp = a.take<double>((size_t)rows_max * l);
  o.rf = a.take<float>(f32_pack_floats(l));
}

// CholeskyQR2 (+ a third pass iff a pass needed the shift): Xq = X R^{-1}.
// lowp_first: the first pass in FP32 (Gram and solve; the Cholesky stays FP64
// with FP32's unit roundoff in its breakdown test and shift), then, when
// passes >= 2, an FP64 pass always follows: Q is FP64-orthonormal and spans
// range(X) to about FP32 accuracy.
// An operand view of a carved digit buffer with these rows and K.
OzOperand oz_view(const OzOperand &b, int64_t rows, int64_t K) {
  OzOperand o = b;
  o.rows = rows;
  o.K = K;
  o.ld = (K + 7) / 8 * 8;
  return o;
}

// C (M x l, ldc; row i to rowmap[i] when given) = X (M x K, ldx) F (K x l,
// ld l) with K <= 128 by digit products on the tensor cores.
int oz_right_product(const OrthBufs &o, const double *X, int64_t M, int64_t K, int64_t ldx,
                     const double *F, int l, double *C, int64_t ldc, const int32_t *rowmap,
                     Ctrl *ctrl, const int *skip, cudaStream_t st) {
  const OzOperand xx = oz_view(o.oz_x, M, K), ff = oz_view(o.oz_ri, l, K);
  RET_IF(oz_split(X, RQLP_F64, M, K, ldx, false, xx, ctrl, skip, st));
  RET_IF(oz_split(F, RQLP_F64, K, l, l, true, ff, ctrl, skip, st));
  return oz_gemm(xx, ff, M, l, K, C, ldc, rowmap, o.oz_part, o.oz_part_floats, ctrl, 0, skip, st);
}

int orth_impl(const double *X, int64_t rows, int l, int64_t ldx, double *Xq, int64_t ldq, double *R,
              const OrthBufs &o, Ctrl *ctrl, int site, int passes, double again_tol,
              cudaStream_t st, bool lowp_first) {
  site %= kShiftSites;
  const int *flag = &ctrl->shift_flag[site];
  int ev;
  // one CholeskyQR pass: src -> dst, R_acc <- R_pass R_acc (skip: conditional pass)
  auto pass = [&](const double *src, int64_t lds, double *dst, int64_t ldd, bool first,
                  const int *skip, double tol, bool lowp = false) -> int {
    // a tall FP64 pass may take its Gram matrix and X R^-1 from digit products
    const bool ozp = o.oz && !lowp && rows > kMaxL;
    ev = prof_start(kProfGram, st);
    if (ozp && kOzGram) {
      const OzOperand xt = oz_view(o.oz_xt, l, rows);
      RET_IF(oz_split(src, RQLP_F64, rows, l, lds, true, xt, ctrl, skip, st));
      RET_IF(oz_gemm(xt, xt, l, l, rows, o.G, l, nullptr, o.oz_part, o.oz_part_floats, ctrl, 0,
                     skip, st));
    } else {
      CK(gram_sym(src, rows, l, lds, o.gpart, o.G, skip, st, lowp));
    }
    prof_stop(kProfGram, ev, st);
    ev = prof_start(kProfChol, st);
    CK(chol_blocked(o.G, l, rows, o.Rp, o.Dinv, ctrl, site, skip, st, tol,
                    lowp ? kEpsF32 : ((ozp && kOzGram) ? kEpsOz : kEpsF64), lowp,
                    lowp ? o.rf : nullptr));
    prof_stop(kProfChol, ev, st);
    ev = prof_start(kProfApply, st);
    if (ozp && kOzApply) {
      // R^-1 = I R^-1 by the blocked solve, then X R^-1 as a digit product
      CK(apply_trsm(o.eye, l, l, l, o.Rp, o.Dinv, o.Rinv, l, skip, st));
      RET_IF(oz_right_product(o, src, rows, l, lds, o.Rinv, l, dst, ldd, nullptr, ctrl, skip, st));
    } else if (rows <= kMaxL && !lowp && skip == nullptr) {
      // a few rows (the l x l QRs): one warp per row solves q R = x
      CK(tri_rows(o.Rp, l, nullptr, l, src, lds, dst, ldd, (int)rows, false, st));
    } else {
      CK(apply_trsm(src, rows, l, lds, o.Rp, o.Dinv, dst, ldd, skip, st, lowp,
                    lowp ? o.rf : nullptr));
    }
    if (R) {
      if (first) {
        CK(copy2d(o.Rp, l, l, l, o.Racc, l, skip, st));
      } else {
        CK(gemm_f64(false, RQLP_F64, o.Rp, l, o.Racc, l, o.Rtmp, l, l, l, l, 1.0, 0.0, o.part,
                    nullptr, skip, st));
        CK(copy2d(o.Rtmp, l, l, l, o.Racc, l, skip, st));
      }
    }
    prof_stop(kProfApply, ev, st);
    return RQLP_OK;
  };
  if (kOzApply && o.oz) CK(set_identity(o.eye, l, l, l, st));
  // X and Xq share no element: a pass may then write Xq while it reads X
  const bool dis = X + (rows - 1) * ldx + l <= Xq || Xq + (rows - 1) * ldq + l <= X;
  int r;
  if (lowp_first && passes >= 2) {
    r = pass(X, ldx, o.tmp, l, true, nullptr, -1.0, true);  // FP32 pass: X -> tmp
    if (r != RQLP_OK) return r;
    r = pass(o.tmp, l, Xq, ldq, false, nullptr, -1.0);      // FP64 pass: tmp -> Xq
  } else if (lowp_first && dis) {
    r = pass(X, ldx, Xq, ldq, true, nullptr, -1.0, true);  // one FP32 pass: X -> Xq
  } else if (lowp_first) {
    r = pass(X, ldx, o.tmp, l, true, nullptr, -1.0, true);  // one FP32 pass, in place
    if (r == RQLP_OK) CK(copy2d(o.tmp, rows, l, l, Xq, ldq, nullptr, st));
  } else if (passes >= 2 && again_tol >= 0.0 && dis) {
    // adaptive, usually one pass: X -> Xq; only when the first pass asks for
    // it, Xq -> tmp -> Xq
    r = pass(X, ldx, Xq, ldq, true, nullptr, again_tol);
    if (r != RQLP_OK) return r;
    r = pass(Xq, ldq, o.tmp, l, false, &ctrl->again_flag[site], -1.0);
    if (r != RQLP_OK) return r;
    CK(copy2d(o.tmp, rows, l, l, Xq, ldq, &ctrl->again_flag[site], st));
  } else if (passes >= 2 && again_tol >= 0.0) {
    // adaptive: the second pass runs only when the first one says it is needed
    r = pass(X, ldx, o.tmp, l, true, nullptr, again_tol);
    if (r != RQLP_OK) return r;
    r = pass(o.tmp, l, Xq, ldq, false, &ctrl->again_flag[site], -1.0);
    if (r != RQLP_OK) return r;
    CK(copy2d(o.tmp, rows, l, l, Xq, ldq, &ctrl->done_flag[site], st));
  } else if (passes >= 2) {
    r = pass(X, ldx, o.tmp, l, true, nullptr, -1.0);   // pass 1: X -> tmp
    if (r != RQLP_OK) return r;
    r = pass(o.tmp, l, Xq, ldq, false, nullptr, -1.0); // pass 2: tmp -> Xq
  } else if (dis) {
    r = pass(X, ldx, Xq, ldq, true, nullptr, -1.0);    // one pass: X -> Xq
  } else {
    r = pass(X, ldx, o.tmp, l, true, nullptr, -1.0);   // one pass, in place: X -> tmp -> Xq
    if (r == RQLP_OK) CK(copy2d(o.tmp, rows, l, l, Xq, ldq, nullptr, st));
  }
  if (r != RQLP_OK) return r;
  // one more pass, only when the device raised the shift flag: Xq -> tmp -> Xq
  // (a lone FP32 pass never raises it: a shifted factor still spans range(X))
  if (!(lowp_first && passes < 2)) {
    r = pass(Xq, ldq, o.tmp, l, false, flag, -1.0);
    if (r != RQLP_OK) return r;
    CK(copy2d(o.tmp, rows, l, l, Xq, ldq, flag, st));
  }
  if (R) CK(copy2d(o.Racc, l, l, l, R, l, nullptr, st));
  return RQLP_OK;
}

int orth(const double *X, int64_t rows, int l, int64_t ldx, double *Xq, int64_t ldq, double *R,
         const OrthBufs &o, Ctrl *ctrl, int site, cudaStream_t st, int passes = 2,
         double again_tol = -1.0, bool lowp_first = false) {
  return orth_impl(X, rows, l, ldx, Xq, ldq, R, o, ctrl, site, passes, again_tol, st, lowp_first);
}

// Mixed forms: a CholeskyQR pass leaves Q orthonormal to about eps cond(X)^2;
// the second pass of CholeskyQR2 runs only when that exceeds 1e-10, far below
// the error of the BF16 products.  The FP64 form always runs both passes.
// the forms whose products with A are FP64-accurate (DFMA, or digits on the
// tensor cores) keep every CholeskyQR pass in FP64
bool fp64_products(int prec) { return prec == RQLP_PREC_FP64 || prec == RQLP_PREC_FP64TC; }
double again_tol_of(const rqlp_opts &o) { return fp64_products(o.prec) ? -1.0 : 1e-10; }

// Everything rqlp() carves from its workspace.
struct Plan {
  Ctrl *ctrl;
  OrthBufs ob;
  double *Y, *V, *Z, *W, *X, *R0t;
  double *Q0, *QB, *Macc, *Racc, *Rt, *Tl, *Vh, *tau, *Qi, *Rprev, *Xs, *sm1;
  double *utw;  // 2 l^2: scratch of the explicit Q from reflectors
  double *rvals;  // l: R-values, diag R0 of the CPQR of B (per block for BRQLP)
  double *Qf, *Lf, *Pf;  // full-width factors before a rank-k truncation (else null)
  int32_t *piv0, *piv1;
  void *cpqr_scratch;
  MixedBufs mx;
  size_t bytes;
};

Plan carve(void *ws, int64_t m, int64_t n, int l, const rqlp_opts &o) {
  Plan p;
  Arena a(ws);
  p.ctrl = a.take<Ctrl>(1);
  const int64_t big = std::max(m, n);
  carve_orth(a, big, l, m, n, p.ob, nullptr);
  p.Y = a.take<double>((size_t)m * l);
  p.V = a.take<double>((size_t)m * l);
  p.Z = a.take<double>((size_t)n * l);
  p.W = a.take<double>((size_t)n * l);
  p.X = a.take<double>((size_t)n * l);
  p.R0t = a.take<double>((size_t)n * l);
  const size_t ll = (size_t)l * l;
  p.Q0 = a.take<double>(ll);
  p.QB = a.take<double>(ll);
  p.Macc = a.take<double>(ll);
  p.Racc = a.take<double>(ll);
  p.Rt = a.take<double>(ll);
  p.Tl = a.take<double>(ll);
  p.Vh = a.take<double>(ll);
  p.tau = a.take<double>((size_t)l);
  p.Qi = a.take<double>(ll);
  p.Rprev = a.take<double>(ll);
  p.Xs = a.take<double>(ll);
  p.sm1 = a.take<double>(ll);
  p.utw = a.take<double>(2 * ll);
  p.rvals = a.take<double>((size_t)l);
  p.Qf = p.Lf = p.Pf = nullptr;
  if (o.truncate_k) {
    p.Qf = a.take<double>((size_t)m * l);
    p.Lf = a.take<double>(ll);
    p.Pf = a.take<double>((size_t)n * l);
  }
  p.piv0 = a.take<int32_t>((size_t)n);
  p.piv1 = a.take<int32_t>((size_t)l);
  p.cpqr_scratch = a.take<char>(cpqr_ws_bytes(std::max<int64_t>(n, l), l));
  carve_mixed(a, m, n, l, o.prec, p.mx);
  carve_orth_oz(a, big, l, p.ob, o.prec != RQLP_PREC_FP64);
  p.bytes = a.off;
  return p;
}

bool valid_opts(const rqlp_opts *o) {
  if (!o) return false;
  if (o->q < 0 || o->q > 16) return false;
  if (o->pivot2 != 0 && o->pivot2 != 1) return false;
  if (!o->pivot2 && (o->d < 1 || o->d > 64)) return false;
  if (o->prec < RQLP_PREC_FP64 || o->prec > RQLP_PREC_FP64TC) return false;
  if (o->block_b < 0) return false;
  if (o->spin_limit_ns < 0) return false;
  if (o->fixed_pivots != 0 && o->fixed_pivots != 1) return false;
  if (o->truncate_k != 0 && o->truncate_k != 1) return false;
  if (o->in_flight < 0) return false;
  return true;
}

bool valid_dims(int64_t m, int64_t n, int32_t k, int32_t p) {
  if (m <= 0 || n <= 0 || k < 1 || p < 0) return false;
  const int64_t l = (int64_t)k + p;
  if (l > kMaxL || l > m || l > n) return false;
  if (m > (1LL << 31) || n > (1LL << 31)) return false;
  return true;
}

// Products with A in the requested precision.
int prod_nn(const Plan &P, const rqlp_opts &o, const void *A, int a_dtype, int64_t m, int64_t n,
            int64_t lda, const double *W, int64_t ldw, int l, double *Y, cudaStream_t st) {
  const int ev = prof_start(kProfProducts, st);
  int r;
  if (o.prec == RQLP_PREC_FP64)
    r = gemm_f64(false, a_dtype, A, lda, W, ldw, Y, l, m, l, n, 1.0, 0.0, P.ob.part, nullptr,
                 nullptr, st) == cudaSuccess ? RQLP_OK : RQLP_ERR_CUDA;
  else
    r = mixed_nn(P.mx, o.prec, m, n, W, ldw, l, Y, P.ctrl, o.spin_limit_ns, st);
  prof_stop(kProfProducts, ev, st);
  return r;
}

int prod_tn(const Plan &P, const rqlp_opts &o, const void *A, int a_dtype, int64_t m, int64_t n,
            int64_t lda, const double *V, int64_t ldv, int l, double *Z, cudaStream_t st) {
  const int ev = prof_start(kProfProducts, st);
  int r;
  if (o.prec == RQLP_PREC_FP64)
    r = gemm_f64(true, a_dtype, A, lda, V, ldv, Z, l, n, l, m, 1.0, 0.0, P.ob.part, nullptr,
                 nullptr, st) == cudaSuccess ? RQLP_OK : RQLP_ERR_CUDA;
  else
    r = mixed_tn(P.mx, o.prec, m, n, V, ldv, l, Z, P.ctrl, o.spin_limit_ns, st);
  prof_stop(kProfProducts, ev, st);
  return r;
}

#define RET(x)                    \
  do {                            \
    int r_ = (x);                 \
    if (r_ != RQLP_OK) return r_; \
  } while (0)

// A second stream for work that does not depend on its neighbours (the
// explicit Q0 of the CPQR runs beside the QR of R0^T).  Not used while the
// stream is being captured (the batched plan captures many problems, and a
// shared side stream would tie their graphs together).
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
// One side stream per caller stream (and host thread), so that problems in
// flight on different streams do not queue behind each other's Q0.  A
// stream being recorded gets none (the batched graph records many problems
// on many branches), unless the recording of one factorization asked for it
// (t_side_in_capture) after creating it outside the capture.
thread_local bool t_side_in_capture = false;
SideStream *side_for(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return nullptr;
  if (cs != cudaStreamCaptureStatusNone && !t_side_in_capture) return nullptr;
  struct Entry {
    cudaStream_t main;
    SideStream sd;
  };
  static thread_local std::vector<Entry> table;
  if (table.capacity() < 64) table.reserve(64);  // entries never move
  for (Entry &e : table)
    if (e.main == st) return &e.sd;
  if (table.size() >= 64) return nullptr;  // many streams: Q0 stays on the caller's stream
  if (cs != cudaStreamCaptureStatusNone) return nullptr;  // nothing is created while recording
  Entry e;
  e.main = st;
  if (cudaStreamCreateWithFlags(&e.sd.s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&e.sd.fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&e.sd.join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  table.push_back(e);
  return &table.back().sd;
}

// The pivoted QLP of the small w x n matrix B, given as Bt = B^T (n x w,
// ld w), followed by the assembly of Q and P (Algorithm 2.1 steps 5-7,
// Algorithm 2.2 steps 5-9).  Vb is the m x w range basis (ld ldv); Q (m x w),
// L (w x w) and P (n x w) are written with leading dimension ldo; piv1 gets w
// entries; rv gets the w R-values diag R0.  fp0 / fp1 (device, may be null):
// given pivots of the two column-pivoted QRs (w entries each), which are then
// taken instead of chosen.
int qlp_stage(const Plan &P, const rqlp_opts &o, int64_t m, int64_t n, int w, const double *Vb,
              int64_t ldv, const double *Bt, double *Q, double *L, double *Pout, int64_t ldo,
              int32_t *piv0, int32_t *piv1, int site0, cudaStream_t st, const int32_t *fp0,
              const int32_t *fp1, double *rv) {
  Ctrl *ctrl = P.ctrl;
  const unsigned long long lim = (unsigned long long)o.spin_limit_ns;
  const unsigned extra = (o.debug_flags & 1) ? 1u : 0u;
  const int l = w;
  // with other factorizations in flight the grid-wide pivoted QR takes half
  // of the SMs: the others' kernels run on the rest while its CTAs wait on
  // their exchanges
  const int cpqr_ctas = o.in_flight >= 2 ? (num_sms() + 1) / 2 : 0;
  int ev = prof_start(kProfCpqr, st);
  CK(cpqr_wide(Bt, n, l, l, P.R0t, l, piv0, P.Vh, P.tau, P.cpqr_scratch, ctrl, lim, extra, st,
               fp0, cpqr_ctas));
  prof_stop(kProfCpqr, ev, st);
  CK(diag_of(P.R0t, l, l, rv, st));  // the R-values of Section 5
  // Q0 from the reflectors, beside the QR of R0^T (joined before Vh is
  // overwritten or Q0 is used)
  SideStream *sd = side_for(st);
  cudaStream_t sq = sd ? sd->s : st;
  if (sd) {
    CK(cudaEventRecord(sd->fork, st));
    CK(cudaStreamWaitEvent(sq, sd->fork, 0));
  }
  ev = prof_start(kProfSmall, sq);
  CK(form_q(P.Vh, l, P.tau, l, l, P.Q0, l, sq, P.utw));
  prof_stop(kProfSmall, ev, sq);
  auto join = [&]() -> int {
    if (sd) {
      CK(cudaEventRecord(sd->join, sq));
      CK(cudaStreamWaitEvent(st, sd->join, 0));
    }
    return RQLP_OK;
  };
  if (o.pivot2) {
    RET(orth(P.R0t, n, l, l, P.X, l, P.Racc, P.ob, ctrl, site0, st, 2, again_tol_of(o)));
    CK(transpose(P.Racc, l, l, l, P.Rt, l, st));
    RET(join());
    CK(cpqr_wide(P.Rt, l, l, l, P.Tl, l, piv1, P.Vh, P.tau, P.cpqr_scratch, ctrl, lim, 0, st,
                 fp1));
    CK(copy2d(P.Tl, l, l, l, L, ldo, nullptr, st));
    CK(form_q(P.Vh, l, P.tau, l, l, P.Qi, l, st, P.utw));
    CK(gather_cols(P.Q0, l, l, l, piv1, P.QB, l, st));
    const int eva = prof_start(kProfAssembly, st);
    if (P.ob.oz)
      RET(oz_right_product(P.ob, P.X, n, l, l, P.Qi, l, Pout, ldo, piv0, ctrl, nullptr, st));
    else
      CK(gemm_f64(false, RQLP_F64, P.X, l, P.Qi, l, Pout, ldo, n, l, l, 1.0, 0.0, P.ob.part, piv0,
                  nullptr, st));
    prof_stop(kProfAssembly, eva, st);
  } else {
    RET(orth(P.R0t, n, l, l, P.X, l, P.Rprev, P.ob, ctrl, site0, st, 2, again_tol_of(o)));
    CK(set_identity(P.QB, l, l, l, st));
    CK(set_identity(P.Macc, l, l, l, st));
    for (int i = 2; i <= o.d; ++i) {
      CK(transpose(P.Rprev, l, l, l, P.Xs, l, st));
      RET(orth(P.Xs, l, l, l, P.Qi, l, P.Rprev, P.ob, ctrl, site0 + i - 1, st, 2,
               again_tol_of(o)));
      double *acc = (i % 2 == 0) ? P.QB : P.Macc;
      CK(gemm_f64(false, RQLP_F64, acc, l, P.Qi, l, P.sm1, l, l, l, l, 1.0, 0.0, P.ob.part, nullptr,
                  nullptr, st));
      CK(copy2d(P.sm1, l, l, l, acc, l, nullptr, st));
    }
    RET(join());
    CK(gemm_f64(false, RQLP_F64, P.Q0, l, P.QB, l, P.sm1, l, l, l, l, 1.0, 0.0, P.ob.part, nullptr,
                nullptr, st));
    CK(copy2d(P.sm1, l, l, l, P.QB, l, nullptr, st));
    const int eva = prof_start(kProfAssembly, st);
    if (o.d <= 2) {
      // no odd inner factor beyond Q(1): P = Pi0 Q(1), a row scatter
      CK(permute_rows(P.X, n, l, l, piv0, Pout, ldo, true, st));
    } else if (P.ob.oz) {
      RET(oz_right_product(P.ob, P.X, n, l, l, P.Macc, l, Pout, ldo, piv0, ctrl, nullptr, st));
    } else {
      CK(gemm_f64(false, RQLP_F64, P.X, l, P.Macc, l, Pout, ldo, n, l, l, 1.0, 0.0, P.ob.part,
                  piv0, nullptr, st));
    }
    prof_stop(kProfAssembly, eva, st);
    if (o.d % 2 == 1) CK(transpose(P.Rprev, l, l, l, L, ldo, st));
    else CK(copy2d(P.Rprev, l, l, l, L, ldo, nullptr, st));
    CK(iota(piv1, l, st));
  }
  const int evq = prof_start(kProfAssembly, st);
  if (P.ob.oz)
    RET(oz_right_product(P.ob, Vb, m, l, ldv, P.QB, l, Q, ldo, nullptr, ctrl, nullptr, st));
  else
    CK(gemm_f64(false, RQLP_F64, Vb, ldv, P.QB, l, Q, ldo, m, l, l, 1.0, 0.0, P.ob.part, nullptr,
                nullptr, st));
  prof_stop(kProfAssembly, evq, st);
  return RQLP_OK;
}

__global__ void k_zero(double *p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 0.0;
}

// Block randomized QLP (Algorithm 4.1).  Per block j of b columns:
// Y_j = A Omega_j; V_j = qr(Y_j); V_j = qr(V_j - V_<j (V_<j^T V_j));
// B_j^T = A^T V_j; the pivoted QLP of B_j; Q_j = V_j Q_B(j), P_j = P_B(j),
// L = blkdiag(L_j).  The deflation A(j) = A(j-1) - V_j B_j is not formed:
// B_j = V_j^T A(j-1) = V_j^T A because V_j is orthogonal to V_<j (Section 4),
// which saves one pass over A per block.
// Block j of Algorithm 4.1 (l columns in all, blocks of o.block_b): Y_j =
// A Omega_j, V_j = qr(Y_j), re-orthonormalized against V_<j, Z = A^T V_j =
// B_j^T (B_j = V_j^T A: V_j is orthogonal to V_<j, so the deflation of
// A(j - 1) changes nothing), and the QLP of B_j into the j-th block columns of
// Q and P and the j-th diagonal block of L.  Leaves B_j^T in P.Z (n x b).
int brqlp_block(const Plan &P, const rqlp_opts &o, const void *A, int a_dtype, int64_t m,
                int64_t n, int64_t lda, int l, const double *Omega, int64_t ldo, double *Q,
                double *L, double *Pout, int32_t *piv0, int32_t *piv1, int j, int &site,
                cudaStream_t st) {
  const int b = o.block_b;
  double *Vj = P.V + (size_t)j * b;  // column block of V (m x l, ld l)
  RET(prod_nn(P, o, A, a_dtype, m, n, lda, Omega + (size_t)j * b, ldo, b, P.Y, st));
  RET(orth(P.Y, m, b, b, Vj, l, nullptr, P.ob, P.ctrl, site++, st));
  if (j > 0) {
    const int jb = j * b;
    // C = V_<j^T V_j (jb x b), then V_j -= V_<j C
    CK(gemm_f64(true, RQLP_F64, P.V, l, Vj, l, P.sm1, b, jb, b, m, 1.0, 0.0, P.ob.part, nullptr,
                nullptr, st));
    CK(gemm_f64(false, RQLP_F64, P.V, l, P.sm1, b, Vj, l, m, b, jb, -1.0, 1.0, P.ob.part,
                nullptr, nullptr, st));
    RET(orth(Vj, m, b, l, Vj, l, nullptr, P.ob, P.ctrl, site++, st));
  }
  RET(prod_tn(P, o, A, a_dtype, m, n, lda, Vj, l, b, P.Z, st));
  int32_t *p0 = (j == 0) ? piv0 : P.piv0;
  RET(qlp_stage(P, o, m, n, b, Vj, l, P.Z, Q + (size_t)j * b, L + (size_t)j * b * l + j * b,
                Pout + (size_t)j * b, l, p0, piv1 + (size_t)j * b, site, st, nullptr, nullptr,
                P.rvals + (size_t)j * b));
  site += o.d + 1;
  return RQLP_OK;
}

int run_brqlp(const Plan &P, const rqlp_opts &o, const void *A, int a_dtype, int64_t m, int64_t n,
              int64_t lda, int l, const double *Omega, int64_t ldo, double *Q, double *L,
              double *Pout, int32_t *piv0, int32_t *piv1, cudaStream_t st) {
  const int h = l / o.block_b;
  k_zero<<<(int)std::min<int64_t>(((int64_t)l * l + 255) / 256, 1024), 256, 0, st>>>(L, (int64_t)l * l);
  count_launch();
  CK(cudaGetLastError());
  int site = 0;
  for (int j = 0; j < h; ++j)
    RET(brqlp_block(P, o, A, a_dtype, m, n, lda, l, Omega, ldo, Q, L, Pout, piv0, piv1, j, site,
                    st));
  return RQLP_OK;
}

// Per-CTA partial sums of squares of an r x c row-major matrix (ld), in
// FP64 and in a fixed order (1-D blocks of 256: eight rows at a time, lanes
// along a row, then the CTA sum), so that the total is reproducible.
template <typename T>
__global__ void __launch_bounds__(256) k_sumsq(const T *__restrict__ X, int64_t r, int64_t c,
                                               int64_t ld, double *__restrict__ part) {
  __shared__ double red[32];
  const int lane = threadIdx.x & 31, rg = threadIdx.x >> 5;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 8 + rg; i < r; i += (int64_t)gridDim.x * 8)
    for (int64_t j = lane; j < c; j += 32) {
      const double v = (double)X[i * ld + j];
      s = fma(v, v, s);
    }
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// ||X||_F^2 of an r x c matrix (FP64 or FP32), summed on the host from the
// CTA partials in index order; synchronizes the stream.  `part` holds at
// least 4 x SMs doubles.
int sum_squares(const void *X, int dtype, int64_t r, int64_t c, int64_t ld, double *part,
                cudaStream_t st, double *out) {
  const int G = (int)std::max<int64_t>(1, std::min<int64_t>((r + 7) / 8, 4LL * num_sms()));
  if (dtype == RQLP_F32)
    k_sumsq<float><<<G, 256, 0, st>>>(static_cast<const float *>(X), r, c, ld, part);
  else
    k_sumsq<double><<<G, 256, 0, st>>>(static_cast<const double *>(X), r, c, ld, part);
  count_launch();
  CK(cudaGetLastError());
  std::vector<double> h((size_t)G);
  CK(cudaMemcpyAsync(h.data(), part, (size_t)G * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  double s = 0.0;
  for (int i = 0; i < G; ++i) s += h[(size_t)i];
  *out = s;
  return RQLP_OK;
}

// Launch shapes for a call with other factorizations in flight
// (rqlp_opts.in_flight >= 2), for the duration of the call: the FP64
// Cholesky on clusters of 8 CTAs, whose SMs are found sooner than 16 free
// SMs of one GPC while other kernels run (the results do not change).  The
// pivoted QR of B takes its half grid in qlp_stage.
struct InFlightShapes {
  Tuning saved;
  explicit InFlightShapes(const rqlp_opts &o) : saved(tuning()) {
    if (o.in_flight >= 2 && tuning().chol_ctas == 0) tuning().chol_ctas = 8;
  }
  ~InFlightShapes() { tuning() = saved; }
};

int run_rqlp(const void *A, int32_t a_dtype, int64_t m, int64_t n, int64_t lda, int32_t k,
             int32_t p, const double *Omega, int64_t ldo, const rqlp_opts &o, double *Q, double *L,
             double *Pout, double *Lvalues, int32_t *piv0, int32_t *piv1, void *ws, size_t ws_bytes,
             cudaStream_t st) {
  const InFlightShapes shapes(o);
  const int l = k + p;
  Plan P = carve(ws, m, n, l, o);
  if (P.bytes > ws_bytes) return RQLP_ERR_WORKSPACE;
  CK(cudaMemsetAsync(P.ctrl, 0, sizeof(Ctrl), st));
  // given pivots are read from the caller's arrays; the pivots the kernels
  // write then go to the workspace
  const int32_t *fp0 = o.fixed_pivots ? piv0 : nullptr;
  const int32_t *fp1 = (o.fixed_pivots && o.pivot2) ? piv1 : nullptr;
  int32_t *pv0 = (piv0 && !o.fixed_pivots) ? piv0 : P.piv0;
  int32_t *pv1 = (piv1 && !o.fixed_pivots) ? piv1 : P.piv1;
  // a rank-k truncation (the rank-k output of the abstract) factors at full
  // width l into the workspace and copies the leading k columns out
  double *Qo = Q, *Lo = L, *Po = Pout, *LVo = Lvalues;
  if (o.truncate_k) {
    Q = P.Qf;
    L = P.Lf;
    Pout = P.Pf;
    Lvalues = nullptr;
  }
  auto finish = [&]() -> int {
    if (!o.truncate_k) return RQLP_OK;
    CK(copy2d(Q, m, k, l, Qo, k, nullptr, st));
    CK(copy2d(L, k, k, l, Lo, k, nullptr, st));
    CK(copy2d(Pout, n, k, l, Po, k, nullptr, st));
    if (LVo) CK(diag_of(L, k, l, LVo, st));
    return RQLP_OK;
  };
  if (o.prec != RQLP_PREC_FP64) {
    const int ev = prof_start(kProfPrep, st);
    RET(mixed_prepare_A(P.mx, o.prec, A, a_dtype, m, n, lda, P.ctrl, st));
    prof_stop(kProfPrep, ev, st);
  }
  int site = 0;
  if (o.block_b > 0) {
    RET(run_brqlp(P, o, A, a_dtype, m, n, lda, l, Omega, ldo, Q, L, Pout, pv0, pv1, st));
    if (Lvalues) CK(diag_of(L, l, l, Lvalues, st));
    return finish();
  }
  // range finder (Section 2) with q power steps
  RET(prod_nn(P, o, A, a_dtype, m, n, lda, Omega, ldo, l, P.Y, st));
  // between power steps one CholeskyQR pass suffices: only the span of the
  // intermediate bases matters; the final V is CholeskyQR2.  In the mixed
  // forms, whose products carry BF16-level errors, the power steps' passes
  // run in FP32 (the span moves by about FP32 rounding).
  const bool lowp = !fp64_products(o.prec);
  for (int i = 0; i < o.q; ++i) {
    RET(orth(P.Y, m, l, l, P.V, l, nullptr, P.ob, P.ctrl, site++, st, 1, -1.0, lowp));
    RET(prod_tn(P, o, A, a_dtype, m, n, lda, P.V, l, l, P.Z, st));
    RET(orth(P.Z, n, l, l, P.W, l, nullptr, P.ob, P.ctrl, site++, st, 1, -1.0, lowp));
    RET(prod_nn(P, o, A, a_dtype, m, n, lda, P.W, l, l, P.Y, st));
  }
  RET(orth(P.Y, m, l, l, P.V, l, nullptr, P.ob, P.ctrl, site++, st, 2, again_tol_of(o)));
  // B^T = A^T V  (Algorithm 2.1 step 4)
  RET(prod_tn(P, o, A, a_dtype, m, n, lda, P.V, l, l, P.Z, st));
  RET(qlp_stage(P, o, m, n, l, P.V, l, P.Z, Q, L, Pout, l, pv0, pv1, site, st, fp0, fp1,
                P.rvals));
  if (Lvalues) CK(diag_of(L, l, l, Lvalues, st));
  return finish();
}

}  // namespace

namespace rqk {
void side_stream_prepare(cudaStream_t st) { side_for(st); }
void side_stream_in_capture(bool on) { t_side_in_capture = on; }
}  // namespace rqk

extern "C" {

const char *rqlp_status_string(int s) {
  switch (s) {
    case RQLP_OK: return "ok";
    case RQLP_WARN_SHIFTED_CHOLQR: return "warning: shifted CholeskyQR pass used";
    case RQLP_ERR_INVALID_ARG: return "invalid argument";
    case RQLP_ERR_NONFINITE: return "non-finite value in the data";
    case RQLP_ERR_RANK_DEFICIENT: return "Gram matrix singular after the shift";
    case RQLP_ERR_TIMEOUT: return "device-side wait timed out";
    case RQLP_ERR_CUDA: return "CUDA runtime error";
    case RQLP_ERR_WORKSPACE: return "workspace too small or misaligned";
    case RQLP_ERR_UNSUPPORTED: return "unsupported option";
    default: return "unknown status";
  }
}

int rqlp_version(void) { return 201; }

size_t rqlp_workspace_size(int64_t m, int64_t n, int32_t k, int32_t p, const rqlp_opts *opts) {
  if (!valid_dims(m, n, k, p) || !valid_opts(opts)) return 0;
  Plan P = carve(nullptr, m, n, k + p, *opts);
  return P.bytes + 256;
}

int rqlp(const void *A, int32_t a_dtype, int64_t m, int64_t n, int64_t lda, int32_t k, int32_t p,
         const double *Omega, int64_t ldo, const rqlp_opts *opts, double *Q, double *L, double *P,
         double *Lvalues, int32_t *piv0, int32_t *piv1, void *ws, size_t ws_bytes,
         rqlp_stream_t stream) {
  if (!valid_dims(m, n, k, p) || !valid_opts(opts)) return RQLP_ERR_INVALID_ARG;
  if (!A || !Omega || !Q || !L || !P || !ws) return RQLP_ERR_INVALID_ARG;
  if (a_dtype != RQLP_F64 && a_dtype != RQLP_F32) return RQLP_ERR_INVALID_ARG;
  const int l = k + p;
  if (lda < n || ldo < l) return RQLP_ERR_INVALID_ARG;
  if (opts->block_b > 0 && (l % opts->block_b != 0)) return RQLP_ERR_INVALID_ARG;
  if (opts->block_b > 0 && opts->q > 0) return RQLP_ERR_UNSUPPORTED;  // Algorithm 4.1 has no power steps
  if (opts->fixed_pivots && opts->block_b > 0) return RQLP_ERR_UNSUPPORTED;
  if (opts->prec == RQLP_PREC_FP64TC && l > 128) return RQLP_ERR_UNSUPPORTED;
  if (opts->fixed_pivots && (!piv0 || (opts->pivot2 && !piv1))) return RQLP_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return RQLP_ERR_WORKSPACE;
  return run_rqlp(A, a_dtype, m, n, lda, k, p, Omega, ldo, *opts, Q, L, P, Lvalues, piv0, piv1, ws,
                  ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

int rqlp_brqlp_tol(const void *A, int32_t a_dtype, int64_t m, int64_t n, int64_t lda, int32_t b,
                   int32_t l_max, double tol, const double *Omega, int64_t ldo,
                   const rqlp_opts *opts, double *Q, double *L, double *P, double *Lvalues,
                   int32_t *piv0, int32_t *piv1, int32_t *l_used, void *ws, size_t ws_bytes,
                   rqlp_stream_t stream) {
  if (!valid_dims(m, n, l_max, 0) || !valid_opts(opts)) return RQLP_ERR_INVALID_ARG;
  if (!A || !Omega || !Q || !L || !P || !l_used || !ws) return RQLP_ERR_INVALID_ARG;
  if (a_dtype != RQLP_F64 && a_dtype != RQLP_F32) return RQLP_ERR_INVALID_ARG;
  if (b < 1 || l_max % b != 0 || !(tol >= 0.0) || lda < n || ldo < l_max)
    return RQLP_ERR_INVALID_ARG;
  if (opts->q > 0) return RQLP_ERR_UNSUPPORTED;  // Algorithm 4.1 has no power steps
  if (opts->fixed_pivots || opts->truncate_k) return RQLP_ERR_UNSUPPORTED;
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return RQLP_ERR_WORKSPACE;
  *l_used = 0;
  rqlp_opts o = *opts;
  o.block_b = b;
  const InFlightShapes shapes(o);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Plan W = carve(ws, m, n, l_max, o);
  if (W.bytes > ws_bytes) return RQLP_ERR_WORKSPACE;
  CK(cudaMemsetAsync(W.ctrl, 0, sizeof(Ctrl), st));
  int32_t *pv0 = piv0 ? piv0 : W.piv0;
  int32_t *pv1 = piv1 ? piv1 : W.piv1;
  if (o.prec != RQLP_PREC_FP64) RET(mixed_prepare_A(W.mx, o.prec, A, a_dtype, m, n, lda, W.ctrl, st));
  const int64_t ll = (int64_t)l_max * l_max;
  k_zero<<<(int)std::min<int64_t>((ll + 255) / 256, 1024), 256, 0, st>>>(L, ll);
  count_launch();
  CK(cudaGetLastError());
  // the stopping rule of eq. 2.1: ||A - V V^T A||_F^2 = ||A||_F^2 - ||B||_F^2
  double a2 = 0.0, b2 = 0.0;
  RET(sum_squares(A, a_dtype, m, n, lda, W.ob.part, st, &a2));
  int used = 0, site = 0;
  for (int j = 0; j < l_max / b; ++j) {
    RET(brqlp_block(W, o, A, a_dtype, m, n, lda, l_max, Omega, ldo, Q, L, P, pv0, pv1, j, site,
                    st));
    double z2 = 0.0;
    RET(sum_squares(W.Z, RQLP_F64, n, b, b, W.ob.part, st, &z2));  // ||B_j||_F^2 (synchronizes)
    int status = 0;
    CK(cudaMemcpy(&status, W.ctrl, sizeof(int), cudaMemcpyDeviceToHost));
    if (status < 0) return status;
    b2 += z2;
    used = j + 1;
    if (a2 - b2 <= tol * tol * a2) break;
  }
  *l_used = used * b;
  if (Lvalues) CK(diag_of(L, used * b, l_max, Lvalues, st));
  return rqlp_read_status(ws, stream);
}

int rqlp_rvalues(const void *ws, int64_t m, int64_t n, int32_t k, int32_t p, const rqlp_opts *opts,
                 double *Rvalues, rqlp_stream_t stream) {
  if (!ws || !Rvalues || !valid_dims(m, n, k, p) || !valid_opts(opts)) return RQLP_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return RQLP_ERR_WORKSPACE;
  Plan P = carve(const_cast<void *>(ws), m, n, k + p, *opts);
  const int cnt = opts->truncate_k ? k : k + p;
  CK(cudaMemcpyAsync(Rvalues, P.rvals, (size_t)cnt * sizeof(double), cudaMemcpyDeviceToDevice,
                     reinterpret_cast<cudaStream_t>(stream)));
  return RQLP_OK;
}

int rqlp_read_status(const void *ws, rqlp_stream_t stream) {
  if (!ws) return RQLP_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return RQLP_ERR_CUDA;
  int s = 0;
  if (cudaMemcpy(&s, ws, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return RQLP_ERR_CUDA;
  return s;
}

size_t rqlp_host_workspace_size(int64_t m, int64_t n, int32_t k, int32_t p, const rqlp_opts *opts,
                                int32_t a_dtype) {
  const size_t base = rqlp_workspace_size(m, n, k, p, opts);
  if (!base) return 0;
  const int64_t l = k + p;
  const size_t esz = a_dtype == RQLP_F32 ? 4 : 8;
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  return up(base) + up((size_t)m * n * esz) + up((size_t)n * l * 8) + up((size_t)m * l * 8) +
         up((size_t)l * l * 8) + up((size_t)n * l * 8) + up((size_t)l * 8) + up((size_t)n * 4) +
         up((size_t)l * 4);
}

int rqlp_host_async(const void *A_host, int32_t a_dtype, int64_t m, int64_t n, int32_t k,
                    int32_t p, const double *Omega_host, const rqlp_opts *opts, double *Q_host,
                    double *L_host, double *P_host, double *Lvalues_host, int32_t *piv0_host,
                    int32_t *piv1_host, void *ws, size_t ws_bytes, rqlp_stream_t stream) {
  if (!valid_dims(m, n, k, p) || !valid_opts(opts)) return RQLP_ERR_INVALID_ARG;
  if (!A_host || !Omega_host || !Q_host || !L_host || !P_host || !ws) return RQLP_ERR_INVALID_ARG;
  if (a_dtype != RQLP_F64 && a_dtype != RQLP_F32) return RQLP_ERR_INVALID_ARG;
  const size_t need = rqlp_host_workspace_size(m, n, k, p, opts, a_dtype);
  if (ws_bytes < need || reinterpret_cast<uintptr_t>(ws) % 256 != 0) return RQLP_ERR_WORKSPACE;
  if (opts->fixed_pivots && (!piv0_host || (opts->pivot2 && !piv1_host)))
    return RQLP_ERR_INVALID_ARG;
  const int64_t l = k + p;
  const int64_t w = opts->truncate_k ? k : l;  // width of the outputs
  const size_t esz = a_dtype == RQLP_F32 ? 4 : 8;
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  char *c = reinterpret_cast<char *>(ws);
  const size_t base = up(rqlp_workspace_size(m, n, k, p, opts));
  char *dA = c + base;
  double *dO = reinterpret_cast<double *>(dA + up((size_t)m * n * esz));
  double *dQ = reinterpret_cast<double *>(reinterpret_cast<char *>(dO) + up((size_t)n * l * 8));
  double *dL = reinterpret_cast<double *>(reinterpret_cast<char *>(dQ) + up((size_t)m * l * 8));
  double *dP = reinterpret_cast<double *>(reinterpret_cast<char *>(dL) + up((size_t)l * l * 8));
  double *dLv = reinterpret_cast<double *>(reinterpret_cast<char *>(dP) + up((size_t)n * l * 8));
  int32_t *dp0 = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(dLv) + up((size_t)l * 8));
  int32_t *dp1 = reinterpret_cast<int32_t *>(reinterpret_cast<char *>(dp0) + up((size_t)n * 4));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  CK(cudaMemcpyAsync(dA, A_host, (size_t)m * n * esz, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(dO, Omega_host, (size_t)n * l * 8, cudaMemcpyHostToDevice, st));
  if (opts->fixed_pivots) {
    // given pivots are inputs: the first l of piv0 (and l of piv1 for RQLP)
    CK(cudaMemcpyAsync(dp0, piv0_host, (size_t)l * 4, cudaMemcpyHostToDevice, st));
    if (opts->pivot2) CK(cudaMemcpyAsync(dp1, piv1_host, (size_t)l * 4, cudaMemcpyHostToDevice, st));
  }
  int r = rqlp(dA, a_dtype, m, n, n, k, p, dO, l, opts, dQ, dL, dP, dLv, dp0, dp1, c, base,
               stream);
  if (r != RQLP_OK) return r;
  CK(cudaMemcpyAsync(Q_host, dQ, (size_t)m * w * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(L_host, dL, (size_t)w * w * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(P_host, dP, (size_t)n * w * 8, cudaMemcpyDeviceToHost, st));
  if (Lvalues_host) CK(cudaMemcpyAsync(Lvalues_host, dLv, (size_t)w * 8, cudaMemcpyDeviceToHost, st));
  if (!opts->fixed_pivots) {
    if (piv0_host) CK(cudaMemcpyAsync(piv0_host, dp0, (size_t)n * 4, cudaMemcpyDeviceToHost, st));
    if (piv1_host) CK(cudaMemcpyAsync(piv1_host, dp1, (size_t)l * 4, cudaMemcpyDeviceToHost, st));
  }
  return RQLP_OK;
}

int rqlp_host(const void *A_host, int32_t a_dtype, int64_t m, int64_t n, int32_t k, int32_t p,
              const double *Omega_host, const rqlp_opts *opts, double *Q_host, double *L_host,
              double *P_host, double *Lvalues_host, int32_t *piv0_host, int32_t *piv1_host,
              void *ws, size_t ws_bytes, rqlp_stream_t stream) {
  const int r = rqlp_host_async(A_host, a_dtype, m, n, k, p, Omega_host, opts, Q_host, L_host,
                                P_host, Lvalues_host, piv0_host, piv1_host, ws, ws_bytes, stream);
  if (r != RQLP_OK) return r;
  return rqlp_read_status(ws, stream);
}

// ---------------------------------------------------------------- stages
size_t rqlp_stage_workspace_size(int64_t rows, int64_t cols, int32_t l, int32_t prec) {
  if (rows <= 0 || cols <= 0 || l < 1 || l > kMaxL) return 0;
  rqlp_opts o;
  std::memset(&o, 0, sizeof(o));
  o.prec = prec;
  o.pivot2 = 1;
  const int64_t m = rows, n = std::max<int64_t>(cols, l);
  Plan P = carve(nullptr, std::max<int64_t>(m, l), n, l, o);
  return P.bytes + 256;
}

int rqlp_sketch(const void *A, int32_t a_dtype, int64_t m, int64_t n, int64_t lda, const double *W,
                int64_t ldw, int32_t l, int32_t prec, double *Y, int64_t ldy, void *ws,
                size_t ws_bytes, rqlp_stream_t stream) {
  if (!A || !W || !Y || !ws || m <= 0 || n <= 0 || l < 1 || l > kMaxL || lda < n || ldw < l ||
      ldy < l || (a_dtype != RQLP_F64 && a_dtype != RQLP_F32))
    return RQLP_ERR_INVALID_ARG;
  if (prec < RQLP_PREC_FP64 || prec > RQLP_PREC_FP64TC) return RQLP_ERR_INVALID_ARG;
  if (prec == RQLP_PREC_FP64TC && l > 128) return RQLP_ERR_UNSUPPORTED;
  rqlp_opts o;
  std::memset(&o, 0, sizeof(o));
  o.prec = prec;
  Plan P = carve(ws, std::max<int64_t>(m, l), std::max<int64_t>(n, l), l, o);
  if (P.bytes > ws_bytes || reinterpret_cast<uintptr_t>(ws) % 256) return RQLP_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  CK(cudaMemsetAsync(P.ctrl, 0, sizeof(Ctrl), st));
  if (prec != RQLP_PREC_FP64) {
    RET(mixed_prepare_A(P.mx, prec, A, a_dtype, m, n, lda, P.ctrl, st));
    double *tmpY = ldy == l ? Y : P.Y;
    RET(mixed_nn(P.mx, prec, m, n, W, ldw, l, tmpY, P.ctrl, 0, st));
    if (tmpY != Y) CK(copy2d(tmpY, m, l, l, Y, ldy, nullptr, st));
    return RQLP_OK;
  }
  CK(gemm_f64(false, a_dtype, A, lda, W, ldw, Y, ldy, m, l, n, 1.0, 0.0, P.ob.part, nullptr,
              nullptr, st));
  return RQLP_OK;
}

int rqlp_project(const void *A, int32_t a_dtype, int64_t m, int64_t n, int64_t lda, const double *V,
                 int64_t ldv, int32_t l, int32_t prec, double *Z, int64_t ldz, void *ws,
                 size_t ws_bytes, rqlp_stream_t stream) {
  if (!A || !V || !Z || !ws || m <= 0 || n <= 0 || l < 1 || l > kMaxL || lda < n || ldv < l ||
      ldz < l || (a_dtype != RQLP_F64 && a_dtype != RQLP_F32))
    return RQLP_ERR_INVALID_ARG;
  if (prec < RQLP_PREC_FP64 || prec > RQLP_PREC_FP64TC) return RQLP_ERR_INVALID_ARG;
  if (prec == RQLP_PREC_FP64TC && l > 128) return RQLP_ERR_UNSUPPORTED;
  rqlp_opts o;
  std::memset(&o, 0, sizeof(o));
  o.prec = prec;
  Plan P = carve(ws, std::max<int64_t>(m, l), std::max<int64_t>(n, l), l, o);
  if (P.bytes > ws_bytes || reinterpret_cast<uintptr_t>(ws) % 256) return RQLP_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  CK(cudaMemsetAsync(P.ctrl, 0, sizeof(Ctrl), st));
  if (prec != RQLP_PREC_FP64) {
    RET(mixed_prepare_A(P.mx, prec, A, a_dtype, m, n, lda, P.ctrl, st));
    double *tmpZ = ldz == l ? Z : P.Z;
    RET(mixed_tn(P.mx, prec, m, n, V, ldv, l, tmpZ, P.ctrl, 0, st));
    if (tmpZ != Z) CK(copy2d(tmpZ, n, l, l, Z, ldz, nullptr, st));
    return RQLP_OK;
  }
  CK(gemm_f64(true, a_dtype, A, lda, V, ldv, Z, ldz, n, l, m, 1.0, 0.0, P.ob.part, nullptr,
              nullptr, st));
  return RQLP_OK;
}

int rqlp_orth(const double *X, int64_t rows, int32_t l, int64_t ldx, double *Qx, int64_t ldq,
              double *R, void *ws, size_t ws_bytes, rqlp_stream_t stream) {
  if (!X || !Qx || !ws || rows <= 0 || l < 1 || l > kMaxL || l > rows || ldx < l || ldq < l)
    return RQLP_ERR_INVALID_ARG;
  rqlp_opts o;
  std::memset(&o, 0, sizeof(o));
  Plan P = carve(ws, rows, l, l, o);
  if (P.bytes > ws_bytes || reinterpret_cast<uintptr_t>(ws) % 256) return RQLP_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  CK(cudaMemsetAsync(P.ctrl, 0, sizeof(Ctrl), st));
  return orth(X, rows, l, ldx, Qx, ldq, R, P.ob, P.ctrl, 0, st);
}

int rqlp_cpqr(const double *Bt, int64_t n, int32_t l, int64_t ldb, double *R0t, int32_t *piv0,
              double *Q0, void *ws, size_t ws_bytes, rqlp_stream_t stream) {
  if (!Bt || !R0t || !piv0 || !ws || n <= 0 || l < 1 || l > kMaxL || l > n || ldb < l)
    return RQLP_ERR_INVALID_ARG;
  rqlp_opts o;
  std::memset(&o, 0, sizeof(o));
  Plan P = carve(ws, l, n, l, o);
  if (P.bytes > ws_bytes || reinterpret_cast<uintptr_t>(ws) % 256) return RQLP_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  CK(cudaMemsetAsync(P.ctrl, 0, sizeof(Ctrl), st));
  CK(cpqr_wide(Bt, n, l, ldb, R0t, l, piv0, P.Vh, P.tau, P.cpqr_scratch, P.ctrl, 0, 0, st));
  if (Q0) CK(form_q(P.Vh, l, P.tau, l, l, Q0, l, st));
  return RQLP_OK;
}

}  // extern "C"

// ---------------------------------------------- deterministic truncated QLP
// Stewart's pivoted QLP truncated at t steps (Section 1, eq. 1.2; the "QLP"
// the paper's Section 5 compares the randomized methods with): the first t
// steps of the column-pivoted Householder QR of A, A Pi0 ~= Q0 R0 with R0 the
// first t rows of R (t x n), then R0^T = Q1 R1 (an unpivoted CholeskyQR2, or,
// with pivot2, the CPQR of its t x t R factor as in Algorithm 2.1), so that
// A ~= Q L P^T with L = R1^T.
namespace {

struct QlpPlan {
  Ctrl *ctrl;
  OrthBufs ob;
  double *At, *R0t, *Vh, *tau, *S, *Wt, *WtT, *Q0, *X, *Racc, *Rt, *Tl, *Qi, *Vh2, *tau2, *utw;
  int32_t *piv0, *piv1;
  void *tall_scratch, *small_scratch;
  size_t bytes;
};

QlpPlan carve_qlp(void *ws, int64_t m, int64_t n, int t) {
  QlpPlan q;
  Arena a(ws);
  q.ctrl = a.take<Ctrl>(1);
  carve_orth(a, n, t, m, n, q.ob, nullptr);
  const size_t tt = (size_t)t * t;
  q.At = a.take<double>((size_t)n * m);
  q.R0t = a.take<double>((size_t)n * t);
  q.Vh = a.take<double>((size_t)m * t);
  q.tau = a.take<double>((size_t)t);
  q.S = a.take<double>(tt);
  q.Wt = a.take<double>(tt);
  q.WtT = a.take<double>(tt);
  q.Q0 = a.take<double>((size_t)m * t);
  q.X = a.take<double>((size_t)n * t);
  q.Racc = a.take<double>(tt);
  q.Rt = a.take<double>(tt);
  q.Tl = a.take<double>(tt);
  q.Qi = a.take<double>(tt);
  q.Vh2 = a.take<double>(tt);
  q.tau2 = a.take<double>((size_t)t);
  q.utw = a.take<double>(2 * tt);
  q.piv0 = a.take<int32_t>((size_t)n);
  q.piv1 = a.take<int32_t>((size_t)t);
  q.tall_scratch = a.take<char>(cpqr_tall_ws_bytes(n, m));
  q.small_scratch = a.take<char>(cpqr_ws_bytes(t, t));
  q.bytes = a.off;
  return q;
}

// Q0 = H_0 ... H_{t-1} [I; 0] (m x t) from the reflectors Vh (m x t, ld t)
// by the compact-WY form I - V T V^T with T^-1 = diag(1 / tau) + striu(V^T V):
// Q0 = [I; 0] - V (T V(:t, :)^T).
int form_q_tall(const QlpPlan &q, int64_t m, int t, double *Q0, cudaStream_t st) {
  CK(gemm_f64(true, RQLP_F64, q.Vh, t, q.Vh, t, q.S, t, t, t, m, 1.0, 0.0, q.ob.part, nullptr,
              nullptr, st));
  CK(tri_rows(q.S, t, q.tau, t, q.Vh, t, q.Wt, t, t, true, st));
  CK(transpose(q.Wt, t, t, t, q.WtT, t, st));
  CK(set_identity(Q0, m, t, t, st));
  CK(gemm_f64(false, RQLP_F64, q.Vh, t, q.WtT, t, Q0, t, m, t, t, -1.0, 1.0, q.ob.part, nullptr,
              nullptr, st));
  return RQLP_OK;
}

int run_qlp(const void *A, int64_t m, int64_t n, int64_t lda, int t, const rqlp_opts &o,
            double *Q, double *L, double *Pout, double *Lvalues, int32_t *piv0, int32_t *piv1,
            void *ws, size_t ws_bytes, cudaStream_t st) {
  QlpPlan q = carve_qlp(ws, m, n, t);
  if (q.bytes > ws_bytes) return RQLP_ERR_WORKSPACE;
  CK(cudaMemsetAsync(q.ctrl, 0, sizeof(Ctrl), st));
  const unsigned long long lim = (unsigned long long)o.spin_limit_ns;
  int32_t *pv0 = piv0 ? piv0 : q.piv0;
  int32_t *pv1 = piv1 ? piv1 : q.piv1;
  // columns of A as rows
  CK(transpose(static_cast<const double *>(A), m, n, lda, q.At, m, st));
  const int ev = prof_start(kProfCpqr, st);
  CK(cpqr_tall(q.At, n, m, t, m, q.R0t, t, pv0, q.Vh, t, q.tau, q.tall_scratch, q.ctrl, lim, st));
  prof_stop(kProfCpqr, ev, st);
  RET(form_q_tall(q, m, t, o.pivot2 ? q.Q0 : Q, st));
  if (o.pivot2) {
    RET(orth(q.R0t, n, t, t, q.X, t, q.Racc, q.ob, q.ctrl, 0, st, 2, -1.0));
    CK(transpose(q.Racc, t, t, t, q.Rt, t, st));
    CK(cpqr_wide(q.Rt, t, t, t, q.Tl, t, pv1, q.Vh2, q.tau2, q.small_scratch, q.ctrl, lim, 0, st));
    CK(copy2d(q.Tl, t, t, t, L, t, nullptr, st));
    CK(form_q(q.Vh2, t, q.tau2, t, t, q.Qi, t, st, q.utw));
    CK(gather_cols(q.Q0, m, t, t, pv1, Q, t, st));
    CK(gemm_f64(false, RQLP_F64, q.X, t, q.Qi, t, Pout, t, n, t, t, 1.0, 0.0, q.ob.part, pv0,
                nullptr, st));
  } else {
    RET(orth(q.R0t, n, t, t, q.X, t, q.Racc, q.ob, q.ctrl, 0, st, 2, -1.0));
    CK(transpose(q.Racc, t, t, t, L, t, st));
    CK(permute_rows(q.X, n, t, t, pv0, Pout, t, true, st));
    CK(iota(pv1, t, st));
  }
  if (Lvalues) CK(diag_of(L, t, t, Lvalues, st));
  return RQLP_OK;
}

}  // namespace

extern "C" {

size_t rqlp_qlp_workspace_size(int64_t m, int64_t n, int32_t t, const rqlp_opts *opts) {
  if (!opts || m <= 0 || n <= 0 || t < 1 || t > kMaxL || t > m || t > n || m > 16384) return 0;
  return carve_qlp(nullptr, m, n, t).bytes + 256;
}

int rqlp_qlp(const void *A, int32_t a_dtype, int64_t m, int64_t n, int64_t lda, int32_t t,
             const rqlp_opts *opts, double *Q, double *L, double *P, double *Lvalues,
             int32_t *piv0, int32_t *piv1, void *ws, size_t ws_bytes, rqlp_stream_t stream) {
  if (!opts || !A || !Q || !L || !P || !ws || lda < n) return RQLP_ERR_INVALID_ARG;
  if (rqlp_qlp_workspace_size(m, n, t, opts) == 0) return RQLP_ERR_INVALID_ARG;
  if (opts->pivot2 != 0 && opts->pivot2 != 1) return RQLP_ERR_INVALID_ARG;
  if (a_dtype != RQLP_F64) return RQLP_ERR_UNSUPPORTED;
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return RQLP_ERR_WORKSPACE;
  return run_qlp(A, m, n, lda, t, *opts, Q, L, P, Lvalues, piv0, piv1, ws, ws_bytes,
                 reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"

// ------------------------------------------------------------------ adjoint
// Reverse-mode derivative of RQLP (Algorithm 2.1, pivot2 = 1) with the
// column pivots held fixed: dA = J^T (dQ, dL, dP).  The forward is recomputed
// (Y is not stored by rqlp()), keeping the range-finder bases and their R
// factors, then every product and QR is swept backwards.  For a thin QR
// X = Q R:  dX = (dQ + Q copyltu(R dR^T - dQ^T Q)) R^{-T};  for the wide
// QR C = Q [U | V] the V block adds C2 dV^T to dQ and Q dV to dC2.  All
// rank-l updates of dA are gathered into one product [L_1 .. L_P][R_1 .. R_P]^T
// with K = (2q + 2) l.
namespace {

struct BwdPlan {
  Plan F;
  double *Vs, *RYs, *Ws, *RZs, *RY, *Q1, *R1;
  double *M, *S, *Rinv, *RinvT, *sm2, *dQ0, *dQB, *dR1, *U, *dU, *dC1, *QBt, *Q0t;
  double *T, *dV, *dW, *dQ1, *dXp, *dX, *dCt, *dBt;
  double *Lcat, *Rcat, *RcatT;
  size_t bytes;
};

BwdPlan carve_bwd(void *ws, int64_t m, int64_t n, int l, const rqlp_opts &o) {
  BwdPlan b;
  b.F = carve(ws, m, n, l, o);
  Arena a(ws ? reinterpret_cast<char *>(ws) + (b.F.bytes + 255) / 256 * 256 : nullptr);
  const int q = o.q, P = 2 * q + 2;
  const size_t ll = (size_t)l * l;
  const int64_t big = std::max(m, n);
  b.Vs = a.take<double>((size_t)std::max(q, 1) * m * l);
  b.RYs = a.take<double>((size_t)std::max(q, 1) * ll);
  b.Ws = a.take<double>((size_t)std::max(q, 1) * n * l);
  b.RZs = a.take<double>((size_t)std::max(q, 1) * ll);
  b.RY = a.take<double>(ll);
  b.Q1 = a.take<double>((size_t)n * l);
  b.R1 = a.take<double>(ll);
  for (double **p : {&b.M, &b.S, &b.Rinv, &b.RinvT, &b.sm2, &b.dQ0, &b.dQB, &b.dR1, &b.U, &b.dU,
                     &b.dC1, &b.QBt, &b.Q0t})
    *p = a.take<double>(ll);
  for (double **p : {&b.T, &b.dV, &b.dW, &b.dQ1, &b.dXp, &b.dX, &b.dCt, &b.dBt})
    *p = a.take<double>((size_t)big * l);
  b.Lcat = a.take<double>((size_t)m * P * l);
  b.Rcat = a.take<double>((size_t)n * P * l);
  b.RcatT = a.take<double>((size_t)P * l * n);
  b.bytes = (b.F.bytes + 255) / 256 * 256 + a.off;
  return b;
}

// dX (rows x l, ld lddx) = (dQ + Q copyltu(M)) R^{-T}, M = R dR^T - dQ^T Q.
int qr_vjp_dev(const BwdPlan &B, const double *Qm, int64_t ldq, const double *R, const double *dQ,
               int64_t lddq, const double *dR, int64_t rows, int l, double *dX, int64_t lddx,
               cudaStream_t st) {
  double *part = B.F.ob.part;
  CK(gemm_f64(true, RQLP_F64, dQ, lddq, Qm, ldq, B.M, l, l, l, rows, -1.0, 0.0, part, nullptr,
              nullptr, st));
  if (dR) {
    CK(transpose(dR, l, l, l, B.sm2, l, st));
    CK(gemm_f64(false, RQLP_F64, R, l, B.sm2, l, B.M, l, l, l, l, 1.0, 1.0, part, nullptr, nullptr,
                st));
  }
  CK(copyltu(B.M, l, B.S, st));
  CK(copy2d(dQ, rows, l, lddq, B.T, l, nullptr, st));
  CK(gemm_f64(false, RQLP_F64, Qm, ldq, B.S, l, B.T, l, rows, l, l, 1.0, 1.0, part, nullptr,
              nullptr, st));
  CK(trinv_upper(R, l, B.Rinv, nullptr, st));
  CK(transpose(B.Rinv, l, l, l, B.RinvT, l, st));
  CK(gemm_f64(false, RQLP_F64, B.T, l, B.RinvT, l, dX, lddx, rows, l, l, 1.0, 0.0, part, nullptr,
              nullptr, st));
  return RQLP_OK;
}

__global__ void k_fill(double *p, int64_t n, double v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

cudaError_t zero(double *p, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_fill<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(p, n, 0.0);
  count_launch();
  return cudaGetLastError();
}

int run_backward(const void *A, int32_t a_dtype, int64_t m, int64_t n, int64_t lda, int l,
                 const double *Omega, int64_t ldo, const rqlp_opts &o, const int32_t *fp0,
                 const int32_t *fp1, const double *dQ, const double *dL, const double *dP,
                 double *dA, int64_t ldda, void *ws, size_t ws_bytes, cudaStream_t st) {
  BwdPlan B = carve_bwd(ws, m, n, l, o);
  if (B.bytes > ws_bytes) return RQLP_ERR_WORKSPACE;
  const Plan &F = B.F;
  Ctrl *ctrl = F.ctrl;
  const int q = o.q, Pc = 2 * q + 2;
  const int64_t ldc = (int64_t)Pc * l;
  const size_t ml = (size_t)m * l, nl = (size_t)n * l, ll = (size_t)l * l;
  double *part = F.ob.part;
  const unsigned long long lim = (unsigned long long)o.spin_limit_ns;
  CK(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st));
  // the recomputed forward's products with A run in the forward's precision,
  // so the mixed forms need their copies of A
  if (o.prec != RQLP_PREC_FP64) RET(mixed_prepare_A(F.mx, o.prec, A, a_dtype, m, n, lda, ctrl, st));
  // ---- forward with intermediates (Algorithm 2.1) ----
  int site = 0;
  RET(prod_nn(F, o, A, a_dtype, m, n, lda, Omega, ldo, l, F.Y, st));
  for (int i = 0; i < q; ++i) {
    RET(orth(F.Y, m, l, l, B.Vs + i * ml, l, B.RYs + i * ll, F.ob, ctrl, site++, st));
    RET(prod_tn(F, o, A, a_dtype, m, n, lda, B.Vs + i * ml, l, l, F.Z, st));
    RET(orth(F.Z, n, l, l, B.Ws + i * nl, l, B.RZs + i * ll, F.ob, ctrl, site++, st));
    RET(prod_nn(F, o, A, a_dtype, m, n, lda, B.Ws + i * nl, l, l, F.Y, st));
  }
  RET(orth(F.Y, m, l, l, F.V, l, B.RY, F.ob, ctrl, site++, st));
  RET(prod_tn(F, o, A, a_dtype, m, n, lda, F.V, l, l, F.Z, st));  // B^T
  CK(cpqr_wide(F.Z, n, l, l, F.R0t, l, F.piv0, F.Vh, F.tau, F.cpqr_scratch, ctrl, lim, 0, st,
               fp0));
  CK(form_q(F.Vh, l, F.tau, l, l, F.Q0, l, st));
  RET(orth(F.R0t, n, l, l, F.X, l, F.Racc, F.ob, ctrl, site++, st));
  CK(transpose(F.Racc, l, l, l, F.Rt, l, st));
  CK(cpqr_wide(F.Rt, l, l, l, F.Tl, l, F.piv1, F.Vh, F.tau, F.cpqr_scratch, ctrl, lim, 0, st,
               fp1));
  CK(form_q(F.Vh, l, F.tau, l, l, F.Qi, l, st));
  CK(gemm_f64(false, RQLP_F64, F.X, l, F.Qi, l, B.Q1, l, n, l, l, 1.0, 0.0, part, nullptr, nullptr,
              st));                                               // Q1 = Qa Qc
  CK(transpose(F.Tl, l, l, l, B.R1, l, st));                     // R1 = L^T
  CK(gather_cols(F.Q0, l, l, l, F.piv1, F.QB, l, st));            // Q_B = Q0 Pi1
  // ---- step 7: Q = V Q_B, L = R1^T, P = Pi0 Q1 ----
  if (dQ) {
    CK(transpose(F.QB, l, l, l, B.QBt, l, st));
    CK(gemm_f64(false, RQLP_F64, dQ, l, B.QBt, l, B.dV, l, m, l, l, 1.0, 0.0, part, nullptr,
                nullptr, st));
    CK(gemm_f64(true, RQLP_F64, F.V, l, dQ, l, B.dQB, l, l, l, m, 1.0, 0.0, part, nullptr, nullptr,
                st));
    CK(zero(B.dQ0, ll, st));
    CK(scatter_cols(B.dQB, l, l, l, F.piv1, B.dQ0, l, st));
  } else {
    CK(zero(B.dV, ml, st));
    CK(zero(B.dQ0, ll, st));
  }
  if (dP) CK(permute_rows(dP, n, l, l, F.piv0, B.dQ1, l, false, st));
  else CK(zero(B.dQ1, nl, st));
  if (dL) {
    CK(transpose(dL, l, l, l, B.dR1, l, st));
    CK(zero_triangle(B.dR1, l, l, true, st));
  } else {
    CK(zero(B.dR1, ll, st));
  }
  // ---- step 6: R0^T Pi1 = Q1 R1 ----
  RET(qr_vjp_dev(B, B.Q1, l, B.R1, B.dQ1, l, B.dR1, n, l, B.dXp, l, st));
  CK(zero(B.dX, nl, st));
  CK(scatter_cols(B.dXp, n, l, l, F.piv1, B.dX, l, st));
  CK(mask_lower_trapezoid(B.dX, n, l, l, st));  // dR0^T: R0 is upper trapezoidal
  // ---- step 5: B Pi0 = Q0 R0, R0 = [U | V] ----
  CK(transpose(F.R0t, l, l, l, B.U, l, st));
  CK(transpose(B.dX, l, l, l, B.dU, l, st));
  if (n > l) {
    CK(gemm_f64(true, RQLP_F64, F.R0t + ll, l, B.dX + ll, l, B.M, l, l, l, n - l, 1.0, 0.0, part,
                nullptr, nullptr, st));
    CK(gemm_f64(false, RQLP_F64, F.Q0, l, B.M, l, B.dQ0, l, l, l, l, 1.0, 1.0, part, nullptr,
                nullptr, st));
  }
  RET(qr_vjp_dev(B, F.Q0, l, B.U, B.dQ0, l, B.dU, l, l, B.dC1, l, st));
  CK(transpose(B.dC1, l, l, l, B.dCt, l, st));
  if (n > l) {
    CK(transpose(F.Q0, l, l, l, B.Q0t, l, st));
    CK(gemm_f64(false, RQLP_F64, B.dX + ll, l, B.Q0t, l, B.dCt + ll, l, n - l, l, l, 1.0, 0.0, part,
                nullptr, nullptr, st));
  }
  CK(permute_rows(B.dCt, n, l, l, F.piv0, B.dBt, l, true, st));  // dB[:, piv0] = dC
  // ---- step 4: B = V^T A ----
  CK(gemm_f64(false, a_dtype, A, lda, B.dBt, l, B.dV, l, m, l, n, 1.0, 1.0, part, nullptr, nullptr,
              st));
  int pc = 0;
  CK(copy2d(F.V, m, l, l, B.Lcat + pc * l, ldc, nullptr, st));
  CK(copy2d(B.dBt, n, l, l, B.Rcat + pc * l, ldc, nullptr, st));
  ++pc;
  // ---- step 3: V = qr(Y_q) ----
  RET(qr_vjp_dev(B, F.V, l, B.RY, B.dV, l, nullptr, m, l, B.Lcat + pc * l, ldc, st));
  // ---- step 2, backwards ----
  for (int i = q - 1; i >= 0; --i) {
    const double *dY = B.Lcat + pc * l;
    CK(copy2d(B.Ws + i * nl, n, l, l, B.Rcat + pc * l, ldc, nullptr, st));  // dA += dY W^T
    ++pc;
    CK(gemm_f64(true, a_dtype, A, lda, dY, ldc, B.dW, l, n, l, m, 1.0, 0.0, part, nullptr, nullptr,
                st));                                                        // dW = A^T dY
    RET(qr_vjp_dev(B, B.Ws + i * nl, l, B.RZs + i * ll, B.dW, l, nullptr, n, l, B.Rcat + pc * l,
                   ldc, st));                                                // dZ
    CK(copy2d(B.Vs + i * ml, m, l, l, B.Lcat + pc * l, ldc, nullptr, st));   // dA += V dZ^T
    CK(gemm_f64(false, a_dtype, A, lda, B.Rcat + pc * l, ldc, B.dV, l, m, l, n, 1.0, 0.0, part,
                nullptr, nullptr, st));                                      // dV = A dZ
    ++pc;
    RET(qr_vjp_dev(B, B.Vs + i * ml, l, B.RYs + i * ll, B.dV, l, nullptr, m, l, B.Lcat + pc * l,
                   ldc, st));                                                // dY_{i-1}
  }
  // ---- step 1: Y_0 = A Omega ----
  CK(copy2d(Omega, n, l, ldo, B.Rcat + pc * l, ldc, nullptr, st));
  ++pc;
  // dA = Lcat Rcat^T (one product, K = (2q + 2) l)
  CK(transpose(B.Rcat, n, ldc, ldc, B.RcatT, n, st));
  CK(gemm_f64(false, RQLP_F64, B.Lcat, ldc, B.RcatT, n, dA, ldda, m, n, ldc, 1.0, 0.0, nullptr,
              nullptr, nullptr, st));
  return RQLP_OK;
}

}  // namespace

extern "C" {

size_t rqlp_backward_workspace_size(int64_t m, int64_t n, int32_t k, int32_t p,
                                    const rqlp_opts *opts) {
  if (!valid_dims(m, n, k, p) || !valid_opts(opts)) return 0;
  if (!opts->pivot2 || opts->block_b != 0 || opts->truncate_k) return 0;
  rqlp_opts o = *opts;
  o.fixed_pivots = 0;
  return carve_bwd(nullptr, m, n, k + p, o).bytes + 256;
}

int rqlp_backward(const void *A, int32_t a_dtype, int64_t m, int64_t n, int64_t lda, int32_t k,
                  int32_t p, const double *Omega, int64_t ldo, const rqlp_opts *opts,
                  const int32_t *piv0, const int32_t *piv1, const double *dQ, const double *dL,
                  const double *dP, double *dA, int64_t ldda, void *ws, size_t ws_bytes,
                  rqlp_stream_t stream) {
  if (!valid_dims(m, n, k, p) || !valid_opts(opts)) return RQLP_ERR_INVALID_ARG;
  if (!A || !Omega || !dA || !ws || lda < n || ldo < k + p || ldda < n) return RQLP_ERR_INVALID_ARG;
  if (a_dtype != RQLP_F64 && a_dtype != RQLP_F32) return RQLP_ERR_INVALID_ARG;
  if (!opts->pivot2 || opts->block_b != 0 || opts->truncate_k) return RQLP_ERR_UNSUPPORTED;
  if ((piv0 == nullptr) != (piv1 == nullptr)) return RQLP_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return RQLP_ERR_WORKSPACE;
  rqlp_opts o = *opts;
  o.fixed_pivots = 0;  // the pivot arrays themselves say whether they are given
  return run_backward(A, a_dtype, m, n, lda, k + p, Omega, ldo, o, piv0, piv1, dQ, dL, dP, dA,
                      ldda, ws, ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
