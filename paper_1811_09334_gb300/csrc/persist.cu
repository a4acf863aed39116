// Batched randomized QLP in one persistent kernel launch.
//
// Every problem of a batch runs the pipeline of rqlp() (Algorithm 2.1 /
// Algorithm 2.2 with q power steps: the sketch Y = A Omega, one CholeskyQR
// pass per power step, CholeskyQR2 of the final basis V, the projection
// B^T = A^T V, the column-pivoted QR of B, the QR of R0^T, the l x l QRs of
// the inner steps and the assembly Q = V Q_B, P = Pi0 ...).  Each step is a
// stage, and each stage is cut into tiles (row blocks of the tall matrices,
// one item for the l x l and pivoting work); a tile is one work item for one
// CTA.  The host lists every item of every problem once, in the order a
// simulated list schedule takes them (ready items by longest remaining
// critical path of their problem, 1 CTA per SM), so that every item comes
// after all items it depends on.  One kernel with one CTA per SM takes the
// items in that order from an atomic counter.  Before an item runs, its CTA
// waits until every tile of the problem's previous stage has finished: a
// per-problem, per-stage counter that finished tiles increment (release at
// GPU scope) and the waiting CTA reads (acquire).  The wait is bounded by
// spin_limit_ns and records RQLP_ERR_TIMEOUT.  Items are taken in a
// topological order and a CTA only ever waits for items that running CTAs
// took before, so the kernel always makes progress.  The CPQR of B of a
// problem whose columns do not fit in one CTA's shared memory is a gang of
// up to 16 items that run together as the multi-CTA pivoting kernel of
// cpqr.cu (one exchange per pivot step); the schedule hands a gang's items
// out one after another, and the launch is cooperative, so every CTA is
// resident and a gang always completes.
//
// Tiles write their results with ordinary stores and the products read the
// BF16 copies through TMA (the async proxy), so every writer fences the
// async proxy before it signals and every TMA issuer after it has waited.
// Stage kernels here are the same algorithms as the single-problem kernels
// (the CPQR pivot loop and the one-CTA Cholesky are shared code); the l x l
// QRs of the inner steps are unpivoted Householder QRs (the CPQR loop with
// the identity as given pivots), which give the same factors as the
// CholeskyQR2 of rqlp() up to rounding.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <queue>
#include <vector>

#include "chol_body.cuh"
#include "cpqr_body.cuh"
#include "persist.cuh"
#include "tc.cuh"

namespace rqk {

PFN_cuTensorMapEncodeTiled_v12000 tma_encode_fn();

namespace {

using namespace tc;

constexpr int kPT = 256;             // threads per CTA
constexpr int kPMaxL = 128;          // widest sketch of the persistent engine
constexpr int kPMaxRing = 4;         // TMA ring stages of the products
constexpr size_t kPSmem = 200 * 1024;  // dynamic shared memory per CTA (after 1 KB alignment)
constexpr int kPrepRows = 128, kPrepCols = 512;  // precision-preparation tile of A
constexpr int kSplitRows = 256;      // rows of Omega per split tile
constexpr int kTcRows = 128;         // rows of a tensor-core product tile
constexpr int kF64Rows = 64;         // rows of an FP64 product tile
constexpr int kGramRows = 128;       // rows per Gram tile
constexpr int kApplyRowsP = 64;      // rows per solve tile
constexpr int kAsmRows = 64;         // rows per assembly tile

enum StageKind : int {
  PK_PREP = 1,   // BF16 pairs of A and A^T
  PK_SPLIT_OM,   // BF16 pair of Omega^T
  PK_PROD,       // a product with A
  PK_GRAM,       // Gram partial of a row tile
  PK_CHOL,       // Cholesky of the summed Gram matrix
  PK_APPLY,      // X R^-1 of a row tile
  PK_CPQR,       // column-pivoted QR of B and the explicit Q0
  PK_TAIL,       // the l x l part of the QLP (second QR, inner QRs)
  PK_ASM,        // Q = V Q_B and the rows of P
  PK_DONE        // the problem's status
};
constexpr int kPKinds = 16;  // stage kinds (index of the per-kind statistics)
enum BufId : int { PB_OM = -1, PB_Y = 0, PB_V, PB_Z, PB_W, PB_R0T, PB_X, PB_COUNT };

struct PStage {
  int kind;
  int cond;      // 0 always; 1 when again_flag[site] is set; 2 when shift_flag[site] is set
  int site;      // CholeskyQR site of the pass
  int lowp;      // FP32 CholeskyQR pass
  int src, dst;  // buffers (PROD: src is the skinny operand, PB_OM for Omega)
  int rows_n;    // the pass or product runs over n rows (else m)
  int aux;       // PROD: 0 = A S, 1 = A^T S; CHOL: 0 no R kept, 1 Racc = R, 2 Racc = R Racc;
                 // APPLY: 0 no BF16 copy, 1 BF16 copy over m (Sm), 2 over n (Sn)
  double again_tol;
};

struct PProb {
  const void *A;
  int a_dtype, l;
  int64_t m, n, lda;
  const double *Om;
  int64_t ldo;
  double *Q, *L, *P, *Lv;
  int32_t *piv0, *piv1;
  double *buf[PB_COUNT];  // m x l or n x l, ld l
  double *gpart;          // Gram partials [tiles][l][l]
  double *G, *Rp, *Dinv, *Racc, *Rtmp, *Q0, *QB, *Qi, *Macc, *T0, *T1, *Vh, *tau;
  int32_t *pscr;          // l pivots of the unpivoted QRs
  ulonglong2 *rec;        // the CPQR loop's record words (one CTA)
  unsigned char *cpx;     // a gang's exchange state (zeroed before every launch)
  Ctrl *ctrl;
  int32_t *status_out;
  int done0;              // first stage counter of this problem
  int lpad;               // l rounded up to 16 (MMA N)
  __nv_bfloat16 *Ah, *Al, *Ath, *Atl, *Snh, *Snl, *Smh, *Sml;
  int64_t ldn8, ldm8;     // leading dimensions of the BF16 arrays over n and over m
  const CUtensorMap *maps;  // Ah, Al, Ath, Atl, Snh, Snl, Smh, Sml
};

struct PPlan {
  const PProb *probs;
  const PStage *stages;
  const int4 *items;  // (problem, stage, tile, 0)
  unsigned *next;
  int *done;
  int *abort;
  const int32_t *iota;
  unsigned long long *stats;  // [3][kPKinds]: busy ns, waiting ns, items per stage kind
  int nstages, nitems, tc, pivot2, d, ring;
  unsigned long long limit_ns;
};

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// CTAs of the CPQR of B (n columns of length l): as many as it takes for
// every CTA's columns (l doubles each, plus 32 bytes of per-column state) to
// sit in shared memory, at most kPGang; one when they fit in one CTA.
constexpr int kPGang = 16;
__host__ __device__ inline int cpqr_gang(int64_t n, int l) {
  const int64_t sv = ((l + 1) & ~1) * 8;
  const int64_t per = (int64_t)l * 8 + 32;
  const int64_t cap = ((int64_t)kPSmem - sv) / per;  // columns per CTA in shared memory
  const int64_t g = cdiv(n, cap > 0 ? cap : 1);
  return (int)(g < 1 ? 1 : (g > kPGang ? kPGang : g));
}

__host__ __device__ inline int64_t stage_rows(const PProb &p, const PStage &s) {
  return s.rows_n ? p.n : p.m;
}

// tiles of a stage of a problem (host and device agree)
__host__ __device__ inline int tiles_of(const PProb &p, const PStage &s, int tc) {
  switch (s.kind) {
    case PK_PREP: return (int)(cdiv(p.m, kPrepRows) * cdiv(p.n, kPrepCols));
    case PK_SPLIT_OM: return (int)cdiv(p.n, kSplitRows);
    case PK_PROD: {
      const int64_t M = s.aux ? p.n : p.m;
      return (int)cdiv(M, tc ? kTcRows : kF64Rows);
    }
    case PK_GRAM: return (int)cdiv(stage_rows(p, s), kGramRows);
    case PK_APPLY: return (int)cdiv(stage_rows(p, s), kApplyRowsP);
    case PK_ASM: return (int)(cdiv(p.m, kAsmRows) + cdiv(p.n, kAsmRows));
    case PK_CPQR: return cpqr_gang(p.n, p.l);
    default: return 1;
  }
}

__device__ __forceinline__ int ld_acquire_i32(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// generic-proxy stores of this thread before async-proxy (TMA) reads
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.global;" ::: "memory");
}
// generic-proxy accesses of shared memory (earlier items) before TMA writes
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// FP64 (or FP32) element of A as FP32, then its BF16 pair: h = bf16(f),
// l = bf16(f - h) (f - h is exact in FP32)
template <typename T>
__device__ __forceinline__ float to_f32(T x) { return as_f32(x); }
__device__ __forceinline__ void bf16_pair(float f, __nv_bfloat16 &h, __nv_bfloat16 &lo) {
  h = __float2bfloat16_rn(f);
  lo = __float2bfloat16_rn(f - __bfloat162float(h));
}

// ---------------------------------------------------------------------------
// Precision preparation (BF16x3 form): a 128 x 512 block of A into the BF16
// pairs Ah, Al (row-major, ld ldn8) and A^T pairs Ath, Atl (ld ldm8).  The
// block is copied into shared memory with cp.async as 16 pieces of 32 x 128
// through a ring of 4 buffers (three pieces in flight while one is split: a
// single CTA per SM needs that many bytes in flight), then split: lanes take
// two neighbouring columns (BF16 pairs stored as 4-byte words), and the
// transposed halves go through shared memory.
constexpr int kTP = kPrepRows + 2;  // transposed rows of 130 BF16: 65 words, odd
constexpr int kPieceRows = 32, kPrepRing = 4;

__device__ __forceinline__ void cp_async_n(void *smem, const void *gmem, int bytes, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int sz = valid ? bytes : 0;
  if (bytes == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(sa), "l"(gmem), "r"(sz)
                 : "memory");
  else if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(sa), "l"(gmem), "r"(sz)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(sa), "l"(gmem), "r"(sz)
                 : "memory");
}

// one 32 x 128 piece (rows pr0.., columns pc0..) into shared memory, zero
// outside A, as one commit group
template <typename T>
__device__ __forceinline__ void prep_load(const PProb &p, const T *A, int64_t pr0, int nr,
                                          int64_t pc0, int nc, bool v16, T *as) {
  constexpr int VE = 16 / (int)sizeof(T);  // elements per 16-byte copy
  if (v16) {
    for (int e = threadIdx.x; e < kPieceRows * (128 / VE); e += kPT) {
      const int r = e / (128 / VE), c = (e - r * (128 / VE)) * VE;
      const bool ok = r < nr && c < nc;
      const T *src = ok ? A + (pr0 + r) * p.lda + pc0 + c : A;
      if (ok && c + VE > nc) {
        for (int j = 0; j < VE; ++j)
          cp_async_n(as + r * 128 + c + j, c + j < nc ? src + j : A, (int)sizeof(T), c + j < nc);
      } else {
        cp_async_n(as + r * 128 + c, src, 16, ok);
      }
    }
  } else {
    for (int e = threadIdx.x; e < kPieceRows * 128; e += kPT) {
      const int r = e >> 7, c = e & 127;
      const bool ok = r < nr && c < nc;
      cp_async_n(as + e, ok ? A + (pr0 + r) * p.lda + pc0 + c : A, (int)sizeof(T), ok);
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <typename T>
__device__ void prep_tile(const PProb &p, int tile, uint8_t *sm) {
  const int nbj = (int)cdiv(p.n, kPrepCols);
  const int64_t r0 = (int64_t)(tile / nbj) * kPrepRows, cb = (int64_t)(tile % nbj) * kPrepCols;
  const T *A = static_cast<const T *>(p.A);
  T *ring = reinterpret_cast<T *>(sm);  // [kPrepRing][32][128]
  __nv_bfloat16 *th =
      reinterpret_cast<__nv_bfloat16 *>(sm + kPrepRing * kPieceRows * 128 * sizeof(T));
  __nv_bfloat16 *tl = th + 128 * kTP;  // th, tl: [128 columns][kTP], 128 rows
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nrb = (int)min((int64_t)kPrepRows, p.m - r0);
  const int64_t cend = min(cb + kPrepCols, p.n);
  const int ncp = (int)cdiv(cend - cb, 128);  // 128-column blocks
  const bool v16 = ((reinterpret_cast<uintptr_t>(A) & 15) == 0) &&
                   (((int64_t)p.lda * (int64_t)sizeof(T)) % 16 == 0);
  constexpr int kQ = kPrepRows / kPieceRows;  // row pieces per column block
  const int npc = kQ * ncp;
  auto piece = [&](int k, int64_t &pr0, int &nr, int64_t &pc0, int &nc) {
    const int cblk = k / kQ, q = k - cblk * kQ;
    pc0 = cb + 128 * cblk;
    nc = (int)min((int64_t)128, p.n - pc0);
    pr0 = r0 + kPieceRows * q;
    nr = (int)max((int64_t)0, min((int64_t)kPieceRows, p.m - pr0));
  };
  for (int k = 0; k < kPrepRing - 1; ++k) {
    if (k < npc) {
      int64_t pr0, pc0;
      int nr, nc;
      piece(k, pr0, nr, pc0, nc);
      prep_load(p, A, pr0, nr, pc0, nc, v16, ring + (size_t)k * kPieceRows * 128);
    } else {
      asm volatile("cp.async.commit_group;" ::: "memory");  // keep the group count
    }
  }
  for (int k = 0; k < npc; ++k) {
    const int kn = k + kPrepRing - 1;
    if (kn < npc) {
      int64_t qr0, qc0;
      int qnr, qnc;
      piece(kn, qr0, qnr, qc0, qnc);
      prep_load(p, A, qr0, qnr, qc0, qnc, v16,
                ring + (size_t)(kn % kPrepRing) * kPieceRows * 128);
    } else {
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    asm volatile("cp.async.wait_group 3;" ::: "memory");  // piece k has landed
    __syncthreads();
    int64_t pr0, pc0;
    int nr, nc;
    piece(k, pr0, nr, pc0, nc);
    const T *a = ring + (size_t)(k % kPrepRing) * kPieceRows * 128;
    const int rofs = kPieceRows * (k % kQ);  // rows of this piece within the transposed tile
    for (int r = warp; r < nr; r += 8) {
      const int64_t i = pr0 + r;
#pragma unroll
      for (int hq = 0; hq < 2; ++hq) {
        const int c = 2 * lane + 64 * hq;
        __nv_bfloat16 h0, l0, h1, l1;
        bf16_pair(to_f32(a[r * 128 + c]), h0, l0);
        bf16_pair(to_f32(a[r * 128 + c + 1]), h1, l1);
        if (c + 1 < nc) {
          *reinterpret_cast<__nv_bfloat162 *>(p.Ah + i * p.ldn8 + pc0 + c) =
              __halves2bfloat162(h0, h1);
          *reinterpret_cast<__nv_bfloat162 *>(p.Al + i * p.ldn8 + pc0 + c) =
              __halves2bfloat162(l0, l1);
        } else if (c < nc) {
          p.Ah[i * p.ldn8 + pc0 + c] = h0;
          p.Al[i * p.ldn8 + pc0 + c] = l0;
        }
        th[c * kTP + rofs + r] = h0;
        tl[c * kTP + rofs + r] = l0;
        th[(c + 1) * kTP + rofs + r] = h1;
        tl[(c + 1) * kTP + rofs + r] = l1;
      }
    }
    __syncthreads();
    if (k % kQ == kQ - 1) {
      // every row piece of this column block is in th / tl: write A^T
      for (int j = warp; j < nc; j += 8) {
        __nv_bfloat16 *dh = p.Ath + (pc0 + j) * p.ldm8 + r0;
        __nv_bfloat16 *dl = p.Atl + (pc0 + j) * p.ldm8 + r0;
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          const int ii = 2 * lane + 64 * hf;
          if (ii + 1 < nrb) {
            *reinterpret_cast<__nv_bfloat162 *>(dh + ii) =
                __halves2bfloat162(th[j * kTP + ii], th[j * kTP + ii + 1]);
            *reinterpret_cast<__nv_bfloat162 *>(dl + ii) =
                __halves2bfloat162(tl[j * kTP + ii], tl[j * kTP + ii + 1]);
          } else if (ii < nrb) {
            dh[ii] = th[j * kTP + ii];
            dl[ii] = tl[j * kTP + ii];
          }
        }
      }
      __syncthreads();
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  fence_proxy_async();
}

// Rows [r0, r0 + nr) (nr <= 256) of a skinny FP64 S (ld lds, l <= 128
// columns) into the BF16 pair of S^T: Sh[c][r0 + r], Sl[c][r0 + r] (ld ldk).
constexpr int kTS = kSplitRows + 2;  // 129 words, odd
__device__ void split_panel_t(const double *S, int64_t lds, int64_t r0, int nr, int l,
                              __nv_bfloat16 *Sh, __nv_bfloat16 *Sl, int64_t ldk, uint8_t *sm) {
  __nv_bfloat16 *th = reinterpret_cast<__nv_bfloat16 *>(sm);  // [l][kTS]
  __nv_bfloat16 *tl = th + kPMaxL * kTS;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int r = warp; r < nr; r += 8)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = lane + 32 * q;
      if (c < l) {
        __nv_bfloat16 h, lo;
        bf16_pair(d2f_rn(S[(r0 + r) * lds + c]), h, lo);
        th[c * kTS + r] = h;
        tl[c * kTS + r] = lo;
      }
    }
  __syncthreads();
  for (int c = warp; c < l; c += 8) {
    __nv_bfloat16 *dh = Sh + (int64_t)c * ldk + r0, *dl = Sl + (int64_t)c * ldk + r0;
    for (int ii = 2 * lane; ii < nr; ii += 64) {
      if (ii + 1 < nr) {
        *reinterpret_cast<__nv_bfloat162 *>(dh + ii) =
            __halves2bfloat162(th[c * kTS + ii], th[c * kTS + ii + 1]);
        *reinterpret_cast<__nv_bfloat162 *>(dl + ii) =
            __halves2bfloat162(tl[c * kTS + ii], tl[c * kTS + ii + 1]);
      } else {
        dh[ii] = th[c * kTS + ii];
        dl[ii] = tl[c * kTS + ii];
      }
    }
  }
  __syncthreads();
  fence_proxy_async();
}

// ---------------------------------------------------------------------------
// A product tile on the tensor cores (BF16x3): 128 rows of C = X Y^T with
// X = A (C = A S, K = n) or A^T (C = A^T S, K = m) and Y the BF16 pair of
// S^T, over the whole K: warp 0 lane 0 streams 128B-swizzled K blocks of 64
// through a ring of shared-memory stages with TMA, warp 1 lane 0 issues the
// three products Xh Yh + Xh Yl + Xl Yh per block into one FP32 accumulator
// in tensor memory, and all eight warps read it back (warps w and w + 4
// share TMEM lanes 32 (w mod 4) .. +31 and split the columns) and store C in
// FP64.  The ring's stage and phase run on across the CTA's items.
struct TcCtx {
  uint64_t *full, *empty, *acc;
  uint32_t tmem;
  int *s_abort;
};

__device__ void prod_tc(const PPlan &P, const PProb &p, const PStage &s, int tile, uint8_t *sm,
                        const TcCtx &c, uint32_t &ring, uint32_t &accph) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool tr = s.aux == 1;
  const int64_t M = tr ? p.n : p.m, K = tr ? p.m : p.n;
  const CUtensorMap *mx = p.maps + (tr ? 2 : 0);
  const CUtensorMap *my = p.maps + (tr ? 6 : 4);
  const int npad = p.lpad;
  const uint32_t xbytes = kTcRows * 128, ybytes = (uint32_t)npad * 128;
  const uint32_t sbytes = 2 * (xbytes + ybytes);
  const int nk = (int)cdiv(K, 64);
  const int row0 = tile * kTcRows;
  const int stages = P.ring;
  if (warp == 0) {
    if (lane == 0) {
      fence_proxy_async();       // the BF16 copies other CTAs wrote, before the TMA reads them
      fence_proxy_async_smem();  // earlier items' use of the stage buffers, before TMA writes
      int issued = 0;
      for (int i = 0; i < nk; ++i) {
        const uint32_t g = ring + (uint32_t)i;
        const int st = (int)(g % (uint32_t)stages);
        const uint32_t ph = (g / (uint32_t)stages) & 1u;
        if (!mbar_wait(&c.empty[st], ph ^ 1u, P.limit_ns) || *(volatile int *)c.s_abort) {
          *c.s_abort = 1;
          break;
        }
        const uint32_t base = smem_u32(sm + (size_t)st * sbytes);
        mbar_expect_tx(&c.full[st], sbytes);
        const int kx = i * 64;
        tma_load_2d(base, mx, kx, row0, &c.full[st]);
        tma_load_2d(base + xbytes, my, kx, 0, &c.full[st]);
        tma_load_2d(base + xbytes + ybytes, mx + 1, kx, row0, &c.full[st]);
        tma_load_2d(base + 2 * xbytes + ybytes, my + 1, kx, 0, &c.full[st]);
        issued = i + 1;
      }
      if (*(volatile int *)c.s_abort) {
        // never leave copies in flight: wait for the last load of each stage
        for (int st = 0; st < stages && st < issued; ++st) {
          const int last = ((issued - 1 - st) / stages) * stages + st;
          const uint32_t g = ring + (uint32_t)last;
          mbar_wait(&c.full[g % (uint32_t)stages], (g / (uint32_t)stages) & 1u, P.limit_ns);
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = instr_desc(kTcRows, npad);
      for (int i = 0; i < nk; ++i) {
        const uint32_t g = ring + (uint32_t)i;
        const int st = (int)(g % (uint32_t)stages);
        const uint32_t ph = (g / (uint32_t)stages) & 1u;
        if (!mbar_wait(&c.full[st], ph, P.limit_ns) || *(volatile int *)c.s_abort) {
          *c.s_abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t xh = smem_u32(sm + (size_t)st * sbytes);
        const uint32_t yh = xh + xbytes, xl = yh + ybytes, yl = xl + xbytes;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t off = (uint32_t)k * 32u;
          mma_bf16(c.tmem, smem_desc(xh + off), smem_desc(yh + off), idesc,
                   (i == 0 && k == 0) ? 0u : 1u);
          mma_bf16(c.tmem, smem_desc(xh + off), smem_desc(yl + off), idesc, 1u);
          mma_bf16(c.tmem, smem_desc(xl + off), smem_desc(yh + off), idesc, 1u);
        }
        mma_commit(&c.empty[st]);
      }
      // arrives once every MMA issued above has completed (also after an abort)
      mma_commit(c.acc);
    }
    __syncwarp();
  }
  const bool ready = mbar_wait(c.acc, accph, P.limit_ns);
  tc_fence_after();
  __syncthreads();
  if (!ready || *(volatile int *)c.s_abort) {
    if (tid == 0) {
      *c.s_abort = 1;
      set_status(p.ctrl, RQLP_ERR_TIMEOUT);
      atomicExch(P.abort, 1);
    }
  } else {
    const int q = warp & 3, half = warp >> 2;
    const int64_t row = row0 + 32 * q + lane;
    double *out = p.buf[s.dst] + row * p.l;
    const int cend = min(npad, half * 64 + 64);
    for (int c0 = half * 64; c0 < cend; c0 += 32) {
      uint32_t r[32];
      tmem_ld32_nowait(c.tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, r);
      tmem_ld_wait();
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 32; ++j)
          if (c0 + j < p.l) out[c0 + j] = f2d(__uint_as_float(r[j]));
      }
    }
  }
  ring += (uint32_t)nk;
  accph ^= 1u;
  tc_fence_before();
}

// ---------------------------------------------------------------------------
// A product tile on the FP64 units (FP64 form): 64 rows of C = A S (K = n)
// or A^T S (K = m), S FP64 (n x l or m x l), K in chunks of 32 through shared
// memory; thread (ty, tx) of 16 x 16 keeps rows ty + 16 a (a < 4) and columns
// tx + 16 b (b < NB = l16 / 16) in registers.
template <int NB>
__device__ __forceinline__ void f64_chunk(const double *Xs, const double *Ss, int kc, int lp16,
                                          int tx, int ty, double (&acc)[4][8]) {
  for (int k = 0; k < kc; ++k) {
    double x[4], y[NB];
#pragma unroll
    for (int a = 0; a < 4; ++a) x[a] = Xs[(ty + 16 * a) * 33 + k];
#pragma unroll
    for (int b = 0; b < NB; ++b) y[b] = Ss[k * lp16 + tx + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < NB; ++b) acc[a][b] = fma(x[a], y[b], acc[a][b]);
  }
}

template <typename T>
__device__ void prod_f64(const PProb &p, const PStage &s, int tile, uint8_t *sm) {
  const bool tr = s.aux == 1;
  const int64_t M = tr ? p.n : p.m, K = tr ? p.m : p.n;
  const T *A = static_cast<const T *>(p.A);
  const double *S = s.src == PB_OM ? p.Om : p.buf[s.src];
  const int64_t lds = s.src == PB_OM ? p.ldo : p.l;
  const int l = p.l, lp16 = (l + 15) / 16 * 16, NB = lp16 / 16;
  double *Xs = reinterpret_cast<double *>(sm);  // [64][33]
  double *Ss = Xs + 64 * 33;                    // [32][lp16]
  const int64_t r0 = (int64_t)tile * kF64Rows;
  const int nr = (int)min((int64_t)kF64Rows, M - r0);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.0;
  for (int64_t k0 = 0; k0 < K; k0 += 32) {
    const int kc = (int)min((int64_t)32, K - k0);
    if (!tr) {
      for (int e = tid; e < 64 * 32; e += kPT) {
        const int i = e >> 5, k = e & 31;
        Xs[i * 33 + k] = (i < nr && k < kc) ? (double)A[(r0 + i) * p.lda + k0 + k] : 0.0;
      }
    } else {
      for (int e = tid; e < 64 * 32; e += kPT) {
        const int k = e >> 6, i = e & 63;
        Xs[i * 33 + k] = (i < nr && k < kc) ? (double)A[(k0 + k) * p.lda + r0 + i] : 0.0;
      }
    }
    for (int e = tid; e < 32 * lp16; e += kPT) {
      const int k = e / lp16, cc = e - k * lp16;
      Ss[e] = (k < kc && cc < l) ? S[(k0 + k) * lds + cc] : 0.0;
    }
    __syncthreads();
    switch (NB) {
      case 1: f64_chunk<1>(Xs, Ss, kc, lp16, tx, ty, acc); break;
      case 2: f64_chunk<2>(Xs, Ss, kc, lp16, tx, ty, acc); break;
      case 3: f64_chunk<3>(Xs, Ss, kc, lp16, tx, ty, acc); break;
      case 4: f64_chunk<4>(Xs, Ss, kc, lp16, tx, ty, acc); break;
      case 5: f64_chunk<5>(Xs, Ss, kc, lp16, tx, ty, acc); break;
      case 6: f64_chunk<6>(Xs, Ss, kc, lp16, tx, ty, acc); break;
      case 7: f64_chunk<7>(Xs, Ss, kc, lp16, tx, ty, acc); break;
      default: f64_chunk<8>(Xs, Ss, kc, lp16, tx, ty, acc); break;
    }
    __syncthreads();
  }
  double *out = p.buf[s.dst];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int i = ty + 16 * a, cc = tx + 16 * b;
      if (i < nr && cc < l) out[(r0 + i) * l + cc] = acc[a][b];
    }
}

// ---------------------------------------------------------------------------
// CholeskyQR pass pieces (the algorithms of cholqr.cu on one CTA each).
//
// Gram tile: the upper triangle of X_t^T X_t for 128 rows, in 4 x 4 register
// tiles of the triangle, the rows staged 32 at a time.  When the triangle has
// at most 128 tiles (l <= 60) the rows of each chunk are dealt to G = 256 /
// tiles groups of threads (every thread busy) and the groups' sums are added
// in a fixed order at the end; otherwise each thread takes up to 3 tiles.
// T = float: each 32-row chunk is rounded to FP32 and summed in FP32, the
// chunks in FP64 (as the FP32 pass of cholqr.cu).
template <typename T>
__device__ void gram_tile(const PProb &p, const PStage &s, int tile, uint8_t *sm) {
  const double *X = p.buf[s.src];
  const int l = p.l;
  const int64_t rows = stage_rows(p, s), r0 = (int64_t)tile * kGramRows;
  const int nr = (int)min((int64_t)kGramRows, rows - r0);
  const int lp = ((l + 3) / 4) * 4 + 1;
  T *xs = reinterpret_cast<T *>(sm);                            // [32][lp]
  double *red = reinterpret_cast<double *>(sm + 32 * 129 * 8);  // [G][tiles][16]
  const int nb = (l + 3) / 4, ntiles = nb * (nb + 1) / 2;
  const int G = (2 * ntiles <= kPT) ? min(8, kPT / ntiles) : 1;
  const int tid = threadIdx.x;
  const int g = G > 1 ? tid / ntiles : 0;
  int bi[3], bj[3];
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    int t = G > 1 ? ((u == 0 && g < G) ? tid % ntiles : -1) : tid + kPT * u, b = 0;
    if (t >= ntiles) t = -1;
    if (t >= 0) {
      while (t >= nb - b) {
        t -= nb - b;
        ++b;
      }
      bi[u] = b;
      bj[u] = b + t;
    } else {
      bi[u] = bj[u] = -1;
    }
  }
  double accd[3][4][4];
#pragma unroll
  for (int u = 0; u < 3; ++u)
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) accd[u][a][b] = 0.0;
  for (int c0 = 0; c0 < nr; c0 += 32) {
    const int cr = min(32, nr - c0);
    __syncthreads();
    for (int e = tid; e < 32 * lp; e += kPT) {
      const int r = e / lp, cc = e - r * lp;
      xs[e] = (r < cr && cc < l) ? from_f64<T>(X[(r0 + c0 + r) * l + cc]) : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      if (bi[u] < 0) continue;
      T acc[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
      for (int r = g; r < cr; r += G) {
        const T *row = xs + r * lp;
        T x[4], y[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) x[a] = row[4 * bi[u] + a];
#pragma unroll
        for (int b = 0; b < 4; ++b) y[b] = row[4 * bj[u] + b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fma(x[a], y[b], acc[a][b]);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) accd[u][a][b] += to_f64(acc[a][b]);
    }
  }
  if (G > 1) {
    // the row groups' partial sums, added in group order
    if (bi[0] >= 0) {
      double *my = red + ((size_t)g * ntiles + tid % ntiles) * 16;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) my[a * 4 + b] = accd[0][a][b];
    }
    __syncthreads();
    if (g == 0 && bi[0] >= 0) {
      for (int h = 1; h < G; ++h) {
        const double *o = red + ((size_t)h * ntiles + tid) * 16;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) accd[0][a][b] += o[a * 4 + b];
      }
    }
    if (g != 0) bi[0] = -1;
  }
  double *out = p.gpart + (int64_t)tile * l * l;
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    if (bi[u] < 0) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = 4 * bi[u] + a;
      if (i >= l) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int j = 4 * bj[u] + b;
        if (j < l && j >= i) out[(int64_t)i * l + j] = accd[u][a][b];
      }
    }
  }
}

// C = A B for l x l matrices in global memory (ld l), one CTA; with
// upper = true both are upper triangular and so is C
__device__ void small_gemm(const double *A, const double *B, double *C, int l, bool upper) {
  for (int e = threadIdx.x; e < l * l; e += kPT) {
    const int i = e / l, j = e - i * l;
    double s0 = 0.0, s1 = 0.0;
    if (!upper || j >= i) {
      const int t0 = upper ? i : 0, t1 = upper ? j + 1 : l;
      int t = t0;
      for (; t + 1 < t1; t += 2) {
        s0 = fma(A[i * l + t], B[t * l + j], s0);
        s1 = fma(A[i * l + t + 1], B[(t + 1) * l + j], s1);
      }
      if (t < t1) s0 = fma(A[i * l + t], B[t * l + j], s0);
    }
    C[e] = s0 + s1;
  }
}

// Sum of the Gram partials (fixed order), the Cholesky (FP64, or FP32 for a
// power step's pass) with its breakdown test, shifted retry and the
// again/shift flags of the site, and the accumulated R of a pass sequence.
__device__ void chol_item(const PProb &p, const PStage &s, uint8_t *sm) {
  const int l = p.l;
  const int64_t rows = stage_rows(p, s);
  const int nt = (int)cdiv(rows, kGramRows);
  const int64_t ll = (int64_t)l * l;
  for (int e = threadIdx.x; e < l * l; e += kPT) {
    const int i = e / l, j = e - i * l;
    if (j < i) continue;
    double a0 = 0.0, a1 = 0.0;
    int t = 0;
    for (; t + 1 < nt; t += 2) {
      a0 += p.gpart[(int64_t)t * ll + e];
      a1 += p.gpart[(int64_t)(t + 1) * ll + e];
    }
    if (t < nt) a0 += p.gpart[(int64_t)t * ll + e];
    const double g = a0 + a1;
    p.G[e] = g;
    p.G[(int64_t)j * l + i] = g;
  }
  __syncthreads();
  double *w = reinterpret_cast<double *>(sm);
  if (s.lowp)
    cholk::chol_body<float>(p.G, l, (double)rows, p.Rp, p.Dinv, p.ctrl, s.site, 1, s.again_tol,
                            kEpsF32, w);
  else
    cholk::chol_body<double>(p.G, l, (double)rows, p.Rp, p.Dinv, p.ctrl, s.site, 1, s.again_tol,
                             kEpsF64, w);
  __syncthreads();
  if (s.aux == 1) {
    for (int e = threadIdx.x; e < l * l; e += kPT) p.Racc[e] = p.Rp[e];
  } else if (s.aux == 2) {
    small_gemm(p.Rp, p.Racc, p.Rtmp, l, true);
    __syncthreads();
    for (int e = threadIdx.x; e < l * l; e += kPT) p.Racc[e] = p.Rtmp[e];
  }
}

// Solve tile: 64 rows of Q = X R^{-1} by the blocked triangular solve of
// cholqr.cu (16-column blocks: the block's residual X[:, b] - Q[:, <b] R[<b, b],
// then times inv(R[b, b])); two groups of 128 threads take 32 rows each, lane
// = row, warp = 4 columns of the block.  dst may be src (the tile is staged
// first).  aux: also the BF16 pair of the result, transposed (the next
// product's skinny operand).
template <typename T>
__device__ void apply_tile(const PProb &p, const PStage &s, int tile, uint8_t *sm) {
  const double *X = p.buf[s.src];
  double *Qd = p.buf[s.dst];
  const int l = p.l, lp = l + 1;
  const int64_t rows = stage_rows(p, s), r0 = (int64_t)tile * kApplyRowsP;
  const int nr = (int)min((int64_t)kApplyRowsP, rows - r0);
  T *qs = reinterpret_cast<T *>(sm);  // [64][lp]
  T *rc = qs + kApplyRowsP * lp;      // [l][16]: rows < c0 of R's block column
  T *dv = rc + l * 16;                // [16][16]: inv(R[b, b])
  const int tid = threadIdx.x;
  const int r = (tid & 31) + 32 * (tid >> 7), j0 = ((tid >> 5) & 3) * 4;
  for (int e = tid; e < kApplyRowsP * l; e += kPT) {
    const int rr = e / l, c = e - rr * l;
    qs[rr * lp + c] = rr < nr ? from_f64<T>(X[(r0 + rr) * l + c]) : (T)0;
  }
  for (int c0 = 0; c0 < l; c0 += 16) {
    const int bs = min(16, l - c0);
    __syncthreads();
    for (int e = tid; e < c0 * 16; e += kPT) {
      const int t = e >> 4, j = e & 15;
      rc[e] = j < bs ? from_f64<T>(p.Rp[(int64_t)t * l + c0 + j]) : (T)0;
    }
    {
      const int i = tid >> 4, j = tid & 15;
      dv[tid] = (i < bs && j < bs) ? from_f64<T>(p.Dinv[(int64_t)(c0 + i) * l + c0 + j]) : (T)0;
    }
    __syncthreads();
    T acc[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) acc[a] = (j0 + a < bs) ? qs[r * lp + c0 + j0 + a] : (T)0;
    for (int t = 0; t < c0; ++t) {
      const T qv = qs[r * lp + t];
#pragma unroll
      for (int a = 0; a < 4; ++a) acc[a] = fma(-qv, rc[t * 16 + j0 + a], acc[a]);
    }
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
      for (int a = 0; a < 4; ++a) out[a] = fma(v, dv[i * 16 + j0 + a], out[a]);
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a)
      if (j0 + a < bs) qs[r * lp + c0 + j0 + a] = out[a];
  }
  __syncthreads();
  for (int e = tid; e < nr * l; e += kPT) {
    const int rr = e / l, c = e - rr * l;
    Qd[(r0 + rr) * l + c] = to_f64(qs[rr * lp + c]);
  }
  if (s.aux) {
    __nv_bfloat16 *Sh = s.aux == 1 ? p.Smh : p.Snh, *Sl = s.aux == 1 ? p.Sml : p.Snl;
    const int64_t ldk = s.aux == 1 ? p.ldm8 : p.ldn8;
    const int lane = tid & 31, warp = tid >> 5;
    for (int c = warp; c < l; c += 8) {
      const int ii = 2 * lane;
      if (ii >= nr) continue;
      __nv_bfloat16 h0, l0, h1, l1;
      bf16_pair(as_f32(qs[ii * lp + c]), h0, l0);
      if (ii + 1 < nr) {
        bf16_pair(as_f32(qs[(ii + 1) * lp + c]), h1, l1);
        *reinterpret_cast<__nv_bfloat162 *>(Sh + (int64_t)c * ldk + r0 + ii) = __halves2bfloat162(h0, h1);
        *reinterpret_cast<__nv_bfloat162 *>(Sl + (int64_t)c * ldk + r0 + ii) = __halves2bfloat162(l0, l1);
      } else {
        Sh[(int64_t)c * ldk + r0 + ii] = h0;
        Sl[(int64_t)c * ldk + r0 + ii] = l0;
      }
    }
    fence_proxy_async();
  }
}

// ---------------------------------------------------------------------------
// Pivoting and the l x l work.
//
// The CPQR pivot loop of cpqr.cu on one CTA (G = 1: no exchange waits) for
// the n x l matrix Bt (the rows of Bt are the columns of the wide matrix B):
// R0t (n x l), the pivots piv (n; given pivots fpiv for the first l steps,
// or null), the reflectors Vh (l x l) and tau.  The columns are kept in
// shared memory when they fit, else they are updated in place in Bt.
__device__ void cpqr_cta(const PPlan &P, const PProb &p, double *Bt, int64_t n, double *R0t,
                         int32_t *piv, const int32_t *fpiv, uint8_t *sm) {
  const int l = p.l;
  for (int64_t i = threadIdx.x; i < n; i += kPT) piv[i] = (int32_t)i;
  __syncthreads();
  cpqrk::CpqrParams c;
  c.Bt = Bt;
  c.n = n;
  c.l = l;
  c.steps = l;
  c.ldv = l;
  c.ldb = l;
  c.R0t = R0t;
  c.ldr = l;
  c.piv = piv;
  c.Vh = p.Vh;
  c.tau = p.tau;
  c.arrive = reinterpret_cast<unsigned *>(p.rec);
  c.win = p.rec;
  c.rec = p.rec;
  c.pcol = p.rec;
  c.gcols = Bt;
  c.ctrl = p.ctrl;
  c.limit_ns = P.limit_ns;
  c.extra = 0;
  c.cpb = (int)n;
  c.fpiv = fpiv;
  const size_t sv = (size_t)((l + 1) & ~1) * sizeof(double);
  const size_t state = (size_t)n * (3 * sizeof(double) + 2 * sizeof(int));
  const size_t slab = (size_t)n * l * sizeof(double);
  c.use_smem = (sv + slab + state <= kPSmem) ? 1 : 0;
  double *w = reinterpret_cast<double *>(sm);
  if (c.use_smem) cpqrk::cpqr_body<true>(c, 1, 0, w);
  else cpqrk::cpqr_body<false>(c, 1, 0, w);
  __syncthreads();
}

// Q (l x l, ld l) = H_0 H_1 ... H_{l-1} from the reflectors of cpqr_cta
// (v_s = e_s + Vh[s+1:, s], tau_s), in shared memory.  Column j of the
// identity is left alone by H_s for s > j, so each column runs its own steps
// s = j .. 0 independently: a group of 4 lanes per column (the dot product
// over rows >= s, then the axpy).
__device__ void form_q_cta(const double *Vh, const double *tau, int l, double *Qout,
                           uint8_t *sm) {
  double *Qs = reinterpret_cast<double *>(sm);
  for (int e = threadIdx.x; e < l * l; e += kPT) {
    const int i = e / l, j = e - i * l;
    Qs[e] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane & 3, grp = threadIdx.x >> 2;
  const unsigned gmask = 0xfu << (lane & ~3);
  for (int j = grp; j < l; j += kPT / 4) {
    for (int s = j; s >= 0; --s) {
      double w = 0.0;
      for (int r = s + g; r < l; r += 4) {
        const double v = (r == s) ? 1.0 : Vh[(int64_t)r * l + s];
        w = fma(v, Qs[r * l + j], w);
      }
      w += __shfl_xor_sync(gmask, w, 1);
      w += __shfl_xor_sync(gmask, w, 2);
      const double tw = tau[s] * w;
      for (int r = s + g; r < l; r += 4) {
        const double v = (r == s) ? 1.0 : Vh[(int64_t)r * l + s];
        Qs[r * l + j] = fma(-tw, v, Qs[r * l + j]);
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < l * l; e += kPT) Qout[e] = Qs[e];
  __syncthreads();
}

// Member b of the gang of G CTAs that factors B together (the multi-CTA
// exchange of cpqr.cu: one tagged candidate record per CTA and pivot step,
// the last arrival picks the winner); the member's columns stay in its
// shared memory.  Member 0 then forms Q0.
__device__ void cpqr_gang_item(const PPlan &P, const PProb &p, int G, int b, uint8_t *sm) {
  const int l = p.l;
  const int64_t n = p.n;
  const int64_t cpb = cdiv(n, G);
  const int64_t c0 = (int64_t)b * cpb, c1 = min(n, c0 + cpb);
  for (int64_t i = c0 + threadIdx.x; i < c1; i += kPT) p.piv0[i] = (int32_t)i;
  __syncthreads();
  cpqrk::CpqrParams c;
  c.Bt = p.buf[PB_Z];
  c.n = n;
  c.l = l;
  c.steps = l;
  c.ldv = l;
  c.ldb = l;
  c.R0t = p.buf[PB_R0T];
  c.ldr = l;
  c.piv = p.piv0;
  c.Vh = p.Vh;
  c.tau = p.tau;
  // the exchange state, laid out as cpqr.cu lays it out for G CTAs
  c.arrive = reinterpret_cast<unsigned *>(p.cpx);
  c.win = reinterpret_cast<ulonglong2 *>(p.cpx + 128);
  c.rec = reinterpret_cast<ulonglong2 *>(p.cpx + 128 + 128 * (size_t)G);
  c.pcol = c.rec + 2 * (size_t)G * cpqrk::kRecWords;
  c.gcols = p.buf[PB_Z];  // the columns in place when they do not fit (not the case by construction)
  c.ctrl = p.ctrl;
  c.limit_ns = P.limit_ns;
  c.extra = 0;
  c.cpb = (int)cpb;
  c.fpiv = nullptr;
  const size_t sv = (size_t)((l + 1) & ~1) * sizeof(double);
  const size_t need = sv + (size_t)cpb * l * sizeof(double) + (size_t)cpb * (3 * 8 + 2 * 4);
  c.use_smem = need <= kPSmem ? 1 : 0;
  double *w = reinterpret_cast<double *>(sm);
  if (c.use_smem) cpqrk::cpqr_body<true>(c, G, b, w);
  else cpqrk::cpqr_body<false>(c, G, b, w);
  __syncthreads();
  if (b != 0 || ld_volatile_i32(&p.ctrl->status) < 0) return;
  form_q_cta(p.Vh, p.tau, l, p.Q0, sm);
}

__device__ void cpqr_item(const PPlan &P, const PProb &p, int tile, uint8_t *sm) {
  const int G = cpqr_gang(p.n, p.l);
  if (G > 1) {
    cpqr_gang_item(P, p, G, tile, sm);
    return;
  }
  cpqr_cta(P, p, p.buf[PB_Z], p.n, p.buf[PB_R0T], p.piv0, nullptr, sm);
  if (ld_volatile_i32(&p.ctrl->status) < 0) return;
  form_q_cta(p.Vh, p.tau, p.l, p.Q0, sm);
}

__device__ void transpose_ll(const double *X, double *Y, int l) {
  for (int e = threadIdx.x; e < l * l; e += kPT) {
    const int i = e / l, j = e - i * l;
    Y[(int64_t)j * l + i] = X[e];
  }
}

__device__ void copy_ll(const double *X, double *Y, int l) {
  for (int e = threadIdx.x; e < l * l; e += kPT) Y[e] = X[e];
}

// The l x l part of the QLP of B.  RQLP (pivot2): the CPQR of Racc (the R of
// the QR of R0^T) gives L (its R^T), piv1 and Qi; Q_B = Q0[:, piv1].
// ERQLP: the QRs of the inner steps R_{i-1}^T = Q(i) R_i (i = 2..d, unpivoted
// Householder), the even factors into Q_B and the odd ones into Macc, then
// Q_B = Q0 Q_B and L = R_d^T (d odd) or R_d.
__device__ void tail_item(const PPlan &P, const PProb &p, uint8_t *sm) {
  const int l = p.l;
  if (P.pivot2) {
    transpose_ll(p.Racc, p.T0, l);
    __syncthreads();
    cpqr_cta(P, p, p.T0, l, p.L, p.piv1, nullptr, sm);
    if (ld_volatile_i32(&p.ctrl->status) < 0) return;
    form_q_cta(p.Vh, p.tau, l, p.Qi, sm);
    for (int e = threadIdx.x; e < l * l; e += kPT) {
      const int i = e / l, j = e - i * l;
      p.QB[e] = p.Q0[(int64_t)i * l + p.piv1[j]];
    }
  } else {
    copy_ll(p.Racc, p.T0, l);  // R_1
    __syncthreads();
    bool qb_id = true, macc_id = true;
    for (int i = 2; i <= P.d; ++i) {
      // B = R_{i-1}^T: the rows of Bt = R_{i-1} are its columns
      cpqr_cta(P, p, p.T0, l, p.T1, p.pscr, P.iota, sm);
      if (ld_volatile_i32(&p.ctrl->status) < 0) return;
      transpose_ll(p.T1, p.T0, l);  // R_i
      form_q_cta(p.Vh, p.tau, l, p.Qi, sm);
      double *acc = (i % 2 == 0) ? p.QB : p.Macc;
      bool &aid = (i % 2 == 0) ? qb_id : macc_id;
      if (aid) {
        copy_ll(p.Qi, acc, l);
        aid = false;
      } else {
        small_gemm(acc, p.Qi, p.Rtmp, l, false);
        __syncthreads();
        copy_ll(p.Rtmp, acc, l);
      }
      __syncthreads();
    }
    if (qb_id) {
      copy_ll(p.Q0, p.QB, l);
    } else {
      small_gemm(p.Q0, p.QB, p.Rtmp, l, false);
      __syncthreads();
      copy_ll(p.Rtmp, p.QB, l);
    }
    if (P.d % 2 == 1) transpose_ll(p.T0, p.L, l);
    else copy_ll(p.T0, p.L, l);
    for (int i = threadIdx.x; i < l; i += kPT) p.piv1[i] = i;
  }
  __syncthreads();
  if (p.Lv)
    for (int i = threadIdx.x; i < l; i += kPT) p.Lv[i] = p.L[(int64_t)i * l + i];
}

// Assembly tile: 64 rows of out = Xr B (B l x l), row i to row rowmap[i]
// when rowmap is given; B staged in shared memory, X rows too; thread
// (ty, tx) of 16 x 16: rows ty + 16 a, columns tx + 16 b.
template <int NB>
__device__ __forceinline__ void rows_gemm_nb(const double *Xs, const double *Bs, int l, int lp16,
                                             int tx, int ty, double (&acc)[4][8]) {
  for (int t = 0; t < l; ++t) {
    double x[4], y[NB];
#pragma unroll
    for (int a = 0; a < 4; ++a) x[a] = Xs[(ty + 16 * a) * (l + 1) + t];
#pragma unroll
    for (int b = 0; b < NB; ++b) y[b] = Bs[t * lp16 + tx + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < NB; ++b) acc[a][b] = fma(x[a], y[b], acc[a][b]);
  }
}

__device__ void rows_gemm(const double *Xr, int64_t rows, int64_t r0, const double *B, int l,
                          double *out, const int32_t *rowmap, uint8_t *sm) {
  const int lp16 = (l + 15) / 16 * 16, NB = lp16 / 16;
  double *Bs = reinterpret_cast<double *>(sm);  // [l][lp16]
  double *Xs = Bs + (size_t)l * lp16;           // [64][l + 1]
  const int nr = (int)min((int64_t)kAsmRows, rows - r0);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int e = tid; e < l * lp16; e += kPT) {
    const int t = e / lp16, c = e - t * lp16;
    Bs[e] = c < l ? B[(int64_t)t * l + c] : 0.0;
  }
  for (int e = tid; e < kAsmRows * l; e += kPT) {
    const int r = e / l, c = e - r * l;
    Xs[r * (l + 1) + c] = r < nr ? Xr[(r0 + r) * l + c] : 0.0;
  }
  __syncthreads();
  double acc[4][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = 0.0;
  switch (NB) {
    case 1: rows_gemm_nb<1>(Xs, Bs, l, lp16, tx, ty, acc); break;
    case 2: rows_gemm_nb<2>(Xs, Bs, l, lp16, tx, ty, acc); break;
    case 3: rows_gemm_nb<3>(Xs, Bs, l, lp16, tx, ty, acc); break;
    case 4: rows_gemm_nb<4>(Xs, Bs, l, lp16, tx, ty, acc); break;
    case 5: rows_gemm_nb<5>(Xs, Bs, l, lp16, tx, ty, acc); break;
    case 6: rows_gemm_nb<6>(Xs, Bs, l, lp16, tx, ty, acc); break;
    case 7: rows_gemm_nb<7>(Xs, Bs, l, lp16, tx, ty, acc); break;
    default: rows_gemm_nb<8>(Xs, Bs, l, lp16, tx, ty, acc); break;
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = ty + 16 * a;
    if (i >= nr) continue;
    const int64_t orow = rowmap ? (int64_t)rowmap[r0 + i] : r0 + i;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int c = tx + 16 * b;
      if (c < l) out[orow * l + c] = acc[a][b];
    }
  }
}

// Q = V Q_B (tiles 0 .. ceil(m / 64) - 1), then the rows of P: P[piv0[i]] =
// X[i] (ERQLP, d <= 2), X[i] Macc (d > 2) or X[i] Qi (RQLP)
__device__ void asm_tile(const PPlan &P, const PProb &p, int tile, uint8_t *sm) {
  const int l = p.l;
  const int tq = (int)cdiv(p.m, kAsmRows);
  if (tile < tq) {
    rows_gemm(p.buf[PB_V], p.m, (int64_t)tile * kAsmRows, p.QB, l, p.Q, nullptr, sm);
    return;
  }
  const int64_t r0 = (int64_t)(tile - tq) * kAsmRows;
  const double *X = p.buf[PB_X];
  if (P.pivot2) {
    rows_gemm(X, p.n, r0, p.Qi, l, p.P, p.piv0, sm);
  } else if (P.d > 2) {
    rows_gemm(X, p.n, r0, p.Macc, l, p.P, p.piv0, sm);
  } else {
    const int nr = (int)min((int64_t)kAsmRows, p.n - r0);
    for (int e = threadIdx.x; e < nr * l; e += kPT) {
      const int r = e / l, c = e - r * l;
      p.P[(int64_t)p.piv0[r0 + r] * l + c] = X[(r0 + r) * l + c];
    }
  }
}

// ---------------------------------------------------------------------------
// The persistent kernel: one CTA per SM takes items from the ordered list.
__device__ void run_item(const PPlan &P, const PProb &p, const PStage &s, int tile, uint8_t *sm,
                         const TcCtx &tcx, uint32_t &ring, uint32_t &accph) {
  const bool f32a = p.a_dtype == RQLP_F32;
  switch (s.kind) {
    case PK_PREP:
      if (f32a) prep_tile<float>(p, tile, sm);
      else prep_tile<double>(p, tile, sm);
      break;
    case PK_SPLIT_OM: {
      const int64_t r0 = (int64_t)tile * kSplitRows;
      split_panel_t(p.Om, p.ldo, r0, (int)min((int64_t)kSplitRows, p.n - r0), p.l, p.Snh, p.Snl,
                    p.ldn8, sm);
      break;
    }
    case PK_PROD:
      if (P.tc) prod_tc(P, p, s, tile, sm, tcx, ring, accph);
      else if (f32a) prod_f64<float>(p, s, tile, sm);
      else prod_f64<double>(p, s, tile, sm);
      break;
    case PK_GRAM:
      if (s.lowp) gram_tile<float>(p, s, tile, sm);
      else gram_tile<double>(p, s, tile, sm);
      break;
    case PK_CHOL: chol_item(p, s, sm); break;
    case PK_APPLY:
      if (s.lowp) apply_tile<float>(p, s, tile, sm);
      else apply_tile<double>(p, s, tile, sm);
      break;
    case PK_CPQR: cpqr_item(P, p, tile, sm); break;
    case PK_TAIL: tail_item(P, p, sm); break;
    case PK_ASM: asm_tile(P, p, tile, sm); break;
    case PK_DONE:
      if (threadIdx.x == 0) *p.status_out = ld_volatile_i32(&p.ctrl->status);
      break;
    default: break;
  }
}

__global__ void __launch_bounds__(kPT, 1) k_persist(const __grid_constant__ PPlan P) {
  extern __shared__ __align__(1024) uint8_t smraw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smraw) + 1023) & ~static_cast<uintptr_t>(1023));
  __shared__ __align__(8) uint64_t bfull[kPMaxRing], bempty[kPMaxRing], bacc;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort, s_skip;
  __shared__ int4 s_item;
  __shared__ unsigned long long s_stat[3][kPKinds];
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid < 3 * kPKinds) (&s_stat[0][0])[tid] = 0ull;
  if (tid == 0) {
    s_abort = 0;
    if (P.tc) {
      for (int s = 0; s < P.ring; ++s) {
        mbar_init(&bfull[s], 1);
        mbar_init(&bempty[s], 1);
      }
      mbar_init(&bacc, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  if (P.tc && warp == 0) tmem_alloc(&s_tmem, 128);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  TcCtx tcx;
  tcx.full = bfull;
  tcx.empty = bempty;
  tcx.acc = &bacc;
  tcx.tmem = P.tc ? s_tmem : 0u;
  tcx.s_abort = &s_abort;
  uint32_t ring = 0, accph = 0;
  unsigned long long t_ready = 0;
  for (;;) {
    if (tid == 0) {
      const unsigned long long t_ask = globaltimer_ns();
      const unsigned idx = atomicAdd(P.next, 1u);
      int4 it = make_int4(-1, 0, 0, 0);
      int skip = 0;
      if (idx < (unsigned)P.nitems) {
        it = P.items[idx];
        const PProb &pb = P.probs[it.x];
        const PStage &sg = P.stages[it.y];
        const bool fin = sg.kind == PK_DONE;
        // after an error (this problem's, or a tensor pipeline that gave up)
        // the items do nothing and need not wait; the status item still waits
        if (!fin && (ld_volatile_i32(P.abort) != 0 || s_abort ||
                     ld_volatile_i32(&pb.ctrl->status) < 0))
          skip = 1;
        if (it.y > 0 && !skip) {
          // every tile of the previous stage of this problem has finished
          const int need = tiles_of(pb, P.stages[it.y - 1], P.tc);
          const int *ctr = P.done + pb.done0 + it.y - 1;
          if (ld_acquire_i32(ctr) < need) {
            const unsigned long long t0 = globaltimer_ns();
            while (ld_acquire_i32(ctr) < need) {
              if (globaltimer_ns() - t0 > P.limit_ns) {
                set_status(pb.ctrl, RQLP_ERR_TIMEOUT);
                atomicExch(&pb.ctrl->timeout_site, 300 + it.y);
                skip = fin ? 0 : 1;
                break;
              }
              __nanosleep(100);
            }
          }
        }
        if (!skip && !fin) {
          if (sg.cond == 1 && ld_volatile_i32(&pb.ctrl->again_flag[sg.site]) == 0) skip = 1;
          if (sg.cond == 2 && ld_volatile_i32(&pb.ctrl->shift_flag[sg.site]) == 0) skip = 1;
        }
      }
      s_item = it;
      s_skip = skip;
      t_ready = globaltimer_ns();
      if (it.x >= 0) s_stat[1][P.stages[it.y].kind & (kPKinds - 1)] += t_ready - t_ask;
    }
    __syncthreads();
    const int4 it = s_item;
    if (it.x < 0) break;
    if (!s_skip) run_item(P, P.probs[it.x], P.stages[it.y], it.z, sm, tcx, ring, accph);
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      atomicAdd(P.done + P.probs[it.x].done0 + it.y, 1);
      const int kd = P.stages[it.y].kind & (kPKinds - 1);
      s_stat[0][kd] += globaltimer_ns() - t_ready;
      s_stat[2][kd] += s_skip ? 0ull : 1ull;
    }
  }
  __syncthreads();
  if (tid < 3 * kPKinds && (&s_stat[0][0])[tid]) atomicAdd(P.stats + tid, (&s_stat[0][0])[tid]);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (P.tc && warp == 0) tmem_dealloc(s_tmem, 128);
}

// ---------------------------------------------------------------------------
// Host side: the stage list, the workspace, the item order.

constexpr int64_t kPMaxN = 6000;  // the CPQR state of n columns (32 bytes each) in shared memory

bool tc_prec(int prec) { return prec == RQLP_PREC_BF16X3; }

std::vector<PStage> build_stages(const rqlp_opts &o) {
  const bool tc = tc_prec(o.prec);
  std::vector<PStage> v;
  int site = 0;
  auto add = [&](int kind, int cond, int st, int lowp, int src, int dst, int rows_n, int aux,
                 double tol) {
    PStage s;
    s.kind = kind;
    s.cond = cond;
    s.site = st;
    s.lowp = lowp;
    s.src = src;
    s.dst = dst;
    s.rows_n = rows_n;
    s.aux = aux;
    s.again_tol = tol;
    v.push_back(s);
  };
  auto pass = [&](int cond, int st, int lowp, int src, int dst, int rows_n, int split, int racc,
                  double tol) {
    add(PK_GRAM, cond, st, lowp, src, dst, rows_n, 0, tol);
    add(PK_CHOL, cond, st, lowp, src, dst, rows_n, racc, tol);
    add(PK_APPLY, cond, st, lowp, src, dst, rows_n, split, tol);
  };
  // one CholeskyQR pass between power steps: FP32 in the BF16x3 form (the
  // span moves by about FP32 rounding, far below the products' error), FP64
  // followed by the shifted pass when its Cholesky broke down in the FP64 form
  auto power_orth = [&](int src, int dst, int rows_n, int split) {
    const int st = site++;
    if (tc) {
      pass(0, st, 1, src, dst, rows_n, split, 0, -1.0);
    } else {
      pass(0, st, 0, src, dst, rows_n, 0, 0, -1.0);
      pass(2, st, 0, dst, dst, rows_n, 0, 0, -1.0);
    }
  };
  // CholeskyQR2 (the second pass only when the first one asks for it in the
  // BF16x3 form), then the shifted pass when a Cholesky broke down
  auto final_orth = [&](int src, int dst, int rows_n, int split, bool keep_r) {
    const int st = site++;
    pass(0, st, 0, src, dst, rows_n, split, keep_r ? 1 : 0, tc ? 1e-10 : -1.0);
    pass(tc ? 1 : 0, st, 0, dst, dst, rows_n, split, keep_r ? 2 : 0, -1.0);
    pass(2, st, 0, dst, dst, rows_n, split, keep_r ? 2 : 0, -1.0);
  };
  if (tc) {
    add(PK_PREP, 0, 0, 0, 0, 0, 0, 0, 0.0);
    add(PK_SPLIT_OM, 0, 0, 0, 0, 0, 1, 0, 0.0);
  }
  add(PK_PROD, 0, 0, 0, PB_OM, PB_Y, 0, 0, 0.0);  // Y = A Omega
  for (int i = 0; i < o.q; ++i) {
    power_orth(PB_Y, PB_V, 0, 1);
    add(PK_PROD, 0, 0, 0, PB_V, PB_Z, 1, 1, 0.0);  // Z = A^T V
    power_orth(PB_Z, PB_W, 1, 2);
    add(PK_PROD, 0, 0, 0, PB_W, PB_Y, 0, 0, 0.0);  // Y = A W
  }
  final_orth(PB_Y, PB_V, 0, tc ? 1 : 0, false);
  add(PK_PROD, 0, 0, 0, PB_V, PB_Z, 1, 1, 0.0);    // B^T = A^T V
  add(PK_CPQR, 0, 0, 0, 0, 0, 1, 0, 0.0);
  final_orth(PB_R0T, PB_X, 1, 0, true);
  add(PK_TAIL, 0, 0, 0, 0, 0, 0, 0, 0.0);
  add(PK_ASM, 0, 0, 0, 0, 0, 0, 0, 0.0);
  add(PK_DONE, 0, 0, 0, 0, 0, 0, 0, 0.0);
  return v;
}

bool supported(const rqlp_problem *probs, int count, const rqlp_opts *o) {
  if (!probs || count <= 0 || !o) return false;
  if (o->prec != RQLP_PREC_FP64 && o->prec != RQLP_PREC_BF16X3) return false;
  if (o->block_b != 0 || o->fixed_pivots != 0 || o->truncate_k != 0) return false;
  if (o->q < 0 || 2 * o->q + 2 > kShiftSites || o->d < 1 || o->d > 4) return false;
  if (o->pivot2 && o->d != 1) return false;
  for (int i = 0; i < count; ++i) {
    const rqlp_problem &p = probs[i];
    const int64_t l = (int64_t)p.k + p.p;
    if (!p.A || !p.Omega || !p.Q || !p.L || !p.P || !p.piv0 || !p.piv1) return false;
    if (p.a_dtype != RQLP_F64 && p.a_dtype != RQLP_F32) return false;
    if (p.k < 1 || p.p < 0 || l > kPMaxL || l > p.n || l > p.m) return false;
    if (p.n > kPMaxN || p.lda < p.n || p.ldo < l || p.m > (1LL << 30)) return false;
  }
  return true;
}

// The workspace: per-launch zeroed region (item counter, abort flag, stage
// counters, control blocks), the tables, then every problem's buffers.
struct Layout {
  unsigned *next;
  int *abort, *done;
  unsigned long long *stats;
  Ctrl *ctrls;
  size_t zero_bytes;
  PStage *stages;
  PProb *probs;
  int4 *items;
  CUtensorMap *maps;
  int32_t *iota;
  std::vector<PProb> hp;
  size_t bytes;
};

// the exchange state of a gang of G CTAs (as cpqr.cu lays it out): the
// arrival counter's line, one winner line per CTA, double-buffered tagged
// candidate records and columns
size_t gang_bytes(int G, int l) {
  return 128 + 128 * (size_t)G + 2 * (size_t)G * cpqrk::kRecWords * sizeof(ulonglong2) +
         2 * (size_t)G * l * sizeof(ulonglong2);
}

void carve_all(void *ws, const rqlp_problem *probs, int count, const rqlp_opts &o, int nstages,
               int64_t nitems, Layout &L) {
  Arena a(ws);
  const bool tc = tc_prec(o.prec);
  char *head = a.take<char>(256);
  L.next = reinterpret_cast<unsigned *>(head);
  L.abort = reinterpret_cast<int *>(head ? head + 128 : nullptr);
  L.done = a.take<int>((size_t)count * nstages);
  L.stats = a.take<unsigned long long>(3 * kPKinds);
  L.ctrls = a.take<Ctrl>((size_t)count);
  // every gang's exchange state starts at zero in every launch
  std::vector<unsigned char *> cpx((size_t)count, nullptr);
  for (int i = 0; i < count; ++i) {
    const int G = cpqr_gang(probs[i].n, probs[i].k + probs[i].p);
    if (G > 1) cpx[(size_t)i] = a.take<unsigned char>(gang_bytes(G, probs[i].k + probs[i].p));
  }
  L.zero_bytes = a.off;
  L.stages = a.take<PStage>((size_t)nstages);
  L.probs = a.take<PProb>((size_t)count);
  L.items = a.take<int4>((size_t)nitems);
  L.maps = tc ? a.take<CUtensorMap>((size_t)count * 8) : nullptr;
  L.iota = a.take<int32_t>(kPMaxL);
  L.hp.assign((size_t)count, PProb());
  for (int i = 0; i < count; ++i) {
    const rqlp_problem &q = probs[i];
    PProb &p = L.hp[(size_t)i];
    std::memset(&p, 0, sizeof(p));
    const int l = q.k + q.p;
    p.A = q.A;
    p.a_dtype = q.a_dtype;
    p.l = l;
    p.m = q.m;
    p.n = q.n;
    p.lda = q.lda;
    p.Om = q.Omega;
    p.ldo = q.ldo;
    p.Q = q.Q;
    p.L = q.L;
    p.P = q.P;
    p.Lv = q.Lvalues;
    p.piv0 = q.piv0;
    p.piv1 = q.piv1;
    p.done0 = i * nstages;
    p.lpad = (l + 15) / 16 * 16;
    const size_t ml = (size_t)q.m * l, nl = (size_t)q.n * l, ll = (size_t)l * l;
    p.buf[PB_Y] = a.take<double>(ml);
    p.buf[PB_V] = a.take<double>(ml);
    p.buf[PB_Z] = a.take<double>(nl);
    p.buf[PB_W] = a.take<double>(nl);
    p.buf[PB_R0T] = a.take<double>(nl);
    p.buf[PB_X] = a.take<double>(nl);
    p.gpart = a.take<double>((size_t)cdiv(std::max(q.m, q.n), kGramRows) * ll);
    double **small[] = {&p.G, &p.Rp, &p.Dinv, &p.Racc, &p.Rtmp, &p.Q0, &p.QB,
                        &p.Qi, &p.Macc, &p.T0, &p.T1, &p.Vh};
    for (double **d : small) *d = a.take<double>(ll);
    p.tau = a.take<double>((size_t)l);
    p.pscr = a.take<int32_t>((size_t)l);
    p.rec = a.take<ulonglong2>(16);
    p.cpx = cpx[(size_t)i];
    p.ctrl = L.ctrls ? L.ctrls + i : nullptr;
    if (tc) {
      p.ldn8 = (q.n + 7) / 8 * 8;
      p.ldm8 = (q.m + 7) / 8 * 8;
      p.Ah = a.take<__nv_bfloat16>((size_t)q.m * p.ldn8);
      p.Al = a.take<__nv_bfloat16>((size_t)q.m * p.ldn8);
      p.Ath = a.take<__nv_bfloat16>((size_t)q.n * p.ldm8);
      p.Atl = a.take<__nv_bfloat16>((size_t)q.n * p.ldm8);
      p.Snh = a.take<__nv_bfloat16>((size_t)l * p.ldn8);
      p.Snl = a.take<__nv_bfloat16>((size_t)l * p.ldn8);
      p.Smh = a.take<__nv_bfloat16>((size_t)l * p.ldm8);
      p.Sml = a.take<__nv_bfloat16>((size_t)l * p.ldm8);
      p.maps = L.maps ? L.maps + (size_t)8 * i : nullptr;
    }
  }
  L.bytes = a.off;
}

// estimated duration (us) of one tile of stage s of problem p on one SM:
// HBM bytes at ~44 GB/s per SM, FP64 FMAs at ~3500 per us per SM
double tile_us(const PProb &p, const PStage &s, bool tc) {
  const double l = p.l, bw = 44e3, f64 = 3.5e3;
  switch (s.kind) {
    case PK_PREP: return 2.0 + (double)kPrepRows * kPrepCols * 16.0 / bw;
    case PK_SPLIT_OM: return 2.0 + kSplitRows * l * 10.0 / bw;
    case PK_PROD: {
      const double K = s.aux ? (double)p.m : (double)p.n;
      return tc ? 3.0 + kTcRows * K * 4.0 / bw : 2.0 + kF64Rows * p.lpad * K / f64;
    }
    case PK_GRAM:
      return (s.cond ? 1.0 : 2.0 + kGramRows * l * l * 0.5 / (s.lowp ? 40.0 * f64 : f64));
    case PK_CHOL: return s.cond ? 1.0 : 5.0 + l * (s.lowp ? 0.6 : 1.5);
    case PK_APPLY:
      return s.cond ? 1.0 : 3.0 + kApplyRowsP * l * l * 0.5 / (s.lowp ? 40.0 * f64 : f64);
    case PK_CPQR: {
      const int G = cpqr_gang(p.n, p.l);
      if (G == 1) return 20.0 + 1.5 * (double)p.n * l * l / f64 + 2.0 * l * l * l / f64;
      // a gang: its share of the FP64 work plus one exchange (~6 us) per pivot step
      return 20.0 + 1.5 * (double)p.n * l * l / f64 / G + 6.0 * l;
    }
    case PK_TAIL: return 20.0 + 4.0 * l * l * l / f64;
    case PK_ASM: return 2.0 + kAsmRows * l * l / f64;
    default: return 1.0;
  }
}

// List schedule of every item on W workers: among the stages whose previous
// stage has finished, the one of largest remaining critical path hands out
// its next tile to the first free worker.  The order tiles are handed out in
// is the item order (each item after every item it depends on).
std::vector<int4> schedule(const std::vector<PProb> &hp, const std::vector<PStage> &st, bool tc,
                           int W) {
  const int P = (int)hp.size(), S = (int)st.size();
  std::vector<double> dur((size_t)P * S), blev((size_t)P * S);
  std::vector<int> tiles((size_t)P * S);
  for (int p = 0; p < P; ++p) {
    double acc = 0.0;
    for (int s = S - 1; s >= 0; --s) {
      const size_t k = (size_t)p * S + s;
      tiles[k] = tiles_of(hp[(size_t)p], st[(size_t)s], tc ? 1 : 0);
      dur[k] = tile_us(hp[(size_t)p], st[(size_t)s], tc);
      acc += dur[k] * (double)cdiv(tiles[k], W);
      blev[k] = acc;
    }
  }
  struct Ready {
    double prio;
    int p, s;
    bool operator<(const Ready &o) const {
      if (prio != o.prio) return prio < o.prio;
      if (p != o.p) return p > o.p;
      return s > o.s;
    }
  };
  struct Pending {
    double t;
    int p, s;
    bool operator<(const Pending &o) const { return t > o.t; }
  };
  std::priority_queue<Ready> ready;
  std::priority_queue<Pending> pending;
  std::priority_queue<double, std::vector<double>, std::greater<double>> workers;
  for (int w = 0; w < W; ++w) workers.push(0.0);
  std::vector<int> handed((size_t)P * S, 0);
  std::vector<double> finish((size_t)P * S, 0.0);
  for (int p = 0; p < P; ++p) ready.push({blev[(size_t)p * S], p, 0});
  std::vector<int4> order;
  size_t total = 0;
  for (int t : tiles) total += (size_t)t;
  order.reserve(total);
  while (order.size() < total) {
    double now = workers.top();
    workers.pop();
    while (!pending.empty() && pending.top().t <= now) {
      const Pending q = pending.top();
      pending.pop();
      ready.push({blev[(size_t)q.p * S + q.s], q.p, q.s});
    }
    if (ready.empty()) {
      now = std::max(now, pending.top().t);
      while (!pending.empty() && pending.top().t <= now) {
        const Pending q = pending.top();
        pending.pop();
        ready.push({blev[(size_t)q.p * S + q.s], q.p, q.s});
      }
    }
    const Ready r = ready.top();
    const size_t k = (size_t)r.p * S + r.s;
    if (st[(size_t)r.s].kind == PK_CPQR && tiles[k] > 1) {
      // a gang: all its tiles one after another, to the next free workers,
      // which start together
      std::vector<double> starts(1, now);
      for (int t = 1; t < tiles[k]; ++t) {
        starts.push_back(workers.top());
        workers.pop();
      }
      double t0 = now;
      for (double x : starts) t0 = std::max(t0, x);
      for (int t = 0; t < tiles[k]; ++t) {
        order.push_back(make_int4(r.p, r.s, handed[k]++, 0));
        workers.push(t0 + dur[k]);
      }
      finish[k] = t0 + dur[k];
    } else {
      const int tile = handed[k]++;
      order.push_back(make_int4(r.p, r.s, tile, 0));
      const double end = now + dur[k];
      finish[k] = std::max(finish[k], end);
      workers.push(end);
    }
    if (handed[k] == tiles[k]) {
      ready.pop();
      if (r.s + 1 < S) pending.push({finish[k], r.p, r.s + 1});
    }
  }
  return order;
}

bool make_map(CUtensorMap *map, const void *base, int64_t rows, int64_t cols, int64_t ld,
              int box_rows) {
  auto fn = tma_encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides,
            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int64_t count_items(const rqlp_problem *probs, int count, const std::vector<PStage> &st, bool tc) {
  int64_t n = 0;
  for (int i = 0; i < count; ++i) {
    PProb p;
    std::memset(&p, 0, sizeof(p));
    p.m = probs[i].m;
    p.n = probs[i].n;
    p.l = probs[i].k + probs[i].p;
    for (const PStage &s : st) n += tiles_of(p, s, tc ? 1 : 0);
  }
  return n;
}

}  // namespace

size_t persist_ws_bytes(const rqlp_problem *probs, int count, const rqlp_opts *o) {
  if (!supported(probs, count, o)) return 0;
  const std::vector<PStage> st = build_stages(*o);
  const int64_t ni = count_items(probs, count, st, tc_prec(o->prec));
  Layout L;
  carve_all(nullptr, probs, count, *o, (int)st.size(), ni, L);
  return L.bytes;
}

int persist_setup(const rqlp_problem *probs, int count, const rqlp_opts *o, void *ws,
                  size_t ws_bytes, int32_t *d_status, PersistLaunch *out) {
  if (!out) return RQLP_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  if (!supported(probs, count, o)) return RQLP_ERR_UNSUPPORTED;
  const bool tc = tc_prec(o->prec);
  const std::vector<PStage> st = build_stages(*o);
  const int S = (int)st.size();
  const int64_t ni = count_items(probs, count, st, tc);
  if (ni >= (1LL << 31)) return RQLP_ERR_UNSUPPORTED;
  Layout L;
  carve_all(ws, probs, count, *o, S, ni, L);
  if (!ws || L.bytes > ws_bytes || reinterpret_cast<uintptr_t>(ws) % 256) return RQLP_ERR_WORKSPACE;
  for (int i = 0; i < count; ++i) L.hp[(size_t)i].status_out = d_status + i;
  // launch shape: one CTA per SM
  const int smem = (int)(kPSmem + 1024);
  if (cudaFuncSetAttribute(k_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
      cudaSuccess)
    return RQLP_ERR_CUDA;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist, kPT, smem) != cudaSuccess ||
      per_sm < 1)
    return RQLP_ERR_CUDA;
  const int grid = num_sms() * per_sm;
  const std::vector<int4> order = schedule(L.hp, st, tc, grid);
  if ((int64_t)order.size() != ni) return RQLP_ERR_INVALID_ARG;
  {
    // every item after all tiles of its problem's previous stage (the order
    // the kernel's progress rests on), every tile exactly once
    std::vector<int> seen((size_t)count * S, 0);
    for (const int4 &it : order) {
      if (it.x < 0 || it.x >= count || it.y < 0 || it.y >= S) return RQLP_ERR_INVALID_ARG;
      const PProb &p = L.hp[(size_t)it.x];
      if (it.y > 0 && seen[(size_t)it.x * S + it.y - 1] != tiles_of(p, st[(size_t)it.y - 1], tc))
        return RQLP_ERR_INVALID_ARG;
      if (it.z != seen[(size_t)it.x * S + it.y]++) return RQLP_ERR_INVALID_ARG;
    }
  }
  int lpad_max = 16;
  for (const PProb &p : L.hp) lpad_max = std::max(lpad_max, p.lpad);
  const size_t sbytes = 2 * ((size_t)kTcRows * 128 + (size_t)lpad_max * 128);
  const int ring = (int)std::min<size_t>(kPMaxRing, kPSmem / sbytes);
  if (tc && ring < 2) return RQLP_ERR_UNSUPPORTED;
  std::vector<CUtensorMap> maps;
  if (tc) {
    maps.resize((size_t)count * 8);
    for (int i = 0; i < count; ++i) {
      const PProb &p = L.hp[(size_t)i];
      CUtensorMap *mp = maps.data() + (size_t)8 * i;
      const bool ok = make_map(mp + 0, p.Ah, p.m, p.n, p.ldn8, kTcRows) &&
                      make_map(mp + 1, p.Al, p.m, p.n, p.ldn8, kTcRows) &&
                      make_map(mp + 2, p.Ath, p.n, p.m, p.ldm8, kTcRows) &&
                      make_map(mp + 3, p.Atl, p.n, p.m, p.ldm8, kTcRows) &&
                      make_map(mp + 4, p.Snh, p.l, p.n, p.ldn8, p.lpad) &&
                      make_map(mp + 5, p.Snl, p.l, p.n, p.ldn8, p.lpad) &&
                      make_map(mp + 6, p.Smh, p.l, p.m, p.ldm8, p.lpad) &&
                      make_map(mp + 7, p.Sml, p.l, p.m, p.ldm8, p.lpad);
      if (!ok) return RQLP_ERR_CUDA;
    }
  }
  std::vector<int32_t> io(kPMaxL);
  for (int i = 0; i < kPMaxL; ++i) io[(size_t)i] = i;
  if (cudaMemcpy(L.stages, st.data(), sizeof(PStage) * st.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(L.probs, L.hp.data(), sizeof(PProb) * L.hp.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(L.items, order.data(), sizeof(int4) * order.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMemcpy(L.iota, io.data(), sizeof(int32_t) * io.size(), cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      (tc && cudaMemcpy(L.maps, maps.data(), sizeof(CUtensorMap) * maps.size(),
                        cudaMemcpyHostToDevice) != cudaSuccess))
    return RQLP_ERR_CUDA;
  PPlan *pp = new PPlan;
  pp->probs = L.probs;
  pp->stages = L.stages;
  pp->items = L.items;
  pp->next = L.next;
  pp->done = L.done;
  pp->abort = L.abort;
  pp->iota = L.iota;
  pp->stats = L.stats;
  pp->nstages = S;
  pp->nitems = (int)ni;
  pp->tc = tc ? 1 : 0;
  pp->pivot2 = o->pivot2 ? 1 : 0;
  pp->d = o->d;
  pp->ring = ring;
  pp->limit_ns = o->spin_limit_ns > 0 ? (unsigned long long)o->spin_limit_ns : kDefaultSpinNs;
  out->params = pp;
  out->param_bytes = sizeof(PPlan);
  out->zero_base = ws;
  out->zero_bytes = L.zero_bytes;
  out->grid = grid;
  out->smem = smem;
  out->items = ni;
  return RQLP_OK;
}

int persist_enqueue(const PersistLaunch &pl, cudaStream_t st) {
  if (!pl.params) return RQLP_ERR_INVALID_ARG;
  if (cudaMemsetAsync(pl.zero_base, 0, pl.zero_bytes, st) != cudaSuccess) return RQLP_ERR_CUDA;
  const PPlan &P = *static_cast<const PPlan *>(pl.params);
  // a cooperative launch: every CTA is resident at once, which the gangs of
  // the CPQR items (CTAs waiting for one another) need
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)pl.grid);
  cfg.blockDim = dim3(kPT);
  cfg.dynamicSmemBytes = (size_t)pl.smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, k_persist, P);
  count_launch();
  return (e == cudaSuccess && cudaGetLastError() == cudaSuccess) ? RQLP_OK : RQLP_ERR_CUDA;
}

int persist_stats(const PersistLaunch &pl, cudaStream_t st, double *busy_us, double *wait_us,
                  int64_t *items) {
  if (!pl.params) return RQLP_ERR_INVALID_ARG;
  const PPlan &P = *static_cast<const PPlan *>(pl.params);
  unsigned long long h[3 * kPKinds];
  if (cudaMemcpyAsync(h, P.stats, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return RQLP_ERR_CUDA;
  for (int k = 0; k < kPKinds; ++k) {
    if (busy_us) busy_us[k] = (double)h[k] * 1e-3;
    if (wait_us) wait_us[k] = (double)h[kPKinds + k] * 1e-3;
    if (items) items[k] = (int64_t)h[2 * kPKinds + k];
  }
  return RQLP_OK;
}

void persist_release(PersistLaunch *pl) {
  if (!pl) return;
  delete static_cast<PPlan *>(pl->params);
  pl->params = nullptr;
}

}  // namespace rqk
