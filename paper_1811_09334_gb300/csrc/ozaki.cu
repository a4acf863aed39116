// FP64-accurate products on the 5th-generation tensor cores.
//
// GB300 runs FP64 at about 1 TFLOP/s, so every O(N l^2) and O(m n l) product
// of the method on FP64 data is bound by the FP64 units.  This file computes
// such products on the BF16 tensor cores with exact digit splitting, the
// scheme of Ozaki, Ogita, Oishi and Rump ("Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59, 2012), laid out for tcgen05:
//
//   * each operand row is scaled by a power of two 2^e with |x| < 2^e and cut
//     into kOzDigits signed 8-bit digits, x = 2^e sum_i d_i 2^(-7-8i) + r,
//     |d_i| <= 128, |r| <= 2^(e-48), computed on the integer pipe from the
//     FP64 bit pattern (no FP64 instruction);
//   * a digit product d_i e_j is an integer of at most 2^14, so a sum of up to
//     1024 of them is exact in the FP32 accumulator: the product of digit
//     pair (i, j) over a K slice of 1024 is exact;
//   * C = 2^(ex+ey) sum_{i,j} 2^(-14-8(i+j)) D_i E_j^T; the pairs of weight
//     group t = i + j = 0..3 are kept exact (one accumulator per pair, the K
//     slices summed as 64-bit integers), the pairs with t = 4, 5 go into one
//     FP32 accumulator with E_j pre-scaled by 2^(-8(t-4)) (their rounding is
//     2^-24 of a term that is itself 2^-32 of the result), and pairs with
//     t >= 6 are dropped (2^-48 of the row scales);
//   * one CTA per job (the pairs of one X digit, at most four accumulators;
//     digit 0's rounded pairs form a seventh job), 128-row tile of C and K
//     slice of 1024: a TMA producer streams 64-byte-swizzled tiles of the X
//     digit and of the Y digits the job needs through a ring of stages, one
//     thread issues tcgen05.mma kind::f16 into the TMEM accumulators, and the
//     epilogue writes FP32 partial sums; a second kernel adds them, applies
//     the weights and the scales, and writes C in FP64.
//
// Every mbarrier wait is bounded (RQLP_ERR_TIMEOUT).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "ozaki.cuh"
#include "tc.cuh"

namespace rqk {

PFN_cuTensorMapEncodeTiled_v12000 tma_encode_fn();

namespace {

using namespace tc;

constexpr int kS = kOzDigits;
constexpr int kC = kOzCopies;
constexpr int kTM = 128;                 // rows of a C tile (MMA M)
constexpr int kTK = 32;                  // K values per stage (one 64-byte swizzle row)
constexpr int kKbExact = 1024 / kTK;     // K blocks per slice: 1024 terms stay exact
constexpr int kMaxAcc = 4;
constexpr int kMaxW = 5;                 // Y digit tiles of one job
constexpr int kExact = 4;                // weight groups t = 0..3 summed exactly
constexpr int kJobs = kS + 1;            // digit 0's rounded pairs form a job of their own
constexpr int kSlots = 16;               // accumulators over all jobs
constexpr int kMaxStages = 6;
constexpr size_t kSmemLimit = 227 * 1024;
constexpr int kExpNone = -1000;          // exponent of an all-zero row

// ------------------------------------------------------------ digits
// Exponent e with |x| < 2^e for a finite nonzero x given its bit pattern;
// zero gives kExpNone, a non-finite value 2000.
__device__ __forceinline__ int exp_bound(unsigned long long ab) {
  const int be = (int)(ab >> 52);
  if (ab == 0ull) return kExpNone;
  if (be == 0x7ff) return 2000;
  return be == 0 ? -1021 : be - 1022;
}

// Digits of x relative to 2^e (|x| < 2^e): the fixed-point magnitude
// |Y| = |x| 2^(62 - e) < 2^62 is cut into bytes of weight 2^(55 - 8i)
// (bits 62..15), rounded at bit 14, and the bytes are turned into signed
// digits from the lowest one up (a byte of 128 or more becomes byte - 256
// with a carry into the next), so that |d_i| <= 128 and the remainder after
// the last digit is at most 2^14, i.e. 2^-48 relative to 2^e; the sign of x
// goes to every digit.  One variable 64-bit shift, the rest 32-bit integer
// operations.  Digits are exact BF16 values, returned as bit patterns.
__device__ __forceinline__ uint16_t bf16_of_small_int(int q) {
  // q in [-128, 128] to FP32 exactly (1.5 2^23 + q has unit spacing); its top
  // 16 bits are the BF16 value
  const float f = __int_as_float(0x4B400000 + q) - 12582912.0f;
  return (uint16_t)(__float_as_uint(f) >> 16);
}

__device__ __forceinline__ void digits_of(double x, int e, uint16_t (&d)[kS]) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int be = (int)((b >> 52) & 0x7ff);
  unsigned long long Y = 0;
  if (be != 0 && be != 0x7ff && e > kExpNone) {
    const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);
    const int sh = (be - 1023) - e + 10;  // |x| 2^(62-e) = m 2^(be-1023-52+62-e), sh <= 9
    if (sh >= 0) Y = m << min(sh, 9);
    else if (sh > -63) Y = m >> (-sh);
  }
  const unsigned yh = (unsigned)(Y >> 32), yl = (unsigned)Y;
  int u[kS];
  u[0] = (int)(yh >> 23);                          // bits 55..62
  u[1] = (int)((yh >> 15) & 0xffu);                // 47..54
  u[2] = (int)((yh >> 7) & 0xffu);                 // 39..46
  u[3] = (int)(((yh << 1) | (yl >> 31)) & 0xffu);  // 31..38
  u[4] = (int)((yl >> 23) & 0xffu);                // 23..30
  u[5] = (int)((yl >> 15) & 0xffu);                // 15..22
  int c = (int)((yl >> 14) & 1u);                  // rounding at bit 14
  const int sgn = (b >> 63) ? -1 : 1;
#pragma unroll
  for (int i = kS - 1; i >= 0; --i) {
    const int v = u[i] + c;
    c = (i > 0 && v >= 128) ? 1 : 0;
    d[i] = bf16_of_small_int(sgn * (v - (c << 8)));
  }
}

// d 2^(-8m) as a BF16 bit pattern (d an integer digit, so no underflow)
__device__ __forceinline__ uint16_t scaled_digit(uint16_t d, int m) {
  return (d & 0x7fffu) ? (uint16_t)(d - (uint16_t)((8 * m) << 7)) : d;
}

__device__ __forceinline__ double as_f64(double x) { return x; }
__device__ __forceinline__ double as_f64(float x) { return f2d(x); }  // integer pipe

// Row exponents (trans = false): one warp per row of S, the largest |x| by
// its bit pattern.  Non-finite data records RQLP_ERR_NONFINITE.
template <typename T>
__global__ void __launch_bounds__(256)
k_oz_exp_rows(const T *__restrict__ S, int64_t r, int64_t c, int64_t ld, int32_t *exps, Ctrl *ctrl,
              const int *skip) {
  if (skip && ld_volatile_i32(skip) == 0) return;
  const int lane = threadIdx.x & 31;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < r;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    unsigned long long mx = 0;
    for (int64_t j = lane; j < c; j += 32) {
      const unsigned long long ab =
          (unsigned long long)__double_as_longlong(as_f64(S[i * ld + j])) & 0x7fffffffffffffffull;
      mx = ab > mx ? ab : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = v > mx ? v : mx;
    }
    if (lane == 0) {
      const int e = exp_bound(mx);
      if (e == 2000) set_status(ctrl, RQLP_ERR_NONFINITE);
      exps[i] = e;
    }
  }
}

// Column exponents (trans = true): (32, 8) blocks over 32 columns and a slab
// of rows, one atomic max per column and block; exps starts at INT_MIN.
template <typename T>
__global__ void __launch_bounds__(256)
k_oz_exp_cols(const T *__restrict__ S, int64_t r, int64_t c, int64_t ld, int32_t *exps, Ctrl *ctrl,
              const int *skip) {
  if (skip && ld_volatile_i32(skip) == 0) return;
  __shared__ int red[8][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t j = (int64_t)blockIdx.x * 32 + tx;
  unsigned long long mx = 0;
  if (j < c)
    for (int64_t i = (int64_t)blockIdx.y * 8 + ty; i < r; i += (int64_t)gridDim.y * 8) {
      const unsigned long long ab =
          (unsigned long long)__double_as_longlong(as_f64(S[i * ld + j])) & 0x7fffffffffffffffull;
      mx = ab > mx ? ab : mx;
    }
  red[ty][tx] = exp_bound(mx);
  __syncthreads();
  if (ty == 0 && j < c) {
    int e = red[0][tx];
    for (int y = 1; y < 8; ++y) e = max(e, red[y][tx]);
    if (e == 2000) set_status(ctrl, RQLP_ERR_NONFINITE);
    atomicMax(exps + j, e);
  }
}

// Digits of the rows of S (trans = false): (32, 8) blocks, each lane two
// neighbouring elements of a row, one BF16 pair store per digit array.
template <typename T>
__global__ void __launch_bounds__(256)
k_oz_digits(const T *__restrict__ S, int64_t r, int64_t c, int64_t ld, const int32_t *__restrict__ exps,
            uint16_t *__restrict__ dig, int64_t ldd, int copies, const int *skip) {
  if (skip && ld_volatile_i32(skip) == 0) return;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t plane = r * ldd;
  for (int64_t i = (int64_t)blockIdx.y * 8 + ty; i < r; i += (int64_t)gridDim.y * 8) {
    const int e = exps[i];
    for (int64_t j = ((int64_t)blockIdx.x * 32 + tx) * 2; j < c; j += (int64_t)gridDim.x * 64) {
      uint16_t d0[kS], d1[kS];
      digits_of(as_f64(S[i * ld + j]), e, d0);
      const bool two = j + 1 < c;
      digits_of(two ? as_f64(S[i * ld + j + 1]) : 0.0, e, d1);
#pragma unroll
      for (int q = 0; q < kS; ++q)
        for (int m = 0; m < copies; ++m) {
          uint16_t *p = dig + (int64_t)(q * copies + m) * plane + i * ldd + j;
          const uint16_t a = scaled_digit(d0[q], m), b = scaled_digit(d1[q], m);
          if (two) *reinterpret_cast<uint32_t *>(p) = (uint32_t)a | ((uint32_t)b << 16);
          else p[0] = a;
        }
    }
  }
}

// Digits of the columns of S (trans = true): 32 x 32 tiles through shared
// memory, S read along its rows and the digit arrays written along K.
template <typename T>
__global__ void __launch_bounds__(256)
k_oz_digits_t(const T *__restrict__ S, int64_t r, int64_t c, int64_t ld,
              const int32_t *__restrict__ exps, uint16_t *__restrict__ dig, int64_t ldd, int copies,
              const int *skip) {
  if (skip && ld_volatile_i32(skip) == 0) return;
  __shared__ uint16_t sh[kS * kC][32][34];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t j0 = (int64_t)blockIdx.x * 32;  // operand rows (columns of S)
  const int64_t plane = c * ldd;
  for (int64_t k0 = (int64_t)blockIdx.y * 32; k0 < r; k0 += (int64_t)gridDim.y * 32) {
    const int64_t j = j0 + tx;
    const int e = j < c ? exps[j] : kExpNone;
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4) {
      const int kr = ty + 8 * q4;
      const int64_t k = k0 + kr;
      uint16_t d[kS];
      digits_of((k < r && j < c) ? as_f64(S[k * ld + j]) : 0.0, e, d);
#pragma unroll
      for (int q = 0; q < kS; ++q)
        for (int m = 0; m < copies; ++m) sh[q * copies + m][tx][kr] = scaled_digit(d[q], m);
    }
    __syncthreads();
    const int arrays = kS * copies;
    for (int a = 0; a < arrays; ++a)
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {
        const int jr = ty + 8 * q4;
        const int64_t jj = j0 + jr, k = k0 + tx;
        if (jj < c && k < r) dig[(int64_t)a * plane + jj * ldd + k] = sh[a][jr][tx];
      }
    __syncthreads();
  }
}

// Both orientations of one matrix at once (the digits of A's rows and of its
// columns, each against its own exponents).  Exponents: tiles of 32 rows x
// 128 columns (8 warps, lanes along the rows, four columns each), one atomic
// max per row and per column and tile; rexp and cexp start at INT_MIN.
template <typename T>
__global__ void __launch_bounds__(256)
k_oz_exps_both(const T *__restrict__ S, int64_t r, int64_t c, int64_t ld, int32_t *rexp,
               int32_t *cexp, Ctrl *ctrl) {
  __shared__ unsigned long long red[8][128];
  const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 128;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long cm[4] = {0, 0, 0, 0}, rm[4] = {0, 0, 0, 0};
#pragma unroll
  for (int p4 = 0; p4 < 4; ++p4) {
    const int64_t i = i0 + warp + 8 * p4;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t j = j0 + lane + 32 * q;
      if (i < r && j < c) {
        const unsigned long long ab =
            (unsigned long long)__double_as_longlong(as_f64(S[i * ld + j])) & 0x7fffffffffffffffull;
        cm[q] = ab > cm[q] ? ab : cm[q];
        rm[p4] = ab > rm[p4] ? ab : rm[p4];
      }
    }
  }
#pragma unroll
  for (int p4 = 0; p4 < 4; ++p4) {
    unsigned long long v = rm[p4];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long w2 = __shfl_xor_sync(0xffffffffu, v, o);
      v = w2 > v ? w2 : v;
    }
    const int64_t i = i0 + warp + 8 * p4;
    if (lane == 0 && i < r) {
      const int ee = exp_bound(v);
      if (ee == 2000) set_status(ctrl, RQLP_ERR_NONFINITE);
      atomicMax(rexp + i, ee);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) red[warp][lane + 32 * q] = cm[q];
  __syncthreads();
  if (threadIdx.x < 128) {
    const int64_t j = j0 + threadIdx.x;
    unsigned long long t = red[0][threadIdx.x];
    for (int w = 1; w < 8; ++w) t = red[w][threadIdx.x] > t ? red[w][threadIdx.x] : t;
    if (j < c) {
      const int ee = exp_bound(t);
      if (ee == 2000) set_status(ctrl, RQLP_ERR_NONFINITE);
      atomicMax(cexp + j, ee);
    }
  }
}

// Digits of the rows (rexp) and of the columns (cexp) of S from one read of
// S: 32 x 32 tiles on (32, 8) blocks; the row digits go out along the rows,
// the column digits through shared memory along the columns.
template <typename T>
__global__ void __launch_bounds__(256)
k_oz_digits_both(const T *__restrict__ S, int64_t r, int64_t c, int64_t ld,
                 const int32_t *__restrict__ rexp, const int32_t *__restrict__ cexp,
                 uint16_t *__restrict__ drow, int64_t ldr, uint16_t *__restrict__ dcol,
                 int64_t ldc) {
  __shared__ uint16_t sh[kS][32][34];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t j0 = (int64_t)blockIdx.x * 32, i0 = (int64_t)blockIdx.y * 32;
  const int64_t prow = r * ldr, pcol = c * ldc;
  const int64_t j = j0 + tx;
  const int ec = j < c ? cexp[j] : kExpNone;
#pragma unroll
  for (int q4 = 0; q4 < 4; ++q4) {
    const int ir = ty + 8 * q4;
    const int64_t i = i0 + ir;
    const bool in = i < r && j < c;
    const double x = in ? as_f64(S[i * ld + j]) : 0.0;
    uint16_t d[kS];
    if (i < r) {
      digits_of(x, rexp[i], d);
      if (j < c)
#pragma unroll
        for (int q = 0; q < kS; ++q) drow[(int64_t)q * prow + i * ldr + j] = d[q];
    }
    digits_of(x, ec, d);
#pragma unroll
    for (int q = 0; q < kS; ++q) sh[q][tx][ir] = d[q];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kS; ++q)
#pragma unroll
    for (int q4 = 0; q4 < 4; ++q4) {
      const int jr = ty + 8 * q4;
      const int64_t jj = j0 + jr, i = i0 + tx;
      if (jj < c && i < r) dcol[(int64_t)q * pcol + jj * ldc + i] = sh[q][jr][tx];
    }
}

// ------------------------------------------------------------ products
// One job: the pairs (i, j) of X digit i that one CTA forms, with the Y
// digit array index (j * kC + m) of each, its accumulator slot, and the
// weight group of each slot (0..3 exact; 4 the rounded rest).
struct OzJob {
  int xi, nw, nacc, slot0;
  int widx[kMaxW];
  int wacc[kMaxW];
  int first[kMaxW];  // the pair that opens its accumulator
  int group[kMaxAcc];
};

struct OzArgs {
  int M, n_pad, ncols, nk, kb_per, stages;
  uint32_t tmem_cols;
  int acc_cols;
  float *part;
  int64_t slot_stride, split_stride;
  int ldp;
  Ctrl *ctrl;
  unsigned long long limit_ns;
  const int *skip;
  int njobs;
  OzJob job[kJobs];
};

__global__ void __launch_bounds__(128, 1)
k_oz_mma(const __grid_constant__ CUtensorMap tX, const __grid_constant__ CUtensorMap tY,
         const __grid_constant__ OzArgs a) {
  // a conditional pass that is not needed: the whole CTA returns before any set-up
  if (a.skip && ld_volatile_i32(a.skip) == 0) return;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[kMaxStages], bar_empty[kMaxStages], bar_acc;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  // the jobs of one (tile, K slice) are neighbours in launch order, so the CTAs
  // that read the same X digit tile run side by side and share it in L2
  const int m_tile = blockIdx.y, split = blockIdx.z;
  const OzJob &jb = a.job[blockIdx.x];
  const int di = jb.xi;
  const uint32_t xbytes = kTM * kTK * 2, ybytes = (uint32_t)a.n_pad * kTK * 2;
  const uint32_t stage_bytes = xbytes + kMaxW * ybytes;
  const uint32_t tx_bytes = xbytes + (uint32_t)jb.nw * ybytes;
  const int kb0 = split * a.kb_per;
  const int nkb = min(a.kb_per, a.nk - kb0);

  if (tid == 0) {
    for (int s = 0; s < a.stages; ++s) {
      mbar_init(&bar_full[s], 1);
      mbar_init(&bar_empty[s], 1);
    }
    mbar_init(&bar_acc, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_abort = 0;
  }
  if (warp == 0) tmem_alloc(&s_tmem, a.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer: the X digit tile and this digit's Y tiles ----
      // (the job's table in registers: no parameter loads inside the loop)
      const int nw = jb.nw;
      int widx[kMaxW];
#pragma unroll
      for (int w = 0; w < kMaxW; ++w) widx[w] = w < nw ? jb.widx[w] : 0;
      int issued = 0;
      for (int i = 0; i < nkb; ++i) {
        const int s = i % a.stages;
        const uint32_t ph = (uint32_t)(i / a.stages) & 1u;
        if (!mbar_wait(&bar_empty[s], ph ^ 1u, a.limit_ns) || *(volatile int *)&s_abort) {
          s_abort = 1;
          break;
        }
        const uint32_t st = smem_u32(smem + (size_t)s * stage_bytes);
        mbar_expect_tx(&bar_full[s], tx_bytes);
        const int kx = (kb0 + i) * kTK;
        tma_load_3d(st, &tX, kx, m_tile * kTM, di, &bar_full[s]);
#pragma unroll
        for (int w = 0; w < kMaxW; ++w)
          if (w < nw) tma_load_3d(st + xbytes + w * ybytes, &tY, kx, 0, widx[w], &bar_full[s]);
        issued = i + 1;
      }
      for (int s = 0; s < a.stages && s < issued; ++s) {
        const int last = ((issued - 1 - s) / a.stages) * a.stages + s;
        mbar_wait(&bar_full[s], (uint32_t)(last / a.stages) & 1u, a.limit_ns);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer ----
      // accumulator address, B-tile offset and opening flag of every pair in
      // registers before the loop (the issuing thread would otherwise wait on
      // a parameter load before each MMA)
      const uint32_t idesc = instr_desc(kTM, a.n_pad);
      const int nw = jb.nw;
      uint32_t td[kMaxW], boff[kMaxW], opens[kMaxW];
#pragma unroll
      for (int w = 0; w < kMaxW; ++w) {
        td[w] = tmem + (uint32_t)((w < nw ? jb.wacc[w] : 0) * a.acc_cols);
        boff[w] = xbytes + (uint32_t)w * ybytes;
        opens[w] = (w < nw && jb.first[w]) ? 1u : 0u;
      }
      for (int i = 0; i < nkb; ++i) {
        const int s = i % a.stages;
        const uint32_t ph = (uint32_t)(i / a.stages) & 1u;
        if (!mbar_wait(&bar_full[s], ph, a.limit_ns) || *(volatile int *)&s_abort) {
          s_abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t xa = smem_u32(smem + (size_t)s * stage_bytes);
#pragma unroll
        for (int k = 0; k < kTK / 16; ++k) {
          // 16 BF16 values (32 bytes) along K inside the 64-byte swizzled row
          const uint32_t off = k * 32;
          const uint64_t adesc = smem_desc_sw64(xa + off);
#pragma unroll
          for (int w = 0; w < kMaxW; ++w) {
            if (w >= nw) break;
            const uint32_t accum = (i == 0 && k == 0 && opens[w]) ? 0u : 1u;
            mma_bf16(td[w], adesc, smem_desc_sw64(xa + boff[w] + off), idesc, accum);
          }
        }
        mma_commit(&bar_empty[s]);
      }
      mma_commit(&bar_acc);
    }
    __syncwarp();
  }

  // ---- epilogue: each accumulator to its FP32 partial-sum slot ----
  const bool ready = mbar_wait(&bar_acc, 0, a.limit_ns);
  tc_fence_after();
  __syncthreads();
  if (!ready || *(volatile int *)&s_abort) {
    if (tid == 0) set_status(a.ctrl, RQLP_ERR_TIMEOUT);
  } else {
    const int row = m_tile * kTM + warp * 32 + lane;
    const uint32_t lanes = (uint32_t)(warp * 32) << 16;
    for (int q = 0; q < jb.nacc; ++q) {
      float *out = a.part + (int64_t)(jb.slot0 + q) * a.slot_stride +
                   (int64_t)split * a.split_stride + (int64_t)row * a.ldp;
      // 64 columns per round: two loads in flight, one wait
      for (int c0 = 0; c0 < a.n_pad; c0 += 64) {
        uint32_t r0[32], r1[32];
        const uint32_t base = tmem + lanes + (uint32_t)(q * a.acc_cols + c0);
        tmem_ld32_nowait(base, r0);
        tmem_ld32_nowait(base + 32, r1);  // columns past n_pad stay inside the accumulator
        tmem_ld_wait();
        if (row < a.M) {
#pragma unroll
          for (int j = 0; j < 32; j += 4)
            if (c0 + j < a.n_pad)
              *reinterpret_cast<uint4 *>(out + c0 + j) = make_uint4(r0[j], r0[j + 1], r0[j + 2], r0[j + 3]);
#pragma unroll
          for (int j = 0; j < 32; j += 4)
            if (c0 + 32 + j < a.n_pad)
              *reinterpret_cast<uint4 *>(out + c0 + 32 + j) =
                  make_uint4(r1[j], r1[j + 1], r1[j + 2], r1[j + 3]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, a.tmem_cols);
}

// The weight group of every partial-sum slot, three bits each (no indexed
// parameter array in the reduction kernels).
struct OzReduce {
  unsigned long long groups;
  int nslots;
  __device__ __forceinline__ int group(int q) const { return (int)((groups >> (3 * q)) & 7ull); }
};

// 2^p as an FP64 value (p within the normal range), built from its bits
__device__ __forceinline__ double pow2(int p) {
  return __longlong_as_double((long long)(1023 + p) << 52);
}

// C = 2^(ex + ey - 38) (G0 2^24 + G1 2^16 + G2 2^8 + G3 + 2^-8 A), with the
// exact groups G summed over slots and K slices as 64-bit integers (exact)
// and the rounded group A in FP32.
__device__ __forceinline__ double oz_combine(long long E, float ap, int e1, int e2) {
  if (e1 <= kExpNone || e2 <= kExpNone) return 0.0;
  const int p = e1 + e2 - 38;
  const double sum = fma((double)ap, 0x1p-8, (double)E);
  return (p > -1022 && p < 1023) ? sum * pow2(p) : ldexp(sum, p);
}

// Many outputs (M N large): one thread per element of C, lanes along a row
// (coalesced partial reads), the slices of each slot loaded four at a time.
__global__ void __launch_bounds__(256)
k_oz_reduce(const float *__restrict__ part, OzReduce rd, int S, int64_t slot_stride,
            int64_t split_stride, int ldp, int64_t M, int ncols, const int32_t *__restrict__ ex,
            const int32_t *__restrict__ ey, double *__restrict__ C, int64_t ldc,
            const int32_t *__restrict__ rowmap, const int *skip) {
  if (skip && ld_volatile_i32(skip) == 0) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; i < M;
       i += (int64_t)gridDim.x * blockDim.y)
    for (int j = threadIdx.x; j < ncols; j += blockDim.x) {
      long long E = 0;
      float ap = 0.f;
      for (int q = 0; q < rd.nslots; ++q) {
        const int grp = rd.group(q);
        const float *p = part + (int64_t)q * slot_stride + i * ldp + j;
        long long gi = 0;
        float fa = 0.f;
        int z = 0;
        for (; z + 4 <= S; z += 4) {
          const float v0 = p[(int64_t)z * split_stride], v1 = p[(int64_t)(z + 1) * split_stride];
          const float v2 = p[(int64_t)(z + 2) * split_stride], v3 = p[(int64_t)(z + 3) * split_stride];
          if (grp < kExact)
            gi += (long long)__float2int_rn(v0) + __float2int_rn(v1) + __float2int_rn(v2) +
                  __float2int_rn(v3);
          else
            fa += (v0 + v1) + (v2 + v3);
        }
        for (; z < S; ++z) {
          const float v = p[(int64_t)z * split_stride];
          if (grp < kExact) gi += __float2int_rn(v);
          else fa += v;
        }
        if (grp < kExact) E += gi << (8 * (kExact - 1 - grp));
        else ap += fa;
      }
      const int64_t dst = rowmap ? (int64_t)rowmap[i] : i;
      C[dst * ldc + j] = oz_combine(E, ap, ex[i], ey[j]);
    }
}

// Few outputs with many partials each (a Gram matrix): one warp per element
// of C, the lanes over (slot, slice) pairs, then a warp reduction (64-bit
// integer for the exact groups, FP32 for the rounded one).
__global__ void __launch_bounds__(256)
k_oz_reduce_deep(const float *__restrict__ part, OzReduce rd, int S, int64_t slot_stride,
                 int64_t split_stride, int ldp, int64_t M, int ncols,
                 const int32_t *__restrict__ ex, const int32_t *__restrict__ ey,
                 double *__restrict__ C, int64_t ldc, const int32_t *__restrict__ rowmap,
                 const int *skip) {
  if (skip && ld_volatile_i32(skip) == 0) return;
  const int lane = threadIdx.x & 31;
  const int64_t nel = M * ncols, items = (int64_t)rd.nslots * S;
  for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < nel;
       e += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t i = e / ncols;
    const int j = (int)(e - i * ncols);
    long long E = 0;
    float ap = 0.f;
    for (int64_t it = lane; it < items; it += 32) {
      const int q = (int)(it / S), z = (int)(it - (int64_t)q * S);
      const float v = part[(int64_t)q * slot_stride + (int64_t)z * split_stride + i * ldp + j];
      const int grp = rd.group(q);
      if (grp < kExact) E += (long long)__float2int_rn(v) << (8 * (kExact - 1 - grp));
      else ap += v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      E += __shfl_xor_sync(0xffffffffu, E, o);
      ap += __shfl_xor_sync(0xffffffffu, ap, o);
    }
    if (lane == 0) {
      const int64_t dst = rowmap ? (int64_t)rowmap[i] : i;
      C[dst * ldc + j] = oz_combine(E, ap, ex[i], ey[j]);
    }
  }
}

// Digit arrays as a 3-D tensor map: K (inner), rows, digit planes `step`
// planes apart (an X operand may read the unscaled planes of a Y array).
bool make_map_3d(CUtensorMap *map, const void *base, int64_t planes, int64_t step, int64_t rows,
                 int64_t K, int64_t ld, int box_rows) {
  auto fn = tma_encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)(step * rows * ld * 2)};
  cuuint32_t box[3] = {(cuuint32_t)kTK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// The jobs (see the file comment): for X digit i the pairs (i, j) with
// t = i + j <= kS - 1; groups t < kExact get one exact accumulator each, the
// others share one rounded accumulator with E_j scaled by 2^(-8 (t - kExact)).
// A digit with more than kMaxAcc accumulators hands its rounded pairs to a
// job of their own (digit 0: four exact groups and the rounded rest).
int build_jobs(OzJob (&job)[kJobs], OzReduce &rd) {
  int nj = 0, slot = 0;
  auto open = [&](int i) -> OzJob & {
    OzJob &jb = job[nj++];
    jb = OzJob{};
    jb.xi = i;
    jb.slot0 = slot;
    return jb;
  };
  auto add = [&](OzJob &jb, int j, int t, int &approx) {
    int acc;
    if (t < kExact) {
      acc = jb.nacc++;
      jb.group[acc] = t;
    } else {
      if (approx < 0) {
        approx = jb.nacc++;
        jb.group[approx] = kExact;
      }
      acc = approx;
    }
    const int w = jb.nw++;
    jb.widx[w] = j * kC + (t < kExact ? 0 : t - kExact);
    jb.wacc[w] = acc;
    jb.first[w] = 1;
    for (int u = 0; u < w; ++u)
      if (jb.wacc[u] == acc) jb.first[w] = 0;
  };
  for (int i = 0; i < kS; ++i) {
    const int nexact = std::max(0, kExact - i), nround = (kS - i) - nexact;
    const bool separate = nexact + (nround > 0 ? 1 : 0) > kMaxAcc;
    OzJob *jb = &open(i);
    int approx = -1;
    for (int j = 0; i + j < kS; ++j) {
      const int t = i + j;
      if (t >= kExact && separate && approx < 0 && jb->nacc == nexact) {
        slot += jb->nacc;
        jb = &open(i);
      }
      add(*jb, j, t, approx);
    }
    slot += jb->nacc;
  }
  rd.nslots = 0;
  rd.groups = 0;
  for (int q = 0; q < nj; ++q)
    for (int u = 0; u < job[q].nacc; ++u)
      rd.groups |= (unsigned long long)job[q].group[u] << (3 * rd.nslots++);
  return nj;
}

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

struct OzPlan {
  int n_pad, nk, kb_per, S, stages;
  size_t smem;
};

OzPlan plan_oz(int64_t K, int N) {
  OzPlan p;
  p.n_pad = (int)round_up(N, 16);
  p.nk = (int)((K + kTK - 1) / kTK);
  p.kb_per = std::min(kKbExact, p.nk);
  p.S = (p.nk + p.kb_per - 1) / p.kb_per;
  const size_t stage = (size_t)kTM * kTK * 2 + (size_t)kMaxW * p.n_pad * kTK * 2;
  p.stages = (int)std::min<size_t>(kMaxStages, (kSmemLimit - 2048) / stage);
  // more than half of the shared memory: one CTA per SM, so that no CTA waits
  // in tcgen05.alloc for another's 512 TMEM columns
  p.smem = std::max<size_t>(p.stages * stage + 1024, 120 * 1024);
  return p;
}

}  // namespace

int ozaki_init() {
  static int done = 0;
  if (done) return RQLP_OK;
  if (!tma_encode_fn()) return RQLP_ERR_CUDA;
  if (cudaFuncSetAttribute(k_oz_mma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(kSmemLimit - 1024)) != cudaSuccess)
    return RQLP_ERR_CUDA;
  done = 1;
  return RQLP_OK;
}

size_t oz_operand_bytes(int64_t rows, int64_t K, int copies) {
  const int64_t ld = round_up(K, 8);
  return (size_t)kS * copies * rows * ld * 2;
}

OzOperand oz_carve(Arena &a, int64_t rows, int64_t K, int copies) {
  OzOperand op;
  op.rows = rows;
  op.K = K;
  op.ld = round_up(K, 8);
  op.copies = copies;
  op.digits = a.take<uint8_t>(oz_operand_bytes(rows, K, copies));
  op.exps = a.take<int32_t>((size_t)rows);
  return op;
}

size_t oz_part_floats(int64_t M, int N, int64_t K) {
  const OzPlan p = plan_oz(K, N);
  return (size_t)kSlots * p.S * round_up(M, kTM) * p.n_pad;
}

int oz_split(const void *S, int dtype, int64_t r, int64_t c, int64_t ld, bool trans,
             const OzOperand &op, Ctrl *ctrl, const int *skip, cudaStream_t st) {
  const int64_t rows = trans ? c : r, K = trans ? r : c;
  if (op.rows != rows || op.K != K || op.ld < K || op.ld % 8 != 0) return RQLP_ERR_INVALID_ARG;
  const int copies = op.copies;
  auto *dig = static_cast<uint16_t *>(op.digits);
  const bool f32 = dtype == RQLP_F32;
  const int sms = num_sms();
  if (!trans) {
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((r + 7) / 8, 8LL * sms));
    if (f32)
      k_oz_exp_rows<float><<<blocks, 256, 0, st>>>(static_cast<const float *>(S), r, c, ld, op.exps, ctrl, skip);
    else
      k_oz_exp_rows<double><<<blocks, 256, 0, st>>>(static_cast<const double *>(S), r, c, ld, op.exps, ctrl, skip);
    count_launch();
    const dim3 g((unsigned)std::max<int64_t>(1, std::min<int64_t>((c + 63) / 64, 64)),
                 (unsigned)std::max<int64_t>(1, std::min<int64_t>((r + 7) / 8, 16LL * sms)));
    if (f32)
      k_oz_digits<float><<<g, dim3(32, 8), 0, st>>>(static_cast<const float *>(S), r, c, ld, op.exps,
                                                     dig, op.ld, copies, skip);
    else
      k_oz_digits<double><<<g, dim3(32, 8), 0, st>>>(static_cast<const double *>(S), r, c, ld,
                                                      op.exps, dig, op.ld, copies, skip);
    count_launch();
  } else {
    if (cudaMemsetAsync(op.exps, 0x80, (size_t)c * sizeof(int32_t), st) != cudaSuccess)
      return RQLP_ERR_CUDA;
    const dim3 ge((unsigned)((c + 31) / 32),
                  (unsigned)std::max<int64_t>(1, std::min<int64_t>((r + 63) / 64, 256)));
    if (f32)
      k_oz_exp_cols<float><<<ge, dim3(32, 8), 0, st>>>(static_cast<const float *>(S), r, c, ld, op.exps, ctrl, skip);
    else
      k_oz_exp_cols<double><<<ge, dim3(32, 8), 0, st>>>(static_cast<const double *>(S), r, c, ld, op.exps, ctrl, skip);
    count_launch();
    const dim3 g((unsigned)((c + 31) / 32),
                 (unsigned)std::max<int64_t>(1, std::min<int64_t>((r + 31) / 32, 8LL * sms)));
    if (f32)
      k_oz_digits_t<float><<<g, dim3(32, 8), 0, st>>>(static_cast<const float *>(S), r, c, ld,
                                                       op.exps, dig, op.ld, copies, skip);
    else
      k_oz_digits_t<double><<<g, dim3(32, 8), 0, st>>>(static_cast<const double *>(S), r, c, ld,
                                                        op.exps, dig, op.ld, copies, skip);
    count_launch();
  }
  return cudaGetLastError() == cudaSuccess ? RQLP_OK : RQLP_ERR_CUDA;
}

int oz_split_both(const void *S, int dtype, int64_t r, int64_t c, int64_t ld,
                  const OzOperand &rows, const OzOperand &cols, Ctrl *ctrl, cudaStream_t st) {
  if (rows.rows != r || rows.K != c || cols.rows != c || cols.K != r || rows.copies != 1 ||
      cols.copies != 1)
    return RQLP_ERR_INVALID_ARG;
  if (cudaMemsetAsync(cols.exps, 0x80, (size_t)c * sizeof(int32_t), st) != cudaSuccess ||
      cudaMemsetAsync(rows.exps, 0x80, (size_t)r * sizeof(int32_t), st) != cudaSuccess)
    return RQLP_ERR_CUDA;
  const bool f32 = dtype == RQLP_F32;
  const dim3 ge((unsigned)((c + 127) / 128), (unsigned)((r + 31) / 32));
  if (f32)
    k_oz_exps_both<float><<<ge, 256, 0, st>>>(static_cast<const float *>(S), r, c, ld, rows.exps,
                                              cols.exps, ctrl);
  else
    k_oz_exps_both<double><<<ge, 256, 0, st>>>(static_cast<const double *>(S), r, c, ld, rows.exps,
                                               cols.exps, ctrl);
  count_launch();
  const dim3 g((unsigned)((c + 31) / 32), (unsigned)((r + 31) / 32));
  auto *dr = static_cast<uint16_t *>(rows.digits);
  auto *dc = static_cast<uint16_t *>(cols.digits);
  if (f32)
    k_oz_digits_both<float><<<g, dim3(32, 8), 0, st>>>(static_cast<const float *>(S), r, c, ld,
                                                        rows.exps, cols.exps, dr, rows.ld, dc,
                                                        cols.ld);
  else
    k_oz_digits_both<double><<<g, dim3(32, 8), 0, st>>>(static_cast<const double *>(S), r, c, ld,
                                                         rows.exps, cols.exps, dr, rows.ld, dc,
                                                         cols.ld);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? RQLP_OK : RQLP_ERR_CUDA;
}

int oz_gemm(const OzOperand &X, const OzOperand &Y, int64_t M, int N, int64_t K, double *C,
            int64_t ldc, const int32_t *rowmap, float *part, int64_t part_floats, Ctrl *ctrl,
            int64_t spin_ns, const int *skip, cudaStream_t st) {
  if (N < 1 || N > 128 || M < 1 || K < 1 || X.rows != M || Y.rows != N || X.K != K || Y.K != K)
    return RQLP_ERR_INVALID_ARG;
  const OzPlan pl = plan_oz(K, N);
  if (pl.stages < 2) return RQLP_ERR_UNSUPPORTED;
  const int64_t Mp = round_up(M, kTM);
  if ((int64_t)oz_part_floats(M, N, K) > part_floats) return RQLP_ERR_WORKSPACE;
  if (ozaki_init() != RQLP_OK) return RQLP_ERR_CUDA;
  CUtensorMap mX, mY;
  if (Y.copies != kC) return RQLP_ERR_INVALID_ARG;
  if (!make_map_3d(&mX, X.digits, kS, X.copies, M, K, X.ld, kTM) ||
      !make_map_3d(&mY, Y.digits, kS * kC, 1, N, K, Y.ld, pl.n_pad))
    return RQLP_ERR_CUDA;
  OzArgs a;
  std::memset(&a, 0, sizeof(a));
  OzReduce rd;
  a.njobs = build_jobs(a.job, rd);
  a.M = (int)M;
  a.n_pad = pl.n_pad;
  a.ncols = N;
  a.nk = pl.nk;
  a.kb_per = pl.kb_per;
  a.stages = pl.stages;
  a.acc_cols = 128;
  a.tmem_cols = 512;
  a.part = part;
  a.ldp = pl.n_pad;
  a.split_stride = Mp * pl.n_pad;
  a.slot_stride = (int64_t)pl.S * a.split_stride;
  a.ctrl = ctrl;
  a.limit_ns = spin_ns > 0 ? (unsigned long long)spin_ns : kDefaultSpinNs;
  a.skip = skip;
  const dim3 grid((unsigned)a.njobs, (unsigned)(Mp / kTM), (unsigned)pl.S);
  k_oz_mma<<<grid, 128, pl.smem, st>>>(mX, mY, a);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return RQLP_ERR_CUDA;
  if (M * N < 32768) {
    // few outputs: a warp per element over its (slot, slice) partials
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((M * N + 7) / 8, 16LL * num_sms()));
    k_oz_reduce_deep<<<blocks, 256, 0, st>>>(part, rd, pl.S, a.slot_stride, a.split_stride, a.ldp,
                                              M, N, X.exps, Y.exps, C, ldc, rowmap, skip);
  } else {
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((M + 7) / 8, 8LL * num_sms()));
    k_oz_reduce<<<blocks, dim3(32, 8), 0, st>>>(part, rd, pl.S, a.slot_stride, a.split_stride,
                                                 a.ldp, M, N, X.exps, Y.exps, C, ldc, rowmap, skip);
  }
  count_launch();
  return cudaGetLastError() == cudaSuccess ? RQLP_OK : RQLP_ERR_CUDA;
}

}  // namespace rqk
