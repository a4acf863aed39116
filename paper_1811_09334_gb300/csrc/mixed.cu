// Mixed-precision products with A on the 5th-generation tensor cores.
//
// The sketch Y = A W, the power-step product Z = A^T V and the projection
// B^T = A^T V (Algorithm 2.1 steps 2 and 4) are the only O(m n l) work of
// the method.  In the BF16x3 form A and the skinny operand are split into
// BF16 pairs, A = Ah + Al and W = Wh + Wl, and three products
// Ah Wh + Ah Wl + Al Wh are accumulated in FP32 (the dropped Al Wl term is
// about 2^-16 of the result); the BF16 form keeps Ah Wh only.
//
// Both products are computed as C[M x N] = X[M x K] Y[N x K]^T with X and Y
// K-major BF16: X = A (M = m, K = n) for the sketch and X = A^T (M = n,
// K = m) for the projection, so A is split once per factorization into
// row- and column-major BF16 copies (a1, one HBM pass).  One CTA owns a
// 128-row tile of C and a slice of K:
//   warp 0 lane 0  TMA producer: 128B-swizzled 128 x 64 tiles of Xh, Xl and
//                  N x 64 tiles of Yh, Yl into a ring of shared-memory stages;
//   warp 1 lane 0  MMA issuer: tcgen05.mma kind::f16, M = 128, N = l padded
//                  to 16, K = 16, FP32 accumulator in TMEM; tcgen05.commit
//                  releases each stage;
//   warps 0-3      epilogue: tcgen05.ld of the accumulator, FP32 partial
//                  sums to global memory (split-K slices are summed in FP64
//                  by a second kernel).
// Every mbarrier wait is bounded; a wait that gives up records
// RQLP_ERR_TIMEOUT, waits (bounded) for its own copies in flight, frees the
// TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "mixed.cuh"
#include "tc.cuh"

namespace rqk {

int mixed_init();

// The driver's tensor-map encoder, reached through the runtime once.
PFN_cuTensorMapEncodeTiled_v12000 tma_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

namespace {

using namespace tc;

constexpr int kTileM = 128;
constexpr int kTileK = 64;                // 64 BF16 = one 128-byte swizzle row
constexpr uint32_t kXBytes = kTileM * kTileK * 2;
constexpr int kMaxStages = 5;  // ring stages: 4 for 128-byte K tiles, up to 5 for 64-byte ones
constexpr size_t kSmemLimit = 227 * 1024;

struct MmaArgs {
  int M;           // rows of C (rows of X)
  int n_pad;       // MMA N (multiple of 16)
  int ncols;       // columns of C that are stored (l)
  int nk;          // K blocks in total
  int kb_per;      // K blocks per split
  int stages;
  uint32_t tmem_cols;
  int nacc;        // accumulators in TMEM, k-block i into number i mod nacc
  int acc_cols;    // TMEM columns between two accumulators
  float *part;     // [split][M][ldp]
  int64_t split_stride;
  int ldp;
  Ctrl *ctrl;
  unsigned long long limit_ns;
};

// SPLIT: three products of the hi/lo pairs; FP8: one E4M3 product with 128
// values per 128-byte K row (K tile of 128 elements instead of 64); TF32:
// FP32 storage read as TF32, 32 values per 128-byte K row.  Every MMA
// consumes 32 bytes of each K row (16 BF16, 8 TF32 or 32 E4M3 values).
template <bool SPLIT, bool FP8 = false, bool TF32 = false, bool SW64 = false>
__global__ void __launch_bounds__(128, 1)
k_mma_bf16(const __grid_constant__ CUtensorMap tXh, const __grid_constant__ CUtensorMap tXl,
           const __grid_constant__ CUtensorMap tYh, const __grid_constant__ CUtensorMap tYl,
           const MmaArgs a) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bar_full[kMaxStages], bar_empty[kMaxStages], bar_acc;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t *smem = reinterpret_cast<uint8_t *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  // SW64 (BF16 only): K tiles of 32 elements in the 64-byte swizzle, half the
  // bytes per stage, so that a wide skinny operand still leaves room for
  // several stages
  constexpr int KT = FP8 ? 128 : TF32 ? 32 : SW64 ? 32 : kTileK;  // K elements per stage
  constexpr uint32_t kXB = SW64 ? kXBytes / 2 : kXBytes;
  constexpr uint32_t kRowB = SW64 ? 64u : 128u;  // bytes of one K row of a tile
  constexpr int kSteps = SW64 ? 2 : 4;           // MMAs of K = 32 bytes per stage
  const uint32_t ybytes = (uint32_t)a.n_pad * kRowB;
  const uint32_t stage_bytes = (SPLIT ? 2u : 1u) * (kXB + ybytes);
  const int m_tile = blockIdx.x, split = blockIdx.y;
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
      // ---- TMA producer ----
      int issued = 0;
      for (int i = 0; i < nkb; ++i) {
        const int s = i % a.stages;
        const uint32_t ph = (uint32_t)(i / a.stages) & 1u;
        if (!mbar_wait(&bar_empty[s], ph ^ 1u, a.limit_ns) || *(volatile int *)&s_abort) {
          s_abort = 1;
          break;
        }
        const uint32_t st = smem_u32(smem + (size_t)s * stage_bytes);
        mbar_expect_tx(&bar_full[s], stage_bytes);
        const int kx = (kb0 + i) * KT, my = m_tile * kTileM;
        tma_load_2d(st, &tXh, kx, my, &bar_full[s]);
        tma_load_2d(st + kXB, &tYh, kx, 0, &bar_full[s]);
        if (SPLIT) {
          tma_load_2d(st + kXB + ybytes, &tXl, kx, my, &bar_full[s]);
          tma_load_2d(st + 2 * kXB + ybytes, &tYl, kx, 0, &bar_full[s]);
        }
        issued = i + 1;
      }
      // never leave with copies in flight: wait for the last load of each stage
      for (int s = 0; s < a.stages && s < issued; ++s) {
        const int last = ((issued - 1 - s) / a.stages) * a.stages + s;
        mbar_wait(&bar_full[s], (uint32_t)(last / a.stages) & 1u, a.limit_ns);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer ----
      const uint32_t idesc = instr_desc(kTileM, a.n_pad, FP8, TF32);
      for (int i = 0; i < nkb; ++i) {
        const int s = i % a.stages;
        const uint32_t ph = (uint32_t)(i / a.stages) & 1u;
        if (!mbar_wait(&bar_full[s], ph, a.limit_ns) || *(volatile int *)&s_abort) {
          s_abort = 1;
          break;
        }
        tc_fence_after();
        const uint32_t xh = smem_u32(smem + (size_t)s * stage_bytes);
        const uint32_t yh = xh + kXB;
        const uint32_t xl = yh + ybytes;
        const uint32_t yl = xl + kXB;
        // the accumulator of this k-block; its first k-block overwrites it
        const uint32_t td = tmem + (uint32_t)((i % a.nacc) * a.acc_cols);
        const uint32_t first = (i < a.nacc) ? 1u : 0u;
#pragma unroll
        for (int k = 0; k < kSteps; ++k) {
          // 32 bytes along K inside the swizzled row: 16 BF16, 8 TF32 or 32 FP8 values
          const uint32_t off = k * 32;
          const uint32_t accum = (first && k == 0) ? 0u : 1u;
          if (FP8) {
            mma_fp8(td, smem_desc(xh + off), smem_desc(yh + off), idesc, accum);
            continue;
          }
          if (TF32) {
            mma_tf32(td, smem_desc(xh + off), smem_desc(yh + off), idesc, accum);
            if (SPLIT) {
              mma_tf32(td, smem_desc(xh + off), smem_desc(yl + off), idesc, 1u);
              mma_tf32(td, smem_desc(xl + off), smem_desc(yh + off), idesc, 1u);
            }
            continue;
          }
          if (SW64) {
            mma_bf16(td, smem_desc_sw64(xh + off), smem_desc_sw64(yh + off), idesc, accum);
            if (SPLIT) {
              mma_bf16(td, smem_desc_sw64(xh + off), smem_desc_sw64(yl + off), idesc, 1u);
              mma_bf16(td, smem_desc_sw64(xl + off), smem_desc_sw64(yh + off), idesc, 1u);
            }
            continue;
          }
          mma_bf16(td, smem_desc(xh + off), smem_desc(yh + off), idesc, accum);
          if (SPLIT) {
            mma_bf16(td, smem_desc(xh + off), smem_desc(yl + off), idesc, 1u);
            mma_bf16(td, smem_desc(xl + off), smem_desc(yh + off), idesc, 1u);
          }
        }
        mma_commit(&bar_empty[s]);
      }
      // arrives once every MMA issued above has completed (also on the abort path)
      mma_commit(&bar_acc);
    }
    __syncwarp();
  }

  // ---- epilogue: TMEM -> FP32 partial sums ----
  const bool ready = mbar_wait(&bar_acc, 0, a.limit_ns);
  tc_fence_after();
  __syncthreads();
  if (!ready || *(volatile int *)&s_abort) {
    if (tid == 0) set_status(a.ctrl, RQLP_ERR_TIMEOUT);
  } else {
    const int row = m_tile * kTileM + warp * 32 + lane;
    float *out = a.part + (int64_t)split * a.split_stride + (int64_t)row * a.ldp;
    const int used = min(a.nacc, nkb);  // accumulators that received a k-block
    for (int c0 = 0; c0 < a.n_pad; c0 += 16) {
      float v[16];
      uint32_t r[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
      for (int q = 1; q < used; ++q) {
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(q * a.acc_cols + c0), r);
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] += __uint_as_float(r[j]);
      }
      if (row < a.M) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j < a.ncols) out[c0 + j] = v[j];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, a.tmem_cols);
}

// C (M x ncols, FP64, ldc) = sum of S FP32 partial slices, divided by the
// row and column scales of a scaled (FP8) product when they are given.
// (32, 8) blocks: lanes along a row of C, warps over rows.
__global__ void k_sum_parts_f32(const float *__restrict__ part, int S, int64_t split_stride,
                                int64_t M, int ncols, int ldp, double *__restrict__ C,
                                int64_t ldc, const float *__restrict__ rscale,
                                const float *__restrict__ cscale) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; i < M;
       i += (int64_t)gridDim.x * blockDim.y)
    for (int j = threadIdx.x; j < ncols; j += blockDim.x) {
      double s = 0.0;
      for (int z = 0; z < S; ++z) s += f2d(part[(int64_t)z * split_stride + i * ldp + j]);
      if (rscale) s /= f2d(rscale[i]) * f2d(cscale[j]);
      C[i * ldc + j] = s;
    }
}

// Per-row maxima of |A| and per-column maxima (one atomic max per column and
// CTA, on the bit patterns of non-negative floats).  CTA = 32 rows.
template <typename T>
__global__ void __launch_bounds__(256)
k_absmax(const T *__restrict__ A, int64_t m, int64_t n, int64_t lda, float *__restrict__ rmax,
         unsigned *__restrict__ cmax_bits) {
  __shared__ float red[32][9];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int nr = (int)min((int64_t)32, m - i0);
  float rmx[32];
#pragma unroll
  for (int r = 0; r < 32; ++r) rmx[r] = 0.f;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    float cm = 0.f;
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      if (r < nr) {
        const float v = fabsf(as_f32(A[(i0 + r) * lda + j]));
        cm = fmaxf(cm, v);
        rmx[r] = fmaxf(rmx[r], v);
      }
    }
    atomicMax(cmax_bits + j, __float_as_uint(cm));
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    float v = rmx[r];
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) red[r][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < nr) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[threadIdx.x][w]);
    rmax[i0 + threadIdx.x] = t;
  }
}

// Power-of-two scale putting the largest magnitude at or below 448 (E4M3 max).
__device__ __forceinline__ float e4m3_scale(float amax) {
  if (!(amax > 0.f) || !isfinite(amax)) return 1.f;
  return exp2f(floorf(log2f(448.f / amax)));
}

__global__ void k_scales(const float *__restrict__ rmax, int64_t m,
                         const unsigned *__restrict__ cmax_bits, int64_t n, float *rscale,
                         float *cscale) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m + n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (i < m) rscale[i] = e4m3_scale(rmax[i]);
    else cscale[i - m] = e4m3_scale(__uint_as_float(cmax_bits[i - m]));
  }
}

// A -> E4M3 row-scaled (m x ld1) and E4M3 column-scaled transpose (n x ld2).
template <typename T>
__global__ void __launch_bounds__(256)
k_quant_a(const T *__restrict__ A, int64_t m, int64_t n, int64_t lda, const float *rscale,
          const float *cscale, __nv_fp8_storage_t *A8, int64_t ld1, __nv_fp8_storage_t *At8,
          int64_t ld2) {
  __shared__ __nv_fp8_storage_t t[32][36];
  const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int k = ty; k < 32; k += 8) {
    const int64_t i = i0 + k, j = j0 + tx;
    if (i < m && j < n) {
      const float v = as_f32(A[i * lda + j]);
      A8[i * ld1 + j] = __nv_cvt_float_to_fp8(v * rscale[i], __NV_SATFINITE, __NV_E4M3);
      t[k][tx] = __nv_cvt_float_to_fp8(v * cscale[j], __NV_SATFINITE, __NV_E4M3);
    }
  }
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const int64_t j = j0 + k, i = i0 + tx;
    if (i < m && j < n) At8[j * ld2 + i] = t[tx][k];
  }
}

// S (K x l, FP64) -> S^T as E4M3 (l x ldk) with one scale per column of S;
// one CTA per column.
__global__ void k_quant_skinny_t(const double *__restrict__ S, int64_t K, int l, int64_t lds,
                                 __nv_fp8_storage_t *S8, int64_t ldk, float *scale) {
  __shared__ float red[32];
  __shared__ float s_sc;
  for (int c = blockIdx.x; c < l; c += gridDim.x) {
    float mx = 0.f;
    for (int64_t k = threadIdx.x; k < K; k += blockDim.x) mx = fmaxf(mx, fabsf(d2f_rn(S[k * lds + c])));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
      s_sc = e4m3_scale(t);
      scale[c] = s_sc;
    }
    __syncthreads();
    const float sc = s_sc;
    for (int64_t k = threadIdx.x; k < K; k += blockDim.x)
      S8[(int64_t)c * ldk + k] = __nv_cvt_float_to_fp8(d2f_rn(S[k * lds + c]) * sc, __NV_SATFINITE,
                                                       __NV_E4M3);
    __syncthreads();
  }
}

// A (m x n, lda) -> Ah, Al (m x ld1) and A^T halves Ath, Atl (n x ld2), BF16.
// Tile of 32 rows x 64 columns per CTA; each thread loads two neighbouring
// elements and stores BF16 pairs, the transposed halves go through shared
// memory.  One HBM pass: read A once, write the four BF16 arrays.
template <typename T>
__global__ void __launch_bounds__(256)
k_split_a(const T *__restrict__ A, int64_t m, int64_t n, int64_t lda, __nv_bfloat16 *Ah,
          __nv_bfloat16 *Al, int64_t ld1, __nv_bfloat16 *Ath, __nv_bfloat16 *Atl, int64_t ld2,
          int with_lo) {
  __shared__ __nv_bfloat16 th[64][34];
  __shared__ __nv_bfloat16 tl[64][34];
  const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 64;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const bool vec = ((lda & 1) == 0) && ((ld1 & 1) == 0) &&
                   ((reinterpret_cast<uintptr_t>(A) & (2 * sizeof(T) - 1)) == 0);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int r = ty + 8 * k;
    const int64_t i = i0 + r, j = j0 + 2 * tx;
    // one FP64 -> FP32 rounding per element, the split
    // in FP32 (FP64 arithmetic runs at 2 operations per clock per SM on this
    // part): f - h is exact in FP32, and the FP32 rounding of v (2^-24) is far
    // below the precision of the pair (about 2^-17)
    float f0 = 0.0f, f1 = 0.0f;
    if (i < m) {
      if (vec && j + 1 < n) {
        if (sizeof(T) == 8) {
          const double2 p = *reinterpret_cast<const double2 *>(A + i * lda + j);
          f0 = (float)p.x;
          f1 = (float)p.y;
        } else {
          const float2 p = *reinterpret_cast<const float2 *>(A + i * lda + j);
          f0 = p.x;
          f1 = p.y;
        }
      } else {
        if (j < n) f0 = as_f32(A[i * lda + j]);
        if (j + 1 < n) f1 = as_f32(A[i * lda + j + 1]);
      }
    }
    const __nv_bfloat16 h0 = __float2bfloat16_rn(f0), h1 = __float2bfloat16_rn(f1);
    const __nv_bfloat16 l0 = __float2bfloat16_rn(f0 - __bfloat162float(h0));
    const __nv_bfloat16 l1 = __float2bfloat16_rn(f1 - __bfloat162float(h1));
    if (i < m) {
      if (vec && j + 1 < n) {
        *reinterpret_cast<__nv_bfloat162 *>(Ah + i * ld1 + j) = __halves2bfloat162(h0, h1);
        if (with_lo) *reinterpret_cast<__nv_bfloat162 *>(Al + i * ld1 + j) = __halves2bfloat162(l0, l1);
      } else {
        if (j < n) {
          Ah[i * ld1 + j] = h0;
          if (with_lo) Al[i * ld1 + j] = l0;
        }
        if (j + 1 < n) {
          Ah[i * ld1 + j + 1] = h1;
          if (with_lo) Al[i * ld1 + j + 1] = l1;
        }
      }
    }
    th[2 * tx][r] = h0;
    th[2 * tx + 1][r] = h1;
    tl[2 * tx][r] = l0;
    tl[2 * tx + 1][r] = l1;
  }
  __syncthreads();
  // transposed: 64 rows (j) x 32 columns (i); a thread writes a BF16 pair of i
  const bool tvec = ((ld2 & 1) == 0);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int jr = (ty + 8 * k) * 2 + (tx >> 4);  // 0..63
    const int ic = (tx & 15) * 2;                 // 0..30
    const int64_t j = j0 + jr, i = i0 + ic;
    if (j >= n || i >= m) continue;
    if (tvec && i + 1 < m) {
      *reinterpret_cast<__nv_bfloat162 *>(Ath + j * ld2 + i) = __halves2bfloat162(th[jr][ic], th[jr][ic + 1]);
      if (with_lo)
        *reinterpret_cast<__nv_bfloat162 *>(Atl + j * ld2 + i) = __halves2bfloat162(tl[jr][ic], tl[jr][ic + 1]);
    } else {
      Ath[j * ld2 + i] = th[jr][ic];
      if (with_lo) Atl[j * ld2 + i] = tl[jr][ic];
      if (i + 1 < m) {
        Ath[j * ld2 + i + 1] = th[jr][ic + 1];
        if (with_lo) Atl[j * ld2 + i + 1] = tl[jr][ic + 1];
      }
    }
  }
}

// S (K x l, FP64, lds) -> S^T halves (l x ldk, BF16).  32 x 32 tiles on
// (32, 8) blocks through shared memory: rows of S are read and rows of S^T
// written along the lanes (both coalesced); blockIdx.x over column tiles of
// S, blockIdx.y over row tiles.
__global__ void k_split_skinny_t(const double *__restrict__ S, int64_t K, int l, int64_t lds,
                                 __nv_bfloat16 *Sh, __nv_bfloat16 *Sl, int64_t ldk, int with_lo) {
  __shared__ __nv_bfloat16 th[32][34], tl[32][34];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int c0 = blockIdx.x * 32;
  for (int64_t k0 = (int64_t)blockIdx.y * 32; k0 < K; k0 += (int64_t)gridDim.y * 32) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int kr = ty + 8 * q;
      const int64_t k = k0 + kr;
      const int c = c0 + tx;
      // the pair split in FP32, as for A
      const float f = (k < K && c < l) ? d2f_rn(S[k * lds + c]) : 0.0f;
      const __nv_bfloat16 h = __float2bfloat16_rn(f);
      th[kr][tx] = h;
      tl[kr][tx] = __float2bfloat16_rn(f - __bfloat162float(h));
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = c0 + ty + 8 * q;
      const int64_t k = k0 + tx;
      if (c < l && k < K) {
        Sh[(int64_t)c * ldk + k] = th[tx][ty + 8 * q];
        if (with_lo) Sl[(int64_t)c * ldk + k] = tl[tx][ty + 8 * q];
      }
    }
    __syncthreads();
  }
}

// FP32 -> TF32 (10-bit significand), round to nearest (ties away from zero);
// the result is an FP32 value whose low 13 significand bits are zero
__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// A (m x n, lda) -> TF32 pairs Ah, Al (m x ld1) and A^T pairs Ath, Atl
// (n x ld2), FP32 storage.  32 x 32 tiles on (32, 8) blocks; the transposed
// pairs go through shared memory.  h = tf32(f), l = tf32(f - h) with f the
// FP32 rounding of A: f - h is exact in FP32, and the pair holds about 22
// significand bits.
template <typename T>
__global__ void __launch_bounds__(256)
k_split_a_tf32(const T *__restrict__ A, int64_t m, int64_t n, int64_t lda, float *Ah, float *Al,
               int64_t ld1, float *Ath, float *Atl, int64_t ld2, int with_lo) {
  __shared__ float th[32][33], tl[32][33];
  const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int r = ty + 8 * k;
    const int64_t i = i0 + r, j = j0 + tx;
    const float f = (i < m && j < n) ? as_f32(A[i * lda + j]) : 0.0f;
    const float h = tf32_rn(f), lo = tf32_rn(f - h);
    if (i < m && j < n) {
      Ah[i * ld1 + j] = h;
      if (with_lo) Al[i * ld1 + j] = lo;
    }
    th[tx][r] = h;
    tl[tx][r] = lo;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int jr = ty + 8 * k;
    const int64_t j = j0 + jr, i = i0 + tx;
    if (j < n && i < m) {
      Ath[j * ld2 + i] = th[jr][tx];
      if (with_lo) Atl[j * ld2 + i] = tl[jr][tx];
    }
  }
}

// S (K x l, FP64, lds) -> S^T TF32 pairs (l x ldk, FP32 storage), tiled as
// k_split_skinny_t
__global__ void k_split_skinny_tf32_t(const double *__restrict__ S, int64_t K, int l, int64_t lds,
                                      float *Sh, float *Sl, int64_t ldk, int with_lo) {
  __shared__ float th[32][33], tl[32][33];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int c0 = blockIdx.x * 32;
  for (int64_t k0 = (int64_t)blockIdx.y * 32; k0 < K; k0 += (int64_t)gridDim.y * 32) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int kr = ty + 8 * q;
      const int64_t k = k0 + kr;
      const int c = c0 + tx;
      const float f = (k < K && c < l) ? d2f_rn(S[k * lds + c]) : 0.0f;
      const float h = tf32_rn(f);
      th[kr][tx] = h;
      tl[kr][tx] = tf32_rn(f - h);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = c0 + ty + 8 * q;
      const int64_t k = k0 + tx;
      if (c < l && k < K) {
        Sh[(int64_t)c * ldk + k] = th[tx][ty + 8 * q];
        if (with_lo) Sl[(int64_t)c * ldk + k] = tl[tx][ty + 8 * q];
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() { return tma_encode_fn(); }

// 2-D tensor map of BF16, E4M3 (fp8) or FP32 (tf32) elements: `rows` x `cols`
// (cols contiguous, ld elements per row), box of box_rows x (128 bytes) with
// the 128-byte swizzle.
bool make_map(CUtensorMap *map, const void *base, int64_t rows, int64_t cols, int64_t ld,
              int box_rows, bool fp8 = false, bool tf32 = false, bool sw64 = false) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int es = fp8 ? 1 : tf32 ? 4 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * es};
  cuuint32_t box[2] = {(cuuint32_t)((sw64 ? 64 : 128) / es), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = fp8    ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                 : tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                        : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  CUresult r = fn(map, dt, 2,
                  const_cast<void *>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  sw64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

struct GemmPlan {
  int n_pad, stages, S, kb_per, nk;
  bool sw64;  // BF16 tiles of 32 K elements in the 64-byte swizzle
  uint32_t tmem_cols;
  size_t smem;
};

GemmPlan plan_gemm(int64_t M, int64_t K, int l, bool split, bool fp8 = false,
                   bool tf32 = false) {
  GemmPlan g;
  g.n_pad = (int)round_up(l, 16);
  size_t ybytes = (size_t)g.n_pad * 128;
  size_t stage = (split ? 2 : 1) * (kXBytes + ybytes);
  g.stages = (int)std::min<size_t>(4, (kSmemLimit - 2048) / stage);
  // a wide skinny operand (the BF16 pair at l > 128) leaves room for two
  // 128-byte stages only: take K tiles of 32 in the 64-byte swizzle instead
  g.sw64 = !fp8 && !tf32 && g.stages < 3;
  if (g.sw64) {
    ybytes = (size_t)g.n_pad * 64;
    stage = (split ? 2 : 1) * (kXBytes / 2 + ybytes);
    g.stages = (int)std::min<size_t>(kMaxStages, (kSmemLimit - 2048) / stage);
  }
  g.smem = g.stages * stage + 1024;
  const int kt = fp8 ? 128 : tf32 ? 32 : g.sw64 ? 32 : kTileK;
  g.nk = (int)((K + kt - 1) / kt);
  const int64_t tiles = (M + kTileM - 1) / kTileM;
  int S = (int)std::max<int64_t>(1, num_sms() / tiles);
  S = std::min(S, std::max(1, g.nk / 4));
  if (tuning().mma_max_splits > 0) S = std::min(S, tuning().mma_max_splits);
  g.kb_per = (g.nk + S - 1) / S;
  g.S = (g.nk + g.kb_per - 1) / g.kb_per;
  g.tmem_cols = g.n_pad <= 32 ? 32 : g.n_pad <= 64 ? 64 : g.n_pad <= 128 ? 128 : 256;
  return g;
}

// C (M x l, FP64, ld l) = X Y^T with X (M x K) and Y (l x K) given as BF16
// pairs (or E4M3 with row scales of X and of Y) with leading dimensions ldx / ldy.
int gemm_xyt(const MixedBufs &mx, bool split, int64_t M, int64_t K, int l, const void *Xh,
             const void *Xl, int64_t ldx, const void *Yh, const void *Yl, int64_t ldy, double *C,
             Ctrl *ctrl, int64_t spin_ns, cudaStream_t st, bool fp8 = false,
             const float *xscale = nullptr, const float *yscale = nullptr, bool tf32 = false) {
  GemmPlan g = plan_gemm(M, K, l, split, fp8, tf32);
  if (g.stages < 2) return RQLP_ERR_UNSUPPORTED;
  if ((int64_t)g.S * M * g.n_pad > mx.part_floats) return RQLP_ERR_WORKSPACE;
  CUtensorMap mXh, mXl, mYh, mYl;
  if (!make_map(&mXh, Xh, M, K, ldx, kTileM, fp8, tf32, g.sw64) ||
      !make_map(&mYh, Yh, l, K, ldy, g.n_pad, fp8, tf32, g.sw64))
    return RQLP_ERR_CUDA;
  if (split) {
    if (!make_map(&mXl, Xl, M, K, ldx, kTileM, false, tf32, g.sw64) ||
        !make_map(&mYl, Yl, l, K, ldy, g.n_pad, false, tf32, g.sw64))
      return RQLP_ERR_CUDA;
  } else {
    mXl = mXh;
    mYl = mYh;
  }
  MmaArgs a;
  a.M = (int)M;
  a.n_pad = g.n_pad;
  a.ncols = l;
  a.nk = g.nk;
  a.kb_per = g.kb_per;
  a.stages = g.stages;
  // TF32 forms: up to four accumulators (at most 512 TMEM columns), each
  // taking every fourth k-block, so that every FP32 accumulation chain in
  // the tensor cores is four times shorter (its error, about 2^-24 per MMA
  // of 8 values, otherwise bounds the TF32x3 product)
  a.nacc = tf32 ? (int)std::min<uint32_t>(4u, 512u / g.tmem_cols) : 1;
  a.acc_cols = (int)g.tmem_cols;
  a.tmem_cols = g.tmem_cols * (uint32_t)a.nacc;
  a.part = mx.part;
  a.ldp = g.n_pad;
  a.split_stride = M * g.n_pad;
  a.ctrl = ctrl;
  a.limit_ns = spin_ns > 0 ? (unsigned long long)spin_ns : kDefaultSpinNs;
  dim3 grid((unsigned)((M + kTileM - 1) / kTileM), (unsigned)g.S);
  if (mixed_init() != RQLP_OK) return RQLP_ERR_CUDA;
  if (fp8) k_mma_bf16<false, true><<<grid, 128, g.smem, st>>>(mXh, mXl, mYh, mYl, a);
  else if (tf32 && split) k_mma_bf16<true, false, true><<<grid, 128, g.smem, st>>>(mXh, mXl, mYh, mYl, a);
  else if (tf32) k_mma_bf16<false, false, true><<<grid, 128, g.smem, st>>>(mXh, mXl, mYh, mYl, a);
  else if (split && g.sw64) k_mma_bf16<true, false, false, true><<<grid, 128, g.smem, st>>>(mXh, mXl, mYh, mYl, a);
  else if (g.sw64) k_mma_bf16<false, false, false, true><<<grid, 128, g.smem, st>>>(mXh, mXl, mYh, mYl, a);
  else if (split) k_mma_bf16<true><<<grid, 128, g.smem, st>>>(mXh, mXl, mYh, mYl, a);
  else k_mma_bf16<false><<<grid, 128, g.smem, st>>>(mXh, mXl, mYh, mYl, a);
  count_launch();
  if (cudaGetLastError() != cudaSuccess) return RQLP_ERR_CUDA;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((M + 7) / 8, 4LL * num_sms()));
  k_sum_parts_f32<<<blocks, dim3(32, 8), 0, st>>>(mx.part, g.S, a.split_stride, M, l, a.ldp, C,
                                                  l, fp8 ? xscale : nullptr,
                                                  fp8 ? yscale : nullptr);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? RQLP_OK : RQLP_ERR_CUDA;
}

int split_skinny(const MixedBufs &mx, bool split, const double *S, int64_t K, int l, int64_t lds,
                 int64_t ldk, cudaStream_t st, bool tf32 = false) {
  const int64_t ktiles = (K + 31) / 32;
  const dim3 grid((unsigned)((l + 31) / 32),
                  (unsigned)std::max<int64_t>(1, std::min<int64_t>(ktiles, 8LL * num_sms())));
  if (tf32)
    k_split_skinny_tf32_t<<<grid, dim3(32, 8), 0, st>>>(S, K, l, lds, static_cast<float *>(mx.Whi),
                                                        static_cast<float *>(mx.Wlo), ldk,
                                                        split ? 1 : 0);
  else
    k_split_skinny_t<<<grid, dim3(32, 8), 0, st>>>(S, K, l, lds,
                                                   static_cast<__nv_bfloat16 *>(mx.Whi),
                                                   static_cast<__nv_bfloat16 *>(mx.Wlo), ldk,
                                                   split ? 1 : 0);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? RQLP_OK : RQLP_ERR_CUDA;
}

}  // namespace

int mixed_init() {
  static int done = 0;
  if (done) return RQLP_OK;
  if (!encode_fn()) return RQLP_ERR_CUDA;
  if (cudaFuncSetAttribute(k_mma_bf16<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(kSmemLimit - 1024)) != cudaSuccess ||
      cudaFuncSetAttribute(k_mma_bf16<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(kSmemLimit - 1024)) != cudaSuccess ||
      cudaFuncSetAttribute(k_mma_bf16<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(kSmemLimit - 1024)) != cudaSuccess ||
      cudaFuncSetAttribute(k_mma_bf16<true, false, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(kSmemLimit - 1024)) != cudaSuccess ||
      cudaFuncSetAttribute(k_mma_bf16<false, false, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(kSmemLimit - 1024)) != cudaSuccess ||
      cudaFuncSetAttribute(k_mma_bf16<true, false, false, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(kSmemLimit - 1024)) != cudaSuccess ||
      cudaFuncSetAttribute(k_mma_bf16<false, false, false, true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(kSmemLimit - 1024)) != cudaSuccess)
    return RQLP_ERR_CUDA;
  done = 1;
  return RQLP_OK;
}

// the forms with a hi/lo pair (three products), and the TF32 forms
static bool is_split(int prec) { return prec == RQLP_PREC_BF16X3 || prec == RQLP_PREC_TF32X3; }
static bool is_tf32(int prec) { return prec == RQLP_PREC_TF32X3 || prec == RQLP_PREC_TF32; }

void carve_mixed(Arena &a, int64_t m, int64_t n, int l, int prec, MixedBufs &mx) {
  mx = MixedBufs{};
  if (prec == RQLP_PREC_FP64) return;
  if (prec == RQLP_PREC_FP64TC) {
    mx.m = m;
    mx.n = n;
    mx.l = l;
    mx.oA = oz_carve(a, m, n, 1);
    mx.oAt = oz_carve(a, n, m, 1);
    mx.oW = oz_carve(a, l, std::max(m, n), kOzCopies);
    mx.opart_floats = (int64_t)std::max(oz_part_floats(m, l, n), oz_part_floats(n, l, m));
    mx.opart = a.take<float>((size_t)mx.opart_floats);
    mx.Ahi = mx.oA.digits;  // marks the buffers as carved
    return;
  }
  if (prec == RQLP_PREC_FP8) {
    mx.m = m;
    mx.n = n;
    mx.l = l;
    const int64_t ld1 = round_up(n, 16), ld2 = round_up(m, 16);
    mx.Ahi = a.take<uint8_t>((size_t)m * ld1);
    mx.Athi = a.take<uint8_t>((size_t)n * ld2);
    mx.Whi = a.take<uint8_t>((size_t)l * round_up(std::max(m, n), 16));
    mx.sA = a.take<float>((size_t)m);
    mx.sAt = a.take<float>((size_t)n);
    mx.sW = a.take<float>((size_t)l);
    mx.rmax = a.take<float>((size_t)m);
    mx.cmax = a.take<unsigned>((size_t)n);
    int64_t pf = 0;
    for (int64_t M : {m, n}) {
      GemmPlan g = plan_gemm(M, (M == m) ? n : m, l, false, true);
      pf = std::max<int64_t>(pf, (int64_t)g.S * M * g.n_pad);
    }
    mx.part_floats = pf;
    mx.part = a.take<float>((size_t)pf);
    return;
  }
  const bool split = is_split(prec), tf32 = is_tf32(prec);
  mx.m = m;
  mx.n = n;
  mx.l = l;
  // BF16 (2 bytes) or FP32-stored TF32 (4 bytes); rows of a multiple of 8
  // elements keep every row 16-byte aligned for the tensor maps
  const size_t es = tf32 ? 4 : 2;
  const int64_t ld1 = round_up(n, 8), ld2 = round_up(m, 8);
  mx.Ahi = a.take<uint8_t>((size_t)m * ld1 * es);
  mx.Alo = split ? a.take<uint8_t>((size_t)m * ld1 * es) : nullptr;
  mx.Athi = a.take<uint8_t>((size_t)n * ld2 * es);
  mx.Atlo = split ? a.take<uint8_t>((size_t)n * ld2 * es) : nullptr;
  const int64_t ldk = round_up(std::max(m, n), 8);
  mx.Whi = a.take<uint8_t>((size_t)l * ldk * es);
  mx.Wlo = split ? a.take<uint8_t>((size_t)l * ldk * es) : nullptr;
  int64_t pf = 0;
  for (int64_t M : {m, n}) {
    const int64_t K = (M == m) ? n : m;
    GemmPlan g = plan_gemm(M, K, l, split, false, tf32);
    pf = std::max<int64_t>(pf, (int64_t)g.S * M * g.n_pad);
  }
  mx.part_floats = pf;
  mx.part = a.take<float>((size_t)pf);
}

int mixed_prepare_A(const MixedBufs &mx, int prec, const void *A, int a_dtype, int64_t m,
                    int64_t n, int64_t lda, Ctrl *ctrl, cudaStream_t st) {
  if (!mx.Ahi) return RQLP_ERR_WORKSPACE;
  if (prec == RQLP_PREC_FP64TC) {
    // digits of the rows of A (for Y = A W) and of its columns (for Z = A^T V)
    return oz_split_both(A, a_dtype, m, n, lda, mx.oA, mx.oAt, ctrl, st);
  }
  if (prec == RQLP_PREC_FP8) {
    if (cudaMemsetAsync(mx.cmax, 0, (size_t)n * sizeof(unsigned), st) != cudaSuccess)
      return RQLP_ERR_CUDA;
    const int rb = (int)((m + 31) / 32);
    if (a_dtype == RQLP_F32)
      k_absmax<float><<<rb, 256, 0, st>>>(static_cast<const float *>(A), m, n, lda, mx.rmax, mx.cmax);
    else
      k_absmax<double><<<rb, 256, 0, st>>>(static_cast<const double *>(A), m, n, lda, mx.rmax, mx.cmax);
    count_launch();
    k_scales<<<(int)std::min<int64_t>((m + n + 255) / 256, 1024), 256, 0, st>>>(mx.rmax, m, mx.cmax, n,
                                                                            mx.sA, mx.sAt);
    count_launch();
    dim3 grid((unsigned)((n + 31) / 32), (unsigned)((m + 31) / 32));
    auto *A8 = static_cast<__nv_fp8_storage_t *>(mx.Ahi);
    auto *At8 = static_cast<__nv_fp8_storage_t *>(mx.Athi);
    if (a_dtype == RQLP_F32)
      k_quant_a<float><<<grid, dim3(32, 8), 0, st>>>(static_cast<const float *>(A), m, n, lda, mx.sA,
                                                      mx.sAt, A8, round_up(n, 16), At8, round_up(m, 16));
    else
      k_quant_a<double><<<grid, dim3(32, 8), 0, st>>>(static_cast<const double *>(A), m, n, lda, mx.sA,
                                                       mx.sAt, A8, round_up(n, 16), At8, round_up(m, 16));
    count_launch();
    return cudaGetLastError() == cudaSuccess ? RQLP_OK : RQLP_ERR_CUDA;
  }
  const bool split = is_split(prec);
  const int64_t ld1 = round_up(n, 8), ld2 = round_up(m, 8);
  if (is_tf32(prec)) {
    dim3 g32((unsigned)((n + 31) / 32), (unsigned)((m + 31) / 32));
    auto *Ah = static_cast<float *>(mx.Ahi);
    auto *Al = static_cast<float *>(mx.Alo);
    auto *Ath = static_cast<float *>(mx.Athi);
    auto *Atl = static_cast<float *>(mx.Atlo);
    if (a_dtype == RQLP_F32)
      k_split_a_tf32<float><<<g32, dim3(32, 8), 0, st>>>(static_cast<const float *>(A), m, n, lda,
                                                          Ah, Al, ld1, Ath, Atl, ld2, split ? 1 : 0);
    else
      k_split_a_tf32<double><<<g32, dim3(32, 8), 0, st>>>(static_cast<const double *>(A), m, n,
                                                           lda, Ah, Al, ld1, Ath, Atl, ld2,
                                                           split ? 1 : 0);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? RQLP_OK : RQLP_ERR_CUDA;
  }
  dim3 grid((unsigned)((n + 63) / 64), (unsigned)((m + 31) / 32));
  auto *Ah = static_cast<__nv_bfloat16 *>(mx.Ahi);
  auto *Al = static_cast<__nv_bfloat16 *>(mx.Alo);
  auto *Ath = static_cast<__nv_bfloat16 *>(mx.Athi);
  auto *Atl = static_cast<__nv_bfloat16 *>(mx.Atlo);
  if (a_dtype == RQLP_F32)
    k_split_a<float><<<grid, dim3(32, 8), 0, st>>>(static_cast<const float *>(A), m, n, lda, Ah, Al,
                                                    ld1, Ath, Atl, ld2, split ? 1 : 0);
  else
    k_split_a<double><<<grid, dim3(32, 8), 0, st>>>(static_cast<const double *>(A), m, n, lda, Ah,
                                                     Al, ld1, Ath, Atl, ld2, split ? 1 : 0);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? RQLP_OK : RQLP_ERR_CUDA;
}

int quant_skinny(const MixedBufs &mx, const double *S, int64_t K, int l, int64_t lds, int64_t ldk,
                 cudaStream_t st) {
  k_quant_skinny_t<<<l, 256, 0, st>>>(S, K, l, lds, static_cast<__nv_fp8_storage_t *>(mx.Whi), ldk,
                                      mx.sW);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? RQLP_OK : RQLP_ERR_CUDA;
}

// The skinny operand S (K x l, FP64) as the Y operand of a digit product
static OzOperand skinny_view(const MixedBufs &mx, int64_t K, int l) {
  OzOperand o = mx.oW;
  o.rows = l;
  o.K = K;
  o.ld = (K + 7) / 8 * 8;
  return o;
}

int mixed_nn(const MixedBufs &mx, int prec, int64_t m, int64_t n, const double *W, int64_t ldw,
             int l, double *Y, Ctrl *ctrl, int64_t spin_ns, cudaStream_t st) {
  if (prec == RQLP_PREC_FP64TC) {
    const OzOperand w = skinny_view(mx, n, l);
    int r = oz_split(W, RQLP_F64, n, l, ldw, true, w, ctrl, nullptr, st);
    if (r != RQLP_OK) return r;
    return oz_gemm(mx.oA, w, m, l, n, Y, l, nullptr, mx.opart, mx.opart_floats, ctrl, spin_ns,
                   nullptr, st);
  }
  if (prec == RQLP_PREC_FP8) {
    const int64_t ldk = round_up(n, 16);
    int r = quant_skinny(mx, W, n, l, ldw, ldk, st);
    if (r != RQLP_OK) return r;
    return gemm_xyt(mx, false, m, n, l, mx.Ahi, nullptr, round_up(n, 16), mx.Whi, nullptr, ldk, Y,
                    ctrl, spin_ns, st, true, mx.sA, mx.sW);
  }
  const bool split = is_split(prec), tf32 = is_tf32(prec);
  const int64_t ldk = round_up(n, 8);
  int r = split_skinny(mx, split, W, n, l, ldw, ldk, st, tf32);
  if (r != RQLP_OK) return r;
  return gemm_xyt(mx, split, m, n, l, mx.Ahi, mx.Alo, round_up(n, 8), mx.Whi, mx.Wlo, ldk, Y, ctrl,
                  spin_ns, st, false, nullptr, nullptr, tf32);
}

int mixed_tn(const MixedBufs &mx, int prec, int64_t m, int64_t n, const double *V, int64_t ldv,
             int l, double *Z, Ctrl *ctrl, int64_t spin_ns, cudaStream_t st) {
  if (prec == RQLP_PREC_FP64TC) {
    const OzOperand v = skinny_view(mx, m, l);
    int r = oz_split(V, RQLP_F64, m, l, ldv, true, v, ctrl, nullptr, st);
    if (r != RQLP_OK) return r;
    return oz_gemm(mx.oAt, v, n, l, m, Z, l, nullptr, mx.opart, mx.opart_floats, ctrl, spin_ns,
                   nullptr, st);
  }
  if (prec == RQLP_PREC_FP8) {
    const int64_t ldk = round_up(m, 16);
    int r = quant_skinny(mx, V, m, l, ldv, ldk, st);
    if (r != RQLP_OK) return r;
    return gemm_xyt(mx, false, n, m, l, mx.Athi, nullptr, round_up(m, 16), mx.Whi, nullptr, ldk, Z,
                    ctrl, spin_ns, st, true, mx.sAt, mx.sW);
  }
  const bool split = is_split(prec), tf32 = is_tf32(prec);
  const int64_t ldk = round_up(m, 8);
  int r = split_skinny(mx, split, V, m, l, ldv, ldk, st, tf32);
  if (r != RQLP_OK) return r;
  return gemm_xyt(mx, split, n, m, l, mx.Athi, mx.Atlo, round_up(m, 8), mx.Whi, mx.Wlo, ldk, Z,
                  ctrl, spin_ns, st, false, nullptr, nullptr, tf32);
}

}  // namespace rqk
