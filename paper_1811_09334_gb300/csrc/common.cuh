// Shared device-side helpers: the control block at the head of every
// workspace, status reporting, fast FP64 reciprocals, integer-pipe roundings
// and shared-memory staging.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rqlp.h"

namespace rqk {

// Control block at offset 0 of a workspace; zeroed at the start of each call.
struct Ctrl {
  int status;               // first error (< 0) or first warning (> 0)
  int shift_flag[15];       // per CholeskyQR site: 1 when a pass needed the shift
  unsigned reserved0[2];
  int timeout_site;         // diagnostics: which wait gave up
  int pad[13];
  int again_flag[16];       // per CholeskyQR site: 1 when a second pass is needed
  int done_flag[16];        // per CholeskyQR site: 1 when one pass was enough
};
static_assert(sizeof(Ctrl) == 256, "Ctrl layout");

constexpr int kMaxL = 256;               // widest sketch supported
constexpr int kShiftSites = 15;
constexpr unsigned long long kDefaultSpinNs = 2000000000ull;

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_volatile_i32(const int *p) {
  return *reinterpret_cast<const volatile int *>(p);
}

// Record a status: errors override warnings, the first error wins.
__device__ inline void set_status(Ctrl *c, int code) {
  int old = ld_volatile_i32(&c->status);
  while (true) {
    if (old < 0) return;
    if (code > 0 && old > 0) return;
    int prev = atomicCAS(&c->status, old, code);
    if (prev == old) return;
    old = prev;
  }
}

// Reciprocal and reciprocal square root for finite x != 0 (x > 0 for the
// square root) with few dependent FP64 operations, which on this GPU cost
// about 64 clocks each: an FP32 estimate from the top bits of x (integer
// operations and one MUFU instruction, ~2^-22 relative error), then one
// third-order Newton step in FP64, whose error O(e^3) lies below FP64
// rounding.  Outside the FP32 exponent range the plain FP64 operation is used.
__device__ __forceinline__ bool fp32_range(long long b) {
  const int e = (int)(b >> 52) & 0x7ff;
  return e > 1023 - 120 && e < 1023 + 120;
}
__device__ __forceinline__ float top_as_float(long long b) {
  const int e = (int)(b >> 52) & 0x7ff;
  const unsigned f = ((unsigned)(b >> 32) & 0x80000000u) | ((unsigned)(e - 1023 + 127) << 23) |
                     (unsigned)((b >> 29) & 0x7fffff);
  return __uint_as_float(f);
}
__device__ __forceinline__ double float_as_double_bits(float y) {
  const unsigned u = __float_as_uint(y);
  const long long e = (long long)((u >> 23) & 0xff) - 127 + 1023;
  return __longlong_as_double(((long long)(u & 0x80000000u) << 32) | (e << 52) |
                              ((long long)(u & 0x7fffff) << 29));
}
__device__ __forceinline__ double rcp_fast(double x) {
  const long long b = __double_as_longlong(x);
  if (!fp32_range(b)) return 1.0 / x;
  float yf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(top_as_float(b)));
  const double y0 = float_as_double_bits(yf);
  const double e = fma(-x, y0, 1.0);  // 1 - x y0
  return fma(y0, fma(e, e, e), y0);   // y0 (1 + e + e^2)
}
__device__ __forceinline__ double rsqrt_fast(double x) {
  const long long b = __double_as_longlong(x);
  if (!fp32_range(b)) return rsqrt(x);
  float yf;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(top_as_float(b)));
  const double y0 = float_as_double_bits(yf);
  const double h = x * y0;
  const double r = fma(-h, y0, 1.0);                // 1 - x y0^2
  return fma(y0, r * fma(0.375, r, 0.5), y0);       // y0 (1 + r/2 + 3 r^2 / 8)
}

// FP64 <-> FP32 conversions on the integer pipe: a conversion instruction
// would occupy the FP64 unit (~64 clocks per warp instruction here), which
// dominates kernels that round every element.  d2f_rn rounds to nearest,
// ties to even (IEEE 754 roundTiesToEven on the 29 dropped significand
// bits); results below the FP32 normal range flush to signed zero, results
// beyond it become infinity, NaN stays NaN.  f2d is exact for normal floats
// and zero (FP32 subnormals flush to zero).
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0x7ff)
    return __uint_as_float(sign | 0x7f800000u |
                           ((b & 0xfffffffffffffULL) != 0 ? 0x400000u : 0u));
  if (e < 1023 - 126) return __uint_as_float(sign);
  if (e > 1023 + 127) return __uint_as_float(sign | 0x7f800000u);
  unsigned f = ((unsigned)(e - 1023 + 127) << 23) | (unsigned)((b >> 29) & 0x7fffffu);
  const unsigned rest = (unsigned)(b & 0x1fffffffULL), half = 0x10000000u;
  if (rest > half || (rest == half && (f & 1u))) f += 1u;  // a carry into the exponent is right
  return __uint_as_float(sign | f);
}
__device__ __forceinline__ double f2d(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long m = (unsigned long long)(u & 0x7fffffu) << 29;
  if (e == 0) return __longlong_as_double((long long)sign);
  if (e == 0xffu) return __longlong_as_double((long long)(sign | 0x7ff0000000000000ULL | m));
  return __longlong_as_double((long long)(sign | ((unsigned long long)(e - 127 + 1023) << 52) | m));
}

template <typename T>
__device__ __forceinline__ float as_f32(T x);
template <>
__device__ __forceinline__ float as_f32<double>(double x) { return d2f_rn(x); }
template <>
__device__ __forceinline__ float as_f32<float>(float x) { return x; }
// FP64 data into the working precision T of a kernel, and back
template <typename T>
__device__ __forceinline__ T from_f64(double x);
template <>
__device__ __forceinline__ double from_f64<double>(double x) { return x; }
template <>
__device__ __forceinline__ float from_f64<float>(double x) { return d2f_rn(x); }
__device__ __forceinline__ double to_f64(double x) { return x; }
__device__ __forceinline__ double to_f64(float x) { return f2d(x); }

// Shared-memory staging.  A plain loop `dst[e] = src[e]` waits one L2 round
// trip per element and thread; in FP64 the copies go out asynchronously
// (cp.async, no registers), all of a thread's elements in flight at once.
// src(e) gives the global address of element e, or nullptr for a zero; dst(e)
// its shared slot.  The FP64 form needs cp_async_wait_all() and a block
// barrier before other threads read the copies.  A conversion to FP32 on the
// way stays a plain loop: batches of eight loads per thread measured slower
// in the FP32 triangular solve (85 against 72 us per 8192-row pass).
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(s), "l"(gmem),
               "r"(valid ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}
template <typename T, typename Src, typename Dst>
__device__ __forceinline__ void stage_smem(int n, const double *any, Src src, Dst dst) {
  if constexpr (sizeof(T) == 8) {
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const double *p = src(e);
      cp_async8(dst(e), p ? p : any, p != nullptr);
    }
  } else {
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
      const double *p = src(e);
      *dst(e) = p ? (T)*p : (T)0;
    }
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the whole CTA; `red` is shared scratch of >= 32 doubles.  All
// threads receive the result.
__device__ inline double block_sum(double v, double *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (warp == 0) {
    t = lane < nw ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) red[0] = t;
  }
  __syncthreads();
  t = red[0];
  __syncthreads();
  return t;
}

}  // namespace rqk
