// rqlp_selftest: the device arithmetic helpers of common.cuh against CUDA's
// own operations (see include/rqlp.h).  Inputs come from a counter-based
// hash (SplitMix64 of the index), so every run checks the same values.
#include "kernels.cuh"

namespace rqk {
namespace {

__device__ int g_selftest_fails[4];

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9e3779b97f4a7c15ULL;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
  return x ^ (x >> 31);
}

__global__ void k_selftest(int count) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const unsigned long long h = splitmix64((unsigned long long)i);
    // FP64 with a random significand and an exponent inside the FP32 normal
    // range (|x| in [2^-120, 2^120)), either sign
    const int e = (int)((h >> 52) % 240) - 120;
    const unsigned long long bits = (h & 0x000fffffffffffffULL) |
                                    ((unsigned long long)(1023 + e) << 52) |
                                    ((h >> 63) ? 0x8000000000000000ULL : 0ULL);
    const double x = __longlong_as_double((long long)bits);
    // 1. FP64 -> FP32
    if (__float_as_uint(d2f_rn(x)) != __float_as_uint(__double2float_rn(x)))
      atomicAdd(&g_selftest_fails[0], 1);
    // 2. FP32 -> FP64
    const float f = __double2float_rn(x);
    if (__double_as_longlong(f2d(f)) != __double_as_longlong((double)f))
      atomicAdd(&g_selftest_fails[1], 1);
    // 3. reciprocal
    const double r = rcp_fast(x), rr = 1.0 / x;
    if (!(fabs(r - rr) <= 0x1p-51 * fabs(rr))) atomicAdd(&g_selftest_fails[2], 1);
    // 4. reciprocal square root of |x|
    const double ax = fabs(x);
    const double q = rsqrt_fast(ax), qq = 1.0 / sqrt(ax);
    if (!(fabs(q - qq) <= 0x1p-51 * qq)) atomicAdd(&g_selftest_fails[3], 1);
  }
}

}  // namespace
}  // namespace rqk

extern "C" int rqlp_selftest(int32_t count, int32_t *fails, rqlp_stream_t stream) {
  if (count <= 0 || count > (1 << 24) || !fails) return RQLP_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int zero[4] = {0, 0, 0, 0};
  if (cudaMemcpyToSymbolAsync(rqk::g_selftest_fails, zero, sizeof(zero), 0,
                              cudaMemcpyHostToDevice, st) != cudaSuccess)
    return RQLP_ERR_CUDA;
  const int blocks = (int)std::min<int64_t>((count + 255) / 256, 4LL * rqk::num_sms());
  rqk::k_selftest<<<blocks, 256, 0, st>>>(count);
  rqk::count_launch();
  if (cudaGetLastError() != cudaSuccess) return RQLP_ERR_CUDA;
  int out[4];
  if (cudaMemcpyFromSymbolAsync(out, rqk::g_selftest_fails, sizeof(out), 0,
                                cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return RQLP_ERR_CUDA;
  for (int k = 0; k < 4; ++k) fails[k] = out[k];
  return RQLP_OK;
}

// ---------------------------------------------------------------------------
// FP64 throughput probe: the denominator of the FP64 rooflines.  Every thread
// runs eight independent FMA chains (enough in flight to keep the FP64 units
// busy), so the kernel is bound by FP64 issue alone; the chains' sums are
// written only when they match an impossible value, which keeps the compiler
// from dropping the work without costing any traffic.
namespace rqk {
namespace {

constexpr int kProbeChains = 8;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_fp64_probe(int iters, double *sink) {
  double a[kProbeChains];
  const double x = 1.0 + 1e-9 * (double)threadIdx.x, y = 0.999999999;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) a[c] = (double)(c + 1);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) a[c] = fma(a[c], y, x);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += a[c];
  if (s == -1.0) sink[0] = s;
}

}  // namespace
}  // namespace rqk

extern "C" int rqlp_fp64_probe(int32_t iters, double *sink, double *flops, rqlp_stream_t stream) {
  if (iters <= 0 || !sink || !flops) return RQLP_ERR_INVALID_ARG;
  const int blocks = 4 * rqk::num_sms();
  rqk::k_fp64_probe<<<blocks, rqk::kProbeThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      iters, sink);
  rqk::count_launch();
  if (cudaGetLastError() != cudaSuccess) return RQLP_ERR_CUDA;
  *flops = 2.0 * rqk::kProbeChains * (double)iters * blocks * rqk::kProbeThreads;
  return RQLP_OK;
}
