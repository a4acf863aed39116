// rqlp_cpqr_static(): the column-pivoted QR of B with no device allocation
// by anyone.
//
// Some callers cannot hand the library a workspace: code that runs under
// another runtime's memory manager which owns all of the device memory, or a
// latency-critical loop that must not call cudaMalloc (it can synchronize
// the whole device).  For them this entry point keeps all of its scratch in
// one file-scope __device__ array of fixed size, which every GPU that loads
// the library holds until the process exits.
#include <mutex>

#include "kernels.cuh"

using namespace rqk;

namespace {

constexpr size_t kStaticScratchBytes = 2u << 20;  // 2 MiB per device

// Control block, reflectors, tau and the pivot tables of one call.
static __device__ __align__(256) unsigned char g_cpqr_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of g_cpqr_scratch on the current device, looked up once per
// device.  In host code the symbol is only a host-side stand-in, so the
// kernels get this address instead.
cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_cpqr_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

size_t up256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

extern "C" int rqlp_cpqr_static(const double *Bt, int64_t n, int32_t l, int64_t ldb, double *R0t,
                                int32_t *piv0, double *Q0, int32_t sync, rqlp_stream_t stream) {
  if (!Bt || !R0t || !piv0 || n <= 0 || l < 1 || l > kMaxL || l > n || ldb < l)
    return RQLP_ERR_INVALID_ARG;
  // fixed layout: Ctrl | Vh (l x l) | tau (l) | pivot tables of the plan
  bool fits = false;
  const size_t tables = cpqr_scratch_bytes_smem_only(n, l, &fits);
  const size_t need = up256(sizeof(Ctrl)) + up256((size_t)l * l * sizeof(double)) +
                      up256((size_t)l * sizeof(double)) + tables;
  if (!fits || need > kStaticScratchBytes) return RQLP_ERR_WORKSPACE;
  void *base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return RQLP_ERR_CUDA;
  char *p = reinterpret_cast<char *>(base);
  Ctrl *ctrl = reinterpret_cast<Ctrl *>(p);
  p += up256(sizeof(Ctrl));
  double *Vh = reinterpret_cast<double *>(p);
  p += up256((size_t)l * l * sizeof(double));
  double *tau = reinterpret_cast<double *>(p);
  p += up256((size_t)l * sizeof(double));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // the array keeps the previous call's contents: the status word and the
  // barrier counters must start at zero
  if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st) != cudaSuccess) return RQLP_ERR_CUDA;
  if (cpqr_wide(Bt, n, l, ldb, R0t, l, piv0, Vh, tau, p, ctrl, 0, 0, st) != cudaSuccess)
    return RQLP_ERR_CUDA;
  if (Q0 && form_q(Vh, l, tau, l, l, Q0, l, st) != cudaSuccess) return RQLP_ERR_CUDA;
  if (!sync) return RQLP_OK;
  if (cudaStreamSynchronize(st) != cudaSuccess) return RQLP_ERR_CUDA;
  int status = 0;
  if (cudaMemcpy(&status, ctrl, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return RQLP_ERR_CUDA;
  return status;
}
