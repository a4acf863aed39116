// Mixed-precision products (placeholder until the tcgen05 kernels land).
#include "mixed.cuh"

namespace rqk {

void carve_mixed(Arena &, int64_t, int64_t, int, int, MixedBufs &mx) {
  mx = MixedBufs{};
}

int mixed_prepare_A(const MixedBufs &, int, const void *, int, int64_t, int64_t, int64_t,
                    cudaStream_t) {
  return RQLP_ERR_UNSUPPORTED;
}

int mixed_nn(const MixedBufs &, int, int64_t, int64_t, const double *, int64_t, int, double *,
             Ctrl *, int64_t, cudaStream_t) {
  return RQLP_ERR_UNSUPPORTED;
}

int mixed_tn(const MixedBufs &, int, int64_t, int64_t, const double *, int64_t, int, double *,
             Ctrl *, int64_t, cudaStream_t) {
  return RQLP_ERR_UNSUPPORTED;
}

}  // namespace rqk
