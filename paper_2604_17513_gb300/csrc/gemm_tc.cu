// Tensor-core global solve (tcgen05, f16 hi/lo split, FP32 accumulation in
// TMEM).  Placeholder until the kernel lands: reports "not supported".
#include "flash_internal.cuh"

namespace flash {

bool tc_available() { return false; }

cudaError_t gemm_tc(const Group &g, float *out, const float *w, const int *done, int mode, cudaStream_t st) {
  (void)g; (void)out; (void)w; (void)done; (void)mode; (void)st;
  return cudaErrorNotSupported;
}

}  // namespace flash
