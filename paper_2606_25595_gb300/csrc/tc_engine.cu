// Tensor-core engine (sm_103a tcgen05): emulated-precision batched complex GEMM.
#include "kernels.cuh"

namespace qtx {
bool tc_available() { return false; }
size_t gemm_tc_scratch_bytes(int, int, int, int, const TcConfig&) { return 0; }
cudaError_t gemm_tc(const GemmArgs<double>&, const TcConfig&, void*, size_t, int*, cudaStream_t) {
  return cudaErrorNotSupported;
}
}  // namespace qtx
