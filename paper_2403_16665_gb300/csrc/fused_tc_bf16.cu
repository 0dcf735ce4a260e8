// Forward kernels with tensor-core radix-16 passes, bf16 split operands.
#include "tc_launch.cuh"

namespace adfft {

cudaError_t tc_prepare_bf16(const FusedLaunch* L, const TwoPassLaunch* L2) {
  return TcKernels<kPrecBf16x3>::prepare(L, L2);
}
cudaError_t tc_launch_fused_bf16(const FusedLaunch& L, const void* in, void* out, cudaStream_t s) {
  return TcKernels<kPrecBf16x3>::launch_fused(L, in, out, s);
}
cudaError_t tc_launch_columns_bf16(const TwoPassLaunch& L, const void* scratch, void* out, cudaStream_t s) {
  return TcKernels<kPrecBf16x3>::launch_columns(L, scratch, out, s);
}

}  // namespace adfft
