// Forward kernels with tensor-core radix-16 passes, fp16 split operands.
#include "tc_launch.cuh"

namespace adfft {

cudaError_t tc_prepare_fp16(const FusedLaunch* L, const TwoPassLaunch* L2) {
  return TcKernels<kPrecFp16x2>::prepare(L, L2);
}
cudaError_t tc_launch_fused_fp16(const FusedLaunch& L, const void* in, void* out, cudaStream_t s) {
  return TcKernels<kPrecFp16x2>::launch_fused(L, in, out, s);
}
cudaError_t tc_launch_columns_fp16(const TwoPassLaunch& L, const void* scratch, void* out, cudaStream_t s) {
  return TcKernels<kPrecFp16x2>::launch_columns(L, scratch, out, s);
}

}  // namespace adfft
