// Instantiations and launcher of the second pass of the two-pass form.
#include "adfft_internal.h"
#include "twopass.cuh"

namespace adfft {

namespace {

using KernelFn = void (*)(const TwoPassArgs);

template <typename V, int VPT>
KernelFn pick_r0(int r0) {
  switch (r0) {
    case 1: return twopass_columns_kernel<V, VPT, 1>;
    case 2: return twopass_columns_kernel<V, VPT, 2>;
    case 4: return twopass_columns_kernel<V, VPT, 4>;
    case 8: return twopass_columns_kernel<V, VPT, 8>;
    default: return twopass_columns_kernel<V, VPT, 16>;
  }
}

KernelFn pick_kernel(const TwoPassLaunch& L) {
  return L.dbl ? pick_r0<double2, 16>(L.r0) : pick_r0<float2, 32>(L.r0);
}

template <typename V, int VPT>
KernelFn pick_adj_r0(int r0) {
  switch (r0) {
    case 1: return twopass_adjoint_columns_kernel<V, VPT, 1>;
    case 2: return twopass_adjoint_columns_kernel<V, VPT, 2>;
    case 4: return twopass_adjoint_columns_kernel<V, VPT, 4>;
    case 8: return twopass_adjoint_columns_kernel<V, VPT, 8>;
    default: return twopass_adjoint_columns_kernel<V, VPT, 16>;
  }
}

KernelFn pick_adj_kernel(const TwoPassLaunch& L) {
  return L.dbl ? pick_adj_r0<double2, 16>(L.r0) : pick_adj_r0<float2, 32>(L.r0);
}

}  // namespace

cudaError_t twopass_prepare(const TwoPassLaunch& L) {
  cudaError_t e = cudaFuncSetAttribute(pick_kernel(L), cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(pick_adj_kernel(L), cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  return e;
}

// Adjoint of the second pass: spectrum g -> scratch rows.  The forward pass's
// geometry: one CTA per block of W columns (packed real input: W column pairs
// m1, R1 - m1, 2 W column regions of shared memory).
cudaError_t twopass_adjoint_launch(const TwoPassLaunch& L, const void* g, void* scratch, cudaStream_t stream) {
  TwoPassArgs t = L.args;
  t.out = const_cast<void*>(g);
  t.scratch = scratch;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(L.grid_x, L.grid_y, 1);
  cfg.blockDim = dim3(L.threads, 1, 1);
  cfg.dynamicSmemBytes = L.smem;
  cfg.stream = stream;
  cfg.numAttrs = 0;
  return cudaLaunchKernelEx(&cfg, pick_adj_kernel(L), t);
}

cudaError_t twopass_launch(const TwoPassLaunch& L, const void* scratch, void* out, cudaStream_t stream) {
  TwoPassArgs t = L.args;
  t.scratch = scratch;
  t.out = out;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(L.grid_x, L.grid_y, 1);
  cfg.blockDim = dim3(L.threads, 1, 1);
  cfg.dynamicSmemBytes = L.smem;
  cfg.stream = stream;
  cfg.numAttrs = 0;
  return cudaLaunchKernelEx(&cfg, pick_kernel(L), t);
}

}  // namespace adfft
