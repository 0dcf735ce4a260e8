// Instantiations and launcher of the chirp-z (Bluestein) kernel.
#include "adfft_internal.h"
#include "bluestein.cuh"

namespace adfft {

namespace {

using KernelFn = void (*)(const BluesteinArgs);

template <typename V, int VPT>
KernelFn pick_r0(int r0) {
  switch (r0) {
    case 1: return bluestein_kernel<V, VPT, 1>;
    case 2: return bluestein_kernel<V, VPT, 2>;
    case 4: return bluestein_kernel<V, VPT, 4>;
    case 8: return bluestein_kernel<V, VPT, 8>;
    default: return bluestein_kernel<V, VPT, 16>;
  }
}

KernelFn pick_kernel(const BluesteinLaunch& L) {
  return L.dbl ? pick_r0<double2, 16>(L.r0) : pick_r0<float2, 32>(L.r0);
}

}  // namespace

cudaError_t bluestein_prepare(const BluesteinLaunch& L) {
  return cudaFuncSetAttribute(pick_kernel(L), cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

cudaError_t bluestein_launch(const BluesteinLaunch& L, const void* in, void* out, cudaStream_t stream) {
  BluesteinArgs b = L.args;
  b.f.in = in;
  b.f.out = out;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b.chunks, L.grid_y, 1);
  cfg.blockDim = dim3(L.threads, 1, 1);
  cfg.dynamicSmemBytes = L.smem;
  cfg.stream = stream;
  cfg.numAttrs = 0;
  return cudaLaunchKernelEx(&cfg, pick_kernel(L), b);
}

namespace {

using AdjKernelFn = void (*)(const BluesteinAdjArgs);

template <typename V, int VPT, int ACC>
AdjKernelFn pick_adj_r0(int r0) {
  switch (r0) {
    case 1: return bluestein_adjoint_kernel<V, VPT, 1, ACC>;
    case 2: return bluestein_adjoint_kernel<V, VPT, 2, ACC>;
    case 4: return bluestein_adjoint_kernel<V, VPT, 4, ACC>;
    case 8: return bluestein_adjoint_kernel<V, VPT, 8, ACC>;
    default: return bluestein_adjoint_kernel<V, VPT, 16, ACC>;
  }
}

AdjKernelFn pick_adj_kernel(const BluesteinAdjLaunch& L) {
  return L.dbl ? pick_adj_r0<double2, 16, kBlaAccF64>(L.r0) : pick_adj_r0<float2, 32, kBlaAccF32>(L.r0);
}

}  // namespace

cudaError_t bluestein_adjoint_prepare(const BluesteinAdjLaunch& L) {
  return cudaFuncSetAttribute(pick_adj_kernel(L), cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

cudaError_t bluestein_adjoint_launch(const BluesteinAdjLaunch& L, const void* g, void* xb, cudaStream_t stream) {
  BluesteinAdjArgs b = L.args;
  b.f.in = g;
  b.f.out = xb;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b.nO, L.grid_y, 1);
  cfg.blockDim = dim3(L.threads, 1, 1);
  cfg.dynamicSmemBytes = L.smem;
  cfg.stream = stream;
  cfg.numAttrs = 0;
  return cudaLaunchKernelEx(&cfg, pick_adj_kernel(L), b);
}

}  // namespace adfft
