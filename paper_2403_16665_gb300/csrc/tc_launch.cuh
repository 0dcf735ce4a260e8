// Launchers of the forward kernels with tensor-core radix-16 passes, one
// precision form per translation unit (instantiated by fused_tc_fp16.cu and
// fused_tc_bf16.cu).
#pragma once

#include "adfft_internal.h"
#include "tc_dft16.cuh"

namespace adfft {

template <int PREC>
struct TcKernels {
  using FusedFn = void (*)(const FusedArgs);
  using ColFn = void (*)(const TwoPassArgs);

  template <int MODE>
  static FusedFn fused_r0(int r0) {
    switch (r0) {
      case 32: return fused_forward_kernel<float2, MODE, 32, 32, PREC>;
      case 1: return fused_forward_kernel<float2, MODE, 32, 1, PREC>;
      case 2: return fused_forward_kernel<float2, MODE, 32, 2, PREC>;
      case 4: return fused_forward_kernel<float2, MODE, 32, 4, PREC>;
      case 8: return fused_forward_kernel<float2, MODE, 32, 8, PREC>;
      default: return fused_forward_kernel<float2, MODE, 32, 16, PREC>;
    }
  }
  static FusedFn fused(const FusedLaunch& L) {
    switch (L.mode) {
      case kLoadComplex: return fused_r0<kLoadComplex>(L.r0);
      case kLoadRealPacked: return fused_r0<kLoadRealPacked>(L.r0);
      case kColumns: return fused_r0<kColumns>(L.r0);
      default: return fused_r0<kLoadRealPlain>(L.r0);
    }
  }
  static ColFn columns(int r0) {
    switch (r0) {
      case 1: return twopass_columns_kernel<float2, 32, 1, PREC>;
      case 2: return twopass_columns_kernel<float2, 32, 2, PREC>;
      case 4: return twopass_columns_kernel<float2, 32, 4, PREC>;
      case 8: return twopass_columns_kernel<float2, 32, 8, PREC>;
      default: return twopass_columns_kernel<float2, 32, 16, PREC>;
    }
  }

  static cudaError_t prepare(const FusedLaunch* L, const TwoPassLaunch* L2) {
    cudaError_t e = cudaSuccess;
    if (L) {
      e = cudaFuncSetAttribute(fused(*L), cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
      if (e == cudaSuccess && L->args.C > 8)
        e = cudaFuncSetAttribute(fused(*L), cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    }
    if (e == cudaSuccess && L2)
      e = cudaFuncSetAttribute(columns(L2->r0), cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    return e;
  }

  static cudaError_t launch_fused(const FusedLaunch& L, const void* in, void* out, cudaStream_t stream) {
    FusedArgs a = L.args;
    a.in = in;
    a.out = out;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.C, L.grid_y, 1);
    cfg.blockDim = dim3(L.threads, 1, 1);
    cfg.dynamicSmemBytes = L.smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = a.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = a.C > 1 ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, fused(L), a);
  }

  static cudaError_t launch_columns(const TwoPassLaunch& L, const void* scratch, void* out, cudaStream_t stream) {
    TwoPassArgs t = L.args;
    t.scratch = scratch;
    t.out = out;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(L.grid_x, L.grid_y, 1);
    cfg.blockDim = dim3(L.threads, 1, 1);
    cfg.dynamicSmemBytes = L.smem;
    cfg.stream = stream;
    cfg.numAttrs = 0;
    return cudaLaunchKernelEx(&cfg, columns(L.r0), t);
  }
};

}  // namespace adfft
