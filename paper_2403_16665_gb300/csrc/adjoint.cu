// Instantiations and launcher of the single-pass adjoint kernel.
#include "adfft_internal.h"
#include "adjoint.cuh"

namespace adfft {

namespace {

using KernelFn = void (*)(const FusedArgs);

template <typename V, int MODE, int VPT>
KernelFn pick_r0(int r0) {
  switch (r0) {
    case 32:
      if constexpr (VPT >= 32) return adjoint_kernel<V, MODE, VPT, 32>;
      else return nullptr;
    case 1: return adjoint_kernel<V, MODE, VPT, 1>;
    case 2: return adjoint_kernel<V, MODE, VPT, 2>;
    case 4: return adjoint_kernel<V, MODE, VPT, 4>;
    case 8: return adjoint_kernel<V, MODE, VPT, 8>;
    default: return adjoint_kernel<V, MODE, VPT, 16>;
  }
}

// compile-time shape of the 4096 x 16384, alpha = 8 class (packed sub-FFT 8192, 8 residues,
// 2 per CTA, 512 threads, padding of 2 slots per 32 elements), as in the forward kernel
using AdjShapeR32N8192P8 = Shape<13, 2, 8, 512, 2, 5, 0, 2>;

KernelFn pick_kernel(const FusedLaunch& L) {
  const FusedArgs& a = L.args;
  if (!L.dbl && L.mode == kLoadRealPacked && L.r0 == 32 && a.logNp == 13 && a.RPC == 2 && a.P == 8 &&
      L.threads == 512 && a.Mt == 2 * a.Mc)
    return adjoint_kernel<float2, kLoadRealPacked, 32, 32, AdjShapeR32N8192P8>;
  if (KernelFn k = spec16k_adjoint(L)) return k;
  const int vpt = fused_values_per_thread(L.dbl);
  if (L.dbl) {
    (void)vpt;
    switch (L.mode) {
      case kLoadComplex: return pick_r0<double2, kLoadComplex, 16>(L.r0);
      case kLoadRealPacked: return pick_r0<double2, kLoadRealPacked, 16>(L.r0);
      case kColumns: return pick_r0<double2, kColumns, 16>(L.r0);
      default: return pick_r0<double2, kLoadRealPlain, 16>(L.r0);
    }
  }
  switch (L.mode) {
    case kLoadComplex: return pick_r0<float2, kLoadComplex, 32>(L.r0);
    case kLoadRealPacked: return pick_r0<float2, kLoadRealPacked, 32>(L.r0);
    case kColumns: return pick_r0<float2, kColumns, 32>(L.r0);
    default: return pick_r0<float2, kLoadRealPlain, 32>(L.r0);
  }
}

}  // namespace

size_t adjoint_smem_bytes(const FusedLaunch& L) {
  const FusedArgs& a = L.args;
  return (size_t)fused_smem_layout(a.tw_lo_n + a.tw_hi_n, 0, a.RPC, a.region, L.dbl ? 16 : 8).total;
}

cudaError_t adjoint_prepare(const FusedLaunch& L) {
  KernelFn k = pick_kernel(L);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e != cudaSuccess) return e;
  if (L.args.C > 8) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

cudaError_t adjoint_launch(const FusedLaunch& L, const void* g, void* xb, cudaStream_t stream) {
  KernelFn k = pick_kernel(L);
  FusedArgs a = L.args;
  a.in = g;
  a.out = xb;
  a.stage_bytes = 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.C, L.grid_y, 1);
  cfg.blockDim = dim3(L.threads, 1, 1);
  cfg.dynamicSmemBytes = adjoint_smem_bytes(L);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = a.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = a.C > 1 ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, a);
}

}  // namespace adfft
