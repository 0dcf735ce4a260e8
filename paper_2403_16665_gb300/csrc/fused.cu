// Instantiations and launchers of the fused single-pass forward kernel.
#include "adfft_internal.h"

namespace adfft {

namespace {

constexpr int kVptF32 = 32;   // complex values per thread per pass, float2
constexpr int kVptF64 = 16;   // complex values per thread per pass, double2

using KernelFn = void (*)(const FusedArgs);

template <typename V, int MODE, int VPT>
KernelFn pick_r0(int r0) {
  switch (r0) {
    case 32:
      if constexpr (VPT >= 32) return fused_forward_kernel<V, MODE, VPT, 32>;
      else return nullptr;
    case 1: return fused_forward_kernel<V, MODE, VPT, 1>;
    case 2: return fused_forward_kernel<V, MODE, VPT, 2>;
    case 4: return fused_forward_kernel<V, MODE, VPT, 4>;
    case 8: return fused_forward_kernel<V, MODE, VPT, 8>;
    default: return fused_forward_kernel<V, MODE, VPT, 16>;
  }
}

// Shapes with a compile-time specialisation (all strides and pass counts constant).
// real fp32, packed sub-FFT 8192, 8 residues, 2 per CTA, 512 threads; padding of 2 slots per 32
// elements (16-byte pairs stay aligned; the radix-32 first pass stores pairs without bank
// conflicts in every quarter-warp), epilogue in pairs of k with 5 pair loads in flight per thread
// (full-spectrum output; the half-spectrum variant below)
using ShapeR32N8192P8 = Shape<13, 2, 8, 512, 2, 5, 5, 2, 1>;
using ShapeR32N8192P8Half = Shape<13, 2, 8, 512, 2, 5, 5, 2, 2>;

// the same with one residue per CTA (clusters of 8, 256 threads: two CTAs per SM)
using ShapeR32N8192P8C8 = Shape<13, 1, 8, 256, 2, 5, 4, 2, 1>;

bool is_r32_n8192_p8(const FusedLaunch& L, int rpc, int threads) {
  const FusedArgs& a = L.args;
  return !L.dbl && L.mode == kLoadRealPacked && L.r0 == 32 && a.logNp == 13 && a.RPC == rpc && a.P == 8 &&
         L.threads == threads && a.Mt == 2 * a.Mc;
}

KernelFn pick_kernel(const FusedLaunch& L) {
  if (L.push) return push_forward(L);
  if (is_r32_n8192_p8(L, 2, 512))
    return L.args.half ? fused_forward_kernel<float2, kLoadRealPacked, kVptF32, 32, 0, ShapeR32N8192P8Half>
                       : fused_forward_kernel<float2, kLoadRealPacked, kVptF32, 32, 0, ShapeR32N8192P8>;
  if (KernelFn k = spec16k_forward(L)) return k;
  if (is_r32_n8192_p8(L, 1, 256) && !L.args.half)
    return fused_forward_kernel<float2, kLoadRealPacked, kVptF32, 32, 0, ShapeR32N8192P8C8>;
  if (L.dbl) {
    switch (L.mode) {
      case kLoadComplex: return pick_r0<double2, kLoadComplex, kVptF64>(L.r0);
      case kLoadRealPacked: return pick_r0<double2, kLoadRealPacked, kVptF64>(L.r0);
      case kColumns: return pick_r0<double2, kColumns, kVptF64>(L.r0);
      default: return pick_r0<double2, kLoadRealPlain, kVptF64>(L.r0);
    }
  }
  switch (L.mode) {
    case kLoadComplex: return pick_r0<float2, kLoadComplex, kVptF32>(L.r0);
    case kLoadRealPacked: return pick_r0<float2, kLoadRealPacked, kVptF32>(L.r0);
    case kColumns: return pick_r0<float2, kColumns, kVptF32>(L.r0);
    default: return pick_r0<float2, kLoadRealPlain, kVptF32>(L.r0);
  }
}

}  // namespace

int fused_values_per_thread(bool dbl) { return dbl ? kVptF64 : kVptF32; }

cudaError_t fused_prepare(const FusedLaunch& L) {
  KernelFn k = pick_kernel(L);
  if (!k) return cudaErrorInvalidConfiguration;
  // the attribute is per kernel and shared by every plan: always allow the full 227 KiB
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  if (e != cudaSuccess) return e;
  if (L.args.C > 8) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int fused_max_active_clusters(const FusedLaunch& L) {
  KernelFn k = pick_kernel(L);
  if (!k) return -1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(L.args.C, L.grid_y, 1);
  cfg.blockDim = dim3(L.threads, 1, 1);
  cfg.dynamicSmemBytes = L.smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = L.args.C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return n;
}

cudaError_t fused_launch(const FusedLaunch& L, const void* in, void* out, cudaStream_t stream) {
  KernelFn k = pick_kernel(L);
  if (!k) return cudaErrorInvalidConfiguration;
  FusedArgs a = L.args;
  a.in = in;
  a.out = out;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.vsplit > 1 ? a.vsplit : a.C, L.grid_y, 1);
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
  return cudaLaunchKernelEx(&cfg, k, a);
}

}  // namespace adfft
