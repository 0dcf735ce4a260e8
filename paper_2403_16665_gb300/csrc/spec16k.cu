// Compile-time shapes of the real fp32 classes with a packed sub-FFT of 16384
// points and one residue per CTA (512 threads, first pass of radix 4, three
// radix-16 passes), for P = 3, 4, 5, 6, 8, 16 residues: N = 32768 or 65536 with
// alpha = 2 .. 8 (ragged batches of the 2^8 .. 2^16 sample mix).  Forward and
// adjoint kernels; a separate translation unit so that it compiles in parallel.
#include "adfft_internal.h"
#include "adjoint.cuh"

namespace adfft {

namespace {

template <int P>
using Shape16k = Shape<14, 1, P, 512, 2, 5, 5, 2, 1>;   // full-spectrum output

template <int P>
using Shape16kHalf = Shape<14, 1, P, 512, 2, 5, 5, 2, 2>;   // half-spectrum output

template <int P>
using AdjShape16k = Shape<14, 1, P, 512, 2, 5, 0, 2>;

bool is_16k(const FusedLaunch& L) {
  const FusedArgs& a = L.args;
  return !L.dbl && L.mode == kLoadRealPacked && L.r0 == 4 && a.logNp == 14 && a.RPC == 1 && L.threads == 512 &&
         a.Mt == 2 * a.Mc;
}

}  // namespace

SpecKernel spec16k_forward(const FusedLaunch& L) {
  if (!is_16k(L)) return nullptr;
  if (L.args.half) {
    switch (L.args.P) {
      case 3: return fused_forward_kernel<float2, kLoadRealPacked, 32, 4, 0, Shape16kHalf<3>>;
      case 4: return fused_forward_kernel<float2, kLoadRealPacked, 32, 4, 0, Shape16kHalf<4>>;
      case 5: return fused_forward_kernel<float2, kLoadRealPacked, 32, 4, 0, Shape16kHalf<5>>;
      case 6: return fused_forward_kernel<float2, kLoadRealPacked, 32, 4, 0, Shape16kHalf<6>>;
      case 8: return fused_forward_kernel<float2, kLoadRealPacked, 32, 4, 0, Shape16kHalf<8>>;
      case 16: return fused_forward_kernel<float2, kLoadRealPacked, 32, 4, 0, Shape16kHalf<16>>;
      default: return nullptr;
    }
  }
  switch (L.args.P) {
    case 3: return fused_forward_kernel<float2, kLoadRealPacked, 32, 4, 0, Shape16k<3>>;
    case 4: return fused_forward_kernel<float2, kLoadRealPacked, 32, 4, 0, Shape16k<4>>;
    case 5: return fused_forward_kernel<float2, kLoadRealPacked, 32, 4, 0, Shape16k<5>>;
    case 6: return fused_forward_kernel<float2, kLoadRealPacked, 32, 4, 0, Shape16k<6>>;
    case 8: return fused_forward_kernel<float2, kLoadRealPacked, 32, 4, 0, Shape16k<8>>;
    case 16: return fused_forward_kernel<float2, kLoadRealPacked, 32, 4, 0, Shape16k<16>>;
    default: return nullptr;
  }
}

SpecKernel spec16k_adjoint(const FusedLaunch& L) {
  if (!is_16k(L)) return nullptr;
  switch (L.args.P) {
    case 3: return adjoint_kernel<float2, kLoadRealPacked, 32, 4, AdjShape16k<3>>;
    case 4: return adjoint_kernel<float2, kLoadRealPacked, 32, 4, AdjShape16k<4>>;
    case 5: return adjoint_kernel<float2, kLoadRealPacked, 32, 4, AdjShape16k<5>>;
    case 6: return adjoint_kernel<float2, kLoadRealPacked, 32, 4, AdjShape16k<6>>;
    case 8: return adjoint_kernel<float2, kLoadRealPacked, 32, 4, AdjShape16k<8>>;
    case 16: return adjoint_kernel<float2, kLoadRealPacked, 32, 4, AdjShape16k<16>>;
    default: return nullptr;
  }
}

}  // namespace adfft
