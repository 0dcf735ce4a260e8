// Instantiations of the push-exchange forward kernel (fused_push.cuh): the real fp32
// classes whose packed sub-FFT runs in one CTA of 256 threads per residue.
#include "adfft_internal.h"
#include "fused_push.cuh"

namespace adfft {

namespace {

// packed sub-FFT 8192 (N = 16384), 8 residues (alpha = 8): the 4096 x 16384 workload
using PushR32N8192P8 = PushShape<13, 8, 256>;

template <class PS>
bool matches(const FusedLaunch& L) {
  const FusedArgs& a = L.args;
  return !L.dbl && L.mode == kLoadRealPacked && a.logNp == PS::LOGNP && a.P == PS::P && a.C == PS::P &&
         a.RPC == 1 && a.q == 1 && a.Mt == 2 * a.Mc && a.stage_bytes == 0;
}

}  // namespace

SpecKernel push_forward(const FusedLaunch& L) {
  if (matches<PushR32N8192P8>(L) && L.r0 == 32) return fused_push_kernel<PushR32N8192P8, 32>;
  return nullptr;
}

// Launch geometry of the push form for this launch (threads, dynamic shared memory), or
// false where no instantiation serves it.
bool push_geometry(const FusedLaunch& L, int* threads, size_t* smem) {
  if (matches<PushR32N8192P8>(L) && L.r0 == 32) {
    *threads = PushR32N8192P8::T;
    *smem = (size_t)push_smem_layout<PushR32N8192P8>(L.args.tw_lo_n + L.args.tw_hi_n).total;
    return true;
  }
  return false;
}

}  // namespace adfft
