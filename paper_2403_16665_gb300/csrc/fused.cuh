// Single-pass ("fused") forward alpha-DFT for sub-FFT lengths that fit in the
// shared memory of one thread-block cluster.
//
// Decomposition (Sec. 3 rewritten in decimation-in-frequency order; see adfft.h):
//   u      : the input as Nc complex elements (real input: u_n = x_{2n} + i x_{2n+1})
//   Mc     : bins of the complex transform of u (Mc = M, or M/2 for packed real input)
//   g = Np : gcd(Mc, Nc), the sub-FFT length (a power of two here)
//   P, q   : Mc/Np residues, Nc/Np fold factor
//   U_{P k + r} = FFT_Np(z_r)[k],   z_r[n] = sum_{f<q} u_{n+f Np} W_Mc^{r (n + f Np)}
// Real input is unpacked in the epilogue:
//   E_j = (U_j + conj U_{Mc-j})/2,  O_j = (U_j - conj U_{Mc-j})/(2i),
//   X_j = E_j + W_M^j O_j,  X_{j+Mc} = E_j - W_M^j O_j,  X_{M-j} = conj X_j.
//
// One cluster of C CTAs owns one signal at a time; CTA c holds residues
// [c*RPC, (c+1)*RPC) of it in shared memory.  Pass 1 (K1) folds and twiddles
// the input straight from global memory into its first radix-R butterfly;
// the remaining Stockham passes (K2) run in shared memory; the epilogue (K3)
// gathers U across the cluster through distributed shared memory so that each
// CTA writes a contiguous, coalesced range of output bins in natural order.
#pragma once

#include <cooperative_groups.h>

#include "fft_device.cuh"

namespace adfft {

namespace cg = cooperative_groups;

// How the kernel reads its input.
enum LoadMode : int {
  kLoadComplex = 0,      // complex input, u = x
  kLoadRealPacked = 1,   // real input, two samples per complex element, unpacked in the epilogue
  kLoadRealPlain = 2     // real input read as complex with zero imaginary part (odd N or odd M)
};

struct FusedArgs {
  const void* in;
  void* out;
  long long batch;
  long long in_stride;   // input scalars (real) or complex elements per signal
  long long M;           // output bins per signal
  int Np, logNp;         // sub-FFT length
  int P, q;              // residues, fold factor
  int RPC, C;            // residues per CTA, CTAs per signal (cluster size)
  int Nc, Mc;            // complex input elements, complex bins
  int Mt;                // twiddle modulus: M for packed real input, Mc otherwise
  int tw_bits, tw_lo_n, tw_hi_n;
  const void* tw;        // lo table (2^tw_bits entries) followed by the hi table
  double scale;
  int region;            // complex elements per residue region in shared memory
  int nrad;              // passes: one of radix R0 (template argument), nrad-1 of radix 16
  FastDiv divP, divRPC;
};

template <typename V>
__device__ __forceinline__ V ld_in(const void* base, long long idx, int mode) {
  using R = typename real_of<V>::type;
  if (mode == kLoadRealPlain) return cmake<V>(__ldg(reinterpret_cast<const R*>(base) + idx), (R)0);
  return __ldg(reinterpret_cast<const V*>(base) + idx);
}

// Twiddles W_{Ns R}^{k i}, i = 1..R-1, applied to v[i] from one table lookup of
// w = W^k: w^(2h) = w^h * w^h, w^(h+l) = w^h * w^l (h the highest power of two
// below i), so no power is more than log2(R) + 1 products away from w.
__host__ __device__ constexpr int high_pow2(int i) { return (i & (i - 1)) == 0 ? i / 2 : (i >= 8 ? 8 : i >= 4 ? 4 : 2); }

template <int R, typename V, int i>
__device__ __forceinline__ void twiddle_powers(V* w, std::integral_constant<int, i>) {
  if constexpr (i < R) {
    constexpr int h = high_pow2(i);
    w[i] = cmul(w[h], w[i - h]);
    twiddle_powers<R, V>(w, std::integral_constant<int, i + 1>());
  }
}

template <int R, typename V>
__device__ __forceinline__ void apply_stage_twiddles(V* v, V w1) {
  if constexpr (R > 1) {
    V w[R];
    w[1] = w1;
    twiddle_powers<R, V>(w, std::integral_constant<int, 2>());
#pragma unroll
    for (int i = 1; i < R; ++i) v[i] = cmul(v[i], w[i]);
  }
}

// Pass 1 (Ns = 1): fold, residue twiddle and the first radix-R butterfly,
// reading u from global memory and writing the CTA's residue regions.
template <int R, typename V>
__device__ __forceinline__ void first_pass(const FusedArgs& a, const void* u, int mode, V* buf,
                                           const TwTable<V>& tab, int r0) {
  const int items = a.Np / R;
  const unsigned T = blockDim.x;
  const unsigned Mt = (unsigned)a.Mt;
  const unsigned s = (unsigned)(a.Mt / a.Mc);
  for (int rl = 0; rl < a.RPC; ++rl) {
    const unsigned long long sr = (unsigned long long)s * (unsigned)(r0 + rl);
    const unsigned d_i = (unsigned)((sr * (unsigned)items) % Mt);
    const unsigned d_f = (unsigned)((sr * (unsigned)a.Np) % Mt);
    const unsigned d_T = (unsigned)((sr * T) % Mt);
    unsigned e_j = (unsigned)((sr * threadIdx.x) % Mt);
    V* dst = buf + rl * a.region;
    for (int j = threadIdx.x; j < items; j += T) {
      V acc[R];
#pragma unroll
      for (int i = 0; i < R; ++i) acc[i] = czero<V>();
      unsigned e_f = e_j;
      for (int f = 0; f < a.q; ++f) {
        unsigned e = e_f;
        const long long nb = (long long)j + (long long)f * a.Np;
#pragma unroll
        for (int i = 0; i < R; ++i) {
          const V x = ld_in<V>(u, nb + (long long)i * items, mode);
          const V w = tab(e);
          acc[i] = cadd(acc[i], cmul(x, w));
          e += d_i;
          if (e >= Mt) e -= Mt;
        }
        e_f += d_f;
        if (e_f >= Mt) e_f -= Mt;
      }
      DFT<R, V>::run(acc);
#pragma unroll
      for (int i = 0; i < R; ++i) dst[pad16(j * R + i)] = acc[i];
      e_j += d_T;
      if (e_j >= Mt) e_j -= Mt;
    }
  }
}

// One in-place Stockham pass of radix R over all residue regions of the CTA.
// Item (rl, j): reads elements j + i*Np/R, twiddles by W_{Ns R}^{(j mod Ns) i},
// runs DFT_R and writes to (j / Ns) * Ns * R + (j mod Ns) + i*Ns.
template <int R, int VPT, typename V>
__device__ __forceinline__ void stockham_pass(const FusedArgs& a, V* buf, const TwTable<V>& tab,
                                              int Ns, int logNs) {
  constexpr int IPT = VPT / R;
  constexpr int LOGR = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : R == 16 ? 4 : 5;
  const int log_items = a.logNp - LOGR;
  const int items_res = 1 << log_items;
  const int items = a.RPC * items_res;
  const int T = blockDim.x;
  const unsigned tw_step = (unsigned)a.Mt / ((unsigned)Ns << LOGR);   // Mt / (Ns R)
  V v[IPT][R];
#pragma unroll
  for (int it = 0; it < IPT; ++it) {
    const int w = threadIdx.x + it * T;
    if (w < items) {
      const int rl = w >> log_items;
      const int j = w & (items_res - 1);
      const V* src = buf + rl * a.region;
#pragma unroll
      for (int i = 0; i < R; ++i) v[it][i] = src[pad16(j + (i << log_items))];
      const int k = j & (Ns - 1);
      if (k != 0) apply_stage_twiddles<R>(v[it], tab((unsigned)k * tw_step));
      DFT<R, V>::run(v[it]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < IPT; ++it) {
    const int w = threadIdx.x + it * T;
    if (w < items) {
      const int rl = w >> log_items;
      const int j = w & (items_res - 1);
      const int k = j & (Ns - 1);
      const int base = ((j >> logNs) << (logNs + LOGR)) + k;
      V* dst = buf + rl * a.region;
#pragma unroll
      for (int i = 0; i < R; ++i) dst[pad16(base + i * Ns)] = v[it][i];
    }
  }
  __syncthreads();
}

// Address of U_idx (0 <= idx < Mc) in the cluster's shared memory.
template <typename V>
__device__ __forceinline__ const V* u_addr(const FusedArgs& a, const V* buf, unsigned idx,
                                           cg::cluster_group& cluster) {
  const unsigned k = fdiv(idx, a.divP);
  const unsigned r = idx - k * (unsigned)a.P;
  const unsigned owner = fdiv(r, a.divRPC);
  const unsigned rl = r - owner * (unsigned)a.RPC;
  const V* p = buf + rl * a.region + pad16((int)k);
  if (a.C > 1) return cluster.map_shared_rank(p, owner);
  return p;
}

// R0: radix of the first pass (1, 2, 4, 8 or 16); every later pass is radix 16.
template <typename V, int MODE, int VPT, int R0>
__global__ void __launch_bounds__(512) fused_forward_kernel(const FusedArgs a) {
  using Rl = typename real_of<V>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* tw_s = reinterpret_cast<V*>(smem_raw);
  const int tw_n = a.tw_lo_n + a.tw_hi_n;
  V* buf = tw_s + ((tw_n + 1) & ~1);
  for (int i = threadIdx.x; i < tw_n; i += blockDim.x) tw_s[i] = reinterpret_cast<const V*>(a.tw)[i];
  __syncthreads();
  TwTable<V> tab{tw_s, tw_s + a.tw_lo_n, a.tw_bits, (1u << a.tw_bits) - 1u};

  cg::cluster_group cluster = cg::this_cluster();
  const int c = (int)blockIdx.x;          // rank within the cluster (grid.x == C)
  const int r0 = c * a.RPC;
  const unsigned T = blockDim.x;
  const Rl S = (Rl)a.scale;
  constexpr int LOGR0 = R0 == 1 ? 0 : R0 == 2 ? 1 : R0 == 4 ? 2 : R0 == 8 ? 3 : 4;

  for (long long sig = blockIdx.y; sig < a.batch; sig += gridDim.y) {
    const void* u;
    if (MODE == kLoadComplex) u = reinterpret_cast<const V*>(a.in) + sig * a.in_stride;
    else u = reinterpret_cast<const Rl*>(a.in) + sig * a.in_stride;
    V* out = reinterpret_cast<V*>(a.out) + sig * a.M;

    // ---- K1: fold + residue twiddle + first radix
    first_pass<R0, V>(a, u, MODE, buf, tab, r0);
    __syncthreads();

    // ---- K2: radix-16 Stockham passes in shared memory
    int Ns = R0, logNs = LOGR0;
    for (int p = 1; p < a.nrad; ++p) {
      stockham_pass<16, VPT, V>(a, buf, tab, Ns, logNs);
      Ns <<= 4;
      logNs += 4;
    }

    // ---- K3: interleave epilogue through distributed shared memory
    if (a.C > 1) cluster.sync(); else __syncthreads();
    if (MODE == kLoadRealPacked) {
      const unsigned Mc = (unsigned)a.Mc;
      const unsigned total = Mc / 2 + 1;
      const unsigned per = (total + a.C - 1) / a.C;
      const unsigned j0 = c * per;
      const unsigned j1 = min(total, j0 + per);
      for (unsigned j = j0 + threadIdx.x; j < j1; j += T) {
        const unsigned jp = (j == 0) ? 0u : Mc - j;
        const V Uj = *u_addr<V>(a, buf, j, cluster);
        const V Ujp = *u_addr<V>(a, buf, jp, cluster);
        const V E = cscale(cadd(Uj, cconj(Ujp)), (Rl)0.5);
        const V O = cscale(cmul_mi(csub(Uj, cconj(Ujp))), (Rl)0.5);
        const V wO = cmul(tab(j), O);
        const V X1 = cscale(cadd(E, wO), S);
        const V X2 = cscale(csub(E, wO), S);
        out[j] = X1;
        out[j + Mc] = X2;
        if (j != 0 && 2 * j != Mc) {
          out[Mc - j] = cconj(X2);
          out[(unsigned long long)a.M - j] = cconj(X1);
        }
      }
    } else {
      const unsigned Mc = (unsigned)a.Mc;
      const unsigned per = (Mc + a.C - 1) / a.C;
      const unsigned m0 = c * per;
      const unsigned m1 = min(Mc, m0 + per);
      for (unsigned m = m0 + threadIdx.x; m < m1; m += T) out[m] = cscale(*u_addr<V>(a, buf, m, cluster), S);
    }
    if (a.C > 1) cluster.sync(); else __syncthreads();
  }
}

}  // namespace adfft
