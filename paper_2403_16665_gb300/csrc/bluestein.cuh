// Chirp-z (Bluestein) evaluation of the alpha-DFT, for any N and M = alpha N.
//
// With m n = (m^2 + n^2 - (m - n)^2) / 2 and the chirp c_j = W_{2M}^{j^2}
// = exp(-pi i j^2 / M):
//     X_m = S c_m sum_{n<N} (x_n c_n) conj(c_{m-n}).
// The output is produced in chunks of B bins [m0, m0 + B): with the chirp
// segment hs[i] = conj(c_{m0 - (N-1) + i}), i < N + B - 1, the linear
// convolution needed for the chunk equals the length-L circular convolution
// (L >= N + B - 1) of a = x c (zero padded) with hs, read at t + N - 1:
//     X_{m0+t} = S c_{m0+t} IFFT_L( FFT_L(a) * FFT_L(hs) )[t + N - 1].
// FFT_L(hs)/L is precomputed per chunk on the host in double precision.
//
// One CTA per (signal, chunk): it forms a in shared memory, runs the forward
// Stockham FFT, multiplies by the chunk's kernel spectrum, runs the inverse
// FFT as conj(FFT(conj(.))), and writes the chunk's B bins contiguously.
#pragma once

#include "fused.cuh"

namespace adfft {

struct BluesteinArgs {
  FusedArgs f;          // FFT view: Np = L, RPC = 1, Mt = L, tw = W_L table, region, nrad
  const void* chirp;    // c_j, j < max(N, M)
  const void* H;        // chunks x L kernel spectra (already divided by L)
  long long N;          // samples per signal
  int B, chunks;        // bins per chunk, chunks per signal
  int real_in;          // input is real (read as complex with zero imaginary part)
};

template <typename V, int VPT, int R0>
__device__ __forceinline__ void run_all_passes(const FusedArgs& a, V* buf, const TwTable<V>& tab) {
  int Ns = 1, logNs = 0;
  constexpr int LOGR0 = R0 == 1 ? 0 : R0 == 2 ? 1 : R0 == 4 ? 2 : R0 == 8 ? 3 : 4;
  if constexpr (R0 > 1) {
    stockham_pass<R0, VPT, V>(a, buf, tab, Ns, logNs);
    Ns = R0;
    logNs = LOGR0;
  }
  for (int p = 1; p < a.nrad; ++p) {
    stockham_pass<16, VPT, V>(a, buf, tab, Ns, logNs);
    Ns <<= 4;
    logNs += 4;
  }
}

template <typename V, int VPT, int R0>
__global__ void __launch_bounds__(512) bluestein_kernel(const BluesteinArgs b) {
  using Rl = typename real_of<V>::type;
  const FusedArgs& a = b.f;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tw_n = a.tw_lo_n + a.tw_hi_n;
  const FusedSmem L = fused_smem_layout(tw_n, 0, 1, a.region, (int)sizeof(V));
  V* tw_s = reinterpret_cast<V*>(smem_raw + L.tw);
  V* buf = reinterpret_cast<V*>(smem_raw + L.buf);
  for (int i = threadIdx.x; i < tw_n; i += blockDim.x) tw_s[i] = reinterpret_cast<const V*>(a.tw)[i];
  __syncthreads();
  TwTable<V> tab{tw_s, tw_s + a.tw_lo_n, a.tw_bits, (1u << a.tw_bits) - 1u};

  const unsigned Lf = (unsigned)a.Np;
  const unsigned T = blockDim.x;
  const int chunk = (int)blockIdx.x;
  const long long m0 = (long long)chunk * b.B;
  const int nb = (int)min((long long)b.B, a.M - m0);
  const V* chirp = reinterpret_cast<const V*>(b.chirp);
  const V* H = reinterpret_cast<const V*>(b.H) + (size_t)chunk * Lf;
  const Rl S = (Rl)a.scale;

  for (long long sig = blockIdx.y; sig < a.batch; sig += gridDim.y) {
    // a_n = x_n c_n, zero padded to L
    for (unsigned i = threadIdx.x; i < Lf; i += T) {
      V v = czero<V>();
      if ((long long)i < b.N) {
        V x;
        const unsigned char* base = reinterpret_cast<const unsigned char*>(a.in) + sig_in_bytes(a, sig);
        if (b.real_in) x = cmake<V>(__ldg(reinterpret_cast<const Rl*>(base) + i), (Rl)0);
        else x = __ldg(reinterpret_cast<const V*>(base) + i);
        v = cmul(x, __ldg(chirp + i));
      }
      buf[pad16((int)i)] = v;
    }
    __syncthreads();
    run_all_passes<V, VPT, R0>(a, buf, tab);
    // times the chunk's kernel spectrum, conjugated for the inverse transform
    for (unsigned i = threadIdx.x; i < Lf; i += T) {
      const int p = pad16((int)i);
      buf[p] = cconj(cmul(buf[p], __ldg(H + i)));
    }
    __syncthreads();
    run_all_passes<V, VPT, R0>(a, buf, tab);
    V* out = reinterpret_cast<V*>(a.out) + sig_out_off(a, sig) + m0;
    for (int t = threadIdx.x; t < nb; t += T) {
      const V y = cconj(buf[pad16(t + (int)b.N - 1)]);
      out[t] = cscale(cmul(y, __ldg(chirp + m0 + t)), S);
    }
    __syncthreads();
  }
}

// Adjoint of the chirp-z evaluation (the backward pass of a chirp-z plan):
//     xb_n = S sum_{m<M} conj(W_M^{mn}) g_m = S conj(c_n) sum_m (g_m conj(c_m)) c_{n-m},
// (conj W_M^{mn} = conj(c_m) conj(c_n) c_{m-n}, and c is even), i.e. the convolution of
// b_m = g_m conj(c_m) (length M) with the chirp itself, read at n < N.  The input is cut
// into blocks of Bi bins [m0, m0 + Bi) and the output into chunks of Bo samples
// [n0, n0 + Bo); with the chirp segment v_i = c_{n0 - m0 - (Bi-1) + i}, i < Bi + Bo - 1,
// a block contributes (u * v)[t + Bi - 1] to output n0 + t (u the block of b), which is
// the length-L circular convolution for L >= Bi + Bo - 1.  FFT_L(v)/L depends on
// n0 - m0 only and is precomputed per difference on the host in double precision.
// One CTA per (signal, output chunk) runs every input block in turn and accumulates its
// chunk in registers; then xb_{n0+t} = S conj(c_{n0+t}) acc_t (its real part for real
// input).
struct BluesteinAdjArgs {
  FusedArgs f;          // FFT view: Np = L, RPC = 1, Mt = L, tw = W_L table, region, nrad
  const void* chirp;    // c_j, j < max(N, M)
  const void* H;        // (nI + nO - 1) x L kernel spectra (divided by L), index o - i + nI - 1
  long long N;          // output samples per signal
  int Bi, Bo, nI, nO;   // input block, output chunk, their counts
  int real_out;         // real input plan: write the real part
};

template <typename V, int VPT, int R0, int ACC>
__global__ void __launch_bounds__(512) bluestein_adjoint_kernel(const BluesteinAdjArgs b) {
  using Rl = typename real_of<V>::type;
  const FusedArgs& a = b.f;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tw_n = a.tw_lo_n + a.tw_hi_n;
  const FusedSmem L = fused_smem_layout(tw_n, 0, 1, a.region, (int)sizeof(V));
  V* tw_s = reinterpret_cast<V*>(smem_raw + L.tw);
  V* buf = reinterpret_cast<V*>(smem_raw + L.buf);
  for (int i = threadIdx.x; i < tw_n; i += blockDim.x) tw_s[i] = reinterpret_cast<const V*>(a.tw)[i];
  __syncthreads();
  TwTable<V> tab{tw_s, tw_s + a.tw_lo_n, a.tw_bits, (1u << a.tw_bits) - 1u};

  const unsigned Lf = (unsigned)a.Np;
  const unsigned T = blockDim.x;
  const int o = (int)blockIdx.x;
  const long long n0 = (long long)o * b.Bo;
  const int nb = (int)min((long long)b.Bo, b.N - n0);
  const long long M = a.M;
  const V* chirp = reinterpret_cast<const V*>(b.chirp);
  const Rl S = (Rl)a.scale;

  for (long long sig = blockIdx.y; sig < a.batch; sig += gridDim.y) {
    const V* g = reinterpret_cast<const V*>(a.in) + sig_out_off(a, sig);
    V acc[ACC];
#pragma unroll
    for (int e = 0; e < ACC; ++e) acc[e] = czero<V>();
    for (int i = 0; i < b.nI; ++i) {
      const long long m0 = (long long)i * b.Bi;
      const long long mb = min((long long)b.Bi, M - m0);
      // u_s = g_{m0+s} conj(c_{m0+s}), zero padded to L
      for (unsigned idx = threadIdx.x; idx < Lf; idx += T) {
        V v = czero<V>();
        if ((long long)idx < mb) v = cmulc(__ldg(g + m0 + idx), __ldg(chirp + m0 + idx));
        buf[pad16((int)idx)] = v;
      }
      __syncthreads();
      run_all_passes<V, VPT, R0>(a, buf, tab);
      const V* H = reinterpret_cast<const V*>(b.H) + (size_t)(o - i + b.nI - 1) * Lf;
      for (unsigned idx = threadIdx.x; idx < Lf; idx += T) {
        const int p = pad16((int)idx);
        buf[p] = cconj(cmul(buf[p], __ldg(H + idx)));
      }
      __syncthreads();
      run_all_passes<V, VPT, R0>(a, buf, tab);
#pragma unroll
      for (int e = 0; e < ACC; ++e) {
        const int t = (int)threadIdx.x + e * (int)T;
        if (t < nb) acc[e] = cadd(acc[e], cconj(buf[pad16(t + b.Bi - 1)]));
      }
      __syncthreads();
    }
    const long long ob = a.offs ? a.offs[2 * sig] / a.in_unit : sig * b.N;
#pragma unroll
    for (int e = 0; e < ACC; ++e) {
      const int t = (int)threadIdx.x + e * (int)T;
      if (t < nb) {
        const V y = cscale(cmulc(acc[e], __ldg(chirp + n0 + t)), S);   // S conj(c_n) acc
        if (b.real_out) reinterpret_cast<Rl*>(a.out)[ob + n0 + t] = y.x;
        else reinterpret_cast<V*>(a.out)[ob + n0 + t] = y;
      }
    }
  }
}

}  // namespace adfft
