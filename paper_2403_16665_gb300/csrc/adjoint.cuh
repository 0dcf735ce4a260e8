// Single-pass adjoint (conjugate transpose) of the alpha-DFT, the backward
// pass of the forward transform:
//
//     xb_n = S * sum_{m<M} exp(+2 pi i m n / M) g_m        (complex input)
//     xb_n = Re of the same                                 (real input)
//
// With the fold decomposition of the forward (m = P k + r, n = n' + Np f):
//     xb_{n'+Np f} = S sum_r conj(W_Mc^{r (n' + Np f)}) * IFFT_Np(g_r)[n'],
//     g_r[k] = g_{P k + r},  IFFT unnormalised (positive exponent).
// For packed real input the Hermitian part h_m = (g_m + conj g_{M-m})/2 is
// folded into the length-Mc complex spectrum
//     ub_j = (h_j + h_{j+Mc}) + i W_M^{-j} (h_j - h_{j+Mc}),   j < Mc,
// whose complex adjoint y (length Nc) carries xb_{2n} = S Re y_n and
// xb_{2n+1} = S Im y_n, so y is stored as the interleaved real output.
//
// One cluster of C CTAs owns one signal: CTA c gathers its residues of g
// (prologue), runs the inverse FFTs as conj(FFT(conj(.))) with the forward
// Stockham passes, and after a cluster barrier reduces over all P residues
// through distributed shared memory for a contiguous range of n.
#pragma once

#include "fused.cuh"

namespace adfft {

template <typename V, int MODE, int VPT, int R0>
__global__ void __launch_bounds__(512) adjoint_kernel(const FusedArgs a) {
  using Rl = typename real_of<V>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int esz = (int)sizeof(V);
  const int tw_n = a.tw_lo_n + a.tw_hi_n;
  const FusedSmem L = fused_smem_layout(tw_n, 0, a.RPC, a.region, esz);
  V* tw_s = reinterpret_cast<V*>(smem_raw + L.tw);
  V* buf = reinterpret_cast<V*>(smem_raw + L.buf);
  for (int i = threadIdx.x; i < tw_n; i += blockDim.x) tw_s[i] = reinterpret_cast<const V*>(a.tw)[i];
  __syncthreads();
  TwTable<V> tab{tw_s, tw_s + a.tw_lo_n, a.tw_bits, (1u << a.tw_bits) - 1u};

  cg::cluster_group cluster = cg::this_cluster();
  const int c = (int)blockIdx.x;
  const int r0 = c * a.RPC;
  const unsigned T = blockDim.x;
  const unsigned P = (unsigned)a.P;
  const unsigned Np = (unsigned)a.Np;
  const unsigned Mc = (unsigned)a.Mc;
  const unsigned Mt = (unsigned)a.Mt;
  const unsigned s = Mt / Mc;
  const Rl S = (Rl)a.scale;
  constexpr int LOGR0 = R0 == 1 ? 0 : R0 == 2 ? 1 : R0 == 4 ? 2 : R0 == 8 ? 3 : R0 == 16 ? 4 : 5;
  constexpr int UNR = 4;

  // this CTA's range of output samples n of the complex core
  const unsigned Nc = (unsigned)a.Nc;
  const unsigned per = (Nc + a.C - 1) / a.C;
  const unsigned n0 = c * per;
  const unsigned n1 = min(Nc, n0 + per);

  for (long long sig = blockIdx.y; sig < a.batch; sig += gridDim.y) {
    const V* g = reinterpret_cast<const V*>(a.in) + ((MODE == kColumns) ? sig * a.M : sig_out_off(a, sig));

    // ---- prologue: conj of the CTA's residues of the (folded) spectrum, natural order
    if (a.C > 1 && sig != (long long)blockIdx.y) cluster_wait();
    const unsigned total = (unsigned)a.RPC * Np;
    for (unsigned t0 = threadIdx.x; t0 < total; t0 += T * UNR) {
      V val[UNR];
#pragma unroll
      for (int e = 0; e < UNR; ++e) {
        const unsigned t = t0 + e * T;
        if (t < total) {
          const unsigned rl = t >> a.logNp, k = t & (Np - 1);
          const unsigned j = k * P + (unsigned)(r0 + rl);
          if (MODE == kLoadRealPacked) {
            const unsigned long long M = (unsigned long long)a.M;
            const V g0 = g[j];
            const V g1 = g[j + Mc];
            const V g2 = g[(M - j) % M];                 // g_{M-j} (g_0 for j = 0)
            const V g3 = g[Mc - j];                      // g_{Mc-j} (g_Mc for j = 0)
            const V h0 = cscale(cadd(g0, cconj(g2)), (Rl)0.5);  // h_j
            const V h1 = cscale(cadd(g1, cconj(g3)), (Rl)0.5);  // h_{j+Mc}
            const V d = cmulc(csub(h0, h1), tab(j));            // W_M^{-j} (h_j - h_{j+Mc})
            val[e] = cadd(cadd(h0, h1), cmul_pi(d));
          } else {
            val[e] = g[j];
          }
        }
      }
#pragma unroll
      for (int e = 0; e < UNR; ++e) {
        const unsigned t = t0 + e * T;
        if (t < total) {
          const unsigned rl = t >> a.logNp, k = t & (Np - 1);
          buf[rl * a.region + pad16((int)k)] = cconj(val[e]);
        }
      }
    }
    __syncthreads();

    // ---- inverse FFTs: forward Stockham passes on the conjugated data
    {
      int Ns = 1, logNs = 0;
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

    // ---- reduction over residues for this CTA's range of n
    if (a.C > 1) { cluster_arrive(); cluster_wait(); } else { __syncthreads(); }
    for (unsigned n = n0 + threadIdx.x; n < n1; n += T) {
      const unsigned np = n & (Np - 1);
      // conj(W_Mc^{r n}) = conj(W_Mt^{s r n}); w = W_Mt^{s n}, powers by products
      const unsigned e1 = (unsigned)(((unsigned long long)s * n) % Mt);
      const V w = tab(e1);
      V wr = cmake<V>(1, 0);
      V acc = czero<V>();
      for (unsigned r = 0; r < P; ++r) {
        const unsigned owner = r / (unsigned)a.RPC, rl = r - owner * (unsigned)a.RPC;
        const V* src = buf + rl * a.region + pad16((int)np);
        const V y = (a.C > 1) ? *cluster.map_shared_rank(src, owner) : *src;
        // the buffer holds FFT(conj .) = conj(IFFT(.)): IFFT value = conj(y)
        acc = cadd(acc, cmulc(cconj(y), wr));
        if ((r & 7u) == 7u) {
          // re-anchor the power chain every 8 steps on an exact table entry
          wr = tab((unsigned)(((unsigned long long)s * (r + 1) * n) % Mt));
        } else {
          wr = cmul(wr, w);
        }
      }
      acc = cscale(acc, S);
      unsigned char* obase = reinterpret_cast<unsigned char*>(a.out);
      if (MODE == kLoadRealPlain) {
        reinterpret_cast<Rl*>(obase + sig_in_bytes(a, sig))[n] = acc.x;
      } else if (MODE == kColumns) {
        // transpose of the two-pass first pass: column (sig mod cols) of the core, stride cols
        reinterpret_cast<V*>(obase + sig_in_bytes(a, sig / a.cols))[(sig % a.cols) + (long long)n * a.cols] = acc;
      } else {
        reinterpret_cast<V*>(obase + sig_in_bytes(a, sig))[n] = acc;
      }
    }
    if (a.C > 1) cluster_arrive_relaxed(); else __syncthreads();
  }
  if (a.C > 1 && (long long)blockIdx.y < a.batch) cluster_wait();
}

}  // namespace adfft
