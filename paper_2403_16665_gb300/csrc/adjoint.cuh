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

// SH: compile-time shape (as for the forward kernel), or RuntimeShape.
template <typename V, int MODE, int VPT, int R0, class SH = RuntimeShape>
__global__ void __launch_bounds__(512) adjoint_kernel(const FusedArgs a) {
  using Rl = typename real_of<V>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int esz = (int)sizeof(V);
  const int tw_n = a.tw_lo_n + a.tw_hi_n;
  const int region = SH::region(a);
  const FusedSmem L = fused_smem_layout(tw_n, 0, SH::rpc(a), region, esz);
  V* tw_s = reinterpret_cast<V*>(smem_raw + L.tw);
  V* buf = reinterpret_cast<V*>(smem_raw + L.buf);
  for (int i = threadIdx.x; i < tw_n; i += blockDim.x) tw_s[i] = reinterpret_cast<const V*>(a.tw)[i];
  __syncthreads();
  TwTable<V> tab{tw_s, tw_s + a.tw_lo_n, a.tw_bits, (1u << a.tw_bits) - 1u};
  // the first signal's prologue stores into the other CTAs' shared memory: every CTA of
  // the cluster must be running before any CTA accesses another's shared memory
  if (a.C > 1) {
    cluster_arrive();
    cluster_wait();
  }

  const int c = (int)blockIdx.x;
  const int r0 = c * SH::rpc(a);
  const unsigned T = (unsigned)SH::threads();
  const unsigned P = (unsigned)SH::p(a);
  const unsigned Np = (unsigned)SH::Np(a);
  const unsigned Mc = (unsigned)a.Mc;
  const unsigned Mt = SH::mt(a);
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

    // ---- prologue: conj of the (folded) spectrum into the residue regions.  The CTAs
    // of the cluster split the bins j between them and read them coalesced (packed real
    // input: j <= Mc/2 together with the partners j + Mc, M - j, Mc - j, which give both
    // ub_j and ub_{Mc-j}); each value goes to the region of residue j mod P, k = j / P,
    // in whichever CTA holds it (distributed shared memory).
    if (a.C > 1 && sig != (long long)blockIdx.y) cluster_wait();
    if constexpr (MODE == kColumns) {
      const unsigned total = (unsigned)SH::rpc(a) * Np;
      for (unsigned t0 = threadIdx.x; t0 < total; t0 += T * UNR) {
        V val[UNR];
#pragma unroll
        for (int e = 0; e < UNR; ++e) {
          const unsigned t = t0 + e * T;
          if (t < total) {
            const unsigned rl = t >> a.logNp, k = t & (Np - 1);
            val[e] = g[k * P + (unsigned)(r0 + rl)];
          }
        }
#pragma unroll
        for (int e = 0; e < UNR; ++e) {
          const unsigned t = t0 + e * T;
          if (t < total) {
            const unsigned rl = t >> a.logNp, k = t & (Np - 1);
            buf[rl * region + SH::pad((int)k)] = cconj(val[e]);
          }
        }
      }
      __syncthreads();
    } else {
      const unsigned jt = (MODE == kLoadRealPacked) ? Mc / 2 + 1 : Mc;
      const unsigned perj = (jt + (unsigned)a.C - 1) / (unsigned)a.C;
      const unsigned ja = (unsigned)c * perj, jb = min(jt, ja + perj);
      const unsigned RPCu = (unsigned)SH::rpc(a);
      // shared::cluster address of element k of residue r
      auto slot = [&](unsigned r, unsigned k) -> uint32_t {
        const unsigned owner = SH::fixed ? r / RPCu : fdiv(r, a.divRPC);
        return dsmem_addr(buf + (r - owner * RPCu) * region + SH::pad((int)k), owner);
      };
      // bins per thread and pass (loads in flight, bounded by registers)
      constexpr int UP = (MODE == kLoadRealPacked) ? (sizeof(V) == 16 ? 1 : 2) : UNR;
      for (unsigned j0 = ja + threadIdx.x; j0 < jb; j0 += T * UP) {
        if constexpr (MODE == kLoadRealPacked) {
          const unsigned long long M = (unsigned long long)a.M;
          V g0[UP], g1[UP], g2[UP], g3[UP];
#pragma unroll
          for (int e = 0; e < UP; ++e) {
            const unsigned j = j0 + e * T;
            if (j < jb) {
              g0[e] = g[j];
              g3[e] = g[Mc - j];        // g_{Mc-j} (g_Mc for j = 0)
              if (a.half) {
                // half-spectrum plans: the bins above M/2 are not part of the map (zero)
                g1[e] = j == 0 ? g3[e] : czero<V>();
                g2[e] = j == 0 ? g0[e] : czero<V>();
              } else {
                g1[e] = g[j + Mc];
                g2[e] = g[(M - j) % M];   // g_{M-j} (g_0 for j = 0)
              }
            }
          }
#pragma unroll
          for (int e = 0; e < UP; ++e) {
            const unsigned j = j0 + e * T;
            if (j < jb) {
              // ub_j = (h_j + h_{j+Mc}) + i W_M^{-j} (h_j - h_{j+Mc}), h_m = (g_m + conj g_{M-m}) / 2
              {
                const V h0 = cscale(cadd(g0[e], cconj(g2[e])), (Rl)0.5);
                const V h1 = cscale(cadd(g1[e], cconj(g3[e])), (Rl)0.5);
                const V d = cmulc(csub(h0, h1), tab(j));
                const unsigned q = SH::fixed ? j / P : fdiv(j, a.divP);
                dsmem_st(slot(j - q * P, q), cconj(cadd(cadd(h0, h1), cmul_pi(d))));
              }
              if (j != 0 && 2 * j != Mc) {
                // ub_{Mc-j}: the same four bins in the roles (g_{Mc-j}, g_{M-j}, g_{j+Mc}, g_j)
                const unsigned jm = Mc - j;
                const V h0 = cscale(cadd(g3[e], cconj(g1[e])), (Rl)0.5);
                const V h1 = cscale(cadd(g2[e], cconj(g0[e])), (Rl)0.5);
                const V d = cmulc(csub(h0, h1), tab(jm));
                const unsigned q = SH::fixed ? jm / P : fdiv(jm, a.divP);
                dsmem_st(slot(jm - q * P, q), cconj(cadd(cadd(h0, h1), cmul_pi(d))));
              }
            }
          }
        } else {
          V v[UP];
#pragma unroll
          for (int e = 0; e < UP; ++e) {
            const unsigned j = j0 + e * T;
            if (j < jb) v[e] = g[j];
          }
#pragma unroll
          for (int e = 0; e < UP; ++e) {
            const unsigned j = j0 + e * T;
            if (j < jb) {
              const unsigned q = SH::fixed ? j / P : fdiv(j, a.divP);
              dsmem_st(slot(j - q * P, q), cconj(v[e]));
            }
          }
        }
      }
      // every CTA's stores have landed before the transforms read them
      if (a.C > 1) { cluster_arrive(); cluster_wait(); } else { __syncthreads(); }
    }

    // ---- inverse FFTs: forward Stockham passes on the conjugated data
    {
      int Ns = 1, logNs = 0;
      if constexpr (R0 > 1) {
        stockham_pass<R0, VPT, V, SH>(a, buf, tab, Ns, logNs);
        Ns = R0;
        logNs = LOGR0;
      }
      if constexpr (SH::fixed) {
#pragma unroll
        for (int p = 1; p < SH_PASSES<SH, LOGR0>::value; ++p) {
          stockham_pass<16, VPT, V, SH>(a, buf, tab, Ns, logNs);
          Ns <<= 4;
          logNs += 4;
        }
      } else {
        for (int p = 1; p < a.nrad; ++p) {
          stockham_pass<16, VPT, V, SH>(a, buf, tab, Ns, logNs);
          Ns <<= 4;
          logNs += 4;
        }
      }
    }

    // ---- reduction over residues for this CTA's range of n: the P residue values of an n
    // are loaded in groups of 8 (fp64: 2), all in flight, before they are summed
    if (a.C > 1) { cluster_arrive(); cluster_wait(); } else { __syncthreads(); }
    {
      const unsigned RPCu = (unsigned)SH::rpc(a);
      constexpr int G = sizeof(V) == 16 ? 2 : 8;    // residue values in flight per n
      constexpr int NH = 1;                          // values of n per thread
      for (unsigned nb = n0 + threadIdx.x; nb < n1; nb += NH * T) {
        V acc[NH], w[NH], wr[NH];
        unsigned nn[NH];
#pragma unroll
        for (int h = 0; h < NH; ++h) {
          acc[h] = czero<V>();
          nn[h] = nb + h * T;
          // conj(W_Mc^{r n}) = conj(W_Mt^{s r n}); w = W_Mt^{s n}, powers by products
          w[h] = tab((unsigned)(((unsigned long long)s * min(nn[h], n1 - 1)) % Mt));
        }
        for (unsigned rb = 0; rb < P; rb += G) {
          V y[NH][G];
#pragma unroll
          for (int h = 0; h < NH; ++h) {
            const unsigned np = nn[h] & (Np - 1);
#pragma unroll
            for (int u = 0; u < G; ++u) {
              const unsigned r = rb + u;
              if (r < P && nn[h] < n1) {
                const unsigned owner = SH::fixed ? r / RPCu : fdiv(r, a.divRPC);
                const V* src = buf + (r - owner * RPCu) * region + SH::pad((int)np);
                y[h][u] = (a.C > 1) ? dsmem_ld(dsmem_addr(src, owner), V{}) : *src;
              }
            }
          }
#pragma unroll
          for (int h = 0; h < NH; ++h) {
            // anchor the power chain on an exact table entry at the start of each group
            wr[h] = tab((unsigned)(((unsigned long long)s * rb * min(nn[h], n1 - 1)) % Mt));
#pragma unroll
            for (int u = 0; u < G; ++u) {
              if (rb + u < P) {
                // the buffer holds FFT(conj .) = conj(IFFT(.)): IFFT value = conj(y)
                acc[h] = cadd(acc[h], cmulc(cconj(y[h][u]), wr[h]));
                wr[h] = cmul(wr[h], w[h]);
              }
            }
          }
        }
#pragma unroll
        for (int h = 0; h < NH; ++h) {
          const unsigned n = nn[h];
          if (n >= n1) continue;
          const V v = cscale(acc[h], S);
          unsigned char* obase = reinterpret_cast<unsigned char*>(a.out);
          if (MODE == kLoadRealPlain) {
            reinterpret_cast<Rl*>(obase + sig_in_bytes(a, sig))[n] = v.x;
          } else if (MODE == kColumns) {
            // transpose of the two-pass first pass: column (sig mod cols) of the core, stride cols
            reinterpret_cast<V*>(obase + sig_in_bytes(a, sig / a.cols))[(sig % a.cols) + (long long)n * a.cols] = v;
          } else {
            reinterpret_cast<V*>(obase + sig_in_bytes(a, sig))[n] = v;
          }
        }
      }
    }
    if (a.C > 1) cluster_arrive_relaxed(); else __syncthreads();
  }
  if (a.C > 1 && (long long)blockIdx.y < a.batch) cluster_wait();
}

}  // namespace adfft
