// Second pass of the two-pass (four-step) form for sub-FFT lengths beyond one
// cluster's shared memory.
//
// With Nc = A B, n = B a + b and m = m1 + R1 m2 (R1 = alpha A, m1 < R1, m2 < B):
//     U_{m1 + R1 m2} = sum_b W_B^{m2 b} [ W_Mc^{m1 b} V_b[m1] ],
//     V_b[m1] = sum_a W_{R1}^{m1 a} u_{B a + b}     (an alpha-DFT of column b).
// The first pass (fused kernel, kColumns mode) writes the bracket to the
// scratch rows S[b][m1].  This pass runs the length-B DFTs over b for a block
// of columns m1 and for the mirror columns R1 - m1, and for packed real input
// unpacks (E_j, O_j) exactly as the single-pass epilogue:
//     X_j = E_j + W_M^j O_j,  X_{j+Mc} = E_j - W_M^j O_j,  X_{M-j} = conj X_j,
// where the partner Mc - j of j = m1 + R1 m2 is (R1 - m1) + R1 (B - 1 - m2)
// (m1 > 0) or R1 ((B - m2) mod B) (m1 = 0).  Consecutive lanes take
// consecutive m1, so every output row segment is written contiguously.
#pragma once

#include "fused.cuh"

namespace adfft {

struct TwoPassArgs {
  FusedArgs f;          // FFT view: Np = B, RPC = 2 W (columns), Mt = B, tw = W_B table, region, nrad
  const void* scratch;  // [batch][B][R1]
  void* out;            // [batch][M]
  long long batch;
  int B, logB;
  long long R1;         // row length alpha A
  long long Mc, M;
  int W;                // column pairs per CTA (4, 8 or 16: a power of two, as is B)
  int real_packed;
  const void* wM;       // two-level W_M table (global memory), for the real unpacking
  int wM_bits, wM_lo_n;
  double scale;
};

template <typename V>
__device__ __forceinline__ V tw_global(const void* t, int lo_n, int bits, unsigned long long e) {
  const V* lo = reinterpret_cast<const V*>(t);
  const V* hi = lo + lo_n;
  return cmul(__ldg(hi + (e >> bits)), __ldg(lo + (e & ((1ull << bits) - 1))));
}

template <typename V, int VPT, int R0, int PREC = 0>
__global__ void __launch_bounds__(512) twopass_columns_kernel(const TwoPassArgs t) {
  using Rl = typename real_of<V>::type;
  const FusedArgs& a = t.f;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tw_n = a.tw_lo_n + a.tw_hi_n;
  const FusedSmem L = fused_smem_layout(tw_n, 0, a.RPC, a.region, (int)sizeof(V));
  V* tw_s = reinterpret_cast<V*>(smem_raw + L.tw);
  V* buf = reinterpret_cast<V*>(smem_raw + L.buf);
  for (int i = threadIdx.x; i < tw_n; i += blockDim.x) tw_s[i] = reinterpret_cast<const V*>(a.tw)[i];
  __syncthreads();
  TwTable<V> tab{tw_s, tw_s + a.tw_lo_n, a.tw_bits, (1u << a.tw_bits) - 1u};

  const unsigned B = (unsigned)t.B;
  const unsigned W = (unsigned)t.W;
  const unsigned long long R1 = (unsigned long long)t.R1;
  const unsigned long long Mc = (unsigned long long)t.Mc;
  const unsigned npairs = (unsigned)(t.real_packed ? R1 / 2 + 1 : R1);
  const unsigned p0 = blockIdx.x * W;
  const unsigned np = min(W, npairs - p0);
  const unsigned T = blockDim.x;
  const Rl S = (Rl)t.scale;
  // columns 0..W-1: m1 = p0 + w;  W..2W-1: the mirrors (R1 - m1) mod R1
  const unsigned ncol = t.real_packed ? 2 * W : W;
  const unsigned lw = 31 - __clz(W), lncol = 31 - __clz(ncol);   // W, ncol: powers of two

  for (long long sig = blockIdx.y; sig < t.batch; sig += gridDim.y) {
    const V* src = reinterpret_cast<const V*>(t.scratch) + (size_t)sig * B * R1;
    // (8 loads in flight per thread before the shared-memory stores)
    constexpr int UL = 8;
    for (unsigned i0 = threadIdx.x; i0 < ncol * B; i0 += T * UL) {
      V v[UL];
#pragma unroll
      for (int e = 0; e < UL; ++e) {
        const unsigned idx = i0 + e * T;
        const unsigned w = idx & (ncol - 1), b = idx >> lncol;   // consecutive threads: consecutive columns
        v[e] = czero<V>();
        const unsigned pw = (w < W) ? w : w - W;
        if (idx < ncol * B && pw < np) {
          const unsigned long long m1 = p0 + pw;
          const unsigned long long col = (w < W) ? m1 : (m1 ? R1 - m1 : 0);
          v[e] = __ldg(src + (size_t)b * R1 + col);
        }
      }
#pragma unroll
      for (int e = 0; e < UL; ++e) {
        const unsigned idx = i0 + e * T;
        if (idx < ncol * B) buf[(idx & (ncol - 1)) * a.region + pad16((int)(idx >> lncol))] = v[e];
      }
    }
    __syncthreads();
    {
      int Ns = 1, logNs = 0;
      constexpr int LOGR0 = R0 == 1 ? 0 : R0 == 2 ? 1 : R0 == 4 ? 2 : R0 == 8 ? 3 : 4;
      if constexpr (R0 > 1) {
        stockham_pass<R0, VPT, V>(a, buf, tab, Ns, logNs);
        Ns = R0;
        logNs = LOGR0;
      }
      for (int p = 1; p < a.nrad; ++p) {
        radix16_pass<PREC, VPT, V>(a, buf, tab, Ns, logNs);
        Ns <<= 4;
        logNs += 4;
      }
    }
    V* out = reinterpret_cast<V*>(t.out) + (t.f.offs ? t.f.offs[2 * sig + 1] : sig * t.M);
    if (t.real_packed) {
      // item (pair w, m2): j = m1 + R1 m2 and its partner in the mirror column
      for (unsigned idx = threadIdx.x; idx < W * B; idx += T) {
        const unsigned w = idx & (W - 1), m2 = idx >> lw;
        if (w >= np) continue;
        const unsigned long long m1 = p0 + w;
        // columns 0 and R1/2 pair with themselves: only half of their m2 are leaders
        const bool self = (m1 == 0) || (2 * m1 == R1);
        if (self && 2 * m2 > B) continue;
        if (self && m1 != 0 && 2 * m2 == B) continue;
        const unsigned m2p = (m1 == 0) ? (B - m2) & (B - 1) : B - 1 - m2;
        const V Uj = buf[w * a.region + pad16((int)m2)];
        const V Up = buf[(W + w) * a.region + pad16((int)m2p)];
        const unsigned long long j = m1 + R1 * m2;
        const V E = cscale(cadd(Uj, cconj(Up)), (Rl)0.5);
        const V O = cscale(cmul_mi(csub(Uj, cconj(Up))), (Rl)0.5);
        const V wO = cmul(tw_global<V>(t.wM, t.wM_lo_n, t.wM_bits, j), O);
        const V X1 = cscale(cadd(E, wO), S);
        const V X2 = cscale(csub(E, wO), S);
        out[j] = X1;
        out[j + Mc] = X2;
        if (j != 0 && 2 * j != Mc) {
          out[Mc - j] = cconj(X2);
          out[(unsigned long long)t.M - j] = cconj(X1);
        }
      }
    } else {
      for (unsigned idx = threadIdx.x; idx < W * B; idx += T) {
        const unsigned w = idx & (W - 1), m2 = idx >> lw;
        if (w >= np) continue;
        const unsigned long long j = p0 + w + R1 * m2;
        out[j] = cscale(buf[w * a.region + pad16((int)m2)], S);
      }
    }
    __syncthreads();
  }
}

// Adjoint of the second pass (first step of the two-pass adjoint): for a block
// of columns m1, forms the (Hermitian-folded, for packed real input)
// spectrum ub_{m1 + R1 m2}, runs the inverse B-point DFT over m2 as
// conj(FFT(conj(.))), multiplies by conj(W_Mc^{m1 b}) and the scale S, and
// writes scratch row b.  The first pass's adjoint (adjoint kernel, kColumns
// mode) then takes the rows to the input samples u_{B a + b}.
// For packed real input the fold of bin j reads g_{M-j} and g_{Mc-j}, which lie
// in the mirror column (R1 - m1) mod R1; a CTA therefore takes W column pairs
// (m1 <= R1/2 in slots 0..W-1, the mirrors in slots W..2W-1, as the forward
// pass does), so that each spectrum value is fetched from HBM once and its
// second read hits in L2.  Columns 0 and R1/2 are their own mirrors and use
// only the first slot.
//   t.out     : the spectrum g [batch][M] (read), offsets from t.f.offs
//   t.scratch : [batch][B][R1] (written)
template <typename V, int VPT, int R0>
__global__ void __launch_bounds__(512) twopass_adjoint_columns_kernel(const TwoPassArgs t) {
  using Rl = typename real_of<V>::type;
  const FusedArgs& a = t.f;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tw_n = a.tw_lo_n + a.tw_hi_n;
  const FusedSmem L = fused_smem_layout(tw_n, 0, a.RPC, a.region, (int)sizeof(V));
  V* tw_s = reinterpret_cast<V*>(smem_raw + L.tw);
  V* buf = reinterpret_cast<V*>(smem_raw + L.buf);
  for (int i = threadIdx.x; i < tw_n; i += blockDim.x) tw_s[i] = reinterpret_cast<const V*>(a.tw)[i];
  __syncthreads();
  TwTable<V> tab{tw_s, tw_s + a.tw_lo_n, a.tw_bits, (1u << a.tw_bits) - 1u};

  const unsigned B = (unsigned)t.B;
  const unsigned W = (unsigned)t.W;
  const unsigned long long R1 = (unsigned long long)t.R1;
  const unsigned long long Mc = (unsigned long long)t.Mc;
  const unsigned long long M = (unsigned long long)t.M;
  const unsigned long long sM = M / Mc;   // W_Mc^e = W_M^{sM e}
  const unsigned npairs = (unsigned)(t.real_packed ? R1 / 2 + 1 : R1);
  const unsigned p0 = blockIdx.x * W;
  const unsigned np = min(W, npairs - p0);
  const unsigned ncol = t.real_packed ? 2 * W : W;   // = a.RPC
  const unsigned lncol = 31 - __clz(ncol);           // W, ncol: powers of two
  const unsigned T = blockDim.x;
  const Rl S = (Rl)t.scale;
  // column of slot s, or -1 for an empty slot (past the last pair, or the mirror of a self-paired column)
  auto slot_col = [&](unsigned s) -> long long {
    const unsigned pw = (s < W) ? s : s - W;
    if (pw >= np) return -1;
    const unsigned long long m1 = p0 + pw;
    if (s < W) return (long long)m1;
    if (m1 == 0 || 2 * m1 == R1) return -1;
    return (long long)(R1 - m1);
  };

  for (long long sig = blockIdx.y; sig < t.batch; sig += gridDim.y) {
    const V* g = reinterpret_cast<const V*>(t.out) + (t.f.offs ? t.f.offs[2 * sig + 1] : sig * t.M);
    // (UA elements' loads in flight per thread before they are combined and stored)
    constexpr int UA = sizeof(V) == 16 ? 1 : 2;
    for (unsigned i0 = threadIdx.x; i0 < ncol * B; i0 += T * UA) {
      V g0[UA], g1[UA], g2[UA], g3[UA];
#pragma unroll
      for (int e = 0; e < UA; ++e) {
        const unsigned idx = i0 + e * T;
        const long long col = (idx < ncol * B) ? slot_col(idx & (ncol - 1)) : -1;
        if (col >= 0) {
          const unsigned long long j = (unsigned long long)col + R1 * (idx >> lncol);
          g0[e] = __ldg(g + j);
          if (t.real_packed) {
            g1[e] = __ldg(g + j + Mc);
            g2[e] = __ldg(g + (j ? M - j : 0));
            g3[e] = __ldg(g + (Mc - j));
          }
        }
      }
#pragma unroll
      for (int e = 0; e < UA; ++e) {
        const unsigned idx = i0 + e * T;
        if (idx >= ncol * B) continue;
        const unsigned w = idx & (ncol - 1), m2 = idx >> lncol;
        const long long col = slot_col(w);
        V v = czero<V>();
        if (col >= 0) {
          const unsigned long long j = (unsigned long long)col + R1 * m2;
          if (t.real_packed) {
            const V h0 = cscale(cadd(g0[e], cconj(g2[e])), (Rl)0.5);
            const V h1 = cscale(cadd(g1[e], cconj(g3[e])), (Rl)0.5);
            const V d = cmulc(csub(h0, h1), tw_global<V>(t.wM, t.wM_lo_n, t.wM_bits, j));
            v = cadd(cadd(h0, h1), cmul_pi(d));
          } else {
            v = g0[e];
          }
        }
        buf[w * a.region + pad16((int)m2)] = cconj(v);
      }
    }
    __syncthreads();
    {
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
    V* rows = reinterpret_cast<V*>(const_cast<void*>(t.scratch)) + (size_t)sig * B * R1;
    for (unsigned idx = threadIdx.x; idx < ncol * B; idx += T) {
      const unsigned w = idx & (ncol - 1), b = idx >> lncol;
      const long long col = slot_col(w);
      if (col < 0) continue;
      const unsigned long long m1 = (unsigned long long)col;
      const V y = cconj(buf[w * a.region + pad16((int)b)]);
      const unsigned long long e = m1 * b * sM;   // m1 b < R1 B = Mc
      rows[(size_t)b * R1 + m1] = cscale(cmulc(y, tw_global<V>(t.wM, t.wM_lo_n, t.wM_bits, e)), S);
    }
    __syncthreads();
  }
}

}  // namespace adfft
