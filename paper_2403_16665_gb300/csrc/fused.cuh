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
// [c*RPC, (c+1)*RPC) of it in shared memory.  The signal's input is brought
// into shared memory by a bulk (TMA) copy issued while the previous signal is
// still being transformed.  Pass 1 (K1) folds and twiddles the staged input
// into its first radix-R butterfly; the remaining radix-16 Stockham passes
// (K2) run in shared memory; the epilogue (K3) gathers U across the cluster
// through distributed shared memory so that each CTA writes a contiguous,
// coalesced range of output bins in natural order.
#pragma once

#include <cooperative_groups.h>

#include "fft_device.cuh"

namespace adfft {

namespace cg = cooperative_groups;

// How the kernel reads its input.
enum LoadMode : int {
  kLoadComplex = 0,      // complex input, u = x
  kLoadRealPacked = 1,   // real input, two samples per complex element, unpacked in the epilogue
  kLoadRealPlain = 2,    // real input read as complex with zero imaginary part (odd N or odd M)
  kColumns = 3           // first pass of the two-pass form: complex columns u_{B a + b} of each
                         // signal (element stride B = cols), output row b twiddled by W_Mpost^{m b}
};

// Status word values written by kernels (0 = no error).
constexpr int kStatusTimeout = -8;

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
  int stage_bytes;       // > 0: each signal's input is bulk-copied into shared memory first
  int* status;           // device status word of the plan
  FastDiv divP, divRPC;
  // per-signal placement for packed (ragged) batches: offs[2 s] = byte offset of
  // signal s in the input, offs[2 s + 1] = its first output bin; NULL means
  // s * in_stride * in_unit bytes and s * M bins
  const long long* offs;
  int in_unit;           // bytes per in_stride unit (real scalar or complex element)
  // kColumns only: columns per signal, and the two-level table of W_Mpost (global memory)
  long long cols;
  const void* post_tw;
  int post_bits, post_lo_n;
  long long Mpost;
  // fault injection for tests (0 = none): the input copy of signal fault_sig1 - 1 is not issued,
  // and waits on input copies give up after wait_limit cycles instead of the default (~2 s)
  long long fault_sig1;
  long long wait_limit;
  // packed real input only: 1 = write the half spectrum X_0 .. X_{M/2} ([batch][M/2 + 1]
  // output), which determines the rest by X_{M-m} = conj X_m
  int half;
  // kColumns only, > 1: that many CTAs per signal without a cluster (C = 1), CTA x holding
  // residues [x RPC, (x + 1) RPC) and writing its own bins m = k P + r (runs of RPC bins)
  int vsplit;
};

// Compile-time shape of a specialised instantiation; a zero field is read from
// FusedArgs at run time instead.  LOGNP: log2 of the sub-FFT length, RPC:
// residues per CTA, P: residues per signal, T: threads per CTA, MTF: Mt / (P Np)
// (2 for packed real input, 1 otherwise).
// PADSH, PW: shared-memory padding of PW slots per 2^PADSH elements (0: 4 and 1,
// i.e. pad16).  With PW = 2 every even element index stays 16-byte aligned, and
// float2 data moves in 16-byte pairs (first-pass stores, epilogue loads).
// EU: independent epilogue loads in flight per thread (0: the generic default).
// HF: output extent of packed real input, 0: read at run time (FusedArgs::half), 1: the full
// spectrum, 2: the half spectrum (fixed at compile time, the epilogue stores carry no test).
template <int LOGNP = 0, int RPC = 0, int P = 0, int T = 0, int MTF = 0, int PADSH = 0, int EU = 0, int PW = 1,
          int HF = 0>
struct Shape {
  static constexpr bool fixed = LOGNP != 0 && RPC != 0 && P != 0 && T != 0 && MTF != 0;
  static constexpr int padsh = PADSH ? PADSH : 4;
  static constexpr int pw = PW;
  static constexpr bool pairs = PW == 2;
  static constexpr int eu = EU;
  __device__ static __forceinline__ bool half(const struct FusedArgs& a);
  __device__ static __forceinline__ int pad(int p) { return p + PW * (p >> padsh); }
  __device__ static __forceinline__ int logNp(const struct FusedArgs& a);
  __device__ static __forceinline__ int Np(const struct FusedArgs& a);
  __device__ static __forceinline__ int rpc(const struct FusedArgs& a);
  __device__ static __forceinline__ int p(const struct FusedArgs& a);
  __device__ static __forceinline__ int threads();
  __device__ static __forceinline__ int region(const struct FusedArgs& a);
  __device__ static __forceinline__ unsigned mt(const struct FusedArgs& a);
};
#define ADFFT_SHAPE_TPL template <int L, int R, int PP, int TT, int F, int PS, int E, int W, int H>
#define ADFFT_SHAPE Shape<L, R, PP, TT, F, PS, E, W, H>
ADFFT_SHAPE_TPL
__device__ __forceinline__ bool ADFFT_SHAPE::half(const FusedArgs& a) { return H ? H == 2 : a.half != 0; }
ADFFT_SHAPE_TPL
__device__ __forceinline__ int ADFFT_SHAPE::logNp(const FusedArgs& a) { return L ? L : a.logNp; }
ADFFT_SHAPE_TPL
__device__ __forceinline__ int ADFFT_SHAPE::Np(const FusedArgs& a) { return L ? (1 << L) : a.Np; }
ADFFT_SHAPE_TPL
__device__ __forceinline__ int ADFFT_SHAPE::rpc(const FusedArgs& a) { return R ? R : a.RPC; }
ADFFT_SHAPE_TPL
__device__ __forceinline__ int ADFFT_SHAPE::p(const FusedArgs& a) { return PP ? PP : a.P; }
ADFFT_SHAPE_TPL
__device__ __forceinline__ int ADFFT_SHAPE::threads() { return TT ? TT : (int)blockDim.x; }
ADFFT_SHAPE_TPL
__device__ __forceinline__ int ADFFT_SHAPE::region(const FusedArgs& a) {
  return L ? ((1 << L) + W * ((1 << L) >> (PS ? PS : 4)) + 2) : a.region;
}
ADFFT_SHAPE_TPL
__device__ __forceinline__ unsigned ADFFT_SHAPE::mt(const FusedArgs& a) {
  return (L && PP && F) ? (unsigned)(F * PP) << L : (unsigned)a.Mt;
}
using RuntimeShape = Shape<>;

// Passes of a fixed shape: one of radix 2^LOGR0, then radix 16.
template <class SH, int LOGR0> struct SH_PASSES;
template <int L, int R, int PP, int TT, int F, int PS, int E, int W, int H, int LOGR0>
struct SH_PASSES<ADFFT_SHAPE, LOGR0> { static constexpr int value = 1 + (L - LOGR0) / 4; };
#undef ADFFT_SHAPE
#undef ADFFT_SHAPE_TPL

// Shared-memory layout of the fused kernel (byte offsets).
struct FusedSmem {
  int tw, stage, buf, total;
};
__host__ __device__ inline FusedSmem fused_smem_layout(int tw_n, int stage_bytes, int rpc, int region,
                                                       int esz) {
  FusedSmem s;
  s.tw = 16;                                         // [0, 16): the mbarrier
  s.stage = s.tw + ((tw_n * esz + 15) & ~15);
  s.buf = s.stage + ((stage_bytes + 15) & ~15);
  s.total = s.buf + rpc * region * esz;
  return s;
}

__device__ __forceinline__ long long sig_in_bytes(const FusedArgs& a, long long s) {
  return a.offs ? a.offs[2 * s] : s * a.in_stride * a.in_unit;
}
__device__ __forceinline__ long long sig_out_off(const FusedArgs& a, long long s) {
  return a.offs ? a.offs[2 * s + 1] : s * (a.half ? a.M / 2 + 1 : a.M);
}

template <typename V>
__device__ __forceinline__ V ld_u(const void* base, int idx, int mode, bool smem) {
  using R = typename real_of<V>::type;
  if (smem) {
    if (mode == kLoadRealPlain) return cmake<V>(reinterpret_cast<const R*>(base)[idx], (R)0);
    return reinterpret_cast<const V*>(base)[idx];
  }
  if (mode == kLoadRealPlain) return cmake<V>(__ldg(reinterpret_cast<const R*>(base) + idx), (R)0);
  return __ldg(reinterpret_cast<const V*>(base) + idx);
}

template <typename V>
__device__ __forceinline__ V ld_col(const void* base, int idx, long long stride) {
  return __ldg(reinterpret_cast<const V*>(base) + (long long)idx * stride);
}

// Multiply v[n][i] (n < NI items, i = 1..R-1) by w^i, w = W^k from one table
// lookup.  Powers are generated on the fly with few live registers:
// w^2 = w w, w^3 = w^2 w, w^4 = w^2 w^2, w^(4b) = w^(4(b-1)) w^4 and
// w^(4b+c) = w^(4b) w^c, so every power is at most five products from w.
template <int R, int NI, typename V>
__device__ __forceinline__ void apply_stage_twiddles(V (*v)[R], V w1) {
  if constexpr (R > 1) {
    const V w2 = cmul(w1, w1);
    const V w3 = cmul(w2, w1);
    const V w4 = cmul(w2, w2);
    V wb = w4;
#pragma unroll
    for (int i = 1; i < R; ++i) {
      const int b = i >> 2, c = i & 3;
      if (b >= 2 && c == 0) wb = cmul(wb, w4);
      V wi;
      if (b == 0) wi = (c == 1) ? w1 : (c == 2) ? w2 : w3;
      else wi = (c == 0) ? wb : cmul(wb, (c == 1) ? w1 : (c == 2) ? w2 : w3);
#pragma unroll
      for (int n = 0; n < NI; ++n) v[n][i] = cmul(v[n][i], wi);
    }
  }
}

// Pass 1 (Ns = 1): fold, residue twiddle and the first radix-R butterfly,
// reading u (staged in shared memory or straight from global memory) and
// writing the CTA's residue regions.  Element n = j + i*Np/R + f*Np of residue r
// is twiddled by W_Mt^{s r n} = W_Mt^{s r j} * c^i * g^f with the per-residue
// constants c = W_Mt^{s r Np/R} and g = W_Mt^{s r Np} (s = Mt/Mc), so each
// (j, r) costs one table lookup.
template <typename V, bool STAGED>
__device__ __forceinline__ V ld_any(const FusedArgs& a, const void* u, const V* su, int idx, int mode) {
  using R = typename real_of<V>::type;
  if constexpr (STAGED) {
    // the staged copy in this CTA's shared memory (typed, so it compiles to shared loads)
    if (mode == kLoadRealPlain) return cmake<V>(reinterpret_cast<const R*>(su)[idx], (R)0);
    return su[idx];
  } else {
    if (mode == kColumns) return ld_col<V>(u, idx, a.cols);
    return ld_u<V>(u, idx, mode, false);
  }
}

template <int R, typename V, bool STAGED, class SH = RuntimeShape>
__device__ __forceinline__ void first_pass(const FusedArgs& a, const void* u, const V* su, int mode,
                                           V* buf, const TwTable<V>& tab, int r0) {
  const int Np = SH::Np(a);
  const int items = Np / R;
  const unsigned T = (unsigned)SH::threads();
  const unsigned Mt = SH::mt(a);
  const unsigned s = SH::fixed ? Mt / ((unsigned)SH::p(a) << SH::logNp(a)) : (unsigned)(a.Mt / a.Mc);
  const int rpc = SH::rpc(a);
  const int region = SH::region(a);
  // one item: elements j + i items (+ f Np) of residue r0 + rl -> R outputs at j R .. j R + R - 1
  auto item = [&](int rl, int j, const V& c1, const V& g1, unsigned e_j) {
    V* dst = buf + rl * region;
    V acc[R];
    // fold: acc[i] = sum_f u[j + i items + f Np] g^f
#pragma unroll
    for (int i = 0; i < R; ++i) acc[i] = ld_any<V, STAGED>(a, u, su, j + i * items, mode);
    if (a.q > 1) {
      V gf = g1;
      for (int f = 1; f < a.q; ++f) {
#pragma unroll
        for (int i = 0; i < R; ++i) acc[i] = cadd(acc[i], cmul(ld_any<V, STAGED>(a, u, su, j + i * items + f * Np, mode), gf));
        gf = cmul(gf, g1);
      }
    }
    // residue twiddle W^{s r j} c^i
    V wi = tab(e_j);
    acc[0] = cmul(acc[0], wi);
#pragma unroll
    for (int i = 1; i < R; ++i) {
      wi = cmul(wi, c1);
      acc[i] = cmul(acc[i], wi);
    }
    DFT<R, V>::run(acc);
    if constexpr (SH::pairs && (R % 2) == 0 && sizeof(V) == 8 && R <= (1 << SH::padsh)) {
      // R outputs of one item lie in one padding block: 16-byte pair stores
      float4* d4 = reinterpret_cast<float4*>(dst + SH::pad(j * R));
#pragma unroll
      for (int i = 0; i < R; i += 2) d4[i / 2] = make_float4(acc[i].x, acc[i].y, acc[i + 1].x, acc[i + 1].y);
    } else {
#pragma unroll
      for (int i = 0; i < R; ++i) dst[SH::pad(j * R + i)] = acc[i];
    }
  };
  if (items < (int)T && (T % (unsigned)items) == 0) {
    // fewer items per residue than threads: thread t keeps item j = t mod items and takes
    // residues t / items, t / items + T / items, ... so that no thread idles while the
    // residues are done in turn (the residue constants are computed once per residue)
    const int rstep = (int)T / items;
    const int j = threadIdx.x % items;
#pragma unroll 1
    for (int rl = threadIdx.x / items; rl < rpc; rl += rstep) {
      const unsigned long long sr = (unsigned long long)s * (unsigned)(r0 + rl);
      const V c1 = tab((unsigned)((sr * (unsigned)items) % Mt));
      const V g1 = tab((unsigned)((sr * (unsigned)Np) % Mt));
      item(rl, j, c1, g1, (unsigned)((sr * (unsigned)j) % Mt));
    }
    return;
  }
#pragma unroll 1
  for (int rl = 0; rl < rpc; ++rl) {
    const unsigned long long sr = (unsigned long long)s * (unsigned)(r0 + rl);
    const V c1 = tab((unsigned)((sr * (unsigned)items) % Mt));
    const V g1 = tab((unsigned)((sr * (unsigned)Np) % Mt));
    const unsigned d_T = (unsigned)((sr * T) % Mt);
    unsigned e_j = (unsigned)((sr * threadIdx.x) % Mt);
    for (int j = threadIdx.x; j < items; j += T) {
      item(rl, j, c1, g1, e_j);
      e_j += d_T;
      if (e_j >= Mt) e_j -= Mt;
    }
  }
}

// One in-place Stockham pass of radix R over all residue regions of the CTA.
// Item (rl, j): reads elements j + i*Np/R, twiddles by W_{Ns R}^{(j mod Ns) i},
// runs DFT_R and writes to (j / Ns) * Ns * R + (j mod Ns) + i*Ns.  When the
// block size is a multiple of Np/R every item of a thread has the same j, and
// the twiddles are computed once for all of its residues.
template <int R, int VPT, typename V, class SH = RuntimeShape>
__device__ __forceinline__ void stockham_pass(const FusedArgs& a, V* buf, const TwTable<V>& tab,
                                              int Ns, int logNs) {
  constexpr int IPT = VPT / R;
  constexpr int LOGR = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : R == 16 ? 4 : 5;
  const int log_items = SH::logNp(a) - LOGR;
  const int items_res = 1 << log_items;
  const int items = SH::rpc(a) * items_res;
  const int T = SH::threads();
  const int region = SH::region(a);
  const bool same_j = (T & (items_res - 1)) == 0;
  const unsigned tw_step = SH::mt(a) / ((unsigned)Ns << LOGR);   // Mt / (Ns R)
  // pad(j + i*S) = pad(j) + i*(S + PW S/2^padsh) for S a multiple of 2^padsh
  constexpr int PADN = 1 << SH::padsh;
  const int in_step = items_res + SH::pw * (items_res >> SH::padsh);
  V v[IPT][R];
#pragma unroll
  for (int it = 0; it < IPT; ++it) {
    const int wi = threadIdx.x + it * T;
    const int rl = wi >> log_items;
    const int j = wi & (items_res - 1);
    const V* src = buf + rl * region;
    if (items_res >= PADN) {
      const V* p0 = src + SH::pad(j);
#pragma unroll
      for (int i = 0; i < R; ++i) v[it][i] = (wi < items) ? p0[i * in_step] : czero<V>();
    } else {
#pragma unroll
      for (int i = 0; i < R; ++i) v[it][i] = (wi < items) ? src[SH::pad(j + (i << log_items))] : czero<V>();
    }
  }
  if (same_j) {
    const int j = threadIdx.x & (items_res - 1);
    apply_stage_twiddles<R, IPT>(v, tab((unsigned)(j & (Ns - 1)) * tw_step));
  } else {
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
      const int j = (threadIdx.x + it * T) & (items_res - 1);
      apply_stage_twiddles<R, 1>(&v[it], tab((unsigned)(j & (Ns - 1)) * tw_step));
    }
  }
#pragma unroll
  for (int it = 0; it < IPT; ++it) DFT<R, V>::run(v[it]);
  __syncthreads();
  const int out_step = Ns + SH::pw * (Ns >> SH::padsh);
#pragma unroll
  for (int it = 0; it < IPT; ++it) {
    const int wi = threadIdx.x + it * T;
    if (wi < items) {
      const int rl = wi >> log_items;
      const int j = wi & (items_res - 1);
      const int k = j & (Ns - 1);
      const int base = ((j >> logNs) << (logNs + LOGR)) + k;
      V* dst = buf + rl * region;
      if (Ns >= PADN) {
        V* p0 = dst + SH::pad(base);
#pragma unroll
        for (int i = 0; i < R; ++i) p0[i * out_step] = v[it][i];
      } else {
#pragma unroll
        for (int i = 0; i < R; ++i) dst[SH::pad(base + i * Ns)] = v[it][i];
      }
    }
  }
  __syncthreads();
}

// independent U loads in flight per thread in the epilogue (bounded by registers)
template <typename V, int MODE>
constexpr int epilogue_unroll() { return sizeof(V) == 16 ? 4 : (MODE == kLoadRealPacked ? 6 : 8); }

// Radix-16 pass hook: the plain FP32/FP64 pass, or the tensor-core form of
// tc_dft16.cuh when PREC != 0 (declared here, defined there).
template <int PREC, int TPT, typename V>
__device__ void stockham_pass_tc(const FusedArgs& a, V* buf, const TwTable<V>& tab, int Ns, int logNs);

template <int PREC, int VPT, typename V, class SH = RuntimeShape>
__device__ __forceinline__ void radix16_pass(const FusedArgs& a, V* buf, const TwTable<V>& tab, int Ns, int logNs) {
  if constexpr (PREC == 0) stockham_pass<16, VPT, V, SH>(a, buf, tab, Ns, logNs);
  else stockham_pass_tc<PREC, VPT / 8, V>(a, buf, tab, Ns, logNs);
}

// R0: radix of the first pass (1, 2, 4, 8 or 16); every later pass is radix 16.
// PREC: arithmetic of the radix-16 passes (0 native, else the tensor-core form).
template <typename V, int MODE, int VPT, int R0, int PREC = 0, class SH = RuntimeShape>
__global__ void __launch_bounds__(512) fused_forward_kernel(const FusedArgs a) {
  using Rl = typename real_of<V>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int esz = (int)sizeof(V);
  const int tw_n = a.tw_lo_n + a.tw_hi_n;
  const FusedSmem L = fused_smem_layout(tw_n, a.stage_bytes, SH::rpc(a), SH::region(a), esz);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  V* tw_s = reinterpret_cast<V*>(smem_raw + L.tw);
  unsigned char* stage = smem_raw + L.stage;
  V* buf = reinterpret_cast<V*>(smem_raw + L.buf);
  // staged: each signal's contiguous input arrives by a bulk copy (prefetched one signal
  // ahead); col_staged (columns of the two-pass form): the CTA gathers its strided column into
  // shared memory once, so the first pass reads it from there for every residue
  const bool staged = a.stage_bytes > 0 && MODE != kColumns;
  const bool col_staged = a.stage_bytes > 0 && MODE == kColumns;

  if (threadIdx.x == 0 && staged) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < tw_n; i += blockDim.x) tw_s[i] = reinterpret_cast<const V*>(a.tw)[i];
  __syncthreads();
  TwTable<V> tab{tw_s, tw_s + a.tw_lo_n, a.tw_bits, (1u << a.tw_bits) - 1u};

  cg::cluster_group cluster = cg::this_cluster();
  const int c = (int)blockIdx.x;          // rank within the cluster (grid.x == C), or residue group
  // (columns split over independent CTAs: each CTA's epilogue covers only its own residues)
  const bool vs = MODE == kColumns && a.vsplit > 1;

  // Epilogue work split: CTA c writes bins j in [c*per, (c+1)*per) (real packed
  // input: j <= Mc/2 and their mirrors), per a multiple of P.  Thread t keeps the
  // residue r_l = t mod P for every j it handles (T' = P * floor(T/P) threads
  // take part), so its shared-memory sources are fixed for the whole kernel.
  const unsigned P = (unsigned)SH::p(a);
  const unsigned RPCu = (unsigned)SH::rpc(a);
  const unsigned EP = vs ? RPCu : P;                          // residues the epilogue covers
  const unsigned Tp = ((unsigned)SH::threads() / EP) * EP;
  const bool lane_ok = threadIdx.x < Tp;
  const unsigned r_l = vs ? c * RPCu + threadIdx.x % EP : threadIdx.x % P;
  const unsigned k_step = Tp / EP;
  const unsigned jtot = (MODE == kLoadRealPacked) ? (unsigned)a.Mc / 2 + 1 : (unsigned)a.Mc;
  // (pair epilogue: per a multiple of 2P, so every CTA's k range starts even)
  constexpr unsigned KG = (SH::pairs && MODE == kLoadRealPacked && sizeof(V) == 8) ? 2u : 1u;
  const unsigned per = vs ? jtot : ((jtot + a.C - 1) / a.C + KG * P - 1) / (KG * P) * (KG * P);
  const unsigned j_first = vs ? 0u : c * per;
  const unsigned j_last = min(jtot, j_first + per) - 1;      // inclusive
  const unsigned k_first = j_first / P + threadIdx.x / EP;
  // shared::cluster addresses of this lane's two source residue regions
  uint32_t base_u, base_p;
  {
    const unsigned rp = (P - r_l) % P;                        // residue of the mirror bin Mc - j
    const unsigned ou = r_l / RPCu, op = rp / RPCu;
    const V* lu = buf + (r_l - ou * RPCu) * SH::region(a);
    const V* lp = buf + (rp - op * RPCu) * SH::region(a);
    base_u = dsmem_addr(lu, (a.C > 1) ? ou : 0u);
    base_p = dsmem_addr(lp, (a.C > 1) ? op : 0u);
  }
  const int r0 = c * SH::rpc(a);
  const Rl S = (Rl)a.scale;
  const bool half_out = SH::half(a);
  constexpr int LOGR0 = R0 == 1 ? 0 : R0 == 2 ? 1 : R0 == 4 ? 2 : R0 == 8 ? 3 : R0 == 16 ? 4 : 5;
  constexpr int kEpilogueUnroll = SH::eu ? SH::eu : epilogue_unroll<V, MODE>();
  uint32_t phase = 0, fail_phase = 0;
  bool failed = false;

  const long long wait_limit = a.wait_limit > 0 ? a.wait_limit : kWaitLimitCycles;
  // prefetch the first signal's input
  if (staged && threadIdx.x == 0 && (long long)blockIdx.y < a.batch) {
    mbar_arrive_expect_tx(bar, (uint32_t)a.stage_bytes);
    if ((long long)blockIdx.y + 1 != a.fault_sig1)
      bulk_copy_g2s(stage, reinterpret_cast<const unsigned char*>(a.in) + sig_in_bytes(a, blockIdx.y),
                    (uint32_t)a.stage_bytes, bar);
  }

  for (long long sig = blockIdx.y; sig < a.batch; sig += gridDim.y) {
    const void* u;
    bool ok = true;   // this thread saw the signal's input land
    if (staged) {
      u = stage;
      if (!failed) ok = mbar_wait_bounded(bar, phase, wait_limit);
    } else if (MODE == kColumns) {
      u = reinterpret_cast<const V*>(reinterpret_cast<const unsigned char*>(a.in) + sig_in_bytes(a, sig / a.cols)) +
          (sig % a.cols);
      if (col_staged) {
        // 4 strided loads in flight per thread; the previous first pass is done with `stage`
        V* st = reinterpret_cast<V*>(stage);
        const unsigned ncol = (unsigned)a.Nc, T = blockDim.x;
        for (unsigned i0 = threadIdx.x; i0 < ncol; i0 += 4 * T) {
          V v[4];
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (i0 + e * T < ncol) v[e] = ld_col<V>(u, (int)(i0 + e * T), a.cols);
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (i0 + e * T < ncol) st[i0 + e * T] = v[e];
        }
        __syncthreads();
      }
    } else {
      u = reinterpret_cast<const unsigned char*>(a.in) + sig_in_bytes(a, sig);
    }
    V* out = reinterpret_cast<V*>(a.out) + ((MODE == kColumns) ? sig * a.M : sig_out_off(a, sig));
    const unsigned col = (MODE == kColumns) ? (unsigned)(sig % a.cols) : 0u;

    // ---- K1: fold + residue twiddle + first radix
    if (a.C > 1 && sig != (long long)blockIdx.y) cluster_wait();
    if (!failed && ok) {
      if (staged || col_staged) first_pass<R0, V, true, SH>(a, u, reinterpret_cast<const V*>(stage), MODE, buf, tab, r0);
      else first_pass<R0, V, false, SH>(a, u, nullptr, MODE, buf, tab, r0);
    }
    if (staged) {
      // the CTA decides as one, on the barrier that ends the first pass: after a wait ran out
      // it transforms no further signal (it keeps taking part in the cluster barriers, so its
      // peers are not left waiting); the first pass has no barrier of its own
      if (__syncthreads_or(!ok) && !failed) {
        failed = true;
        fail_phase = phase;
        if (threadIdx.x == 0 && a.status) atomicExch(a.status, kStatusTimeout);
      }
      phase ^= 1u;
    } else {
      __syncthreads();
    }

    // prefetch the next signal's input while this one is transformed
    const long long nxt = sig + gridDim.y;
    if (staged && threadIdx.x == 0 && nxt < a.batch && !failed) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(bar, (uint32_t)a.stage_bytes);
      if (nxt + 1 != a.fault_sig1)
        bulk_copy_g2s(stage, reinterpret_cast<const unsigned char*>(a.in) + sig_in_bytes(a, nxt),
                      (uint32_t)a.stage_bytes, bar);
    }

    // ---- K2: radix-16 Stockham passes in shared memory
    int Ns = R0, logNs = LOGR0;
    if (failed) {
      // no transform after a failed wait: only the cluster barriers below
    } else if constexpr (SH::fixed) {
      constexpr int kPasses = SH_PASSES<SH, LOGR0>::value;
#pragma unroll
      for (int p = 1; p < kPasses; ++p) {
        radix16_pass<PREC, VPT, V, SH>(a, buf, tab, Ns, logNs);
        Ns <<= 4;
        logNs += 4;
      }
    } else {
      for (int p = 1; p < a.nrad; ++p) {
        radix16_pass<PREC, VPT, V, SH>(a, buf, tab, Ns, logNs);
        Ns <<= 4;
        logNs += 4;
      }
    }

    // ---- K3: interleave epilogue through distributed shared memory
    if (a.C > 1) { cluster_arrive(); cluster_wait(); } else { __syncthreads(); }
    if (lane_ok && !failed) {
      if constexpr (KG == 2) {
        // pairs of k: thread (r_l, kq) handles k = 2 kq and 2 kq + 1 of residue r_l, i.e. bins
        // j0 = 2 kq P + r_l and j1 = j0 + P; U[k], U[k+1] come in one 16-byte load, and so do
        // the mirror values U[Np-2-k], U[Np-1-k] (residue P - r_l), except for r_l = 0
        const unsigned Mc = (unsigned)a.Mc;
        const unsigned half = Mc / 2;
        const unsigned lim = min(half, j_last);
        const unsigned Npu = (unsigned)SH::Np(a);
        const unsigned kq_first = j_first / (2 * P) + threadIdx.x / P;
        const Rl hS = S * (Rl)0.5;
        const V wP = tab(P);   // W_M^P
        for (unsigned kq = kq_first; 2 * kq * P + r_l <= lim; kq += k_step * kEpilogueUnroll) {
          V Ua[kEpilogueUnroll][2], Ub[kEpilogueUnroll][2];
#pragma unroll
          for (int e = 0; e < kEpilogueUnroll; ++e) {
            const unsigned k = 2 * (kq + e * k_step);
            if (k * P + r_l <= lim) {
              dsmem_ld_pair(base_u + (uint32_t)SH::pad((int)k) * 8u, Ua[e][0], Ua[e][1]);
              if (r_l != 0) {
                // mirror of k is Np-1-k, of k+1 is Np-2-k: the pair starting at Np-2-k
                dsmem_ld_pair(base_p + (uint32_t)SH::pad((int)(Npu - 2 - k)) * 8u, Ub[e][1], Ub[e][0]);
              } else {
                Ub[e][0] = dsmem_ld(base_p + (uint32_t)SH::pad((int)((Npu - k) & (Npu - 1))) * 8u, V{});
                Ub[e][1] = dsmem_ld(base_p + (uint32_t)SH::pad((int)(Npu - 1 - k)) * 8u, V{});
              }
            }
          }
#pragma unroll
          for (int e = 0; e < kEpilogueUnroll; ++e) {
            const unsigned k = 2 * (kq + e * k_step);
            V X1[2], X2[2];
            // (S/2)(-i) W_M^j for j = k P + r_l, and for j + P by one product with W_M^P
            V wn = tab(k * P + r_l);
            wn = cmake<V>(hS * wn.y, -hS * wn.x);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const unsigned j = (k + h) * P + r_l;
              if (h == 1) wn = cmul(wn, wP);
              // X_j = (S/2)(A + (-i) W_M^j B), X_{j+Mc} = (S/2)(A - (-i) W_M^j B),
              // A = U_j + conj U_{Mc-j}, B = U_j - conj U_{Mc-j}
              const V A = cadd(Ua[e][h], cconj(Ub[e][h]));
              const V B = csub(Ua[e][h], cconj(Ub[e][h]));
              const V t = cmul(wn, B);
              const V hA = cscale(A, hS);
              X1[h] = cadd(hA, t);
              X2[h] = csub(hA, t);
              if (j <= lim) {
                st_stream(out + j, X1[h]);
                if (!half_out || j == 0) st_stream(out + j + Mc, X2[h]);
              }
            }
            // mirror bins: lanes of residue 0 store their two values in the opposite order, so
            // each warp-wide store covers whole 32-byte runs Mc - j (the runs end at multiples of P)
            const bool sw = (r_l == 0);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const V y1 = sw ? X1[1 - h] : X1[h];   // constant indices: registers, not memory
              const V y2 = sw ? X2[1 - h] : X2[h];
              const unsigned j = (k + (sw ? 1 - h : h)) * P + r_l;
              if (j <= lim && j != 0 && 2 * j != Mc) {
                st_stream(out + (Mc - j), cconj(y2));
                if (!half_out) st_stream(out + ((unsigned long long)a.M - j), cconj(y1));
              }
            }
          }
        }
      } else if (MODE == kLoadRealPacked) {
        const unsigned Mc = (unsigned)a.Mc;
        const unsigned half = Mc / 2;
        for (unsigned kb = k_first; kb * P + r_l <= min(half, j_last); kb += k_step * kEpilogueUnroll) {
          V Ua[kEpilogueUnroll], Ub[kEpilogueUnroll];
#pragma unroll
          for (int e = 0; e < kEpilogueUnroll; ++e) {
            const unsigned k = kb + e * k_step;
            const unsigned j = k * P + r_l;
            if (j <= half && j <= j_last) {
              const unsigned Npu = (unsigned)SH::Np(a);
              const unsigned kp = (r_l == 0) ? (Npu - k) & (Npu - 1) : Npu - 1 - k;
              Ua[e] = dsmem_ld(base_u + (uint32_t)SH::pad((int)k) * (uint32_t)sizeof(V), V{});
              Ub[e] = dsmem_ld(base_p + (uint32_t)SH::pad((int)kp) * (uint32_t)sizeof(V), V{});
            }
          }
#pragma unroll
          for (int e = 0; e < kEpilogueUnroll; ++e) {
            const unsigned k = kb + e * k_step;
            const unsigned j = k * P + r_l;
            if (j <= half && j <= j_last) {
              const V E = cscale(cadd(Ua[e], cconj(Ub[e])), (Rl)0.5);
              const V O = cscale(cmul_mi(csub(Ua[e], cconj(Ub[e]))), (Rl)0.5);
              const V wO = cmul(tab(j), O);
              const V X1 = cscale(cadd(E, wO), S);
              const V X2 = cscale(csub(E, wO), S);
              st_stream(out + j, X1);
              if (!half_out || j == 0) st_stream(out + j + Mc, X2);
              if (j != 0 && 2 * j != Mc) {
                st_stream(out + (Mc - j), cconj(X2));
                if (!half_out) st_stream(out + ((unsigned long long)a.M - j), cconj(X1));
              }
            }
          }
        }
      } else {
        // kColumns: row twiddle W_Mpost^{m col}; along a thread's bins m steps by k_step P, so
        // the twiddle steps by one product with W_Mpost^{k_step P col}, re-anchored on the
        // table at every group of kEpilogueUnroll bins
        const V* plo = reinterpret_cast<const V*>(a.post_tw);
        const V* phi = plo + a.post_lo_n;
        const unsigned long long pmask = (1ull << a.post_bits) - 1;
        auto post_tab = [&](unsigned long long e2) { return cmul(__ldg(phi + (e2 >> a.post_bits)), __ldg(plo + (e2 & pmask))); };
        V pstep = czero<V>();
        if (MODE == kColumns)
          pstep = post_tab(((unsigned long long)k_step * P * col) % (unsigned long long)a.Mpost);
        for (unsigned kb = k_first; kb * P + r_l <= j_last; kb += k_step * kEpilogueUnroll) {
          V Ua[kEpilogueUnroll];
#pragma unroll
          for (int e = 0; e < kEpilogueUnroll; ++e) {
            const unsigned k = kb + e * k_step;
            if (k * P + r_l <= j_last) Ua[e] = dsmem_ld(base_u + (uint32_t)SH::pad((int)k) * (uint32_t)sizeof(V), V{});
          }
          V pw = czero<V>();
          if (MODE == kColumns)
            pw = post_tab(((unsigned long long)(kb * P + r_l) * col) % (unsigned long long)a.Mpost);
#pragma unroll
          for (int e = 0; e < kEpilogueUnroll; ++e) {
            const unsigned k = kb + e * k_step;
            const unsigned m = k * P + r_l;
            if (m <= j_last) {
              V y = cscale(Ua[e], S);
              if (MODE == kColumns) {
                y = cmul(y, pw);
                pw = cmul(pw, pstep);
              }
              st_stream(out + m, y);
            }
          }
        }
      }
    }
    // this CTA has read what it needs from the cluster; the wait that pairs with
    // this arrive comes before the next signal overwrites shared memory
    if (a.C > 1) cluster_arrive_relaxed(); else __syncthreads();
  }
  if (a.C > 1 && (long long)blockIdx.y < a.batch) cluster_wait();
  // a copy can only still be in flight after a timed-out wait: give it time to land
  if (failed && threadIdx.x == 0) mbar_wait_bounded(bar, fail_phase, wait_limit);
}

}  // namespace adfft
