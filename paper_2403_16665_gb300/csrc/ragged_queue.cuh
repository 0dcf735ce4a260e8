// One persistent kernel for a whole ragged batch (signals of uneven N and alpha), driven
// by a work queue of tiles.
//
// The decomposition is the fold form of fused.cuh per signal (Sec. 3 in decimation-in-
// frequency order): U_{P k + r} = FFT_Np(z_r)[k], z_r[n] = sum_{f<q} u_{n + f Np}
// W_Mt^{s r (n + f Np)}, with the real unpacking X_j = E_j + W_M^j O_j, X_{j+Mc} =
// E_j - W_M^j O_j, X_{M-j} = conj X_j of packed real input.  Every signal belongs to a
// shape class (Np, P, q, Mc, twiddle table) and is served by tiles of three kinds:
//
//   whole   the signal's P residue FFTs fit one CTA: fold, FFT and unpack in shared
//           memory, natural-order stores (a tile takes up to 64 signals of its class side
//           by side: one fold per signal, then the Stockham passes and the unpacking over
//           all of them);
//   fft     R of the P residues of a longer signal: fold and FFT in shared memory, U_r
//           written to a global scratch area (residue-major, coalesced), then the
//           signal's counter is raised (release);
//   unpack  a range of leader bins j of a longer signal: waits (acquire, bounded) until
//           all its fft tiles are counted, gathers U_j and U_{Mc-j} from the scratch (L2),
//           unpacks and stores.
//
// CTAs take tiles in queue order from an atomic head; the host puts a signal's fft tiles
// before its unpack tiles, so a CTA waiting in an unpack tile only waits for tiles already
// taken by running CTAs (the grid is at most the resident CTAs), and fft tiles never wait.
#pragma once

#include "fused.cuh"

namespace adfft {

struct RqClass {
  int Np, logNp, P, q, Nc, Mc;
  int Mt;                 // twiddle modulus (M for packed real input, Mc otherwise)
  int region, nrad, r0;   // shared-memory region per residue, passes, first radix
  int tw_bits, tw_lo_n, tw_hi_n;
  int real_packed;        // 1: packed real input, unpacked to M = 2 Mc bins
  long long tw_off;       // float2 offset of the class's table in the table array
  long long M;            // bins per signal
  float scale;            // S
  FastDiv divP;
};

enum RqTileKind : int { kRqWhole = 0, kRqFft = 1, kRqUnpack = 2 };
constexpr int kRqMaxGroup = 64;   // signals of one whole tile at most

struct RqTile {
  int kind, cls;
  int sig;     // signal (whole: the first of `a1` consecutive queue signals of the class)
  int a0, a1;  // fft: residues [a0, a0 + a1); unpack: leaders [a0, a1); whole: -, count
  int pad;
};

struct RqSignal {
  long long in_bytes;   // byte offset of the signal's input
  long long out_bin;    // first output bin
  long long scratch;    // float2 offset of its U in the scratch area (fft / unpack signals)
  int nfft;             // its fft tiles
  int pad;
};

struct RqArgs {
  const void* in;
  void* out;
  const RqTile* tiles;
  int ntiles;
  const RqClass* classes;
  const RqSignal* sigs;
  const int* whole_sigs;   // signals of the whole tiles, tile after tile
  const float2* tables;
  float2* scratch;
  int* counters;           // [0]: queue head; [1 + s]: fft tiles done of signal s
  int* status;
  int tw_max;              // largest table (entries) of any class
  long long wait_limit;
};

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// FusedArgs view of a class, for the shared first pass and Stockham passes.
__device__ __forceinline__ FusedArgs rq_fused_args(const RqClass& c, int rpc) {
  FusedArgs a;
  memset(&a, 0, sizeof(a));
  a.Np = c.Np;
  a.logNp = c.logNp;
  a.P = c.P;
  a.q = c.q;
  a.RPC = rpc;
  a.C = 1;
  a.Nc = c.Nc;
  a.Mc = c.Mc;
  a.Mt = c.Mt;
  a.region = c.region;
  a.nrad = c.nrad;
  return a;
}

// fold + twiddle + first radix of residues [r0, r0 + rpc) of one signal into buf
template <int R0>
__device__ __forceinline__ void rq_first(const FusedArgs& a, const void* u, int mode, float2* buf,
                                         const TwTable<float2>& tab, int r0) {
  first_pass<R0, float2, false, RuntimeShape>(a, u, nullptr, mode, buf, tab, r0);
}

// the radix-16 Stockham passes over all a.RPC regions of buf (after the first pass of radix R0);
// starts and ends with the CTA synchronised (every pass ends with a barrier)
template <int R0>
__device__ __forceinline__ void rq_passes(const FusedArgs& a, float2* buf, const TwTable<float2>& tab) {
  constexpr int LOGR0 = R0 == 1 ? 0 : R0 == 2 ? 1 : R0 == 4 ? 2 : R0 == 8 ? 3 : R0 == 16 ? 4 : 5;
  int Ns = R0, logNs = LOGR0;
  __syncthreads();
  for (int p = 1; p < a.nrad; ++p) {
    stockham_pass<16, 32, float2, RuntimeShape>(a, buf, tab, Ns, logNs);
    Ns <<= 4;
    logNs += 4;
  }
}

__device__ __forceinline__ void rq_first_any(const FusedArgs& a, int r0radix, const void* u, int mode, float2* buf,
                                             const TwTable<float2>& tab, int r0) {
  switch (r0radix) {
    case 1: rq_first<1>(a, u, mode, buf, tab, r0); break;
    case 2: rq_first<2>(a, u, mode, buf, tab, r0); break;
    case 4: rq_first<4>(a, u, mode, buf, tab, r0); break;
    case 8: rq_first<8>(a, u, mode, buf, tab, r0); break;
    case 16: rq_first<16>(a, u, mode, buf, tab, r0); break;
    default: rq_first<32>(a, u, mode, buf, tab, r0); break;
  }
}

__device__ __forceinline__ void rq_passes_any(const FusedArgs& a, int r0radix, float2* buf,
                                              const TwTable<float2>& tab) {
  switch (r0radix) {
    case 1: rq_passes<1>(a, buf, tab); break;
    case 2: rq_passes<2>(a, buf, tab); break;
    case 4: rq_passes<4>(a, buf, tab); break;
    case 8: rq_passes<8>(a, buf, tab); break;
    case 16: rq_passes<16>(a, buf, tab); break;
    default: rq_passes<32>(a, buf, tab); break;
  }
}

// Unpack leader j (packed real: j <= Mc/2; complex: j < Mc) of one signal, with U fetched
// by `getU(q)` (q = bin of the complex core), and store its natural-order bins.
// (packed real: Uj = U_j and Up = U_{Mc - j}; complex: Uj = U_j, Up unused)
__device__ __forceinline__ void rq_unpack_vals(const RqClass& c, const TwTable<float2>& tab, float2* out,
                                               unsigned j, float2 Uj, float2 Up) {
  const unsigned Mc = (unsigned)c.Mc;
  const float S = c.scale;
  if (c.real_packed) {
    const float hS = 0.5f * S;
    const float2 A = cadd(Uj, cconj(Up));
    const float2 B = csub(Uj, cconj(Up));
    float2 wn = tab(j);
    wn = cmake<float2>(hS * wn.y, -hS * wn.x);   // (S/2)(-i) W_M^j
    const float2 t = cmul(wn, B);
    const float2 hA = cscale(A, hS);
    const float2 X1 = cadd(hA, t), X2 = csub(hA, t);
    st_stream(out + j, X1);
    st_stream(out + j + Mc, X2);
    if (j != 0 && 2 * j != Mc) {
      st_stream(out + (Mc - j), cconj(X2));
      st_stream(out + ((unsigned long long)c.M - j), cconj(X1));
    }
  } else {
    st_stream(out + j, cscale(Uj, S));
  }
}

template <class GetU>
__device__ __forceinline__ void rq_unpack_one(const RqClass& c, const TwTable<float2>& tab, float2* out,
                                              unsigned j, GetU getU) {
  const unsigned Mc = (unsigned)c.Mc;
  rq_unpack_vals(c, tab, out, j, getU(j), c.real_packed ? getU(j ? Mc - j : 0u) : czero<float2>());
}

// (a template so that only the translation unit that launches it instantiates it)
template <int UNUSED = 0>
__global__ void __launch_bounds__(512) ragged_queue_kernel(const RqArgs g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw_s = reinterpret_cast<float2*>(smem_raw);
  float2* buf = reinterpret_cast<float2*>(smem_raw + ((g.tw_max * 8 + 15) & ~15));
  __shared__ int s_tile, s_fail;
  __shared__ long long s_out[kRqMaxGroup];   // first output bin of each signal of a whole tile
  int cached_cls = -1;
  if (threadIdx.x == 0) s_fail = 0;
  for (;;) {
    __syncthreads();   // the previous tile is done with shared memory and s_tile
    if (threadIdx.x == 0) s_tile = atomicAdd(g.counters, 1);
    __syncthreads();
    const int ti = s_tile;
    if (ti >= g.ntiles || s_fail) break;
    const RqTile t = g.tiles[ti];
    const RqClass c = g.classes[t.cls];
    if (t.cls != cached_cls) {
      const int tw_n = c.tw_lo_n + c.tw_hi_n;
      for (int i = threadIdx.x; i < tw_n; i += blockDim.x) tw_s[i] = g.tables[c.tw_off + i];
      cached_cls = t.cls;
      __syncthreads();
    }
    const TwTable<float2> tab{tw_s, tw_s + c.tw_lo_n, c.tw_bits, (1u << c.tw_bits) - 1u};
    const int mode = c.real_packed ? kLoadRealPacked : kLoadComplex;
    if (t.kind == kRqWhole) {
      // the t.a1 signals of the group side by side: signal w in regions [w P, (w + 1) P)
      const int nw = t.a1;
      const FusedArgs a1 = rq_fused_args(c, c.P);
      for (int w = threadIdx.x; w < nw; w += blockDim.x) s_out[w] = g.sigs[g.whole_sigs[t.sig + w]].out_bin;
      for (int w = 0; w < nw; ++w) {
        const RqSignal sg = g.sigs[g.whole_sigs[t.sig + w]];
        const void* u = reinterpret_cast<const unsigned char*>(g.in) + sg.in_bytes;
        rq_first_any(a1, c.r0, u, mode, buf + (size_t)w * c.P * c.region, tab, 0);
      }
      rq_passes_any(rq_fused_args(c, nw * c.P), c.r0, buf, tab);
      const unsigned jt = c.real_packed ? (unsigned)c.Mc / 2 + 1 : (unsigned)c.Mc;
      const unsigned total = (unsigned)nw * jt;
      for (unsigned i = threadIdx.x; i < total; i += blockDim.x) {
        const unsigned w = i / jt, j = i - w * jt;
        const float2* bw = buf + (size_t)w * c.P * c.region;
        float2* out = reinterpret_cast<float2*>(g.out) + s_out[w];
        rq_unpack_one(c, tab, out, j, [&](unsigned q) {
          const unsigned k = fdiv(q, c.divP);
          return bw[(q - k * (unsigned)c.P) * (unsigned)c.region + (unsigned)pad16((int)k)];
        });
      }
    } else if (t.kind == kRqFft) {
      const FusedArgs a = rq_fused_args(c, t.a1);
      const RqSignal sg = g.sigs[t.sig];
      const void* u = reinterpret_cast<const unsigned char*>(g.in) + sg.in_bytes;
      rq_first_any(a, c.r0, u, mode, buf, tab, t.a0);
      rq_passes_any(a, c.r0, buf, tab);
      // U_r[k] of residues a0 .. a0 + a1 - 1 to the scratch, residue-major
      float2* dst = g.scratch + sg.scratch + (long long)t.a0 * c.Np;
      const unsigned total = (unsigned)t.a1 * (unsigned)c.Np;
      for (unsigned i = threadIdx.x; i < total; i += blockDim.x) {
        const unsigned rl = i >> c.logNp, k = i & ((unsigned)c.Np - 1u);
        __stcg(dst + i, buf[rl * (unsigned)c.region + (unsigned)pad16((int)k)]);
      }
      __threadfence();   // every thread's scratch stores before the count (release)
      __syncthreads();
      if (threadIdx.x == 0) atomicAdd(g.counters + 1 + t.sig, 1);
    } else {
      const RqSignal sg = g.sigs[t.sig];
      if (threadIdx.x == 0) {
        const long long t0 = clock64();
        while (ld_acquire_gpu(g.counters + 1 + t.sig) < sg.nfft) {
          if (clock64() - t0 > g.wait_limit) {
            s_fail = 1;
            if (g.status) atomicExch(g.status, kStatusTimeout);
            break;
          }
        }
      }
      __syncthreads();
      if (s_fail) break;
      const float2* U = g.scratch + sg.scratch;
      float2* out = reinterpret_cast<float2*>(g.out) + sg.out_bin;
      for (unsigned j = (unsigned)t.a0 + threadIdx.x; j < (unsigned)t.a1; j += blockDim.x)
        rq_unpack_one(c, tab, out, j, [&](unsigned q) {
          const unsigned k = fdiv(q, c.divP);
          return __ldcg(U + (long long)(q - k * (unsigned)c.P) * c.Np + k);
        });
    }
  }
}

}  // namespace adfft
