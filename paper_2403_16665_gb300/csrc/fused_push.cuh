// Single-pass forward alpha-DFT for packed real input with one residue per CTA
// (clusters of C = P CTAs, two CTAs per SM) and a PUSH exchange.
//
// Same decomposition as fused.cuh (Sec. 3 in decimation-in-frequency order):
//   U_{P k + r} = FFT_Np(z_r)[k],  z_r[n] = u_n W_Mc^{r n}   (u_n = x_{2n} + i x_{2n+1}, q = 1)
// and the real unpacking of the epilogue
//   X_j = (S/2)(A + (-i) W_M^j B),  X_{j+Mc} = (S/2)(A - (-i) W_M^j B),
//   A = U_j + conj U_{Mc-j},  B = U_j - conj U_{Mc-j},  X_{M-j} = conj X_j.
//
// CTA c of the cluster transforms residue r = c of the signal.  For the output it owns
// the bins j in [JC c, JC c + JC) (JC = Np/2) and j + Mc, and the mirror bins Mc - j',
// M - j' for j' in (JC c, JC c + JC]; over the cluster these four ranges partition
// [0, M).  They need U_j and U_{Mc-j} for every residue, i.e. one run of k and one
// mirrored run of k from each of the other CTAs.  Instead of reading those runs from
// the peers' shared memory (distributed-shared-memory loads, which sustain only a few
// bytes per clock per SM), every CTA PUSHES the runs its peers need into their landing
// zones with bulk copies (the TMA engine), in two halves of the k range:
//
//   FFT(s) into buf                                  [waits: my last pushes have landed]
//   for h in {0, 1}:
//     push half h of buf to the P-1 peers           [waits: every peer's landing is free]
//     wait until my landing holds half h from all peers
//     unpack from buf (own residue) + landing, coalesced stores
//     tell every peer that my landing is free again
//
// Three mbarriers per CTA carry the protocol: `full` (bytes pushed into my landing),
// `landed` (peers report that my half-1 pushes arrived, so buf may be overwritten) and
// `freeb` (peers report that their landing is free).  Every wait is bounded; a timed-out
// wait sets the plan's status word and the CTA stops issuing work.  A CTA touches peer
// shared memory only between the initial and the final cluster barrier.
//
// Stores: each warp step writes 32 consecutive bins of each of the four ranges; the mirror
// ranges are written one bin shifted (lanes exchange values by shuffles) so that every warp
// store covers whole 32-byte sectors.
#pragma once

#include "fused.cuh"

namespace adfft {

template <int LOGNP_, int P_, int T_>
struct PushShape {
  static constexpr int LOGNP = LOGNP_, NP = 1 << LOGNP_, P = P_, T = T_;
  // FFT view of the shape: one residue per CTA, packed real input (Mt = 2 P Np), padding of
  // 2 slots per 32 elements (16-byte pairs stay aligned)
  using SH = Shape<LOGNP_, 1, P_, T_, 2, 5, 0, 2>;
  static constexpr int LOGP = P == 2 ? 1 : P == 4 ? 2 : P == 8 ? 3 : P == 16 ? 4 : 5;
  static constexpr int REGION = NP + 2 * (NP >> 5) + 2;   // = SH::region
  static constexpr int JC = NP / 2;          // leader bins j per CTA (Mc / (2 C))
  static constexpr int JH = JC / 2;          // per half
  static constexpr int KC = JC / P;          // k per CTA
  static constexpr int KH = KC / 2;          // k per half
  static constexpr int NA = KH + 32;         // direct run (k), 32-aligned start
  static constexpr int NB = KH + 64;         // mirrored run (k), at most
  static constexpr int PADA = NA / 32 * 34, PADB = NB / 32 * 34;
  // landing elements per peer: the runs, padded so that consecutive slots start 12 elements
  // apart modulo 16 (96 bytes): the 8-byte loads of one warp step, 4 consecutive elements from
  // each of 8 sources, then spread over the 32 banks two sources per bank group
  static constexpr int SLOT0 = PADA + PADB;
  static constexpr int SLOT = SLOT0 + ((12 - SLOT0 % 16) % 16 + 16) % 16;
  static constexpr int WARPS = T / 32;
  static constexpr int STEPS = JH / 32 / WARPS;   // 32-bin steps per warp per half
  static_assert((1 << LOGP) == P && P >= 2 && P <= 32, "P: a power of two");
  static_assert(KH % 32 == 0 && KH >= 32, "half runs of whole 32-element blocks");
  static_assert(STEPS * 32 * WARPS == JH, "warp steps");
  static_assert((SLOT * 8) % 16 == 0 && (PADA * 8) % 16 == 0 && (REGION * 8) % 16 == 0, "bulk copy alignment");

  // start (k) and padded length of the runs a CTA of rank c needs in half h
  __host__ __device__ static constexpr int a0(int c, int h) { return KC * c + KH * h; }
  __host__ __device__ static constexpr int b0(int c, int h) { return NP - a0(c, h) - KH - 32; }
  __host__ __device__ static constexpr int padb(int c, int h) { return (a0(c, h) == 0 ? NA : NB) / 32 * 34; }
  // bytes pushed into the landing of rank c for half h (P-1 peers)
  __host__ __device__ static constexpr unsigned bytes_in(int c, int h) {
    return (unsigned)(P - 1) * (unsigned)(PADA + padb(c, h)) * 8u;
  }
};

// Shared-memory layout (bytes): [0, 64) mbarriers (0, 8, 16) and a failure flag (32),
// twiddle table, buf, landing.
struct PushSmem {
  int tw, buf, land, total;
};
template <class PS>
__host__ __device__ inline PushSmem push_smem_layout(int tw_n) {
  PushSmem s;
  s.tw = 64;
  s.buf = s.tw + ((tw_n * 8 + 15) & ~15);
  s.land = s.buf + PS::REGION * 8;
  s.total = s.land + (PS::P - 1) * PS::SLOT * 8;
  return s;
}

__device__ __forceinline__ int pad32x2(int x) { return x + 2 * (x >> 5); }

template <class PS, int R0>
__global__ void __launch_bounds__(PS::T, 2) fused_push_kernel(const FusedArgs a) {
  using V = float2;
  using SH = typename PS::SH;
  constexpr int P = PS::P, NP = PS::NP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // (no static shared memory: the launcher sets the dynamic limit to the whole 227 KiB)
  volatile int& s_fail = *reinterpret_cast<int*>(smem_raw + 32);
  const int tw_n = a.tw_lo_n + a.tw_hi_n;
  const PushSmem L = push_smem_layout<PS>(tw_n);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* landed = full + 1;
  uint64_t* freeb = full + 2;
  V* tw_s = reinterpret_cast<V*>(smem_raw + L.tw);
  V* buf = reinterpret_cast<V*>(smem_raw + L.buf);
  V* land = reinterpret_cast<V*>(smem_raw + L.land);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c = (int)blockIdx.x;   // cluster rank = residue

  if (tid == 0) {
    mbar_init(full, 1);
    mbar_init(landed, P - 1);
    mbar_init(freeb, P - 1);
    fence_mbar_init();
    s_fail = 0;
  }
  for (int i = tid; i < tw_n; i += PS::T) tw_s[i] = reinterpret_cast<const V*>(a.tw)[i];
  __syncthreads();
  const TwTable<V> tab{tw_s, tw_s + a.tw_lo_n, a.tw_bits, (1u << a.tw_bits) - 1u};
  // every CTA's barriers are initialised before any remote access
  cluster_arrive();
  cluster_wait();

  const bool has_work = (long long)blockIdx.y < a.batch;
  // peers of this CTA: rank (c + 1 + i) % P for i < P - 1; my slot in peer d's landing is
  // (c - d - 1) mod P
  bool armed = false;   // `full` expects bytes for phase ph_full
  if (has_work) {
    if (tid == 0) mbar_arrive_expect_tx(full, PS::bytes_in(c, 0));
    armed = true;
    if (tid < P - 1) mbar_arrive_remote(dsmem_addr(freeb, (uint32_t)((c + 1 + tid) % P)));
  }

  const unsigned Mc = (unsigned)a.Mc;
  const unsigned long long M = (unsigned long long)a.M;
  const float hS = (float)a.scale * 0.5f;
  uint32_t ph_full = 0, ph_landed = 0, ph_free = 0;
  bool failed = false;
  auto fail_now = [&]() {
    s_fail = 1;
    if (a.status) atomicExch(a.status, kStatusTimeout);
  };

  for (long long sig = blockIdx.y; sig < a.batch; sig += gridDim.y) {
    if (sig != (long long)blockIdx.y) {
      // buf may be overwritten once every peer has received my previous half-1 pushes
      if (tid == 0 && !mbar_wait_cluster_bounded(landed, ph_landed)) fail_now();
      ph_landed ^= 1u;
      __syncthreads();
      if (s_fail) { failed = true; break; }
    }
    const void* u = reinterpret_cast<const unsigned char*>(a.in) + sig_in_bytes(a, sig);
    V* out = reinterpret_cast<V*>(a.out) + sig_out_off(a, sig);

    // ---- K1 + K2: residue twiddle, first radix, radix-16 Stockham passes (residue c)
    first_pass<R0, V, false, SH>(a, u, nullptr, kLoadRealPacked, buf, tab, c);
    __syncthreads();
    {
      constexpr int LOGR0 = R0 == 16 ? 4 : 5;
      int Ns = R0, logNs = LOGR0;
#pragma unroll
      for (int p = 1; p < SH_PASSES<SH, LOGR0>::value; ++p) {
        stockham_pass<16, 32, V, SH>(a, buf, tab, Ns, logNs);
        Ns <<= 4;
        logNs += 4;
      }
    }
    const bool more = sig + gridDim.y < a.batch;

    for (int h = 0; h < 2; ++h) {
      // ---- push half h of my residue to every peer
      if (warp == 0) {
        if (lane == 0 && !mbar_wait_cluster_bounded(freeb, ph_free)) fail_now();
        __syncwarp();
        if (lane < P - 1 && !s_fail) {
          const int d = (c + 1 + lane) % P;
          const int slot = (c - d - 1 + 2 * P) % P;
          fence_proxy_async_smem();
          const uint32_t dst = dsmem_addr(land + slot * PS::SLOT, (uint32_t)d);
          const uint32_t bar = dsmem_addr(full, (uint32_t)d);
          bulk_push_s2c(dst, buf + SH::pad(PS::a0(d, h)), PS::PADA * 8u, bar);
          bulk_push_s2c(dst + PS::PADA * 8u, buf + SH::pad(PS::b0(d, h)), (uint32_t)PS::padb(d, h) * 8u, bar);
        }
      }
      ph_free ^= 1u;
      // ---- wait for my landing (every thread observes the phase)
      if (!mbar_wait_cluster_bounded(full, ph_full)) fail_now();
      __syncthreads();
      if (s_fail) { failed = true; break; }
      ph_full ^= 1u;
      armed = false;
      if (h == 1 && warp == 0 && lane < P - 1)
        mbar_arrive_remote(dsmem_addr(landed, (uint32_t)((c + 1 + lane) % P)));

      // ---- epilogue of half h
      const int A0 = PS::a0(c, h), B0 = PS::b0(c, h);
      const unsigned jb = (unsigned)(PS::JC * c + PS::JH * h + warp * (PS::STEPS * 32));
      // Per lane the residue r = lane mod P is fixed, so the sources of U_j (residue r, k) and of
      // U_{Mc-j} (residue rm, k') are fixed too: this CTA's buf when the residue is c, else the
      // peer's slot in the landing.  Runs start at multiples of 32, so the padded index of k in
      // either place is base + pad32x2(k - run start); branch-free per lane.
      const V* sm = reinterpret_cast<const V*>(smem_raw);
      const int r_l = lane & (P - 1);
      const int rm_l = (P - r_l) & (P - 1);
      const int base_d = (r_l == c) ? L.buf / 8 + SH::pad(A0)
                                    : L.land / 8 + ((r_l - c - 1 + 2 * P) % P) * PS::SLOT;
      const int base_m = (rm_l == c) ? L.buf / 8 + SH::pad(B0)
                                     : L.land / 8 + ((rm_l - c - 1 + 2 * P) % P) * PS::SLOT + PS::PADA;
      auto unpack = [&](unsigned j, V& X1, V& X2) {
        const int k = (int)(j >> PS::LOGP);
        // mirror index: P (Np - 1 - k) + (P - r) for r > 0, P ((Np - k) mod Np) for r = 0
        const int km = r_l ? NP - 1 - k : (NP - k) & (NP - 1);
        const V Uj = sm[base_d + pad32x2(k - A0)];
        const V Up = sm[base_m + pad32x2(km - B0)];
        V wn = tab(j);
        wn = cmake<V>(hS * wn.y, -hS * wn.x);   // (S/2)(-i) W_M^j
        const V A = cadd(Uj, cconj(Up));
        const V B = csub(Uj, cconj(Up));
        const V t = cmul(wn, B);
        const V hA = cscale(A, hS);
        X1 = cadd(hA, t);
        X2 = csub(hA, t);
      };
      V P1 = czero<V>(), P2 = czero<V>();
#pragma unroll 2
      for (int t = 0; t <= PS::STEPS; ++t) {
        const unsigned j0 = jb + 32u * (unsigned)t;
        V X1, X2;
        unpack(j0 + (unsigned)lane, X1, X2);
        if (t < PS::STEPS) {
          st_stream(out + j0 + lane, X1);
          st_stream(out + Mc + j0 + lane, X2);
        }
        if (t > 0) {
          // mirror bins of the previous step, shifted by one: lane l stores Mc - j' and M - j'
          // for j' = jp + 32 - l (lane 32 - l of the previous step; lane 0 of this step for l = 0)
          const int src = (32 - lane) & 31;
          const float m1x = __shfl_sync(0xffffffffu, P1.x, src), m1y = __shfl_sync(0xffffffffu, P1.y, src);
          const float m2x = __shfl_sync(0xffffffffu, P2.x, src), m2y = __shfl_sync(0xffffffffu, P2.y, src);
          const float n1x = __shfl_sync(0xffffffffu, X1.x, 0), n1y = __shfl_sync(0xffffffffu, X1.y, 0);
          const float n2x = __shfl_sync(0xffffffffu, X2.x, 0), n2y = __shfl_sync(0xffffffffu, X2.y, 0);
          const V v1 = lane ? cmake<V>(m1x, m1y) : cmake<V>(n1x, n1y);
          const V v2 = lane ? cmake<V>(m2x, m2y) : cmake<V>(n2x, n2y);
          const unsigned jp = j0 - 32u;
          st_stream(out + (Mc - jp - 32u + (unsigned)lane), cconj(v2));
          st_stream(out + (M - jp - 32u + (unsigned)lane), cconj(v1));
        }
        P1 = X1;
        P2 = X2;
      }
      // ---- my landing is free again
      __syncthreads();
      if (tid == 0) {
        fence_proxy_async_smem();
        if (h == 0) mbar_arrive_expect_tx(full, PS::bytes_in(c, 1));
        else if (more) mbar_arrive_expect_tx(full, PS::bytes_in(c, 0));
      }
      armed = (h == 0) || more;
      __syncthreads();
      if (warp == 0 && lane < P - 1) mbar_arrive_remote(dsmem_addr(freeb, (uint32_t)((c + 1 + lane) % P)));
    }
    if (failed) break;
  }
  // a failed CTA lets copies still in flight towards its landing arrive before the cluster ends
  if (failed && armed && tid == 0) mbar_wait_cluster_bounded(full, ph_full);
  cluster_arrive();
  cluster_wait();
}

}  // namespace adfft
