// Device building blocks of the alpha-densified DFT kernels (sm_103a).
//
// - complex arithmetic on float2 / double2,
// - DFT_R in registers (R = 1..32) with compile-time constant roots of unity,
// - a two-level table of W_Mt^e = exp(-2 pi i e / Mt) staged in shared memory,
// - division by a run-time invariant (multiply-high + shift),
// - the shared-memory index padding used by every Stockham pass.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace adfft {

template <typename V> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };

template <typename V> __device__ __forceinline__ V cmake(typename real_of<V>::type x,
                                                         typename real_of<V>::type y) {
  V r; r.x = x; r.y = y; return r;
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return cmake<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return cmake<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return cmake<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {
  return cmake<V>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename V> __device__ __forceinline__ V cconj(V a) { return cmake<V>(a.x, -a.y); }
template <typename V> __device__ __forceinline__ V cscale(V a, typename real_of<V>::type s) {
  return cmake<V>(a.x * s, a.y * s);
}
// a * (-i)
template <typename V> __device__ __forceinline__ V cmul_mi(V a) { return cmake<V>(a.y, -a.x); }
// a * (+i)
template <typename V> __device__ __forceinline__ V cmul_pi(V a) { return cmake<V>(-a.y, a.x); }
template <typename V> __device__ __forceinline__ V czero() { return cmake<V>(0, 0); }

// cos(2 pi t / 32) and sin(2 pi t / 32) for t = 0..8 (the first octant and a half).
__host__ __device__ constexpr double kCos32(int t) {
  return t == 0 ? 1.0 : t == 1 ? 0.98078528040323044913 : t == 2 ? 0.92387953251128675613
       : t == 3 ? 0.83146961230254523708 : t == 4 ? 0.70710678118654752440
       : t == 5 ? 0.55557023301960222474 : t == 6 ? 0.38268343236508977173
       : t == 7 ? 0.19509032201612826785 : 0.0;
}
__host__ __device__ constexpr double kSin32(int t) { return kCos32(8 - t); }

// z * exp(-2 pi i t / 32) for a compile-time t in [0, 16).
template <typename V, int t> __device__ __forceinline__ V mul_root32(V z) {
  using R = typename real_of<V>::type;
  static_assert(t >= 0 && t < 16, "root index");
  if constexpr (t == 0) {
    return z;
  } else if constexpr (t == 8) {
    return cmul_mi(z);                                   // -i
  } else if constexpr (t == 4 || t == 12) {
    constexpr R h = (R)0.70710678118654752440;
    // t=4: (1 - i)/sqrt2 ; t=12: (-1 - i)/sqrt2
    if constexpr (t == 4) return cmake<V>((z.x + z.y) * h, (z.y - z.x) * h);
    else return cmake<V>((z.y - z.x) * h, -(z.x + z.y) * h);
  } else if constexpr (t < 8) {
    constexpr R c = (R)kCos32(t), s = (R)kSin32(t);
    return cmake<V>(z.x * c + z.y * s, z.y * c - z.x * s);
  } else {
    // exp(-2 pi i t/32) = -i * exp(-2 pi i (t-8)/32)
    constexpr R c = (R)kCos32(t - 8), s = (R)kSin32(t - 8);
    V w = cmake<V>(z.x * c + z.y * s, z.y * c - z.x * s);
    return cmul_mi(w);
  }
}

// In-register forward DFT of length R (power of two <= 32), natural order in and out:
//   v[k] <- sum_r v[r] exp(-2 pi i r k / R).
// Radix-2 decimation in frequency, unrolled at compile time.
template <int R, typename V> struct DFT {
  static __device__ __forceinline__ void run(V* v) {
    constexpr int H = R / 2;
    V a[H], b[H];
#pragma unroll
    for (int r = 0; r < H; ++r) {
      a[r] = cadd(v[r], v[r + H]);
      b[r] = csub(v[r], v[r + H]);
    }
    twiddle_half(b, std::integral_constant<int, 0>());
    DFT<H, V>::run(a);
    DFT<H, V>::run(b);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      v[2 * k] = a[k];
      v[2 * k + 1] = b[k];
    }
  }
  template <int r>
  static __device__ __forceinline__ void twiddle_half(V* b, std::integral_constant<int, r>) {
    if constexpr (r < R / 2) {
      b[r] = mul_root32<V, (r * (32 / R)) % 32>(b[r]);
      twiddle_half(b, std::integral_constant<int, r + 1>());
    }
  }
};
template <typename V> struct DFT<1, V> {
  static __device__ __forceinline__ void run(V*) {}
};

// Two-level table of W_Mt^e = exp(-2 pi i e/Mt), 0 <= e < Mt:
//   W_Mt^e = hi[e >> bits] * lo[e & (2^bits - 1)].
// Both levels are computed on the host in double precision and rounded once.
template <typename V> struct TwTable {
  const V* lo;
  const V* hi;
  int bits;
  unsigned mask;
  __device__ __forceinline__ V operator()(unsigned e) const { return cmul(hi[e >> bits], lo[e & mask]); }
};

// Unsigned division by a run-time invariant d >= 1 for dividends n < 2^31:
//   q = (umulhi(n, mul) + n) >> shift, with shift = ceil(log2 d),
//   mul = floor(2^32 (2^shift - d) / d) + 1.
struct FastDiv {
  uint32_t d, mul, shift;
};
__host__ inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  uint32_t l = 0;
  while ((1ull << l) < d) ++l;
  f.shift = l;
  f.mul = (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
  return f;
}
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
  return (__umulhi(n, f.mul) + n) >> f.shift;
}

// Shared-memory element index with one pad slot per 16 elements: keeps the
// strided writes of the first Stockham passes (stride R in elements) and the
// unit-stride reads on distinct banks for 8- and 16-byte elements.
__device__ __forceinline__ int pad16(int p) { return p + (p >> 4); }

}  // namespace adfft

namespace adfft {

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA engine) and mbarriers, sm_90+ PTX.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Orders this thread's (and, after a CTA barrier, the CTA's) generic-proxy
// shared-memory accesses before later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned),
// completion signalled on `bar` as transaction bytes.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
// Wait for phase `phase` of `bar` to complete, giving up after ~2 s of SM clock.
constexpr long long kWaitLimitCycles = 4000000000ll;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase,
                                                  long long limit = kWaitLimitCycles) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, phase)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}


// mbarrier wait with cluster-scope acquire: makes visible what peers released before their
// (remote) arrives on this barrier.  Gives up after ~2 s of SM clock.
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cluster_bounded(uint64_t* bar, uint32_t phase) {
  const long long t0 = clock64();
  while (!mbar_try_wait_cluster(bar, phase)) {
    if (clock64() - t0 > kWaitLimitCycles) return false;
  }
  return true;
}
// Arrive (release, cluster scope) on an mbarrier of another CTA of the cluster, given its
// shared::cluster address.
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from this CTA's shared
// memory into the shared memory of another CTA of the cluster (dst and its mbarrier given as
// shared::cluster addresses); completion is signalled on that mbarrier as transaction bytes.
__device__ __forceinline__ void bulk_push_s2c(uint32_t dst_cluster, const void* src, uint32_t bytes,
                                              uint32_t bar_cluster) {
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst_cluster),
      "r"(smem_u32(src)), "r"(bytes), "r"(bar_cluster)
      : "memory");
}

// Split cluster barrier (all threads of every CTA of the cluster take part).
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
// Arrive without release semantics: for a barrier whose only job is to say
// "this CTA has finished reading its peers' shared memory" (every such load has
// been consumed by then), so it need not wait for the thread's global stores.
__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Distributed shared memory: 32-bit shared::cluster address of `p` (a pointer
// into this CTA's shared memory) in the shared memory of cluster rank `rank`.
__device__ __forceinline__ uint32_t dsmem_addr(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ float2 dsmem_ld(uint32_t addr, float2) {
  float2 v;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void dsmem_st(uint32_t addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void dsmem_st(uint32_t addr, double2 v) {
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(addr), "d"(v.x), "d"(v.y) : "memory");
}
// Two adjacent float2 elements (16 bytes, 16-byte aligned address).
__device__ __forceinline__ void dsmem_ld_pair(uint32_t addr, float2& a, float2& b) {
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(a.x), "=f"(a.y), "=f"(b.x), "=f"(b.y)
               : "r"(addr)
               : "memory");
}
__device__ __forceinline__ double2 dsmem_ld(uint32_t addr, double2) {
  double2 v;
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(addr) : "memory");
  return v;
}

// Streaming (evict-first) global stores for outputs that are written once.
__device__ __forceinline__ void st_stream(float2* p, float2 v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(double2* p, double2 v) { __stcs(p, v); }

}  // namespace adfft
