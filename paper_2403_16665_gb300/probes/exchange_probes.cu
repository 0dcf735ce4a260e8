// Micro-benchmarks of the data paths the fused kernels' output exchange can take on this
// GPU (measurement tool, not part of the library):
//   write   - 4 GiB of complex64 output written coalesced, as per-CTA strided residue runs
//             (runs that share 32-byte sectors with other CTAs), and as single-bin strides;
//   dsmem   - every CTA of a cluster receives 64 KiB from its peers per iteration, by
//             distributed-shared-memory loads (pull) or by bulk shared::cta -> shared::cluster
//             copies (push), for clusters of 4, 8 and 16 at one or two CTAs per SM;
//   overlap - a push exchange of 96 KiB and 256 KiB of output per CTA (clusters of 4), alone
//             and together, output by ordinary stores or by bulk stores;
//   l2      - the same exchange through an L2-resident global scratch buffer instead;
//   place   - which SMs the CTAs of a cluster land on when two CTAs fit on one SM.
// Build and run: python -m paper_2403_16665_gb300.profile --probes
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>
#include <cooperative_groups.h>
namespace cg = cooperative_groups;
#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("err %s line %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

namespace write_probe {
// Write-pattern micro-benchmark: 4096 x 131072 float2 (4 GiB) output.
constexpr long long SIG = 4096, MB = 131072;

__global__ void k_coal(float4* o, long long n4) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x)
    __stcs(o + i, make_float4(1.f, 2.f, 3.f, 4.f));
}
// P=64, 8 units per signal; unit t owns residues {4t..4t+3} U {61-4t..64-4t} (t=0: {61,62,63} + 32)
template <bool SPREAD>
__global__ void k_d3(float2* o) {
  const long long units = SIG * 8;
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    long long s; int t;
    if (SPREAD) { t = (int)(u / SIG); s = u % SIG; } else { s = u / 8; t = (int)(u % 8); }
    float2* base = o + s * MB;
    for (int idx = threadIdx.x; idx < 2048 * 4; idx += blockDim.x) {
      const int k = idx >> 2, d = idx & 3;
      __stcs(base + 64 * k + 4 * t + d, make_float2(1.f, (float)d));
      if (t > 0 || d < 3) __stcs(base + 64 * k + 61 - 4 * t + d, make_float2(2.f, (float)d));
      else __stcs(base + 64 * k + 32, make_float2(3.f, 0.f));
    }
  }
}
// P=8 single residue per unit (stride-8 bins)
__global__ void k_stride8(float2* o) {
  const long long units = SIG * 8;
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    const long long s = u / 8; const int t = (int)(u % 8);
    float2* base = o + s * MB;
    for (int k = threadIdx.x; k < 16384; k += blockDim.x) __stcs(base + 8 * k + t, make_float2(1.f, 0.f));
  }
}
// P=32, 4 units: {4t..4t+3} U {29-4t .. 32-4t} (t=0: {29,30,31} + 16)
__global__ void k_p32(float2* o) {
  const long long units = SIG * 4;
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    const long long s = u / 4; const int t = (int)(u % 4);
    float2* base = o + s * MB;
    for (int idx = threadIdx.x; idx < 4096 * 4; idx += blockDim.x) {
      const int k = idx >> 2, d = idx & 3;
      __stcs(base + 32 * k + 4 * t + d, make_float2(1.f, (float)d));
      if (t > 0 || d < 3) __stcs(base + 32 * k + 29 - 4 * t + d, make_float2(2.f, (float)d));
      else __stcs(base + 32 * k + 16, make_float2(3.f, 0.f));
    }
  }
}
int run_all() {
  float2* o; size_t bytes = SIG * MB * sizeof(float2);
  CK(cudaMalloc(&o, bytes));
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
  auto run = [&](const char* name, auto launch) {
    for (int i = 0; i < 3; ++i) launch();
    cudaEventRecord(a);
    for (int i = 0; i < 10; ++i) launch();
    cudaEventRecord(b); cudaEventSynchronize(b);
    float ms; cudaEventElapsedTime(&ms, a, b); ms /= 10;
    printf("%-28s %8.3f ms  %8.1f GB/s  (%s)\n", name, ms, bytes / ms / 1e6, cudaGetErrorString(cudaGetLastError()));
  };
  run("coalesced float4", [&] { k_coal<<<sms * 4, 512>>>((float4*)o, (long long)(bytes / 16)); });
  for (int cps = 2; cps <= 4; cps += 1) {
    char nm[64];
    snprintf(nm, 64, "d3 P64 8 units %d/SM", cps); run(nm, [&] { k_d3<false><<<sms * cps, 256>>>(o); });
  }
  run("d3 P64 spread units 3/SM", [&] { k_d3<true><<<sms * 3, 256>>>(o); });
  run("p32 4 units 1/SM 512t", [&] { k_p32<<<sms, 512>>>(o); });
  run("p32 4 units 2/SM 512t", [&] { k_p32<<<sms * 2, 512>>>(o); });
  run("stride8 3/SM", [&] { k_stride8<<<sms * 3, 256>>>(o); });
  CK(cudaDeviceSynchronize());
  return 0;
}

}  // namespace write_probe

namespace dsmem_probe {
// DSMEM exchange micro-benchmark: every CTA of a cluster of CL receives BUFB bytes
// (BUFB/CL from each peer) per iteration, by pull loads or by bulk push copies.

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t mapa(uint32_t a, uint32_t rank) { uint32_t r; asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank)); return r; }
__device__ __forceinline__ float4 ld_dsm(uint32_t a) { float4 v; asm volatile("ld.shared::cluster.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a) : "memory"); return v; }
__device__ __forceinline__ void cl_sync() { asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory"); }
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t c) { asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(b)), "r"(c) : "memory"); }
__device__ __forceinline__ void expect_tx(uint64_t* b, uint32_t bytes) { asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(b)), "r"(bytes) : "memory"); }
__device__ __forceinline__ bool try_wait(uint64_t* b, uint32_t ph) { uint32_t ok; asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\nselp.u32 %0,1,0,p;\n}" : "=r"(ok) : "r"(smem_u32(b)), "r"(ph) : "memory"); return ok; }
__device__ __forceinline__ void push(uint32_t dst_cluster, const void* src, uint32_t bytes, uint32_t bar_cluster) {
  asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" :: "r"(dst_cluster), "r"(smem_u32(src)), "r"(bytes), "r"(bar_cluster) : "memory");
}

template <int MODE, int CL, int BUFB, int NCH, int UL>
__global__ void xk(int iters, long long* cyc, float* sink) {
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t* bar = (uint64_t*)sm;
  unsigned char* buf = sm + 128;
  unsigned char* land = buf + BUFB;
  const uint32_t me = cg::this_cluster().block_rank();
  for (int i = threadIdx.x; i < BUFB / 4; i += blockDim.x) ((float*)buf)[i] = (float)(i + me);
  if (threadIdx.x == 0) { mbar_init(bar, 1); asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
  __syncthreads();
  cl_sync();
  float acc = 0.f;
  long long t0 = clock64();
  uint32_t ph = 0;
  constexpr int CH = BUFB / CL;          // bytes this CTA gets from each peer
  for (int it = 0; it < iters; ++it) {
    if (MODE == 0) {
      // pull: thread reads 16-byte items; item idx -> peer idx / (CH/16), offset
      const int items = BUFB / 16;
      for (int i0 = threadIdx.x; i0 < items; i0 += blockDim.x * UL) {
        float4 v[UL];
#pragma unroll
        for (int u = 0; u < UL; ++u) {
          const int i = i0 + u * blockDim.x;
          if (i < items) {
            const int p = i / (CH / 16), off = (i % (CH / 16)) * 16 + me * CH;
            v[u] = ld_dsm(mapa(smem_u32(buf + off), p));
          } else v[u] = make_float4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < UL; ++u) acc += v[u].x + v[u].w;
      }
      cl_sync();
    } else {
      // push: thread 0 expects BUFB bytes, then pushes my chunk for each peer (NCH pieces each)
      if (threadIdx.x == 0) expect_tx(bar, BUFB);
      cl_sync();   // every landing zone is free and expecting
      if (threadIdx.x < CL) {
        const uint32_t p = threadIdx.x;
        const uint32_t dbar = mapa(smem_u32(bar), p);
        for (int c = 0; c < NCH; ++c) {
          const uint32_t off = c * (CH / NCH);
          push(mapa(smem_u32(land + me * CH + off), p), buf + p * CH + off, CH / NCH, dbar);
        }
      }
      long long w0 = clock64();
      while (!try_wait(bar, ph)) { if (clock64() - w0 > 2000000000ll) break; }
      ph ^= 1;
      for (int i = threadIdx.x; i < BUFB / 16; i += blockDim.x * 8) acc += ((float*)land)[i * 4];
      // sources: wait own pushes' reads before the next iteration
      if (threadIdx.x < CL) asm volatile("cp.async.bulk.commit_group;\ncp.async.bulk.wait_group.read 0;" ::: "memory");
      __syncthreads();
    }
  }
  long long t1 = clock64();
  cl_sync();
  if (threadIdx.x == 0 && blockIdx.x == 0) *cyc = t1 - t0;
  if (acc == 123.f) sink[threadIdx.x] = acc;
}

template <int MODE, int CL, int BUFB, int NCH, int UL>
int run(const char* name, int threads, int smem_extra, int sms) {
  auto k = xk<MODE, CL, BUFB, NCH, UL>;
  const int smem = 128 + 2 * BUFB + smem_extra;
  CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  CK(cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension; at[0].val.clusterDim.x = CL; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
  cfg.attrs = at; cfg.numAttrs = 1; cfg.blockDim = dim3(threads); cfg.dynamicSmemBytes = smem;
  cfg.gridDim = dim3(CL);
  int ncl = 0; CK(cudaOccupancyMaxActiveClusters(&ncl, k, &cfg));
  cfg.gridDim = dim3(CL * ncl);
  long long* cyc; float* sink; CK(cudaMalloc(&cyc, 8)); CK(cudaMalloc(&sink, 4096));
  const int iters = 2000;
  CK(cudaLaunchKernelEx(&cfg, k, 10, cyc, sink));
  CK(cudaDeviceSynchronize());
  cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
  cudaEventRecord(a);
  CK(cudaLaunchKernelEx(&cfg, k, iters, cyc, sink));
  cudaEventRecord(b); CK(cudaEventSynchronize(b));
  float ms; cudaEventElapsedTime(&ms, a, b);
  long long c; cudaMemcpy(&c, cyc, 8, cudaMemcpyDeviceToHost);
  const double bytes = (double)BUFB * CL * ncl * iters;
  printf("%-34s clusters %3d (CTAs %4d) smem %6d thr %4d: %7.0f cyc/iter, %6.1f B/clk/CTA, agg %7.1f GB/s\n", name, ncl, CL * ncl, smem, threads,
         (double)c / iters, (double)BUFB * iters / c, bytes / ms / 1e6);
  cudaFree(cyc); cudaFree(sink);
  return 0;
}

int run_all() {
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  printf("SMs %d\n", sms);
  // 1 CTA per SM (big smem)
  run<0, 8, 65536, 1, 4>("pull  CL8 64K UL4 1/SM", 512, 60000, sms);
  run<0, 8, 65536, 1, 8>("pull  CL8 64K UL8 1/SM", 512, 60000, sms);
  run<0, 8, 65536, 1, 8>("pull  CL8 64K UL8 1/SM 256t", 256, 60000, sms);
  run<1, 8, 65536, 1, 1>("push  CL8 64K 8KB x1 1/SM", 512, 60000, sms);
  run<1, 8, 65536, 2, 1>("push  CL8 64K 4KB x2 1/SM", 512, 60000, sms);
  run<1, 8, 65536, 8, 1>("push  CL8 64K 1KB x8 1/SM", 512, 60000, sms);
  run<0, 4, 65536, 1, 8>("pull  CL4 64K UL8 1/SM", 512, 60000, sms);
  run<1, 4, 65536, 1, 1>("push  CL4 64K 16KB 1/SM", 512, 60000, sms);
  run<1, 16, 65536, 1, 1>("push  CL16 64K 4KB 1/SM", 512, 60000, sms);
  // 2 CTAs per SM
  run<0, 8, 32768, 1, 8>("pull  CL8 32K UL8 2/SM", 256, 30000, sms);
  run<1, 8, 32768, 1, 1>("push  CL8 32K 4KB 2/SM", 256, 30000, sms);
  run<1, 16, 32768, 1, 1>("push  CL16 32K 2KB 2/SM", 256, 30000, sms);
  return 0;
}

}  // namespace dsmem_probe

namespace overlap_probe {
// Does a DSMEM push exchange overlap with the output stream?  Clusters of 4 CTAs (1 per SM);
// per iteration every CTA receives 96 KB from its 3 peers (push bulk copies) and/or writes
// 256 KB of output (LSU stores, or bulk stores from shared memory).
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t mapa(uint32_t a, uint32_t rank) { uint32_t r; asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank)); return r; }
__device__ __forceinline__ void cl_sync() { asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory"); }
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t c) { asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(smem_u32(b)), "r"(c) : "memory"); }
__device__ __forceinline__ void expect_tx(uint64_t* b, uint32_t bytes) { asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(smem_u32(b)), "r"(bytes) : "memory"); }
__device__ __forceinline__ bool try_wait(uint64_t* b, uint32_t ph) { uint32_t ok; asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\nselp.u32 %0,1,0,p;\n}" : "=r"(ok) : "r"(smem_u32(b)), "r"(ph) : "memory"); return ok; }
__device__ __forceinline__ void push(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" :: "r"(dst), "r"(smem_u32(src)), "r"(bytes), "r"(bar) : "memory");
}
__device__ __forceinline__ void bulk_store(void* g, const void* s, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" :: "l"(g), "r"(smem_u32(s)), "r"(bytes) : "memory");
}

constexpr int CL = 4, XB = 98304, PEERB = XB / 3, OUTB = 262144;   // 96 KB exchange, 256 KB out
template <bool EX, int OUTMODE, int CHUNK>
__global__ void __launch_bounds__(512) k2(int iters, float4* out, long long out_units, long long* cyc, float* sink, int* fail) {
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t* bar = (uint64_t*)sm;
  unsigned char* src = sm + 128;              // 96 KB: what this CTA sends (32 KB per peer)
  unsigned char* land = src + XB;             // 96 KB: 3 slots of 32 KB
  const uint32_t me = cg::this_cluster().block_rank();
  for (int i = threadIdx.x; i < XB / 4; i += blockDim.x) ((float*)src)[i] = (float)(i ^ me);
  if (threadIdx.x == 0) { mbar_init(bar, 1); asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
  __syncthreads();
  cl_sync();
  const int G = gridDim.x;
  uint32_t ph = 0;
  float acc = 0.f;
  long long t0 = clock64();
  for (int t = 0; t < iters; ++t) {
    if (EX) {
      if (threadIdx.x == 0) expect_tx(bar, XB);
      cl_sync();
      if (threadIdx.x < 3 * (PEERB / CHUNK)) {
        const int q = threadIdx.x / (PEERB / CHUNK), c = threadIdx.x % (PEERB / CHUNK);
        const uint32_t p = (me + 1 + q) % CL;                 // peer
        const uint32_t slot = (me + CL - p - 1) % CL;          // my slot index in the peer's landing (0..2)
        push(mapa(smem_u32(land + slot * PEERB + c * CHUNK), p), src + q * PEERB + c * CHUNK, CHUNK, mapa(smem_u32(bar), p));
      }
    }
    if (OUTMODE) {
      const long long unit = ((long long)t * G + blockIdx.x) % out_units;
      float4* o = out + unit * (OUTB / 16);
      if (OUTMODE == 1) {
        for (int i = threadIdx.x; i < OUTB / 16; i += 512) __stcs(o + i, make_float4(acc, 1.f, 2.f, 3.f));
      } else if (threadIdx.x == 0) {
        // 256 KB from the 96 KB source region in 8 bulk stores of 32 KB
        for (int c = 0; c < 8; ++c) bulk_store(o + c * (32768 / 16), src + (c % 3) * 32768, 32768);
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
    }
    if (EX) {
      long long w0 = clock64();
      while (!try_wait(bar, ph)) { if (clock64() - w0 > 2000000000ll) { atomicExch(fail, 1); break; } }
      ph ^= 1;
      acc += ((float*)land)[threadIdx.x * 16];
      if (threadIdx.x < 3 * (PEERB / CHUNK)) asm volatile("cp.async.bulk.commit_group;\ncp.async.bulk.wait_group.read 0;" ::: "memory");
    }
    if (OUTMODE == 2 && threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    __syncthreads();
  }
  long long t1 = clock64();
  if (OUTMODE == 2 && threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  cl_sync();
  if (threadIdx.x == 0 && blockIdx.x == 0) *cyc = t1 - t0;
  if (acc == 123.f) sink[threadIdx.x] = acc;
}

template <bool EX, int OUTMODE, int CHUNK>
int run(const char* name) {
  auto k = k2<EX, OUTMODE, CHUNK>;
  const int smem = 128 + 2 * XB;
  CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension; at[0].val.clusterDim.x = CL; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
  cfg.attrs = at; cfg.numAttrs = 1; cfg.blockDim = dim3(512); cfg.dynamicSmemBytes = smem; cfg.gridDim = dim3(CL);
  int ncl = 0; CK(cudaOccupancyMaxActiveClusters(&ncl, k, &cfg));
  cfg.gridDim = dim3(CL * ncl);
  const long long out_units = 16384;   // 4 GiB
  float4* out; long long* cyc; float* sink; int* fail;
  CK(cudaMalloc(&out, (size_t)out_units * OUTB)); CK(cudaMalloc(&cyc, 8)); CK(cudaMalloc(&sink, 4096)); CK(cudaMalloc(&fail, 4));
  CK(cudaMemset(fail, 0, 4));
  const int G = CL * ncl, iters = (int)(out_units / G);
  cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
  float ms = 0;
  for (int rep = 0; rep < 2; ++rep) {
    cudaEventRecord(a);
    CK(cudaLaunchKernelEx(&cfg, k, iters, out, out_units, cyc, sink, fail));
    cudaEventRecord(b); CK(cudaEventSynchronize(b));
    cudaEventElapsedTime(&ms, a, b);
  }
  long long c; int f; cudaMemcpy(&c, cyc, 8, cudaMemcpyDeviceToHost); cudaMemcpy(&f, fail, 4, cudaMemcpyDeviceToHost);
  const double units = (double)G * iters;
  printf("%-30s CTAs %d iters %d: %7.0f cyc/iter, %.3f ms (per 16384 units %.3f ms), xch %.0f GB/s, out %.0f GB/s%s\n", name, G, iters,
         (double)c / iters, ms, ms * 16384.0 / units, EX ? units * XB / ms / 1e6 : 0.0, OUTMODE ? units * OUTB / ms / 1e6 : 0.0, f ? " FAIL" : "");
  cudaFree(out); cudaFree(cyc); cudaFree(sink); cudaFree(fail);
  return 0;
}
int run_all() {
  run<true, 0, 1024>("exch 96K (1KB copies)");
  run<true, 0, 4096>("exch 96K (4KB copies)");
  run<false, 1, 1024>("out LSU 256K");
  run<false, 2, 1024>("out bulk 256K");
  run<true, 1, 1024>("exch + out LSU");
  run<true, 2, 1024>("exch + out bulk");
  run<true, 2, 4096>("exch4K + out bulk");
  return 0;
}

}  // namespace overlap_probe

namespace l2_probe {
// L2 exchange micro-benchmark: persistent CTAs in groups of 8 (no clusters); per iteration each
// CTA writes 64 KB (its "residue") to a scratch slot, the group synchronises through a global
// counter, then each CTA reads 64 KB (16 runs of 4 KB, from all 8 slots) and optionally writes
// 128 KiB of output.

__device__ __forceinline__ unsigned ld_acq(const unsigned* p) { unsigned v; asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory"); return v; }
__device__ __forceinline__ void red_rel(unsigned* p, unsigned v) { asm volatile("red.release.gpu.global.add.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory"); }

template <bool EXCH, bool OUT, int UL, int FMA>
__global__ void __launch_bounds__(256) lk(int iters, float4* scratch, unsigned* cnt, float4* out, long long out_units, long long* cyc, float* sink, int* fail) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int G = gridDim.x, b = blockIdx.x, grp = b / 8, rank = b % 8;
  float acc = 0.f;
  long long t0 = clock64();
  for (int t = 0; t < iters; ++t) {
    // pretend compute: FMA chain
    float z = (float)threadIdx.x;
    for (int i = 0; i < FMA; ++i) z = fmaf(z, 1.0001f, 0.5f);
    acc += z;
    if (EXCH) {
      float4* slot = scratch + ((size_t)(grp * 2 + (t & 1)) * 8 + rank) * 4096;   // 64 KB = 4096 float4
      for (int i = threadIdx.x; i < 4096; i += 256) slot[i] = make_float4(acc, (float)i, (float)t, 1.f);
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        red_rel(cnt + grp * 32, 1u);
        const unsigned want = 8u * (unsigned)(t + 1);
        long long w0 = clock64();
        while (ld_acq(cnt + grp * 32) < want) { if (clock64() - w0 > 2000000000ll) { atomicExch(fail, 1); break; } }
      }
      __syncthreads();
      // read 16 runs of 4 KB: run (p, h): slot p, offset (rank*2 + h) * 256 float4
      const float4* base = scratch + (size_t)(grp * 2 + (t & 1)) * 8 * 4096;
      for (int i0 = threadIdx.x; i0 < 4096; i0 += 256 * UL) {
        float4 v[UL];
#pragma unroll
        for (int u = 0; u < UL; ++u) {
          const int i = i0 + u * 256;
          const int run = i >> 8, p = run >> 1, h = run & 1;
          v[u] = __ldcg(base + (size_t)p * 4096 + (rank * 2 + h) * 256 + (i & 255));
        }
#pragma unroll
        for (int u = 0; u < UL; ++u) acc += v[u].x + v[u].w;
      }
    }
    if (OUT) {
      const long long unit = ((long long)t * G + b) % out_units;
      float4* o = out + unit * 8192;   // 128 KiB
      for (int i = threadIdx.x; i < 8192; i += 256) __stcs(o + i, make_float4(acc, 1.f, 2.f, 3.f));
    }
  }
  long long t1 = clock64();
  if (threadIdx.x == 0 && b == 0) *cyc = t1 - t0;
  if (acc == 123.f) sink[threadIdx.x] = acc;
}

template <bool EXCH, bool OUT, int UL, int FMA>
int run(const char* name, int cps, int smem) {
  auto k = lk<EXCH, OUT, UL, FMA>;
  CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  int occ = 0; CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, 256, smem));
  if (occ < cps) { printf("%s: occupancy %d < %d\n", name, occ, cps); return 0; }
  const int G = (sms * cps) / 8 * 8;
  float4 *scratch, *out; unsigned* cnt; long long* cyc; float* sink; int* fail;
  const long long out_units = 32768;   // 4 GiB of output
  CK(cudaMalloc(&scratch, (size_t)(G / 8) * 2 * 8 * 65536));
  CK(cudaMalloc(&out, (size_t)out_units * 131072));
  CK(cudaMalloc(&cnt, (G / 8) * 32 * 4)); CK(cudaMalloc(&cyc, 8)); CK(cudaMalloc(&sink, 4096)); CK(cudaMalloc(&fail, 4));
  const int iters = 32768 / G * 4;
  cudaEvent_t a, c; cudaEventCreate(&a); cudaEventCreate(&c);
  float ms = 0;
  for (int rep = 0; rep < 2; ++rep) {
    CK(cudaMemset(cnt, 0, (G / 8) * 32 * 4)); CK(cudaMemset(fail, 0, 4));
    cudaEventRecord(a);
    k<<<G, 256, smem>>>(iters, scratch, cnt, out, out_units, cyc, sink, fail);
    cudaEventRecord(c); CK(cudaEventSynchronize(c));
    cudaEventElapsedTime(&ms, a, c);
  }
  long long cy; int f; cudaMemcpy(&cy, cyc, 8, cudaMemcpyDeviceToHost); cudaMemcpy(&f, fail, 4, cudaMemcpyDeviceToHost);
  const double units = (double)G * iters;
  printf("%-36s G %4d iters %4d: %7.0f cyc/iter/CTA, %7.3f ms, per 32768 units %.3f ms, xch %6.1f GB/s, out %6.1f GB/s%s\n", name, G, iters,
         (double)cy / iters, ms, ms * 32768.0 / units, EXCH ? units * 65536 / ms / 1e6 : 0.0, OUT ? units * 131072 / ms / 1e6 : 0.0, f ? " FAIL" : "");
  cudaFree(scratch); cudaFree(out); cudaFree(cnt); cudaFree(cyc); cudaFree(sink); cudaFree(fail);
  return 0;
}

int run_all() {
  run<true, false, 8, 0>("exch only 2/SM UL8", 2, 80000);
  run<true, false, 16, 0>("exch only 2/SM UL16", 2, 80000);
  run<true, false, 8, 0>("exch only 3/SM UL8", 3, 70000);
  run<false, true, 8, 0>("out only 2/SM", 2, 80000);
  run<true, true, 8, 0>("exch+out 2/SM UL8", 2, 80000);
  run<true, true, 8, 0>("exch+out 3/SM UL8", 3, 70000);
  run<true, true, 8, 2000>("exch+out+2000fma 2/SM", 2, 80000);
  run<false, true, 8, 2000>("out+2000fma 2/SM", 2, 80000);
  return 0;
}

}  // namespace l2_probe

namespace place_probe {
// Where does the hardware place the CTAs of 8-CTA clusters when two CTAs fit on one SM?
__global__ void pk(int* smid, int spin) {
  extern __shared__ unsigned char sm[];
  unsigned s; asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
  if (threadIdx.x == 0) smid[blockIdx.x] = (int)s;
  long long t0 = clock64(); while (clock64() - t0 < spin) {}
  sm[threadIdx.x] = 1;
  cg::this_cluster().sync();
}
int run(int CL, int smem, int threads) {
  cudaFuncSetAttribute(pk, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(pk, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {}; cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension; at[0].val.clusterDim.x = CL; at[0].val.clusterDim.y = 1; at[0].val.clusterDim.z = 1;
  cfg.attrs = at; cfg.numAttrs = 1; cfg.blockDim = dim3(threads); cfg.dynamicSmemBytes = smem; cfg.gridDim = dim3(CL);
  int ncl = 0; cudaOccupancyMaxActiveClusters(&ncl, pk, &cfg);
  cfg.gridDim = dim3(CL * ncl);
  int* d; cudaMalloc(&d, 4 * CL * ncl);
  cudaLaunchKernelEx(&cfg, pk, d, 2000000);
  cudaError_t e = cudaDeviceSynchronize();
  int h[4096]; cudaMemcpy(h, d, 4 * CL * ncl, cudaMemcpyDeviceToHost);
  int same = 0, diff = 0, cnt[256] = {0}, first[256]; for (int i = 0; i < 256; ++i) first[i] = -1;
  for (int b = 0; b < CL * ncl; ++b) { int s = h[b]; cnt[s]++; if (first[s] < 0) first[s] = b / CL; else if (first[s] == b / CL) same++; else diff++; }
  int used = 0; for (int i = 0; i < 256; ++i) used += cnt[i] > 0;
  printf("CL %2d smem %6d thr %d: clusters %d, SMs used %d, co-resident pairs same cluster %d, different clusters %d (%s)\n", CL, smem, threads, ncl, used, same, diff, cudaGetErrorString(e));
  printf("  cluster 0 SMs:"); for (int r = 0; r < CL; ++r) printf(" %d", h[r]); printf("\n");
  cudaFree(d); return 0;
}
int run_all() { run(8, 100000, 256); run(8, 70000, 256); run(4, 100000, 256); run(16, 100000, 256); run(2, 100000, 256); run(8, 200000, 256); return 0; }

}  // namespace place_probe


int main(int argc, char** argv) {
  const char* which = argc > 1 ? argv[1] : "all";
  int rc = 0;
  if (!strcmp(which, "all") || !strcmp(which, "write")) { printf("== write\n"); rc |= write_probe::run_all(); }
  if (!strcmp(which, "all") || !strcmp(which, "dsmem")) { printf("== dsmem\n"); rc |= dsmem_probe::run_all(); }
  if (!strcmp(which, "all") || !strcmp(which, "overlap")) { printf("== overlap\n"); rc |= overlap_probe::run_all(); }
  if (!strcmp(which, "all") || !strcmp(which, "l2")) { printf("== l2\n"); rc |= l2_probe::run_all(); }
  if (!strcmp(which, "all") || !strcmp(which, "place")) { printf("== place\n"); rc |= place_probe::run_all(); }
  return rc;
}
