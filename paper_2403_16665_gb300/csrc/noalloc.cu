// adfft_execute_noalloc: the forward transform for callers that cannot
// allocate device memory.
//
// It runs the two-pass (four-step) form of the transform, whose intermediate
// needs scratch memory, with that scratch (and the twiddle tables the passes
// read) in one file-scope static device array instead of plan-owned
// allocations.  Nothing here calls cudaMalloc, cudaFree or any other
// allocating routine; the host side only does arithmetic, one-time symbol and
// function-attribute set-up, and kernel launches.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "adfft_internal.h"

namespace adfft {

namespace {

// Fixed device storage: 1 MiB of twiddle tables followed by 32 MiB of scratch
// for the pass-1 intermediate ([batch][B][R1] complex64).  Every GPU that loads
// the library holds this array until the process exits.
constexpr size_t kNoAllocTableBytes = size_t(1) << 20;
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_mem[kNoAllocTableBytes + kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_noalloc_addr[kMaxDevices];   // device address of g_noalloc_mem, per device, once set up
// Sizes (R1, Mc, B, M) whose tables the array holds on each device, so that consecutive
// calls with the same sizes do not rewrite them; all zero = none.  Guarded by g_setup_mutex.
long long g_table_key[kMaxDevices][4];

int64_t gcd_i64(int64_t a, int64_t b) {
  while (b) {
    const int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}
bool pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
int log2i(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l;
}

// Two-level table of W_X (lo: 2^bits entries, hi: ceil(X / 2^bits) entries)
// written by one thread per entry, in double precision and rounded to float.
__global__ void noalloc_table_kernel(float2* dst, long long X, int bits, int lo_n, int total) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  long long e = (i < lo_n) ? (long long)i : (long long)(i - lo_n) << bits;
  e %= X;
  const long long k = (2 * e > X) ? e - X : e;   // symmetric range
  double s, c;
  sincospi(2.0 * (double)k / (double)X, &s, &c);
  dst[i] = make_float2((float)c, (float)-s);
}

struct Table {
  size_t offset;   // bytes into the table region
  int bits, lo_n, hi_n;
};

bool add_table(long long X, size_t* used, Table* t) {
  t->bits = (log2i(X) + 1) / 2;
  t->lo_n = 1 << t->bits;
  t->hi_n = (int)((X + t->lo_n - 1) >> t->bits);
  t->offset = *used;
  const size_t bytes = ((size_t)(t->lo_n + t->hi_n) * sizeof(float2) + 255) & ~size_t(255);
  if (*used + bytes > kNoAllocTableBytes) return false;
  *used += bytes;
  return true;
}

cudaError_t launch_table(unsigned char* base, const Table& t, long long X, cudaStream_t s) {
  const int total = t.lo_n + t.hi_n;
  noalloc_table_kernel<<<(total + 255) / 256, 256, 0, s>>>(reinterpret_cast<float2*>(base + t.offset), X,
                                                            t.bits, t.lo_n, total);
  return cudaGetLastError();
}

// One-time set-up for the current device: device address of the static array.
int device_setup(void** addr, int* dev_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return ADFFT_ERR_CUDA;
  }
  *dev_out = dev;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_mem);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return ADFFT_ERR_CUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *addr = g_noalloc_addr[dev];
  return ADFFT_OK;
}

}  // namespace
}  // namespace adfft

extern "C" int adfft_execute_noalloc(int64_t N, int64_t M, int64_t batch, int dtype, const void* d_in,
                                     void* d_out, void* stream) {
  using namespace adfft;
  if (N < 1 || M < 1 || batch < 0 || !d_in || !d_out) return ADFFT_ERR_INVALID_ARG;
  if (dtype != ADFFT_R32 && dtype != ADFFT_C64) return ADFFT_ERR_NOT_SUPPORTED;
  if ((((uintptr_t)d_in) & 15u) || (((uintptr_t)d_out) & 15u)) return ADFFT_ERR_MISALIGNED;
  const bool real = (dtype == ADFFT_R32);
  // core shape: packed real input needs even N and M; sizes are checked before pointers
  int64_t Nc = N, Mc = M;
  if (real) {
    if ((N % 2) || (M % 2)) return ADFFT_ERR_UNSUPPORTED_SIZE;
    Nc = N / 2;
    Mc = M / 2;
  }
  if (!pow2(Nc) || Nc < 4 || M >= (int64_t(1) << 30)) return ADFFT_ERR_UNSUPPORTED_SIZE;
  if ((size_t)batch * (size_t)Mc * sizeof(float2) > kNoAllocScratchBytes) return ADFFT_ERR_UNSUPPORTED_SIZE;
  const size_t in_bytes = (size_t)batch * (size_t)N * (real ? 4 : 8);
  const size_t out_bytes = (size_t)batch * (size_t)M * 8;
  {
    const uintptr_t a = (uintptr_t)d_in, b = (uintptr_t)d_out;
    if (in_bytes && out_bytes && a < b + out_bytes && b < a + in_bytes) return ADFFT_ERR_OVERLAP;
  }
  if (batch == 0) return ADFFT_OK;

  // Geometry of the two passes (same rules as the two-pass plan form):
  // pass 1 = alpha-DFT of B strided columns of A samples (R1 bins each) in one
  // cluster of C <= 8 CTAs; pass 2 = B-point FFTs over W column pairs per CTA.
  constexpr size_t kSmem = 227 * 1024;
  constexpr int kVpt = 32, kThreads = 512;
  FusedLaunch L1{};
  TwoPassLaunch L2{};
  int64_t A = 0, B = 0, R1 = 0;
  int W = 0, ncol = 0;
  bool found = false;
  for (int max_c : {4, 8}) {
    for (A = Nc / 2; A >= 2; A >>= 1) {
      B = Nc / A;
      if (B > 2048) break;
      if ((Mc * A) % Nc) continue;
      R1 = Mc * A / Nc;
      if (real && (R1 % 2)) continue;
      W = (B <= 512) ? 16 : (B <= 1024) ? 8 : 4;
      ncol = real ? 2 * W : W;
      const int64_t region2 = B + B / 16 + 2;
      const int bits2 = (log2i(B) + 1) / 2;
      const int tw2_n = (1 << bits2) + (int)((B + (1 << bits2) - 1) >> bits2);
      if ((size_t)fused_smem_layout(tw2_n, 0, ncol, (int)region2, 8).total > kSmem) continue;
      if ((int64_t)ncol * B > (int64_t)kVpt * kThreads) continue;
      // pass 1
      const int64_t Np = gcd_i64(R1, A), P = R1 / Np, q = A / Np;
      if (!pow2(Np) || q > 64) continue;
      const int bits1 = (log2i(R1) + 1) / 2;
      const int tw1_n = (1 << bits1) + (int)((R1 + (1 << bits1) - 1) >> bits1);
      const int64_t region1 = Np + Np / 16 + 2;
      int C = -1;
      for (int c = 1; c <= std::min<int64_t>(P, max_c); ++c) {
        if (P % c) continue;
        if ((P / c) * Np > (int64_t)kVpt * kThreads) continue;
        if ((size_t)fused_smem_layout(tw1_n, 0, (int)(P / c), (int)region1, 8).total > kSmem) continue;
        C = c;
        break;
      }
      if (C < 0) continue;
      FusedArgs& a = L1.args;
      memset(&a, 0, sizeof(a));
      a.batch = batch * B;
      a.in_stride = Nc;
      a.M = R1;
      a.Np = (int)Np;
      a.logNp = log2i(Np);
      a.P = (int)P;
      a.q = (int)q;
      a.RPC = (int)(P / C);
      a.C = C;
      a.Nc = (int)A;
      a.Mc = (int)R1;
      a.Mt = (int)R1;
      a.tw_bits = bits1;
      a.scale = 1.0;
      a.region = (int)region1;
      a.stage_bytes = 0;
      a.status = nullptr;
      a.cols = B;
      a.in_unit = 8;
      a.Mpost = Mc;
      const int lr0 = (a.logNp == 0) ? 0 : (a.logNp % 4 ? a.logNp % 4 : 4);
      a.nrad = 1 + (a.logNp - lr0) / 4;
      a.divP = make_fastdiv((uint32_t)P);
      a.divRPC = make_fastdiv((uint32_t)(P / C));
      L1.mode = kColumns;
      L1.r0 = 1 << lr0;
      L1.dbl = false;
      // the epilogue gives every residue at least one thread of each CTA (threads >= P),
      // as the plan path does; a shape that would need more than kThreads is skipped
      {
        const int64_t t1 = std::max<int64_t>(((P / C) * Np + kVpt - 1) / kVpt, P);
        const int64_t t1r = std::max<int64_t>(32, (t1 + 31) / 32 * 32);
        if (t1r > kThreads) continue;
        L1.threads = (int)t1r;
      }
      L1.grid_y = (int)std::min<int64_t>(batch * B, 65535);
      L1.smem = (size_t)fused_smem_layout(tw1_n, 0, a.RPC, a.region, 8).total;
      if (C > 1 && fused_max_active_clusters(L1) < 1) continue;
      // pass 2
      TwoPassArgs& t = L2.args;
      memset(&t, 0, sizeof(t));
      FusedArgs& f = t.f;
      f.Np = (int)B;
      f.logNp = log2i(B);
      f.P = 1;
      f.q = 1;
      f.RPC = ncol;
      f.C = 1;
      f.Nc = (int)B;
      f.Mc = (int)B;
      f.Mt = (int)B;
      f.tw_bits = bits2;
      f.region = (int)region2;
      f.scale = 1.0;
      const int lr2 = (f.logNp == 0) ? 0 : (f.logNp % 4 ? f.logNp % 4 : 4);
      f.nrad = 1 + (f.logNp - lr2) / 4;
      t.batch = batch;
      t.B = (int)B;
      t.logB = f.logNp;
      t.R1 = R1;
      t.Mc = Mc;
      t.M = M;
      t.W = W;
      t.real_packed = real ? 1 : 0;
      t.scale = 1.0 / (double)N;
      L2.r0 = 1 << lr2;
      L2.dbl = false;
      L2.threads = std::max(32, (int)(((int64_t)ncol * B / kVpt + 31) / 32 * 32));
      L2.grid_x = (int)(((real ? R1 / 2 + 1 : R1) + W - 1) / W);
      L2.grid_y = (int)std::min<int64_t>(batch, 65535);
      L2.smem = (size_t)fused_smem_layout(tw2_n, 0, ncol, (int)region2, 8).total;
      found = true;
      break;
    }
    if (found) break;
  }
  if (!found) return ADFFT_ERR_UNSUPPORTED_SIZE;

  // tables inside the static array
  size_t used = 0;
  Table t1, tp, t2, tm;
  if (!add_table(R1, &used, &t1) || !add_table(Mc, &used, &tp) || !add_table(B, &used, &t2) ||
      !add_table(M, &used, &tm))
    return ADFFT_ERR_UNSUPPORTED_SIZE;

  void* base_v = nullptr;
  int dev = 0;
  int rc = device_setup(&base_v, &dev);
  if (rc != ADFFT_OK) return rc;
  unsigned char* base = static_cast<unsigned char*>(base_v);
  unsigned char* scratch = base + kNoAllocTableBytes;
  L1.args.tw = base + t1.offset;
  L1.args.tw_lo_n = t1.lo_n;
  L1.args.tw_hi_n = t1.hi_n;
  L1.args.post_tw = base + tp.offset;
  L1.args.post_bits = tp.bits;
  L1.args.post_lo_n = tp.lo_n;
  L2.args.f.tw = base + t2.offset;
  L2.args.f.tw_lo_n = t2.lo_n;
  L2.args.f.tw_hi_n = t2.hi_n;
  L2.args.wM = base + tm.offset;
  L2.args.wM_bits = tm.bits;
  L2.args.wM_lo_n = tm.lo_n;

  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = fused_prepare(L1);
  if (e == cudaSuccess) e = twopass_prepare(L2);
  {
    // the tables depend on (R1, Mc, B, M) only: rewrite them when the previous call on
    // this device used other sizes (calls are serialised on the GPU by contract)
    const long long key[4] = {(long long)R1, (long long)Mc, (long long)B, (long long)M};
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    const bool same = memcmp(g_table_key[dev], key, sizeof(key)) == 0;
    if (e == cudaSuccess && !same) {
      memset(g_table_key[dev], 0, sizeof(key));
      e = launch_table(base, t1, R1, s);
      if (e == cudaSuccess) e = launch_table(base, tp, Mc, s);
      if (e == cudaSuccess) e = launch_table(base, t2, B, s);
      if (e == cudaSuccess) e = launch_table(base, tm, M, s);
      if (e == cudaSuccess) memcpy(g_table_key[dev], key, sizeof(key));
    }
  }
  if (e == cudaSuccess) e = fused_launch(L1, d_in, scratch, s);
  if (e == cudaSuccess) e = twopass_launch(L2, scratch, d_out, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    memset(g_table_key[dev], 0, sizeof(g_table_key[dev]));
    return ADFFT_ERR_CUDA;
  }
  return ADFFT_OK;
}
