// Host side of the adfft C ABI: plan validation, algorithm and launch-shape
// selection, FP64-derived tables, and the extern "C" entry points.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <new>
#include <vector>

#include "adfft_internal.h"

namespace adfft {

// ---- fault injection for tests (environment variable ADFFT_FAULT, read at plan creation) ----
//   alloc:<k>      the k-th device allocation of the plan creation (k >= 1) fails as out of memory
//   launch         every launch of the plan's kernels fails (ADFFT_ERR_CUDA, nothing launched)
//   copy_skip:<s>  the fused kernel does not issue the input copy of signal s and gives up
//                  waiting for it after ~10 ms: the plan then reports ADFFT_ERR_TIMEOUT
// Unset (the normal case): no effect.
namespace {
thread_local int g_alloc_count = 0;     // device allocations of the plan creation under way
thread_local int g_alloc_fail_at = 0;   // the one that fails (0: none)
}  // namespace

FaultSpec read_fault_spec() {
  FaultSpec f;
  const char* v = getenv("ADFFT_FAULT");
  if (!v || !*v) return f;
  if (strncmp(v, "alloc:", 6) == 0) f.alloc_at = atoi(v + 6);
  else if (strcmp(v, "launch") == 0) f.launch = true;
  else if (strncmp(v, "copy_skip:", 10) == 0) f.copy_skip = atoll(v + 10);
  return f;
}

// cudaMalloc through the allocation fault hook.
cudaError_t dev_malloc(void** p, size_t bytes) {
  if (g_alloc_fail_at > 0 && ++g_alloc_count == g_alloc_fail_at) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

namespace {

thread_local int g_last_error = ADFFT_OK;

constexpr size_t kSmemLimit = 227 * 1024;   // dynamic shared memory per CTA on sm_103a
constexpr int kMaxCluster = kFoldMaxCluster;   // non-portable cluster size limit
constexpr int kMaxFold = 64;                // largest fold factor q the fused kernel takes
constexpr int kMaxThreads = 512;

int64_t gcd64(int64_t a, int64_t b) {
  while (b) {
    int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

int ilog2(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l;
}

// exp(-2 pi i e / Mt) in double precision, e reduced to the symmetric range first.
void root_of_unity(int64_t e, int64_t Mt, double* c, double* s) {
  e %= Mt;
  if (e < 0) e += Mt;
  int64_t k = (2 * e > Mt) ? e - Mt : e;
  double ang = (2.0 * M_PI * (double)k) / (double)Mt;
  *c = cos(ang);
  *s = -sin(ang);
}

// Two-level table of W_Mt: lo[l] = W^l (l < 2^bits), hi[h] = W^(h 2^bits).
template <typename T>
std::vector<T> build_two_level(int64_t Mt, int bits, int* lo_n, int* hi_n) {
  *lo_n = 1 << bits;
  *hi_n = (int)((Mt + *lo_n - 1) >> bits);
  std::vector<T> t((size_t)2 * (*lo_n + *hi_n));
  for (int l = 0; l < *lo_n; ++l) {
    double c, s;
    root_of_unity(l, Mt, &c, &s);
    t[2 * l] = (T)c;
    t[2 * l + 1] = (T)s;
  }
  for (int h = 0; h < *hi_n; ++h) {
    double c, s;
    root_of_unity((int64_t)h << bits, Mt, &c, &s);
    t[2 * (*lo_n + h)] = (T)c;
    t[2 * (*lo_n + h) + 1] = (T)s;
  }
  return t;
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return ADFFT_OK;
  if (e == cudaErrorMemoryAllocation) return ADFFT_ERR_OOM;
  return ADFFT_ERR_CUDA;
}

template <typename T>
int upload(void** dst, const std::vector<T>& v);

// Configure a fused fold+FFT launch for the complex core of Nc input elements
// and Mc bins (twiddle modulus Mt); stage_bytes > 0 asks for bulk-copy input
// staging of that many bytes per signal, used if it fits.  The choice fixes the
// sub-FFT length Np, a power of two dividing both Mc and Nc (P = Mc/Np residues
// and a fold of q = Nc/Np blocks: the identity holds for any common divisor),
// the cluster size (0: the smallest that fits) and whether staging may be
// used.  Allocates the twiddle table in *d_tw unless one is passed in.
// Returns ADFFT_OK or why the shape does not fit.
// Two-pass forward, FP32: pass 1 with each column's residues over independent CTAs of this
// many residues (runs of that many bins, 32 bytes at 4), instead of one CTA or cluster per column.
constexpr bool kTwoPassSplitForward = true;
constexpr int kTwoPassSplitResidues = 4;

int configure_fused(bool dbl, int mode, int64_t Nc, int64_t Mc, int64_t Mt, int64_t batch,
                    int64_t stage_bytes, int max_cluster, double scale, int* status,
                    FusedLaunch& L, void** d_tw, const FoldChoice& choice = FoldChoice{}) {
  const int64_t g = gcd64(Mc, Nc);
  const int64_t Np = choice.np > 0 ? choice.np : (g & -g);
  if (!is_pow2(Np) || g % Np) return ADFFT_ERR_UNSUPPORTED_SIZE;
  const int64_t P = Mc / Np, q = Nc / Np;
  if (q > kMaxFold || P > (int64_t(1) << 30)) return ADFFT_ERR_UNSUPPORTED_SIZE;
  if (Mt >= (int64_t(1) << 31)) return ADFFT_ERR_UNSUPPORTED_SIZE;
  const size_t esz = dbl ? 16 : 8;
  const int vpt = fused_values_per_thread(dbl);
  const int max_vals = vpt * kMaxThreads;

  const int bits = (ilog2(Mt) + 1) / 2;
  int lo_n, hi_n;
  const int tw_n = (1 << bits) + (int)((Mt + (1 << bits) - 1) >> bits);
  const int64_t region = Np + Np / 16 + 2;
  const bool push = choice.stage == 2;   // bulk push exchange: one residue per CTA, no staging
  const bool can_stage = choice.stage != 0 && !push && stage_bytes > 0 && (stage_bytes % 16) == 0 &&
                         stage_bytes <= (int64_t)kSmemLimit;
  const int vs = choice.vsplit > 1 ? choice.vsplit : 0;   // independent CTAs per column
  if (vs && (mode != kColumns || push || P % vs)) return ADFFT_ERR_UNSUPPORTED_SIZE;
  int C = -1, stage = 0;
  size_t smem = 0;
  for (int pass = 0; pass < 2 && C < 0; ++pass) {
    if (pass == 0 && !can_stage) continue;
    if (pass == 1 && choice.stage == 1) continue;
    const int st = (pass == 0) ? (int)stage_bytes : 0;
    for (int c = 1; c <= std::min<int64_t>(P, max_cluster); ++c) {
      if (P % c) continue;
      if (choice.cluster > 0 && c != choice.cluster) continue;
      if (push && c != P) continue;
      if (vs && c != 1) continue;
      const int64_t rpc = vs ? P / vs : P / c;
      if (rpc * Np > max_vals) continue;
      const FusedSmem lay = fused_smem_layout(tw_n, st, (int)rpc, (int)region, (int)esz);
      if ((size_t)lay.total > kSmemLimit) continue;
      C = c;
      stage = st;
      smem = (size_t)lay.total;
      break;
    }
  }
  if (C < 0) return ADFFT_ERR_UNSUPPORTED_SIZE;
  const int64_t RPC = vs ? P / vs : P / C;

  FusedArgs& a = L.args;
  memset(&a, 0, sizeof(a));
  a.batch = batch;
  a.M = (mode == kLoadRealPacked) ? 2 * Mc : Mc;
  a.in_stride = (mode == kLoadComplex || mode == kColumns) ? Nc : (mode == kLoadRealPacked ? 2 * Nc : Nc);
  a.Np = (int)Np;
  a.logNp = ilog2(Np);
  a.P = (int)P;
  a.q = (int)q;
  a.RPC = (int)RPC;
  a.C = C;
  a.Nc = (int)Nc;
  a.Mc = (int)Mc;
  a.Mt = (int)Mt;
  a.tw_bits = bits;
  a.scale = scale;
  a.region = (int)region;
  a.stage_bytes = stage;
  a.status = status;
  a.cols = 1;
  a.vsplit = vs;
  a.in_unit = (mode == kLoadComplex || mode == kColumns) ? (int)esz : (int)(esz / 2);
  // passes: a first pass of radix R0 = 2^(log2 Np mod 4) (16 if that is 0), then radix 16;
  // for complex64 data a remainder of 2 is merged with one radix-16 pass into radix 32
  const int L2 = a.logNp;
  int lr0 = (L2 == 0) ? 0 : (L2 % 4 ? L2 % 4 : 4);
  if (!dbl && lr0 == 1 && L2 >= 5) lr0 = 5;
  a.nrad = 1 + (L2 - lr0) / 4;
  L.r0 = 1 << lr0;
  a.divP = make_fastdiv((uint32_t)P);
  a.divRPC = make_fastdiv((uint32_t)RPC);

  // table W_Mt (depends on Mt and the precision only: a table passed in is reused)
  lo_n = 1 << bits;
  hi_n = (int)((Mt + lo_n - 1) >> bits);
  a.tw_lo_n = lo_n;
  a.tw_hi_n = hi_n;
  if (!*d_tw) {
    size_t tw_bytes;
    std::vector<unsigned char> host;
    if (dbl) {
      auto t = build_two_level<double>(Mt, bits, &lo_n, &hi_n);
      tw_bytes = t.size() * sizeof(double);
      host.assign((unsigned char*)t.data(), (unsigned char*)t.data() + tw_bytes);
    } else {
      auto t = build_two_level<float>(Mt, bits, &lo_n, &hi_n);
      tw_bytes = t.size() * sizeof(float);
      host.assign((unsigned char*)t.data(), (unsigned char*)t.data() + tw_bytes);
    }
    cudaError_t e = dev_malloc(d_tw, tw_bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      *d_tw = nullptr;
      return cuda_status(e);
    }
    e = cudaMemcpy(*d_tw, host.data(), tw_bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_status(e);
  }
  a.tw = *d_tw;

  int threads = (int)((RPC * Np + vpt - 1) / vpt);
  // the epilogue gives every residue it covers at least one thread of each CTA
  threads = (int)std::max<int64_t>(threads, vs ? RPC : P);
  threads = std::max(32, (threads + 31) / 32 * 32);
  if (threads > kMaxThreads) return ADFFT_ERR_UNSUPPORTED_SIZE;
  L.mode = mode;
  L.dbl = dbl;
  L.threads = threads;
  L.grid_y = (int)std::max<int64_t>(1, std::min<int64_t>(batch, 65535));
  L.smem = smem;
  L.push = false;
  if (push) {
    // only the compile-time shapes of fused_push.cu serve this form
    int pt = 0;
    size_t ps = 0;
    L.push = true;
    if (!push_geometry(L, &pt, &ps) || ps > kSmemLimit) {
      L.push = false;
      return ADFFT_ERR_UNSUPPORTED_SIZE;
    }
    L.threads = pt;
    L.smem = ps;
  }
  cudaError_t e = fused_prepare(L);
  if (e == cudaSuccess) e = adjoint_prepare(L);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(e);
  }
  int resident = fused_max_active_clusters(L);
  if (vs && resident > 0) resident = std::max(1, resident / vs);   // columns in flight
  if (C > 1 && resident < 1) return ADFFT_ERR_UNSUPPORTED_SIZE;
  // persistent grid: clusters loop over signals, so the table load and launch are paid once
  // per cluster and the next signal's input is fetched while the current one is transformed
  if (choice.grid > 0) L.grid_y = (int)std::min<int64_t>(L.grid_y, choice.grid);
  else if (choice.grid == 0 && resident > 0) L.grid_y = std::min(L.grid_y, resident);
  return ADFFT_OK;
}

}  // namespace

// How the plan's input maps onto the complex core: mode, Nc, Mc.
void core_shape(const Plan& p, int* mode, int64_t* Nc, int64_t* Mc) {
  if (!p.real) {
    *mode = kLoadComplex;
    *Nc = p.N;
    *Mc = p.M;
  } else if (p.N % 2 == 0 && p.M % 2 == 0) {
    *mode = kLoadRealPacked;
    *Nc = p.N / 2;
    *Mc = p.M / 2;
  } else {
    *mode = kLoadRealPlain;
    *Nc = p.N;
    *Mc = p.M;
  }
}

// Configure the fused single-pass fold+FFT path.  Without a forced choice the
// sub-FFT length is the largest power of two dividing gcd(Mc, Nc), halved
// while no cluster fits (and the fold factor stays within kTuneMaxFold), the
// cluster the smallest that fits, with input staging where it fits.
int setup_fold(Plan& p, const FoldChoice* forced) {
  int mode;
  int64_t Nc, Mc;
  core_shape(p, &mode, &Nc, &Mc);
  const int64_t Mt = (mode == kLoadRealPacked) ? p.M : Mc;
  const int64_t sig_bytes = p.stage_ok ? (int64_t)p.N * (int64_t)p.in_elem : 0;
  if (p.half && (mode != kLoadRealPacked || (forced && forced->stage == 2))) return ADFFT_ERR_UNSUPPORTED_SIZE;
  const int64_t g = gcd64(Mc, Nc);
  int rc = ADFFT_ERR_UNSUPPORTED_SIZE;
  FoldChoice ch{};
  FusedLaunch L{};   // configured here, taken only on success (the plan keeps its shape otherwise)
  if (forced) {
    ch = *forced;
    rc = configure_fused(p.dbl, mode, Nc, Mc, Mt, p.batch, sig_bytes, kMaxCluster, p.scale, p.d_status,
                         L, &p.d_tw, ch);
  } else {
    const int64_t np0 = g & -g;
    for (int64_t np = np0; np >= 1; np /= 2) {
      if (np != np0 && Nc / np > kTuneMaxFold) break;
      ch = FoldChoice{np, 0, -1};
      rc = configure_fused(p.dbl, mode, Nc, Mc, Mt, p.batch, sig_bytes, kMaxCluster, p.scale, p.d_status,
                           L, &p.d_tw, ch);
      if (rc != ADFFT_ERR_UNSUPPORTED_SIZE) break;
    }
  }
  if (rc != ADFFT_OK) return rc;
  p.fused = L;
  p.fused.args.in_stride = p.N;   // complex elements or real scalars per signal
  p.fused.args.in_unit = (int)p.in_elem;
  p.fused.args.M = p.M;
  p.fused.args.offs = p.d_offs;
  p.fused.args.half = p.half ? 1 : 0;
  if (p.half) {
    // half-spectrum output has kernels of its own: set their launch attributes too
    cudaError_t e = fused_prepare(p.fused);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p.fold_ok = false;
      return cuda_status(e);
    }
  }
  if (p.fault.copy_skip >= 0) {
    p.fused.args.fault_sig1 = p.fault.copy_skip + 1;
    p.fused.args.wait_limit = 20000000;   // ~10 ms of SM clock
  }
  p.fold_choice = FoldChoice{p.fused.args.Np, p.fused.args.C,
                             p.fused.push ? 2 : (p.fused.args.stage_bytes > 0 ? 1 : 0), ch.grid};
  p.fold_ok = true;
  return ADFFT_OK;
}

bool split_forward_ok(const Plan& p, int64_t P1) {
  return kTwoPassSplitForward && !p.dbl && P1 > kTwoPassSplitResidues && P1 % kTwoPassSplitResidues == 0;
}

// Configure the two-pass (four-step) path for power-of-two Nc: Nc = A B, pass 1 the
// alpha-DFTs of the B columns of length A, pass 2 the B-point FFTs.  Without a forced A
// (p.tp_force_A == 0): where the FP32 forward can split pass 1 over independent CTAs, the
// longest A with B >= 512 whose pass 1 fits a cluster of at most 4 CTAs (for the adjoint);
// else the longest A whose pass-1 transform fits one CTA (each CTA then reads its strided
// column once), else clusters of at most 4, then 8 CTAs.  (8 x 2^22, alpha 16: A = 4096,
// forward 3.93 ms, against 4.60 ms at A = 1024.)
int setup_twopass(Plan& p) {
  int mode;
  int64_t Nc, Mc;
  if (p.tp_ok) return ADFFT_OK;
  core_shape(p, &mode, &Nc, &Mc);
  if (mode == kLoadRealPlain || !is_pow2(Nc) || Nc < 4) return ADFFT_ERR_UNSUPPORTED_SIZE;
  const size_t esz = p.dbl ? 16 : 8;
  const int vpt = fused_values_per_thread(p.dbl);
  const bool forced = p.tp_force_A > 0;
  // rounds of (largest cluster for pass 1, smallest B, pass 1 must split for the forward)
  struct Round {
    int max_c;
    int64_t min_B;
    bool split;
  };
  static const Round kDefault[] = {{4, 512, true}, {1, 0, false}, {4, 0, false}, {8, 0, false}};
  static const Round kForced[] = {{4, 0, false}, {8, 0, false}, {16, 0, false}};
  const Round* rounds = forced ? kForced : kDefault;
  const int nrounds = forced ? 3 : 4;
  for (int ri = 0; ri < nrounds; ++ri) {
    const int max_c = rounds[ri].max_c;
    for (int64_t A = Nc / 2; A >= 16; A >>= 1) {
      const int64_t B = Nc / A;
      if (B > 2048) break;
      if (B < rounds[ri].min_B) continue;
      if (forced && A != p.tp_force_A) continue;
      if ((Mc * A) % Nc != 0) continue;
      const int64_t R1 = Mc * A / Nc;
      if (mode == kLoadRealPacked && (R1 % 2) != 0) continue;
      if (rounds[ri].split) {
        const int64_t g1 = gcd64(R1, A);
        if (!split_forward_ok(p, R1 / (g1 & -g1))) continue;
      }
      // pass 2 geometry: W column pairs per CTA.  Output rows are written in runs of W bins
      // (32 bytes at W = 4); more columns per CTA (longer runs) cost shared memory and so
      // concurrency: measured on 8 x 2^22, alpha 16, W = 4 is best for the forward from B = 1024
      // to 2048 (B = 1024: 4.40 ms against 4.53 ms at W = 8), W = 2 and 1 lose (6.1, 7.8 ms at
      // B = 2048); at B = 512 W = 4 and 8 tie for the forward and W = 8 is 0.3 ms faster for
      // the adjoint (7.09 against 7.41 ms), W = 16 slower for both
      const int W = (B <= 256) ? 16 : (B <= 512) ? 8 : 4;
      const int ncol = (mode == kLoadRealPacked) ? 2 * W : W;
      const int64_t region = B + B / 16 + 2;
      const int bits2 = (ilog2(B) + 1) / 2;
      const int tw_n2 = (1 << bits2) + (int)((B + (1 << bits2) - 1) >> bits2);
      const FusedSmem lay2 = fused_smem_layout(tw_n2, 0, ncol, (int)region, (int)esz);
      if ((size_t)lay2.total > kSmemLimit) continue;
      if ((int64_t)ncol * B > (int64_t)vpt * kMaxThreads) continue;
      // pass 1: alpha-DFT of the B columns (A samples -> R1 bins each)
      FusedLaunch L1{};
      void* tw1 = nullptr;
      // the column (A complex elements) is gathered into shared memory once per CTA where it fits
      int rc = configure_fused(p.dbl, kColumns, A, R1, R1, p.batch * B, A * (int64_t)esz, max_c, 1.0, p.d_status,
                               L1, &tw1);
      if (rc != ADFFT_OK) {
        if (tw1) cudaFree(tw1);
        if (rc == ADFFT_ERR_UNSUPPORTED_SIZE) continue;
        return rc;
      }
      p.d_tp_tw1 = tw1;
      L1.args.cols = B;
      L1.args.in_stride = Nc;
      L1.args.M = R1;
      L1.args.Mpost = Mc;
      int lo_n, hi_n;
      const int pbits = (ilog2(Mc) + 1) / 2;
      if (p.dbl) {
        if ((rc = upload(&p.d_tp_post, build_two_level<double>(Mc, pbits, &lo_n, &hi_n))) != ADFFT_OK) return rc;
      } else {
        if ((rc = upload(&p.d_tp_post, build_two_level<float>(Mc, pbits, &lo_n, &hi_n))) != ADFFT_OK) return rc;
      }
      L1.args.post_tw = p.d_tp_post;
      L1.args.post_bits = pbits;
      L1.args.post_lo_n = lo_n;
      p.tp1 = L1;
      // FP32 forward: the column's residues over independent CTAs of kTwoPassSplitResidues
      // residues each (no cluster exchange; every CTA writes runs of that many bins)
      p.tp1f_ok = false;
      const int64_t P1 = L1.args.P;
      if (split_forward_ok(p, L1.args.P)) {
        FusedLaunch F{};
        FoldChoice fc{};
        fc.np = L1.args.Np;
        fc.vsplit = (int)(P1 / kTwoPassSplitResidues);
        const int rcf = configure_fused(p.dbl, kColumns, A, R1, R1, p.batch * B, A * (int64_t)esz, 1, 1.0,
                                        p.d_status, F, &tw1, fc);
        if (rcf == ADFFT_OK) {
          const FusedArgs& s1 = L1.args;
          F.args.cols = s1.cols;
          F.args.in_stride = s1.in_stride;
          F.args.M = s1.M;
          F.args.Mpost = s1.Mpost;
          F.args.post_tw = s1.post_tw;
          F.args.post_bits = s1.post_bits;
          F.args.post_lo_n = s1.post_lo_n;
          p.tp1f = F;
          p.tp1f_ok = true;
        } else if (rcf != ADFFT_ERR_UNSUPPORTED_SIZE) {
          return rcf;
        }
      }
      // pass 2 tables: W_B (shared memory), W_M (global, real unpacking)
      TwoPassLaunch& L2 = p.tp2;
      TwoPassArgs& t = L2.args;
      memset(&t, 0, sizeof(t));
      FusedArgs& f = t.f;
      f.Np = (int)B;
      f.logNp = ilog2(B);
      f.P = 1;
      f.q = 1;
      f.RPC = ncol;
      f.C = 1;
      f.Nc = (int)B;
      f.Mc = (int)B;
      f.Mt = (int)B;
      f.tw_bits = bits2;
      f.region = (int)region;
      f.scale = 1.0;
      f.status = p.d_status;
      const int lb = f.logNp;
      const int lr0 = (lb == 0) ? 0 : (lb % 4 ? lb % 4 : 4);
      f.nrad = 1 + (lb - lr0) / 4;
      L2.r0 = 1 << lr0;
      const int mbits = (ilog2(p.M) + 1) / 2;
      if (p.dbl) {
        if ((rc = upload(&p.d_tp_tw2, build_two_level<double>(B, bits2, &lo_n, &hi_n))) != ADFFT_OK) return rc;
        f.tw_lo_n = lo_n;
        f.tw_hi_n = hi_n;
        if ((rc = upload(&p.d_tp_wM, build_two_level<double>(p.M, mbits, &lo_n, &hi_n))) != ADFFT_OK) return rc;
      } else {
        if ((rc = upload(&p.d_tp_tw2, build_two_level<float>(B, bits2, &lo_n, &hi_n))) != ADFFT_OK) return rc;
        f.tw_lo_n = lo_n;
        f.tw_hi_n = hi_n;
        if ((rc = upload(&p.d_tp_wM, build_two_level<float>(p.M, mbits, &lo_n, &hi_n))) != ADFFT_OK) return rc;
      }
      f.tw = p.d_tp_tw2;
      t.wM = p.d_tp_wM;
      t.wM_bits = mbits;
      t.wM_lo_n = lo_n;
      t.batch = p.batch;
      t.B = (int)B;
      t.logB = ilog2(B);
      t.R1 = R1;
      t.Mc = Mc;
      t.M = p.M;
      t.W = W;
      t.real_packed = (mode == kLoadRealPacked) ? 1 : 0;
      t.scale = p.scale;
      L2.dbl = p.dbl;
      L2.threads = std::max(32, (int)(((int64_t)ncol * B / vpt + 31) / 32 * 32));
      const int64_t npairs = (mode == kLoadRealPacked) ? R1 / 2 + 1 : R1;
      L2.grid_x = (int)((npairs + W - 1) / W);
      L2.grid_y = (int)std::max<int64_t>(1, std::min<int64_t>(p.batch, 65535));
      L2.smem = (size_t)lay2.total;
      if (L2.grid_x > 0x7fffffff) return ADFFT_ERR_UNSUPPORTED_SIZE;
      cudaError_t e = twopass_prepare(L2);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_status(e);
      }
      // scratch [batch][B][R1]
      p.ws_bytes = (size_t)p.batch * (size_t)Mc * esz;
      if (p.ws_bytes) {
        e = dev_malloc(&p.d_ws, p.ws_bytes);
        if (e != cudaSuccess) {
          cudaGetLastError();
          p.d_ws = nullptr;
          return cuda_status(e);
        }
      }
      p.tp1.args.offs = p.d_offs;
      p.tp1f.args.offs = p.d_offs;
      t.f.offs = p.d_offs;
      p.tp_A = A;
      p.tp_B = B;
      p.tp_ok = true;
      return ADFFT_OK;
    }
  }
  return ADFFT_ERR_UNSUPPORTED_SIZE;
}

// Free the two-pass form's tables and workspace (the plan keeps its other forms).
void release_twopass(Plan& p) {
  for (void** q : {&p.d_tp_tw1, &p.d_tp_post, &p.d_tp_tw2, &p.d_tp_wM, &p.d_ws}) {
    if (*q) cudaFree(*q);
    *q = nullptr;
  }
  p.ws_bytes = 0;
  p.tp_ok = false;
  p.tp1f_ok = false;
  p.tp_A = p.tp_B = 0;
}

int64_t plan_gcd(int64_t a, int64_t b) { return gcd64(a, b); }

std::vector<float> twiddle_table_f32(int64_t Mt, int* bits, int* lo_n, int* hi_n) {
  *bits = (ilog2(Mt) + 1) / 2;
  return build_two_level<float>(Mt, *bits, lo_n, hi_n);
}

namespace {

// In-place iterative radix-2 FFT in double precision (host), forward sign.
void host_fft(std::vector<std::complex<double>>& a) {
  const size_t n = a.size();
  for (size_t i = 1, j = 0; i < n; ++i) {
    size_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (size_t len = 2; len <= n; len <<= 1) {
    for (size_t i = 0; i < n; i += len) {
      for (size_t k = 0; k < len / 2; ++k) {
        double c, s;
        root_of_unity((int64_t)k, (int64_t)len, &c, &s);
        const std::complex<double> w(c, s);
        const std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w;
        a[i + k] = u + v;
        a[i + k + len / 2] = u - v;
      }
    }
  }
}

// chirp c_j = exp(-pi i (j^2 mod 2M) / M), exact integer reduction of j^2
std::complex<double> chirp(int64_t j, int64_t M) {
  if (j < 0) j = -j;
  const int64_t twoM = 2 * M;
  const int64_t jj = (int64_t)(((__int128)j * j) % twoM);
  double c, s;
  root_of_unity(jj, twoM, &c, &s);
  return {c, s};
}

template <typename T>
int upload(void** dst, const std::vector<T>& v) {
  const size_t bytes = v.size() * sizeof(T);
  cudaError_t e = dev_malloc(dst, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *dst = nullptr;
    return cuda_status(e);
  }
  e = cudaMemcpy(*dst, v.data(), bytes, cudaMemcpyHostToDevice);
  return cuda_status(e);
}

template <typename T>
std::vector<T> flatten(const std::vector<std::complex<double>>& v) {
  std::vector<T> o(2 * v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    o[2 * i] = (T)v[i].real();
    o[2 * i + 1] = (T)v[i].imag();
  }
  return o;
}

}  // namespace

// Configure the chirp-z adjoint (any N, M): input blocks and output chunks of one transform
// length L (a single tile where N + M - 1 fits), FP64-derived chirp and kernel spectra.
int setup_bluestein_adjoint(Plan& p) {
  if (p.bla_ok) return ADFFT_OK;
  const int64_t Lmax = p.dbl ? 8192 : 16384;
  const int acc = p.dbl ? kBlaAccF64 : kBlaAccF32;
  const int vpt = fused_values_per_thread(p.dbl);
  const size_t esz = p.dbl ? 16 : 8;
  int64_t L = 1, Bi, Bo;
  if (p.N + p.M - 1 <= Lmax && p.N <= (int64_t)acc * kMaxThreads) {
    while (L < p.N + p.M - 1) L <<= 1;
    Bi = p.M;
    Bo = p.N;
  } else {
    L = Lmax;
    Bi = Bo = L / 2;
  }
  const int64_t nI = (p.M + Bi - 1) / Bi, nO = (p.N + Bo - 1) / Bo;
  if (nO > 65535 || p.M >= (int64_t(1) << 31)) return ADFFT_ERR_UNSUPPORTED_SIZE;
  int threads = (int)std::max<int64_t>(L / vpt, (Bo + acc - 1) / acc);
  threads = std::max(32, (threads + 31) / 32 * 32);
  if (threads > kMaxThreads) return ADFFT_ERR_UNSUPPORTED_SIZE;
  const int bits = (ilog2(L) + 1) / 2;
  const int tw_n = (1 << bits) + (int)((L + (1 << bits) - 1) >> bits);
  const int64_t region = L + L / 16 + 2;
  const FusedSmem lay = fused_smem_layout(tw_n, 0, 1, (int)region, (int)esz);
  if ((size_t)lay.total > kSmemLimit) return ADFFT_ERR_UNSUPPORTED_SIZE;
  // host tables: chirp, kernel spectra of every block difference d = (o - i) Bo (single tile: 0)
  std::vector<std::complex<double>> ch((size_t)std::max(p.N, p.M));
  for (size_t j = 0; j < ch.size(); ++j) ch[j] = chirp((int64_t)j, p.M);
  const int64_t nd = nI + nO - 1;
  std::vector<std::complex<double>> H((size_t)(nd * L));
  std::vector<std::complex<double>> seg((size_t)L);
  for (int64_t k = 0; k < nd; ++k) {
    const int64_t d = (k - (nI - 1)) * Bo;
    std::fill(seg.begin(), seg.end(), std::complex<double>(0, 0));
    for (int64_t i = 0; i < Bi + Bo - 1 && i < L; ++i) seg[(size_t)i] = chirp(d - (Bi - 1) + i, p.M);
    host_fft(seg);
    for (int64_t t = 0; t < L; ++t) H[(size_t)(k * L + t)] = seg[(size_t)t] / (double)L;
  }
  int lo_n, hi_n, rc;
  if (p.dbl) {
    if ((rc = upload(&p.d_bla_tw, build_two_level<double>(L, bits, &lo_n, &hi_n))) != ADFFT_OK) return rc;
    if ((rc = upload(&p.d_bla_chirp, flatten<double>(ch))) != ADFFT_OK) return rc;
    if ((rc = upload(&p.d_bla_H, flatten<double>(H))) != ADFFT_OK) return rc;
  } else {
    if ((rc = upload(&p.d_bla_tw, build_two_level<float>(L, bits, &lo_n, &hi_n))) != ADFFT_OK) return rc;
    if ((rc = upload(&p.d_bla_chirp, flatten<float>(ch))) != ADFFT_OK) return rc;
    if ((rc = upload(&p.d_bla_H, flatten<float>(H))) != ADFFT_OK) return rc;
  }
  BluesteinAdjLaunch& BL = p.bla;
  BluesteinAdjArgs& b = BL.args;
  memset(&b, 0, sizeof(b));
  FusedArgs& a = b.f;
  a.batch = p.batch;
  a.M = p.M;
  a.Np = (int)L;
  a.logNp = ilog2(L);
  a.P = 1;
  a.q = 1;
  a.RPC = 1;
  a.C = 1;
  a.Nc = (int)L;
  a.Mc = (int)L;
  a.Mt = (int)L;
  a.tw_bits = bits;
  a.tw_lo_n = lo_n;
  a.tw_hi_n = hi_n;
  a.tw = p.d_bla_tw;
  a.scale = p.scale;
  a.region = (int)region;
  const int lr0 = (a.logNp == 0) ? 0 : (a.logNp % 4 ? a.logNp % 4 : 4);
  a.nrad = 1 + (a.logNp - lr0) / 4;
  a.in_unit = (int)p.in_elem;
  a.offs = p.d_offs;
  b.chirp = p.d_bla_chirp;
  b.H = p.d_bla_H;
  b.N = p.N;
  b.Bi = (int)Bi;
  b.Bo = (int)Bo;
  b.nI = (int)nI;
  b.nO = (int)nO;
  b.real_out = p.real ? 1 : 0;
  BL.r0 = 1 << lr0;
  BL.dbl = p.dbl;
  BL.threads = threads;
  BL.grid_y = (int)std::max<int64_t>(1, std::min<int64_t>(p.batch, 65535));
  BL.smem = (size_t)lay.total;
  cudaError_t e = bluestein_adjoint_prepare(BL);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(e);
  }
  p.bla_ok = true;
  return ADFFT_OK;
}

// Configure the chirp-z path (any N, M); returns ADFFT_OK or why it does not apply.
int setup_bluestein(Plan& p) {
  if (p.blu_ok) return ADFFT_OK;
  const int64_t Lmax = p.dbl ? 8192 : 16384;
  // chunks of B = L - N + 1 >= N + 1 bins: at most 2M/N + 1 kernel spectra of length L
  if (2 * p.N > Lmax) return ADFFT_ERR_UNSUPPORTED_SIZE;
  int64_t L = 1;
  while (L < p.N + p.M - 1 && L < Lmax) L <<= 1;
  while (L < 2 * p.N) L <<= 1;
  const int64_t B = L - p.N + 1;
  const int64_t chunks = (p.M + B - 1) / B;
  if (chunks > 4096 || p.M >= (int64_t(1) << 31)) return ADFFT_ERR_UNSUPPORTED_SIZE;
  const int vpt = fused_values_per_thread(p.dbl);
  const size_t esz = p.dbl ? 16 : 8;
  const int bits = (ilog2(L) + 1) / 2;
  const int tw_n = (1 << bits) + (int)((L + (1 << bits) - 1) >> bits);
  const int64_t region = L + L / 16 + 2;
  const FusedSmem lay = fused_smem_layout(tw_n, 0, 1, (int)region, (int)esz);
  if ((size_t)lay.total > kSmemLimit) return ADFFT_ERR_UNSUPPORTED_SIZE;

  // host tables: W_L, chirp, per-chunk FFT_L(hs)/L
  int lo_n, hi_n;
  std::vector<std::complex<double>> ch((size_t)std::max(p.N, p.M));
  for (size_t j = 0; j < ch.size(); ++j) ch[j] = chirp((int64_t)j, p.M);
  std::vector<std::complex<double>> H((size_t)(chunks * L));
  std::vector<std::complex<double>> seg((size_t)L);
  for (int64_t c = 0; c < chunks; ++c) {
    const int64_t m0 = c * B;
    std::fill(seg.begin(), seg.end(), std::complex<double>(0, 0));
    for (int64_t i = 0; i < p.N + B - 1 && i < L; ++i) seg[(size_t)i] = std::conj(chirp(m0 - (p.N - 1) + i, p.M));
    host_fft(seg);
    for (int64_t k = 0; k < L; ++k) H[(size_t)(c * L + k)] = seg[(size_t)k] / (double)L;
  }
  int rc;
  if (p.dbl) {
    auto tw = build_two_level<double>(L, bits, &lo_n, &hi_n);
    if ((rc = upload(&p.d_blu_tw, tw)) != ADFFT_OK) return rc;
    if ((rc = upload(&p.d_chirp, flatten<double>(ch))) != ADFFT_OK) return rc;
    if ((rc = upload(&p.d_H, flatten<double>(H))) != ADFFT_OK) return rc;
  } else {
    auto tw = build_two_level<float>(L, bits, &lo_n, &hi_n);
    if ((rc = upload(&p.d_blu_tw, tw)) != ADFFT_OK) return rc;
    if ((rc = upload(&p.d_chirp, flatten<float>(ch))) != ADFFT_OK) return rc;
    if ((rc = upload(&p.d_H, flatten<float>(H))) != ADFFT_OK) return rc;
  }
  BluesteinLaunch& BL = p.blu;
  BluesteinArgs& b = BL.args;
  memset(&b, 0, sizeof(b));
  FusedArgs& a = b.f;
  a.batch = p.batch;
  a.M = p.M;
  a.Np = (int)L;
  a.logNp = ilog2(L);
  a.P = 1;
  a.q = 1;
  a.RPC = 1;
  a.C = 1;
  a.Nc = (int)L;
  a.Mc = (int)L;
  a.Mt = (int)L;
  a.tw_bits = bits;
  a.tw_lo_n = lo_n;
  a.tw_hi_n = hi_n;
  a.tw = p.d_blu_tw;
  a.scale = p.scale;
  a.region = (int)region;
  const int L2 = a.logNp;
  const int lr0 = (L2 == 0) ? 0 : (L2 % 4 ? L2 % 4 : 4);
  a.nrad = 1 + (L2 - lr0) / 4;
  a.status = p.d_status;
  a.in_stride = p.N;
  a.in_unit = (int)p.in_elem;
  b.chirp = p.d_chirp;
  b.H = p.d_H;
  b.N = p.N;
  b.B = (int)B;
  b.chunks = (int)chunks;
  b.real_in = p.real ? 1 : 0;
  a.offs = p.d_offs;
  BL.r0 = 1 << lr0;
  BL.dbl = p.dbl;
  BL.threads = std::max(32, (int)((L / vpt + 31) / 32 * 32));
  BL.grid_y = (int)std::max<int64_t>(1, std::min<int64_t>(p.batch, 65535));
  BL.smem = (size_t)lay.total;
  cudaError_t e = bluestein_prepare(BL);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(e);
  }
  p.blu_ok = true;
  return ADFFT_OK;
}


int cuda_status_of(cudaError_t e) { return cuda_status(e); }

int launch_forward(Plan& p, const void* in, void* out, cudaStream_t s) {
  if (p.fault.launch) return ADFFT_ERR_CUDA;   // injected launch failure: nothing is launched
  cudaError_t e;
  const bool tc = p.precision != ADFFT_PREC_NATIVE;
  const bool f16 = p.precision == ADFFT_PREC_FP16X2;
  if (p.algo == ADFFT_ALGO_BLUESTEIN) {
    e = bluestein_launch(p.blu, in, out, s);
  } else if (p.algo == ADFFT_ALGO_FOLD && p.fold_ok) {
    e = !tc ? fused_launch(p.fused, in, out, s)
            : f16 ? tc_launch_fused_fp16(p.fused, in, out, s) : tc_launch_fused_bf16(p.fused, in, out, s);
  } else if (p.tp_ok) {
    e = !tc ? fused_launch(p.tp1f_ok ? p.tp1f : p.tp1, in, p.d_ws, s)
            : f16 ? tc_launch_fused_fp16(p.tp1, in, p.d_ws, s) : tc_launch_fused_bf16(p.tp1, in, p.d_ws, s);
    if (e == cudaSuccess)
      e = !tc ? twopass_launch(p.tp2, p.d_ws, out, s)
              : f16 ? tc_launch_columns_fp16(p.tp2, p.d_ws, out, s) : tc_launch_columns_bf16(p.tp2, p.d_ws, out, s);
  } else {
    return ADFFT_ERR_NOT_SUPPORTED;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(e);
  }
  return ADFFT_OK;
}

int launch_adjoint(Plan& p, const void* g, void* xb, cudaStream_t s) {
  if (p.fault.launch) return ADFFT_ERR_CUDA;
  cudaError_t e;
  // the selected fold form, else whichever fold form the plan has (the chirp-z form has no adjoint kernel)
  const bool use_tp = p.tp_ok && (p.algo == ADFFT_ALGO_FOUR_STEP || !p.fold_ok);
  if (p.algo == ADFFT_ALGO_BLUESTEIN || (!p.fold_ok && !p.tp_ok)) {
    // chirp-z plans: the adjoint's own tables are set up at its first call
    const int rc = setup_bluestein_adjoint(p);
    if (rc != ADFFT_OK) return rc == ADFFT_ERR_UNSUPPORTED_SIZE ? ADFFT_ERR_NOT_SUPPORTED : rc;
    e = bluestein_adjoint_launch(p.bla, g, xb, s);
  } else if (!use_tp && p.fold_ok) {
    e = adjoint_launch(p.fused, g, xb, s);
  } else if (use_tp) {
    // transpose of the two passes, in reverse order, through the same workspace
    e = twopass_adjoint_launch(p.tp2, g, p.d_ws, s);
    if (e == cudaSuccess) e = adjoint_launch(p.tp1, p.d_ws, xb, s);
  } else {
    return ADFFT_ERR_NOT_SUPPORTED;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(e);
  }
  return ADFFT_OK;
}

int prepare_precision(Plan& p) {
  if (p.precision == ADFFT_PREC_NATIVE) return ADFFT_OK;
  const bool f16 = p.precision == ADFFT_PREC_FP16X2;
  cudaError_t e = cudaSuccess;
  if (p.fold_ok) e = f16 ? tc_prepare_fp16(&p.fused, nullptr) : tc_prepare_bf16(&p.fused, nullptr);
  if (e == cudaSuccess && p.tp_ok) e = f16 ? tc_prepare_fp16(&p.tp1, &p.tp2) : tc_prepare_bf16(&p.tp1, &p.tp2);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(e);
  }
  return ADFFT_OK;
}

namespace {

void release(Plan& p) {
  if (p.ragged) ragged_release(p);
  for (void** q : {&p.d_blu_tw, &p.d_chirp, &p.d_H, &p.d_bla_tw, &p.d_bla_chirp, &p.d_bla_H, &p.d_tp_tw1,
                   &p.d_tp_post, &p.d_tp_tw2, &p.d_tp_wM, &p.d_ws}) {
    if (*q) cudaFree(*q);
    *q = nullptr;
  }
  if (p.d_status) cudaFree(p.d_status);
  p.d_status = nullptr;
  if (p.d_tw) cudaFree(p.d_tw);
  if (p.d_stage_in) cudaFree(p.d_stage_in);
  if (p.d_stage_out) cudaFree(p.d_stage_out);
  p.d_tw = p.d_stage_in = p.d_stage_out = nullptr;
}

adfft_plan_t fail(int code, adfft_plan_s* h) {
  if (h) {
    release(h->p);
    delete h;
  }
  g_last_error = code;
  return nullptr;
}

bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return na && nb && x < y + nb && y < x + na;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace
}  // namespace adfft

using adfft::Plan;

extern "C" {

const char* adfft_status_string(int s) {
  switch (s) {
    case ADFFT_OK: return "ADFFT_OK";
    case ADFFT_ERR_INVALID_ARG: return "ADFFT_ERR_INVALID_ARG";
    case ADFFT_ERR_INVALID_ALPHA: return "ADFFT_ERR_INVALID_ALPHA";
    case ADFFT_ERR_UNSUPPORTED_SIZE: return "ADFFT_ERR_UNSUPPORTED_SIZE";
    case ADFFT_ERR_MISALIGNED: return "ADFFT_ERR_MISALIGNED";
    case ADFFT_ERR_OVERLAP: return "ADFFT_ERR_OVERLAP";
    case ADFFT_ERR_CUDA: return "ADFFT_ERR_CUDA";
    case ADFFT_ERR_OOM: return "ADFFT_ERR_OOM";
    case ADFFT_ERR_TIMEOUT: return "ADFFT_ERR_TIMEOUT";
    case ADFFT_ERR_NOT_SUPPORTED: return "ADFFT_ERR_NOT_SUPPORTED";
    default: return "ADFFT_ERR_UNKNOWN";
  }
}

int adfft_last_error(void) { return adfft::g_last_error; }

adfft_plan_t adfft_plan_create_bins(int64_t N, int64_t M, int64_t batch, int dtype) {
  using namespace adfft;
  if (N < 1 || batch < 0 || dtype < ADFFT_R32 || dtype > ADFFT_C128) return fail(ADFFT_ERR_INVALID_ARG, nullptr);
  if (M < 1) return fail(ADFFT_ERR_INVALID_ALPHA, nullptr);
  if (N > (int64_t(1) << 40) || M > (int64_t(1) << 40)) return fail(ADFFT_ERR_UNSUPPORTED_SIZE, nullptr);
  adfft_plan_s* h = new (std::nothrow) adfft_plan_s;
  if (!h) return fail(ADFFT_ERR_OOM, nullptr);
  Plan& p = h->p;
  p.N = N;
  p.M = M;
  p.batch = batch;
  p.dtype = dtype;
  p.real = (dtype == ADFFT_R32 || dtype == ADFFT_R64);
  p.dbl = (dtype == ADFFT_R64 || dtype == ADFFT_C128);
  p.in_elem = p.real ? (p.dbl ? 8 : 4) : (p.dbl ? 16 : 8);
  p.out_elem = p.dbl ? 16 : 8;
  p.scale = 1.0 / (double)N;
  p.fault = read_fault_spec();
  g_alloc_count = 0;
  g_alloc_fail_at = p.fault.alloc_at;
  struct Disarm {
    ~Disarm() { g_alloc_fail_at = 0; }
  } disarm;
  if (cudaGetDevice(&p.device) != cudaSuccess) {
    cudaGetLastError();
    return fail(ADFFT_ERR_CUDA, h);
  }
  {
    cudaError_t e = dev_malloc(reinterpret_cast<void**>(&p.d_status), sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p.d_status, 0, sizeof(int));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(cuda_status(e), h);
    }
  }
  const int rc_fold = setup_fold(p);
  if (rc_fold != ADFFT_OK && rc_fold != ADFFT_ERR_UNSUPPORTED_SIZE) return fail(rc_fold, h);
  if (!p.fold_ok) {
    const int rc_tp = setup_twopass(p);
    if (rc_tp != ADFFT_OK && rc_tp != ADFFT_ERR_UNSUPPORTED_SIZE) return fail(rc_tp, h);
  }
  // the chirp-z form is set up here only when no fold form applies (else on request)
  if (!p.fold_ok && !p.tp_ok) {
    const int rc_blu = setup_bluestein(p);
    if (rc_blu != ADFFT_OK && rc_blu != ADFFT_ERR_UNSUPPORTED_SIZE) return fail(rc_blu, h);
  }
  if (p.fold_ok) p.algo = ADFFT_ALGO_FOLD;
  else if (p.tp_ok) p.algo = ADFFT_ALGO_FOUR_STEP;
  else if (p.blu_ok) p.algo = ADFFT_ALGO_BLUESTEIN;
  else return fail(ADFFT_ERR_UNSUPPORTED_SIZE, h);
  p.auto_algo = p.algo;
  autotune_apply_cached(p);   // a launch shape recorded by the autotuner for these sizes, if any
  g_last_error = ADFFT_OK;
  return h;
}

adfft_plan_t adfft_plan_create(int64_t N, double alpha, int64_t batch, int dtype) {
  if (!(alpha > 0.0) || !isfinite(alpha)) return adfft::fail(ADFFT_ERR_INVALID_ALPHA, nullptr);
  if (N < 1) return adfft::fail(ADFFT_ERR_INVALID_ARG, nullptr);
  const double Md = alpha * (double)N;
  if (!(Md < 9.0e15)) return adfft::fail(ADFFT_ERR_UNSUPPORTED_SIZE, nullptr);
  const double Mr = nearbyint(Md);
  if (fabs(Md - Mr) > 1e-9 * Md || Mr < 1.0) return adfft::fail(ADFFT_ERR_INVALID_ALPHA, nullptr);
  return adfft_plan_create_bins(N, (int64_t)Mr, batch, dtype);
}

adfft_plan_t adfft_plan_create_ragged(const int64_t* N, const double* alpha, int64_t count, int dtype) {
  int err = ADFFT_OK;
  adfft_plan_s* h = adfft::ragged_create(N, alpha, count, dtype, &err);
  if (!h) return adfft::fail(err, nullptr);
  adfft::g_last_error = ADFFT_OK;
  return h;
}

int adfft_plan_offsets(adfft_plan_t plan, int64_t* in_off, int64_t* out_off) {
  if (!plan) return ADFFT_ERR_INVALID_ARG;
  const Plan& p = plan->p;
  if (p.ragged) {
    for (int64_t i = 0; i <= p.r_count; ++i) {
      if (in_off) in_off[i] = p.r_in_off[(size_t)i];
      if (out_off) out_off[i] = p.r_out_off[(size_t)i];
    }
    return ADFFT_OK;
  }
  for (int64_t i = 0; i <= p.batch; ++i) {
    if (in_off) in_off[i] = i * p.N;
    if (out_off) out_off[i] = i * p.M;
  }
  return ADFFT_OK;
}

int adfft_plan_destroy(adfft_plan_t plan) {
  if (!plan) return ADFFT_OK;
  cudaDeviceSynchronize();
  cudaGetLastError();
  adfft::release(plan->p);
  delete plan;
  return ADFFT_OK;
}

int adfft_plan_set_scale(adfft_plan_t plan, double S) {
  if (!plan || !isfinite(S)) return ADFFT_ERR_INVALID_ARG;
  if (plan->p.ragged) return ADFFT_ERR_NOT_SUPPORTED;   // each ragged signal keeps S = 1/N_i
  plan->p.scale = S;
  plan->p.fused.args.scale = S;
  plan->p.blu.args.f.scale = S;
  plan->p.tp2.args.scale = S;
  return ADFFT_OK;
}

int adfft_plan_set_algorithm(adfft_plan_t plan, int algo) {
  using namespace adfft;
  if (!plan) return ADFFT_ERR_INVALID_ARG;
  Plan& p = plan->p;
  if (p.ragged) return (algo == ADFFT_ALGO_AUTO) ? ADFFT_OK : ADFFT_ERR_NOT_SUPPORTED;
  if (algo == ADFFT_ALGO_AUTO) {
    p.algo = p.auto_algo;
    return ADFFT_OK;
  }
  if (p.half && algo != ADFFT_ALGO_FOLD) return ADFFT_ERR_NOT_SUPPORTED;   // half spectrum: single pass only
  if (algo == ADFFT_ALGO_FOLD) {
    // the single-pass fold form, else (sub-FFT beyond one cluster) its two-pass variant
    if (p.half && !p.fold_ok) return ADFFT_ERR_NOT_SUPPORTED;
    if (!p.fold_ok && !p.tp_ok) return ADFFT_ERR_NOT_SUPPORTED;
    p.algo = p.fold_ok ? ADFFT_ALGO_FOLD : ADFFT_ALGO_FOUR_STEP;
    return ADFFT_OK;
  }
  int rc = ADFFT_OK;
  if (algo == ADFFT_ALGO_FOUR_STEP) {
    rc = setup_twopass(p);
    if (rc == ADFFT_OK) rc = prepare_precision(p);
  } else if (algo == ADFFT_ALGO_BLUESTEIN) {
    rc = setup_bluestein(p);
  } else {
    return ADFFT_ERR_INVALID_ARG;
  }
  if (rc == ADFFT_ERR_UNSUPPORTED_SIZE) return ADFFT_ERR_NOT_SUPPORTED;
  if (rc != ADFFT_OK) return rc;
  p.algo = algo;
  return ADFFT_OK;
}

int adfft_plan_set_ragged_form(adfft_plan_t plan, int form) {
  using namespace adfft;
  if (!plan || (form != ADFFT_RAGGED_CLASSES && form != ADFFT_RAGGED_QUEUE)) return ADFFT_ERR_INVALID_ARG;
  if (!plan->p.ragged) return ADFFT_ERR_NOT_SUPPORTED;
  return ragged_set_form(plan->p, form);
}

int adfft_ragged_queue_layout(const int64_t* N, const double* alpha, int64_t count, int dtype, int32_t lag,
                              int32_t* tiles, int64_t tile_capacity, int64_t* ntiles, int64_t* whole,
                              int64_t whole_capacity, int64_t* nwhole) {
  return adfft::ragged_queue_layout(N, alpha, count, dtype, (int)lag, tiles, tile_capacity, ntiles, whole,
                                    whole_capacity, nwhole);
}

int adfft_plan_set_output(adfft_plan_t plan, int mode) {
  using namespace adfft;
  if (!plan || (mode != ADFFT_OUTPUT_FULL && mode != ADFFT_OUTPUT_HALF)) return ADFFT_ERR_INVALID_ARG;
  Plan& p = plan->p;
  const bool want = mode == ADFFT_OUTPUT_HALF;
  if (want == p.half) return ADFFT_OK;
  if (want) {
    // real input packed two samples per element (even N and M), single-pass fold form
    int m;
    int64_t Nc, Mc;
    core_shape(p, &m, &Nc, &Mc);
    if (p.ragged || m != kLoadRealPacked || !p.fold_ok) return ADFFT_ERR_NOT_SUPPORTED;
  }
  const bool old = p.half;
  const FoldChoice keep = p.fold_choice;
  p.half = want;
  FoldChoice c = keep;
  if (want && c.stage == 2) c.stage = -1;   // the push form writes the full spectrum only
  int rc = p.fold_ok ? setup_fold(p, &c) : ADFFT_OK;
  if (rc != ADFFT_OK) {
    p.half = old;
    setup_fold(p, &keep);
    return rc == ADFFT_ERR_UNSUPPORTED_SIZE ? ADFFT_ERR_NOT_SUPPORTED : rc;
  }
  if (p.fold_ok) p.algo = ADFFT_ALGO_FOLD;
  return ADFFT_OK;
}

int adfft_plan_set_launch_shape(adfft_plan_t plan, int64_t fft_len, int cluster, int staged, int grid) {
  using namespace adfft;
  if (!plan || fft_len < 0 || cluster < 0 || cluster > kFoldMaxCluster || staged < -1 || staged > 2 || grid < -1)
    return ADFFT_ERR_INVALID_ARG;
  Plan& p = plan->p;
  if (p.ragged) return ADFFT_ERR_NOT_SUPPORTED;
  FoldChoice c{fft_len, cluster, staged, grid};
  int rc = setup_fold(p, &c);
  if (rc == ADFFT_OK) rc = prepare_precision(p);
  if (rc == ADFFT_ERR_UNSUPPORTED_SIZE) return ADFFT_ERR_NOT_SUPPORTED;
  if (rc != ADFFT_OK) return rc;
  p.algo = ADFFT_ALGO_FOLD;
  return ADFFT_OK;
}

int adfft_plan_set_precision(adfft_plan_t plan, int mode) {
  using namespace adfft;
  if (!plan) return ADFFT_ERR_INVALID_ARG;
  Plan& p = plan->p;
  if (mode == ADFFT_PREC_NATIVE) {
    p.precision = mode;
    return ADFFT_OK;
  }
  if (mode != ADFFT_PREC_FP16X2 && mode != ADFFT_PREC_BF16X3) return ADFFT_ERR_INVALID_ARG;
  // tensor-core radix-16 passes: complex64 data in the fold forms (not chirp-z, not ragged)
  if (p.dbl || p.ragged || (!p.fold_ok && !p.tp_ok)) return ADFFT_ERR_NOT_SUPPORTED;
  const int old = p.precision;
  p.precision = mode;
  const int rc = prepare_precision(p);
  if (rc != ADFFT_OK) p.precision = old;
  return rc;
}

int adfft_plan_get_info(adfft_plan_t plan, adfft_plan_info_t* info) {
  if (!plan || !info) return ADFFT_ERR_INVALID_ARG;
  const Plan& p = plan->p;
  memset(info, 0, sizeof(*info));
  info->N = p.N;
  info->M = p.M;
  info->batch = p.batch;
  info->dtype = p.dtype;
  info->algo = p.algo;
  info->out_bins = p.ragged ? 0 : p.out_bins();
  if (p.ragged) {
    info->batch = p.r_count;
    info->fft_len = 0;
    info->residues = (int64_t)p.r_sub.size();   // shape classes
    info->fold = 0;
    info->cluster = 0;
    int passes = 1;
    bool tuned = !p.r_sub.empty();
    for (auto* sp : p.r_sub) {
      passes = std::max(passes, sp->p.algo == ADFFT_ALGO_FOUR_STEP ? 2 : 1);
      tuned = tuned && sp->p.tuned;
    }
    info->passes = passes;
    info->scale = 0.0;
    info->tuned = tuned ? 1 : 0;
    return ADFFT_OK;
  }
  if (p.algo == ADFFT_ALGO_BLUESTEIN) {
    info->fft_len = p.blu.args.f.Np;
    info->residues = p.blu.args.chunks;
    info->fold = 0;
    info->cluster = 1;
  } else if (p.algo == ADFFT_ALGO_FOUR_STEP) {
    info->fft_len = p.tp_A * p.tp_B;      // the sub-FFT length, split A x B over two passes
    info->four_step_a = (int32_t)p.tp_A;
    info->residues = p.tp1.args.P;
    info->fold = p.tp1.args.q;
    info->cluster = p.tp1.args.C;
  } else {
    info->fft_len = p.fused.args.Np;
    info->residues = p.fused.args.P;
    info->fold = p.fused.args.q;
    info->cluster = p.fused.args.C;
  }
  info->passes = (p.algo == ADFFT_ALGO_FOUR_STEP) ? 2 : 1;
  info->scale = p.scale;
  info->staged = (p.algo != ADFFT_ALGO_FOLD) ? 0 : p.fused.push ? 2 : (p.fused.args.stage_bytes > 0 ? 1 : 0);
  info->grid = (p.algo == ADFFT_ALGO_FOLD) ? p.fused.grid_y : (p.algo == ADFFT_ALGO_FOUR_STEP) ? p.tp1.grid_y : 0;
  info->tuned = p.tuned ? 1 : 0;
  return ADFFT_OK;
}

size_t adfft_plan_workspace_bytes(adfft_plan_t plan) {
  if (!plan) return 0;
  size_t total = plan->p.ws_bytes;
  for (auto* sp : plan->p.r_sub) total += sp->p.ws_bytes;
  return total;
}

int adfft_execute(adfft_plan_t plan, const void* d_in, void* d_out, void* stream) {
  using namespace adfft;
  if (!plan || !d_in || !d_out) return ADFFT_ERR_INVALID_ARG;
  Plan& p = plan->p;
  if (!aligned16(d_in) || !aligned16(d_out)) return ADFFT_ERR_MISALIGNED;
  if (overlaps(d_in, p.in_bytes(), d_out, p.out_bytes())) return ADFFT_ERR_OVERLAP;
  if (p.ragged) return ragged_execute(p, d_in, d_out, (cudaStream_t)stream, 0);
  if (p.batch == 0) return ADFFT_OK;
  return launch_forward(p, d_in, d_out, (cudaStream_t)stream);
}

int adfft_execute_adjoint(adfft_plan_t plan, const void* d_grad_out, void* d_grad_in, void* stream) {
  using namespace adfft;
  if (!plan || !d_grad_out || !d_grad_in) return ADFFT_ERR_INVALID_ARG;
  Plan& p = plan->p;
  if (!aligned16(d_grad_out) || !aligned16(d_grad_in)) return ADFFT_ERR_MISALIGNED;
  if (overlaps(d_grad_out, p.out_bytes(), d_grad_in, p.in_bytes())) return ADFFT_ERR_OVERLAP;
  if (p.ragged) return ragged_execute(p, d_grad_out, d_grad_in, (cudaStream_t)stream, 1);
  if (p.batch == 0) return ADFFT_OK;
  return launch_adjoint(p, d_grad_out, d_grad_in, (cudaStream_t)stream);
}

int adfft_execute_host(adfft_plan_t plan, const void* h_in, void* h_out, void* stream) {
  using namespace adfft;
  if (!plan || !h_in || !h_out) return ADFFT_ERR_INVALID_ARG;
  Plan& p = plan->p;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t ib = p.in_bytes(), ob = p.out_bytes();
  if (p.batch == 0) return ADFFT_OK;
  if (!p.d_stage_in) {
    cudaError_t e = cudaMalloc(&p.d_stage_in, ib);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p.d_stage_in = nullptr;
      return cuda_status(e);
    }
  }
  if (!p.d_stage_out) {
    cudaError_t e = cudaMalloc(&p.d_stage_out, ob);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p.d_stage_out = nullptr;
      return cuda_status(e);
    }
  }
  cudaError_t e = cudaMemcpyAsync(p.d_stage_in, h_in, ib, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_status(e);
  int rc = adfft_execute(plan, p.d_stage_in, p.d_stage_out, stream);
  if (rc != ADFFT_OK) return rc;
  e = cudaMemcpyAsync(h_out, p.d_stage_out, ob, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  return adfft_plan_sync_status(plan, stream);
}

int adfft_plan_sync_status(adfft_plan_t plan, void* stream) {
  using namespace adfft;
  if (!plan) return ADFFT_ERR_INVALID_ARG;
  Plan& p = plan->p;
  cudaStream_t s = (cudaStream_t)stream;
  if (p.ragged) {
    // the shape classes' kernels report into their sub-plans' status words, the queue
    // kernel into its own
    int rc = ADFFT_OK;
    for (auto* sp : p.r_sub) {
      const int r = adfft_plan_sync_status(sp, stream);
      if (rc == ADFFT_OK) rc = r;
    }
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_status(e);
    }
    int q = 0;
    const int rq = ragged_queue_status(p, &q);
    if (rc == ADFFT_OK) rc = rq != ADFFT_OK ? rq : (q != 0 ? ADFFT_ERR_TIMEOUT : ADFFT_OK);
    return rc;
  }
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, p.d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(e);
  }
  if (h != 0) {
    e = cudaMemsetAsync(p.d_status, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_status(e);
    }
    return h == kStatusTimeout ? ADFFT_ERR_TIMEOUT : ADFFT_ERR_CUDA;
  }
  return ADFFT_OK;
}

}  // extern "C"
