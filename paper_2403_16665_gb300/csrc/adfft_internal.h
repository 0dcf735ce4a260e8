// Internal plan representation and kernel launchers of the adfft library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "adfft.h"
#include "fft_device.cuh"
#include "fused.cuh"
#include "bluestein.cuh"
#include "twopass.cuh"
#include "ragged_queue.cuh"

struct adfft_plan_s;

namespace adfft {

constexpr int kRaggedStreams = 4;   // side streams a ragged plan's graph forks over

// Launch geometry of the fused single-pass kernel.
struct FusedLaunch {
  FusedArgs args;
  int mode;        // LoadMode
  int r0;          // radix of the first pass
  bool dbl;        // double2 (true) or float2 elements
  int threads;
  int grid_y;
  size_t smem;
  bool push = false;   // exchange by bulk push copies (fused_push.cuh) instead of peer loads
};

// Launch-shape choice of the fused fold path (set by the plan's default rule
// or by the autotuner).
struct FoldChoice {
  int64_t np = 0;    // sub-FFT length: a power of two dividing gcd(Mc, Nc); 0 = the largest such
  int cluster = 0;   // CTAs per cluster; 0 = the smallest that fits
  int stage = -1;    // input staging through shared memory: 1 required, 0 never, -1 where it fits;
                     // 2: no staging, residues exchanged by bulk push copies (fused_push.cuh)
  int grid = 0;      // clusters launched: 0 = as many as can be resident at once (each loops over
                     // signals), -1 = one per signal, > 0 = that many
  int vsplit = 0;    // columns of the two-pass form only, > 1: residues split over that many
                     // independent CTAs per column (no cluster), each writing its own bins
};

// Launch geometry of the chirp-z kernel.
struct BluesteinLaunch {
  BluesteinArgs args;
  int r0;
  bool dbl;
  int threads;
  int grid_y;
  size_t smem;
};

// Launch geometry of the chirp-z adjoint kernel.
struct BluesteinAdjLaunch {
  BluesteinAdjArgs args;
  int r0;
  bool dbl;
  int threads;
  int grid_y;
  size_t smem;
};

// Launch geometry of the second pass of the two-pass form.
struct TwoPassLaunch {
  TwoPassArgs args;
  int r0;
  bool dbl;
  int threads;
  int grid_x, grid_y;
  size_t smem;
};

// Test fault injection requested through ADFFT_FAULT (plan.cu).
struct FaultSpec {
  int alloc_at = 0;          // fail the k-th device allocation of plan creation (0: none)
  bool launch = false;       // every launch of the plan fails without launching
  long long copy_skip = -1;  // the fused kernel skips the input copy of this signal (-1: none)
};
FaultSpec read_fault_spec();
cudaError_t dev_malloc(void** p, size_t bytes);

struct Plan {
  FaultSpec fault{};
  int64_t N = 0, M = 0, batch = 0;
  int dtype = 0;
  bool real = false, dbl = false;
  int algo = ADFFT_ALGO_FOLD;
  int precision = ADFFT_PREC_NATIVE;
  double scale = 1.0;
  int device = 0;
  size_t in_elem = 0, out_elem = 0;   // bytes per input scalar/complex, per output complex

  int auto_algo = ADFFT_ALGO_FOLD;    // what ADFFT_ALGO_AUTO selects (default rule or autotuner)
  bool stage_ok = true;               // input staging allowed (bulk copies need 16-byte aligned signals)
  const long long* d_offs = nullptr;  // ragged sub-plans: device {input byte, output bin} offsets per signal
  bool tuned = false;                 // launch shape set by the autotuner (or its cache)

  // fold + FFT (fused) path
  bool fold_ok = false;
  FoldChoice fold_choice{};           // the choice p.fused was configured with
  FusedLaunch fused{};
  void* d_tw = nullptr;               // twiddle table of the fused path
  int* d_status = nullptr;            // device status word (0, or ADFFT_ERR_TIMEOUT)

  // chirp-z path
  bool blu_ok = false;
  BluesteinLaunch blu{};
  void* d_blu_tw = nullptr;           // W_L table
  void* d_chirp = nullptr;            // chirp c_j
  void* d_H = nullptr;                // per-chunk kernel spectra
  // chirp-z adjoint (set up at the first adjoint call of a plan without a fold form)
  bool bla_ok = false;
  BluesteinAdjLaunch bla{};
  void* d_bla_tw = nullptr;           // W_L table of the adjoint's transform length
  void* d_bla_chirp = nullptr;        // chirp c_j, j < max(N, M)
  void* d_bla_H = nullptr;            // kernel spectra per block difference

  // two-pass path (sub-FFT beyond one cluster): pass 1 = fused kColumns launch, pass 2 = columns
  bool tp_ok = false;
  int64_t tp_A = 0, tp_B = 0;
  int64_t tp_force_A = 0;             // two-pass split chosen by the autotuner (0: the default rule)
  FusedLaunch tp1{};
  FusedLaunch tp1f{};      // pass 1 forward with the residues split over independent CTAs
  bool tp1f_ok = false;    // (FP32 forward only; the adjoint and precision forms use tp1)
  TwoPassLaunch tp2{};
  void* d_tp_tw1 = nullptr;           // pass-1 W_R1 table
  void* d_tp_post = nullptr;          // pass-1 row twiddles W_Mc
  void* d_tp_tw2 = nullptr;           // pass-2 W_B table
  void* d_tp_wM = nullptr;            // pass-2 W_M table (real unpacking)
  void* d_ws = nullptr;               // scratch [batch][B][R1]
  size_t ws_bytes = 0;

  // ragged plan: one uniform sub-plan per (N, M) shape class, all launched from one CUDA graph
  bool ragged = false;
  int64_t r_count = 0;
  std::vector<int64_t> r_in_off, r_out_off;    // count + 1 packed offsets
  std::vector<adfft_plan_s*> r_sub;             // sub-plans (own their tables and workspace)
  std::vector<void*> r_offs;                    // per class: device {in, out} offsets of its signals
  cudaStream_t r_streams[kRaggedStreams] = {};
  cudaEvent_t r_fork = nullptr, r_join[kRaggedStreams] = {};
  cudaGraphExec_t r_graph[2] = {nullptr, nullptr};   // forward, adjoint
  // ragged forward as one persistent kernel over a tile queue (ragged_queue.cuh)
  bool rq_ok = false;                 // the queue form serves this plan
  bool rq_on = false;                 // the forward uses it (adfft_plan_set_ragged_form)
  RqArgs rq{};                        // kernel arguments (buffers of the plan)
  int rq_grid = 0;
  size_t rq_smem = 0;
  std::vector<void*> rq_bufs;         // device allocations of the queue form
  const void* r_graph_in[2] = {nullptr, nullptr};
  void* r_graph_out[2] = {nullptr, nullptr};

  // host-memory staging of adfft_execute_host
  void* d_stage_in = nullptr;
  void* d_stage_out = nullptr;

  // packed offsets (uniform plans: i*N, i*M)
  std::vector<int64_t> in_off, out_off;

  size_t in_bytes() const { return (size_t)batch * (size_t)N * in_elem; }
  bool half = false;                  // real input: output X_0 .. X_{M/2} only (adfft_plan_set_output)
  int64_t out_bins() const { return half ? M / 2 + 1 : M; }
  size_t out_bytes() const { return (size_t)batch * (size_t)out_bins() * out_elem; }
};

// Compile-time-shape kernels of the real classes with a 16384-point packed sub-FFT and one
// residue per CTA (spec16k.cu); nullptr when the launch is not of that class.
using SpecKernel = void (*)(const FusedArgs);
SpecKernel spec16k_forward(const FusedLaunch& L);
SpecKernel spec16k_adjoint(const FusedLaunch& L);

// Push-exchange forward kernels (fused_push.cu): the kernel for a launch whose args (C = P,
// one residue per CTA, packed real fp32, no staging) it serves, else nullptr; and its
// threads and dynamic shared memory.
SpecKernel push_forward(const FusedLaunch& L);
bool push_geometry(const FusedLaunch& L, int* threads, size_t* smem);

// Kernel launchers (fused.cu).  Return a cudaError_t.
cudaError_t fused_prepare(const FusedLaunch& L);   // sets function attributes once
cudaError_t fused_launch(const FusedLaunch& L, const void* in, void* out, cudaStream_t stream);
int fused_max_active_clusters(const FusedLaunch& L);
int fused_values_per_thread(bool dbl);

// Adjoint launchers (adjoint.cu): same launch shape as the forward, no input staging.
cudaError_t adjoint_prepare(const FusedLaunch& L);
cudaError_t adjoint_launch(const FusedLaunch& L, const void* g, void* xb, cudaStream_t stream);
size_t adjoint_smem_bytes(const FusedLaunch& L);

// Plan set-up steps (plan.cu).  Each returns ADFFT_OK, ADFFT_ERR_UNSUPPORTED_SIZE
// when the form does not apply to the plan's sizes, or a CUDA/allocation error.
void core_shape(const Plan& p, int* mode, int64_t* Nc, int64_t* Mc);
int setup_fold(Plan& p, const FoldChoice* forced = nullptr);
int setup_twopass(Plan& p);
int setup_bluestein(Plan& p);
int setup_bluestein_adjoint(Plan& p);
void release_twopass(Plan& p);
int prepare_precision(Plan& p);   // function attributes of the precision-form kernels in use
int64_t plan_gcd(int64_t a, int64_t b);
// two-level W_Mt table (lo entries then hi entries, interleaved re, im) rounded to float once
std::vector<float> twiddle_table_f32(int64_t Mt, int* bits, int* lo_n, int* hi_n);
constexpr int kFoldMaxCluster = 16;   // largest cluster the fused kernel is launched with
constexpr int kTuneMaxFold = 16;      // largest fold factor q the autotuner and default rule consider

// Autotuner (autotune.cu): apply a cached choice at plan creation; time and choose.
void autotune_apply_cached(Plan& p);
int autotune_plan(Plan& p, const void* in, void* out, cudaStream_t s, int iters, int flags);
void ragged_invalidate(Plan& p);   // drop captured graphs (launch shapes changed)

// Launch the plan's forward / adjoint kernels (no argument checks).
int launch_forward(Plan& p, const void* in, void* out, cudaStream_t s);
int launch_adjoint(Plan& p, const void* g, void* xb, cudaStream_t s);
int cuda_status_of(cudaError_t e);

// Ragged plans (ragged.cu).
adfft_plan_s* ragged_create(const int64_t* N, const double* alpha, int64_t count, int dtype, int* err);
int ragged_execute(Plan& p, const void* in, void* out, cudaStream_t s, int which);
void ragged_release(Plan& p);
int ragged_queue_layout(const int64_t* N, const double* alpha, int64_t count, int dtype, int lag,
                        int32_t* tiles_out, int64_t tile_capacity, int64_t* ntiles, int64_t* whole_out,
                        int64_t whole_capacity, int64_t* nwhole);
int ragged_set_form(Plan& p, int form);              // ADFFT_RAGGED_CLASSES / ADFFT_RAGGED_QUEUE
int ragged_queue_status(Plan& p, int* status);       // read and clear the queue kernel's status word

// Two-pass second-pass launchers (twopass.cu).
cudaError_t twopass_prepare(const TwoPassLaunch& L);
cudaError_t twopass_launch(const TwoPassLaunch& L, const void* scratch, void* out, cudaStream_t stream);
cudaError_t twopass_adjoint_launch(const TwoPassLaunch& L, const void* g, void* scratch, cudaStream_t stream);

// Tensor-core (precision form) launchers (fused_tc_fp16.cu, fused_tc_bf16.cu).
cudaError_t tc_prepare_fp16(const FusedLaunch* L, const TwoPassLaunch* L2);
cudaError_t tc_launch_fused_fp16(const FusedLaunch& L, const void* in, void* out, cudaStream_t s);
cudaError_t tc_launch_columns_fp16(const TwoPassLaunch& L, const void* scratch, void* out, cudaStream_t s);
cudaError_t tc_prepare_bf16(const FusedLaunch* L, const TwoPassLaunch* L2);
cudaError_t tc_launch_fused_bf16(const FusedLaunch& L, const void* in, void* out, cudaStream_t s);
cudaError_t tc_launch_columns_bf16(const TwoPassLaunch& L, const void* scratch, void* out, cudaStream_t s);

// Chirp-z launchers (bluestein.cu).
cudaError_t bluestein_prepare(const BluesteinLaunch& L);
cudaError_t bluestein_launch(const BluesteinLaunch& L, const void* in, void* out, cudaStream_t stream);
cudaError_t bluestein_adjoint_prepare(const BluesteinAdjLaunch& L);
cudaError_t bluestein_adjoint_launch(const BluesteinAdjLaunch& L, const void* g, void* xb, cudaStream_t stream);
constexpr int kBlaAccF32 = 16, kBlaAccF64 = 8;   // output samples per thread of the chirp-z adjoint

}  // namespace adfft

struct adfft_plan_s {
  adfft::Plan p;
};
