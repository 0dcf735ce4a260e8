// Ragged plans: many signals of different N and alpha, packed back to back.
//
// Signals are grouped into shape classes (N, M).  Each class gets a uniform
// sub-plan whose launches read and write through a device table of per-signal
// offsets, so the class's signals stay where the caller packed them.  The
// first execute for a given (input, output) pair captures every class launch
// into one CUDA graph, forked over a few internal streams so that small classes
// run side by side; later executes replay that graph on the caller's stream
// with a single cudaGraphLaunch.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "adfft_internal.h"

namespace adfft {

namespace {

void set_offsets(Plan& sub, const long long* d_offs) {
  sub.d_offs = d_offs;
  sub.fused.args.offs = d_offs;
  sub.blu.args.f.offs = d_offs;
  sub.tp1.args.offs = d_offs;
  sub.tp2.args.f.offs = d_offs;
}

void destroy_graphs(Plan& p) {
  for (int w = 0; w < 2; ++w) {
    if (p.r_graph[w]) cudaGraphExecDestroy(p.r_graph[w]);
    p.r_graph[w] = nullptr;
    p.r_graph_in[w] = nullptr;
    p.r_graph_out[w] = nullptr;
  }
}

int capture(Plan& p, const void* in, void* out, int which) {
  cudaStream_t s0 = p.r_streams[0];
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_status_of(e);
  int rc = ADFFT_OK;
  e = cudaEventRecord(p.r_fork, s0);
  for (int k = 1; k < kRaggedStreams && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(p.r_streams[k], p.r_fork, 0);
  if (e != cudaSuccess) rc = cuda_status_of(e);
  // largest classes first, spread round-robin over the streams
  std::vector<std::pair<double, size_t>> order;
  for (size_t i = 0; i < p.r_sub.size(); ++i) {
    const Plan& q = p.r_sub[i]->p;
    order.push_back({-(double)q.batch * (double)(q.M + q.N), i});
  }
  std::sort(order.begin(), order.end());
  for (size_t t = 0; t < order.size() && rc == ADFFT_OK; ++t) {
    Plan& q = p.r_sub[order[t].second]->p;
    cudaStream_t st = p.r_streams[t % kRaggedStreams];
    rc = (which == 0) ? launch_forward(q, in, out, st) : launch_adjoint(q, in, out, st);
  }
  for (int k = 1; k < kRaggedStreams; ++k) {
    cudaError_t e2 = cudaEventRecord(p.r_join[k], p.r_streams[k]);
    if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s0, p.r_join[k], 0);
    if (e2 != cudaSuccess && rc == ADFFT_OK) rc = cuda_status_of(e2);
  }
  e = cudaStreamEndCapture(s0, &graph);
  if (e != cudaSuccess && rc == ADFFT_OK) rc = cuda_status_of(e);
  if (rc != ADFFT_OK) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc;
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status_of(e);
  }
  if (p.r_graph[which]) cudaGraphExecDestroy(p.r_graph[which]);
  p.r_graph[which] = exec;
  p.r_graph_in[which] = in;
  p.r_graph_out[which] = out;
  return ADFFT_OK;
}

}  // namespace

void ragged_invalidate(Plan& p) { destroy_graphs(p); }

void ragged_release(Plan& p) {
  destroy_graphs(p);
  for (auto* sp : p.r_sub) adfft_plan_destroy(sp);
  p.r_sub.clear();
  for (void* d : p.r_offs)
    if (d) cudaFree(d);
  p.r_offs.clear();
  for (int k = 0; k < kRaggedStreams; ++k) {
    if (p.r_streams[k]) cudaStreamDestroy(p.r_streams[k]);
    if (p.r_join[k]) cudaEventDestroy(p.r_join[k]);
    p.r_streams[k] = nullptr;
    p.r_join[k] = nullptr;
  }
  if (p.r_fork) cudaEventDestroy(p.r_fork);
  p.r_fork = nullptr;
}

adfft_plan_s* ragged_create(const int64_t* N, const double* alpha, int64_t count, int dtype, int* err) {
  *err = ADFFT_OK;
  if (!N || !alpha || count < 0) {
    *err = ADFFT_ERR_INVALID_ARG;
    return nullptr;
  }
  if (dtype != ADFFT_R32 && dtype != ADFFT_C64) {
    *err = ADFFT_ERR_NOT_SUPPORTED;
    return nullptr;
  }
  std::vector<int64_t> Ms((size_t)count);
  for (int64_t i = 0; i < count; ++i) {
    if (N[i] < 1) {
      *err = ADFFT_ERR_INVALID_ARG;
      return nullptr;
    }
    const double a = alpha[i];
    if (!(a > 0.0) || !isfinite(a)) {
      *err = ADFFT_ERR_INVALID_ALPHA;
      return nullptr;
    }
    const double Md = a * (double)N[i];
    const double Mr = nearbyint(Md);
    if (fabs(Md - Mr) > 1e-9 * Md || Mr < 1.0) {
      *err = ADFFT_ERR_INVALID_ALPHA;
      return nullptr;
    }
    Ms[(size_t)i] = (int64_t)Mr;
  }
  adfft_plan_s* h = new (std::nothrow) adfft_plan_s;
  if (!h) {
    *err = ADFFT_ERR_OOM;
    return nullptr;
  }
  Plan& p = h->p;
  p.ragged = true;
  p.r_count = count;
  p.dtype = dtype;
  p.real = (dtype == ADFFT_R32);
  p.dbl = false;
  p.in_elem = p.real ? 4 : 8;
  p.out_elem = 8;
  p.r_in_off.assign((size_t)count + 1, 0);
  p.r_out_off.assign((size_t)count + 1, 0);
  for (int64_t i = 0; i < count; ++i) {
    p.r_in_off[(size_t)i + 1] = p.r_in_off[(size_t)i] + N[i];
    p.r_out_off[(size_t)i + 1] = p.r_out_off[(size_t)i] + Ms[(size_t)i];
  }
  // the packed buffers, as one "signal" for the size and overlap checks
  p.batch = 1;
  p.N = p.r_in_off[(size_t)count];
  p.M = p.r_out_off[(size_t)count];
  auto bail = [&](int code) {
    ragged_release(p);
    delete h;
    *err = code;
    return (adfft_plan_s*)nullptr;
  };
  if (cudaGetDevice(&p.device) != cudaSuccess) {
    cudaGetLastError();
    return bail(ADFFT_ERR_CUDA);
  }
  // shape classes
  std::map<std::pair<int64_t, int64_t>, std::vector<int64_t>> classes;
  for (int64_t i = 0; i < count; ++i) classes[{N[i], Ms[(size_t)i]}].push_back(i);
  for (auto& kv : classes) {
    const int64_t n = kv.first.first, m = kv.first.second;
    const std::vector<int64_t>& members = kv.second;
    adfft_plan_s* sub = adfft_plan_create_bins(n, m, (int64_t)members.size(), dtype);
    if (!sub) return bail(adfft_last_error());
    p.r_sub.push_back(sub);
    std::vector<long long> offs(2 * members.size());
    bool stage_ok = true;
    for (size_t k = 0; k < members.size(); ++k) {
      offs[2 * k] = p.r_in_off[(size_t)members[k]] * (long long)p.in_elem;   // bytes
      offs[2 * k + 1] = p.r_out_off[(size_t)members[k]];                      // bins
      if (offs[2 * k] % 16) stage_ok = false;
    }
    void* d = nullptr;
    cudaError_t e = cudaMalloc(&d, offs.size() * sizeof(long long));
    if (e == cudaSuccess) e = cudaMemcpy(d, offs.data(), offs.size() * sizeof(long long), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (d) cudaFree(d);
      return bail(cuda_status_of(e));
    }
    p.r_offs.push_back(d);
    set_offsets(sub->p, static_cast<const long long*>(d));
    if (!stage_ok) {
      // bulk copies need 16-byte aligned sources: re-plan the class without input staging
      sub->p.stage_ok = false;
      if (sub->p.fold_ok && sub->p.fused.args.stage_bytes > 0) {
        FoldChoice c = sub->p.fold_choice;
        c.stage = 0;
        c.cluster = 0;
        const int rc = setup_fold(sub->p, &c);
        if (rc != ADFFT_OK) return bail(rc);
      }
    }
  }
  for (int k = 0; k < kRaggedStreams; ++k) {
    if (cudaStreamCreateWithFlags(&p.r_streams[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p.r_join[k], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return bail(ADFFT_ERR_CUDA);
    }
  }
  if (cudaEventCreateWithFlags(&p.r_fork, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return bail(ADFFT_ERR_CUDA);
  }
  return h;
}

int ragged_execute(Plan& p, const void* in, void* out, cudaStream_t s, int which) {
  if (p.r_count == 0) return ADFFT_OK;
  if (which == 1) {
    for (auto* sp : p.r_sub)
      if (!sp->p.fold_ok && !sp->p.tp_ok) return ADFFT_ERR_NOT_SUPPORTED;
  }
  if (!p.r_graph[which] || p.r_graph_in[which] != in || p.r_graph_out[which] != out) {
    int rc = capture(p, in, out, which);
    if (rc != ADFFT_OK) return rc;
  }
  cudaError_t e = cudaGraphLaunch(p.r_graph[which], s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status_of(e);
  }
  return ADFFT_OK;
}

}  // namespace adfft
