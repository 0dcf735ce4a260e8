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

void release_queue(Plan& p);
int launch_queue(Plan& p, const void* in, void* out, cudaStream_t s);

void set_offsets(Plan& sub, const long long* d_offs) {
  sub.d_offs = d_offs;
  sub.fused.args.offs = d_offs;
  sub.blu.args.f.offs = d_offs;
  sub.tp1.args.offs = d_offs;
  sub.tp1f.args.offs = d_offs;
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
  if (which == 0 && p.rq_on) {
    rc = launch_queue(p, in, out, s0);
    order.clear();
  }
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
  release_queue(p);
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

namespace {

// Small tiles: 4096 points and 128 threads give 4 independent CTAs per SM (shared memory
// and registers both allow 4), which hides the latency of each CTA's fold / pass / store
// phases behind the others better than one 512-thread CTA with 16384 points.
constexpr int kRqThreads = 128;
constexpr int kRqTilePoints = 4096;         // complex points of U one tile holds in shared memory
constexpr int kRqLeadersPerTile = 8192;     // leader bins of one unpack tile

template <typename T>
int rq_upload(Plan& p, const std::vector<T>& v, T** dst) {
  void* d = nullptr;
  const size_t bytes = std::max<size_t>(16, v.size() * sizeof(T));
  cudaError_t e = cudaMalloc(&d, bytes);
  if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (d) cudaFree(d);
    return cuda_status_of(e);
  }
  p.rq_bufs.push_back(d);
  *dst = static_cast<T*>(d);
  return ADFFT_OK;
}

// signals of a class that one whole tile transforms side by side
int whole_group(const RqClass& k) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(kRqMaxGroup, kRqTilePoints / ((int64_t)k.P * k.Np)));
}

// ---- layout of the queue form on the host (no CUDA call: adfft_ragged_queue_layout uses it too)

// Queue geometry of a shape class from its core shape (load mode, Nc input elements, Mc bins)
// and its M output bins: packed real (even N and M) or complex input, the largest
// power-of-two sub-FFT dividing gcd(Mc, Nc) that one tile holds, with a fold of at most 64.
// ADFFT_ERR_UNSUPPORTED_SIZE where the queue form has no geometry for the class.
int rq_geometry(int mode, int64_t Nc, int64_t Mc, int64_t M, RqClass& k) {
  if (mode != kLoadRealPacked && mode != kLoadComplex) return ADFFT_ERR_UNSUPPORTED_SIZE;
  const int64_t gg = plan_gcd(Mc, Nc);
  int64_t Np = gg & -gg;
  while (Np > kRqTilePoints) Np /= 2;
  if (Nc / Np > 64 || Mc >= (int64_t(1) << 30)) return ADFFT_ERR_UNSUPPORTED_SIZE;
  memset(&k, 0, sizeof(k));
  k.Np = (int)Np;
  k.logNp = 0;
  while ((1 << k.logNp) < k.Np) ++k.logNp;
  k.P = (int)(Mc / Np);
  k.q = (int)(Nc / Np);
  k.Nc = (int)Nc;
  k.Mc = (int)Mc;
  k.Mt = (int)(mode == kLoadRealPacked ? M : Mc);
  k.region = k.Np + k.Np / 16 + 2;
  int lr0 = (k.logNp == 0) ? 0 : (k.logNp % 4 ? k.logNp % 4 : 4);
  if (lr0 == 1 && k.logNp >= 5) lr0 = 5;   // radix 2 merged with one radix-16 pass into radix 32
  k.nrad = 1 + (k.logNp - lr0) / 4;
  k.r0 = 1 << lr0;
  k.real_packed = mode == kLoadRealPacked ? 1 : 0;
  k.M = M;
  k.divP = make_fastdiv((uint32_t)k.P);
  return ADFFT_OK;
}

bool rq_split(const RqClass& k) { return (int64_t)k.P * k.Np > kRqTilePoints; }

struct RqLayout {
  std::vector<RqTile> tiles;
  std::vector<int> whole;           // signals of the whole tiles, tile after tile
  std::vector<int> nfft;            // per signal: its fft tiles (0: a whole signal)
  std::vector<long long> scratch;   // per signal: float2 offset of its U in the scratch area
  long long scratch_total = 0;
};

// Tile order: split signals (residues beyond one tile) largest first, each signal's fft tiles
// followed, at least `lag` tiles later (about one wave of resident CTAs, so that an unpack
// tile seldom waits for fft tiles still running), by its unpack tiles; then the whole tiles of
// each class, classes with the most work first.  An unpack tile waits only for fft tiles
// earlier in the queue, which never wait: no cycle.
void rq_layout(const std::vector<RqClass>& cls, const std::vector<std::vector<int64_t>>& members, int64_t count,
               int lag, RqLayout& L) {
  const size_t ncls = cls.size();
  L.tiles.clear();
  L.whole.clear();
  L.nfft.assign((size_t)count, 0);
  L.scratch.assign((size_t)count, 0);
  L.scratch_total = 0;
  std::vector<int> cls_of((size_t)count, -1);
  for (size_t c = 0; c < ncls; ++c)
    for (int64_t s : members[c]) cls_of[(size_t)s] = (int)c;
  std::vector<std::pair<int64_t, int64_t>> split;   // (-M, signal)
  for (int64_t s = 0; s < count; ++s) {
    const RqClass& k = cls[(size_t)cls_of[(size_t)s]];
    if (rq_split(k)) {
      L.scratch[(size_t)s] = L.scratch_total;
      L.scratch_total += (long long)k.P * k.Np;
      const int rpt = std::min(k.P, kRqTilePoints / k.Np);
      L.nfft[(size_t)s] = (k.P + rpt - 1) / rpt;
      split.push_back({-k.M, s});
    }
  }
  std::sort(split.begin(), split.end());
  auto unpack_tiles = [&](int64_t s) {
    const int c = cls_of[(size_t)s];
    const RqClass& k = cls[(size_t)c];
    const int jt = k.real_packed ? k.Mc / 2 + 1 : k.Mc;
    for (int j0 = 0; j0 < jt; j0 += kRqLeadersPerTile)
      L.tiles.push_back(RqTile{kRqUnpack, c, (int)s, j0, std::min(jt, j0 + kRqLeadersPerTile), 0});
  };
  std::vector<std::pair<size_t, int64_t>> pending;   // (tiles emitted after its fft tiles, signal)
  size_t next = 0;
  for (size_t i = 0; i < split.size(); ++i) {
    const int64_t s = split[i].second;
    const int c = cls_of[(size_t)s];
    const RqClass& k = cls[(size_t)c];
    const int rpt = std::min(k.P, kRqTilePoints / k.Np);
    for (int r = 0; r < k.P; r += rpt) L.tiles.push_back(RqTile{kRqFft, c, (int)s, r, std::min(rpt, k.P - r), 0});
    pending.push_back({L.tiles.size(), s});
    while (next < pending.size() && pending[next].first + (size_t)lag <= L.tiles.size())
      unpack_tiles(pending[next++].second);
  }
  while (next < pending.size()) unpack_tiles(pending[next++].second);
  std::vector<std::pair<int64_t, size_t>> corder;
  for (size_t c = 0; c < ncls; ++c) {
    const RqClass& k = cls[c];
    if (rq_split(k)) continue;
    const int64_t n = k.real_packed ? 2 * (int64_t)k.Nc : (int64_t)k.Nc;
    corder.push_back({-(int64_t)members[c].size() * (k.M + n), c});
  }
  std::sort(corder.begin(), corder.end());
  for (auto& co : corder) {
    const size_t c = co.second;
    const int per = whole_group(cls[c]);
    for (size_t i = 0; i < members[c].size(); i += per) {
      const int cnt = (int)std::min<size_t>(per, members[c].size() - i);
      L.tiles.push_back(RqTile{kRqWhole, (int)c, (int)L.whole.size(), 0, cnt, 0});
      for (int w = 0; w < cnt; ++w) L.whole.push_back((int)members[c][i + w]);
    }
  }
}

// Build the tile queue of the persistent form from the shape classes' fold geometry.
// Returns ADFFT_OK (p.rq_ok set), ADFFT_ERR_UNSUPPORTED_SIZE when a class has no
// single-CTA fold geometry (then only the class graph serves the plan), or an error.
int build_queue(Plan& p, const std::vector<std::vector<int64_t>>& members) {
  const size_t ncls = p.r_sub.size();
  std::vector<RqClass> cls(ncls);
  std::vector<float> tables;
  int tw_max = 0;
  size_t buf_max = 0;
  for (size_t c = 0; c < ncls; ++c) {
    const Plan& q = p.r_sub[c]->p;
    if (q.dbl) return ADFFT_ERR_UNSUPPORTED_SIZE;
    int mode;
    int64_t Nc, Mc;
    core_shape(q, &mode, &Nc, &Mc);
    RqClass& k = cls[c];
    const int rcg = rq_geometry(mode, Nc, Mc, q.M, k);
    if (rcg != ADFFT_OK) return rcg;
    k.scale = (float)q.scale;
    int bits, lo_n, hi_n;
    std::vector<float> t = twiddle_table_f32(k.Mt, &bits, &lo_n, &hi_n);
    k.tw_bits = bits;
    k.tw_lo_n = lo_n;
    k.tw_hi_n = hi_n;
    k.tw_off = (long long)(tables.size() / 2);
    tables.insert(tables.end(), t.begin(), t.end());
    tw_max = std::max(tw_max, lo_n + hi_n);
    // regions a tile holds: R of the residues of a split signal, or the P residues of each
    // signal of a whole tile
    const int rpt = rq_split(k) ? std::min(k.P, kRqTilePoints / k.Np) : whole_group(k) * k.P;
    buf_max = std::max(buf_max, (size_t)rpt * (size_t)k.region * 8);
  }
  const size_t smem = (((size_t)tw_max * 8 + 15) & ~size_t(15)) + buf_max;
  if (smem > 200 * 1024) return ADFFT_ERR_UNSUPPORTED_SIZE;
  cudaError_t e = cudaFuncSetAttribute(ragged_queue_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0, sms = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ragged_queue_kernel<0>, kRqThreads, smem);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p.device);
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return ADFFT_ERR_UNSUPPORTED_SIZE;
  }
  const int resident = per_sm * sms;

  RqLayout lay;
  rq_layout(cls, members, p.r_count, resident, lay);
  const std::vector<RqTile>& tiles = lay.tiles;
  const std::vector<int>& whole = lay.whole;
  const long long scratch = lay.scratch_total;
  std::vector<RqSignal> sigs((size_t)p.r_count);
  for (int64_t s = 0; s < p.r_count; ++s) {
    RqSignal& g = sigs[(size_t)s];
    memset(&g, 0, sizeof(g));
    g.in_bytes = p.r_in_off[(size_t)s] * (long long)p.in_elem;
    g.out_bin = p.r_out_off[(size_t)s];
    g.scratch = lay.scratch[(size_t)s];
    g.nfft = lay.nfft[(size_t)s];
  }
  if (tiles.size() > 0x7fffffff || p.r_count > 0x7ffffffe) return ADFFT_ERR_UNSUPPORTED_SIZE;

  RqArgs& a = p.rq;
  memset(&a, 0, sizeof(a));
  RqTile* d_tiles = nullptr;
  RqClass* d_cls = nullptr;
  RqSignal* d_sigs = nullptr;
  int* d_whole = nullptr;
  float* d_tab = nullptr;
  int rc;
  if ((rc = rq_upload(p, tiles, &d_tiles)) != ADFFT_OK) return rc;
  if ((rc = rq_upload(p, cls, &d_cls)) != ADFFT_OK) return rc;
  if ((rc = rq_upload(p, sigs, &d_sigs)) != ADFFT_OK) return rc;
  if ((rc = rq_upload(p, whole, &d_whole)) != ADFFT_OK) return rc;
  if ((rc = rq_upload(p, tables, &d_tab)) != ADFFT_OK) return rc;
  void* d_scr = nullptr;
  void* d_cnt = nullptr;
  void* d_st = nullptr;
  e = cudaMalloc(&d_scr, std::max<size_t>(16, (size_t)scratch * 8));
  if (e == cudaSuccess) p.rq_bufs.push_back(d_scr);
  if (e == cudaSuccess) e = cudaMalloc(&d_cnt, (size_t)(p.r_count + 1) * sizeof(int));
  if (e == cudaSuccess) p.rq_bufs.push_back(d_cnt);
  if (e == cudaSuccess) e = cudaMalloc(&d_st, sizeof(int));
  if (e == cudaSuccess) p.rq_bufs.push_back(d_st);
  if (e == cudaSuccess) e = cudaMemset(d_st, 0, sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status_of(e);
  }
  a.tiles = d_tiles;
  a.ntiles = (int)tiles.size();
  a.classes = d_cls;
  a.sigs = d_sigs;
  a.whole_sigs = d_whole;
  a.tables = reinterpret_cast<const float2*>(d_tab);
  a.scratch = static_cast<float2*>(d_scr);
  a.counters = static_cast<int*>(d_cnt);
  a.status = static_cast<int*>(d_st);
  a.tw_max = tw_max;
  a.wait_limit = kWaitLimitCycles;
  p.rq_smem = smem;
  // every CTA resident at once: a CTA waiting in an unpack tile never waits for one that
  // has not started
  p.rq_grid = std::max(1, std::min(resident, (int)tiles.size()));
  p.rq_ok = true;
  return ADFFT_OK;
}

void release_queue(Plan& p) {
  for (void* d : p.rq_bufs)
    if (d) cudaFree(d);
  p.rq_bufs.clear();
  p.rq_ok = p.rq_on = false;
}

int launch_queue(Plan& p, const void* in, void* out, cudaStream_t s) {
  RqArgs a = p.rq;
  a.in = in;
  a.out = out;
  cudaError_t e = cudaMemsetAsync(a.counters, 0, (size_t)(p.r_count + 1) * sizeof(int), s);
  if (e == cudaSuccess) {
    ragged_queue_kernel<0><<<p.rq_grid, kRqThreads, p.rq_smem, s>>>(a);
    e = cudaGetLastError();
  }
  return cuda_status_of(e);
}

}  // namespace

// The queue layout of a ragged batch from its shapes alone (host only, no CUDA call): the shape
// classes are formed and ordered as a ragged plan forms them ((N, M) in increasing order).
int ragged_queue_layout(const int64_t* N, const double* alpha, int64_t count, int dtype, int lag,
                        int32_t* tiles_out, int64_t tile_capacity, int64_t* ntiles, int64_t* whole_out,
                        int64_t whole_capacity, int64_t* nwhole) {
  if (!N || !alpha || count < 0 || lag < 0 || !ntiles || !nwhole) return ADFFT_ERR_INVALID_ARG;
  if (dtype != ADFFT_R32 && dtype != ADFFT_C64) return ADFFT_ERR_NOT_SUPPORTED;
  std::map<std::pair<int64_t, int64_t>, std::vector<int64_t>> classes;
  for (int64_t i = 0; i < count; ++i) {
    const double a = alpha[i];
    if (N[i] < 1) return ADFFT_ERR_INVALID_ARG;
    if (!(a > 0.0) || !isfinite(a)) return ADFFT_ERR_INVALID_ALPHA;
    const double Md = a * (double)N[i];
    const double Mr = nearbyint(Md);
    if (fabs(Md - Mr) > 1e-9 * Md || Mr < 1.0) return ADFFT_ERR_INVALID_ALPHA;
    classes[{N[i], (int64_t)Mr}].push_back(i);
  }
  std::vector<RqClass> cls;
  std::vector<std::vector<int64_t>> members;
  for (auto& kv : classes) {
    const int64_t n = kv.first.first, m = kv.first.second;
    int mode;
    int64_t Nc, Mc;
    if (dtype == ADFFT_C64) {
      mode = kLoadComplex;
      Nc = n;
      Mc = m;
    } else if (n % 2 == 0 && m % 2 == 0) {
      mode = kLoadRealPacked;
      Nc = n / 2;
      Mc = m / 2;
    } else {
      return ADFFT_ERR_NOT_SUPPORTED;
    }
    RqClass k;
    if (rq_geometry(mode, Nc, Mc, m, k) != ADFFT_OK) return ADFFT_ERR_NOT_SUPPORTED;
    cls.push_back(k);
    members.push_back(kv.second);
  }
  RqLayout lay;
  rq_layout(cls, members, count, lag, lay);
  *ntiles = (int64_t)lay.tiles.size();
  *nwhole = (int64_t)lay.whole.size();
  if (tiles_out) {
    if (tile_capacity < *ntiles) return ADFFT_ERR_INVALID_ARG;
    for (size_t i = 0; i < lay.tiles.size(); ++i) {
      const RqTile& t = lay.tiles[i];
      int32_t* o = tiles_out + 5 * i;
      o[0] = t.kind;
      o[1] = t.cls;
      o[2] = t.sig;
      o[3] = t.a0;
      o[4] = t.a1;
    }
  }
  if (whole_out) {
    if (whole_capacity < *nwhole) return ADFFT_ERR_INVALID_ARG;
    for (size_t i = 0; i < lay.whole.size(); ++i) whole_out[i] = lay.whole[i];
  }
  return ADFFT_OK;
}

int ragged_set_form(Plan& p, int form) {
  if (form == ADFFT_RAGGED_QUEUE && !p.rq_ok) return ADFFT_ERR_NOT_SUPPORTED;
  const bool on = form == ADFFT_RAGGED_QUEUE;
  if (on != p.rq_on) {
    p.rq_on = on;
    destroy_graphs(p);
  }
  return ADFFT_OK;
}

int ragged_queue_status(Plan& p, int* status) {
  *status = 0;
  if (!p.rq_ok) return ADFFT_OK;
  cudaError_t e = cudaMemcpy(status, p.rq.status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && *status != 0) e = cudaMemset(p.rq.status, 0, sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status_of(e);
  }
  return ADFFT_OK;
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
  // packed real classes read their samples in pairs (8-byte loads): a real signal with even N
  // and M must start at an even sample offset
  if (p.real) {
    for (int64_t i = 0; i < count; ++i) {
      if (N[i] % 2 == 0 && Ms[(size_t)i] % 2 == 0 && (p.r_in_off[(size_t)i] % 2) != 0) {
        delete h;
        *err = ADFFT_ERR_NOT_SUPPORTED;
        return nullptr;
      }
    }
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
  std::vector<std::vector<int64_t>> members;
  for (auto& kv : classes) members.push_back(kv.second);
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
  // the persistent queue form, where every class has a single-CTA fold geometry
  if (count > 0) {
    const int rc = build_queue(p, members);
    if (rc != ADFFT_OK && rc != ADFFT_ERR_UNSUPPORTED_SIZE) return bail(rc);
    if (rc != ADFFT_OK) release_queue(p);
  }
  return h;
}

int ragged_execute(Plan& p, const void* in, void* out, cudaStream_t s, int which) {
  if (p.r_count == 0) return ADFFT_OK;
  if (which == 1) {
    // chirp-z classes set up their adjoint's tables (device allocations) outside the capture
    for (auto* sp : p.r_sub) {
      if (sp->p.fold_ok || sp->p.tp_ok) continue;
      const int rc = setup_bluestein_adjoint(sp->p);
      if (rc != ADFFT_OK) return rc == ADFFT_ERR_UNSUPPORTED_SIZE ? ADFFT_ERR_NOT_SUPPORTED : rc;
    }
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
