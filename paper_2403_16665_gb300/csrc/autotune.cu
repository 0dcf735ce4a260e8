// Autotuner: times the candidate launch shapes of a plan's forward transform
// and keeps the fastest, with a process-wide cache keyed by GPU model, driver
// and sizes (saved to and loaded from a small JSON file).
//
// Candidates of the fold form: every sub-FFT length Np (a power of two dividing
// gcd(Mc, Nc), down to 64 while the fold factor q = Nc/Np stays within
// kTuneMaxFold), every cluster size that divides P = Mc/Np and holds P/C
// residue FFTs in one CTA's shared memory, with and without input staging,
// with a resident-size (persistent) grid or one cluster per signal.
// The two-pass form is a further candidate where it applies.  Every candidate
// is a configuration the same kernels take at any size: tuning changes which
// shape runs, never what is computed (results agree to rounding).
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "adfft_internal.h"

namespace adfft {

namespace {

struct Key {
  std::string device;
  int64_t N, M, batch;
  int dtype, precision;
  bool operator<(const Key& o) const {
    return std::tie(device, N, M, batch, dtype, precision) <
           std::tie(o.device, o.N, o.M, o.batch, o.dtype, o.precision);
  }
};

struct Entry {
  int algo = ADFFT_ALGO_FOLD;   // ADFFT_ALGO_FOLD or ADFFT_ALGO_FOUR_STEP
  FoldChoice fold{};
  int64_t tp_a = 0;             // four-step: length A of the pass-1 transforms (0: default rule)
  double ms = 0.0;              // time per forward transform when tuned
};

std::mutex g_mu;
std::map<Key, Entry> g_cache;
std::map<int, std::string> g_device_ids;

// "<name>|sm_<cc>|cuda-driver <version>" of a device (looked up once per device).
std::string device_id(int device) {
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_device_ids.find(device);
    if (it != g_device_ids.end()) return it->second;
  }
  cudaDeviceProp prop;
  std::string id = "unknown";
  if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) {
    int drv = 0;
    if (cudaDriverGetVersion(&drv) != cudaSuccess) drv = 0;
    char buf[400];
    snprintf(buf, sizeof buf, "%s|sm_%d%d|cuda-driver %d", prop.name, prop.major, prop.minor, drv);
    id = buf;
  } else {
    cudaGetLastError();
  }
  std::lock_guard<std::mutex> lk(g_mu);
  g_device_ids[device] = id;
  return id;
}

Key key_of(const Plan& p, const std::string& dev) {
  return Key{dev, p.N, p.M, p.batch, p.dtype, p.precision};
}

// Apply an entry to a plan; on failure the plan keeps its current shape.
int apply(Plan& p, const Entry& e) {
  if (e.algo == ADFFT_ALGO_FOUR_STEP) {
    if (p.tp_ok && p.tp_A != e.tp_a && e.tp_a > 0) release_twopass(p);
    p.tp_force_A = e.tp_a;
    int rc = setup_twopass(p);
    if (rc == ADFFT_OK) rc = prepare_precision(p);
    if (rc != ADFFT_OK) return rc;
    p.algo = p.auto_algo = ADFFT_ALGO_FOUR_STEP;
    return ADFFT_OK;
  }
  int rc = setup_fold(p, &e.fold);
  if (rc == ADFFT_OK) rc = prepare_precision(p);
  if (rc != ADFFT_OK) return rc;
  p.algo = p.auto_algo = ADFFT_ALGO_FOLD;
  return ADFFT_OK;
}

std::vector<FoldChoice> fold_candidates(const Plan& p) {
  std::vector<FoldChoice> out;
  if (p.dbl && p.precision != ADFFT_PREC_NATIVE) return out;
  int mode;
  int64_t Nc, Mc;
  core_shape(p, &mode, &Nc, &Mc);
  const int64_t g = plan_gcd(Mc, Nc);
  const int64_t np0 = g & -g;
  const int vals = fused_values_per_thread(p.dbl) * 512;   // complex values one CTA holds
  for (int64_t np = np0; np >= 1; np /= 2) {
    if (np != np0 && (Nc / np > kTuneMaxFold || np < 64)) break;
    const int64_t P = Mc / np;
    for (int c = 1; c <= kFoldMaxCluster && c <= P; ++c) {
      if (P % c || (P / c) * np > vals) continue;
      for (int st : {1, 0})
        for (int grid : {0, -1}) out.push_back(FoldChoice{np, c, st, grid});
      // bulk push exchange (one residue per CTA; configure rejects shapes it has no kernel for)
      if (c == P && !p.dbl && mode == kLoadRealPacked && !p.half) out.push_back(FoldChoice{np, c, 2, 0});
    }
  }
  return out;
}

// Mean time per forward launch of the plan as configured now (ms), or a negative status;
// with xb != nullptr each step is a forward and the adjoint of its spectrum into xb.
double time_forward(Plan& p, const void* in, void* out, void* xb, cudaStream_t s, int iters, cudaEvent_t e0,
                    cudaEvent_t e1) {
  auto step = [&]() {
    int r = launch_forward(p, in, out, s);
    if (r == ADFFT_OK && xb) r = launch_adjoint(p, out, xb, s);
    return r;
  };
  int rc = step();   // warm-up (also first-touch of tables)
  if (rc != ADFFT_OK) return (double)rc;
  if (cudaEventRecord(e0, s) != cudaSuccess) return (double)ADFFT_ERR_CUDA;
  for (int i = 0; i < iters && rc == ADFFT_OK; ++i) rc = step();
  if (rc != ADFFT_OK) return (double)rc;
  if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
    cudaGetLastError();
    return (double)ADFFT_ERR_CUDA;
  }
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
    cudaGetLastError();
    return (double)ADFFT_ERR_CUDA;
  }
  return (double)ms / iters;
}

int tune_uniform(Plan& p, const void* in, void* out, void* xb, cudaStream_t s, int iters, cudaEvent_t e0,
                 cudaEvent_t e1) {
  if (p.algo == ADFFT_ALGO_BLUESTEIN && !p.fold_ok && !p.tp_ok) return ADFFT_OK;   // nothing to choose
  const bool had_tp = p.tp_ok;
  const Entry start{p.algo == ADFFT_ALGO_FOUR_STEP ? ADFFT_ALGO_FOUR_STEP : ADFFT_ALGO_FOLD, p.fold_choice, p.tp_A,
                    0.0};
  const int saved_algo = p.algo;
  // a failed timing run leaves the plan as it was before tuning (then reports the error)
  auto restore = [&](int err) {
    apply(p, start);
    p.algo = saved_algo;
    return err;
  };
  Entry best{};
  best.ms = -1.0;
  std::vector<Entry> timed;   // every candidate that ran, for the final runoff
  for (const FoldChoice& c : fold_candidates(p)) {
    if (setup_fold(p, &c) != ADFFT_OK) continue;   // does not fit (or cannot launch): skip
    if (prepare_precision(p) != ADFFT_OK) continue;
    p.algo = ADFFT_ALGO_FOLD;
    const double ms = time_forward(p, in, out, xb, s, iters, e0, e1);
    if (ms < 0.0) return restore((int)ms);
    timed.push_back(Entry{ADFFT_ALGO_FOLD, p.fold_choice, 0, ms});
    if (best.ms < 0.0 || ms < best.ms) best = timed.back();
  }
  // the four-step form with every split Nc = A B it takes (B up to 2048)
  {
    int mode;
    int64_t Nc, Mc;
    core_shape(p, &mode, &Nc, &Mc);
    const bool pow2 = Nc >= 4 && (Nc & (Nc - 1)) == 0 && mode != kLoadRealPlain && !p.half;
    for (int64_t A = pow2 ? Nc / 2 : 0; A >= 16 && Nc / A <= 2048; A >>= 1) {
      if (p.tp_ok) release_twopass(p);
      p.tp_force_A = A;
      const int rc_tp = setup_twopass(p);
      if (rc_tp == ADFFT_OK && prepare_precision(p) == ADFFT_OK) {
        p.algo = ADFFT_ALGO_FOUR_STEP;
        const double ms = time_forward(p, in, out, xb, s, iters, e0, e1);
        if (ms < 0.0) {
          p.tp_force_A = 0;
          return restore((int)ms);
        }
        timed.push_back(Entry{ADFFT_ALGO_FOUR_STEP, FoldChoice{}, A, ms});
        if (best.ms < 0.0 || ms < best.ms) best = timed.back();
      } else if (rc_tp != ADFFT_OK && rc_tp != ADFFT_ERR_UNSUPPORTED_SIZE) {
        release_twopass(p);   // a partial set-up (allocation failure): drop it, tuning goes on
      } else if (rc_tp != ADFFT_OK) {
        release_twopass(p);
      }
    }
    p.tp_force_A = 0;
  }
  // runoff: the candidates within 5 % of the best (at most 3) are timed again in three
  // alternating rounds and the smallest time of each decides, so that one noisy sweep
  // timing does not pick a shape that is slower in steady state
  if (best.ms > 0.0) {
    std::stable_sort(timed.begin(), timed.end(), [](const Entry& x, const Entry& y) { return x.ms < y.ms; });
    std::vector<Entry> top;
    for (const Entry& e : timed)
      if (e.ms <= best.ms * 1.05 && top.size() < 3) top.push_back(e);
    if (top.size() > 1) {
      std::vector<double> tmin(top.size(), -1.0);
      for (int round = 0; round < 3; ++round)
        for (size_t i = 0; i < top.size(); ++i) {
          if (apply(p, top[i]) != ADFFT_OK) continue;
          const double ms = time_forward(p, in, out, xb, s, iters, e0, e1);
          if (ms < 0.0) return restore((int)ms);
          if (tmin[i] < 0.0 || ms < tmin[i]) tmin[i] = ms;
        }
      size_t bi = 0;
      for (size_t i = 1; i < top.size(); ++i)
        if (tmin[i] >= 0.0 && (tmin[bi] < 0.0 || tmin[i] < tmin[bi])) bi = i;
      if (tmin[bi] >= 0.0) {
        best = top[bi];
        best.ms = tmin[bi];
      }
    }
  }
  if (best.ms < 0.0) {
    p.algo = saved_algo;
    return apply(p, start) == ADFFT_OK ? ADFFT_OK : ADFFT_ERR_UNSUPPORTED_SIZE;
  }
  int rc = apply(p, best);
  if (rc != ADFFT_OK) return rc;
  if (best.algo == ADFFT_ALGO_FOLD && !had_tp && p.tp_ok) release_twopass(p);   // workspace not needed
  p.tuned = true;
  const std::string dev = device_id(p.device);
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[key_of(p, dev)] = best;
  return ADFFT_OK;
}

// ---- JSON file: {"adfft_autotune": 1, "entries": [{...}, ...]} -------------

void json_string(std::string& o, const std::string& v) {
  o += '"';
  for (char ch : v) {
    if (ch == '"' || ch == '\\') {
      o += '\\';
      o += ch;
    } else if ((unsigned char)ch < 0x20) {
      char b[8];
      snprintf(b, sizeof b, "\\u%04x", (unsigned)(unsigned char)ch);
      o += b;
    } else {
      o += ch;
    }
  }
  o += '"';
}

struct Parser {
  const char* s;
  const char* e;
  bool ok = true;
  void ws() {
    while (s < e && (*s == ' ' || *s == '\n' || *s == '\r' || *s == '\t')) ++s;
  }
  bool eat(char c) {
    ws();
    if (s < e && *s == c) {
      ++s;
      return true;
    }
    return false;
  }
  bool str(std::string& out) {
    ws();
    if (s >= e || *s != '"') return ok = false;
    ++s;
    out.clear();
    while (s < e && *s != '"') {
      if (*s == '\\') {
        if (++s >= e) return ok = false;
        if (*s == 'u') {
          if (e - s < 5) return ok = false;
          char hex[5] = {s[1], s[2], s[3], s[4], 0};
          char* endp = nullptr;
          const long v = strtol(hex, &endp, 16);
          if (endp != hex + 4 || v > 0x7f) return ok = false;
          out += (char)v;
          s += 5;
          continue;
        }
        out += *s++;
      } else {
        out += *s++;
      }
    }
    if (s >= e) return ok = false;
    ++s;
    return true;
  }
  bool num(double& v) {
    ws();
    char buf[64];
    size_t n = 0;
    while (s < e && n < sizeof(buf) - 1 && (strchr("+-.eE", *s) || (*s >= '0' && *s <= '9'))) buf[n++] = *s++;
    buf[n] = 0;
    if (!n) return ok = false;
    char* endp = nullptr;
    v = strtod(buf, &endp);
    if (endp != buf + n) return ok = false;
    return true;
  }
};

bool parse_entry(Parser& ps, Key& k, Entry& en) {
  if (!ps.eat('{')) return false;
  bool have_dev = false;
  int have = 0;
  if (ps.eat('}')) return false;
  do {
    std::string name;
    if (!ps.str(name) || !ps.eat(':')) return false;
    if (name == "device") {
      if (!ps.str(k.device)) return false;
      have_dev = true;
      continue;
    }
    double v;
    if (!ps.num(v)) return false;
    if (name == "N") k.N = (int64_t)v, have |= 1;
    else if (name == "M") k.M = (int64_t)v, have |= 2;
    else if (name == "batch") k.batch = (int64_t)v, have |= 4;
    else if (name == "dtype") k.dtype = (int)v, have |= 8;
    else if (name == "precision") k.precision = (int)v, have |= 16;
    else if (name == "algo") en.algo = (int)v, have |= 32;
    else if (name == "fft_len") en.fold.np = (int64_t)v, have |= 64;
    else if (name == "cluster") en.fold.cluster = (int)v, have |= 128;
    else if (name == "staged") en.fold.stage = (int)v, have |= 256;
    else if (name == "grid") en.fold.grid = (int)v;
    else if (name == "four_step_a") en.tp_a = (int64_t)v;
    else if (name == "ms") en.ms = v;
  } while (ps.eat(','));
  if (!ps.eat('}')) return false;
  if (!have_dev || have != 511) return false;
  if (en.algo != ADFFT_ALGO_FOLD && en.algo != ADFFT_ALGO_FOUR_STEP) return false;
  if (en.fold.stage < 0 || en.fold.stage > 2) return false;
  if (en.fold.grid < -1 || en.tp_a < 0) return false;
  return true;
}

}  // namespace

void autotune_apply_cached(Plan& p) {
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_cache.empty()) return;
  }
  if (p.ragged || p.algo == ADFFT_ALGO_BLUESTEIN) return;
  const std::string dev = device_id(p.device);
  Entry e;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key_of(p, dev));
    if (it == g_cache.end()) return;
    e = it->second;
  }
  if (apply(p, e) == ADFFT_OK) p.tuned = true;   // else the default shape stays
}

int autotune_plan(Plan& p, const void* in, void* out, cudaStream_t s, int iters, int flags) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    return ADFFT_ERR_CUDA;
  }
  // forward + adjoint: the adjoint writes into a temporary buffer of the input's size
  void* xb = nullptr;
  if (flags & ADFFT_TUNE_WITH_ADJOINT) {
    const cudaError_t e = cudaMalloc(&xb, std::max<size_t>(16, p.in_bytes()));
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return e == cudaErrorMemoryAllocation ? ADFFT_ERR_OOM : ADFFT_ERR_CUDA;
    }
  }
  int rc = ADFFT_OK;
  if (p.ragged) {
    for (auto* sp : p.r_sub) {
      rc = tune_uniform(sp->p, in, out, xb, s, iters, e0, e1);
      if (rc != ADFFT_OK) break;
    }
    ragged_invalidate(p);   // the next execute captures the new shapes
  } else {
    rc = tune_uniform(p, in, out, xb, s, iters, e0, e1);
  }
  if (xb) {
    cudaStreamSynchronize(s);
    cudaFree(xb);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // namespace adfft

using adfft::Plan;

extern "C" {

int adfft_plan_autotune(adfft_plan_t plan, const void* d_in, void* d_out, void* stream, int iters, int flags) {
  if (!plan || !d_in || !d_out || iters < 0 || iters > 100 || (flags & ~ADFFT_TUNE_WITH_ADJOINT))
    return ADFFT_ERR_INVALID_ARG;
  Plan& p = plan->p;
  if (((uintptr_t)d_in & 15u) || ((uintptr_t)d_out & 15u)) return ADFFT_ERR_MISALIGNED;
  const size_t ni = p.in_bytes(), no = p.out_bytes();
  const uintptr_t a = (uintptr_t)d_in, b = (uintptr_t)d_out;
  if (ni && no && a < b + no && b < a + ni) return ADFFT_ERR_OVERLAP;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    cudaGetLastError();
    return ADFFT_ERR_CUDA;
  }
  if (cs != cudaStreamCaptureStatusNone) return ADFFT_ERR_NOT_SUPPORTED;
  return adfft::autotune_plan(p, d_in, d_out, s, iters ? iters : 3, flags);
}

int adfft_autotune_save(const char* path) {
  using namespace adfft;
  if (!path) return ADFFT_ERR_INVALID_ARG;
  std::string o = "{\"adfft_autotune\": 1, \"entries\": [";
  {
    std::lock_guard<std::mutex> lk(g_mu);
    bool first = true;
    for (const auto& kv : g_cache) {
      const Key& k = kv.first;
      const Entry& e = kv.second;
      o += first ? "\n  {" : ",\n  {";
      first = false;
      o += "\"device\": ";
      json_string(o, k.device);
      char buf[512];
      snprintf(buf, sizeof buf,
               ", \"N\": %lld, \"M\": %lld, \"batch\": %lld, \"dtype\": %d, \"precision\": %d, "
               "\"algo\": %d, \"fft_len\": %lld, \"cluster\": %d, \"staged\": %d, \"grid\": %d, "
               "\"four_step_a\": %lld, \"ms\": %.6g}",
               (long long)k.N, (long long)k.M, (long long)k.batch, k.dtype, k.precision, e.algo,
               (long long)e.fold.np, e.fold.cluster, e.fold.stage == 2 ? 2 : (e.fold.stage == 1 ? 1 : 0), e.fold.grid, (long long)e.tp_a,
               e.ms);
      o += buf;
    }
  }
  o += "\n]}\n";
  FILE* f = fopen(path, "wb");
  if (!f) return ADFFT_ERR_INVALID_ARG;
  const bool ok = fwrite(o.data(), 1, o.size(), f) == o.size();
  return (fclose(f) == 0 && ok) ? ADFFT_OK : ADFFT_ERR_INVALID_ARG;
}

int adfft_autotune_load(const char* path) {
  using namespace adfft;
  if (!path) return ADFFT_ERR_INVALID_ARG;
  FILE* f = fopen(path, "rb");
  if (!f) return ADFFT_ERR_INVALID_ARG;
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof buf, f)) > 0) {
    text.append(buf, n);
    if (text.size() > (64u << 20)) {
      fclose(f);
      return ADFFT_ERR_INVALID_ARG;
    }
  }
  fclose(f);
  Parser ps{text.data(), text.data() + text.size()};
  std::vector<std::pair<Key, Entry>> got;
  if (!ps.eat('{')) return ADFFT_ERR_INVALID_ARG;
  bool have_tag = false, have_entries = false;
  do {
    std::string name;
    if (!ps.str(name) || !ps.eat(':')) return ADFFT_ERR_INVALID_ARG;
    if (name == "adfft_autotune") {
      double v;
      if (!ps.num(v) || v != 1.0) return ADFFT_ERR_INVALID_ARG;
      have_tag = true;
    } else if (name == "entries") {
      if (!ps.eat('[')) return ADFFT_ERR_INVALID_ARG;
      if (!ps.eat(']')) {
        do {
          Key k{};
          Entry e{};
          if (!parse_entry(ps, k, e)) return ADFFT_ERR_INVALID_ARG;
          got.push_back({k, e});
        } while (ps.eat(','));
        if (!ps.eat(']')) return ADFFT_ERR_INVALID_ARG;
      }
      have_entries = true;
    } else {
      return ADFFT_ERR_INVALID_ARG;
    }
  } while (ps.eat(','));
  if (!ps.eat('}') || !have_tag || !have_entries || !ps.ok) return ADFFT_ERR_INVALID_ARG;
  ps.ws();
  if (ps.s != ps.e) return ADFFT_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& kv : got) g_cache[kv.first] = kv.second;
  return ADFFT_OK;
}

int adfft_autotune_clear(void) {
  std::lock_guard<std::mutex> lk(adfft::g_mu);
  adfft::g_cache.clear();
  return ADFFT_OK;
}

}  // extern "C"
