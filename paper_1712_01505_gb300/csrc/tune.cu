// Launch-shape autotuner for the stencil kernels.
//
// On the first launch of a key (kernel, lattice, precision, right-hand sides)
// every candidate shape is timed with CUDA events on the caller's stream (about
// 2 ms of launches per candidate, twice, interleaved); the fastest is cached for
// the life of the process and,
// when QCD_TUNECACHE names a file, appended to it and read back by later
// processes.  Candidates must be idempotent (out-of-place stencils).  While a
// stream is being captured into a CUDA graph nothing can be timed, so an
// unknown key then falls back to the first candidate without caching it; the
// same when the kernels' stop word (the solver's) is raised, which would make
// every candidate an empty launch.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "internal.h"

namespace qcd {

namespace {
std::mutex g_mu;
std::map<std::string, LaunchCfg> g_cache;
bool g_loaded = false;
int g_mode = 1;

const char* cache_path() {
  const char* p = getenv("QCD_TUNECACHE");
  return (p && *p) ? p : nullptr;
}

void load_cache_locked() {
  if (g_loaded) return;
  g_loaded = true;
  const char* path = cache_path();
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char line[512];
  while (fgets(line, sizeof line, f)) {
    // format: <key>\t<block>\t<tile>
    char* t1 = strchr(line, '\t');
    if (!t1) continue;
    *t1 = 0;
    int b = 0, t = 0;
    if (sscanf(t1 + 1, "%d\t%d", &b, &t) == 2 && b > 0 && t != 0) g_cache[line] = {b, t};
  }
  fclose(f);
}

void append_cache(const std::string& key, const LaunchCfg& c) {
  const char* path = cache_path();
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s\t%d\t%d\n", key.c_str(), c.block, c.tile);
  fclose(f);
}
}  // namespace

bool tuning_enabled() { return g_mode != 0; }
void set_tuning(int mode) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_mode = mode;
}

bool pdl_enabled() {
  static const bool on = [] {
    const char* e = getenv("QCD_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

LaunchCfg tune(const std::string& key, const std::vector<LaunchCfg>& cands,
               void (*run)(void* ctx, const LaunchCfg& cfg), void* ctx, cudaStream_t st,
               bool allow_timing, const int* stop) {
  if (cands.empty()) raise(QCD_ERR_ARG, "tune: no candidates for %s", key.c_str());
  {
    std::lock_guard<std::mutex> lk(g_mu);
    load_cache_locked();
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
      for (const auto& c : cands)
        if (c.block == it->second.block && c.tile == it->second.tile) return it->second;
    }
    if (g_mode == 0 || !allow_timing) return cands[0];
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  QCD_CK(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone || cands.size() == 1) return cands[0];
  if (stop) {
    // a kernel whose stop word is raised returns at once: timing it would time empty
    // launches, so an unknown key then takes the first candidate without caching it
    int v = 0;
    QCD_CK(cudaMemcpyAsync(&v, stop, sizeof v, cudaMemcpyDeviceToHost, st));
    QCD_CK(cudaStreamSynchronize(st));
    if (v != 0) return cands[0];
  }

  cudaEvent_t e0, e1;
  QCD_CK(cudaEventCreate(&e0));
  QCD_CK(cudaEventCreate(&e1));
  // every candidate: one warm-up launch, then two passes over all candidates
  // (interleaved, so that clock or thermal drift does not favour one), each
  // timing enough back-to-back launches to cover about 2 ms; a candidate's time
  // is its smaller per-launch average
  auto time_reps = [&](const LaunchCfg& c, int reps) {
    QCD_CK(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r) run(ctx, c);
    QCD_CK(cudaEventRecord(e1, st));
    QCD_CK(cudaEventSynchronize(e1));
    note_launches(reps - 1);
    QCD_LAUNCH_CK();
    float ms = 0;
    QCD_CK(cudaEventElapsedTime(&ms, e0, e1));
    return ms / reps;
  };
  std::vector<int> reps(cands.size());
  std::vector<float> best_of(cands.size(), 1e30f);
  for (size_t i = 0; i < cands.size(); ++i) {
    run(ctx, cands[i]);  // warm-up
    QCD_LAUNCH_CK();
    const float once = time_reps(cands[i], 1);
    reps[i] = once > 0.f ? (int)std::min(50.f, std::max(3.f, 2.0f / once)) : 50;
  }
  for (int pass = 0; pass < 2; ++pass)
    for (size_t i = 0; i < cands.size(); ++i) best_of[i] = std::min(best_of[i], time_reps(cands[i], reps[i]));
  LaunchCfg best = cands[0];
  float best_ms = 1e30f;
  for (size_t i = 0; i < cands.size(); ++i) {
    if (getenv("QCD_TUNE_VERBOSE"))
      fprintf(stderr, "[qcd tune]   %s block %d tile %d: %.4f ms\n", key.c_str(), cands[i].block, cands[i].tile,
              best_of[i]);
    if (best_of[i] < best_ms) {
      best_ms = best_of[i];
      best = cands[i];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (getenv("QCD_TUNE_VERBOSE"))
    fprintf(stderr, "[qcd tune] %s -> block %d tile %d (%.4f ms per launch)\n", key.c_str(), best.block,
            best.tile, best_ms);
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[key] = best;
  append_cache(key, best);
  return best;
}

}  // namespace qcd
