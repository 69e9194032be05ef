// Launch-shape autotuner: times each candidate once per problem key and caches the winner.
//
// The first call with a new (kernel, dtype, parity, dagger, volume, nrhs) key runs every
// candidate shape on the caller's own arguments (one warm-up and three timed launches
// each, CUDA events on the caller's stream) and keeps the fastest; later calls reuse the
// choice.  Calls made while the stream is being captured into a graph never tune (they use
// the default shape).  WMG_DSLASH_VARIANT=<i> in the environment forces a shape.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <tuple>

#include "common.cuh"
#include "internal.h"

namespace wmg {

namespace {
typedef std::tuple<int, int, int, int, int> Key;
std::map<Key, std::pair<int, float>> g_cache;
std::mutex g_mu;
std::string g_report;
}  // namespace

int tuned_variant(int dtype, int parity, int dagger, int V, int nrhs, cudaStream_t st, int nvar,
                  const std::function<void(int)>& run) {
  static int forced = [] {
    const char* e = std::getenv("WMG_DSLASH_VARIANT");
    return e ? std::atoi(e) : -1;
  }();
  if (forced >= 0 && forced < nvar) return forced;
  Key key(dtype, parity, dagger, V, nrhs);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) return it->second.first;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return 0;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1;
  int best = 0;
  float best_ms = 1e30f;
  for (int v = 0; v < nvar; ++v) {
    run(v);
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3; ++r) run(v);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return -1;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    count_launch(4);
    if (ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::lock_guard<std::mutex> lk(g_mu);
  g_cache[key] = std::make_pair(best, best_ms / 3.0f);
  return best;
}

const char* tune_report() {
  std::lock_guard<std::mutex> lk(g_mu);
  std::ostringstream os;
  os << "[";
  bool first = true;
  for (auto& kv : g_cache) {
    if (!first) os << ",";
    first = false;
    os << "{\"kernel\":\"dslash\",\"dtype\":" << std::get<0>(kv.first)
       << ",\"parity\":" << std::get<1>(kv.first) << ",\"dagger\":" << std::get<2>(kv.first)
       << ",\"volume\":" << std::get<3>(kv.first) << ",\"nrhs\":" << std::get<4>(kv.first)
       << ",\"variant\":" << kv.second.first << ",\"ms\":" << kv.second.second << "}";
  }
  os << "]";
  g_report = os.str();
  return g_report.c_str();
}

}  // namespace wmg

extern "C" const char* mg_autotune_report(void) { return wmg::tune_report(); }
