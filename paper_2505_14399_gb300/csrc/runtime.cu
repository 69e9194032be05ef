// Error reporting, geometry validation and host/device staging of ABI arguments.
#include <atomic>
#include <cstring>
#include <map>
#include <unordered_map>
#include <utility>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace wmg {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int status, const std::string& msg) {
  g_last_error = msg;
  return status;
}

void count_launch(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int make_geom(Geom& g, const int dims[4], double kappa, const double w[4], const int bc[4],
              bool need_even) {
  long long V = 1;
  for (int m = 0; m < 4; ++m) {
    if (dims[m] < 1) return fail(MG_EINVAL, "lattice extent < 1");
    if (need_even && (dims[m] & 1)) return fail(MG_EINVAL, "parity form needs even extents");
    if (bc[m] != 1 && bc[m] != -1) return fail(MG_EINVAL, "bc_phase must be +1 or -1");
    g.L[m] = dims[m];
    g.w[m] = w[m];
    g.bc[m] = bc[m];
    V *= dims[m];
  }
  if (V > (1LL << 30)) return fail(MG_EINVAL, "lattice volume too large");
  g.V = (int)V;
  g.kappa = kappa;
  return MG_OK;
}

// ------------------------------------------------------------------ memory cache
// Device and pinned-host blocks released by the library are kept, per device and rounded
// size, and handed out again: building and destroying hierarchies of the same shape in a
// loop then costs no cudaMalloc / cudaFree (both of which synchronise the device).  On an
// allocation failure the cache is returned to the driver and the allocation retried.
// Callers release blocks only when no queued work still uses them.
namespace {

struct MemCache {
  std::mutex mu;
  std::multimap<std::pair<int, size_t>, void*> free_dev, free_host;
  std::unordered_map<void*, std::pair<int, size_t>> live_dev, live_host;
};

MemCache& mem_cache() {
  static MemCache* c = new MemCache();   // never destroyed: blocks may be freed at exit
  return *c;
}

size_t round_block(size_t b) {
  size_t g = b < ((size_t)1 << 20) ? 512 : ((size_t)2 << 20);
  if (b == 0) b = 1;
  return (b + g - 1) / g * g;
}

int cached_alloc(void** p, size_t bytes, bool host) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::pair<int, size_t> key(dev, round_block(bytes));
  MemCache& c = mem_cache();
  std::lock_guard<std::mutex> lock(c.mu);
  auto& fl = host ? c.free_host : c.free_dev;
  auto& live = host ? c.live_host : c.live_dev;
  auto it = fl.find(key);
  if (it != fl.end()) {
    *p = it->second;
    fl.erase(it);
    live[*p] = key;
    return MG_OK;
  }
  cudaError_t e = host ? cudaMallocHost(p, key.second) : cudaMalloc(p, key.second);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    cudaDeviceSynchronize();
    for (auto& kv : fl) {
      if (host) cudaFreeHost(kv.second);
      else cudaFree(kv.second);
    }
    fl.clear();
    e = host ? cudaMallocHost(p, key.second) : cudaMalloc(p, key.second);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(e == cudaErrorMemoryAllocation ? MG_ENOMEM : MG_ECUDA,
                std::string(host ? "pinned" : "device") + " allocation of " +
                    std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
  }
  live[*p] = key;
  return MG_OK;
}

void cached_free(void* p, bool host) {
  if (!p) return;
  MemCache& c = mem_cache();
  std::lock_guard<std::mutex> lock(c.mu);
  auto& live = host ? c.live_host : c.live_dev;
  auto it = live.find(p);
  if (it == live.end()) return;
  (host ? c.free_host : c.free_dev).emplace(it->second, p);
  live.erase(it);
}

}  // namespace

int* device_error_word() {
  static std::mutex mu;
  static int* word = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!word) {
    if (cudaMallocHost(&word, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      word = nullptr;
      return nullptr;
    }
    *word = 0;
  }
  return word;
}

int take_device_error() {
  int* w = device_error_word();
  if (!w) return 0;
  int v = *(volatile int*)w;
  *(volatile int*)w = 0;
  return v;
}

int dev_alloc_bytes(void** p, size_t bytes) { return cached_alloc(p, bytes, false); }
void dev_free(void* p) { cached_free(p, false); }
int host_alloc_bytes(void** p, size_t bytes) { return cached_alloc(p, bytes, true); }
void host_free(void* p) { cached_free(p, true); }

int smem_attr_raw(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> done;
  int dev = 0;
  WMG_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  size_t& have = done[{dev, fn}];
  if (have >= bytes) return MG_OK;
  WMG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  have = bytes;
  return MG_OK;
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
      n = 148;
  }
  return n;
}

int is_device_pointer(const void* p, bool* dev) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *dev = false;
    return MG_OK;
  }
  *dev = (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
  return MG_OK;
}

Staged::~Staged() {
  if (owned && dev) cudaFreeAsync(dev, stream);
}

int stage_in(Staged& s, const void* p, size_t bytes, cudaStream_t st) {
  bool dev = false;
  WMG_TRY(is_device_pointer(p, &dev));
  s.stream = st;
  if (dev) {
    s.dev = const_cast<void*>(p);
    s.owned = false;
    return MG_OK;
  }
  WMG_CUDA(cudaMallocAsync(&s.dev, bytes, st));
  s.owned = true;
  WMG_CUDA(cudaMemcpyAsync(s.dev, p, bytes, cudaMemcpyHostToDevice, st));
  return MG_OK;
}

int stage_out_alloc(Staged& s, void* p, size_t bytes, cudaStream_t st) {
  bool dev = false;
  WMG_TRY(is_device_pointer(p, &dev));
  s.stream = st;
  if (dev) {
    s.dev = p;
    s.owned = false;
    return MG_OK;
  }
  WMG_CUDA(cudaMallocAsync(&s.dev, bytes, st));
  s.owned = true;
  return MG_OK;
}

int stage_out_finish(Staged& s, void* p, size_t bytes, cudaStream_t st) {
  if (!s.owned) return MG_OK;
  WMG_CUDA(cudaMemcpyAsync(p, s.dev, bytes, cudaMemcpyDeviceToHost, st));
  // host destination: the caller reads it after return
  WMG_CUDA(cudaStreamSynchronize(st));
  return MG_OK;
}

// ------------------------------------------------------------------ per-kernel timing
namespace {
struct ProfRec {
  const char* name;
  double bytes, flops, issued;
  int ev0, ev1;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<cudaEvent_t> g_prof_events;
std::vector<ProfRec> g_prof_recs;
size_t g_prof_next = 0;
std::vector<int> g_prof_open;   // stack of open records (launches do not nest across threads)
std::string g_prof_json;
}  // namespace

bool prof_enabled() { return g_prof_on; }

void prof_begin(const char* name, double bytes, double flops, double issued, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (g_prof_next + 2 > g_prof_events.size()) {
    g_prof_open.push_back(-1);
    return;
  }
  int e0 = (int)g_prof_next++, e1 = (int)g_prof_next++;
  cudaEventRecord(g_prof_events[e0], st);
  g_prof_recs.push_back({name, bytes, flops, issued, e0, e1});
  g_prof_open.push_back((int)g_prof_recs.size() - 1);
}

void prof_end(cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (g_prof_open.empty()) return;
  int r = g_prof_open.back();
  g_prof_open.pop_back();
  if (r >= 0) cudaEventRecord(g_prof_events[g_prof_recs[r].ev1], st);
}

}  // namespace wmg

extern "C" int mg_profile_enable(int enable, int max_launches) {
  using namespace wmg;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_recs.clear();
  g_prof_open.clear();
  g_prof_next = 0;
  if (enable) {
    size_t need = (size_t)(max_launches > 0 ? max_launches : 100000) * 2;
    while (g_prof_events.size() < need) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return fail(MG_ECUDA, "mg_profile_enable: event");
      g_prof_events.push_back(e);
    }
  }
  g_prof_on = enable != 0;
  return MG_OK;
}

extern "C" const char* mg_profile_report(void) {
  using namespace wmg;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  struct Agg {
    long long n = 0;
    double ms = 0, bytes = 0, flops = 0, issued = 0;
  };
  std::map<std::string, Agg> agg;
  for (auto& r : g_prof_recs) {
    float ms = 0;
    if (cudaEventSynchronize(g_prof_events[r.ev1]) != cudaSuccess ||
        cudaEventElapsedTime(&ms, g_prof_events[r.ev0], g_prof_events[r.ev1]) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    Agg& a = agg[r.name];
    a.n += 1;
    a.ms += ms;
    a.bytes += r.bytes;
    a.flops += r.flops;
    a.issued += r.issued;
  }
  std::ostringstream os;
  os << "{";
  bool first = true;
  for (auto& kv : agg) {
    if (!first) os << ",";
    first = false;
    os << "\"" << kv.first << "\":{\"launches\":" << kv.second.n << ",\"ms\":" << kv.second.ms
       << ",\"bytes\":" << kv.second.bytes << ",\"flops\":" << kv.second.flops;
    if (kv.second.issued > 0) os << ",\"issued_flops\":" << kv.second.issued;
    os << "}";
  }
  os << "}";
  g_prof_json = os.str();
  return g_prof_json.c_str();
}

extern "C" const char* mg_last_error(void) { return wmg::g_last_error.c_str(); }

extern "C" long long mg_kernel_launches(void) { return wmg::g_launches.load(); }

extern "C" void mg_params_default(mg_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  for (int m = 0; m < 4; ++m) {
    p->dims[m] = 4;
    p->block[m] = 2;
    p->hop_weight[m] = 1.0;
    p->bc_phase[m] = 1;
  }
  p->kappa = 0.12;
  p->k = 24;
  p->r = 24;
  p->n_s = 2;
  p->sweeps = 5;
  p->seed = 3000;
  p->setup_dtype = MG_C64;
  p->solve_dtype = MG_C64;
  p->post_smooth = 8;
  p->coarse_tol = 0.03;
  p->coarse_restart = 32;
  p->coarse_maxiter = 2000;
  p->outer_restart = 16;
  p->inner_tol = 1e-5;
  p->svd_refine = -1;
  p->coarse_persistent = 1;
  p->fp64_emulation = -1;
  p->link_compress = -1;
  p->schur_smoother = 0;
}
