// Shared device/host helpers of the GB300 Wilson multigrid library.
#pragma once

#include <utility>

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>

#include "../../include/wilson_mg.h"

namespace wmg {

// ------------------------------------------------------------------ error handling
void set_error(const std::string& msg);
int fail(int status, const std::string& msg);
void count_launch(long long n = 1);
// Pinned, device-visible error word: a kernel whose bounded wait gives up stores a non-zero
// code there; take_device_error() returns it (0 if none) and clears it.  Read only after the
// stream that ran the kernel has been synchronised.
int* device_error_word();
int take_device_error();
// Library-wide caching allocator (device memory and pinned host memory); see runtime.cu.
int dev_alloc_bytes(void** p, size_t bytes);
void dev_free(void* p);
int host_alloc_bytes(void** p, size_t bytes);
void host_free(void* p);
template <typename T>
inline int dev_alloc(T** p, size_t bytes) { return dev_alloc_bytes(reinterpret_cast<void**>(p), bytes); }
template <typename T>
inline int host_alloc(T** p, size_t bytes) { return host_alloc_bytes(reinterpret_cast<void**>(p), bytes); }

#define WMG_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return ::wmg::fail(e_ == cudaErrorMemoryAllocation ? MG_ENOMEM : MG_ECUDA,    \
                         std::string(#call) + ": " + cudaGetErrorString(e_));       \
  } while (0)

#define WMG_LAUNCHED()                                                              \
  do {                                                                              \
    ::wmg::count_launch();                                                          \
    cudaError_t e_ = cudaGetLastError();                                            \
    if (e_ != cudaSuccess)                                                          \
      return ::wmg::fail(MG_ECUDA, std::string("kernel launch at ") + __FILE__ +    \
                         ":" + std::to_string(__LINE__) + ": " +                    \
                         cudaGetErrorString(e_));                                   \
  } while (0)

#define WMG_TRY(expr)                                                               \
  do {                                                                              \
    int s_ = (expr);                                                                \
    if (s_ != MG_OK) return s_;                                                     \
  } while (0)

// ------------------------------------------------------------------ dependent launches
// Programmatic dependent launch: a kernel started with launch_dep() may be scheduled while
// the previous kernel on its stream is still finishing (its launch latency and prologue
// overlap that tail).  Every such kernel calls dep_entry() before touching global memory:
// griddepcontrol.wait returns once the previous grid has completed and its writes are
// visible (immediately for a kernel launched the ordinary way), and
// griddepcontrol.launch_dependents lets the next kernel be scheduled in turn.
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void dep_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void dep_entry() {
  dep_wait();
  dep_trigger();
}

template <typename... KArgs, typename... Args>
cudaError_t launch_dep(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

#define WMG_LAUNCH_DEP(...)                                                         \
  do {                                                                              \
    cudaError_t e_ = ::wmg::launch_dep(__VA_ARGS__);                                \
    ::wmg::count_launch();                                                          \
    if (e_ != cudaSuccess)                                                          \
      return ::wmg::fail(MG_ECUDA, std::string("kernel launch at ") + __FILE__ +    \
                         ":" + std::to_string(__LINE__) + ": " +                    \
                         cudaGetErrorString(e_));                                   \
  } while (0)

// ------------------------------------------------------------------ per-kernel timing
// When enabled (mg_profile_enable), every instrumented launch is bracketed by CUDA events
// on its own stream; mg_profile_report() aggregates durations with the launch's
// algorithmic bytes and flops per kernel name.  Disabled: one branch per launch.
bool prof_enabled();
// bytes, flops: the algorithmic figures of the launch; issued: flops the tensor pipe executes
// for them, when that differs (exact digit-plane products), else 0
void prof_begin(const char* name, double bytes, double flops, double issued, cudaStream_t st);
void prof_end(cudaStream_t st);
struct ProfScope {
  bool on;
  cudaStream_t st;
  ProfScope(const char* name, double bytes, double flops, cudaStream_t s) : on(prof_enabled()), st(s) {
    if (on) prof_begin(name, bytes, flops, 0.0, s);
  }
  ProfScope(const char* name, double bytes, double flops, double issued, cudaStream_t s)
      : on(prof_enabled()), st(s) {
    if (on) prof_begin(name, bytes, flops, issued, s);
  }
  ~ProfScope() {
    if (on) prof_end(st);
  }
};

// ------------------------------------------------------------------ complex numbers
template <typename R>
struct cplx {
  R re, im;
};

template <typename R>
__host__ __device__ __forceinline__ cplx<R> mk(R a, R b) { return cplx<R>{a, b}; }
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator+(cplx<R> a, cplx<R> b) {
  return {a.re + b.re, a.im + b.im};
}
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator-(cplx<R> a, cplx<R> b) {
  return {a.re - b.re, a.im - b.im};
}
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator-(cplx<R> a) { return {-a.re, -a.im}; }
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator*(cplx<R> a, cplx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__host__ __device__ __forceinline__ cplx<R> operator*(R s, cplx<R> a) { return {s * a.re, s * a.im}; }
template <typename R>
__host__ __device__ __forceinline__ cplx<R>& operator+=(cplx<R>& a, cplx<R> b) {
  a.re += b.re; a.im += b.im; return a;
}
template <typename R>
__host__ __device__ __forceinline__ cplx<R>& operator-=(cplx<R>& a, cplx<R> b) {
  a.re -= b.re; a.im -= b.im; return a;
}
template <typename R>
__host__ __device__ __forceinline__ cplx<R> conj(cplx<R> a) { return {a.re, -a.im}; }
// conj(a) * b
template <typename R>
__host__ __device__ __forceinline__ cplx<R> cmulc(cplx<R> a, cplx<R> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// i * a and -i * a
template <typename R>
__host__ __device__ __forceinline__ cplx<R> ti(cplx<R> a) { return {-a.im, a.re}; }
template <typename R>
__host__ __device__ __forceinline__ cplx<R> tmi(cplx<R> a) { return {a.im, -a.re}; }
template <typename R>
__host__ __device__ __forceinline__ R norm2(cplx<R> a) { return a.re * a.re + a.im * a.im; }
// a += b * c   (complex FMA)
template <typename R>
__host__ __device__ __forceinline__ void cfma(cplx<R>& a, cplx<R> b, cplx<R> c) {
  a.re = fma(b.re, c.re, a.re); a.re = fma(-b.im, c.im, a.re);
  a.im = fma(b.re, c.im, a.im); a.im = fma(b.im, c.re, a.im);
}
// a += conj(b) * c
template <typename R>
__host__ __device__ __forceinline__ void cfmac(cplx<R>& a, cplx<R> b, cplx<R> c) {
  a.re = fma(b.re, c.re, a.re); a.re = fma(b.im, c.im, a.re);
  a.im = fma(b.re, c.im, a.im); a.im = fma(-b.im, c.re, a.im);
}

typedef cplx<double> zd;
typedef cplx<float> zf;

// ------------------------------------------------------------------ storage traits
// Each storage type S provides: element type, compute real type, load/store of one
// complex number at an element index.
struct StC128 {
  typedef double2 elem;
  typedef double real;
  static __device__ __forceinline__ cplx<double> ld(const elem* p, size_t i) {
    double2 v = __ldg(p + i); return {v.x, v.y};
  }
  static __device__ __forceinline__ void st(elem* p, size_t i, cplx<double> v) {
    p[i] = make_double2(v.re, v.im);
  }
};
struct StC64 {
  typedef float2 elem;
  typedef float real;
  static __device__ __forceinline__ cplx<float> ld(const elem* p, size_t i) {
    float2 v = __ldg(p + i); return {v.x, v.y};
  }
  static __device__ __forceinline__ void st(elem* p, size_t i, cplx<float> v) {
    p[i] = make_float2(v.re, v.im);
  }
};
struct StF16 {
  typedef __half2 elem;
  typedef float real;
  static __device__ __forceinline__ cplx<float> ld(const elem* p, size_t i) {
    float2 v = __half22float2(p[i]); return {v.x, v.y};
  }
  static __device__ __forceinline__ void st(elem* p, size_t i, cplx<float> v) {
    p[i] = __floats2half2_rn(v.re, v.im);
  }
};
struct StBF16 {
  typedef __nv_bfloat162 elem;
  typedef float real;
  static __device__ __forceinline__ cplx<float> ld(const elem* p, size_t i) {
    float2 v = __bfloat1622float2(p[i]); return {v.x, v.y};
  }
  static __device__ __forceinline__ void st(elem* p, size_t i, cplx<float> v) {
    p[i] = __floats2bfloat162_rn(v.re, v.im);
  }
};

inline size_t dtype_bytes(int dtype) {
  switch (dtype) {
    case MG_C128: return 16;
    case MG_C64: return 8;
    case MG_F16: return 4;
    case MG_BF16: return 4;
  }
  return 0;
}

// ------------------------------------------------------------------ lattice geometry
struct Geom {
  int L[4];
  int V;
  double kappa;
  double w[4];
  int bc[4];
};

int make_geom(Geom& g, const int dims[4], double kappa, const double w[4], const int bc[4],
              bool need_even);

int num_sms();

// Raises the dynamic shared-memory limit of kernel `fn` on the current device to at least
// `bytes`: the attribute is per device, so the record of what was set is kept per (device,
// kernel), under a lock.
int smem_attr_raw(const void* fn, size_t bytes);
template <typename F>
inline int smem_attr(F* fn, size_t bytes) {
  return smem_attr_raw(reinterpret_cast<const void*>(fn), bytes);
}

// ------------------------------------------------------------------ host staging
// A field argument that may live on the host: returns a device pointer (the same
// pointer if it is already device/managed memory) and whether a copy was made.
struct Staged {
  void* dev = nullptr;
  bool owned = false;
  cudaStream_t stream = 0;
  ~Staged();
};
int is_device_pointer(const void* p, bool* dev);
int stage_in(Staged& s, const void* p, size_t bytes, cudaStream_t st);
int stage_out_alloc(Staged& s, void* p, size_t bytes, cudaStream_t st);
int stage_out_finish(Staged& s, void* p, size_t bytes, cudaStream_t st);

}  // namespace wmg
