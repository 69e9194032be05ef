// Arithmetic-rate probe: the FP64 and FP32 FMA throughput of the device, the denominators
// of the ALU-bound kernels' rooflines (FP64 Jacobi/Gram/Galerkin; double-float Gram,
// update and Galerkin, which run on the FP32 units).
#include <cuda_runtime.h>

#include "common.cuh"
#include "internal.h"

namespace wmg {

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;    // independent dependency chains per thread
constexpr int PROBE_UNROLL = 16;

// Every thread runs PROBE_CHAINS independent x <- x * a + b chains; a < 1 keeps them bounded.
// The result is stored so that the chains cannot be removed.
template <typename T>
__global__ void __launch_bounds__(PROBE_THREADS)
fma_probe_kernel(T* out, T a, T b, int iters) {
  T x[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < PROBE_UNROLL; ++u) {
#pragma unroll
      for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = fma(x[c], a, b);
    }
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int probe(double* tflops, int iters, cudaStream_t st) {
  int occ = 0;
  WMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fma_probe_kernel<T>,
                                                         PROBE_THREADS, 0));
  if (occ < 1) occ = 1;
  int blocks = occ * num_sms();
  T* out = nullptr;
  WMG_CUDA(cudaMallocAsync(&out, sizeof(T) * (size_t)blocks * PROBE_THREADS, st));
  cudaEvent_t e0, e1;
  WMG_CUDA(cudaEventCreate(&e0));
  WMG_CUDA(cudaEventCreate(&e1));
  float best = 0;
  int status = MG_OK;
  for (int rep = 0; rep < 4 && status == MG_OK; ++rep) {
    cudaEventRecord(e0, st);
    fma_probe_kernel<T><<<blocks, PROBE_THREADS, 0, st>>>(out, (T)0.9999999, (T)1e-7, iters);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      status = fail(MG_ECUDA, "fma probe launch failed");
      break;
    }
    count_launch();
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0 || ms < best)) best = ms;   // first launch is warm-up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, st);
  if (status != MG_OK) return status;
  WMG_CUDA(cudaStreamSynchronize(st));
  double fmas = (double)blocks * PROBE_THREADS * iters * PROBE_UNROLL * PROBE_CHAINS;
  *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  return MG_OK;
}

}  // namespace

}  // namespace wmg

extern "C" int mg_probe_fma_peak(int dtype, double* tflops, void* stream) {
  if (!tflops) return wmg::fail(MG_EINVAL, "mg_probe_fma_peak: NULL output");
  cudaStream_t st = (cudaStream_t)stream;
  // about 15 ms per launch at the nominal FP64 (1.25 TFLOP/s) and FP32 (80 TFLOP/s) rates
  if (dtype == MG_C128) return wmg::probe<double>(tflops, 256, st);
  if (dtype == MG_C64) return wmg::probe<float>(tflops, 16384, st);
  return wmg::fail(MG_EINVAL, "mg_probe_fma_peak: dtype must be MG_C128 or MG_C64");
}
