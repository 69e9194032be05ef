// Complex-Gaussian random fields from Philox4x32-10 (random initial guesses of Eq. 2).
//
// Philox4x32-10 follows its published definition (Salmon, Moraes, Dror, Shaw, SC'11):
// 10 rounds of two 32x32->64-bit multiplies of counter words 0 and 2 by fixed odd
// constants, hi/lo halves permuted and xored with the key, key bumped by the Weyl
// constants between rounds.  Counter (site, component, vector id, 0), key (seed low,
// seed high); the four words make two 53-bit uniforms and Box-Muller gives
// Re = sqrt(-2 ln(1 - u_a)) cos(2 pi u_b), Im = sqrt(-2 ln(1 - u_a)) sin(2 pi u_b).
#include "common.cuh"
#include "internal.h"

namespace wmg {

namespace {

__device__ __forceinline__ void philox_round(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  uint32_t lo0 = M0 * c[0], hi0 = __umulhi(M0, c[0]);
  uint32_t lo1 = M1 * c[2], hi1 = __umulhi(M1, c[2]);
  uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
  c[0] = n0;
  c[1] = lo1;
  c[2] = n2;
  c[3] = lo0;
}

__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    philox_round(c, k0, k1);
  }
}

// FP32 fields: the same Philox words and the same 53-bit uniforms, with the transforms
// in FP32 (GB300's FP64 transcendentals are slow).  1 - u_a is formed exactly as the
// integer 2^53 - m_a before rounding to float, so the tail is not lost to cancellation;
// small u_a goes through log1pf.  Relative error against the FP64 map ~1e-7.
__global__ void gaussian_kernel_f32(zf* out, uint32_t k0, uint32_t k1, unsigned id0, int V,
                                    int nc, uint32_t w3, size_t total) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    size_t per = (size_t)V * nc;
    unsigned v = (unsigned)(e / per);
    size_t rem = e % per;
    uint32_t c[4] = {(uint32_t)(rem / nc), (uint32_t)(rem % nc), id0 + v, w3};
    philox10(c, k0, k1);
    unsigned long long ma = ((unsigned long long)(c[0] >> 5) << 26) | (c[1] >> 6);
    unsigned long long mb = ((unsigned long long)(c[2] >> 5) << 26) | (c[3] >> 6);
    const float s53 = 1.1102230246251565e-16f;  // 2^-53
    float ua = __ull2float_rn(ma) * s53;
    float l;
    if (ua < 0.5f) l = log1pf(-ua);
    else l = logf(__ull2float_rn((1ull << 53) - ma) * s53);
    float rho = sqrtf(-2.0f * l);
    float ub = __ull2float_rn(mb) * s53;
    float sn, cs;
    sincospif(2.0f * ub, &sn, &cs);
    out[e] = {rho * cs, rho * sn};
  }
}

template <typename R>
__global__ void gaussian_kernel(cplx<R>* out, uint32_t k0, uint32_t k1, unsigned id0, int V,
                                int nc, uint32_t w3, size_t total) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (size_t)gridDim.x * blockDim.x) {
    size_t per = (size_t)V * nc;
    unsigned v = (unsigned)(e / per);
    size_t rem = e % per;
    uint32_t c[4] = {(uint32_t)(rem / nc), (uint32_t)(rem % nc), id0 + v, w3};
    philox10(c, k0, k1);
    const double s53 = 1.1102230246251565e-16;  // 2^-53
    double ua = ((double)(c[0] >> 5) * 67108864.0 + (double)(c[1] >> 6)) * s53;
    double ub = ((double)(c[2] >> 5) * 67108864.0 + (double)(c[3] >> 6)) * s53;
    double rho = sqrt(-2.0 * log(1.0 - ua));
    double sn, cs;
    sincos(2.0 * 3.141592653589793 * ub, &sn, &cs);
    out[e] = {(R)(rho * cs), (R)(rho * sn)};
  }
}

}  // namespace

template <typename R>
int gaussian_fill_n(cplx<R>* out, unsigned long long seed, unsigned id0, int nvec, int nsites,
                    int ncomp, unsigned word3, cudaStream_t st) {
  size_t total = (size_t)nvec * nsites * ncomp;
  size_t g = (total + 255) / 256;
  size_t cap = (size_t)num_sms() * 16;
  unsigned grid = (unsigned)(g < cap ? (g < 1 ? 1 : g) : cap);
  uint32_t k0 = (uint32_t)(seed & 0xffffffffu), k1 = (uint32_t)(seed >> 32);
  if (sizeof(R) == 4)
    gaussian_kernel_f32<<<grid, 256, 0, st>>>((zf*)out, k0, k1, id0, nsites, ncomp, word3, total);
  else
    gaussian_kernel<R><<<grid, 256, 0, st>>>(out, k0, k1, id0, nsites, ncomp, word3, total);
  WMG_LAUNCHED();
  return MG_OK;
}

template <typename R>
int gaussian_fill(cplx<R>* out, unsigned long long seed, unsigned id0, int nvec, int V,
                  cudaStream_t st) {
  return gaussian_fill_n<R>(out, seed, id0, nvec, V, 12, 0u, st);
}

template int gaussian_fill<float>(zf*, unsigned long long, unsigned, int, int, cudaStream_t);
template int gaussian_fill<double>(zd*, unsigned long long, unsigned, int, int, cudaStream_t);
template int gaussian_fill_n<float>(zf*, unsigned long long, unsigned, int, int, int, unsigned,
                                    cudaStream_t);
template int gaussian_fill_n<double>(zd*, unsigned long long, unsigned, int, int, int, unsigned,
                                     cudaStream_t);

}  // namespace wmg
