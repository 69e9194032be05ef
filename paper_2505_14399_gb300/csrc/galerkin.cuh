// Shared pieces of the Galerkin coarse-operator build (Eq. 5): hop geometry, the staging batch
// size, the exact double-float i sigma_mu, and the tensor-pipe forward-hop kernel's launcher.
#pragma once

#include "common.cuh"
#include "df64.cuh"
#include "internal.h"

namespace wmg {

struct HopGeom {
  int L[4], stride[4];
  double w[4];
  int bc[4];
  double kappa;
};

constexpr int GNB = 8;       // fine sites staged per batch

// (i sigma_mu psi)[s] in df64 (sign changes and swaps only: exact)
__device__ __forceinline__ zdf isigma_df(int mu, int s, zdf p0, zdf p1) {
  if (mu == 0) return s == 0 ? zdf_ti(p1) : zdf_ti(p0);
  if (mu == 1) return s == 0 ? p1 : zdf_neg(p0);
  return s == 0 ? zdf_ti(p0) : zdf_tmi(p1);
}

// Whether the tensor-pipe forward-hop kernel handles this k and blocking (2k <= 48, its
// shared memory fits one CTA).
bool galerkin_tc_supported(int k, const Blocking& B);
// bf16 flops that kernel issues for one build at nb sites per batch (its digit-plane
// products, padding included).
double galerkin_tc_issued_flops(int k, const Blocking& B, int nb);
// Sites per staging batch of the tensor-pipe kernel for this build (8 or 4; autotuned where
// both fit, which runs the kernel on these arguments).
int galerkin_tc_batch(int* nb, zd* Op, zd* Xpart, const zdf* Pdf, int k, const zdf* Ldf,
                      const HopGeom& g, const Blocking& B, int* range_flag, cudaStream_t st);
// The forward-hop blocks of the double-float Galerkin build on the tensor pipe (same outputs
// as the FP32-unit kernel: Y_+mu blocks into Op, in-aggregate partials into Xpart), nb sites
// per staging batch.  Raises *range_flag (device int) if a staged entry is outside the
// fixed-point range (|v| >= 2 or not finite), in which case the caller rebuilds with the
// FP32-unit kernel.
int galerkin_hops_tc(zd* Op, zd* Xpart, const zdf* Pdf, int k, const zdf* Ldf, const HopGeom& g,
                     const Blocking& B, int nb, int* range_flag, cudaStream_t st);

}  // namespace wmg
