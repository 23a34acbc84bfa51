// map.cu -- maintenance of the Gaussian set between mapping steps (appendix "Gaussian
// Initialization and Joint Mapping": Eq. app-ema and the pruning bounds on the observation
// count, visibility score, covariance trace and opacity). Elementwise over the Gaussians.
#include <math.h>

#include <algorithm>

#include "rgs_internal.cuh"

namespace rgs {
namespace {

constexpr int kMapThreads = 256;

// Eq. app-ema: mu_bar <- (1 - eta) mu_bar + eta mu.
__global__ void __launch_bounds__(kMapThreads) map_ema_kernel(int64_t n3,
                                                              const float* __restrict__ means,
                                                              float* __restrict__ ema,
                                                              float eta) {
  chain_wait();
  for (int64_t k = (int64_t)blockIdx.x * kMapThreads + threadIdx.x; k < n3;
       k += (int64_t)gridDim.x * kMapThreads)
    ema[k] = fmaf(eta, means[k] - ema[k], ema[k]);
}

// Kept iff alpha >= min_opacity, tr(Sigma) <= max_trace and not (observed at least
// min_observations times with a visibility score below min_visibility); counts the kept ones
// (one atomic per warp).
__global__ void __launch_bounds__(kMapThreads) prune_mask_kernel(
    int n, const float* __restrict__ log_scales, const float* __restrict__ logits,
    const uint32_t* __restrict__ obs_count, const float* __restrict__ vis_score,
    float min_opacity, float max_trace, uint32_t min_observations, float min_visibility,
    uint8_t* __restrict__ keep, uint32_t* __restrict__ n_keep) {
  chain_wait();
  const int i = blockIdx.x * kMapThreads + threadIdx.x;
  bool k = false;
  if (i < n) {
    const float alpha = 1.0f / (1.0f + expf(-logits[i]));
    const float tr = expf(2.0f * log_scales[3 * i]) + expf(2.0f * log_scales[3 * i + 1]) +
                     expf(2.0f * log_scales[3 * i + 2]);
    const bool weak = obs_count[i] >= min_observations && vis_score[i] < min_visibility;
    k = alpha >= min_opacity && tr <= max_trace && !weak;
    keep[i] = k ? 1 : 0;
  }
  const unsigned votes = __ballot_sync(0xffffffffu, k);
  if ((threadIdx.x & 31) == 0 && votes) atomicAdd(n_keep, (uint32_t)__popc(votes));
}

}  // namespace

cudaError_t launch_map_ema(int64_t n, const float* means, float* ema, float eta,
                           cudaStream_t stream) {
  const int64_t n3 = 3 * n;
  const unsigned blocks = (unsigned)std::min<int64_t>((n3 + kMapThreads - 1) / kMapThreads, 8 * 152);
  const cudaError_t e = launch_chained(map_ema_kernel, dim3(blocks), dim3(kMapThreads), stream,
                                       n3, means, ema, eta);
  RGS_LAUNCHED();
  return e;
}

cudaError_t launch_prune_mask(int64_t n, const float* log_scales, const float* logits,
                              const uint32_t* obs_count, const float* vis_score, float min_opacity,
                              float max_trace, uint32_t min_observations, float min_visibility,
                              uint8_t* keep, uint32_t* n_keep, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(n_keep, 0, sizeof(uint32_t), stream);
  if (e != cudaSuccess || n == 0) return e;
  e = launch_chained(prune_mask_kernel, dim3((unsigned)((n + kMapThreads - 1) / kMapThreads)),
                     dim3(kMapThreads), stream, (int)n, log_scales, logits, obs_count, vis_score,
                     min_opacity, max_trace, min_observations, min_visibility, keep, n_keep);
  RGS_LAUNCHED();
  return e;
}

}  // namespace rgs
