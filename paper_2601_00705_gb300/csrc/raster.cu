// raster.cu -- pair duplication, tile ranges, and the forward / backward alpha blends.
//
// Forward blend (Section 3.1, Eq. alpha; Section 3.2.2): one CTA per (view, tile); the tile's
// Gaussians, already in near-to-far order, are staged through shared memory in batches of one
// Gaussian per thread and every thread composites its own pixel front to back with early exit.
// Backward blend: the same tiles are walked back to front from each pixel's last contributor,
// recovering the transmittance by division from the saved final value, so no per-pixel list is
// stored; per-Gaussian screen-space gradients are reduced across the warp before one atomic per
// value and warp.
#include "rgs_internal.cuh"

namespace rgs {
namespace {

constexpr int kDupThreads = 256;

__global__ void __launch_bounds__(kDupThreads) duplicate_kernel(
    const __grid_constant__ Views views, int n, const uint32_t* __restrict__ order,
    const uint32_t* __restrict__ offsets, const uint32_t* __restrict__ ntiles,
    const float4* __restrict__ rec0, const float4* __restrict__ rec1,
    const Counters* __restrict__ counters_in, uint32_t capacity, uint32_t* __restrict__ keys,
    uint32_t* __restrict__ vals, Counters* __restrict__ counters) {
  const uint32_t k = blockIdx.x * kDupThreads + threadIdx.x;
  if (k >= counters_in->n_visible) return;
  const uint32_t vi = order[k];
  const int v = (int)(vi / (uint32_t)n);
  const uint32_t begin = offsets[k];
  const uint32_t cnt = ntiles[vi];
  const uint32_t end = begin + cnt;  // this entry's slots: [begin, end)
  if (end > capacity) atomicOr(&counters->status, (uint32_t)kStatusPairOverflow);
  const ViewParams& vp = views.v[v];
  uint32_t off = begin;
  Ellipse e;
  if (make_ellipse(rec0[vi], rec1[vi], e)) {
    for_each_tile_row(e, views.tile_w, views.tile_h, vp.tiles_x, vp.tiles_y,
                      [&](int ty, int tx0, int tx1) {
                        const uint32_t row = (uint32_t)(vp.tile_base + ty * vp.tiles_x);
                        for (int tx = tx0; tx <= tx1; ++tx, ++off) {
                          if (off < end && off < capacity) {
                            keys[off] = row + (uint32_t)tx;
                            vals[off] = vi;
                          }
                        }
                      });
  }
  // The counting pass visits the same tiles, so this never runs; if it ever did, the unused
  // slots get the out-of-range key total_tiles, which sorts last and owns no tile range.
  for (; off < end && off < capacity; ++off) {
    keys[off] = (uint32_t)views.total_tiles;
    vals[off] = vi;
  }
}

__global__ void store_pair_count_kernel(Counters* counters, uint32_t capacity) {
  const uint32_t p = counters->n_pairs;
  counters->n_pairs_stored = p < capacity ? p : capacity;
}

__global__ void tile_ranges_kernel(const uint32_t* __restrict__ keys,
                                   const Counters* __restrict__ counters, uint32_t total_tiles,
                                   uint2* __restrict__ ranges) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t n = counters->n_pairs_stored;
  if (p >= n) return;
  const uint32_t key = keys[p];
  if (key >= total_tiles) return;
  if (p == 0 || keys[p - 1] != key) ranges[key].x = p;
  if (p == n - 1 || keys[p + 1] != key) ranges[key].y = p + 1;
}

// ------------------------------------------------------------------------------------------
// Forward blend.
// ------------------------------------------------------------------------------------------
template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH) blend_forward_kernel(
    const __grid_constant__ Views views, const Consts c, const uint2* __restrict__ ranges,
    const uint32_t* __restrict__ pair_vals, const float4* __restrict__ rec0,
    const float4* __restrict__ rec1, const float4* __restrict__ rec2, float* __restrict__ color,
    float* __restrict__ depth, float* __restrict__ alpha_out, float* __restrict__ t_final,
    int32_t* __restrict__ last_index, Counters* __restrict__ counters) {
  constexpr int kThreads = TW * TH;
  __shared__ float4 s0[kThreads], s1[kThreads], s2[kThreads];
  __shared__ unsigned long long s_eval[kThreads / 32], s_contrib[kThreads / 32];
  const int gtile = blockIdx.x;
  const int v = view_of_tile(views, gtile);
  const ViewParams& vp = views.v[v];
  const int local = gtile - vp.tile_base;
  const int ty = local / vp.tiles_x, tx = local - ty * vp.tiles_x;
  const int px = tx * TW + (int)(threadIdx.x % TW);
  const int py = ty * TH + (int)(threadIdx.x / TW);
  const bool inside = px < vp.width && py < vp.height;
  const float fx = (float)px, fy = (float)py;
  const uint2 range = ranges[gtile];

  float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, D = 0.0f;
  int32_t last = -1;
  uint32_t evals = 0, contribs = 0;
  bool done = !inside;
  for (uint32_t start = range.x; start < range.y; start += kThreads) {
    if (__syncthreads_count(done) == kThreads) break;
    const uint32_t j = start + threadIdx.x;
    if (j < range.y) {
      const uint32_t vi = pair_vals[j];
      s0[threadIdx.x] = rec0[vi];
      s1[threadIdx.x] = rec1[vi];
      s2[threadIdx.x] = rec2[vi];
    }
    __syncthreads();
    const int cnt = (int)min((uint32_t)kThreads, range.y - start);
    for (int k = 0; k < cnt && !done; ++k) {
      ++evals;
      const float4 g0 = s0[k];
      const float4 g1 = s1[k];
      const float power = gauss_power(__fsub_rn(fx, g0.x), __fsub_rn(fy, g0.y), g1.x, g1.y, g1.z);
      const float a = fminf(c.alpha_max, gauss_alpha_raw(g0.z, power));
      if (a < c.alpha_min) continue;
      const float Tn = __fmul_rn(T, __fsub_rn(1.0f, a));
      if (Tn < c.t_min) {
        done = true;
        break;
      }
      const float w = a * T;
      const float4 g2 = s2[k];
      C0 = fmaf(w, g2.x, C0);
      C1 = fmaf(w, g2.y, C1);
      C2 = fmaf(w, g2.z, C2);
      D = fmaf(w, g0.w, D);
      T = Tn;
      ++contribs;
      last = (int32_t)(start + k);
    }
  }
  if (inside) {
    const long long pix = vp.pixel_offset + (long long)py * vp.width + px;
    color[3 * pix + 0] = fmaf(T, c.bg[0], C0);
    color[3 * pix + 1] = fmaf(T, c.bg[1], C1);
    color[3 * pix + 2] = fmaf(T, c.bg[2], C2);
    depth[pix] = D;
    alpha_out[pix] = 1.0f - T;
    t_final[pix] = T;
    last_index[pix] = last;
  }
  // Evaluated (pixel, Gaussian) positions, for the roofline accounting.
  unsigned long long e = evals, n_c = contribs;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_xor_sync(0xffffffffu, e, o);
    n_c += __shfl_xor_sync(0xffffffffu, n_c, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s_eval[threadIdx.x >> 5] = e;
    s_contrib[threadIdx.x >> 5] = n_c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0, sc = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) {
      s += s_eval[w];
      sc += s_contrib[w];
    }
    atomicAdd(&counters->n_eval, s);
    atomicAdd(&counters->n_contrib, sc);
  }
}

// ------------------------------------------------------------------------------------------
// Backward blend.
// ------------------------------------------------------------------------------------------
template <int TW, int TH>
__global__ void __launch_bounds__(TW * TH) blend_backward_kernel(
    const __grid_constant__ Views views, const Consts c, const uint2* __restrict__ ranges,
    const uint32_t* __restrict__ pair_vals, const float4* __restrict__ rec0,
    const float4* __restrict__ rec1, const float4* __restrict__ rec2,
    const float* __restrict__ t_final, const int32_t* __restrict__ last_index,
    const float* __restrict__ d_color, const float* __restrict__ d_depth,
    const float* __restrict__ d_alpha, float* __restrict__ g2d) {
  constexpr int kThreads = TW * TH;
  __shared__ float4 s0[kThreads], s1[kThreads], s2[kThreads];
  __shared__ uint32_t s_vi[kThreads];
  __shared__ int s_max_last[kThreads / 32];
  const int gtile = blockIdx.x;
  const int v = view_of_tile(views, gtile);
  const ViewParams& vp = views.v[v];
  const int local = gtile - vp.tile_base;
  const int ty = local / vp.tiles_x, tx = local - ty * vp.tiles_x;
  const int px = tx * TW + (int)(threadIdx.x % TW);
  const int py = ty * TH + (int)(threadIdx.x / TW);
  const bool inside = px < vp.width && py < vp.height;
  const float fx = (float)px, fy = (float)py;
  const uint2 range = ranges[gtile];
  const int lane = threadIdx.x & 31;

  float Tfin = 1.0f, gC0 = 0.0f, gC1 = 0.0f, gC2 = 0.0f, gD = 0.0f, gA = 0.0f;
  int32_t last = -1;
  if (inside) {
    const long long pix = vp.pixel_offset + (long long)py * vp.width + px;
    Tfin = t_final[pix];
    last = last_index[pix];
    if (d_color) {
      gC0 = d_color[3 * pix + 0];
      gC1 = d_color[3 * pix + 1];
      gC2 = d_color[3 * pix + 2];
    }
    if (d_depth) gD = d_depth[pix];
    if (d_alpha) gA = d_alpha[pix];
  }
  // Only list positions up to the largest last-contributor index of the tile matter.
  int m = last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) s_max_last[threadIdx.x >> 5] = m;
  __syncthreads();
  int max_last = -1;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) max_last = max(max_last, s_max_last[w]);
  if (max_last < (int)range.x) return;

  float T = Tfin;                                   // transmittance after the current position
  float S0 = Tfin * c.bg[0], S1 = Tfin * c.bg[1], S2 = Tfin * c.bg[2];  // colour behind
  float SD = 0.0f;                                  // depth behind
  const int first = (int)range.x;
  for (int bend = max_last + 1; bend > first; bend -= kThreads) {
    const int bstart = max(first, bend - kThreads);
    __syncthreads();
    const int j = bstart + (int)threadIdx.x;
    if (j < bend) {
      const uint32_t vi = pair_vals[j];
      s_vi[threadIdx.x] = vi;
      s0[threadIdx.x] = rec0[vi];
      s1[threadIdx.x] = rec1[vi];
      s2[threadIdx.x] = rec2[vi];
    }
    __syncthreads();
    for (int jj = bend - 1; jj >= bstart; --jj) {
      const int k = jj - bstart;
      float g[10];
#pragma unroll
      for (int s = 0; s < 10; ++s) g[s] = 0.0f;
      bool contrib = false;
      if (jj <= last) {
        const float4 g0 = s0[k];
        const float4 g1 = s1[k];
        const float dx = __fsub_rn(fx, g0.x), dy = __fsub_rn(fy, g0.y);
        const float power = gauss_power(dx, dy, g1.x, g1.y, g1.z);
        const float oG = gauss_alpha_raw(g0.z, power);
        const float a = fminf(c.alpha_max, oG);
        if (a >= c.alpha_min) {
          contrib = true;
          const float om = __fsub_rn(1.0f, a);
          const float rom = 1.0f / om;
          T = T * rom;  // transmittance in front of this Gaussian
          const float w = a * T;
          const float4 g2 = s2[k];
          g[kGR] = gC0 * w;
          g[kGG] = gC1 * w;
          g[kGB] = gC2 * w;
          g[kGZ] = gD * w;
          float dLda = gC0 * (g2.x * T - S0 * rom) + gC1 * (g2.y * T - S1 * rom) +
                       gC2 * (g2.z * T - S2 * rom);
          dLda += gD * (g0.w * T - SD * rom);
          dLda += gA * Tfin * rom;
          S0 = fmaf(w, g2.x, S0);
          S1 = fmaf(w, g2.y, S1);
          S2 = fmaf(w, g2.z, S2);
          SD = fmaf(w, g0.w, SD);
          if (oG < c.alpha_max) {
            const float G = __expf(power);
            g[kGOp] = dLda * G;
            const float dp = dLda * a;  // d alpha / d power = o G = alpha
            g[kGMx] = dp * (g1.x * dx + g1.y * dy);
            g[kGMy] = dp * (g1.y * dx + g1.z * dy);
            g[kGCa] = -0.5f * dp * dx * dx;
            g[kGCb] = -dp * dx * dy;
            g[kGCc] = -0.5f * dp * dy * dy;
          }
        }
      }
      if (__any_sync(0xffffffffu, contrib)) {
#pragma unroll
        for (int s = 0; s < 10; ++s) {
          float x = g[s];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
          g[s] = x;
        }
        if (lane < 10) {
          float val = g[0];
#pragma unroll
          for (int s = 1; s < 10; ++s) val = (lane == s) ? g[s] : val;
          atomicAdd(g2d + (size_t)s_vi[k] * kG2Stride + lane, val);
        }
      }
    }
  }
}

template <int TW, int TH>
cudaError_t launch_blends_t(bool forward, const Views& views, const Consts& c,
                            const uint2* ranges, const uint32_t* pair_vals, const float4* rec0,
                            const float4* rec1, const float4* rec2, float* color, float* depth,
                            float* alpha, float* t_final, int32_t* last_index,
                            const float* d_color, const float* d_depth, const float* d_alpha,
                            float* g2d, Counters* counters, cudaStream_t stream) {
  if (views.total_tiles == 0) return cudaSuccess;
  if (forward) {
    blend_forward_kernel<TW, TH><<<views.total_tiles, TW * TH, 0, stream>>>(
        views, c, ranges, pair_vals, rec0, rec1, rec2, color, depth, alpha, t_final,
        last_index, counters);
  } else {
    blend_backward_kernel<TW, TH><<<views.total_tiles, TW * TH, 0, stream>>>(
        views, c, ranges, pair_vals, rec0, rec1, rec2, t_final, last_index, d_color, d_depth,
        d_alpha, g2d);
  }
  RGS_LAUNCHED();
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_duplicate(const Views& views, int n, const uint32_t* order,
                             const uint32_t* offsets, const uint32_t* ntiles, const float4* rec0,
                             const float4* rec1, int64_t visible_cap, uint32_t capacity,
                             uint32_t* keys, uint32_t* vals, Counters* counters,
                             cudaStream_t stream) {
  if (visible_cap > 0) {
    const unsigned blocks = (unsigned)((visible_cap + kDupThreads - 1) / kDupThreads);
    duplicate_kernel<<<blocks, kDupThreads, 0, stream>>>(views, n, order, offsets, ntiles, rec0,
                                                         rec1, counters, capacity, keys, vals,
                                                         counters);
    RGS_LAUNCHED();
  }
  store_pair_count_kernel<<<1, 1, 0, stream>>>(counters, capacity);
  RGS_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_tile_ranges(const uint32_t* keys, const Counters* counters, uint2* ranges,
                               int total_tiles, uint32_t capacity, cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)total_tiles, stream);
  if (e != cudaSuccess) return e;
  if (capacity > 0)
    tile_ranges_kernel<<<(capacity + 255) / 256, 256, 0, stream>>>(keys, counters,
                                                                   (uint32_t)total_tiles, ranges);
    RGS_LAUNCHED();
  return cudaGetLastError();
}

cudaError_t launch_blend(bool forward, const Views& views, const Consts& c, const uint2* ranges,
                         const uint32_t* pair_vals, const float4* rec0, const float4* rec1,
                         const float4* rec2, float* color, float* depth, float* alpha,
                         float* t_final, int32_t* last_index, const float* d_color,
                         const float* d_depth, const float* d_alpha, float* g2d,
                         Counters* counters, cudaStream_t stream) {
  const int tw = views.tile_w, th = views.tile_h;
#define RGS_BLEND(W, H)                                                                          \
  return launch_blends_t<W, H>(forward, views, c, ranges, pair_vals, rec0, rec1, rec2, color,   \
                               depth, alpha, t_final, last_index, d_color, d_depth, d_alpha, g2d, \
                               counters, stream)
  if (tw == 8 && th == 8) RGS_BLEND(8, 8);
  if (tw == 32 && th == 8) RGS_BLEND(32, 8);
  RGS_BLEND(16, 16);
#undef RGS_BLEND
}

}  // namespace rgs
