// raster.cu -- pair duplication, tile ranges, and the forward / backward alpha blends.
//
// Forward blend (Section 3.1, Eq. alpha; Section 3.2.2): one CTA per (view, tile), the tiles
// taken longest run first; the tile's Gaussians, already in near-to-far order, are staged
// through shared memory in batches of one Gaussian per thread and every thread composites its
// pixels front to back with early exit.
// Backward blend: the same tiles are walked back to front from each pixel's last contributor,
// recovering the transmittance by division from the saved final value, so no per-pixel list is
// stored; per-Gaussian screen-space gradient sums are reduced per warp through shared memory, in
// groups of Gaussians, before one atomic per value and Gaussian.
#include <algorithm>
#include <type_traits>

#include "rgs_internal.cuh"

namespace rgs {
namespace {

constexpr int kDupThreads = 256;
constexpr int kDupWarps = kDupThreads / 32;
// Footprints of up to this many tiles are walked by their own lane into a per-warp staging
// buffer in shared memory, from which the warp writes them out coalesced; larger ones are walked
// by the whole warp, up to 32 tile rows at a time with the rows' tiles dealt out over the lanes.
constexpr uint32_t kDupSerialMax = 32;
constexpr int kDupStage = 32 * kDupSerialMax;  // staged pairs per warp and round

// First lane whose inclusive count exceeds idx (idx < the warp total).
__device__ __forceinline__ int lane_of(int incl, int idx) {
  int lo = 0, hi = 31;
#pragma unroll
  for (int step = 0; step < 5; ++step) {
    const int mid = (lo + hi) >> 1;
    if (__shfl_sync(0xffffffffu, incl, mid) > idx) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// One (tile, vi) pair per tile touched by each visible entry, into the entry's slots
// [offsets[k], offsets[k] + ntiles[vi]) of the pair list (so the list is in the entries' depth
// order). The counting pass in the projection visits the same tiles, so every slot is written;
// if that ever failed, the unused slots get the out-of-range key total_tiles, which sorts last
// and owns no tile range.
__global__ void __launch_bounds__(kDupThreads) duplicate_kernel(
    const __grid_constant__ Views views, int n, const uint32_t* __restrict__ order,
    const uint32_t* __restrict__ offsets, const uint32_t* __restrict__ ntiles,
    const float4* __restrict__ rec0, const float4* __restrict__ rec1, float log2_alpha_min,
    uint32_t visible_cap, uint32_t capacity, uint32_t* __restrict__ keys,
    uint32_t* __restrict__ vals, Counters* __restrict__ counters) {
  chain_wait();
  __shared__ uint32_t s_stage[kDupWarps][kDupStage];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* stage = s_stage[warp];
  // The sorted list holds at most visible_cap entries; more (only possible under stream
  // capture) are recorded in the status word. The pair count the tile sort uses is stored here.
  const uint32_t n_visible_raw = counters->n_visible;
  const uint32_t n_visible = min(n_visible_raw, visible_cap);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (n_visible_raw > visible_cap) atomicOr(&counters->status, (uint32_t)kStatusVisibleOverflow);
    counters->n_visible_kept = n_visible;
    const uint32_t p = counters->n_pairs;
    counters->n_pairs_stored = p < capacity ? p : capacity;
  }
  const uint32_t sentinel = (uint32_t)views.total_tiles;
  // Lane l of global warp w takes entry k = round * 32 W + l W + w (W warps in the grid): the
  // nearest entries, whose footprints are the largest, come first in the depth order and are
  // spread one per warp instead of filling the first warps.
  const uint32_t n_warps = gridDim.x * kDupWarps;
  const uint32_t gwarp = blockIdx.x * kDupWarps + warp;
  for (uint64_t round_base = 0; round_base + gwarp < n_visible; round_base += 32ull * n_warps) {
    const uint64_t k64 = round_base + (uint64_t)lane * n_warps + gwarp;
    const uint32_t k = k64 < n_visible ? (uint32_t)k64 : n_visible;
    uint32_t vi = 0, begin = 0, cnt = 0;
    bool ok = false;
    if (k < n_visible) {
      vi = order[k];
      begin = offsets[k];
      cnt = ntiles[vi];
      if ((uint64_t)begin + cnt > capacity)
        atomicOr(&counters->status, (uint32_t)kStatusPairOverflow);
    }
    const int v = (int)(vi / (uint32_t)max(n, 1));
    // Every lane sets up its own entry's tile cover once; a large footprint's cover is then
    // handed to the whole warp by shuffles instead of being recomputed by every lane.
    TileCover tc;
    if (k < n_visible) {
      Ellipse e;
      const ViewParams& vp = views.v[v];
      ok = make_ellipse(rec0[vi], rec1[vi], log2_alpha_min, e) &&
           tc.init(e, views.tile_w, views.tile_h, vp.tiles_x, vp.tiles_y);
    }
    // Small footprints: stage, then write out.
    const bool small = k < n_visible && cnt <= kDupSerialMax;
    const int c_small = small ? (int)cnt : 0;
    int incl = c_small;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int staged = __shfl_sync(0xffffffffu, incl, 31);
    if (small) {
      int q = incl - c_small;
      const int q_end = incl;
      if (ok) {
        const ViewParams& vp = views.v[v];
        for (int ty = tc.ty0; ty <= tc.ty1; ++ty) {
          int tx0, tx1;
          if (!tc.span(ty, tx0, tx1)) continue;
          const uint32_t row = (uint32_t)(vp.tile_base + ty * vp.tiles_x);
          for (int tx = tx0; tx <= tx1 && q < q_end; ++tx) stage[q++] = row + tx;
        }
      }
      for (; q < q_end; ++q) stage[q] = sentinel;
    }
    __syncwarp();
    for (int b = 0; b < staged; b += 32) {
      const int idx = b + lane;
      const int src = lane_of(incl, idx);
      const int src_incl = __shfl_sync(0xffffffffu, incl, src);
      const int src_cnt = __shfl_sync(0xffffffffu, c_small, src);
      const uint32_t src_begin = __shfl_sync(0xffffffffu, begin, src);
      const uint32_t src_vi = __shfl_sync(0xffffffffu, vi, src);
      if (idx < staged) {
        const uint32_t off = src_begin + (uint32_t)(idx - (src_incl - src_cnt));
        if (off < capacity) {
          keys[off] = stage[idx];
          vals[off] = src_vi;
        }
      }
    }
    __syncwarp();
    // Large footprints: the whole warp, one entry at a time.
    unsigned big = __ballot_sync(0xffffffffu, k < n_visible && cnt > kDupSerialMax);
    while (big) {
      const int src = __ffs(big) - 1;
      big &= big - 1;
      const uint32_t vib = __shfl_sync(0xffffffffu, vi, src);
      const uint32_t bbeg = __shfl_sync(0xffffffffu, begin, src);
      const uint32_t bend = min(bbeg + __shfl_sync(0xffffffffu, cnt, src), capacity);
      uint32_t done = 0;  // pairs written so far (rows before the current chunk)
      if (__shfl_sync(0xffffffffu, (int)ok, src)) {
        const TileCover tb = tc.broadcast(src);
        const ViewParams& vp = views.v[__shfl_sync(0xffffffffu, v, src)];
        {
          for (int r0 = tb.ty0; r0 <= tb.ty1; r0 += 32) {
            // Lane l takes tile row r0 + l; the rows' tiles are then dealt out 32 at a time.
            const int ty = r0 + lane;
            int tx0 = 0, tx1 = -1;
            if (ty > tb.ty1 || !tb.span(ty, tx0, tx1)) {
              tx0 = 0;
              tx1 = -1;
            }
            const int w = tx1 - tx0 + 1;
            int rincl = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
              const int y = __shfl_up_sync(0xffffffffu, rincl, o);
              if (lane >= o) rincl += y;
            }
            const int total = __shfl_sync(0xffffffffu, rincl, 31);
            for (int b = 0; b < total; b += 32) {
              const int idx = b + lane;
              const int row = lane_of(rincl, idx);
              const int r_incl = __shfl_sync(0xffffffffu, rincl, row);
              const int r_w = __shfl_sync(0xffffffffu, w, row);
              const int r_tx0 = __shfl_sync(0xffffffffu, tx0, row);
              const uint32_t off = bbeg + done + (uint32_t)idx;
              if (idx < total && off < bend) {
                keys[off] = (uint32_t)(vp.tile_base + (r0 + row) * vp.tiles_x + r_tx0 + idx -
                                       (r_incl - r_w));
                vals[off] = vib;
              }
            }
            done += (uint32_t)total;
          }
        }
      }
      for (uint32_t off = bbeg + done + lane; off < bend; off += 32) {
        keys[off] = sentinel;
        vals[off] = vib;
      }
    }
  }
}

// Keeps at most `capacity` visible entries (the sorted-list capacity under stream capture): the
// entries beyond it are dropped from this forward and the overflow is recorded.
__global__ void store_pair_count_kernel(Counters* counters, uint32_t capacity) {
  chain_wait();
  const uint32_t p = counters->n_pairs;
  counters->n_pairs_stored = p < capacity ? p : capacity;
  if (counters->n_visible > 0) atomicOr(&counters->status, (uint32_t)kStatusVisibleOverflow);
  counters->n_visible_kept = 0;
}

// ------------------------------------------------------------------------------------------
// Staging of a batch of Gaussians in shared memory, with the row terms of the tile's anchor row
// y_a (anchor_terms). For an even number of pixels per thread every per-Gaussian operand is
// stored twice, as (x, x) pairs, so the packed f32x2 arithmetic of two pixels reads its broadcast
// operands straight from shared memory:
//   [0] (mx hi, mx hi), (mx lo, mx lo)   [1] (l11, l11), (c21, c21)
//   [2] (l21, l21), (l22, l22)           [3] (s_a, s_a), (-log2 o, -log2 o)
//   [4] (r, r), (g, g)                   [5] (b, b), (z, z)
// With one pixel per thread rows 0..2 hold (mx hi, mx lo, l11, c21), (l21, l22, s_a, -log2 o)
// and rec2 as float4.
// ------------------------------------------------------------------------------------------
template <int R, int N>
__device__ __forceinline__ void stage_gaussian(ulonglong2 (&sp)[R][N], int t, float4 r0,
                                               float4 r1, float4 r2, float y_a) {
  const AnchorTerms at = anchor_terms(r0, r1, y_a);
  const float nlo = -r1.w;
  if constexpr (R == 6) {
    sp[0][t] = make_ulonglong2(f2_make(r0.x, r0.x), f2_make(r0.z, r0.z));
    sp[1][t] = make_ulonglong2(f2_make(r1.x, r1.x), f2_make(at.c21, at.c21));
    sp[2][t] = make_ulonglong2(f2_make(r1.y, r1.y), f2_make(r1.z, r1.z));
    sp[3][t] = make_ulonglong2(f2_make(at.s_a, at.s_a), f2_make(nlo, nlo));
    sp[4][t] = make_ulonglong2(f2_make(r2.x, r2.x), f2_make(r2.y, r2.y));
    sp[5][t] = make_ulonglong2(f2_make(r2.z, r2.z), f2_make(r2.w, r2.w));
  } else {
    reinterpret_cast<float4*>(sp[0])[t] = make_float4(r0.x, r0.z, r1.x, at.c21);
    reinterpret_cast<float4*>(sp[1])[t] = make_float4(r1.y, r1.z, at.s_a, nlo);
    reinterpret_cast<float4*>(sp[2])[t] = r2;
  }
}

// ------------------------------------------------------------------------------------------
// Forward blend. A CTA covers one TW x TH tile with TW * TH / PPT threads; thread t owns the
// PPT vertically adjacent pixels (x, y0 + k), k < PPT, of column x = t % TW, so every Gaussian
// staged in shared memory is read once per thread and evaluated for PPT pixels. With an even PPT
// the pixels go in pairs through packed f32x2 arithmetic: a pixel that does not composite a
// Gaussian gets weight +0, which leaves its colour, depth and transmittance bit-identical, so the
// result equals the one-pixel-per-thread kernel's. Alpha is zeroed where it is below alpha_min
// before the weight is formed, so a live pixel composites its weight unconditionally and only
// the rare stop (its transmittance would fall below t_min) branches. A pixel that has stopped, or
// lies off the image, gets a row offset of 1e18 from the anchor row: its exponent is then
// astronomically large, its alpha 0, and it keeps its colour and transmittance with no per-pixel
// test in the loop.
// For the backward each pixel saves the last list position it may composite: the one before its
// stop, or the tile's last position if it never stops (between its last contributor and that
// position no Gaussian covers it, so the backward takes the same decisions there).
// ------------------------------------------------------------------------------------------
template <int TW, int TH, int PPT>
__global__ void __launch_bounds__(TW * TH / PPT) blend_forward_kernel(
    const __grid_constant__ Views views, const Consts c, const uint2* __restrict__ ranges,
    const uint32_t* __restrict__ pair_vals, const float4* __restrict__ rec0,
    const float4* __restrict__ rec1, const float4* __restrict__ rec2, float* __restrict__ color,
    float* __restrict__ depth, float* __restrict__ alpha_out, float* __restrict__ t_final,
    int32_t* __restrict__ last_index, const uint32_t* __restrict__ tile_order,
    Counters* __restrict__ counters) {
  chain_wait();
  constexpr int kThreads = TW * TH / PPT;
  constexpr bool kPacked = PPT % 2 == 0;
  constexpr int P2 = kPacked ? PPT / 2 : 1;
  static_assert(kThreads % 32 == 0, "whole warps only");
  __shared__ ulonglong2 sp[kPacked ? 6 : 3][kThreads];
  __shared__ unsigned long long s_eval[kThreads / 32];
  const int gtile = (int)tile_order[blockIdx.x];
  const int v = view_of_tile(views, gtile);
  const ViewParams& vp = views.v[v];
  const int local = gtile - vp.tile_base;
  const int ty = local / vp.tiles_x, tx = local - ty * vp.tiles_x;
  const int px = tx * TW + (int)(threadIdx.x % TW);
  const int py0 = ty * TH + (int)(threadIdx.x / TW) * PPT;
  const float fx = (float)px;
  // Anchor row of the tile's row terms, and the thread's first row relative to it.
  const float y_a = (float)(ty * TH + TH / 2);
  const int r0_ = (int)(threadIdx.x / TW) * PPT - TH / 2;
  const uint2 range = ranges[gtile];

  float T[PPT], C0[PPT], C1[PPT], C2[PPT], D[PPT];
  f32x2 T2[P2], C02[P2], C12[P2], C22[P2], D2[P2], FR[P2];
  uint32_t visited_end[PPT];  // one past the last list position the pixel visited
  bool done[PPT];             // the pixel has stopped (or is off the image)
  int live = 0;               // pixels of the thread that have not stopped
  // Row offset of a pixel that takes no further part: every Gaussian's alpha there is 0.
  constexpr float kFarRow = 1e18f;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    done[k] = !(px < vp.width && py0 + k < vp.height);
    T[k] = 1.0f;
    C0[k] = C1[k] = C2[k] = D[k] = 0.0f;
    visited_end[k] = done[k] ? range.x : range.y;
    live += done[k] ? 0 : 1;
  }
#pragma unroll
  for (int q = 0; q < P2; ++q) {
    const int k0 = kPacked ? 2 * q : 0, k1 = kPacked ? 2 * q + 1 : 0;
    T2[q] = f2_make(1.0f, 1.0f);
    C02[q] = C12[q] = C22[q] = D2[q] = f2_make(0.0f, 0.0f);
    FR[q] = f2_make(done[k0] ? kFarRow : (float)(r0_ + k0), done[k1] ? kFarRow : (float)(r0_ + k1));
  }
  const f32x2 FX = f2_make(fx, fx);

  // One staged Gaussian (list position pos, slot g) against the thread's pixel pairs.
  auto composite_pairs = [&](uint32_t pos, int g) {
    const ulonglong2 X = sp[0][g], L1 = sp[1][g], L2 = sp[2][g], L3 = sp[3][g];
    const ulonglong2 CA = sp[4 % (kPacked ? 6 : 3)][g], CB = sp[5 % (kPacked ? 6 : 3)][g];
    // Whitened offset t at the anchor row of the thread's column (Eq. alpha's exponent).
    const f32x2 dx = f2_sub(f2_sub(FX, X.x), X.y);
    const f32x2 TA = f2_fma(L1.x, dx, L1.y);
#pragma unroll
    for (int q = 0; q < P2; ++q) {
      const int k0 = 2 * q, k1 = 2 * q + 1;
      const f32x2 tt = f2_fma(FR[q], L2.x, TA);
      const f32x2 ss = f2_fma(FR[q], L2.y, L3.x);
      const f32x2 nq = f2_fma(tt, tt, f2_fma(ss, ss, L3.y));  // -log2(o G)
      const float a0 = fminf(c.alpha_max, ex2_neg_approx(f2_lo(nq)));
      const float a1 = fminf(c.alpha_max, ex2_neg_approx(f2_hi(nq)));
      // w = alpha T and the transmittance after this Gaussian T' = T - w; an uncovered pixel
      // (alpha < alpha_min) has w = +0 and T' = T.
      f32x2 w = f2_mul(f2_make(a0 >= c.alpha_min ? a0 : 0.0f, a1 >= c.alpha_min ? a1 : 0.0f),
                       T2[q]);
      f32x2 Tn = f2_sub(T2[q], w);
      const bool stop0 = f2_lo(Tn) < c.t_min, stop1 = f2_hi(Tn) < c.t_min;
      if (stop0 || stop1) {  // once per pixel: it composites nothing from here on
        const float t0 = f2_lo(T2[q]), t1 = f2_hi(T2[q]);
        w = f2_make(stop0 ? 0.0f : f2_lo(w), stop1 ? 0.0f : f2_hi(w));
        Tn = f2_make(stop0 ? t0 : f2_lo(Tn), stop1 ? t1 : f2_hi(Tn));
        FR[q] = f2_make(stop0 ? kFarRow : f2_lo(FR[q]), stop1 ? kFarRow : f2_hi(FR[q]));
        if (stop0) visited_end[k0] = pos + 1;
        if (stop1) visited_end[k1] = pos + 1;
        done[k0] = done[k0] || stop0;
        done[k1] = done[k1] || stop1;
        live -= (int)stop0 + (int)stop1;
      }
      C02[q] = f2_fma(w, CA.x, C02[q]);
      C12[q] = f2_fma(w, CA.y, C12[q]);
      C22[q] = f2_fma(w, CB.x, C22[q]);
      D2[q] = f2_fma(w, CB.y, D2[q]);
      T2[q] = Tn;
    }
  };

  for (uint32_t start = range.x; start < range.y; start += kThreads) {
    if (__syncthreads_count(live == 0) == kThreads) break;
    const uint32_t j = start + threadIdx.x;
    if (j < range.y) {
      const uint32_t vi = pair_vals[j];
      stage_gaussian(sp, threadIdx.x, rec0[vi], rec1[vi], rec2[vi], y_a);
    }
    __syncthreads();
    const int cnt = (int)min((uint32_t)kThreads, range.y - start);
    // The warp leaves the batch together, once none of its pixels is live: a stopped pixel
    // composites nothing more (its alpha is 0), and a loop without per-thread exits ran 9 %
    // faster than one that let each thread leave on its own.
    for (int g = 0; g < cnt; ++g) {
      if (!__any_sync(0xffffffffu, live > 0)) break;
      const uint32_t pos = start + g;
      if constexpr (kPacked) {
        // Always with the clamp: a warp-uniform clamp-free variant (as in the backward) made
        // this loop slower (two copies of its body), measured 3.64 against 3.21 ms on the
        // 16-view 1080p window.
        composite_pairs(pos, g);
      } else {
        const float4 g0 = reinterpret_cast<const float4*>(sp[0])[g];
        const float4 g1 = reinterpret_cast<const float4*>(sp[1])[g];
        const float4 g2 = reinterpret_cast<const float4*>(sp[2])[g];
        const float ta = __fmaf_rn(g0.z, __fsub_rn(__fsub_rn(fx, g0.x), g0.y), g0.w);
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          if (!done[k]) {
            const float nq = neg_log2_og(ta, g1.z, g1.x, g1.y, g1.w, (float)(r0_ + k));
            const float a = fminf(c.alpha_max, ex2_neg_approx(nq));
            if (a >= c.alpha_min) {
              const float w = __fmul_rn(a, T[k]);
              const float Tn = __fsub_rn(T[k], w);
              if (Tn < c.t_min) {
                done[k] = true;
                visited_end[k] = pos + 1;
                --live;
              } else {
                C0[k] = fmaf(w, g2.x, C0[k]);
                C1[k] = fmaf(w, g2.y, C1[k]);
                C2[k] = fmaf(w, g2.z, C2[k]);
                D[k] = fmaf(w, g2.w, D[k]);
                T[k] = Tn;
              }
            }
          }
        }
      }
    }
  }
  if constexpr (kPacked) {
#pragma unroll
    for (int q = 0; q < P2; ++q) {
      T[2 * q] = f2_lo(T2[q]);
      T[2 * q + 1] = f2_hi(T2[q]);
      C0[2 * q] = f2_lo(C02[q]);
      C0[2 * q + 1] = f2_hi(C02[q]);
      C1[2 * q] = f2_lo(C12[q]);
      C1[2 * q + 1] = f2_hi(C12[q]);
      C2[2 * q] = f2_lo(C22[q]);
      C2[2 * q + 1] = f2_hi(C22[q]);
      D[2 * q] = f2_lo(D2[q]);
      D[2 * q + 1] = f2_hi(D2[q]);
    }
  }
  uint32_t evals = 0;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    evals += visited_end[k] - range.x;
    const int py = py0 + k;
    if (px < vp.width && py < vp.height) {
      const long long pix = vp.pixel_offset + (long long)py * vp.width + px;
      color[3 * pix + 0] = fmaf(T[k], c.bg[0], C0[k]);
      color[3 * pix + 1] = fmaf(T[k], c.bg[1], C1[k]);
      color[3 * pix + 2] = fmaf(T[k], c.bg[2], C2[k]);
      depth[pix] = D[k];
      alpha_out[pix] = 1.0f - T[k];
      t_final[pix] = T[k];
      // The last position the pixel may composite (stop position - 1, or the tile's last).
      last_index[pix] = done[k] ? (int32_t)visited_end[k] - 2 : (int32_t)range.y - 1;
    }
  }
  // Visited (pixel, Gaussian) positions, for the roofline accounting.
  unsigned long long e = evals;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0) s_eval[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) s += s_eval[w];
    atomicAdd(&counters->n_eval, s);
  }
}

// ------------------------------------------------------------------------------------------
// Per-warp reduction of the visited Gaussians' gradient sums through shared memory. Each visit
// writes the lane's kVals partial sums as one column of kVals rows (row b * kVals + k for the
// b-th Gaussian of the group, RedLayout); after kBatch visits (or at the end of a staged batch)
// every lane adds up whole rows (eight 16-byte reads of a row padded to 36 floats, so that both
// the column writes and the row reads are free of bank conflicts) and parks the row total in
// the padding. Lane b then turns Gaussian b's totals into its whitened moments and issues the
// atomics. Per visit this costs kVals shared stores and a share of the row sums, in place of a
// shuffle butterfly with its selects after every Gaussian.
//
// The lane's values: k = 0..2: sdp, sr, srr (the sums of dp, dp r and dp r^2 over its pixels,
// r the row offset from the tile's anchor row), k = 3..5: t_a sdp, t_a sr, t_a^2 sdp (t_a the
// whitened offset of its column at the anchor row), k = 6..8 (9): the colour (depth) weights.
// ------------------------------------------------------------------------------------------
constexpr int kRedPad = 36;

template <bool kAux>
struct RedLayout {
  static constexpr int kVals = kAux ? 10 : 9;
  static constexpr int kBatch = kAux ? 6 : 7;  // kVals * kBatch <= 64: two row passes
  static constexpr int kRows = kVals * kBatch;
};

// Adds up row r (32 lane values) and parks the total in its first padding float.
__device__ __forceinline__ void reduce_row(float* red, int r) {
  const ulonglong2* row = reinterpret_cast<const ulonglong2*>(red + r * kRedPad);
  f32x2 s[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const ulonglong2 v = row[c];
    s[c] = f2_add(v.x, v.y);
  }
#pragma unroll
  for (int h = 4; h > 0; h >>= 1)
#pragma unroll
    for (int c = 0; c < h; ++c) s[c] = f2_add(s[c], s[c + h]);
  red[r * kRedPad + 32] = f2_lo(s[0]) + f2_hi(s[0]);
}

// ------------------------------------------------------------------------------------------
// Backward blend (same pixel layout as the forward).
// ------------------------------------------------------------------------------------------
// kAux: a depth or accumulated-opacity upstream gradient is present. Without one (a colour-only
// loss) the per-pixel depth / opacity gradient state and its arithmetic drop out; the results
// are those of the general kernel with those gradients zero.
template <int TW, int TH, int PPT, bool kAux>
__global__ void __launch_bounds__(TW * TH / PPT) blend_backward_kernel(
    const __grid_constant__ Views views, const Consts c, const uint2* __restrict__ ranges,
    const uint32_t* __restrict__ pair_vals, const float4* __restrict__ rec0,
    const float4* __restrict__ rec1, const float4* __restrict__ rec2,
    const float* __restrict__ t_final, const int32_t* __restrict__ last_index,
    const float* __restrict__ d_color, const float* __restrict__ d_depth,
    const float* __restrict__ d_alpha, const uint32_t* __restrict__ tile_order,
    float* __restrict__ g2d) {
  chain_wait();
  constexpr int kThreads = TW * TH / PPT;
  constexpr bool kPacked = PPT % 2 == 0;
  constexpr int P2 = kPacked ? PPT / 2 : 1;
  static_assert(kThreads % 32 == 0, "whole warps only");
  using RL = RedLayout<kAux>;
  __shared__ ulonglong2 sp[kPacked ? 6 : 3][kThreads];
  __shared__ uint32_t s_vi[kThreads];
  __shared__ int s_max_last[kThreads / 32];
  __shared__ __align__(16) float s_red[kThreads / 32][RL::kRows * kRedPad];
  const int gtile = (int)tile_order[blockIdx.x];
  const int v = view_of_tile(views, gtile);
  const ViewParams& vp = views.v[v];
  const int local = gtile - vp.tile_base;
  const int ty = local / vp.tiles_x, tx = local - ty * vp.tiles_x;
  const int px = tx * TW + (int)(threadIdx.x % TW);
  const int py0 = ty * TH + (int)(threadIdx.x / TW) * PPT;
  const float fx = (float)px;
  // Anchor row of the tile's row terms, and the thread's first row relative to it (as in the
  // forward, so both blends compute every pixel's exponent to the same bits).
  const float y_a = (float)(ty * TH + TH / 2);
  const int r0_ = (int)(threadIdx.x / TW) * PPT - TH / 2;
  const uint2 range = ranges[gtile];
  const int lane = threadIdx.x & 31;
  float* const red = s_red[threadIdx.x >> 5];

  // Per pixel: transmittance behind the current position, the upstream gradients, and
  // U = sum_ch dL/dC_ch S_ch + dL/dD S_D, where S is the colour / depth composited behind the
  // current position (background included), so dL/dalpha = T q + (dL/dA T_final - U) / (1 - alpha)
  // with q = dL/dC . c + dL/dD z.
  float T[PPT], U[PPT], gC0[PPT], gC1[PPT], gC2[PPT], gD[PPT], gAT[PPT];
  int32_t last[PPT];
  int thread_last = -1;
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    float Tfin = 1.0f;
    gC0[k] = gC1[k] = gC2[k] = gD[k] = gAT[k] = 0.0f;
    last[k] = -1;
    const int py = py0 + k;
    if (px < vp.width && py < vp.height) {
      const long long pix = vp.pixel_offset + (long long)py * vp.width + px;
      Tfin = t_final[pix];
      last[k] = last_index[pix];
      if (d_color) {
        gC0[k] = d_color[3 * pix + 0];
        gC1[k] = d_color[3 * pix + 1];
        gC2[k] = d_color[3 * pix + 2];
      }
      if (kAux && d_depth) gD[k] = d_depth[pix];
      if (kAux && d_alpha) gAT[k] = d_alpha[pix] * Tfin;
    }
    T[k] = Tfin;
    U[k] = Tfin * (gC0[k] * c.bg[0] + gC1[k] * c.bg[1] + gC2[k] * c.bg[2]);
    thread_last = max(thread_last, last[k]);
  }
  // The same state as (pixel 2q, pixel 2q + 1) pairs for the packed arithmetic.
  f32x2 T2[P2], U2[P2], GC02[P2], GC12[P2], GC22[P2], GD2[P2], GAT2[P2], FR[P2];
#pragma unroll
  for (int q = 0; q < P2; ++q) {
    const int k0 = kPacked ? 2 * q : 0, k1 = kPacked ? 2 * q + 1 : 0;
    T2[q] = f2_make(T[k0], T[k1]);
    U2[q] = f2_make(U[k0], U[k1]);
    GC02[q] = f2_make(gC0[k0], gC0[k1]);
    GC12[q] = f2_make(gC1[k0], gC1[k1]);
    GC22[q] = f2_make(gC2[k0], gC2[k1]);
    GD2[q] = f2_make(gD[k0], gD[k1]);
    GAT2[q] = f2_make(gAT[k0], gAT[k1]);
    FR[q] = f2_make((float)(r0_ + k0), (float)(r0_ + k1));
  }
  const f32x2 FX = f2_make(fx, fx), ONE2 = f2_make(1.0f, 1.0f), ZERO2 = f2_make(0.0f, 0.0f);
  // Only list positions up to the largest last-contributor index of the tile matter.
  int m = thread_last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) s_max_last[threadIdx.x >> 5] = m;
  // At or below the smallest last-contributor index of the warp every pixel of the warp is
  // live, and the per-pixel test of the list position drops out (warp-uniform).
  int thread_min_last = last[0];
#pragma unroll
  for (int k = 1; k < PPT; ++k) thread_min_last = min(thread_min_last, last[k]);
  const int warp_min_last = __reduce_min_sync(0xffffffffu, thread_min_last);
  __syncthreads();
  int max_last = -1;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) max_last = max(max_last, s_max_last[w]);
  if (max_last < (int)range.x) return;

  // One Gaussian (list position jj, staged at g) against the thread's pixels; kCheckLast tests
  // each pixel's last-contributor index.
  // kClamp: the Gaussian may reach alpha_max somewhere (clamp, and no gradient through a
  // clamped alpha); without it neither can happen and both tests drop out. The lane's partial
  // sums go to column `lane` of the rows from `rows` on (zeros where it covers nothing).
  auto visit = [&](int jj, int g, float* rows, auto check_last, auto clamp_tag) {
    constexpr bool kCheckLast = decltype(check_last)::value;
    constexpr bool kClamp = decltype(clamp_tag)::value;
    (void)kClamp;  // the one-pixel path always clamps
    // Per-thread sums of dp = dL/dpower over the thread's pixels, weighted by their row offset
    // r from the anchor row: sdp = sum dp, sr = sum dp r, srr = sum dp r^2. Every pixel of the
    // column has w = (t, s) = (t_a + r l21, s_a + r l22), so the whitened moments follow from
    // these three and t_a once per Gaussian.
    float sdp = 0.0f, sr = 0.0f, srr = 0.0f, ta = 0.0f, gr = 0.0f, gg = 0.0f, gb = 0.0f,
          gz = 0.0f;
    if (!kCheckLast || jj <= thread_last) {
      if constexpr (kPacked) {
        const ulonglong2 X = sp[0][g], L1 = sp[1][g], L2 = sp[2][g], L3 = sp[3][g];
        const ulonglong2 CA = sp[4 % (kPacked ? 6 : 3)][g], CB = sp[5 % (kPacked ? 6 : 3)][g];
        const f32x2 dx2 = f2_sub(f2_sub(FX, X.x), X.y);
        const f32x2 TA = f2_fma(L1.x, dx2, L1.y);
        f32x2 aR = ZERO2, aG = ZERO2, aB = ZERO2, aZ = ZERO2, mP = ZERO2, mY = ZERO2,
              mYY = ZERO2;
        (void)aZ;
#pragma unroll
        for (int q = 0; q < P2; ++q) {
          const int k0 = 2 * q, k1 = 2 * q + 1;
          const f32x2 tt = f2_fma(FR[q], L2.x, TA);
          const f32x2 ss = f2_fma(FR[q], L2.y, L3.x);
          const f32x2 nq = f2_fma(tt, tt, f2_fma(ss, ss, L3.y));  // -log2(o G)
          const float oG0 = ex2_neg_approx(f2_lo(nq)), oG1 = ex2_neg_approx(f2_hi(nq));
          const float a0 = kClamp ? fminf(c.alpha_max, oG0) : oG0;
          const float a1 = kClamp ? fminf(c.alpha_max, oG1) : oG1;
          const bool cov0 = (!kCheckLast || jj <= last[k0]) && a0 >= c.alpha_min;
          const bool cov1 = (!kCheckLast || jj <= last[k1]) && a1 >= c.alpha_min;
          // A pixel this Gaussian does not cover gets alpha 0 and 1 / (1 - alpha) = 1 (the
          // hardware reciprocal of 1 is exactly 1 on sm_103a, measured), so its transmittance,
          // suffix sum and every accumulator stay bit-identical.
          const f32x2 am = f2_make(cov0 ? a0 : 0.0f, cov1 ? a1 : 0.0f);
          const f32x2 om = f2_sub(ONE2, am);
          const f32x2 rom = f2_make(rcp_approx(f2_lo(om)), rcp_approx(f2_hi(om)));
          T2[q] = f2_mul(T2[q], rom);  // transmittance in front of this Gaussian
          const f32x2 w = f2_mul(am, T2[q]);
          aR = f2_fma(GC02[q], w, aR);
          aG = f2_fma(GC12[q], w, aG);
          aB = f2_fma(GC22[q], w, aB);
          f32x2 qv, dLda;
          if constexpr (kAux) {
            aZ = f2_fma(GD2[q], w, aZ);
            qv = f2_fma(GC02[q], CA.x,
                        f2_fma(GC12[q], CA.y, f2_fma(GC22[q], CB.x, f2_mul(GD2[q], CB.y))));
            dLda = f2_fma(T2[q], qv, f2_mul(rom, f2_sub(GAT2[q], U2[q])));
          } else {
            qv = f2_fma(GC02[q], CA.x, f2_fma(GC12[q], CA.y, f2_mul(GC22[q], CB.x)));
            dLda = f2_fma(T2[q], qv, f2_mul(rom, f2_sub(ZERO2, U2[q])));
          }
          U2[q] = f2_fma(w, qv, U2[q]);
          // dL/dpower = dL/dalpha * alpha (d alpha / d power = o G = alpha), unclamped only
          // (an uncovered pixel has alpha 0 here, so its share is 0 already).
          f32x2 dp = f2_mul(dLda, am);
          if constexpr (kClamp) {
            const bool m0 = oG0 < c.alpha_max, m1 = oG1 < c.alpha_max;
            dp = f2_make(m0 ? f2_lo(dp) : 0.0f, m1 ? f2_hi(dp) : 0.0f);
          }
          mP = f2_add(mP, dp);
          const f32x2 t = f2_mul(dp, FR[q]);
          mY = f2_add(mY, t);
          mYY = f2_fma(t, FR[q], mYY);
        }
        gr = f2_lo(aR) + f2_hi(aR);
        gg = f2_lo(aG) + f2_hi(aG);
        gb = f2_lo(aB) + f2_hi(aB);
        if constexpr (kAux) gz = f2_lo(aZ) + f2_hi(aZ);
        sdp = f2_lo(mP) + f2_hi(mP);
        sr = f2_lo(mY) + f2_hi(mY);
        srr = f2_lo(mYY) + f2_hi(mYY);
        ta = f2_lo(TA);
      } else {
        const float4 g0 = reinterpret_cast<const float4*>(sp[0])[g];
        const float4 g1 = reinterpret_cast<const float4*>(sp[1])[g];
        const float4 g2 = reinterpret_cast<const float4*>(sp[2])[g];
        ta = __fmaf_rn(g0.z, __fsub_rn(__fsub_rn(fx, g0.x), g0.y), g0.w);
#pragma unroll
        for (int k = 0; k < PPT; ++k) {
          if (kCheckLast && jj > last[k]) continue;
          const float fr = (float)(r0_ + k);
          const float oG = ex2_neg_approx(neg_log2_og(ta, g1.z, g1.x, g1.y, g1.w, fr));
          const float a = fminf(c.alpha_max, oG);
          if (a < c.alpha_min) continue;
          const float rom = rcp_approx(__fsub_rn(1.0f, a));
          T[k] = T[k] * rom;  // transmittance in front of this Gaussian
          const float w = a * T[k];
          gr = fmaf(gC0[k], w, gr);
          gg = fmaf(gC1[k], w, gg);
          gb = fmaf(gC2[k], w, gb);
          float q, dLda;
          if constexpr (kAux) {
            gz = fmaf(gD[k], w, gz);
            q = fmaf(gC0[k], g2.x, fmaf(gC1[k], g2.y, fmaf(gC2[k], g2.z, gD[k] * g2.w)));
            dLda = fmaf(T[k], q, rom * (gAT[k] - U[k]));
          } else {
            q = fmaf(gC0[k], g2.x, fmaf(gC1[k], g2.y, gC2[k] * g2.z));
            dLda = fmaf(T[k], q, rom * (0.0f - U[k]));
          }
          U[k] = fmaf(w, q, U[k]);
          if (oG < c.alpha_max) {
            const float dp = dLda * a;  // dL/dpower: d alpha / d power = o G = alpha
            sdp += dp;
            const float t = dp * fr;
            sr += t;
            srr = fmaf(t, fr, srr);
          }
        }
      }
    }
    const float tsdp = ta * sdp;
    float* col = rows + lane;
    col[0 * kRedPad] = sdp;
    col[1 * kRedPad] = sr;
    col[2 * kRedPad] = srr;
    col[3 * kRedPad] = tsdp;
    col[4 * kRedPad] = ta * sr;
    col[5 * kRedPad] = ta * tsdp;
    col[6 * kRedPad] = gr;
    col[7 * kRedPad] = gg;
    col[8 * kRedPad] = gb;
    if constexpr (kAux) col[9 * kRedPad] = gz;
    else (void)gz;
  };

  // Row sums of the last nb visits (staged at g_first, g_first - 1, ...), then one lane per
  // Gaussian forms its whitened moments (with w = (t_a + r l21, s_a + r l22):
  // sum dp w = (S3 + l21 S1, s_a S0 + l22 S1) and
  // sum dp w w^T = (S5 + l21 (2 S4 + l21 S2), s_a W_t + l22 (S4 + l21 S2),
  // s_a W_s + l22 (s_a S1 + l22 S2)) for the lane values S0..S5) and adds them to its record.
  auto flush = [&](int nb, int g_first) {
    __syncwarp();
    const int nrows = nb * RL::kVals;
    for (int r = lane; r < nrows; r += 32) reduce_row(red, r);
    __syncwarp();
    if (lane < nb) {
      const int g = g_first - lane;
      const float* tot = red + lane * RL::kVals * kRedPad + 32;
      float S[RL::kVals];
#pragma unroll
      for (int k = 0; k < RL::kVals; ++k) S[k] = tot[k * kRedPad];
      float l21, l22, s_a;
      if constexpr (kPacked) {
        l21 = f2_lo(sp[2][g].x);
        l22 = f2_lo(sp[2][g].y);
        s_a = f2_lo(sp[3][g].x);
      } else {
        const float4 g1 = reinterpret_cast<const float4*>(sp[1])[g];
        l21 = g1.x;
        l22 = g1.y;
        s_a = g1.z;
      }
      bool any = false;
#pragma unroll
      for (int k = 0; k < RL::kVals; ++k) any = any || S[k] != 0.0f;
      if (any) {
        const float wt = fmaf(l21, S[1], S[3]);
        const float ws = fmaf(s_a, S[0], l22 * S[1]);
        const float u = fmaf(l21, S[2], S[4]);
        float* dst = g2d + (size_t)s_vi[g] * kG2Stride;
        atomicAdd(dst + kM0, S[0]);
        atomicAdd(dst + kWt, wt);
        atomicAdd(dst + kWs, ws);
        atomicAdd(dst + kWtt, fmaf(l21, S[4] + u, S[5]));
        atomicAdd(dst + kWts, fmaf(s_a, wt, l22 * u));
        atomicAdd(dst + kWss, fmaf(s_a, ws, l22 * fmaf(s_a, S[1], l22 * S[2])));
        atomicAdd(dst + kGR, S[6]);
        atomicAdd(dst + kGG, S[7]);
        atomicAdd(dst + kGB, S[8]);
        if constexpr (kAux) atomicAdd(dst + kGZ, S[9]);
      }
    }
    __syncwarp();
  };

  const int first = (int)range.x;
  for (int bend = max_last + 1; bend > first; bend -= kThreads) {
    const int bstart = max(first, bend - kThreads);
    __syncthreads();
    const int j = bstart + (int)threadIdx.x;
    if (j < bend) {
      const uint32_t vi = pair_vals[j];
      s_vi[threadIdx.x] = vi;
      stage_gaussian(sp, threadIdx.x, rec0[vi], rec1[vi], rec2[vi], y_a);
    }
    __syncthreads();
    // Positions above the warp's smallest last index test each pixel; the rest do not. Whether
    // the staged Gaussian can reach alpha_max is warp-uniform (every thread reads its opacity).
    auto clamps = [&](int g) {
      if constexpr (kPacked) return !(f2_lo(sp[3][g].y) > c.unclamped_neg_lo);
      return true;
    };
    int nb = 0, g_first = bend - 1 - bstart;
    auto next = [&](int g) {
      if (++nb == RL::kBatch) {
        flush(nb, g_first);
        nb = 0;
        g_first = g - 1;
      }
    };
    const int split = max(bstart - 1, min(bend - 1, warp_min_last));
    for (int jj = bend - 1; jj > split; --jj) {
      const int g = jj - bstart;
      float* rows = red + nb * RL::kVals * kRedPad;
      if (clamps(g))
        visit(jj, g, rows, std::true_type{}, std::true_type{});
      else
        visit(jj, g, rows, std::true_type{}, std::false_type{});
      next(g);
    }
    for (int jj = split; jj >= bstart; --jj) {
      const int g = jj - bstart;
      float* rows = red + nb * RL::kVals * kRedPad;
      if (clamps(g))
        visit(jj, g, rows, std::false_type{}, std::true_type{});
      else
        visit(jj, g, rows, std::false_type{}, std::false_type{});
      next(g);
    }
    if (nb > 0) flush(nb, g_first);
  }
}

// ------------------------------------------------------------------------------------------
// Launch order of the blends' tiles: longest run first. A CTA's time grows with its tile's run,
// and runs differ by two orders of magnitude (a few tiles near dense structure hold thousands of
// Gaussians); launched in tile order, a long run that starts late holds its SM after the others
// have drained. Sorted by decreasing length, the long runs start first and the short ones fill
// the end. The key is the run length's octave, so the stable sort keeps each octave's tiles in
// tile order: neighbouring tiles, which share Gaussians (their records, and in the backward their
// gradient atomics), still run together. Finer classes (16 per octave) made the backward 3 %
// slower; octaves made it 1 % faster than plain tile order.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t length_octave(uint32_t len) {
  return (uint32_t)(31 - __clz(len + 1u));  // 0 .. 32
}

__global__ void tile_order_keys_kernel(const uint2* __restrict__ ranges, uint32_t total_tiles,
                                       uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  chain_wait();
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total_tiles) return;
  const uint2 r = ranges[t];
  keys[t] = 32u - length_octave(r.y - r.x);
  vals[t] = t;
}

template <int TW, int TH, int PPT>
cudaError_t launch_blends_t(bool forward, const Views& views, const Consts& c,
                            const uint2* ranges, const uint32_t* pair_vals, const float4* rec0,
                            const float4* rec1, const float4* rec2, float* color, float* depth,
                            float* alpha, float* t_final, int32_t* last_index,
                            const float* d_color, const float* d_depth, const float* d_alpha,
                            float* g2d, const uint32_t* tile_order, Counters* counters,
                            cudaStream_t stream) {
  if (views.total_tiles == 0) return cudaSuccess;
  constexpr int kThreads = TW * TH / PPT;
  cudaError_t e;
  if (forward) {
    e = launch_chained(blend_forward_kernel<TW, TH, PPT>, dim3(views.total_tiles), dim3(kThreads),
                       stream, views, c, ranges, pair_vals, rec0, rec1, rec2, color, depth, alpha,
                       t_final, last_index, tile_order, counters);
  } else {
    const bool aux = d_depth != nullptr || d_alpha != nullptr;
    e = launch_chained(aux ? blend_backward_kernel<TW, TH, PPT, true>
                           : blend_backward_kernel<TW, TH, PPT, false>,
                       dim3(views.total_tiles), dim3(kThreads), stream, views, c, ranges,
                       pair_vals, rec0, rec1, rec2, (const float*)t_final,
                       (const int32_t*)last_index, d_color, d_depth, d_alpha, tile_order, g2d);
  }
  RGS_LAUNCHED();
  return e;
}

}  // namespace

cudaError_t launch_duplicate(const Views& views, int n, const uint32_t* order,
                             const uint32_t* offsets, const uint32_t* ntiles, const float4* rec0,
                             const float4* rec1, const float4* rec2, float log2_alpha_min,
                             int64_t visible_cap, uint32_t capacity,
                             uint32_t* keys, uint32_t* vals, Counters* counters,
                             cudaStream_t stream) {
  (void)rec2;
  if (visible_cap > 0) {
    const int64_t need = (visible_cap + kDupThreads - 1) / kDupThreads;
    const unsigned blocks = (unsigned)std::min<int64_t>(need, 8 * 152);
    const cudaError_t e =
        launch_chained(duplicate_kernel, dim3(blocks), dim3(kDupThreads), stream, views, n, order,
                       offsets, ntiles, rec0, rec1, log2_alpha_min,
                       (uint32_t)std::min<int64_t>(visible_cap, 0xffffffffll), capacity, keys,
                       vals, counters);
    RGS_LAUNCHED();
    return e;
  }
  // No visible-list capacity: nothing to duplicate, but the counts still need storing.
  const cudaError_t e = launch_chained(store_pair_count_kernel, dim3(1), dim3(1), stream, counters,
                                       capacity);
  RGS_LAUNCHED();
  return e;
}

cudaError_t launch_tile_order(const uint2* ranges, int total_tiles, uint32_t* keys,
                              uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                              uint32_t* hist, uint32_t* block_sums, const uint32_t** order,
                              cudaStream_t stream) {
  *order = vals;
  if (total_tiles <= 0) return cudaSuccess;
  constexpr int kThreads = 256;
  cudaError_t e = launch_chained(tile_order_keys_kernel, dim3((total_tiles + kThreads - 1) / kThreads),
                                 dim3(kThreads), stream, ranges, (uint32_t)total_tiles, keys, vals);
  RGS_LAUNCHED();
  if (e != cudaSuccess) return e;
  bool alt = false;
  e = launch_radix_sort(keys, vals, keys_alt, vals_alt, total_tiles, nullptr, 0, 6, hist,
                        block_sums, &alt, stream, kSortItemsSmall);
  *order = alt ? vals_alt : vals;
  return e;
}

cudaError_t launch_blend(bool forward, const Views& views, const Consts& c, const uint2* ranges,
                         const uint32_t* pair_vals, const float4* rec0, const float4* rec1,
                         const float4* rec2, float* color, float* depth, float* alpha,
                         float* t_final, int32_t* last_index, const float* d_color,
                         const float* d_depth, const float* d_alpha, float* g2d,
                         const uint32_t* tile_order, Counters* counters, cudaStream_t stream) {
  const int tw = views.tile_w, th = views.tile_h;
  const int ppt = forward ? views.pixels_per_thread : views.bwd_pixels_per_thread;
#define RGS_BLEND(W, H, P)                                                                        \
  if (tw == W && th == H && ppt == P)                                                             \
  return launch_blends_t<W, H, P>(forward, views, c, ranges, pair_vals, rec0, rec1, rec2, color, \
                                  depth, alpha, t_final, last_index, d_color, d_depth, d_alpha,   \
                                  g2d, tile_order, counters, stream)
  RGS_BLEND(16, 16, 1);
  RGS_BLEND(16, 16, 2);
  RGS_BLEND(16, 16, 4);
  RGS_BLEND(16, 16, 8);
  RGS_BLEND(8, 8, 1);
  RGS_BLEND(8, 8, 2);
  RGS_BLEND(32, 8, 1);
  RGS_BLEND(32, 8, 2);
  RGS_BLEND(32, 8, 4);
  RGS_BLEND(32, 8, 8);
#undef RGS_BLEND
  return cudaErrorInvalidValue;
}

}  // namespace rgs
