// rgs_internal.cuh -- shared declarations and device helpers of the sm_103a rasterizer.
//
// Layout in HBM (V views, N Gaussians, "vi" = v * N + i):
//   rec0[vi] = (mean2d.x hi, mean2d.y hi, mean2d.x lo, mean2d.y lo)   float4, the projected
//              mean as an unevaluated double-float sum, so that p - mu^I is accurate to ~1e-7 px
//              even at 1080p coordinates
//   rec1[vi] = (l11, l21, l22, log2 o)                    float4, lower-triangular factor of the
//              base-2-scaled conic (see below)
//   rec2[vi] = (r, g, b, depth z)                          float4
//   ntiles[vi]: tiles touched (0 = culled / invisible)
//   g2d[vi * 16 + s]: the backward blend's sums over the covered pixels of dL/dpower moments
//              and of the colour / depth weights (see G2Slot), reused by the backward
//              preprocess for its per-view intermediate results
//   pair list: key = global tile id, value = vi; sorted so that each tile's run is in
//              (depth, index) order; ranges[gtile] = [first, last + 1) of the run.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rgs.h"

namespace rgs {

constexpr int kMaxViews = RGS_MAX_VIEWS;
constexpr int kG2Stride = 16;  // floats per (view, Gaussian) gradient record (64 bytes)

// Slots the backward blend accumulates per (view, Gaussian), with dp = dL/dpower of a covered,
// unclamped pixel and (t, s) = L^T (p - mu^I) the pixel's whitened offset (see the coverage
// helpers below):
//   kM0 = sum dp, kWt = sum dp t, kWs = sum dp s, kWtt = sum dp t^2, kWts = sum dp t s,
//   kWss = sum dp s^2; kGR/kGG/kGB/kGZ = dL/d(colour, depth) = sum dL/dC alpha T.
// The screen-space gradients are linear in these sums (L and the opacity are constant per
// (view, Gaussian)), so the backward preprocess forms them once per record. Whitened moments
// stay well conditioned where moments of p - mu^I do not: for a thin footprint whose centre lies
// thousands of pixels off the image, sum dp (p - mu)(p - mu)^T is dominated by the long axis and
// the thin-axis part that the covariance gradient needs is lost to FP32 accumulation.
enum G2Slot { kM0 = 0, kWt, kWs, kWtt, kWts, kWss, kGR, kGG, kGB, kGZ };

struct ViewParams {
  int width, height;
  int tiles_x, tiles_y;
  int tile_base;            // first global tile id of this view
  int pad0;
  long long pixel_offset;   // first pixel of this view in the concatenated images
  float fx, fy, cx, cy;
  float R[9];               // world-to-camera rotation, row-major
  float t[3];
  float cam_center[3];      // -R^T t
  float lim_u, lim_w;       // guard band of x/z and y/z used by the projection Jacobian
};

// Every kernel receives the views by value (a __grid_constant__ parameter block), so a captured
// CUDA graph carries its own camera data and no host-to-device copy is needed per call.
struct Views {
  int n_views;
  int total_tiles;
  long long total_pixels;
  int tile_w, tile_h;
  int pixels_per_thread;    // vertically adjacent pixels per forward-blend thread
  int bwd_pixels_per_thread;  // the same for the backward blend
  // Device pose records [n_views][16] = R (9, row-major), t (3), c = -R^T t (3), pad; when set,
  // they replace the poses in v[] (a pose that lives on the device, e.g. one a tracking loop
  // updates without the host). Null: the poses in v[].
  const float* pose_dev;
  ViewParams v[kMaxViews];
};

// The pose of view v that the launch uses: R (row-major), t and the camera centre.
struct PoseRef {
  const float* R;
  const float* t;
  const float* c;
};
__device__ __forceinline__ PoseRef view_pose(const Views& views, int v) {
  if (views.pose_dev) {
    const float* p = views.pose_dev + 16 * v;
    return PoseRef{p, p + 9, p + 12};
  }
  const ViewParams& vp = views.v[v];
  return PoseRef{vp.R, vp.t, vp.cam_center};
}
// The same with the pose's location fixed at compile time (kDevice: the device records), for
// kernels whose host-pose variant should read the parameter block directly.
template <bool kDevice>
__device__ __forceinline__ PoseRef view_pose(const Views& views, int v) {
  if constexpr (kDevice) {
    const float* p = views.pose_dev + 16 * v;
    return PoseRef{p, p + 9, p + 12};
  } else {
    const ViewParams& vp = views.v[v];
    return PoseRef{vp.R, vp.t, vp.cam_center};
  }
}

struct Consts {
  float alpha_min, alpha_max, t_min, znear, eps2d;
  float bg[3];
  float log2_alpha_min;  // log2(alpha_min), rounded once on the host
  // A staged Gaussian with -log2(o) above this value cannot reach alpha_max at any pixel
  // (o G <= o < alpha_max by a margin far beyond the error of the hardware exponential), so the
  // blends skip the clamp and its gradient kink test for it: 1e-5 - log2(alpha_max).
  float unclamped_neg_lo;
};

// Device status bits.
enum StatusBits : uint32_t {
  kStatusPairOverflow = 1u,     // the pair list outgrew its capacity
  kStatusVisibleOverflow = 2u,  // the visible entries outgrew the sorted-list capacity
  kStatusScanWait = 4u,         // a single-pass scan gave up waiting for an earlier block
};

// Device counters of one forward.
struct Counters {
  uint32_t n_visible;       // compacted (view, Gaussian) entries
  uint32_t n_pairs;         // duplicated pairs
  uint32_t n_pairs_stored;  // min(n_pairs, capacity)
  uint32_t status;
  uint32_t n_nonfinite;
  uint32_t n_candidates;    // entries the cull pass keeps for full projection
  uint32_t n_visible_kept;  // min(n_visible, visible-list capacity): the entries sorted and used
  uint32_t pad;
  unsigned long long n_eval;     // (pixel, Gaussian) positions the forward blend visited
  unsigned long long n_contrib;  // reserved (0): composites are not counted
};

// Programmatic dependent launch. Every kernel of the library is launched with programmatic
// stream serialization allowed (launch_chained below): once every block of the previous kernel
// of the stream has exited, the next kernel is scheduled without waiting for the previous grid
// to be retired. In every block, before any early return or any access to data of earlier
// kernels, it waits for the previous kernel to complete with its memory visible. Since each
// kernel completes only after that wait, the previous kernel's completion implies the completion
// of all earlier ones. No kernel lets its successor start before its own blocks have exited:
// with successors scheduled as soon as their predecessor had started, a long chain of short
// kernels captured in a graph replayed wrong results.
__device__ __forceinline__ void chain_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_chained(void (*kernel)(KArgs...), dim3 grid, dim3 block,
                                  cudaStream_t stream, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Host-side count of kernels the library has launched on the calling thread.
inline uint64_t& launch_counter() {
  static thread_local uint64_t count = 0;
  return count;
}
#define RGS_LAUNCHED() (++::rgs::launch_counter())

// ------------------------------------------------------------------------------------------
// Small device helpers.
// ------------------------------------------------------------------------------------------

__device__ __forceinline__ int view_of_tile(const Views& views, int gtile) {
  int lo = 0, hi = views.n_views - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (views.v[mid].tile_base <= gtile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Error-free product and sum (Dekker / Knuth) used by the compensated dot product below.
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// a b - c d with Kahan's FMA scheme: within about one ulp of the exact value even when the two
// products nearly cancel.
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d) {
  const float w = __fmul_rn(c, d);
  const float e = __fmaf_rn(-c, d, w);
  const float f = __fmaf_rn(a, b, -w);
  return __fadd_rn(f, e);
}

// r . m + t with the compensated dot product "Dot2" of Ogita, Rump and Oishi (SIAM J. Sci.
// Comput. 26(6), 2005): as accurate as evaluation in twice the working precision. Returns the
// result as an unevaluated sum hi + lo (|lo| <= ulp(hi) / 2), hi being the float32 rounding of
// the accurate value. The camera-space depth taken from hi is therefore the float32 rounding of
// the exact depth, so the near-to-far sort key does not depend on operation order.
__device__ __forceinline__ float dot3_plus_dd(float r0, float r1, float r2, float m0, float m1,
                                              float m2, float t, float& lo) {
  float p, s, h, e, q;
  two_prod(r0, m0, p, s);
  two_prod(r1, m1, h, e);
  two_sum(p, h, p, q);
  s = __fadd_rn(s, __fadd_rn(q, e));
  two_prod(r2, m2, h, e);
  two_sum(p, h, p, q);
  s = __fadd_rn(s, __fadd_rn(q, e));
  two_sum(p, t, p, q);
  s = __fadd_rn(s, q);
  const float hi = __fadd_rn(p, s);
  lo = __fsub_rn(s, __fsub_rn(hi, p));
  return hi;
}

// Hardware base-2 exponential and reciprocal (PTX ex2.approx / rcp.approx): fixed instruction
// sequences, so every kernel that evaluates the same input gets the same bits.
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Coverage of a pixel by a projected Gaussian, alpha = min(alpha_max, o G), with
// G = exp(-1/2 d^T Q d) and d = p - mu^I (Section 3.1, Eq. alpha). The record stores the lower
// triangular factor L of the base-2-scaled conic, (log2(e) / 2) Q = L L^T, and lo = log2(o), so
//   log2(o G) = lo - (t^2 + s^2),  (t, s) = L^T d = (l11 dx + l21 dy, l22 dy).
// The whitened offsets t and s are O(1) wherever the Gaussian is visible, so the exponent keeps
// its accuracy for thin footprints far from their centre, where the expanded quadratic form
// a dx^2 + 2 b dx dy + c dy^2 cancels terms of 10^4 and more.
// A blend CTA evaluates its tile's pixels against one staged Gaussian: the row terms at the
// tile's anchor row y_a (its middle row), c21 = l21 (y_a - mu_y) and s_a = l22 (y_a - mu_y), are
// computed once per (Gaussian, tile); a thread then forms t_a = l11 dx + c21 once for its column,
// and each pixel at row offset r = y - y_a costs t = t_a + r l21, s = s_a + r l22 and two FMAs
// for t^2 + s^2 - lo. Every operation is explicitly rounded and a pixel's value depends only on
// its tile row, so both blends take identical coverage decisions whatever their pixels per
// thread.
struct AnchorTerms {
  float c21, s_a;
};
__device__ __forceinline__ AnchorTerms anchor_terms(float4 r0, float4 r1, float y_a) {
  const float dya = __fsub_rn(__fsub_rn(y_a, r0.y), r0.w);
  return AnchorTerms{__fmul_rn(r1.y, dya), __fmul_rn(r1.z, dya)};
}
// t at the anchor row of column px.
__device__ __forceinline__ float column_t(float px, float4 r0, float l11, float c21) {
  return __fmaf_rn(l11, __fsub_rn(__fsub_rn(px, r0.x), r0.z), c21);
}
// t^2 + s^2 - log2(o) = -log2(o G) at row offset r.
__device__ __forceinline__ float neg_log2_og(float t_a, float s_a, float l21, float l22,
                                             float neg_lo, float r) {
  const float t = __fmaf_rn(r, l21, t_a), s = __fmaf_rn(r, l22, s_a);
  return __fmaf_rn(t, t, __fmaf_rn(s, s, neg_lo));
}
// 2^(-x): o G from neg_log2_og.
__device__ __forceinline__ float ex2_neg_approx(float x) {
  float y;
  asm("{\n\t.reg .f32 n;\n\tneg.f32 n, %1;\n\tex2.approx.ftz.f32 %0, n;\n\t}" : "=f"(y) : "f"(x));
  return y;
}

// Packed FP32 pairs (PTX .f32x2 on the sm_100 family): one instruction performs the same IEEE
// round-to-nearest operation on both halves of a 64-bit register pair, so two pixels that share
// every operand but their own state cost one issue slot. Results are bit-identical to the
// scalar __fadd_rn / __fsub_rn / __fmul_rn / __fmaf_rn.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2_make(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float f2_lo(f32x2 v) {
  float lo;
  asm("{\n\t.reg .f32 t;\n\tmov.b64 {%0, t}, %1;\n\t}" : "=f"(lo) : "l"(v));
  return lo;
}
__device__ __forceinline__ float f2_hi(f32x2 v) {
  float hi;
  asm("{\n\t.reg .f32 t;\n\tmov.b64 {t, %0}, %1;\n\t}" : "=f"(hi) : "l"(v));
  return hi;
}
__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f32x2 f2_sub(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

constexpr float kLn2 = 0.69314718055994531f;
constexpr float kLog2e = 1.4426950408889634f;

// ------------------------------------------------------------------------------------------
// Tile coverage of a projected Gaussian: the tiles whose pixel centres may lie inside the
// alpha >= alpha_min ellipse {d : |L^T d|^2 <= kappa}, kappa = log2 o - log2 alpha_min, padded by
// kTilePad pixels so that the per-pixel FP32 test in the blend can never find a covered pixel
// outside the listed tiles. The two tests differ only by rounding: a few ulps relative to the
// footprint's extent (the blend adds the low part of the mean, below 1e-4 px; the extent here
// comes from approximate reciprocals and square roots), and kappa is widened by 1e-4 relative
// below, so a sixteenth of a pixel is a wide margin. Each listed tile without a covered pixel
// costs a full pass over the tile in both blends. Visits tile rows ty0..ty1 and, per row, the
// column span [tx0, tx1] of the ellipse restricted to the row's pixel band.
// ------------------------------------------------------------------------------------------
constexpr float kTilePad = 0.0625f;

struct Ellipse {
  float mx, my;           // centre
  float l11, l21, l22;    // factor of the scaled conic (the record's rec1.xyz)
  float kappa;
};

// From the stored records (rec0.xy = mean hi parts, rec1 = factor and log2 o).
__device__ __forceinline__ bool make_ellipse(float4 r0, float4 r1, float log2_alpha_min,
                                             Ellipse& e) {
  const float kappa = __fsub_rn(r1.w, log2_alpha_min);
  if (!(r1.x > 0.0f) || !(r1.z > 0.0f) || !(kappa >= 0.0f)) return false;
  e.mx = r0.x;
  e.my = r0.y;
  e.l11 = r1.x;
  e.l21 = r1.y;
  e.l22 = r1.z;
  e.kappa = kappa;
  return true;
}

// sqrt through the hardware reciprocal square root: not correctly rounded, but a fixed
// instruction sequence, so every kernel that calls it gets the same bits for the same input.
__device__ __forceinline__ float sqrt_fixed(float x) {
  return x > 0.0f ? __fmul_rn(x, rsqrtf(x)) : 0.0f;
}

// Every operation below is a single instruction with no contraction (explicitly rounded
// arithmetic, hardware approximations of reciprocals and square roots), so the counting pass in
// the projection and the emitting pass of the duplication visit exactly the same tiles. The
// approximations err by a few ulp, far inside the 1-pixel padding.
//
// TileCover holds the per-footprint constants; span(ty) gives the column span of one tile row,
// so that rows can be walked in sequence (for_each_tile_row) or in parallel, one per lane.
struct TileCover {
  int ty0, ty1, bx0, bx1;
  bool box_only;  // a single row or column of tiles: every row spans the padded box
  int tile_w, tile_h, tiles_x;
  float mx, my, kap, rx, ry, inv_tw, x_lo, x_hi, inv_syy, s, h, dy_star;

  // False when the footprint touches no tile.
  __device__ __forceinline__ bool init(const Ellipse& e, int tw, int th, int tiles_x_,
                                       int tiles_y) {
    tile_w = tw;
    tile_h = th;
    tiles_x = tiles_x_;
    mx = e.mx;
    my = e.my;
    kap = __fadd_rn(__fmul_rn(e.kappa, 1.0001f), 1e-6f);
    // With (t, s) = L^T d: |s| <= sqrt(kap) bounds dy by sqrt(kap) / l22; for a given dy,
    // |t| <= sqrt(kap - s^2) gives dx in -l21 / l11 dy +- sqrt(kap - (l22 dy)^2) / l11, whose
    // extremes lie at dy* = -+ rx l11 l21 / (l21^2 + l22^2) with half-width
    // rx = sqrt(kap (1 + (l21 / l22)^2)) / l11.
    const float sk = sqrt_fixed(kap);
    const float il11 = __fdiv_rn(1.0f, e.l11), il22 = __fdiv_rn(1.0f, e.l22);
    const float r = __fmul_rn(e.l21, il22);
    rx = __fmul_rn(__fmul_rn(sk, sqrt_fixed(__fmaf_rn(r, r, 1.0f))), il11);
    ry = __fmul_rn(sk, il22);
    inv_tw = 1.0f / (float)tw;  // powers of two
    const float inv_th = 1.0f / (float)th;
    const float y_lo = __fsub_rn(__fsub_rn(e.my, ry), kTilePad);
    const float y_hi = __fadd_rn(__fadd_rn(e.my, ry), kTilePad);
    x_lo = __fsub_rn(__fsub_rn(e.mx, rx), kTilePad);
    x_hi = __fadd_rn(__fadd_rn(e.mx, rx), kTilePad);
    // Clamp before converting to int: the extents of near-degenerate Gaussians can be huge.
    const float fty0 = floorf(fminf(fmaxf(__fmul_rn(y_lo, inv_th), -1.0f), (float)tiles_y));
    const float fty1 = floorf(fminf(fmaxf(__fmul_rn(y_hi, inv_th), -1.0f), (float)tiles_y));
    const float ftx0 = floorf(fminf(fmaxf(__fmul_rn(x_lo, inv_tw), -1.0f), (float)tiles_x));
    const float ftx1 = floorf(fminf(fmaxf(__fmul_rn(x_hi, inv_tw), -1.0f), (float)tiles_x));
    ty0 = max(0, (int)fty0);
    ty1 = min(tiles_y - 1, (int)fty1);
    bx0 = max(0, (int)ftx0);
    bx1 = min(tiles_x - 1, (int)ftx1);
    if (ty0 > ty1 || bx0 > bx1) return false;
    box_only = ty0 == ty1 || bx0 == bx1;
    // x | y of the ellipse: centre mx + s dy, half-width h sqrt(kap - dy^2 / syy), with
    // s = -l21 / l11, h = 1 / l11, 1 / syy = l22^2.
    inv_syy = __fmul_rn(e.l22, e.l22);
    s = __fmul_rn(-e.l21, il11);
    h = il11;
    dy_star = __fmul_rn(rx, __fdiv_rn(-__fmul_rn(e.l11, e.l21),
                                      __fmaf_rn(e.l21, e.l21, __fmul_rn(e.l22, e.l22))));
    return true;
  }

  // The cover set up by lane src of the warp, in every lane (all lanes must call it).
  __device__ __forceinline__ TileCover broadcast(int src) const {
    TileCover o;
    const unsigned m = 0xffffffffu;
    o.ty0 = __shfl_sync(m, ty0, src);
    o.ty1 = __shfl_sync(m, ty1, src);
    o.bx0 = __shfl_sync(m, bx0, src);
    o.bx1 = __shfl_sync(m, bx1, src);
    o.box_only = __shfl_sync(m, (int)box_only, src) != 0;
    o.tile_w = __shfl_sync(m, tile_w, src);
    o.tile_h = __shfl_sync(m, tile_h, src);
    o.tiles_x = __shfl_sync(m, tiles_x, src);
    o.mx = __shfl_sync(m, mx, src);
    o.my = __shfl_sync(m, my, src);
    o.kap = __shfl_sync(m, kap, src);
    o.rx = __shfl_sync(m, rx, src);
    o.ry = __shfl_sync(m, ry, src);
    o.inv_tw = __shfl_sync(m, inv_tw, src);
    o.x_lo = __shfl_sync(m, x_lo, src);
    o.x_hi = __shfl_sync(m, x_hi, src);
    o.inv_syy = __shfl_sync(m, inv_syy, src);
    o.s = __shfl_sync(m, s, src);
    o.h = __shfl_sync(m, h, src);
    o.dy_star = __shfl_sync(m, dy_star, src);
    return o;
  }

  // Column span [tx0, tx1] of tile row ty (ty0 <= ty <= ty1); false if the row is not touched.
  __device__ __forceinline__ bool span(int ty, int& tx0, int& tx1) const {
    if (box_only) {
      tx0 = bx0;
      tx1 = bx1;
      return true;
    }
    const float b0 = fmaxf(__fsub_rn(__fsub_rn((float)(ty * tile_h), kTilePad), my), -ry);
    const float b1 =
        fminf(__fsub_rn(__fadd_rn((float)(ty * tile_h + tile_h - 1), kTilePad), my), ry);
    float xmax, xmin;
    if (b0 > b1) {
      // The band lies in the padding only: keep the whole padded width.
      xmax = x_hi;
      xmin = x_lo;
    } else {
      if (dy_star >= b0 && dy_star <= b1) {
        xmax = __fadd_rn(mx, rx);
      } else {
        const float d = fminf(fmaxf(dy_star, b0), b1);
        const float hw =
            __fmul_rn(h, sqrt_fixed(__fsub_rn(kap, __fmul_rn(__fmul_rn(d, d), inv_syy))));
        xmax = __fadd_rn(__fadd_rn(mx, __fmul_rn(s, d)), hw);
      }
      if (-dy_star >= b0 && -dy_star <= b1) {
        xmin = __fsub_rn(mx, rx);
      } else {
        const float d = fminf(fmaxf(-dy_star, b0), b1);
        const float hw =
            __fmul_rn(h, sqrt_fixed(__fsub_rn(kap, __fmul_rn(__fmul_rn(d, d), inv_syy))));
        xmin = __fsub_rn(__fadd_rn(mx, __fmul_rn(s, d)), hw);
      }
      xmax = __fadd_rn(xmax, kTilePad);
      xmin = __fsub_rn(xmin, kTilePad);
    }
    tx0 = max(bx0, (int)floorf(fminf(fmaxf(__fmul_rn(xmin, inv_tw), -1.0f), (float)tiles_x)));
    tx1 = min(bx1, (int)floorf(fminf(fmaxf(__fmul_rn(xmax, inv_tw), -1.0f), (float)tiles_x)));
    return tx0 <= tx1;
  }
};

template <typename RowFn>
__device__ __forceinline__ void for_each_tile_row(const Ellipse& e, int tile_w, int tile_h,
                                                  int tiles_x, int tiles_y, RowFn&& fn) {
  TileCover tc;
  if (!tc.init(e, tile_w, tile_h, tiles_x, tiles_y)) return;
  for (int ty = tc.ty0; ty <= tc.ty1; ++ty) {
    int tx0, tx1;
    if (tc.span(ty, tx0, tx1)) fn(ty, tx0, tx1);
  }
}

// ------------------------------------------------------------------------------------------
// Host-side launchers (defined in the .cu files). All take device pointers and a stream.
// ------------------------------------------------------------------------------------------
struct ScanScratch {
  uint32_t* block_sums;  // >= scan_blocks(n) + 1 entries
};

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

inline int64_t scan_blocks(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

// Bookkeeping of one single-pass scan (chained scan with decoupled look-back): a ticket counter
// and one 64-bit state word per tile of kScanTile elements, all zero before the launch.
struct Lookback {
  uint32_t* ticket = nullptr;
  unsigned long long* tiles = nullptr;  // null: the scan runs without look-back
  uint32_t* status = nullptr;           // kStatusScanWait is recorded here
  int64_t capacity = 0;                 // tile states in the area
};
// Visibility bitmask of a forward: one row of vis_bit_words_per_view(n) words per view, bit i of
// row v set iff entry (v, i) touches a tile. The allocation for up to vn_cap entries holds every
// n_views x n layout with n_views * n <= vn_cap.
inline int64_t vis_bit_words_per_view(int64_t n) { return (n + 31) / 32; }
inline int64_t vis_bit_words_cap(int64_t vn_cap) { return (vn_cap + 31) / 32 + kMaxViews; }

// Tile states of one Lookback area serving up to n_cap elements: a scan of n_cap elements
// takes scan_blocks(n_cap) tiles; the bitmask compaction of n_views x n <= n_cap entries
// (tiles of 256 words, n_views <= RGS_MAX_VIEWS <= 256) takes at most n_cap / 8192 + 2.
static_assert(RGS_MAX_VIEWS <= 256, "bound of the bitmask compaction's tiles");
inline int64_t lookback_tiles(int64_t n_cap) { return scan_blocks(n_cap) + 2; }
// Bytes of one Lookback area (a 16-byte header, then the tile states).
inline size_t lookback_bytes(int64_t n_cap) { return 16 + 8 * (size_t)lookback_tiles(n_cap); }
inline Lookback lookback_at(void* area, uint32_t* status, int64_t n_cap) {
  Lookback lb;
  lb.ticket = static_cast<uint32_t*>(area);
  lb.tiles = reinterpret_cast<unsigned long long*>(static_cast<char*>(area) + 16);
  lb.status = status;
  lb.capacity = lookback_tiles(n_cap);
  return lb;
}

// Exclusive scan of in[0..n) (n read from n_dev if non-null, capped at n_cap) into out, total
// into *total (may be null).
cudaError_t launch_exclusive_scan(const uint32_t* in, uint32_t* out, int64_t n_cap,
                                  const uint32_t* n_dev, uint32_t* total, uint32_t* block_sums,
                                  cudaStream_t stream);

// The same scan in one launch through zeroed look-back bookkeeping.
cudaError_t launch_exclusive_scan_single_pass(const uint32_t* in, uint32_t* out, int64_t n,
                                              uint32_t* total, Lookback lb, cudaStream_t stream);

// Compaction of the visible entries, in (view, Gaussian) order: for every set bit i of row v of
// the visibility bitmask (n_views rows for n Gaussians), writes keys[pos] = float bits of
// rec2[v n + i].w (depth) and vals[pos] = list[pos] = v n + i (vals feeds the depth sort, list
// keeps the order for the colour pass and the backward's per-entry pass); the count into *n_out.
// One single-pass launch; lb must be zeroed.
cudaError_t launch_compact_visible(const uint32_t* vis_bits, int n_views, int n,
                                   const float4* rec2, uint32_t* keys, uint32_t* vals,
                                   uint32_t* list, uint32_t* n_out, Lookback lb,
                                   cudaStream_t stream);

// offs[k] = exclusive scan of ntiles[order[k]] for k < *n_dev; total into *total.
cudaError_t launch_gather_scan(const uint32_t* ntiles, const uint32_t* order, int64_t n_cap,
                               const uint32_t* n_dev, uint32_t* offs, uint32_t* total,
                               uint32_t* block_sums, Lookback lb, cudaStream_t stream);

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;       // keys per thread for large sorts (2048 per block)
constexpr int kSortItemsSmall = 4;  // for sorts whose live count is far below the capacity
constexpr int kRadixBins = 256;

inline int64_t sort_blocks(int64_t n, int items = kSortItems) {
  return (n + kSortThreads * items - 1) / (kSortThreads * items);
}
// Scratch for a sort of up to n_cap elements: the digit-major histogram table plus one row
// total per digit (u32 counts).
inline int64_t sort_hist_entries(int64_t n_cap, int items = kSortItems) {
  return (sort_blocks(n_cap, items) + 1) * kRadixBins;
}

// Mapping regulariser and maintenance state, fused into the per-Gaussian backward phase
// (Eq. reg, Eq. app-ema). A null pointer disables its part.
struct MapReg {
  float lambda_iso, lambda_alpha, lambda_mu;
  const float* ema_means;  // [n][3] anchor of the position term
  uint32_t* obs_count;     // [n]: += number of views of the forward that see the Gaussian
  float* vis_score;        // [n]: += that number times its opacity
  float* values;           // [n] scratch: the Gaussian's share of R (for the reduction)
  double* value;           // [1]: R summed over the Gaussians
};

// Per-view camera data in double precision (built on the host from the float cameras).
struct SeedCams {
  int n_views;
  int pad;
  long long pixel_offset[kMaxViews];
  int width[kMaxViews], height[kMaxViews];
  double P[kMaxViews][12];   // K [R | t], row-major 3x4
  double R[kMaxViews][9];
  double t[kMaxViews][3];
  double c[kMaxViews][3];    // camera centre -R^T t
  double fx[kMaxViews], fy[kMaxViews], cx[kMaxViews], cy[kMaxViews];
};

struct SeedConsts {
  double min_parallax, max_reproj, tie_eps, plane_radius, s_par_cap, alpha_lo, alpha_hi, voxel;
};

cudaError_t launch_triangulate(const SeedCams& cams, const SeedConsts& c, int64_t m, int k,
                               const int32_t* ref_view, const double* ref_xy,
                               const int32_t* nb_view, const double* nb_xy, const float* nb_conf,
                               uint32_t* valid, double* X, int32_t* best, double* err,
                               double* angle, float* kappa, cudaStream_t stream);
cudaError_t launch_seed_flags(int64_t m, int n_views, const uint32_t* valid,
                              const int32_t* ref_view, uint32_t* flags, cudaStream_t stream);
cudaError_t launch_compact_points(int64_t m, const uint32_t* valid, const uint32_t* pos,
                                  uint32_t* vidx, cudaStream_t stream);
cudaError_t launch_seed_points(const SeedCams& cams, const SeedConsts& c, int s, int k, int sh_k,
                               const uint32_t* vidx, const int32_t* ref_view,
                               const int32_t* nb_view, const double* X, const double* err,
                               const double* angle, const float* kappa, const float* obs,
                               const float* gain_bias, uint32_t* lo, uint32_t* hi,
                               uint32_t* slot, uint32_t* t0, uint32_t* t1, uint32_t* hist,
                               uint32_t* block_sums, unsigned long long* skey, double* sX,
                               float* means, float* log_scales, float* quats, float* logits,
                               float* sh, float* normals, uint32_t* keep, cudaStream_t stream);
cudaError_t launch_scatter_seeds(int s, int sh_k, const uint32_t* keep, const uint32_t* pos,
                                 const uint32_t* vidx, const float* means,
                                 const float* log_scales, const float* quats,
                                 const float* logits, const float* sh, const float* normals,
                                 int32_t* o_index, float* o_means, float* o_log_scales,
                                 float* o_quats, float* o_logits, float* o_sh, float* o_normals,
                                 cudaStream_t stream);

// Largest n the single-cluster sort takes on `device` (0: cluster launches unavailable); sorts
// with n_cap up to it run as one launch and always return their result in the alternate buffers.
int64_t cluster_sort_capacity(int device);

// Stable LSD radix sort of (keys, vals) by bits [begin_bit, end_bit); ping-pongs between the
// (keys, vals) and (keys_alt, vals_alt) buffers and returns in *result_in_alt whether the
// sorted data ended in the alternate buffers. vals may be null (keys only).
cudaError_t launch_radix_sort(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt,
                              uint32_t* vals_alt, int64_t n_cap, const uint32_t* n_dev,
                              int begin_bit, int end_bit, uint32_t* hist, uint32_t* block_sums,
                              bool* result_in_alt, cudaStream_t stream,
                              int items = kSortItems);

}  // namespace rgs
