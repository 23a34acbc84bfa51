// rgs_api.cu -- the C ABI (include/rgs.h): context, per-forward saved state, device memory,
// and the launch sequence of the forward and backward passes.
//
// Forward launch sequence for a batch of V views (one launch per stage covers every view):
//   1. preprocess      per Gaussian, all views: projected records + tile counts  (Eq. proj)
//   2. compact         visible (view, Gaussian) entries with their depth keys
//   3. depth sort      stable radix sort of the visible entries by float32 depth
//   4. offsets         exclusive scan of tile counts in depth order
//   5. duplicate       one (tile, vi) pair per touched tile, emitted in depth order
//   6. tile sort       stable radix sort of the pairs by global tile id; stability keeps each
//                      tile's run in (depth, index) order
//   7. ranges          [first, last + 1) of each tile's run
//   8. blend           front-to-back compositing per tile                          (Eq. alpha)
// Backward: backward blend (screen-space gradients) then backward preprocess (parameter and
// twist gradients, Eq. muCjac / muIjac / sigmaIjac) and the twist reduction.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "rgs_internal.cuh"

namespace rgs {
cudaError_t launch_preprocess_forward(const Views& views, const Consts& c,
                                      const rgs_gaussians& g, float4* rec0, float4* rec1,
                                      float4* rec2, uint32_t* ntiles, uint32_t* cand,
                                      uint32_t* vis_bits, bool defer_colour, Counters* counters,
                                      cudaStream_t stream);
cudaError_t launch_ranges_colour(const uint32_t* keys, int total_tiles, uint2* ranges,
                                 uint32_t pair_capacity, const Views& views,
                                 const rgs_gaussians& g, const uint32_t* list, int64_t vis_cap,
                                 bool colour, float4* rec1, float4* rec2, Counters* counters,
                                 cudaStream_t stream);
int preprocess_backward_blocks(int64_t vn);
cudaError_t launch_preprocess_backward(const Views& views, const Consts& c,
                                       const rgs_gaussians& g, unsigned long long* vis_mask,
                                       const uint32_t* list, const Counters* counters,
                                       int64_t vn, float* g2d, uint32_t grad_mask,
                                       float* d_means, float* d_log_scales, float* d_quats,
                                       float* d_logits, float* d_sh, float* pose_partial,
                                       float* d_pose, const MapReg* reg, cudaStream_t stream);
cudaError_t launch_duplicate(const Views& views, int n, const uint32_t* order,
                             const uint32_t* offsets, const uint32_t* ntiles, const float4* rec0,
                             const float4* rec1, const float4* rec2, float log2_alpha_min,
                             int64_t visible_cap, uint32_t capacity,
                             uint32_t* keys, uint32_t* vals, Counters* counters,
                             cudaStream_t stream);
cudaError_t launch_blend(bool forward, const Views& views, const Consts& c, const uint2* ranges,
                         const uint32_t* pair_vals, const float4* rec0, const float4* rec1,
                         const float4* rec2, float* color, float* depth, float* alpha,
                         float* t_final, int32_t* last_index, const float* d_color,
                         const float* d_depth, const float* d_alpha, float* g2d,
                         const uint32_t* tile_order, Counters* counters, cudaStream_t stream);
cudaError_t launch_tile_order(const uint2* ranges, int total_tiles, uint32_t* keys,
                              uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                              uint32_t* hist, uint32_t* block_sums, const uint32_t** order,
                              cudaStream_t stream);
}  // namespace rgs

using namespace rgs;

namespace {

constexpr size_t kAlign = 256;
constexpr int kEvBwd0 = 9;                    // first backward event
constexpr int kNumEvents = kEvBwd0 + 3;       // 9 forward marks + 3 backward marks

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// A device allocation carved into aligned sub-buffers.
struct Region {
  void* base = nullptr;
  size_t bytes = 0;
};

struct State {
  // Inputs of the last forward (the backward reuses them).
  rgs_gaussians g{};
  Views views{};
  Consts consts{};
  int64_t vn = 0;            // n_views * n
  bool has_forward = false;

  // Capacities and regions.
  int64_t vn_cap = 0, n_cap = 0, pix_cap = 0, tile_cap = 0, pair_cap = 0, pose_cap = 0;
  // Sorted-list capacity for the visible entries (not an allocation: the buffers hold vn_cap
  // entries); the depth sort, the offsets scan and the duplication are sized by it.
  int64_t vis_cap = 0;
  Region r_vn, r_n, r_pix, r_tile, r_pair, r_scratch, r_pose, r_counters;

  // Per (view, Gaussian).
  float4 *rec0 = nullptr, *rec1 = nullptr, *rec2 = nullptr;
  uint32_t* ntiles = nullptr;
  uint32_t *vis_keys[2] = {nullptr, nullptr}, *vis_vals[2] = {nullptr, nullptr};
  uint32_t* offsets = nullptr;
  // The visible entries in (view, Gaussian) order (the compaction's output, kept past the depth
  // sort): the colour pass and the backward's per-entry pass walk it, so that neighbouring
  // threads read neighbouring Gaussians and mostly share a view.
  uint32_t* vis_list = nullptr;
  float* g2d = nullptr;
  // Visibility bits of the last forward: row v (ceil(n / 32) words) has bit i set iff entry
  // (v, i) touches a tile.
  uint32_t* vis_bits = nullptr;
  // Per Gaussian: bit v set by the backward's phase 1 for every view v that sees it, cleared by
  // phase 2 (zero between backward calls).
  unsigned long long* vis_mask = nullptr;
  const uint32_t* order = nullptr;  // depth-sorted visible entries (one of vis_vals)
  // Per pixel / tile / pair.
  float* t_final = nullptr;
  int32_t* last_index = nullptr;
  uint2* ranges = nullptr;
  // Launch order of the blends' tiles (longest run first) and the buffers of its sort.
  uint32_t *tile_keys[2] = {nullptr, nullptr}, *tile_vals[2] = {nullptr, nullptr};
  const uint32_t* tile_order = nullptr;
  uint32_t *pair_keys[2] = {nullptr, nullptr}, *pair_vals[2] = {nullptr, nullptr};
  const uint32_t* sorted_vals = nullptr;
  // Scratch.
  uint32_t* hist = nullptr;
  uint32_t* block_sums = nullptr;
  int64_t hist_cap = 0, sums_cap = 0;
  float* pose_partial = nullptr;
  Counters* counters = nullptr;
  float* pose_records = nullptr;  // [kMaxViews][16] device poses of a posed forward
  Region r_reg;                   // per-Gaussian regulariser values (first mapping backward)
  float* reg_vals = nullptr;
  int64_t reg_cap = 0;
  // Phase timing: event k is recorded at the start (k = 0) / end of each forward phase, and
  // kEvBwd0 .. at the start / end of each backward phase.
  cudaEvent_t ev[kNumEvents] = {};
  bool fwd_timed = false, bwd_timed = false;
  uint32_t fwd_launches = 0, bwd_launches = 0;
};

}  // namespace

namespace rgs {
cudaError_t launch_pose_prepare(const float* world_to_cam, int n_views, float* records,
                                cudaStream_t stream);
cudaError_t launch_grad_weight(const Views& views, const float* obs, float tau_grad, float* w_out,
                               cudaStream_t stream);
cudaError_t launch_track_loss(const Views& views, const float* color, const float* alpha,
                              const float* obs, const float* w_grad, float tau_alpha,
                              bool fit_exposure, double* sums, float* d_color, double* loss,
                              float* gain_bias, cudaStream_t stream);
cudaError_t launch_pose_adam(int n_views, float lr, float beta1, float beta2, float eps,
                             int iterations, const float* d_pose, float* adam_state,
                             int32_t* step, float* world_to_cam, cudaStream_t stream);
cudaError_t launch_covisibility(const float* alpha_a, const float* alpha_b, int64_t n,
                                int n_pairs, float tau, unsigned long long* counts, float* iou,
                                cudaStream_t stream);
cudaError_t launch_map_ema(int64_t n, const float* means, float* ema, float eta,
                           cudaStream_t stream);
cudaError_t launch_prune_mask(int64_t n, const float* log_scales, const float* logits,
                              const uint32_t* obs_count, const float* vis_score, float min_opacity,
                              float max_trace, uint32_t min_observations, float min_visibility,
                              uint8_t* keep, uint32_t* n_keep, cudaStream_t stream);
}  // namespace rgs

struct TuneChoice {
  int tile_w, tile_h, ppt, bwd_ppt;
};

struct rgs_ctx {
  int device = 0;
  bool timing = false;
  std::map<std::string, TuneChoice> tune_cache;
  std::string last_error;
  std::map<uint64_t, State*> states;
  uint64_t next_id = 1;
  Counters* host_counters = nullptr;  // pinned
  double* track_sums = nullptr;       // device [kMaxViews][4]: exposure-fit sums
  Region r_seed;                      // seed-initialisation scratch, grown on demand
};

namespace {

rgs_status fail(rgs_ctx* ctx, rgs_status s, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return s;
}

rgs_status cuda_fail(rgs_ctx* ctx, cudaError_t e, const char* where) {
  return fail(ctx, e == cudaErrorMemoryAllocation ? RGS_ERR_NOMEM : RGS_ERR_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define RGS_CUDA(call, where)                                \
  do {                                                       \
    cudaError_t _e = (call);                                 \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, where); \
  } while (0)

void free_region(Region& r) {
  if (r.base) cudaFree(r.base);
  r.base = nullptr;
  r.bytes = 0;
}

cudaError_t alloc_region(Region& r, size_t bytes) {
  free_region(r);
  if (bytes == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(&r.base, bytes);
  if (e != cudaSuccess) {
    r.base = nullptr;
    return e;
  }
  r.bytes = bytes;
  return cudaSuccess;
}

template <typename T>
T* carve(char*& p, int64_t count) {
  T* out = reinterpret_cast<T*>(p);
  p += align_up(sizeof(T) * (size_t)std::max<int64_t>(count, 1));
  return out;
}

bool is_capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
  return st != cudaStreamCaptureStatusNone;
}

// Scratch for the scans and sorts of up to `items` elements.
rgs_status ensure_scratch(rgs_ctx* ctx, State& s, int64_t items, bool capturing) {
  // The depth sort and the sort of the tiles' launch order run with small blocks over the
  // per-Gaussian and tile capacities, the tile sort with large blocks over the pair capacity;
  // the table must fit each.
  const int64_t small = std::max<int64_t>(std::max(s.vn_cap, s.tile_cap), 1);
  const int64_t hist = std::max(sort_hist_entries(small, kSortItemsSmall),
                                sort_hist_entries(std::max<int64_t>(items, 1)));
  const int64_t sums = std::max(scan_blocks(hist), scan_blocks(std::max<int64_t>(items, 1))) + 1;
  if (hist <= s.hist_cap && sums <= s.sums_cap) return RGS_OK;
  if (capturing) return fail(ctx, RGS_ERR_CAPACITY, "scratch too small during stream capture");
  RGS_CUDA(cudaDeviceSynchronize(), "sync before scratch growth");
  const size_t bytes = align_up(sizeof(uint32_t) * hist) + align_up(sizeof(uint32_t) * sums);
  RGS_CUDA(alloc_region(s.r_scratch, bytes), "allocate sort scratch");
  char* p = static_cast<char*>(s.r_scratch.base);
  s.hist = carve<uint32_t>(p, hist);
  s.block_sums = carve<uint32_t>(p, sums);
  s.hist_cap = hist;
  s.sums_cap = sums;
  return RGS_OK;
}

rgs_status ensure_vn(rgs_ctx* ctx, State& s, int64_t vn, int64_t n, int64_t pose_entries,
                     bool capturing, cudaStream_t stream) {
  if (n > s.n_cap) {
    if (capturing) return fail(ctx, RGS_ERR_CAPACITY, "per-Gaussian buffers grow during capture");
    RGS_CUDA(cudaDeviceSynchronize(), "sync before growth");
    RGS_CUDA(alloc_region(s.r_n, sizeof(unsigned long long) * n), "allocate visibility masks");
    s.vis_mask = static_cast<unsigned long long*>(s.r_n.base);
    RGS_CUDA(cudaMemsetAsync(s.vis_mask, 0, sizeof(unsigned long long) * n, stream),
             "zero visibility masks");
    s.n_cap = n;
  }
  if (vn > s.vn_cap) {
    if (capturing) return fail(ctx, RGS_ERR_CAPACITY, "per-Gaussian buffers grow during capture");
    RGS_CUDA(cudaDeviceSynchronize(), "sync before growth");
    const int64_t cap = vn;
    size_t bytes = 3 * align_up(sizeof(float4) * cap) + 7 * align_up(sizeof(uint32_t) * cap) +
                   align_up(sizeof(float) * kG2Stride * cap) +
                   align_up(sizeof(uint32_t) * vis_bit_words_cap(cap));
    RGS_CUDA(alloc_region(s.r_vn, bytes), "allocate per-Gaussian buffers");
    char* p = static_cast<char*>(s.r_vn.base);
    s.rec0 = carve<float4>(p, cap);
    s.rec1 = carve<float4>(p, cap);
    s.rec2 = carve<float4>(p, cap);
    s.ntiles = carve<uint32_t>(p, cap);
    s.vis_keys[0] = carve<uint32_t>(p, cap);
    s.vis_keys[1] = carve<uint32_t>(p, cap);
    s.vis_vals[0] = carve<uint32_t>(p, cap);
    s.vis_vals[1] = carve<uint32_t>(p, cap);
    s.offsets = carve<uint32_t>(p, cap);
    s.vis_list = carve<uint32_t>(p, cap);
    s.g2d = carve<float>(p, kG2Stride * cap);
    s.vis_bits = carve<uint32_t>(p, vis_bit_words_cap(cap));
    // The screen-space gradient accumulators start at zero; every backward leaves them zero.
    RGS_CUDA(cudaMemsetAsync(s.g2d, 0, sizeof(float) * kG2Stride * cap, stream), "zero g2d");
    s.vn_cap = cap;
  }
  if (pose_entries > s.pose_cap) {
    if (capturing) return fail(ctx, RGS_ERR_CAPACITY, "pose buffers grow during capture");
    RGS_CUDA(cudaDeviceSynchronize(), "sync before growth");
    RGS_CUDA(alloc_region(s.r_pose, sizeof(float) * pose_entries), "allocate pose partials");
    s.pose_partial = static_cast<float*>(s.r_pose.base);
    s.pose_cap = pose_entries;
  }
  return RGS_OK;
}

rgs_status ensure_pix_tiles(rgs_ctx* ctx, State& s, int64_t pixels, int64_t tiles,
                            bool capturing) {
  if (pixels > s.pix_cap) {
    if (capturing) return fail(ctx, RGS_ERR_CAPACITY, "pixel buffers grow during capture");
    RGS_CUDA(cudaDeviceSynchronize(), "sync before growth");
    RGS_CUDA(alloc_region(s.r_pix, align_up(sizeof(float) * pixels) +
                                        align_up(sizeof(int32_t) * pixels)),
             "allocate pixel state");
    char* p = static_cast<char*>(s.r_pix.base);
    s.t_final = carve<float>(p, pixels);
    s.last_index = carve<int32_t>(p, pixels);
    s.pix_cap = pixels;
  }
  if (tiles > s.tile_cap) {
    if (capturing) return fail(ctx, RGS_ERR_CAPACITY, "tile buffers grow during capture");
    RGS_CUDA(cudaDeviceSynchronize(), "sync before growth");
    RGS_CUDA(alloc_region(s.r_tile, align_up(sizeof(uint2) * tiles) +
                                         4 * align_up(sizeof(uint32_t) * tiles)),
             "allocate tile ranges");
    char* p = static_cast<char*>(s.r_tile.base);
    s.ranges = carve<uint2>(p, tiles);
    s.tile_keys[0] = carve<uint32_t>(p, tiles);
    s.tile_keys[1] = carve<uint32_t>(p, tiles);
    s.tile_vals[0] = carve<uint32_t>(p, tiles);
    s.tile_vals[1] = carve<uint32_t>(p, tiles);
    s.tile_cap = tiles;
  }
  return RGS_OK;
}

rgs_status ensure_pairs(rgs_ctx* ctx, State& s, int64_t pairs) {
  if (pairs <= s.pair_cap) return RGS_OK;
  RGS_CUDA(cudaDeviceSynchronize(), "sync before growth");
  const int64_t cap = std::max<int64_t>(pairs + pairs / 4, 4096);
  if (cap >= (int64_t)UINT32_MAX) return fail(ctx, RGS_ERR_INVALID_ARG, "pair list exceeds 2^32");
  RGS_CUDA(alloc_region(s.r_pair, 4 * align_up(sizeof(uint32_t) * cap)), "allocate pair lists");
  char* p = static_cast<char*>(s.r_pair.base);
  s.pair_keys[0] = carve<uint32_t>(p, cap);
  s.pair_keys[1] = carve<uint32_t>(p, cap);
  s.pair_vals[0] = carve<uint32_t>(p, cap);
  s.pair_vals[1] = carve<uint32_t>(p, cap);
  s.pair_cap = cap;
  return RGS_OK;
}

State* find_state(rgs_ctx* ctx, uint64_t id) {
  auto it = ctx->states.find(id);
  return it == ctx->states.end() ? nullptr : it->second;
}

rgs_status get_or_create_state(rgs_ctx* ctx, uint64_t* handle, State** out) {
  if (!handle) return fail(ctx, RGS_ERR_INVALID_ARG, "state handle pointer is null");
  if (*handle == 0) {
    State* s = new State();
    for (cudaEvent_t& e : s->ev) {
      if (cudaEventCreate(&e) != cudaSuccess) {
        e = nullptr;
        delete s;
        return fail(ctx, RGS_ERR_CUDA, "cudaEventCreate failed");
      }
    }
    const uint64_t id = ctx->next_id++;
    ctx->states[id] = s;
    *handle = id;
    *out = s;
    return RGS_OK;
  }
  State* s = find_state(ctx, *handle);
  if (!s) return fail(ctx, RGS_ERR_STATE, "unknown state handle");
  *out = s;
  return RGS_OK;
}

void destroy_state(State* s) {
  for (cudaEvent_t& e : s->ev)
    if (e) cudaEventDestroy(e);
  free_region(s->r_vn);
  free_region(s->r_n);
  free_region(s->r_pix);
  free_region(s->r_tile);
  free_region(s->r_pair);
  free_region(s->r_scratch);
  free_region(s->r_pose);
  free_region(s->r_counters);
  free_region(s->r_reg);
  delete s;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

rgs_status build_views(rgs_ctx* ctx, const rgs_camera* cams, int n_views, const rgs_config& cfg,
                       Views& views, Consts& consts) {
  if (!cams) return fail(ctx, RGS_ERR_INVALID_ARG, "cams is null");
  if (n_views < 1 || n_views > kMaxViews)
    return fail(ctx, RGS_ERR_INVALID_ARG, "n_views must be in 1..RGS_MAX_VIEWS");
  const int tw = cfg.tile_w, th = cfg.tile_h;
  const int ppt = cfg.pixels_per_thread == 0 ? 4 : cfg.pixels_per_thread;
  const int bwd_ppt = cfg.backward_pixels_per_thread == 0 ? ppt : cfg.backward_pixels_per_thread;
  if (!((tw == 16 && th == 16) || (tw == 8 && th == 8) || (tw == 32 && th == 8)))
    return fail(ctx, RGS_ERR_INVALID_ARG, "tile shape must be 16x16, 8x8 or 32x8");
  if (!(ppt == 1 || ppt == 2 || ppt == 4 || ppt == 8) || (tw * th / ppt) % 32 != 0)
    return fail(ctx, RGS_ERR_INVALID_ARG,
                "pixels_per_thread must be 1, 2, 4 or 8 with whole warps per tile");
  if (!(bwd_ppt == 1 || bwd_ppt == 2 || bwd_ppt == 4 || bwd_ppt == 8) ||
      (tw * th / bwd_ppt) % 32 != 0)
    return fail(ctx, RGS_ERR_INVALID_ARG,
                "backward_pixels_per_thread must be 0, 1, 2, 4 or 8 with whole warps per tile");
  std::memset(&views, 0, sizeof(views));
  views.n_views = n_views;
  views.tile_w = tw;
  views.tile_h = th;
  views.pixels_per_thread = ppt;
  views.bwd_pixels_per_thread = bwd_ppt;
  long long pix = 0;
  long long tiles = 0;
  for (int v = 0; v < n_views; ++v) {
    const rgs_camera& c = cams[v];
    if (c.width < 1 || c.height < 1 || c.width > 16384 || c.height > 16384)
      return fail(ctx, RGS_ERR_INVALID_ARG, "camera size out of range");
    if (!(c.fx > 0.0f) || !(c.fy > 0.0f) || !std::isfinite(c.cx) || !std::isfinite(c.cy))
      return fail(ctx, RGS_ERR_INVALID_ARG, "camera intrinsics invalid");
    for (int k = 0; k < 12; ++k)
      if (!std::isfinite(c.world_to_cam[k]))
        return fail(ctx, RGS_ERR_INVALID_ARG, "camera pose is not finite");
    ViewParams& vp = views.v[v];
    vp.width = c.width;
    vp.height = c.height;
    vp.tiles_x = (c.width + tw - 1) / tw;
    vp.tiles_y = (c.height + th - 1) / th;
    vp.tile_base = (int)tiles;
    vp.pixel_offset = pix;
    vp.fx = c.fx;
    vp.fy = c.fy;
    vp.cx = c.cx;
    vp.cy = c.cy;
    for (int a = 0; a < 3; ++a) {
      for (int b = 0; b < 3; ++b) vp.R[3 * a + b] = c.world_to_cam[4 * a + b];
      vp.t[a] = c.world_to_cam[4 * a + 3];
    }
    for (int a = 0; a < 3; ++a) {
      double s = 0.0;
      for (int b = 0; b < 3; ++b) s -= (double)vp.R[3 * b + a] * (double)vp.t[b];
      vp.cam_center[a] = (float)s;
    }
    if (cfg.jac_clamp > 0.0f) {
      vp.lim_u = (float)((double)cfg.jac_clamp * 0.5 * c.width / c.fx);
      vp.lim_w = (float)((double)cfg.jac_clamp * 0.5 * c.height / c.fy);
    } else {
      vp.lim_u = vp.lim_w = 0.0f;
    }
    tiles += (long long)vp.tiles_x * vp.tiles_y;
    pix += (long long)c.width * c.height;
  }
  if (tiles >= (1ll << 31) || pix >= (1ll << 31))
    return fail(ctx, RGS_ERR_INVALID_ARG, "too many pixels or tiles in one batch");
  views.total_tiles = (int)tiles;
  views.total_pixels = pix;
  consts.alpha_min = cfg.alpha_min;
  consts.alpha_max = cfg.alpha_max;
  consts.t_min = cfg.t_min;
  consts.znear = cfg.znear;
  consts.eps2d = cfg.eps2d;
  for (int k = 0; k < 3; ++k) consts.bg[k] = cfg.bg[k];
  consts.log2_alpha_min = (float)std::log2((double)cfg.alpha_min);
  consts.unclamped_neg_lo = (float)(1e-5 - std::log2((double)cfg.alpha_max));
  if (!(cfg.alpha_min > 0.0f) || !(cfg.alpha_max > cfg.alpha_min) || !(cfg.alpha_max < 1.0f) ||
      !(cfg.t_min > 0.0f) || !(cfg.eps2d >= 0.0f) || !(cfg.znear > 0.0f) ||
      !std::isfinite(cfg.znear))
    return fail(ctx, RGS_ERR_INVALID_ARG, "config values out of range");
  return RGS_OK;
}

// Records phase event k of state s when timing is enabled (as a graph node under capture).
cudaError_t mark(const rgs_ctx* ctx, State& s, int k, cudaStream_t stream, bool capturing) {
  if (!ctx->timing) return cudaSuccess;
  return cudaEventRecordWithFlags(s.ev[k], stream,
                                  capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
}

int bits_for(uint32_t count) {  // bits needed to represent values in [0, count)
  int b = 0;
  while (b < 32 && (count - 1) >> b) ++b;
  return std::max(b, 1);
}

}  // namespace

extern "C" {

void rgs_config_default(rgs_config* cfg) {
  if (!cfg) return;
  cfg->alpha_min = 1.0f / 255.0f;
  cfg->alpha_max = 0.99f;
  cfg->t_min = 1e-4f;
  cfg->znear = 0.2f;
  cfg->eps2d = 0.3f;
  cfg->jac_clamp = 1.3f;
  cfg->bg[0] = cfg->bg[1] = cfg->bg[2] = 0.0f;
  cfg->tile_w = 16;
  cfg->tile_h = 16;
  cfg->pixels_per_thread = 4;
  cfg->backward_pixels_per_thread = 0;
  cfg->sh_ready_event = nullptr;
}

rgs_status rgs_create(rgs_ctx** out, int device) {
  if (!out) return RGS_ERR_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count)
    return RGS_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return RGS_ERR_CUDA;
  rgs_ctx* ctx = new rgs_ctx();
  ctx->device = device;
  // Decide once, outside any stream capture, whether sorts can run as one cluster launch.
  (void)cluster_sort_capacity(device);
  if (cudaMallocHost(&ctx->host_counters, sizeof(Counters)) != cudaSuccess) {
    delete ctx;
    return RGS_ERR_NOMEM;
  }
  if (cudaMalloc(&ctx->track_sums, sizeof(double) * 4 * kMaxViews) != cudaSuccess) {
    cudaFreeHost(ctx->host_counters);
    delete ctx;
    return RGS_ERR_NOMEM;
  }
  *out = ctx;
  return RGS_OK;
}

void rgs_destroy(rgs_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  for (auto& kv : ctx->states) destroy_state(kv.second);
  ctx->states.clear();
  if (ctx->host_counters) cudaFreeHost(ctx->host_counters);
  if (ctx->track_sums) cudaFree(ctx->track_sums);
  free_region(ctx->r_seed);
  delete ctx;
}

const char* rgs_last_error(const rgs_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

rgs_status rgs_autotune(rgs_ctx* ctx, const rgs_gaussians* g, const rgs_camera* cams,
                        int32_t n_views, rgs_config* cfg, float* ms_out, void* stream_ptr) {
  if (!ctx || !g || !cams || !cfg) return RGS_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (ms_out) *ms_out = 0.0f;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
  if (is_capturing(stream)) return fail(ctx, RGS_ERR_INVALID_ARG, "autotune under stream capture");
  if (n_views < 1 || n_views > kMaxViews)
    return fail(ctx, RGS_ERR_INVALID_ARG, "n_views must be in 1..RGS_MAX_VIEWS");
  std::string key = std::to_string(g->n) + ":" + std::to_string(g->sh_degree);
  int64_t pixels = 0;
  for (int v = 0; v < n_views; ++v) {
    key += ":" + std::to_string(cams[v].width) + "x" + std::to_string(cams[v].height);
    pixels += (int64_t)cams[v].width * cams[v].height;
  }
  auto hit = ctx->tune_cache.find(key);
  if (hit != ctx->tune_cache.end()) {
    cfg->tile_w = hit->second.tile_w;
    cfg->tile_h = hit->second.tile_h;
    cfg->pixels_per_thread = hit->second.ppt;
    cfg->backward_pixels_per_thread = hit->second.bwd_ppt;
    return RGS_OK;
  }
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, RGS_ERR_CUDA, "cudaSetDevice");
  const int K = (g->sh_degree + 1) * (g->sh_degree + 1);
  const int64_t n = g->n;
  // Scratch: images [P,5], upstream colour gradient [P,3], parameter and pose gradients.
  const int64_t n1 = std::max<int64_t>(n, 1);
  const size_t bytes = align_up(sizeof(float) * 5 * pixels) + align_up(sizeof(float) * 3 * pixels) +
                       3 * align_up(sizeof(float) * 4 * n1) + align_up(sizeof(float) * n1) +
                       align_up(sizeof(float) * 3 * K * n1) + align_up(sizeof(float) * 6 * n_views);
  char* base = nullptr;
  RGS_CUDA(cudaMalloc(&base, bytes), "autotune scratch");
  char* p = base;
  float* img = carve<float>(p, 5 * pixels);
  float* upc = carve<float>(p, 3 * pixels);
  float* d_means = carve<float>(p, 4 * n1);
  float* d_ls = carve<float>(p, 4 * n1);
  float* d_q = carve<float>(p, 4 * n1);
  float* d_o = carve<float>(p, n1);
  float* d_sh = carve<float>(p, 3 * K * n1);
  float* dpose = carve<float>(p, 6 * n_views);
  rgs_status result = RGS_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
  uint64_t state = 0;
  do {
    // Every byte 0x3a makes each upstream value 7.1e-4: a non-zero colour gradient, so that the
    // trials' backward blends issue their gradient atomics as under a real loss (with zeros the
    // all-zero sums skip them, which favoured the settings with more atomics).
    if (cudaMemsetAsync(upc, 0x3a, sizeof(float) * 3 * pixels, stream) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaEventCreate(&e2) != cudaSuccess) {
      result = fail(ctx, RGS_ERR_CUDA, "autotune setup");
      break;
    }
    rgs_images out{img, img + 3 * pixels, img + 4 * pixels};
    rgs_image_grads up{upc, nullptr, nullptr};
    const uint32_t mask = RGS_GRAD_ALL;
    struct Shape {
      int tile_w, tile_h;
    };
    const Shape shapes[] = {{16, 16}, {8, 8}, {32, 8}};
    const int ppts[] = {4, 8, 2, 1};
    float best = 1e30f;
    TuneChoice choice{16, 16, 4, 4};
    for (const Shape& sh : shapes) {
      // The blends share only the tile shape, so per shape the forward and the backward setting
      // are chosen independently.
      float best_f = 1e30f, best_b = 1e30f;
      int ppt_f = 0, ppt_b = 0;
      for (const int ppt : ppts) {
        if ((sh.tile_w * sh.tile_h / ppt) % 32 != 0) continue;
        rgs_config trial = *cfg;
        trial.tile_w = sh.tile_w;
        trial.tile_h = sh.tile_h;
        trial.pixels_per_thread = ppt;
        trial.backward_pixels_per_thread = ppt;
        trial.sh_ready_event = nullptr;  // the trials run on coefficients already on the device
        // The fastest of four timed runs (after one warm-up) of each blend: the minimum is the
        // least disturbed by the eager forward's host synchronisations and other tenants.
        float t_f = 1e30f, t_b = 1e30f;
        for (int it = 0; it < 5 && result == RGS_OK; ++it) {
          cudaEventRecord(e0, stream);
          rgs_status st = rgs_render_forward(ctx, g, cams, n_views, &trial, &out, &state, stream);
          cudaEventRecord(e1, stream);
          if (st == RGS_OK)
            st = rgs_render_backward(ctx, state, &up, mask, d_means, d_ls, d_q, d_o, d_sh, dpose,
                                     stream);
          cudaEventRecord(e2, stream);
          float ms_f = 0.0f, ms_b = 0.0f;
          if (st != RGS_OK) {
            result = st;
          } else if (cudaEventSynchronize(e2) != cudaSuccess ||
                     cudaEventElapsedTime(&ms_f, e0, e1) != cudaSuccess ||
                     cudaEventElapsedTime(&ms_b, e1, e2) != cudaSuccess) {
            result = fail(ctx, RGS_ERR_CUDA, "autotune timing");
          } else if (it > 0) {  // the first run is the warm-up
            t_f = fminf(t_f, ms_f);
            t_b = fminf(t_b, ms_b);
          }
        }
        if (result != RGS_OK) break;
        if (t_f < best_f) {
          best_f = t_f;
          ppt_f = ppt;
        }
        if (t_b < best_b) {
          best_b = t_b;
          ppt_b = ppt;
        }
      }
      if (result != RGS_OK) break;
      if (ppt_f != 0 && best_f + best_b < best) {
        best = best_f + best_b;
        choice = TuneChoice{sh.tile_w, sh.tile_h, ppt_f, ppt_b};
      }
    }
    if (result != RGS_OK) break;
    ctx->tune_cache[key] = choice;
    cfg->tile_w = choice.tile_w;
    cfg->tile_h = choice.tile_h;
    cfg->pixels_per_thread = choice.ppt;
    cfg->backward_pixels_per_thread = choice.bwd_ppt;
    if (ms_out) *ms_out = best;
  } while (false);
  cudaStreamSynchronize(stream);
  if (state) {
    auto it = ctx->states.find(state);
    if (it != ctx->states.end()) {
      destroy_state(it->second);
      ctx->states.erase(it);
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e2) cudaEventDestroy(e2);
  cudaFree(base);
  return result;
}

rgs_status rgs_release_state(rgs_ctx* ctx, uint64_t handle) {
  if (!ctx) return RGS_ERR_INVALID_ARG;
  State* s = find_state(ctx, handle);
  if (!s) return fail(ctx, RGS_ERR_STATE, "unknown state handle");
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();  // queued work may still read the state's buffers
  destroy_state(s);
  ctx->states.erase(handle);
  return RGS_OK;
}

rgs_status rgs_reserve(rgs_ctx* ctx, uint64_t* handle, int64_t pair_capacity, void* stream) {
  (void)stream;
  if (!ctx) return RGS_ERR_INVALID_ARG;
  State* s = nullptr;
  rgs_status st = get_or_create_state(ctx, handle, &s);
  if (st != RGS_OK) return st;
  cudaSetDevice(ctx->device);
  if (pair_capacity > 0) {
    st = ensure_pairs(ctx, *s, pair_capacity);
    if (st != RGS_OK) return st;
    st = ensure_scratch(ctx, *s, std::max<int64_t>(s->pair_cap, s->vn_cap), false);
    if (st != RGS_OK) return st;
  }
  return RGS_OK;
}

namespace {
rgs_status render_forward(rgs_ctx* ctx, const rgs_gaussians* g, const rgs_camera* cams,
                          int32_t n_views, const float* world_to_cam, const rgs_config* cfg_in,
                          rgs_images* out, uint64_t* handle, void* stream_ptr);
}  // namespace

rgs_status rgs_render_forward(rgs_ctx* ctx, const rgs_gaussians* g, const rgs_camera* cams,
                              int32_t n_views, const rgs_config* cfg_in, rgs_images* out,
                              uint64_t* handle, void* stream_ptr) {
  return render_forward(ctx, g, cams, n_views, nullptr, cfg_in, out, handle, stream_ptr);
}

rgs_status rgs_render_forward_posed(rgs_ctx* ctx, const rgs_gaussians* g,
                                    const rgs_camera* cams, int32_t n_views,
                                    const float* world_to_cam, const rgs_config* cfg_in,
                                    rgs_images* out, uint64_t* handle, void* stream_ptr) {
  if (!ctx) return RGS_ERR_INVALID_ARG;
  if (!world_to_cam) {
    ctx->last_error = "world_to_cam is null";
    return RGS_ERR_INVALID_ARG;
  }
  return render_forward(ctx, g, cams, n_views, world_to_cam, cfg_in, out, handle, stream_ptr);
}

namespace {
rgs_status render_forward(rgs_ctx* ctx, const rgs_gaussians* g, const rgs_camera* cams,
                          int32_t n_views, const float* world_to_cam, const rgs_config* cfg_in,
                          rgs_images* out, uint64_t* handle, void* stream_ptr) {
  if (!ctx) return RGS_ERR_INVALID_ARG;
  ctx->last_error.clear();
  cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
  if (!g || !out) return fail(ctx, RGS_ERR_INVALID_ARG, "null gaussians or output struct");
  if (g->n < 0 || g->sh_degree < 0 || g->sh_degree > 3)
    return fail(ctx, RGS_ERR_INVALID_ARG, "n must be >= 0 and sh_degree in 0..3");
  if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh))
    return fail(ctx, RGS_ERR_INVALID_ARG, "null Gaussian parameter pointer");
  if (g->n > 0 && (!aligned16(g->means) || !aligned16(g->log_scales) || !aligned16(g->quats) ||
                   !aligned16(g->opacity_logits) || !aligned16(g->sh)))
    return fail(ctx, RGS_ERR_INVALID_ARG, "Gaussian parameter pointers must be 16-byte aligned");
  if (!out->color || !out->depth || !out->alpha)
    return fail(ctx, RGS_ERR_INVALID_ARG, "null output image pointer");
  rgs_config cfg;
  if (cfg_in) cfg = *cfg_in; else rgs_config_default(&cfg);
  Views views;
  Consts consts;
  rgs_status st = build_views(ctx, cams, n_views, cfg, views, consts);
  if (st != RGS_OK) return st;
  const int64_t vn = (int64_t)n_views * g->n;
  if (vn >= (1ll << 31)) return fail(ctx, RGS_ERR_INVALID_ARG, "n_views * n must be < 2^31");
  if (cudaSetDevice(ctx->device) != cudaSuccess)
    return fail(ctx, RGS_ERR_CUDA, "cudaSetDevice failed");
  const bool capturing = is_capturing(stream);
  State* s = nullptr;
  st = get_or_create_state(ctx, handle, &s);
  if (st != RGS_OK) return st;
  s->has_forward = false;
  const int64_t pose_entries = (int64_t)preprocess_backward_blocks(vn) * n_views * 6;
  st = ensure_vn(ctx, *s, vn, g->n, pose_entries, capturing, stream);
  if (st != RGS_OK) return st;
  st = ensure_pix_tiles(ctx, *s, views.total_pixels, views.total_tiles, capturing);
  if (st != RGS_OK) return st;
  st = ensure_scratch(ctx, *s, std::max<int64_t>(vn, s->pair_cap), capturing);
  if (st != RGS_OK) return st;
  // Pose records, then the counters and the bookkeeping of the two single-pass scans (the
  // compaction and the pair offsets), which one memset zeroes at the start of every forward.
  const size_t pose_bytes = align_up(sizeof(float) * 16 * kMaxViews);
  const size_t lb_bytes = align_up(lookback_bytes(s->vn_cap));
  const size_t reset_bytes = align_up(sizeof(Counters)) + 2 * lb_bytes;
  if (s->r_counters.bytes < pose_bytes + reset_bytes) {
    if (capturing) return fail(ctx, RGS_ERR_CAPACITY, "counters grow during capture");
    if (s->r_counters.base) RGS_CUDA(cudaDeviceSynchronize(), "sync before counters growth");
    RGS_CUDA(alloc_region(s->r_counters, pose_bytes + reset_bytes), "allocate counters");
  }
  s->pose_records = static_cast<float*>(s->r_counters.base);
  s->counters = reinterpret_cast<Counters*>(static_cast<char*>(s->r_counters.base) + pose_bytes);
  char* lb_area = reinterpret_cast<char*>(s->counters) + align_up(sizeof(Counters));
  if (world_to_cam) views.pose_dev = s->pose_records;
  s->g = *g;
  s->views = views;
  s->consts = consts;
  s->vn = vn;
  Counters* cnt = s->counters;
  const uint64_t launches0 = launch_counter();
  s->fwd_timed = ctx->timing;
  RGS_CUDA(cudaMemsetAsync(cnt, 0, reset_bytes, stream), "reset counters");
  // Tiles without pairs keep the empty range [0, 0); the range kernel writes the others.
  RGS_CUDA(cudaMemsetAsync(s->ranges, 0, sizeof(uint2) * (size_t)views.total_tiles, stream),
           "reset tile ranges");
  RGS_CUDA(mark(ctx, *s, 0, stream, capturing), "event");
  // Device poses: records (R, t, camera centre) for the projection kernels and the backward.
  if (world_to_cam)
    RGS_CUDA(launch_pose_prepare(world_to_cam, n_views, s->pose_records, stream), "pose records");

  // 1. Projection.
  // The cull pass's candidate list lives in the depth sort's second key buffer, which is free
  // until the sort starts.
  // The colours are evaluated in the projection, unless the caller's SH coefficients may still
  // be in flight: then after the sorts, behind the caller's event.
  const bool defer_colour = cfg.sh_ready_event != nullptr;
  RGS_CUDA(launch_preprocess_forward(views, consts, *g, s->rec0, s->rec1, s->rec2, s->ntiles,
                                     s->vis_keys[1], s->vis_bits, defer_colour, cnt, stream),
           "preprocess");
  RGS_CUDA(mark(ctx, *s, 1, stream, capturing), "event");
  // 2. Visible entries with depth keys, in (view, Gaussian) order.
  RGS_CUDA(launch_compact_visible(s->vis_bits, n_views, g->n, s->rec2, s->vis_keys[0],
                                  s->vis_vals[0], s->vis_list, &cnt->n_visible,
                                  lookback_at(lb_area, &cnt->status, s->vn_cap), stream),
           "compact");
  RGS_CUDA(mark(ctx, *s, 2, stream, capturing), "event");
  // Size the sorted list of visible entries (outside capture: read the count back; under
  // capture the capacity of the last eager call holds, and a larger count is clamped to it and
  // recorded in the status word).
  if (!capturing) {
    RGS_CUDA(cudaMemcpyAsync(ctx->host_counters, cnt, sizeof(Counters), cudaMemcpyDeviceToHost,
                             stream),
             "read counters");
    RGS_CUDA(cudaStreamSynchronize(stream), "sync for visible count");
    const int64_t nv = ctx->host_counters->n_visible;
    if (nv > s->vis_cap) s->vis_cap = std::max<int64_t>(nv + nv / 4, 1024);
  } else if (s->vis_cap == 0) {
    s->vis_cap = vn;
  }
  const int64_t vis_cap = std::min<int64_t>(s->vis_cap, vn);
  // 3. Stable sort by depth (positive float bits order like the values; the sign bit is 0).
  bool alt = false;
  RGS_CUDA(launch_radix_sort(s->vis_keys[0], s->vis_vals[0], s->vis_keys[1], s->vis_vals[1],
                             vis_cap, &cnt->n_visible, 0, 31, s->hist, s->block_sums, &alt,
                             stream, kSortItemsSmall),
           "depth sort");
  s->order = s->vis_vals[alt ? 1 : 0];
  RGS_CUDA(mark(ctx, *s, 3, stream, capturing), "event");
  // 4. Pair offsets in depth order.
  RGS_CUDA(launch_gather_scan(s->ntiles, s->order, vis_cap, &cnt->n_visible, s->offsets,
                              &cnt->n_pairs, s->block_sums,
                              lookback_at(lb_area + lb_bytes, &cnt->status, s->vn_cap), stream),
           "pair offsets");
  RGS_CUDA(mark(ctx, *s, 4, stream, capturing), "event");
  // Size the pair list (outside capture: read the count back and grow if needed).
  int64_t pair_bound = s->pair_cap;
  if (!capturing) {
    RGS_CUDA(cudaMemcpyAsync(ctx->host_counters, cnt, sizeof(Counters), cudaMemcpyDeviceToHost,
                             stream),
             "read counters");
    RGS_CUDA(cudaStreamSynchronize(stream), "sync for pair count");
    const int64_t pairs = ctx->host_counters->n_pairs;
    st = ensure_pairs(ctx, *s, pairs);
    if (st != RGS_OK) return st;
    st = ensure_scratch(ctx, *s, std::max<int64_t>(vn, s->pair_cap), false);
    if (st != RGS_OK) return st;
    pair_bound = pairs;
  } else if (s->pair_cap == 0) {
    return fail(ctx, RGS_ERR_CAPACITY, "pair list has no capacity under capture: rgs_reserve");
  }
  const uint32_t capacity = (uint32_t)s->pair_cap;
  // 5. Duplicate (tile, vi) pairs in depth order.
  RGS_CUDA(launch_duplicate(views, g->n, s->order, s->offsets, s->ntiles, s->rec0, s->rec1,
                            s->rec2, consts.log2_alpha_min, vis_cap, capacity, s->pair_keys[0],
                            s->pair_vals[0], cnt, stream),
           "duplicate");
  RGS_CUDA(mark(ctx, *s, 5, stream, capturing), "event");
  // 6. Stable sort by global tile id.
  alt = false;
  // Keys are tile ids in [0, total_tiles]; total_tiles itself marks an unused slot.
  const int tile_bits = bits_for((uint32_t)views.total_tiles + 1u);
  RGS_CUDA(launch_radix_sort(s->pair_keys[0], s->pair_vals[0], s->pair_keys[1], s->pair_vals[1],
                             std::min<int64_t>(pair_bound, s->pair_cap), &cnt->n_pairs_stored, 0,
                             tile_bits, s->hist, s->block_sums, &alt, stream),
           "tile sort");
  const uint32_t* sorted_keys = s->pair_keys[alt ? 1 : 0];
  s->sorted_vals = s->pair_vals[alt ? 1 : 0];
  RGS_CUDA(mark(ctx, *s, 6, stream, capturing), "event");
  // 7. Tile ranges.
  // Tile ranges and, when deferred, the colours of the visible entries, in one launch: the
  // colours are then the first read of the SH coefficients, so the caller's upload of them may
  // run until here.
  if (defer_colour)
    RGS_CUDA(cudaStreamWaitEvent(stream, static_cast<cudaEvent_t>(cfg.sh_ready_event), 0),
             "wait for the SH coefficients");
  RGS_CUDA(launch_ranges_colour(sorted_keys, views.total_tiles, s->ranges,
                                (uint32_t)std::min<int64_t>(pair_bound, s->pair_cap), views, *g,
                                s->vis_list, vis_cap, defer_colour, s->rec1, s->rec2, cnt,
                                stream),
           "tile ranges and colours");
  RGS_CUDA(launch_tile_order(s->ranges, views.total_tiles, s->tile_keys[0], s->tile_vals[0],
                             s->tile_keys[1], s->tile_vals[1], s->hist, s->block_sums,
                             &s->tile_order, stream),
           "tile order");
  RGS_CUDA(mark(ctx, *s, 7, stream, capturing), "event");
  // 8. Blend.
  RGS_CUDA(launch_blend(true, views, consts, s->ranges, s->sorted_vals, s->rec0, s->rec1,
                        s->rec2, out->color, out->depth, out->alpha, s->t_final, s->last_index,
                        nullptr, nullptr, nullptr, nullptr, s->tile_order, cnt, stream),
           "blend forward");
  RGS_CUDA(mark(ctx, *s, 8, stream, capturing), "event");
  s->fwd_launches = (uint32_t)(launch_counter() - launches0);
  s->has_forward = true;
  return RGS_OK;
}
}  // namespace

namespace {
rgs_status render_backward(rgs_ctx* ctx, uint64_t handle, const rgs_image_grads* grads,
                           uint32_t grad_mask, float* d_means, float* d_log_scales,
                           float* d_quats, float* d_opacity_logits, float* d_sh, float* d_pose,
                           const rgs_map_reg* reg, void* stream_ptr);
}  // namespace

rgs_status rgs_render_backward(rgs_ctx* ctx, uint64_t handle, const rgs_image_grads* grads,
                               uint32_t grad_mask, float* d_means, float* d_log_scales,
                               float* d_quats, float* d_opacity_logits, float* d_sh,
                               float* d_pose, void* stream_ptr) {
  return render_backward(ctx, handle, grads, grad_mask, d_means, d_log_scales, d_quats,
                         d_opacity_logits, d_sh, d_pose, nullptr, stream_ptr);
}

rgs_status rgs_render_backward_mapping(rgs_ctx* ctx, uint64_t handle,
                                       const rgs_image_grads* grads, uint32_t grad_mask,
                                       float* d_means, float* d_log_scales, float* d_quats,
                                       float* d_opacity_logits, float* d_sh, float* d_pose,
                                       const rgs_map_reg* reg, void* stream_ptr) {
  return render_backward(ctx, handle, grads, grad_mask, d_means, d_log_scales, d_quats,
                         d_opacity_logits, d_sh, d_pose, reg, stream_ptr);
}

namespace {
rgs_status render_backward(rgs_ctx* ctx, uint64_t handle, const rgs_image_grads* grads,
                           uint32_t grad_mask, float* d_means, float* d_log_scales,
                           float* d_quats, float* d_opacity_logits, float* d_sh, float* d_pose,
                           const rgs_map_reg* reg, void* stream_ptr) {
  if (!ctx) return RGS_ERR_INVALID_ARG;
  ctx->last_error.clear();
  cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
  State* s = find_state(ctx, handle);
  if (!s) return fail(ctx, RGS_ERR_STATE, "unknown state handle");
  if (!s->has_forward) return fail(ctx, RGS_ERR_STATE, "state holds no completed forward");
  if (grad_mask & ~RGS_GRAD_ALL) return fail(ctx, RGS_ERR_INVALID_ARG, "unknown grad_mask bits");
  const int n = s->g.n;
  struct Need { uint32_t bit; const void* p; const char* name; bool vec4; };
  const Need needs[] = {{RGS_GRAD_MEANS, d_means, "d_means", false},
                        {RGS_GRAD_SCALES, d_log_scales, "d_log_scales", false},
                        {RGS_GRAD_QUATS, d_quats, "d_quats", true},
                        {RGS_GRAD_OPACITY, d_opacity_logits, "d_opacity_logits", false},
                        {RGS_GRAD_SH, d_sh, "d_sh", true},
                        {RGS_GRAD_POSE, d_pose, "d_pose", false}};
  for (const Need& nd : needs) {
    if (!(grad_mask & nd.bit)) continue;
    if (!nd.p && (n > 0 || nd.bit == RGS_GRAD_POSE))
      return fail(ctx, RGS_ERR_INVALID_ARG, std::string(nd.name) + " is null but requested");
    if (nd.p && nd.vec4 && !aligned16(nd.p))
      return fail(ctx, RGS_ERR_INVALID_ARG, std::string(nd.name) + " must be 16-byte aligned");
  }
  const float* dc = grads ? grads->d_color : nullptr;
  const float* dd = grads ? grads->d_depth : nullptr;
  const float* da = grads ? grads->d_alpha : nullptr;
  if (cudaSetDevice(ctx->device) != cudaSuccess)
    return fail(ctx, RGS_ERR_CUDA, "cudaSetDevice failed");
  const bool capturing = is_capturing(stream);
  MapReg mreg{};
  if (reg) {
    if (!std::isfinite(reg->lambda_iso) || !std::isfinite(reg->lambda_alpha) ||
        !std::isfinite(reg->lambda_mu))
      return fail(ctx, RGS_ERR_INVALID_ARG, "regulariser weights must be finite");
    mreg.lambda_iso = reg->lambda_iso;
    mreg.lambda_alpha = reg->lambda_alpha;
    mreg.lambda_mu = reg->lambda_mu;
    mreg.ema_means = reg->ema_means;
    mreg.obs_count = reg->obs_count;
    mreg.vis_score = reg->vis_score;
    mreg.value = reg->value;
    if (reg->value && n > 0) {
      if (s->reg_cap < n) {
        if (capturing)
          return fail(ctx, RGS_ERR_CAPACITY, "regulariser scratch: make a first call outside capture");
        free_region(s->r_reg);
        RGS_CUDA(alloc_region(s->r_reg, sizeof(float) * (size_t)n), "allocate regulariser scratch");
        s->reg_vals = static_cast<float*>(s->r_reg.base);
        s->reg_cap = n;
      }
      mreg.values = s->reg_vals;
    }
  }
  const uint64_t launches0 = launch_counter();
  s->bwd_timed = ctx->timing;
  RGS_CUDA(mark(ctx, *s, kEvBwd0, stream, capturing), "event");
  RGS_CUDA(launch_blend(false, s->views, s->consts, s->ranges, s->sorted_vals, s->rec0, s->rec1,
                        s->rec2, nullptr, nullptr, nullptr, s->t_final, s->last_index, dc, dd, da,
                        s->g2d, s->tile_order, s->counters, stream),
           "blend backward");
  RGS_CUDA(mark(ctx, *s, kEvBwd0 + 1, stream, capturing), "event");
  RGS_CUDA(launch_preprocess_backward(s->views, s->consts, s->g, s->vis_mask, s->vis_list,
                                      s->counters, s->vn, s->g2d, grad_mask, d_means,
                                      d_log_scales, d_quats, d_opacity_logits, d_sh,
                                      s->pose_partial, d_pose, reg ? &mreg : nullptr, stream),
           "preprocess backward");
  RGS_CUDA(mark(ctx, *s, kEvBwd0 + 2, stream, capturing), "event");
  s->bwd_launches = (uint32_t)(launch_counter() - launches0);
  return RGS_OK;
}
}  // namespace

rgs_status rgs_set_phase_timing(rgs_ctx* ctx, int32_t enable) {
  if (!ctx) return RGS_ERR_INVALID_ARG;
  ctx->timing = enable != 0;
  return RGS_OK;
}

rgs_status rgs_phase_times(rgs_ctx* ctx, uint64_t handle, float* ms, int32_t n,
                           void* stream_ptr) {
  if (!ctx || !ms || n < 0) return RGS_ERR_INVALID_ARG;
  State* s = find_state(ctx, handle);
  if (!s) return fail(ctx, RGS_ERR_STATE, "unknown state handle");
  for (int k = 0; k < n; ++k) ms[k] = 0.0f;
  cudaSetDevice(ctx->device);
  RGS_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream_ptr)), "sync for timing");
  // Forward phases k = 0..7 lie between events k and k + 1; backward phases 8, 9 between the
  // backward events.
  for (int k = 0; k < n && k < RGS_PHASE_COUNT; ++k) {
    const bool fwd = k < RGS_PHASE_BLEND_BACKWARD;
    if (fwd ? !s->fwd_timed : !s->bwd_timed) continue;
    const int e0 = fwd ? k : kEvBwd0 + (k - RGS_PHASE_BLEND_BACKWARD);
    float t = 0.0f;
    RGS_CUDA(cudaEventElapsedTime(&t, s->ev[e0], s->ev[e0 + 1]), "event timing");
    ms[k] = t;
  }
  return RGS_OK;
}

rgs_status rgs_query_stats(rgs_ctx* ctx, uint64_t handle, rgs_stats* out, void* stream_ptr) {
  if (!ctx || !out) return RGS_ERR_INVALID_ARG;
  State* s = find_state(ctx, handle);
  if (!s) return fail(ctx, RGS_ERR_STATE, "unknown state handle");
  std::memset(out, 0, sizeof(*out));
  out->pair_capacity = s->pair_cap;
  out->state_bytes = (int64_t)(s->r_vn.bytes + s->r_n.bytes + s->r_pix.bytes + s->r_tile.bytes +
                               s->r_pair.bytes + s->r_scratch.bytes + s->r_pose.bytes +
                               s->r_counters.bytes);
  if (!s->counters) return RGS_OK;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
  cudaSetDevice(ctx->device);
  RGS_CUDA(cudaMemcpyAsync(ctx->host_counters, s->counters, sizeof(Counters),
                           cudaMemcpyDeviceToHost, stream),
           "read counters");
  RGS_CUDA(cudaStreamSynchronize(stream), "sync for stats");
  const Counters& c = *ctx->host_counters;
  out->n_visible = c.n_visible;
  out->n_pairs = c.n_pairs;
  out->n_eval = (int64_t)c.n_eval;
  out->n_contrib = (int64_t)c.n_contrib;
  out->n_nonfinite = c.n_nonfinite;
  out->status = c.status;
  out->kernel_launches = s->fwd_launches + s->bwd_launches;
  return RGS_OK;
}

rgs_status rgs_copy_tile_lists(rgs_ctx* ctx, uint64_t handle, uint32_t* host_vals,
                               int64_t vals_cap, uint32_t* host_ranges, int64_t* n_pairs,
                               void* stream_ptr) {
  if (!ctx || !n_pairs) return RGS_ERR_INVALID_ARG;
  State* s = find_state(ctx, handle);
  if (!s || !s->has_forward) return fail(ctx, RGS_ERR_STATE, "state holds no completed forward");
  cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
  cudaSetDevice(ctx->device);
  RGS_CUDA(cudaMemcpyAsync(ctx->host_counters, s->counters, sizeof(Counters),
                           cudaMemcpyDeviceToHost, stream),
           "read counters");
  RGS_CUDA(cudaStreamSynchronize(stream), "sync");
  const int64_t np = ctx->host_counters->n_pairs_stored;
  *n_pairs = np;
  if (host_vals && np <= vals_cap && np > 0)
    RGS_CUDA(cudaMemcpyAsync(host_vals, s->sorted_vals, sizeof(uint32_t) * np,
                             cudaMemcpyDeviceToHost, stream),
             "copy pair list");
  if (host_ranges && s->views.total_tiles > 0)
    RGS_CUDA(cudaMemcpyAsync(host_ranges, s->ranges, sizeof(uint2) * s->views.total_tiles,
                             cudaMemcpyDeviceToHost, stream),
             "copy tile ranges");
  RGS_CUDA(cudaStreamSynchronize(stream), "sync");
  return RGS_OK;
}

rgs_status rgs_copy_records(rgs_ctx* ctx, uint64_t handle, float* host_rec,
                            uint32_t* host_ntiles, void* stream_ptr) {
  if (!ctx || !host_rec) return RGS_ERR_INVALID_ARG;
  State* s = find_state(ctx, handle);
  if (!s || !s->has_forward) return fail(ctx, RGS_ERR_STATE, "state holds no completed forward");
  cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
  cudaSetDevice(ctx->device);
  const int64_t vn = s->vn;
  if (vn > 0) {
    const float4* recs[3] = {s->rec0, s->rec1, s->rec2};
    for (int k = 0; k < 3; ++k)
      RGS_CUDA(cudaMemcpy2DAsync(host_rec + 4 * k, 12 * sizeof(float), recs[k], sizeof(float4),
                                 sizeof(float4), (size_t)vn, cudaMemcpyDeviceToHost, stream),
               "copy records");
    if (host_ntiles)
      RGS_CUDA(cudaMemcpyAsync(host_ntiles, s->ntiles, sizeof(uint32_t) * vn,
                               cudaMemcpyDeviceToHost, stream),
               "copy tile counts");
  }
  std::vector<uint32_t> bits;
  const int64_t n = s->g.n, words = vis_bit_words_per_view(n);
  if (host_ntiles && vn > 0 && n > 0) {
    bits.resize((size_t)(vn / n) * words);
    RGS_CUDA(cudaMemcpyAsync(bits.data(), s->vis_bits, sizeof(uint32_t) * bits.size(),
                             cudaMemcpyDeviceToHost, stream),
             "copy visibility bits");
  }
  RGS_CUDA(cudaStreamSynchronize(stream), "sync");
  // The forward writes tile counts for its projection candidates only; an entry whose
  // visibility bit is clear touches no tile.
  if (!bits.empty())
    for (int64_t vi = 0; vi < vn; ++vi) {
      const int64_t v = vi / n, i = vi - v * n;
      if (!((bits[(size_t)(v * words + i / 32)] >> (i % 32)) & 1u)) host_ntiles[vi] = 0u;
    }
  return RGS_OK;
}

rgs_status rgs_radix_sort_u32(rgs_ctx* ctx, uint32_t* keys, uint32_t* vals, int64_t n,
                              int32_t begin_bit, int32_t end_bit, void* stream_ptr) {
  if (!ctx) return RGS_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (n < 0 || n >= (1ll << 31) || (n > 0 && !keys) || begin_bit < 0 || end_bit > 32 ||
      begin_bit >= end_bit)
    return fail(ctx, RGS_ERR_INVALID_ARG, "bad sort arguments");
  if (n == 0) return RGS_OK;
  cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
  cudaSetDevice(ctx->device);
  const int64_t hist = sort_hist_entries(n);
  const int64_t sums = std::max(scan_blocks(hist), scan_blocks(n)) + 1;
  char* base = nullptr;
  const size_t bytes = 2 * align_up(sizeof(uint32_t) * n) + align_up(sizeof(uint32_t) * hist) +
                       align_up(sizeof(uint32_t) * sums);
  RGS_CUDA(cudaMalloc(&base, bytes), "allocate sort scratch");
  char* p = base;
  uint32_t* kalt = carve<uint32_t>(p, n);
  uint32_t* valt = carve<uint32_t>(p, n);
  uint32_t* h = carve<uint32_t>(p, hist);
  uint32_t* bs = carve<uint32_t>(p, sums);
  bool alt = false;
  cudaError_t e = launch_radix_sort(keys, vals, kalt, vals ? valt : nullptr, n, nullptr,
                                    begin_bit, end_bit, h, bs, &alt, stream);
  if (e == cudaSuccess && alt) {
    e = cudaMemcpyAsync(keys, kalt, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, stream);
    if (e == cudaSuccess && vals)
      e = cudaMemcpyAsync(vals, valt, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, stream);
  }
  cudaError_t e2 = cudaStreamSynchronize(stream);
  cudaFree(base);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "radix sort");
  if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "radix sort sync");
  return RGS_OK;
}

rgs_status rgs_exclusive_scan_u32(rgs_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n,
                                  uint32_t* total_out, void* stream_ptr) {
  if (!ctx) return RGS_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (n < 0 || n >= (1ll << 31) || (n > 0 && (!in || !out)))
    return fail(ctx, RGS_ERR_INVALID_ARG, "bad scan arguments");
  cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
  cudaSetDevice(ctx->device);
  const int64_t sums = scan_blocks(n) + 1;
  uint32_t* bs = nullptr;
  RGS_CUDA(cudaMalloc(&bs, sizeof(uint32_t) * sums), "allocate scan scratch");
  cudaError_t e = launch_exclusive_scan(in, out, n, nullptr, total_out, bs, stream);
  cudaError_t e2 = cudaStreamSynchronize(stream);
  cudaFree(bs);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "scan");
  if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "scan sync");
  return RGS_OK;
}

int64_t rgs_single_pass_scan_bytes(int64_t n) {
  return n < 0 ? 0 : (int64_t)lookback_bytes(n);
}

rgs_status rgs_exclusive_scan_u32_single_pass(const uint32_t* in, uint32_t* out, int64_t n,
                                              uint32_t* total_out, void* work, int64_t work_bytes,
                                              uint32_t* status, void* stream_ptr) {
  if (n < 0 || n >= (1ll << 31) || (n > 0 && (!in || !out)) || !work || !status ||
      (reinterpret_cast<uintptr_t>(work) & 15u) != 0 ||
      work_bytes < rgs_single_pass_scan_bytes(n))
    return RGS_ERR_INVALID_ARG;
  if (n == 0) {
    if (total_out &&
        cudaMemsetAsync(total_out, 0, sizeof(uint32_t), static_cast<cudaStream_t>(stream_ptr)) !=
            cudaSuccess)
      return RGS_ERR_CUDA;
    return RGS_OK;
  }
  Lookback lb = lookback_at(work, status, n);
  const cudaError_t e = launch_exclusive_scan_single_pass(
      in, out, n, total_out, lb, static_cast<cudaStream_t>(stream_ptr));
  return e == cudaSuccess ? RGS_OK : RGS_ERR_CUDA;
}

}  // extern "C"

// ---- Tracking step ----

void rgs_track_config_default(rgs_track_config* cfg) {
  if (!cfg) return;
  cfg->tau_alpha = 0.5f;
  cfg->tau_grad = 0.05f;
  cfg->fit_exposure = 1;
}

void rgs_adam_config_default(rgs_adam_config* cfg) {
  if (!cfg) return;
  cfg->lr = 5e-3f;
  cfg->beta1 = 0.9f;
  cfg->beta2 = 0.999f;
  cfg->eps = 1e-8f;
  cfg->iterations = 0;
}

rgs_status rgs_track_grad_weight(rgs_ctx* ctx, const rgs_camera* cams, int32_t n_views,
                                 const float* observed, float tau_grad, float* w,
                                 void* stream_ptr) {
  if (!ctx) return RGS_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (!observed || !w) return fail(ctx, RGS_ERR_INVALID_ARG, "null image pointer");
  if (!(tau_grad > 0.0f) || !std::isfinite(tau_grad))
    return fail(ctx, RGS_ERR_INVALID_ARG, "tau_grad must be positive");
  rgs_config cfg;
  rgs_config_default(&cfg);
  Views views;
  Consts consts;
  rgs_status st = build_views(ctx, cams, n_views, cfg, views, consts);
  if (st != RGS_OK) return st;
  if (cudaSetDevice(ctx->device) != cudaSuccess)
    return fail(ctx, RGS_ERR_CUDA, "cudaSetDevice failed");
  RGS_CUDA(launch_grad_weight(views, observed, tau_grad, w, static_cast<cudaStream_t>(stream_ptr)),
           "gradient weights");
  return RGS_OK;
}

rgs_status rgs_track_loss(rgs_ctx* ctx, const rgs_camera* cams, int32_t n_views,
                          const rgs_track_config* tcfg_in, const float* color,
                          const float* alpha, const float* observed, const float* w_grad,
                          float* d_color, double* loss, float* gain_bias, void* stream_ptr) {
  if (!ctx) return RGS_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (!color || !alpha || !observed || !d_color || !loss || !gain_bias)
    return fail(ctx, RGS_ERR_INVALID_ARG, "null pointer");
  rgs_track_config tcfg;
  if (tcfg_in) tcfg = *tcfg_in; else rgs_track_config_default(&tcfg);
  if (!(tcfg.tau_alpha > 0.0f) || !std::isfinite(tcfg.tau_alpha))
    return fail(ctx, RGS_ERR_INVALID_ARG, "tau_alpha must be positive");
  rgs_config cfg;
  rgs_config_default(&cfg);
  Views views;
  Consts consts;
  rgs_status st = build_views(ctx, cams, n_views, cfg, views, consts);
  if (st != RGS_OK) return st;
  if (cudaSetDevice(ctx->device) != cudaSuccess)
    return fail(ctx, RGS_ERR_CUDA, "cudaSetDevice failed");
  RGS_CUDA(launch_track_loss(views, color, alpha, observed, w_grad, tcfg.tau_alpha,
                             tcfg.fit_exposure != 0, ctx->track_sums, d_color, loss, gain_bias,
                             static_cast<cudaStream_t>(stream_ptr)),
           "tracking loss");
  return RGS_OK;
}

rgs_status rgs_pose_adam_step(rgs_ctx* ctx, int32_t n_views, const rgs_adam_config* acfg_in,
                              const float* d_pose, float* adam_state, int32_t* step,
                              float* world_to_cam, void* stream_ptr) {
  if (!ctx) return RGS_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (n_views < 1 || n_views > kMaxViews)
    return fail(ctx, RGS_ERR_INVALID_ARG, "n_views must be in 1..RGS_MAX_VIEWS");
  if (!d_pose || !adam_state || !step || !world_to_cam)
    return fail(ctx, RGS_ERR_INVALID_ARG, "null pointer");
  rgs_adam_config a;
  if (acfg_in) a = *acfg_in; else rgs_adam_config_default(&a);
  if (!(a.lr >= 0.0f) || !std::isfinite(a.lr) || !(a.beta1 >= 0.0f && a.beta1 < 1.0f) ||
      !(a.beta2 >= 0.0f && a.beta2 < 1.0f) || !(a.eps > 0.0f) || a.iterations < 0)
    return fail(ctx, RGS_ERR_INVALID_ARG, "Adam constants out of range");
  if (cudaSetDevice(ctx->device) != cudaSuccess)
    return fail(ctx, RGS_ERR_CUDA, "cudaSetDevice failed");
  RGS_CUDA(launch_pose_adam(n_views, a.lr, a.beta1, a.beta2, a.eps, a.iterations, d_pose,
                            adam_state, step, world_to_cam, static_cast<cudaStream_t>(stream_ptr)),
           "pose update");
  return RGS_OK;
}

// ---- Dense initialisation ----

void rgs_seed_config_default(rgs_seed_config* cfg) {
  if (!cfg) return;
  cfg->min_parallax = (float)(M_PI / 180.0);
  cfg->max_reproj = 2.0f;
  cfg->tie_eps = 1e-3f;
  cfg->plane_radius = 0.05f;
  cfg->s_par_cap = 10.0f;
  cfg->alpha_lo = 0.1f;
  cfg->alpha_hi = 0.9f;
  cfg->voxel = 0.0f;
}

namespace {

rgs_status seed_setup(rgs_ctx* ctx, const rgs_camera* cams, int32_t n_views,
                      const rgs_seed_config* cfg_in, SeedCams& sc, SeedConsts& c) {
  if (!cams) return fail(ctx, RGS_ERR_INVALID_ARG, "cams is null");
  if (n_views < 1 || n_views > kMaxViews)
    return fail(ctx, RGS_ERR_INVALID_ARG, "n_views must be in 1..RGS_MAX_VIEWS");
  rgs_seed_config cfg;
  if (cfg_in) cfg = *cfg_in; else rgs_seed_config_default(&cfg);
  if (!(cfg.min_parallax >= 0.0f) || !(cfg.max_reproj > 0.0f) || !(cfg.tie_eps >= 0.0f) ||
      !(cfg.plane_radius > 0.0f) || !(cfg.s_par_cap >= 1.0f) || !(cfg.alpha_lo > 0.0f) ||
      !(cfg.alpha_hi < 1.0f) || !(cfg.alpha_lo <= cfg.alpha_hi) || !(cfg.voxel >= 0.0f) ||
      !std::isfinite(cfg.plane_radius) || !std::isfinite(cfg.voxel))
    return fail(ctx, RGS_ERR_INVALID_ARG, "seed config values out of range");
  std::memset(&sc, 0, sizeof(sc));
  sc.n_views = n_views;
  long long pix = 0;
  for (int v = 0; v < n_views; ++v) {
    const rgs_camera& cm = cams[v];
    if (cm.width < 1 || cm.height < 1 || cm.width > 16384 || cm.height > 16384 ||
        !(cm.fx > 0.0f) || !(cm.fy > 0.0f))
      return fail(ctx, RGS_ERR_INVALID_ARG, "camera size or intrinsics invalid");
    sc.pixel_offset[v] = pix;
    sc.width[v] = cm.width;
    sc.height[v] = cm.height;
    sc.fx[v] = cm.fx;
    sc.fy[v] = cm.fy;
    sc.cx[v] = cm.cx;
    sc.cy[v] = cm.cy;
    for (int a = 0; a < 3; ++a) {
      for (int b = 0; b < 3; ++b) sc.R[v][3 * a + b] = cm.world_to_cam[4 * a + b];
      sc.t[v][a] = cm.world_to_cam[4 * a + 3];
    }
    for (int j = 0; j < 4; ++j) {
      const double r0 = j < 3 ? sc.R[v][j] : sc.t[v][0];
      const double r1 = j < 3 ? sc.R[v][3 + j] : sc.t[v][1];
      const double r2 = j < 3 ? sc.R[v][6 + j] : sc.t[v][2];
      sc.P[v][j] = sc.fx[v] * r0 + sc.cx[v] * r2;
      sc.P[v][4 + j] = sc.fy[v] * r1 + sc.cy[v] * r2;
      sc.P[v][8 + j] = r2;
    }
    for (int a = 0; a < 3; ++a) {
      double s = 0.0;
      for (int b = 0; b < 3; ++b) s -= sc.R[v][3 * b + a] * sc.t[v][b];
      sc.c[v][a] = s;
    }
    pix += (long long)cm.width * cm.height;
  }
  c.min_parallax = cfg.min_parallax;
  c.max_reproj = cfg.max_reproj;
  c.tie_eps = cfg.tie_eps;
  c.plane_radius = cfg.plane_radius;
  c.s_par_cap = cfg.s_par_cap;
  c.alpha_lo = cfg.alpha_lo;
  c.alpha_hi = cfg.alpha_hi;
  c.voxel = cfg.voxel;
  return RGS_OK;
}

}  // namespace

rgs_status rgs_triangulate(rgs_ctx* ctx, const rgs_camera* cams, int32_t n_views, int64_t m,
                           int32_t k, const int32_t* ref_view, const double* ref_xy,
                           const int32_t* nb_view, const double* nb_xy, const float* nb_conf,
                           const rgs_seed_config* cfg, uint32_t* valid, double* X, int32_t* best,
                           double* err, double* angle, float* kappa, void* stream_ptr) {
  if (!ctx) return RGS_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (m < 0 || m >= (1ll << 31) || k < 1 || k > 8)
    return fail(ctx, RGS_ERR_INVALID_ARG, "m must be in 0..2^31-1 and k in 1..8");
  if (m > 0 && (!ref_view || !ref_xy || !nb_view || !nb_xy || !nb_conf || !valid || !X || !best ||
                !err || !angle || !kappa))
    return fail(ctx, RGS_ERR_INVALID_ARG, "null array");
  SeedCams sc;
  SeedConsts c;
  rgs_status st = seed_setup(ctx, cams, n_views, cfg, sc, c);
  if (st != RGS_OK) return st;
  if (cudaSetDevice(ctx->device) != cudaSuccess)
    return fail(ctx, RGS_ERR_CUDA, "cudaSetDevice failed");
  RGS_CUDA(launch_triangulate(sc, c, m, k, ref_view, ref_xy, nb_view, nb_xy, nb_conf, valid, X,
                              best, err, angle, kappa, static_cast<cudaStream_t>(stream_ptr)),
           "triangulate");
  return RGS_OK;
}

rgs_status rgs_init_seeds(rgs_ctx* ctx, const rgs_camera* cams, int32_t n_views, int64_t m,
                          int32_t k, const int32_t* ref_view, const int32_t* nb_view,
                          const uint32_t* valid, const double* X, const double* err,
                          const double* angle, const float* kappa, const float* observed,
                          const float* gain_bias, int32_t sh_degree, const rgs_seed_config* cfg,
                          int32_t* index, float* means, float* log_scales, float* quats,
                          float* opacity_logits, float* sh, float* normals, int64_t* n_seeds,
                          void* stream_ptr) {
  if (!ctx) return RGS_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (!n_seeds) return fail(ctx, RGS_ERR_INVALID_ARG, "n_seeds is null");
  *n_seeds = 0;
  if (m < 0 || m >= (1ll << 31) || k < 1 || k > 8 || sh_degree < 0 || sh_degree > 3)
    return fail(ctx, RGS_ERR_INVALID_ARG, "m, k or sh_degree out of range");
  if (m > 0 && (!ref_view || !nb_view || !valid || !X || !err || !angle || !kappa || !observed ||
                !gain_bias || !index || !means || !log_scales || !quats || !opacity_logits ||
                !sh || !normals))
    return fail(ctx, RGS_ERR_INVALID_ARG, "null array");
  SeedCams sc;
  SeedConsts c;
  rgs_status st = seed_setup(ctx, cams, n_views, cfg, sc, c);
  if (st != RGS_OK) return st;
  if (m == 0) return RGS_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess)
    return fail(ctx, RGS_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
  const int sh_k = (sh_degree + 1) * (sh_degree + 1);
  const int64_t hist = sort_hist_entries(m);
  const int64_t sums = std::max(scan_blocks(hist), scan_blocks(m)) + 1;
  const size_t bytes = 12 * align_up(sizeof(uint32_t) * m) + align_up(sizeof(uint32_t) * hist) +
                       align_up(sizeof(uint32_t) * sums) + align_up(sizeof(uint64_t) * m) +
                       align_up(sizeof(double) * 3 * m) +
                       align_up(sizeof(float) * (size_t)m * (3 + 3 + 4 + 1 + 3 + 3 * sh_k));
  // The scratch region is kept in the context and only grows: repeated calls (one per new
  // keyframe) neither allocate nor free.
  if (ctx->r_seed.bytes < bytes)
    RGS_CUDA(alloc_region(ctx->r_seed, bytes), "allocate seeding scratch");
  char* p = static_cast<char*>(ctx->r_seed.base);
  uint32_t* flags = carve<uint32_t>(p, m);
  uint32_t* pos = carve<uint32_t>(p, m);
  uint32_t* vidx = carve<uint32_t>(p, m);
  uint32_t* lo = carve<uint32_t>(p, m);
  uint32_t* hi = carve<uint32_t>(p, m);
  uint32_t* slot = carve<uint32_t>(p, m);
  uint32_t* t0 = carve<uint32_t>(p, m);
  uint32_t* t1 = carve<uint32_t>(p, m);
  uint32_t* keep = carve<uint32_t>(p, m);
  uint32_t* kpos = carve<uint32_t>(p, m);
  uint32_t* totals = carve<uint32_t>(p, m);  // [0]: accepted points, [1]: kept seeds
  carve<uint32_t>(p, m);                     // spare
  uint32_t* h = carve<uint32_t>(p, hist);
  uint32_t* bs = carve<uint32_t>(p, sums);
  unsigned long long* skey = carve<unsigned long long>(p, m);
  double* sX = carve<double>(p, 3 * m);
  float* f_means = carve<float>(p, 3 * m);
  float* f_ls = carve<float>(p, 3 * m);
  float* f_q = carve<float>(p, 4 * m);
  float* f_o = carve<float>(p, m);
  float* f_n = carve<float>(p, 3 * m);
  float* f_sh = carve<float>(p, 3 * sh_k * m);
  rgs_status result = RGS_OK;
  uint32_t host_tot[2] = {0, 0};
  do {
    cudaError_t e = launch_seed_flags(m, n_views, valid, ref_view, flags, stream);
    if (e == cudaSuccess) e = launch_exclusive_scan(flags, pos, m, nullptr, totals, bs, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_tot, totals, sizeof(uint32_t),
                                              cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) { result = cuda_fail(ctx, e, "seed compaction"); break; }
    const int s = (int)host_tot[0];
    e = launch_compact_points(m, flags, pos, vidx, stream);
    if (e == cudaSuccess)
      e = launch_seed_points(sc, c, s, k, sh_k, vidx, ref_view, nb_view, X, err, angle, kappa,
                             observed, gain_bias, lo, hi, slot, t0, t1, h, bs, skey, sX, f_means,
                             f_ls, f_q, f_o, f_sh, f_n, keep, stream);
    if (e == cudaSuccess && s > 0)
      e = launch_exclusive_scan(keep, kpos, s, nullptr, totals + 1, bs, stream);
    if (e == cudaSuccess && s > 0)
      e = cudaMemcpyAsync(host_tot + 1, totals + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                          stream);
    if (e == cudaSuccess)
      e = launch_scatter_seeds(s, sh_k, keep, kpos, vidx, f_means, f_ls, f_q, f_o, f_sh, f_n,
                               index, means, log_scales, quats, opacity_logits, sh, normals,
                               stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) { result = cuda_fail(ctx, e, "seed initialisation"); break; }
    *n_seeds = s > 0 ? (int64_t)host_tot[1] : 0;
  } while (false);
  cudaStreamSynchronize(stream);
  return result;
}

rgs_status rgs_covisibility(rgs_ctx* ctx, const float* alpha_a, const float* alpha_b, int64_t n,
                            int32_t n_pairs, float tau, uint64_t* counts, float* iou,
                            void* stream_ptr) {
  if (!ctx) return RGS_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (n < 0 || n_pairs < 0 || n_pairs > 65535 || !std::isfinite(tau))
    return fail(ctx, RGS_ERR_INVALID_ARG, "n, n_pairs (0..65535) or tau out of range");
  if (n_pairs > 0 && (!counts || !iou || (n > 0 && (!alpha_a || !alpha_b))))
    return fail(ctx, RGS_ERR_INVALID_ARG, "null array");
  if (n_pairs == 0) return RGS_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess)
    return fail(ctx, RGS_ERR_CUDA, "cudaSetDevice failed");
  RGS_CUDA(launch_covisibility(alpha_a, alpha_b, n, n_pairs, tau,
                               reinterpret_cast<unsigned long long*>(counts), iou,
                               static_cast<cudaStream_t>(stream_ptr)),
           "co-visibility");
  return RGS_OK;
}

// ---- Mapping maintenance ----

rgs_status rgs_map_ema(rgs_ctx* ctx, int64_t n, const float* means, float* ema_means, float eta,
                       void* stream_ptr) {
  if (!ctx) return RGS_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (n < 0 || !(eta > 0.0f && eta < 1.0f))
    return fail(ctx, RGS_ERR_INVALID_ARG, "n must be >= 0 and eta in (0, 1)");
  if (n > 0 && (!means || !ema_means)) return fail(ctx, RGS_ERR_INVALID_ARG, "null array");
  if (n == 0) return RGS_OK;
  if (cudaSetDevice(ctx->device) != cudaSuccess)
    return fail(ctx, RGS_ERR_CUDA, "cudaSetDevice failed");
  RGS_CUDA(launch_map_ema(n, means, ema_means, eta, static_cast<cudaStream_t>(stream_ptr)),
           "anchor update");
  return RGS_OK;
}

void rgs_prune_config_default(rgs_prune_config* cfg) {
  if (!cfg) return;
  cfg->min_opacity = 0.005f;
  cfg->max_trace = 1.0f;
  cfg->min_observations = 5;
  cfg->min_visibility = 1.0f;
}

rgs_status rgs_prune_mask(rgs_ctx* ctx, int64_t n, const float* log_scales,
                          const float* opacity_logits, const uint32_t* obs_count,
                          const float* vis_score, const rgs_prune_config* cfg_in, uint8_t* keep,
                          uint32_t* n_keep, void* stream_ptr) {
  if (!ctx) return RGS_ERR_INVALID_ARG;
  ctx->last_error.clear();
  if (n < 0 || n >= (1ll << 31)) return fail(ctx, RGS_ERR_INVALID_ARG, "n out of range");
  if (!n_keep || (n > 0 && (!log_scales || !opacity_logits || !obs_count || !vis_score || !keep)))
    return fail(ctx, RGS_ERR_INVALID_ARG, "null array");
  rgs_prune_config cfg;
  if (cfg_in) cfg = *cfg_in; else rgs_prune_config_default(&cfg);
  if (!std::isfinite(cfg.min_opacity) || !std::isfinite(cfg.min_visibility) ||
      std::isnan(cfg.max_trace))
    return fail(ctx, RGS_ERR_INVALID_ARG, "prune bounds out of range");
  if (cudaSetDevice(ctx->device) != cudaSuccess)
    return fail(ctx, RGS_ERR_CUDA, "cudaSetDevice failed");
  RGS_CUDA(launch_prune_mask(n, log_scales, opacity_logits, obs_count, vis_score,
                             cfg.min_opacity, cfg.max_trace, cfg.min_observations,
                             cfg.min_visibility, keep, n_keep,
                             static_cast<cudaStream_t>(stream_ptr)),
           "prune mask");
  return RGS_OK;
}
