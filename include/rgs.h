/*
 * rgs.h -- C ABI of the GB300 (sm_103a) differentiable 3D Gaussian-splatting rasterizer.
 *
 * The library renders a set of anisotropic 3D Gaussians into one or more pinhole views and
 * back-propagates image gradients to every Gaussian parameter and to each view's SE(3) pose.
 *
 *   Forward  (Section 3.1, Eq. proj and Eq. alpha; Appendix C.1, Eq. app-sh):
 *     mu^C = R mu^W + t, mu^I = pi(mu^C), Sigma^I = J R Sigma^W R^T J^T + eps2d I,
 *     Sigma^W = R_q diag(exp(2 log_scale)) R_q^T, colour from real spherical harmonics of the
 *     viewing direction, opacity o = sigmoid(logit); per pixel the covering Gaussians are
 *     composited front to back, C = sum_i c_i alpha_i prod_{j<i} (1 - alpha_j).
 *   Backward (Section 3.1, differentiability in colour, opacity, mean, covariance and pose;
 *     Section 3.2.3, Eq. leftupdate, Eq. muCjac, Eq. muIjac, Eq. sigmaIjac): gradients of the
 *     rendered colour, depth and accumulated opacity with respect to means, log-scales,
 *     quaternions, opacity logits, SH coefficients, and the twist xi = (rho, omega) of the left
 *     update T_WC <- exp(xi^) T_WC, evaluated at xi = 0.
 *
 * Conventions
 *   - Every array is a DEVICE pointer on the context's device unless stated otherwise, FP32,
 *     C-contiguous, and owned by the caller. Nothing is copied: a device array passed to
 *     rgs_render_forward must stay alive and unchanged until the matching rgs_render_backward
 *     (and rgs_release_state) has completed on the stream.
 *   - Images of all views are concatenated: view v occupies pixels [offset_v, offset_v + W_v H_v)
 *     with offset_v = sum_{u<v} W_u H_u, row-major inside a view; colour is [P,3] interleaved.
 *   - Pixel (x, y) is sampled at image coordinates (x, y). A Gaussian covers a pixel iff
 *     alpha = min(alpha_max, o G) >= alpha_min; compositing stops before the Gaussian whose
 *     inclusion would drop the transmittance below t_min; near-to-far order is by camera-space
 *     depth of the Gaussian centre (rounded to float32), ties by Gaussian index.
 *   - Outputs: colour = sum w_i c_i + T_final bg, depth = sum w_i z_i, alpha = 1 - T_final.
 *   - All calls are asynchronous on `stream` (a cudaStream_t passed as void*, NULL = legacy
 *     default stream). Gradient buffers are overwritten, not accumulated.
 *   - Errors are returned as rgs_status; rgs_last_error() gives a message. No call throws or aborts.
 *   - A context is not thread-safe: serialise calls on one context.
 */
#ifndef RGS_H_
#define RGS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RGS_MAX_VIEWS 64

typedef enum {
  RGS_OK = 0,
  RGS_ERR_INVALID_ARG = 1, /* a null, misaligned or out-of-range argument */
  RGS_ERR_CUDA = 2,        /* a CUDA runtime call failed (message in rgs_last_error) */
  RGS_ERR_CAPACITY = 3,    /* the (view, tile) pair list outgrew its capacity during stream
                              capture; results are incomplete. Re-run outside capture (which
                              grows it) or call rgs_reserve first */
  RGS_ERR_NOMEM = 4,       /* device allocation failed */
  RGS_ERR_STATE = 5,       /* unknown or released state handle */
  RGS_ERR_TOO_LARGE = 6,   /* more elements than a fixed-scratch entry point supports */
} rgs_status;

/* Opaque context: owns per-forward saved state (projected records, sorted pair lists, tile
 * ranges, per-pixel final transmittance and last-contributor index) and sort scratch. */
typedef struct rgs_ctx rgs_ctx;

/* The Gaussian set (Section 3.1; Appendix C.1). Device pointers, FP32, caller-owned.
 *   means [n,3] world frame; log_scales [n,3]; quats [n,4] as (w, x, y, z), normalised inside
 *   (need not be unit); opacity_logits [n]; sh [n,K,3], K = (sh_degree+1)^2, basis order
 *   l = 0..sh_degree, m = -l..l. Each pointer must be 16-byte aligned. */
typedef struct {
  int32_t n;
  int32_t sh_degree; /* 0..3 */
  const float* means;
  const float* log_scales;
  const float* quats;
  const float* opacity_logits;
  const float* sh;
} rgs_gaussians;

/* One pinhole view (HOST struct). world_to_cam is the row-major 3x4 [R | t] of T_WC,
 * mu^C = R mu^W + t; R must be a rotation. Camera axes: x right, y down, z forward. */
typedef struct {
  int32_t width, height;
  float fx, fy, cx, cy;
  float world_to_cam[12];
} rgs_camera;

/* Renderer constants (HOST struct); rgs_config_default fills the defaults shown. */
typedef struct {
  float alpha_min;  /* 1/255: a Gaussian covers a pixel iff min(alpha_max, o G) >= alpha_min */
  float alpha_max;  /* 0.99 */
  float t_min;      /* 1e-4: transmittance stop */
  float znear;      /* 0.2: Gaussians with camera depth <= znear are culled */
  float eps2d;      /* 0.3 px^2: dilation added to Sigma^I before inversion */
  float jac_clamp;  /* 1.3: J uses x/z, y/z clamped to +-jac_clamp*(W/2)/fx, (H/2)/fy; 0 = off */
  float bg[3];      /* background colour, added as bg * T_final */
  int32_t tile_w;   /* tile shape of the binning and blend: 16x16 (default), 8x8 or 32x8 */
  int32_t tile_h;
  int32_t pixels_per_thread; /* vertically adjacent pixels per forward-blend thread: 1, 2, 4 or
                                8 (4 and 8 not with 8x8 tiles); 0 = default (4). Results do not
                                depend on it or on the tile shape beyond atomics-order rounding of
                                the gradients */
  int32_t backward_pixels_per_thread; /* the same for the backward blend (same rules); 0 = equal to
                                         pixels_per_thread. The two blends share only the tile
                                         shape: the per-pixel state between them is stored in
                                         image order */
  void* sh_ready_event; /* optional cudaEvent_t, or NULL. NULL: the projection evaluates the
                           colours (Eq. app-sh) and culls entries with a non-finite coefficient.
                           An event: the forward reads the SH coefficients only after the tile
                           lists are built (the colours of the visible entries are evaluated just
                           before the forward blend) and waits for the event on its stream right
                           there, so that the caller's upload of the coefficients can overlap the
                           projection and the sorts; an entry with a non-finite coefficient then
                           stays in the lists but covers no pixel. Images and gradients are the
                           same either way. The event must have been recorded (on any stream)
                           before the call; under stream capture the wait becomes a graph
                           dependency. */
} rgs_config;

/* Forward outputs (device, caller-owned, P = sum_v W_v H_v): color [P,3], depth [P], alpha [P]. */
typedef struct {
  float* color;
  float* depth;
  float* alpha;
} rgs_images;

/* Upstream gradients of a scalar loss with respect to the forward outputs (device, [P,3], [P],
 * [P]); a NULL member means zero. */
typedef struct {
  const float* d_color;
  const float* d_depth;
  const float* d_alpha;
} rgs_image_grads;

/* Bits of grad_mask for rgs_render_backward. */
#define RGS_GRAD_MEANS 1u
#define RGS_GRAD_SCALES 2u
#define RGS_GRAD_QUATS 4u
#define RGS_GRAD_OPACITY 8u
#define RGS_GRAD_SH 16u
#define RGS_GRAD_POSE 32u
#define RGS_GRAD_ALL 63u

/* Counters of the last forward on a state (read back with a stream synchronisation). */
typedef struct {
  int64_t n_visible;       /* (view, Gaussian) pairs that touch at least one tile */
  int64_t n_pairs;         /* duplicated (view, tile, Gaussian) entries (of the visible entries
                              kept, when status bit 2 is set) */
  int64_t n_eval;          /* (pixel, Gaussian) list positions visited by the forward blend */
  int64_t n_contrib;       /* reserved: 0 (the forward blend counts visited positions only) */
  int64_t n_nonfinite;     /* (view, Gaussian) culled for non-finite inputs (with an SH event,
                              non-finite SH coefficients are found, and counted, for the entries
                              that reach the tile lists) */
  int64_t pair_capacity;   /* allocated pair-list capacity */
  int64_t state_bytes;     /* device bytes held by the state */
  uint32_t status;         /* device status bits: 1 = pair list overflowed its capacity;
                              2 = more visible entries than the sorted-list capacity (both only
                              under stream capture; the output is then incomplete); 4 = a
                              single-pass scan gave up a bounded wait for another block (the
                              output is then wrong; not expected) */
  uint32_t kernel_launches; /* kernels launched by the last forward plus the last backward */
} rgs_stats;

/* Creates a context on CUDA device `device`. Returns RGS_ERR_INVALID_ARG for a null out pointer
 * or bad device, RGS_ERR_CUDA if the device cannot be used. */
rgs_status rgs_create(rgs_ctx** ctx, int device);

/* Frees every state and scratch buffer (synchronises the device). NULL is a no-op. */
void rgs_destroy(rgs_ctx* ctx);

/* Fills the defaults listed in rgs_config. */
void rgs_config_default(rgs_config* cfg);

/* Message of the last failed call on this context ("" if none). Valid until the next call. */
const char* rgs_last_error(const rgs_ctx* ctx);

/* Renders n_views (1..RGS_MAX_VIEWS) views of the Gaussian set in one batched launch sequence
 * (Section 3.1, Eq. proj and Eq. alpha; the keyframe window of the mapping loss, Eq. map-loss).
 *   g: Gaussian set (n may be 0: empty images, alpha 0, colour = bg).
 *   cams: HOST array of n_views cameras; each W, H in 1..16384.
 *   cfg: HOST config, or NULL for the defaults.
 *   out: device output images.
 *   state: in/out. If *state is 0 a new state is created and its handle written back; otherwise
 *     the named state is reused (its previous contents are replaced). The state keeps the data
 *     the backward needs.
 * Outside stream capture the call synchronises the stream twice (after the visibility
 * compaction and after the pair count) to size the sorted list of visible entries and the pair
 * list. Under stream capture it never synchronises and keeps the sizes of the last call outside
 * capture; if a list would overflow, the kernels record it, the output is incomplete and
 * rgs_query_stats reports status bit 1 (pairs) or 2 (visible entries). */
rgs_status rgs_render_forward(rgs_ctx* ctx, const rgs_gaussians* g, const rgs_camera* cams,
                              int32_t n_views, const rgs_config* cfg, rgs_images* out,
                              uint64_t* state, void* stream);

/* Back-propagates upstream image gradients through the forward saved in `state`
 * (Section 3.1; Section 3.2.3 Eq. muCjac, Eq. muIjac, Eq. sigmaIjac). The Gaussian arrays and
 * cameras of that forward are used; they must be unchanged.
 *   grads: HOST struct of device pointers (members may be NULL = zero).
 *   grad_mask: RGS_GRAD_* bits; outputs whose bit is clear may be NULL and are not written.
 *   d_means [n,3], d_log_scales [n,3], d_quats [n,4], d_opacity_logits [n], d_sh [n,K,3]:
 *     summed over all views of the forward; overwritten.
 *   d_pose [n_views,6]: (rho, omega) per view, the gradient with respect to the twist of the
 *     left update at xi = 0; overwritten. */
rgs_status rgs_render_backward(rgs_ctx* ctx, uint64_t state, const rgs_image_grads* grads,
                               uint32_t grad_mask, float* d_means, float* d_log_scales,
                               float* d_quats, float* d_opacity_logits, float* d_sh,
                               float* d_pose, void* stream);

/* Autotuner: picks the blend tile shape and the pixels per thread of each blend (the per-thread
 * batch depth) that make one forward + backward of this exact workload fastest on this GPU. For
 * every tile shape (16x16, 8x8, 32x8) and every pixels-per-thread value it admits (1, 2, 4, 8)
 * the forward and the backward are timed separately with CUDA events (one warm-up and the
 * fastest of four timed runs, a uniform non-zero upstream colour gradient, all gradients
 * requested) in scratch buffers of its own; per tile shape the fastest forward and the fastest
 * backward setting are combined, and the
 * tile shape with the smallest sum wins. The choice is written into cfg->tile_w, cfg->tile_h,
 * cfg->pixels_per_thread and cfg->backward_pixels_per_thread (other fields are kept) and cached
 * in the context under (n, sh_degree, the views' sizes); a later call with the same key returns
 * the cached choice without timing. Results do not depend on the choice beyond atomics-order
 * rounding of the gradients. Synchronises `stream`; allocates and frees device memory. Under
 * stream capture it returns RGS_ERR_INVALID_ARG. ms_out (may be NULL) receives the winner's
 * forward + backward time in milliseconds (0 when served from the cache). */
rgs_status rgs_autotune(rgs_ctx* ctx, const rgs_gaussians* g, const rgs_camera* cams,
                        int32_t n_views, rgs_config* cfg, float* ms_out, void* stream);

/* Frees a state's device memory (after its queued work completes). */
rgs_status rgs_release_state(rgs_ctx* ctx, uint64_t state);

/* Grows a state's pair-list capacity to at least `pair_capacity` entries (0 = leave), so that a
 * later forward under stream capture does not overflow. Creates the state if *state is 0. */
rgs_status rgs_reserve(rgs_ctx* ctx, uint64_t* state, int64_t pair_capacity, void* stream);

/* Reads the counters of the last forward on `state` (synchronises `stream`). */
rgs_status rgs_query_stats(rgs_ctx* ctx, uint64_t state, rgs_stats* out, void* stream);

/* ---- Tracking step (Section 3.2 and its appendix: Eq. app-bright, app-ls, app-trackloss,
 * app-weight; Eq. leftupdate). One tracking iteration on the device, with no host round trip:
 *   rgs_render_forward_posed -> rgs_track_loss -> rgs_render_backward (RGS_GRAD_POSE)
 *   -> rgs_pose_adam_step, which updates the device poses the next forward reads.
 * With the observation's gradient weights from rgs_track_grad_weight (once per frame), the
 * iteration can be captured in a CUDA graph and replayed. ---- */

/* rgs_render_forward with the world-to-camera poses taken from DEVICE memory:
 *   world_to_cam: device [n_views][12] floats, row-major [R|t] as in rgs_camera (4-byte
 *     aligned); read by this call's first kernel, so it may be updated (e.g. by
 *     rgs_pose_adam_step) as soon as the call's work is queued; the backward uses the poses of
 *     this forward. The poses in cams are ignored (sizes and intrinsics are used). NULL is
 *     RGS_ERR_INVALID_ARG.
 * Given the same pose values, the result is bit-identical to rgs_render_forward's. */
rgs_status rgs_render_forward_posed(rgs_ctx* ctx, const rgs_gaussians* g, const rgs_camera* cams,
                                    int32_t n_views, const float* world_to_cam,
                                    const rgs_config* cfg, rgs_images* out, uint64_t* state,
                                    void* stream);

/* Loss constants (HOST struct); rgs_track_config_default fills the defaults shown. The paper
 * fixes neither threshold. */
typedef struct {
  float tau_alpha;      /* 0.5: w_alpha = clip(alpha / tau_alpha, 0, 1) */
  float tau_grad;       /* 0.05: w_grad = clip(||grad I||_2 / tau_grad, 0, 1) (intensities in [0, 1]) */
  int32_t fit_exposure; /* 1: fit (g, b) per view by least squares (Eq. app-ls); 0: g = 1, b = 0 */
} rgs_track_config;
void rgs_track_config_default(rgs_track_config* cfg);

/* Gradient weights of observed frames (Eq. app-weight): w[p] = clip(||grad I(p)||_2 / tau_grad,
 * 0, 1), with grad I from central differences per channel (one-sided on the image border, zero
 * along an axis of extent 1) and the norm over both axes and the three channels.
 *   observed: device [P,3] (views concatenated as in rgs_images); w: device [P] output.
 *   cams: HOST array (sizes are used). tau_grad > 0. */
rgs_status rgs_track_grad_weight(rgs_ctx* ctx, const rgs_camera* cams, int32_t n_views,
                                 const float* observed, float tau_grad, float* w, void* stream);

/* Exposure-compensated, weighted L1 tracking loss of each view and its gradient with respect to
 * the rendered colour (Eq. app-bright, app-ls, app-trackloss, app-weight):
 *   (g_v, b_v) = argmin_{g,b} sum_{p in v} ||I(p) - g C(p) - b||_2^2   (closed form, FP64;
 *                a constant render gives g = 1 and b matching the means)
 *   loss[v]    = sum_{p in v} w(p) ||I(p) - (g_v C(p) + b_v)||_1,
 *   w(p)       = clip(alpha(p) / tau_alpha, 0, 1) * w_grad(p)   (w_grad NULL: 1)
 *   d_color(p) = -w(p) g_v sign(I(p) - g_v C(p) - b_v)   per channel (sign(0) = 0).
 * (g, b) and w are held fixed in the gradient: they are re-estimated from every render.
 *   cams: HOST array (sizes are used); cfg: HOST or NULL (defaults).
 *   color [P,3], alpha [P]: a forward's outputs; observed [P,3]; w_grad [P] or NULL (device).
 *   d_color [P,3]: device output, the upstream colour gradient for rgs_render_backward.
 *   loss: device double [n_views]; gain_bias: device float [n_views][2] = (g, b).
 * Uses a fixed scratch of the context: calls on one context whose executions overlap on the
 * GPU race on it. Never synchronises; may be captured. */
rgs_status rgs_track_loss(rgs_ctx* ctx, const rgs_camera* cams, int32_t n_views,
                          const rgs_track_config* cfg, const float* color, const float* alpha,
                          const float* observed, const float* w_grad, float* d_color,
                          double* loss, float* gain_bias, void* stream);

/* Adam constants (HOST struct); rgs_adam_config_default fills the defaults shown. */
typedef struct {
  float lr;           /* 5e-3: base learning rate */
  float beta1, beta2; /* 0.9, 0.999 */
  float eps;          /* 1e-8 */
  int32_t iterations; /* K > 0: cosine schedule lr_k = lr (1 + cos(pi min(k, K) / K)) / 2 for
                         step k = 0, 1, ...; 0: constant lr. Default 0 */
} rgs_adam_config;
void rgs_adam_config_default(rgs_adam_config* cfg);

/* One Adam step on the twist of every view and the left update T <- exp(xi^) T (Eq. leftupdate),
 * with xi = -lr_k mhat / (sqrt(vhat) + eps) from d_pose = dL/dxi at xi = 0 (rgs_render_backward's
 * (rho, omega)), and the closed-form SE(3) exponential (R <- R_d R, t <- R_d t + V rho). FP64
 * arithmetic; all arrays are DEVICE memory:
 *   d_pose [n_views][6]; adam_state [n_views][12] = (m[6], v[6]), zero before the first step;
 *   step: one int32, the number of steps taken (0 before the first), incremented;
 *   world_to_cam [n_views][12], row-major [R|t], updated in place.
 * Never synchronises; may be captured. */
rgs_status rgs_pose_adam_step(rgs_ctx* ctx, int32_t n_views, const rgs_adam_config* cfg,
                              const float* d_pose, float* adam_state, int32_t* step,
                              float* world_to_cam, void* stream);

/* Phases timed by rgs_phase_times, in this order. */
#define RGS_PHASE_PREPROCESS 0     /* projection, SH colour, tile counts (Eq. proj, Eq. app-sh) */
#define RGS_PHASE_COMPACT 1        /* visible (view, Gaussian) entries with depth keys */
#define RGS_PHASE_DEPTH_SORT 2     /* radix sort of the visible entries by depth */
#define RGS_PHASE_OFFSETS 3        /* pair offsets (scan of tile counts in depth order) */
#define RGS_PHASE_DUPLICATE 4      /* (tile, Gaussian) pair emission */
#define RGS_PHASE_TILE_SORT 5      /* radix sort of the pairs by tile */
#define RGS_PHASE_RANGES 6         /* per-tile [first, last + 1) (with an SH event, also the
                                      colours of the visible entries) */
#define RGS_PHASE_BLEND_FORWARD 7  /* front-to-back compositing (Eq. alpha) */
#define RGS_PHASE_BLEND_BACKWARD 8 /* back-to-front screen-space gradients */
#define RGS_PHASE_PREPROCESS_BACKWARD 9 /* parameter and twist gradients (Eq. muCjac..sigmaIjac) */
#define RGS_PHASE_COUNT 10

/* Enables (enable != 0) or disables CUDA-event timing of the phases above on every later forward
 * and backward of this context (also inside stream capture, where the events become graph
 * nodes). Costs one event record per phase. */
rgs_status rgs_set_phase_timing(rgs_ctx* ctx, int32_t enable);

/* Device milliseconds of each phase of the most recent forward and backward on `state`
 * (ms[RGS_PHASE_COUNT]; a phase that did not run reads 0). Synchronises `stream`. Outside stream
 * capture, the depth-sort and duplicate phases of a forward include the host synchronisations
 * that size the visible list and the pair list. */
rgs_status rgs_phase_times(rgs_ctx* ctx, uint64_t state, float* ms, int32_t n, void* stream);

/* ---- Diagnostics: copies of a state's binning results (synchronise `stream`). ----
 * rgs_copy_tile_lists: the sorted pair list (the (view, Gaussian) index vi = view * n + i of each
 * pair, tile runs in near-to-far order) into host_vals (capacity vals_cap entries; the number of
 * pairs is written to *n_pairs even when it exceeds vals_cap, in which case nothing is copied),
 * and the [first, last + 1) range of every global tile into host_ranges (2 u32 per tile; global
 * tile ids count view by view, row-major inside a view).
 * rgs_copy_records: the projected records of every (view, Gaussian) into host_rec
 * ([n_views * n][12] floats: mean2d hi x, y, lo x, y; the whitening factor l11, l21, l22, lower
 * triangular with L L^T = (log2 e / 2) (Sigma^I)^-1, and log2 o; r, g, b and camera-space depth),
 * and the touched-tile counts into host_ntiles (may be NULL).
 * A record is meaningful only where its tile count is non-zero. */
rgs_status rgs_copy_tile_lists(rgs_ctx* ctx, uint64_t state, uint32_t* host_vals, int64_t vals_cap,
                               uint32_t* host_ranges, int64_t* n_pairs, void* stream);
rgs_status rgs_copy_records(rgs_ctx* ctx, uint64_t state, float* host_rec, uint32_t* host_ntiles,
                            void* stream);

/* ---- Primitives of the binning stage, exposed for testing (Section 3.1: the front-to-back
 * ordered covering set is built by a key sort). Device pointers, caller-owned. ---- */

/* Stable LSD radix sort of n (key, value) pairs by key bits [begin_bit, end_bit), in place.
 * keys/vals: device u32 arrays of n entries (vals may be NULL for a keys-only sort). Uses the
 * context's scratch memory. 0 <= begin_bit < end_bit <= 32. */
rgs_status rgs_radix_sort_u32(rgs_ctx* ctx, uint32_t* keys, uint32_t* vals, int64_t n,
                              int32_t begin_bit, int32_t end_bit, void* stream);

/* Exclusive prefix sum of n u32 values into out (device arrays; out may equal in), and the
 * total into *total_out (device u32, may be NULL). */
rgs_status rgs_exclusive_scan_u32(rgs_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n,
                                  uint32_t* total_out, void* stream);

/* ---- Mapping (Section 3.5 Eq. map-loss and Eq. reg; appendix Eq. app-ema and the maintenance
 * of observation counts, visibility scores and pruning). ---- */
typedef struct {
  float lambda_iso;        /* weight of sum_i |Sigma_i - tr(Sigma_i) / 3 I|_F */
  float lambda_alpha;      /* weight of sum_i psi(alpha_i), psi = -log(alpha) - log(1 - alpha) */
  float lambda_mu;         /* weight of sum_i |mu_i - mu_bar_i|^2 */
  const float* ema_means;  /* DEVICE [n][3] anchor mu_bar, or NULL: no position term */
  uint32_t* obs_count;     /* DEVICE [n] or NULL: += number of views of the forward that see i */
  float* vis_score;        /* DEVICE [n] or NULL: += that number times alpha_i */
  double* value;           /* DEVICE [1] or NULL: R summed over all Gaussians */
} rgs_map_reg;

/* rgs_render_backward plus the mapping regulariser R of Eq. reg over all n Gaussians (seen or
 * not): its gradients are added to the requested parameter gradients (isotropy: log-scales
 * only, since the Frobenius norm is invariant under the rotation, zero at the isotropic kink;
 * psi: opacity logits, d psi / d logit = 2 alpha - 1; position: means, the anchor held
 * fixed), its value is written to reg->value, and the counters are advanced. Parameters with
 * non-finite values contribute nothing. The first call with reg->value set on a state allocates
 * a per-Gaussian scratch and must be made outside stream capture. reg NULL: rgs_render_backward. */
rgs_status rgs_render_backward_mapping(rgs_ctx* ctx, uint64_t state, const rgs_image_grads* grads,
                                       uint32_t grad_mask, float* d_means, float* d_log_scales,
                                       float* d_quats, float* d_opacity_logits, float* d_sh,
                                       float* d_pose, const rgs_map_reg* reg, void* stream);

/* Anchor update after a mapping step (Eq. app-ema): ema = (1 - eta) ema + eta means, over n
 * Gaussians (DEVICE [n][3] each); 0 < eta < 1. Never synchronises. */
rgs_status rgs_map_ema(rgs_ctx* ctx, int64_t n, const float* means, float* ema_means, float eta,
                       void* stream);

/* Pruning bounds (HOST struct; the paper gives no values): a Gaussian is kept iff
 *   alpha >= min_opacity, tr(Sigma^W) = sum_k exp(2 log_scale_k) <= max_trace, and not
 *   (obs_count >= min_observations and vis_score < min_visibility).
 * Defaults: 0.005, 1.0, 5, 1.0 (observed five times with a summed opacity below one). */
typedef struct {
  float min_opacity;
  float max_trace;
  uint32_t min_observations;
  float min_visibility;
} rgs_prune_config;
void rgs_prune_config_default(rgs_prune_config* cfg);

/* keep[i] = 1 or 0 by the bounds above (DEVICE u8 [n]); n_keep: DEVICE u32 [1], the number
 * kept. Inputs DEVICE [n][3] log-scales, [n] logits, [n] counts, [n] scores. Never
 * synchronises. */
rgs_status rgs_prune_mask(rgs_ctx* ctx, int64_t n, const float* log_scales,
                          const float* opacity_logits, const uint32_t* obs_count,
                          const float* vis_score, const rgs_prune_config* cfg, uint8_t* keep,
                          uint32_t* n_keep, void* stream);

/* Co-visibility of frame pairs for keyframe scheduling (Eq. iou, with the per-pixel visibility
 * masks of the appendix "Keyframe Scheduling by Co-Visibility"): for pair j,
 *   V_a = {p : alpha_a[j n + p] > tau},  V_b = {p : alpha_b[j n + p] > tau},
 *   counts[j] = (|V_a n V_b|, |V_a u V_b|),  iou[j] = |V_a n V_b| / |V_a u V_b| (0 if empty).
 *   alpha_a, alpha_b: DEVICE [n_pairs][n] accumulated opacities (e.g. rgs_images.alpha of two
 *     renders of the same size); counts: DEVICE u64 [n_pairs][2]; iou: DEVICE float [n_pairs].
 * Never synchronises; may be captured. */
rgs_status rgs_covisibility(rgs_ctx* ctx, const float* alpha_a, const float* alpha_b, int64_t n,
                            int32_t n_pairs, float tau, uint64_t* counts, float* iou,
                            void* stream);

/* ---- Dense initialisation (Section 3.3 "Multi-view Triangulation" and "Gaussian Parameter
 * Initialization"; appendix "Gaussian Initialization and Joint Mapping", Eq. app-sigma-init,
 * Eq. app-alpha-init). Matched pixels of a keyframe window become Gaussian seeds: a two-view
 * DLT in double precision per (reference pixel, neighbour), the best hypothesis per pixel, then
 * one seed per accepted point. The paper fixes none of the constants below. ---- */
typedef struct {
  float min_parallax; /* radians: smallest baseline angle of an accepted hypothesis; 1 degree */
  float max_reproj;   /* pixels: largest RMS reprojection error over the two views; 2 */
  float tie_eps;      /* pixels: errors within this of the lowest are ties (larger angle wins); 1e-3 */
  float plane_radius; /* world units: neighbourhood of the plane fit for the normal; 0.05 */
  float s_par_cap;    /* s_par <= s_par_cap * s_perp; 10 */
  float alpha_lo;     /* opacity = alpha_lo + (alpha_hi - alpha_lo) * kappa_bar; 0.1 */
  float alpha_hi;     /* 0.9 */
  float voxel;        /* world units: keep one seed per cube of this edge; 0 = keep all (default) */
} rgs_seed_config;
void rgs_seed_config_default(rgs_seed_config* cfg);

/* Two-view linear triangulation of m reference pixels against up to k (1..8) neighbours each:
 *   A = [x_r P_r^3 - P_r^1; y_r P_r^3 - P_r^2; x_n P_n^3 - P_n^1; y_n P_n^3 - P_n^2],
 *   X~ = argmin_{|X~| = 1} |A X~| (smallest right singular vector, one-sided Jacobi in FP64),
 *   X = X~[0:3] / X~[3], P = K [R | t] of each view.
 * A hypothesis is accepted if X is in front of both cameras, the angle between the two rays at X
 * is at least min_parallax and the RMS reprojection error over the two views is at most
 * max_reproj; the lowest error wins, errors within tie_eps of it are ties decided by the larger
 * angle, then the lower neighbour slot.
 *   cams: HOST array of n_views cameras (intrinsics and poses); cfg: HOST or NULL (defaults).
 *   DEVICE arrays: ref_view [m] int32, ref_xy [m][2] double (pixel (x, y) at (x, y)),
 *     nb_view [m][k] int32 (-1 or out of range: no match), nb_xy [m][k][2] double,
 *     nb_conf [m][k] float (per-match confidence in [0, 1]);
 *   outputs: valid [m] u32 (1 accepted), X [m][3] double, best [m] int32 (slot, -1),
 *     err [m] double (pixels), angle [m] double (radians), kappa [m] float (mean confidence of
 *     the matches, Eq. conf).
 * Never synchronises; may be captured. */
rgs_status rgs_triangulate(rgs_ctx* ctx, const rgs_camera* cams, int32_t n_views, int64_t m,
                           int32_t k, const int32_t* ref_view, const double* ref_xy,
                           const int32_t* nb_view, const double* nb_xy, const float* nb_conf,
                           const rgs_seed_config* cfg, uint32_t* valid, double* X, int32_t* best,
                           double* err, double* angle, float* kappa, void* stream);

/* Gaussian seeds of the accepted points of rgs_triangulate (same m, k, views and arrays):
 *   mean = X; normal v = eigenvector of the smallest eigenvalue of the covariance of the
 *   accepted points within plane_radius of X (FP64 Jacobi), turned towards the reference camera
 *   (fewer than 3 points: the direction to the reference camera); rotation [t1, t2, v] (the
 *   tangent frame of Duff et al. 2017) as a quaternion (w, x, y, z), w >= 0; scales
 *   (s_perp, s_perp, s_par) with s_perp = det(J J^T)^(-1/4) for the projection Jacobian J at X
 *   in the reference view and s_par = min(s_perp (1 + err / 1 px) / sin(angle), s_par_cap s_perp)
 *   (Eq. app-sigma-init); opacity alpha_lo + (alpha_hi - alpha_lo) kappa as a logit
 *   (Eq. app-alpha-init); colour = per-channel median of the exposure-corrected bilinear samples
 *   (I - b) / g over the reference and matched views where X projects inside (SH DC
 *   (c - 0.5) / Y_0, higher orders 0); then, if voxel > 0, one seed per cube of edge voxel
 *   (highest kappa, then lowest index).
 *   observed: DEVICE [P][3] frames (views concatenated as in rgs_images); gain_bias: DEVICE
 *     [n_views][2] exposure (g, b) of each view; sh_degree 0..3.
 *   outputs (DEVICE, capacity m seeds, in increasing reference-pixel order): index [m] int32
 *     (the reference pixel of each seed), means [m][3], log_scales [m][3], quats [m][4],
 *     opacity_logits [m], sh [m][K][3], normals [m][3]; n_seeds: HOST, the number written.
 * Uses a device scratch region held by the context (allocated on the first call and again when m
 * outgrows it, freed by rgs_destroy), so two calls on one context must not run at the same time;
 * synchronises `stream`; not for stream capture. */
rgs_status rgs_init_seeds(rgs_ctx* ctx, const rgs_camera* cams, int32_t n_views, int64_t m,
                          int32_t k, const int32_t* ref_view, const int32_t* nb_view,
                          const uint32_t* valid, const double* X, const double* err,
                          const double* angle, const float* kappa, const float* observed,
                          const float* gain_bias, int32_t sh_degree, const rgs_seed_config* cfg,
                          int32_t* index, float* means, float* log_scales, float* quats,
                          float* opacity_logits, float* sh, float* normals, int64_t* n_seeds,
                          void* stream);

/* ---- Allocation-free variant (the paper has no counterpart: this serves library users). ----
 *
 * rgs_exclusive_scan_u32_static computes exactly what rgs_exclusive_scan_u32 computes, but
 * allocates nothing: no cudaMalloc, no cudaFree, no context. It is for callers that cannot
 * allocate device memory at call time, such as a real-time tracking loop that must not block on
 * the driver's allocator in the middle of a frame, or a process whose device memory is already
 * reserved in full by another framework's caching allocator.
 *   in, out: device u32 arrays of n elements (out may equal in); total_out: device u32 or NULL.
 *   n: 0 <= n <= RGS_STATIC_SCAN_MAX_N; larger n returns RGS_ERR_TOO_LARGE before any GPU work.
 *   stream: cudaStream_t as void* (NULL = legacy default stream). Runs on the current device.
 * Its scratch (one u32 per 4096 elements) is a fixed 64 KiB device array inside the library,
 * held by every GPU that loads the library until the process exits. Every call looks up that
 * array's device address in the current context (cudaGetSymbolAddress), so the first call on a
 * device also loads the library's device code there: make that first call before any stream
 * capture. All calls on a device share the array and keep the last call's contents; nothing in
 * it needs to start at zero. Calls whose executions overlap on the GPU (different streams, or
 * different host threads, without ordering) race on the array: serialise them.
 * Asynchronous: unlike rgs_exclusive_scan_u32, which synchronises its stream before returning,
 * this call only enqueues the scan on `stream`; synchronise the stream before reading out or
 * total_out on the host. Returns RGS_ERR_INVALID_ARG for null arrays with n > 0 and RGS_ERR_CUDA
 * if a CUDA call fails. */
#define RGS_STATIC_SCAN_MAX_N (1 << 26)
rgs_status rgs_exclusive_scan_u32_static(const uint32_t* in, uint32_t* out, int64_t n,
                                         uint32_t* total_out, void* stream);

/* Single-pass exclusive scan (the forward's compaction and pair offsets run on it): one launch,
 * the blocks chaining their prefixes by decoupled look-back (Merrill and Garland, 2016) through
 * caller-owned bookkeeping, so that nothing is allocated and nothing synchronises.
 *   in, out: device u32 arrays of n elements (out may equal in); total_out: device u32 or NULL.
 *   n: 0 <= n < 2^31.
 *   work: device memory of at least rgs_single_pass_scan_bytes(n) bytes, 16-byte aligned, ALL
 *     ZERO when the scan starts (e.g. cudaMemsetAsync on the same stream); the scan leaves it
 *     non-zero. work_bytes: its size.
 *   status: device u32; the scan ORs in 4 if a block gave up its bounded wait (about a second)
 *     for an earlier block's prefix. That is never expected; it means the work area was not
 *     zero or the device is not running the earlier blocks, and the output is then wrong.
 *   stream: cudaStream_t as void*. Asynchronous: no host synchronisation.
 * Returns RGS_ERR_INVALID_ARG for null or misaligned pointers, a negative or too large n or a
 * small work area, before any GPU work; RGS_ERR_CUDA if the launch fails. */
int64_t rgs_single_pass_scan_bytes(int64_t n);
rgs_status rgs_exclusive_scan_u32_single_pass(const uint32_t* in, uint32_t* out, int64_t n,
                                              uint32_t* total_out, void* work, int64_t work_bytes,
                                              uint32_t* status, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RGS_H_ */
