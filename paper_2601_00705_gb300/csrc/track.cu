// track.cu -- the tracking step around the renderer (Section 3.2 and its appendix: Eq.
// app-bright, app-ls, app-trackloss, app-weight; Eq. leftupdate):
//   * pose records: device poses [V][12] -> R, t and the camera centre -R^T t per view, so
//     the projection kernels can read a pose that only the device holds;
//   * gradient weights w_grad(x) = clip(||grad I(x)||_2 / tau_grad, 0, 1) of an observed frame;
//   * the exposure fit (g, b) = argmin sum_x ||I(x) - g I^(x) - b||^2 per view, the weighted L1
//     loss sum_x w_alpha(x) w_grad(x) ||I(x) - (g I^(x) + b)||_1 and its gradient with respect to
//     the rendered colour, which is the upstream gradient of the backward;
//   * one Adam step on the twist xi of every view, applied as T <- exp(xi^) T;
//   * co-visibility of frame pairs for the keyframe test (Eq. iou): intersection and union of
//     the pixels whose accumulated opacity exceeds a threshold.
// All passes are elementwise or reductions over the images (HBM-bound) except the pose update
// (one thread per view).
#include <math.h>

#include <algorithm>

#include "rgs_internal.cuh"

namespace rgs {
namespace {

constexpr int kTrackThreads = 256;

// ------------------------------------------------------------------------------------------
// Pose records: R (9), t (3), c = -R^T t (3), pad. The centre is accumulated in double and
// rounded once, as the host does for poses given in rgs_camera, so both routes give the same
// records bit for bit.
// ------------------------------------------------------------------------------------------
__global__ void pose_prepare_kernel(const float* __restrict__ world_to_cam, int n_views,
                                    float* __restrict__ records) {
  chain_wait();
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_views) return;
  const float* w = world_to_cam + 12 * v;
  float R[9], t[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) R[3 * a + b] = w[4 * a + b];
    t[a] = w[4 * a + 3];
  }
  float* r = records + 16 * v;
#pragma unroll
  for (int k = 0; k < 9; ++k) r[k] = R[k];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    r[9 + a] = t[a];
    double s = 0.0;
#pragma unroll
    for (int b = 0; b < 3; ++b) s -= (double)R[3 * b + a] * (double)t[b];
    r[12 + a] = (float)s;
  }
  r[15] = 0.0f;
}

// Pixel k of view v's pixels, walked by the blocks of grid row v.
__device__ __forceinline__ void view_pixels(const Views& views, int v, long long& first,
                                            int& count, int& width, int& height) {
  const ViewParams& vp = views.v[v];
  first = vp.pixel_offset;
  width = vp.width;
  height = vp.height;
  count = vp.width * vp.height;
}

// ------------------------------------------------------------------------------------------
// Gradient weights (Eq. app-weight): per channel, central differences inside the image and
// one-sided differences on its border (zero along an axis of extent 1); the norm is taken over
// both axes and the three channels.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kTrackThreads) grad_weight_kernel(
    const __grid_constant__ Views views, const float* __restrict__ obs, float inv_tau,
    float* __restrict__ w_out) {
  chain_wait();
  const int v = blockIdx.y;
  long long first;
  int count, W, H;
  view_pixels(views, v, first, count, W, H);
  for (int k = blockIdx.x * kTrackThreads + threadIdx.x; k < count;
       k += gridDim.x * kTrackThreads) {
    const int y = k / W, x = k - y * W;
    const int xl = x > 0 ? x - 1 : x, xr = x < W - 1 ? x + 1 : x;
    const int yu = y > 0 ? y - 1 : y, yd = y < H - 1 ? y + 1 : y;
    const float sx = (xr - xl) == 2 ? 0.5f : 1.0f, sy = (yd - yu) == 2 ? 0.5f : 1.0f;
    const float* row = obs + 3 * (first + (long long)y * W);
    const float* up = obs + 3 * (first + (long long)yu * W);
    const float* dn = obs + 3 * (first + (long long)yd * W);
    float s = 0.0f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const float gx = (xr == xl) ? 0.0f : (row[3 * xr + ch] - row[3 * xl + ch]) * sx;
      const float gy = (yd == yu) ? 0.0f : (dn[3 * x + ch] - up[3 * x + ch]) * sy;
      s = fmaf(gx, gx, fmaf(gy, gy, s));
    }
    w_out[first + k] = fminf(fmaxf(sqrtf(s) * inv_tau, 0.0f), 1.0f);
  }
}

// Block-wide sum of NV values per thread, in double, into (double) accumulators with atomics.
template <int NV>
__device__ __forceinline__ void block_sum_to(const float (&x)[NV], double* __restrict__ acc) {
  __shared__ double s_part[kTrackThreads / 32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NV; ++j) {
    float v = x[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_part[warp][j] = (double)v;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kTrackThreads / 32; ++w) t += s_part[w][threadIdx.x];
    atomicAdd(acc + threadIdx.x, t);
  }
}

// ------------------------------------------------------------------------------------------
// Exposure fit, pass 1 (Eq. app-ls): per view, sum r, sum r^2, sum o, sum r o over the three
// channels of every pixel (r rendered, o observed). Per-thread partial sums in FP32 over a few
// dozen values, FP64 from the warp totals on.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kTrackThreads) track_sums_kernel(
    const __grid_constant__ Views views, const float* __restrict__ color,
    const float* __restrict__ obs, double* __restrict__ sums) {
  chain_wait();
  const int v = blockIdx.y;
  long long first;
  int count, W, H;
  view_pixels(views, v, first, count, W, H);
  float x[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  for (int k = blockIdx.x * kTrackThreads + threadIdx.x; k < count;
       k += gridDim.x * kTrackThreads) {
    const long long p = first + k;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const float r = color[3 * p + ch], o = obs[3 * p + ch];
      x[0] += r;
      x[1] = fmaf(r, r, x[1]);
      x[2] += o;
      x[3] = fmaf(r, o, x[3]);
    }
  }
  block_sum_to<4>(x, sums + 4 * v);
}

// (g, b) of view v from its sums; without a unique fit (a constant render) g = 1 and b matches
// the means.
__device__ __forceinline__ void exposure_of(const double* s, double n, bool fit, double& g,
                                            double& b) {
  if (!fit) {
    g = 1.0;
    b = 0.0;
    return;
  }
  const double sr = s[0], srr = s[1], so = s[2], sro = s[3];
  const double den = n * srr - sr * sr;
  if (n > 0.0 && den > 1e-12 * n * n) {
    g = (n * sro - sr * so) / den;
    b = (so - g * sr) / n;
  } else {
    g = 1.0;
    b = n > 0.0 ? (so - sr) / n : 0.0;
  }
}

// ------------------------------------------------------------------------------------------
// Pass 2 (Eq. app-bright, app-trackloss, app-weight): with r' = g r + b,
//   loss_v = sum_x w(x) sum_ch |o - r'|,  w = clip(alpha / tau_alpha, 0, 1) w_grad,
//   dL/dr_ch = -w g sign(o - r'),
// with (g, b) and w held fixed (they are re-estimated from every render, and no gradient flows
// into them). Writes the upstream colour gradient, the loss per view and (g, b) per view.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kTrackThreads) track_loss_kernel(
    const __grid_constant__ Views views, const float* __restrict__ color,
    const float* __restrict__ alpha, const float* __restrict__ obs,
    const float* __restrict__ w_grad, const double* __restrict__ sums, float inv_tau_alpha,
    int fit_exposure, float* __restrict__ d_color, double* __restrict__ loss,
    float* __restrict__ gain_bias) {
  chain_wait();
  const int v = blockIdx.y;
  long long first;
  int count, W, H;
  view_pixels(views, v, first, count, W, H);
  double gd, bd;
  exposure_of(sums + 4 * v, 3.0 * (double)count, fit_exposure != 0, gd, bd);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    gain_bias[2 * v] = (float)gd;
    gain_bias[2 * v + 1] = (float)bd;
  }
  const float g = (float)gd, b = (float)bd;
  float part[1] = {0.0f};
  for (int k = blockIdx.x * kTrackThreads + threadIdx.x; k < count;
       k += gridDim.x * kTrackThreads) {
    const long long p = first + k;
    float w = fminf(fmaxf(alpha[p] * inv_tau_alpha, 0.0f), 1.0f);
    if (w_grad) w *= w_grad[p];
    float l1 = 0.0f;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const float res = obs[3 * p + ch] - fmaf(g, color[3 * p + ch], b);
      l1 += fabsf(res);
      const float sg = res > 0.0f ? 1.0f : (res < 0.0f ? -1.0f : 0.0f);
      d_color[3 * p + ch] = -w * g * sg;
    }
    part[0] = fmaf(w, l1, part[0]);
  }
  block_sum_to<1>(part, loss + v);
}

// ------------------------------------------------------------------------------------------
// Pose update: one Adam step on the twist xi = (rho, omega) of every view from dL/dxi at
// xi = 0, then T <- exp(xi^) T (Eq. leftupdate) with the closed-form SE(3) exponential:
//   R_d = I + A W + B W^2,  V = I + B W + C W^2,  t_d = V rho,  W = [omega]_x,
//   A = sin(th) / th, B = (1 - cos(th)) / th^2, C = (th - sin(th)) / th^3, th = |omega|
// (Taylor series for small th); R <- R_d R, t <- R_d t + t_d. The learning rate of step k
// (k = 0, 1, ...) is lr * (1 + cos(pi min(k, K) / K)) / 2 with K = iterations, or lr when
// K = 0. In FP64; the pose is stored back in FP32.
// ------------------------------------------------------------------------------------------
__global__ void pose_adam_kernel(int n_views, float lr, float beta1, float beta2, float eps,
                                 int iterations, const float* __restrict__ d_pose,
                                 float* __restrict__ adam_state, int32_t* __restrict__ step,
                                 float* __restrict__ world_to_cam) {
  chain_wait();
  const int v = threadIdx.x;
  const int k = *step;
  __syncthreads();  // every thread has read the step count before it advances
  if (v < n_views) {
    double lr_k = lr;
    if (iterations > 0) {
      const double kk = (double)(k < iterations ? k : iterations);
      lr_k = 0.5 * (double)lr * (1.0 + cos(M_PI * kk / (double)iterations));
    }
    const double c1 = 1.0 - pow((double)beta1, (double)(k + 1));
    const double c2 = 1.0 - pow((double)beta2, (double)(k + 1));
    double xi[6];
    float* m = adam_state + 12 * v;
    float* s2 = m + 6;
    for (int j = 0; j < 6; ++j) {
      const double gj = d_pose[6 * v + j];
      const double mj = (double)beta1 * m[j] + (1.0 - (double)beta1) * gj;
      const double vj = (double)beta2 * s2[j] + (1.0 - (double)beta2) * gj * gj;
      m[j] = (float)mj;
      s2[j] = (float)vj;
      xi[j] = -lr_k * (mj / c1) / (sqrt(vj / c2) + (double)eps);
    }
    const double w0 = xi[3], w1 = xi[4], w2 = xi[5];
    const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
    double A, B, C;
    if (th2 < 1e-10) {
      A = 1.0 - th2 / 6.0;
      B = 0.5 - th2 / 24.0;
      C = 1.0 / 6.0 - th2 / 120.0;
    } else {
      const double th = sqrt(th2);
      A = sin(th) / th;
      B = (1.0 - cos(th)) / th2;
      C = (th - sin(th)) / (th2 * th);
    }
    // W = [omega]_x and W^2.
    const double Wm[9] = {0.0, -w2, w1, w2, 0.0, -w0, -w1, w0, 0.0};
    double W2[9];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        double s = 0.0;
        for (int c = 0; c < 3; ++c) s += Wm[3 * a + c] * Wm[3 * c + b];
        W2[3 * a + b] = s;
      }
    double Rd[9], Vm[9];
    for (int j = 0; j < 9; ++j) {
      const double id = (j % 4 == 0) ? 1.0 : 0.0;
      Rd[j] = id + A * Wm[j] + B * W2[j];
      Vm[j] = id + B * Wm[j] + C * W2[j];
    }
    float* T = world_to_cam + 12 * v;
    double R[9], t[3];
    for (int a = 0; a < 3; ++a) {
      for (int b = 0; b < 3; ++b) R[3 * a + b] = T[4 * a + b];
      t[a] = T[4 * a + 3];
    }
    for (int a = 0; a < 3; ++a) {
      double tn = 0.0;
      for (int b = 0; b < 3; ++b) {
        double rn = 0.0;
        for (int c = 0; c < 3; ++c) rn += Rd[3 * a + c] * R[3 * c + b];
        T[4 * a + b] = (float)rn;
        tn += Rd[3 * a + b] * t[b] + Vm[3 * a + b] * xi[b];
      }
      T[4 * a + 3] = (float)tn;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *step = k + 1;
}

// ------------------------------------------------------------------------------------------
// Co-visibility (Eq. iou, with the per-pixel visibility masks of the keyframe scheduling): for
// pair j, V_a = {p : alpha_a(p) > tau}, V_b likewise, counts |V_a n V_b| and |V_a u V_b| over
// the n pixels of the pair's two images; IoU = intersection / union (0 for an empty union).
// Grid rows are pairs; each block reduces its share with ballots and one atomic per count.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kTrackThreads) covis_count_kernel(
    const float* __restrict__ alpha_a, const float* __restrict__ alpha_b, int64_t n, float tau,
    unsigned long long* __restrict__ counts) {
  chain_wait();
  const int j = blockIdx.y;
  const float* a = alpha_a + (size_t)j * n;
  const float* b = alpha_b + (size_t)j * n;
  unsigned long long inter = 0, uni = 0;
  for (int64_t p = (int64_t)blockIdx.x * kTrackThreads + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * kTrackThreads) {
    const bool va = a[p] > tau, vb = b[p] > tau;
    inter += (va && vb) ? 1u : 0u;
    uni += (va || vb) ? 1u : 0u;
  }
  __shared__ unsigned long long s_i[kTrackThreads / 32], s_u[kTrackThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    inter += __shfl_xor_sync(0xffffffffu, inter, o);
    uni += __shfl_xor_sync(0xffffffffu, uni, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s_i[threadIdx.x >> 5] = inter;
    s_u[threadIdx.x >> 5] = uni;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long ti = 0, tu = 0;
    for (int w = 0; w < kTrackThreads / 32; ++w) {
      ti += s_i[w];
      tu += s_u[w];
    }
    atomicAdd(counts + 2 * j, ti);
    atomicAdd(counts + 2 * j + 1, tu);
  }
}

__global__ void covis_iou_kernel(int n_pairs, const unsigned long long* __restrict__ counts,
                                 float* __restrict__ iou) {
  chain_wait();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n_pairs)
    iou[j] = counts[2 * j + 1] ? (float)((double)counts[2 * j] / (double)counts[2 * j + 1]) : 0.0f;
}

// Grid rows per view, columns enough to cover the largest view (at most 2 waves of blocks).
dim3 view_grid(const Views& views) {
  int max_px = 1;
  for (int v = 0; v < views.n_views; ++v)
    max_px = max(max_px, views.v[v].width * views.v[v].height);
  const int want = (max_px + kTrackThreads * 4 - 1) / (kTrackThreads * 4);
  const int cap = max(1, 2 * 152 * 4 / views.n_views);
  return dim3((unsigned)min(want, cap), (unsigned)views.n_views);
}

}  // namespace

cudaError_t launch_pose_prepare(const float* world_to_cam, int n_views, float* records,
                                cudaStream_t stream) {
  const cudaError_t e = launch_chained(pose_prepare_kernel, dim3(1), dim3(kMaxViews), stream,
                                       world_to_cam, n_views, records);
  RGS_LAUNCHED();
  return e;
}

cudaError_t launch_grad_weight(const Views& views, const float* obs, float tau_grad, float* w_out,
                               cudaStream_t stream) {
  const cudaError_t e = launch_chained(grad_weight_kernel, view_grid(views), dim3(kTrackThreads),
                                       stream, views, obs, 1.0f / tau_grad, w_out);
  RGS_LAUNCHED();
  return e;
}

cudaError_t launch_track_loss(const Views& views, const float* color, const float* alpha,
                              const float* obs, const float* w_grad, float tau_alpha,
                              bool fit_exposure, double* sums, float* d_color, double* loss,
                              float* gain_bias, cudaStream_t stream) {
  const int V = views.n_views;
  cudaError_t e = cudaMemsetAsync(sums, 0, sizeof(double) * 4 * V, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(double) * V, stream);
  if (e != cudaSuccess) return e;
  const dim3 grid = view_grid(views);
  if (fit_exposure) {
    e = launch_chained(track_sums_kernel, grid, dim3(kTrackThreads), stream, views, color, obs,
                       sums);
    RGS_LAUNCHED();
    if (e != cudaSuccess) return e;
  }
  e = launch_chained(track_loss_kernel, grid, dim3(kTrackThreads), stream, views, color, alpha,
                     obs, w_grad, (const double*)sums, 1.0f / tau_alpha, fit_exposure ? 1 : 0,
                     d_color, loss, gain_bias);
  RGS_LAUNCHED();
  return e;
}

cudaError_t launch_covisibility(const float* alpha_a, const float* alpha_b, int64_t n,
                                int n_pairs, float tau, unsigned long long* counts, float* iou,
                                cudaStream_t stream) {
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * 2 * n_pairs, stream);
  if (e != cudaSuccess || n_pairs == 0) return e;
  if (n > 0) {
    const int64_t want = (n + kTrackThreads * 8 - 1) / (kTrackThreads * 8);
    const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, 4 * 152 / n_pairs + 1));
    e = launch_chained(covis_count_kernel, dim3(gx, (unsigned)n_pairs), dim3(kTrackThreads),
                       stream, alpha_a, alpha_b, n, tau, counts);
    RGS_LAUNCHED();
    if (e != cudaSuccess) return e;
  }
  e = launch_chained(covis_iou_kernel, dim3((unsigned)((n_pairs + 255) / 256)), dim3(256), stream,
                     n_pairs, (const unsigned long long*)counts, iou);
  RGS_LAUNCHED();
  return e;
}

cudaError_t launch_pose_adam(int n_views, float lr, float beta1, float beta2, float eps,
                             int iterations, const float* d_pose, float* adam_state,
                             int32_t* step, float* world_to_cam, cudaStream_t stream) {
  const cudaError_t e = launch_chained(pose_adam_kernel, dim3(1), dim3(kMaxViews), stream,
                                       n_views, lr, beta1, beta2, eps, iterations, d_pose,
                                       adam_state, step, world_to_cam);
  RGS_LAUNCHED();
  return e;
}

}  // namespace rgs
