// preprocess.cu -- per-Gaussian projection (forward) and its adjoint with the SE(3) pose
// gradient (backward).
//
// Forward (Section 3.1, Eq. proj; Appendix C.1, Eq. app-sh), two passes: a cull pass over every
// (view, Gaussian) that keeps the entries whose footprint may reach the image, then a full
// projection of those candidates that writes the projected records and tile counts.
// Backward (Section 3.2.3, Eq. muCjac, Eq. muIjac, Eq. sigmaIjac), two phases: per visible entry,
// the view-dependent chain rule and the block-reduced twist gradient of the view; then per
// Gaussian, the sum over the views that see it and the chain to the parameters, so every
// parameter gradient is written once, with no atomics.
#include <algorithm>

#include "rgs_internal.cuh"

namespace rgs {
namespace {

constexpr int kPreThreads = 128;
constexpr int kCullMaxViewsPerThread = 8;  // views one cull thread takes (its candidate buffer)

// Real spherical harmonics of a unit direction, degree <= DEG (basis index l*l + l + m).
// Y_{l,m} = sqrt(2) Re / Im of the complex harmonic with the Condon-Shortley phase, as
// polynomials; the constants are 1/(2 sqrt(pi)), sqrt(3/(4pi)), sqrt(15/pi)/2, sqrt(5/pi)/4,
// sqrt(15/pi)/4, sqrt(35/(2pi))/4, sqrt(105/pi)/2, sqrt(21/(2pi))/4, sqrt(7/pi)/4, sqrt(105/pi)/4.
constexpr float kSH0 = 0.28209479177387814f;
constexpr float kSH1 = 0.4886025119029199f;
constexpr float kSH2a = 1.0925484305920792f;
constexpr float kSH2b = 0.31539156525252005f;
constexpr float kSH2c = 0.5462742152960396f;
constexpr float kSH30 = 0.5900435899266435f;
constexpr float kSH31 = 2.890611442640554f;
constexpr float kSH32 = 0.4570457994644658f;
constexpr float kSH33 = 0.3731763325901154f;
constexpr float kSH35 = 1.445305721320277f;

template <int DEG>
__device__ __forceinline__ void sh_basis(float x, float y, float z, float* Y) {
  Y[0] = kSH0;
  if (DEG >= 1) {
    Y[1] = -kSH1 * y;
    Y[2] = kSH1 * z;
    Y[3] = -kSH1 * x;
  }
  if (DEG >= 2) {
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = kSH2a * x * y;
    Y[5] = -kSH2a * y * z;
    Y[6] = kSH2b * (2.0f * zz - xx - yy);
    Y[7] = -kSH2a * x * z;
    Y[8] = kSH2c * (xx - yy);
    if (DEG >= 3) {
      Y[9] = -kSH30 * y * (3.0f * xx - yy);
      Y[10] = kSH31 * x * y * z;
      Y[11] = -kSH32 * y * (4.0f * zz - xx - yy);
      Y[12] = kSH33 * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
      Y[13] = -kSH32 * x * (4.0f * zz - xx - yy);
      Y[14] = kSH35 * z * (xx - yy);
      Y[15] = -kSH30 * x * (xx - 3.0f * yy);
    }
  }
}

// sum_k w[k] * grad Y_k(x, y, z) (gradient of the polynomials above).
template <int DEG>
__device__ __forceinline__ void sh_basis_vjp(float x, float y, float z, const float* w,
                                             float& gx, float& gy, float& gz) {
  gx = gy = gz = 0.0f;
  if (DEG >= 1) {
    gy += -kSH1 * w[1];
    gz += kSH1 * w[2];
    gx += -kSH1 * w[3];
  }
  if (DEG >= 2) {
    gx += kSH2a * y * w[4];
    gy += kSH2a * x * w[4];
    gy += -kSH2a * z * w[5];
    gz += -kSH2a * y * w[5];
    gx += -2.0f * kSH2b * x * w[6];
    gy += -2.0f * kSH2b * y * w[6];
    gz += 4.0f * kSH2b * z * w[6];
    gx += -kSH2a * z * w[7];
    gz += -kSH2a * x * w[7];
    gx += 2.0f * kSH2c * x * w[8];
    gy += -2.0f * kSH2c * y * w[8];
    if (DEG >= 3) {
      const float xx = x * x, yy = y * y, zz = z * z;
      gx += -kSH30 * 6.0f * x * y * w[9];
      gy += -kSH30 * 3.0f * (xx - yy) * w[9];
      gx += kSH31 * y * z * w[10];
      gy += kSH31 * x * z * w[10];
      gz += kSH31 * x * y * w[10];
      gx += kSH32 * 2.0f * x * y * w[11];
      gy += -kSH32 * (4.0f * zz - xx - 3.0f * yy) * w[11];
      gz += -kSH32 * 8.0f * y * z * w[11];
      gx += -kSH33 * 6.0f * x * z * w[12];
      gy += -kSH33 * 6.0f * y * z * w[12];
      gz += kSH33 * (6.0f * zz - 3.0f * xx - 3.0f * yy) * w[12];
      gx += -kSH32 * (4.0f * zz - 3.0f * xx - yy) * w[13];
      gy += kSH32 * 2.0f * x * y * w[13];
      gz += -kSH32 * 8.0f * x * z * w[13];
      gx += kSH35 * 2.0f * x * z * w[14];
      gy += -kSH35 * 2.0f * y * z * w[14];
      gz += kSH35 * (xx - yy) * w[14];
      gx += -kSH30 * 3.0f * (xx - yy) * w[15];
      gy += kSH30 * 6.0f * x * y * w[15];
    }
  }
}

// Per-Gaussian, view-independent quantities.
struct GaussianLocal {
  float m[3];
  float qn[4];       // unit quaternion (w, x, y, z)
  float qnorm;       // |q| before normalisation
  float Rq[9];       // rotation of the Gaussian, row-major
  float s[3];        // scales exp(log_scale)
  float M[9];        // Rq diag(s)
  float Sw[6];       // Sigma^W = M M^T: xx, xy, xz, yy, yz, zz
  float smax2;       // largest squared scale (largest eigenvalue of Sigma^W)
  float opacity;
};

__device__ __forceinline__ void gaussian_local(const float* m, const float* ls, const float* q,
                                               float logit, GaussianLocal& g) {
  g.m[0] = m[0];
  g.m[1] = m[1];
  g.m[2] = m[2];
  g.qnorm = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const float inv = 1.0f / g.qnorm;
  const float w = q[0] * inv, x = q[1] * inv, y = q[2] * inv, z = q[3] * inv;
  g.qn[0] = w;
  g.qn[1] = x;
  g.qn[2] = y;
  g.qn[3] = z;
  g.Rq[0] = 1.0f - 2.0f * (y * y + z * z);
  g.Rq[1] = 2.0f * (x * y - w * z);
  g.Rq[2] = 2.0f * (x * z + w * y);
  g.Rq[3] = 2.0f * (x * y + w * z);
  g.Rq[4] = 1.0f - 2.0f * (x * x + z * z);
  g.Rq[5] = 2.0f * (y * z - w * x);
  g.Rq[6] = 2.0f * (x * z - w * y);
  g.Rq[7] = 2.0f * (y * z + w * x);
  g.Rq[8] = 1.0f - 2.0f * (x * x + y * y);
#pragma unroll
  for (int k = 0; k < 3; ++k) g.s[k] = expf(ls[k]);
  g.smax2 = fmaxf(g.s[0], fmaxf(g.s[1], g.s[2]));
  g.smax2 *= g.smax2;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) g.M[3 * a + b] = g.Rq[3 * a + b] * g.s[b];
  const float* M = g.M;
  g.Sw[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
  g.Sw[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
  g.Sw[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
  g.Sw[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
  g.Sw[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
  g.Sw[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
  g.opacity = 1.0f / (1.0f + expf(-logit));
}

// Projection of one Gaussian into one view (Eq. proj).
struct ViewProj {
  float mc[3];             // camera-space mean (each component the float32 rounding of exact)
  float u, w;              // x/z, y/z
  float uc, wc;            // clamped for J
  bool u_cl, w_cl;
  float J00, J02, J11, J12;
  float T[6];              // J R, row-major 2x3
  float TS[6];             // T Sigma^W
  float cov[3];            // Sigma^I + eps: xx, xy, yy
  float chol[3];           // l11, l21, l22: (log2(e) / 2) (Sigma^I + eps)^-1 = L L^T
  float mean2d[2];         // projected mean, hi parts
  float mean2d_lo[2];      // and lo parts (mean2d + mean2d_lo = fx u + cx, fy w + cy)
};

// Returns false if the Gaussian is culled in this view (behind znear or degenerate).
__device__ __forceinline__ bool project_view(const GaussianLocal& g, const ViewParams& vp,
                                             const PoseRef& ps, const Consts& c, ViewProj& p) {
  const float* R = ps.R;
  float lo[3];
  p.mc[0] = dot3_plus_dd(R[0], R[1], R[2], g.m[0], g.m[1], g.m[2], ps.t[0], lo[0]);
  p.mc[1] = dot3_plus_dd(R[3], R[4], R[5], g.m[0], g.m[1], g.m[2], ps.t[1], lo[1]);
  p.mc[2] = dot3_plus_dd(R[6], R[7], R[8], g.m[0], g.m[1], g.m[2], ps.t[2], lo[2]);
  const float z = p.mc[2];
  if (!(z > c.znear)) return false;
  const float rz = 1.0f / z;
  p.u = __fdiv_rn(p.mc[0], z);
  p.w = __fdiv_rn(p.mc[1], z);
  // Projected mean in double-float: u = x / z to about 2^-44 from the double-float x and z,
  // then fx u + cx with error-free products and sums.
  {
    const float uq[2] = {p.u, p.w};
    const float f[2] = {vp.fx, vp.fy}, cc[2] = {vp.cx, vp.cy};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      float r = __fmaf_rn(-uq[a], z, p.mc[a]);           // exact remainder of the hi parts
      r = __fsub_rn(__fadd_rn(r, lo[a]), __fmul_rn(uq[a], lo[2]));
      const float ul = __fmul_rn(r, rz);                  // u = uq + ul
      float ph, pl, sh, sl;
      two_prod(f[a], uq[a], ph, pl);
      pl = __fmaf_rn(f[a], ul, pl);
      two_sum(ph, cc[a], sh, sl);
      sl = __fadd_rn(sl, pl);
      p.mean2d[a] = __fadd_rn(sh, sl);
      p.mean2d_lo[a] = __fsub_rn(sl, __fsub_rn(p.mean2d[a], sh));
    }
  }
  p.uc = p.u;
  p.wc = p.w;
  p.u_cl = p.w_cl = false;
  if (vp.lim_u > 0.0f) {
    if (p.u > vp.lim_u) { p.uc = vp.lim_u; p.u_cl = true; }
    if (p.u < -vp.lim_u) { p.uc = -vp.lim_u; p.u_cl = true; }
    if (p.w > vp.lim_w) { p.wc = vp.lim_w; p.w_cl = true; }
    if (p.w < -vp.lim_w) { p.wc = -vp.lim_w; p.w_cl = true; }
  }
  p.J00 = vp.fx * rz;
  p.J02 = -vp.fx * p.uc * rz;
  p.J11 = vp.fy * rz;
  p.J12 = -vp.fy * p.wc * rz;
  // T = J R.
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    p.T[k] = p.J00 * R[k] + p.J02 * R[6 + k];
    p.T[3 + k] = p.J11 * R[3 + k] + p.J12 * R[6 + k];
  }
  // TS = T Sigma^W, Sigma^I = TS T^T + eps I.
  const float* S = g.Sw;
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const float t0 = p.T[3 * r], t1 = p.T[3 * r + 1], t2 = p.T[3 * r + 2];
    p.TS[3 * r + 0] = t0 * S[0] + t1 * S[1] + t2 * S[2];
    p.TS[3 * r + 1] = t0 * S[1] + t1 * S[3] + t2 * S[4];
    p.TS[3 * r + 2] = t0 * S[2] + t1 * S[4] + t2 * S[5];
  }
  // Sigma^I = A A^T + eps I with A = T M (M = Rq diag(s), so that Sigma^W = M M^T). Its
  // determinant comes from the Cauchy-Binet sum of squared 2x2 minors of A, each minor a
  // difference of products evaluated with Kahan's FMA scheme: no cancellation between the two
  // large products ac and b^2, so the conic of a thin, far-stretched ellipse keeps its accuracy.
  float A[6];
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      A[3 * r + k] = p.T[3 * r] * g.M[k] + p.T[3 * r + 1] * g.M[3 + k] + p.T[3 * r + 2] * g.M[6 + k];
  const float sxx = A[0] * A[0] + A[1] * A[1] + A[2] * A[2];
  const float syy = A[3] * A[3] + A[4] * A[4] + A[5] * A[5];
  p.cov[0] = sxx + c.eps2d;
  p.cov[1] = A[0] * A[3] + A[1] * A[4] + A[2] * A[5];
  p.cov[2] = syy + c.eps2d;
  const float m01 = diff_of_products(A[0], A[4], A[1], A[3]);
  const float m02 = diff_of_products(A[0], A[5], A[2], A[3]);
  const float m12 = diff_of_products(A[1], A[5], A[2], A[4]);
  const float det = m01 * m01 + m02 * m02 + m12 * m12 + c.eps2d * (sxx + syy) + c.eps2d * c.eps2d;
  if (!(det > 0.0f)) return false;
  // Lower-triangular factor of the base-2-scaled conic k Q (k = log2(e) / 2, Q = the inverse of
  // Sigma^I + eps I) from the covariance entries and the accurate determinant, with no
  // subtraction: l11 = sqrt(k Syy / det), l21 = -k Sxy / (det l11), l22 = sqrt(k / Syy); then
  // l11^2 = k Q_xx, l11 l21 = k Q_xy and l21^2 + l22^2 = k Q_yy.
  constexpr float k = 0.5f * kLog2e;
  const float idet = 1.0f / det;
  p.chol[0] = sqrtf(k * p.cov[2] * idet);
  p.chol[1] = -k * p.cov[1] * idet / p.chol[0];
  p.chol[2] = sqrtf(k / p.cov[2]);
  return true;
}

template <int DEG>
__device__ __forceinline__ void load_sh(const float* __restrict__ sh, int i, float* c) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  const float* p = sh + (size_t)i * 3 * K;
  if ((3 * K) % 4 == 0) {
    const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int k = 0; k < 3 * K / 4; ++k) {
      const float4 v = __ldg(p4 + k);
      c[4 * k] = v.x;
      c[4 * k + 1] = v.y;
      c[4 * k + 2] = v.z;
      c[4 * k + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 3 * K; ++k) c[k] = __ldg(p + k);
  }
}

// Forward, pass 1 (cull): one thread per (Gaussian, chunk of views). Only the camera-space mean,
// the projected centre and the footprint-radius bound of project_view are computed, and the
// entries that may touch the image are appended to `cand` (gathered in
// shared memory, then one global atomic per block; their order does not matter). Pass 2 then
// projects only those, so its warps are not held up by the large majority of entries that fall
// outside the image.
__global__ void __launch_bounds__(kPreThreads) cull_kernel(
    const __grid_constant__ Views views, const Consts c, int n, const float* __restrict__ means,
    const float* __restrict__ log_scales, const float* __restrict__ quats,
    const float* __restrict__ logits, uint32_t* __restrict__ ntiles, uint32_t* __restrict__ cand,
    uint32_t* __restrict__ vis_bits, int bit_words, Counters* __restrict__ counters,
    int views_per_chunk) {
  static_assert(kPreThreads % 32 == 0, "whole words of the visibility bitmask per block");
  chain_wait();
  __shared__ uint32_t s_cand[kPreThreads * kCullMaxViewsPerThread];
  __shared__ uint32_t s_count, s_base;
  if (threadIdx.x == 0) s_count = 0;
  __syncthreads();
  const int i = blockIdx.x * kPreThreads + threadIdx.x;
  const bool in_range = i < n;
  const int lane = threadIdx.x & 31;
  const int v_begin = blockIdx.y * views_per_chunk;
  const int v_end = min(views.n_views, v_begin + views_per_chunk);
  float m[3] = {0, 0, 0}, ls[3] = {0, 0, 0}, q[4] = {1, 0, 0, 0}, logit = 0.0f;
  if (in_range) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      m[k] = __ldg(means + 3 * (size_t)i + k);
      ls[k] = __ldg(log_scales + 3 * (size_t)i + k);
    }
    const float4 q4 = __ldg(reinterpret_cast<const float4*>(quats) + i);
    q[0] = q4.x;
    q[1] = q4.y;
    q[2] = q4.z;
    q[3] = q4.w;
    logit = __ldg(logits + i);
  }
  bool finite = in_range && isfinite(logit);
#pragma unroll
  for (int k = 0; k < 3; ++k) finite = finite && isfinite(m[k]) && isfinite(ls[k]);
#pragma unroll
  for (int k = 0; k < 4; ++k) finite = finite && isfinite(q[k]);
  const float qn2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  finite = finite && qn2 > 0.0f && isfinite(qn2);
  if (in_range && !finite) atomicAdd(&counters->n_nonfinite, (uint32_t)(v_end - v_begin));
  float smax = fmaxf(ls[0], fmaxf(ls[1], ls[2]));
  const float smax2 = finite ? expf(2.0f * smax) : 0.0f;
  const float opacity = 1.0f / (1.0f + expf(-logit));
  const float kappa = finite ? 2.0f * logf(opacity / c.alpha_min) : -1.0f;
  for (int v = v_begin; v < v_end; ++v) {
    const ViewParams& vp = views.v[v];
    const PoseRef ps = view_pose(views, v);
    const size_t vi = (size_t)v * n + i;
    bool keep = false;
    if (finite && kappa >= 0.0f) {
      const float* R = ps.R;
      // Plain FMA dot products: the cull only has to keep every Gaussian the projection keeps.
      // Their error is below 8 units of roundoff of the summed magnitudes, so a Gaussian is
      // dropped for the near plane only when even z + that bound is at or below it (the
      // projection then decides with its compensated depth); the projected centre's error is
      // far inside the radius bound's 4 px slack.
      const float z = fmaf(R[6], m[0], fmaf(R[7], m[1], fmaf(R[8], m[2], ps.t[2])));
      const float z_err =
          4.8e-7f * (fabsf(R[6] * m[0]) + fabsf(R[7] * m[1]) + fabsf(R[8] * m[2]) + fabsf(ps.t[2]));
      if (z + z_err > c.znear && z > 0.0f) {
        const float x = fmaf(R[0], m[0], fmaf(R[1], m[1], fmaf(R[2], m[2], ps.t[0])));
        const float y = fmaf(R[3], m[0], fmaf(R[4], m[1], fmaf(R[5], m[2], ps.t[1])));
        const float rz = 1.0f / z;
        const float u = x * rz, w = y * rz;
        float uc = u, wc = w;
        if (vp.lim_u > 0.0f) {
          uc = fminf(fmaxf(u, -vp.lim_u), vp.lim_u);
          wc = fminf(fmaxf(w, -vp.lim_w), vp.lim_w);
        }
        const float jf2 = (vp.fx * vp.fx * (1.0f + uc * uc) + vp.fy * vp.fy * (1.0f + wc * wc)) *
                          (rz * rz);
        // A rigorous bound of the alpha >= alpha_min footprint radius: the largest eigenvalue of
        // Sigma^I is at most ||J||_F^2 smax^2 + eps, so the radius is at most
        // sqrt(kappa (||J||_F^2 smax^2 + eps)); widened by 2 % and 4 px, beyond the 1-px padding
        // of the tile coverage and the rounding of this cheaper mean.
        const float rad = sqrtf(kappa * fmaf(jf2, smax2, c.eps2d)) * 1.02f + 4.0f;
        const float mx = fmaf(vp.fx, u, vp.cx), my = fmaf(vp.fy, w, vp.cy);
        keep = !(mx + rad < 0.0f || mx - rad > (float)(vp.width - 1) || my + rad < 0.0f ||
                 my - rad > (float)(vp.height - 1));
      }
    }
    // The block's Gaussians own whole words of row v of the visibility bitmask. Tile counts are
    // written by the projection for its candidates only: the later passes read them only for
    // entries whose visibility bit is set.
    if (threadIdx.x < kPreThreads / 32) {
      const int w = blockIdx.x * (kPreThreads / 32) + threadIdx.x;
      if (w < bit_words) vis_bits[(size_t)v * bit_words + w] = 0u;
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, keep);
    if (ballot) {
      const int leader = __ffs(ballot) - 1;
      uint32_t base = 0;
      if (lane == leader) base = atomicAdd(&s_count, (uint32_t)__popc(ballot));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (keep) s_cand[base + __popc(ballot & ((1u << lane) - 1u))] = (uint32_t)vi;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) s_base = s_count ? atomicAdd(&counters->n_candidates, s_count) : 0u;
  __syncthreads();
  for (uint32_t t = threadIdx.x; t < s_count; t += kPreThreads) cand[s_base + t] = s_cand[t];
}

// Colour of a Gaussian from its SH coefficients (Eq. app-sh) for the direction camera centre ->
// mean, clamped at 0. Both passes that evaluate it call this, so their results are the same bits.
template <int DEG>
__device__ __forceinline__ void sh_colour(const float* shc, const float* m, const PoseRef& ps,
                                          float* rgb) {
  constexpr int K = (DEG + 1) * (DEG + 1);
  float d0 = m[0] - ps.c[0], d1 = m[1] - ps.c[1], d2 = m[2] - ps.c[2];
  const float rn = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
  d0 *= rn;
  d1 *= rn;
  d2 *= rn;
  float Y[16];
  sh_basis<DEG>(d0, d1, d2, Y);
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    float acc = 0.5f;
#pragma unroll
    for (int a = 0; a < K; ++a) acc += shc[3 * a + ch] * Y[a];
    rgb[ch] = fmaxf(acc, 0.0f);
  }
}

// Forward, pass 2 (project): one thread per candidate entry (grid-stride). Full projection
// (Eq. proj), tile count and, for DEG >= 0, the colour; writes the entry's records and tile count.
// An entry with a non-finite SH coefficient is culled here and counted. With DEG = -1 (the
// caller's SH coefficients may still be in flight) the colour is left to the pass after the
// sorts (rec2.xyz = 0 until then). Entries that are not candidates keep ntiles = 0 and unwritten
// records.
template <int DEG, bool kDevPose>
__global__ void __launch_bounds__(kPreThreads) project_kernel(
    const __grid_constant__ Views views, const Consts c, int n, const float* __restrict__ means,
    const float* __restrict__ log_scales, const float* __restrict__ quats,
    const float* __restrict__ logits, const float* __restrict__ sh,
    const uint32_t* __restrict__ cand, float4* __restrict__ rec0, float4* __restrict__ rec1,
    float4* __restrict__ rec2, uint32_t* __restrict__ ntiles, uint32_t* __restrict__ vis_bits,
    int bit_words, Counters* __restrict__ counters) {
  chain_wait();
  constexpr int K = DEG >= 0 ? (DEG + 1) * (DEG + 1) : 1;
  const uint32_t n_cand = counters->n_candidates;
  for (uint32_t k = blockIdx.x * kPreThreads + threadIdx.x; k < n_cand;
       k += gridDim.x * kPreThreads) {
    const uint32_t vi = cand[k];
    const int v = (int)(vi / (uint32_t)n);
    const int i = (int)(vi - (uint32_t)v * (uint32_t)n);
    float m[3], ls[3], q[4];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      m[a] = __ldg(means + 3 * (size_t)i + a);
      ls[a] = __ldg(log_scales + 3 * (size_t)i + a);
    }
    const float4 q4 = __ldg(reinterpret_cast<const float4*>(quats) + i);
    q[0] = q4.x;
    q[1] = q4.y;
    q[2] = q4.z;
    q[3] = q4.w;
    float shc[3 * K];
    if constexpr (DEG >= 0) {
      load_sh<DEG>(sh, i, shc);
      bool sh_finite = true;
#pragma unroll
      for (int a = 0; a < 3 * K; ++a) sh_finite = sh_finite && isfinite(shc[a]);
      if (!sh_finite) {
        atomicAdd(&counters->n_nonfinite, 1u);
        continue;
      }
    }
    GaussianLocal g;
    gaussian_local(m, ls, q, __ldg(logits + i), g);
    const ViewParams& vp = views.v[v];
    const PoseRef ps = view_pose<kDevPose>(views, v);
    ViewProj p;
    if (!project_view(g, vp, ps, c, p)) continue;
    const float4 r0 = make_float4(p.mean2d[0], p.mean2d[1], p.mean2d_lo[0], p.mean2d_lo[1]);
    const float4 r1 = make_float4(p.chol[0], p.chol[1], p.chol[2], log2f(g.opacity));
    float rgb[3] = {0.0f, 0.0f, 0.0f};
    if constexpr (DEG >= 0) sh_colour<DEG>(shc, g.m, ps, rgb);
    const float4 r2 = make_float4(rgb[0], rgb[1], rgb[2], p.mc[2]);
    uint32_t count = 0;
    Ellipse e;
    if (make_ellipse(r0, r1, c.log2_alpha_min, e))
      for_each_tile_row(e, views.tile_w, views.tile_h, vp.tiles_x, vp.tiles_y,
                        [&](int, int tx0, int tx1) { count += (uint32_t)(tx1 - tx0 + 1); });
    rec0[vi] = r0;
    rec1[vi] = r1;
    rec2[vi] = r2;
    ntiles[vi] = count;
    if (count > 0) atomicOr(&vis_bits[(size_t)v * bit_words + (i >> 5)], 1u << (i & 31));
  }
}

// Forward, pass 3 (after the tile lists are built, before the blend), one launch of two
// independent parts.
//  * Blocks [0, range_blocks): tile ranges. Thread t looks at the eight sorted keys 8t .. 8t + 7
//    (two 16-byte loads; the key arrays are 256-byte aligned) and the key before them, and writes
//    the run boundaries among them into `ranges` (zero on entry: tiles without pairs keep
//    [0, 0)).
//  * The other blocks: one thread per visible entry, in (view, Gaussian) order (grid-stride
//    over `list`, the compacted list: neighbouring threads read neighbouring Gaussians' SH
//    rows; in depth order the reads are scattered, which costs ~0.15 ms on 3M Gaussians whose
//    coefficients do not fit in L2). The colour from the SH
//    coefficients for the direction camera centre -> Gaussian (Eq. app-sh), clamped at 0, into
//    rec2.xyz. An entry with a non-finite coefficient gets log2 opacity -inf, so that it covers
//    no pixel in either blend, and is counted as culled.
constexpr int kRangesColourThreads = 256;
constexpr int kRangesKeys = 8;  // sorted keys per thread of the range part (two 16-byte loads)

template <int DEG, bool kDevPose>
__global__ void __launch_bounds__(kRangesColourThreads) ranges_colour_kernel(
    const uint32_t* __restrict__ keys, uint32_t total_tiles, uint2* __restrict__ ranges,
    uint32_t range_blocks, const __grid_constant__ Views views, int n,
    const float* __restrict__ means, const float* __restrict__ sh,
    const uint32_t* __restrict__ list, float4* __restrict__ rec1, float4* __restrict__ rec2,
    Counters* __restrict__ counters) {
  chain_wait();
  if (blockIdx.x < range_blocks) {
    const uint32_t np = counters->n_pairs_stored;
    const uint32_t p0 = (uint32_t)kRangesKeys * (blockIdx.x * kRangesColourThreads + threadIdx.x);
    if (p0 >= np) return;
    uint32_t k[kRangesKeys + 1];  // k[0] = key before p0 (or none), k[1..] = keys p0 ..
    k[0] = p0 > 0 ? keys[p0 - 1] : 0xffffffffu;
    if (p0 + kRangesKeys <= np) {
#pragma unroll
      for (int h = 0; h < kRangesKeys / 4; ++h) {
        const uint4 q = *reinterpret_cast<const uint4*>(keys + p0 + 4 * h);
        k[4 * h + 1] = q.x;
        k[4 * h + 2] = q.y;
        k[4 * h + 3] = q.z;
        k[4 * h + 4] = q.w;
      }
    } else {
#pragma unroll
      for (int j = 0; j < kRangesKeys; ++j) k[j + 1] = p0 + j < np ? keys[p0 + j] : 0xffffffffu;
    }
    const uint32_t next = p0 + kRangesKeys < np ? keys[p0 + kRangesKeys] : 0xffffffffu;
#pragma unroll
    for (int j = 0; j < kRangesKeys; ++j) {
      const uint32_t p = p0 + j;
      const uint32_t key = k[j + 1];
      if (p >= np || key >= total_tiles) continue;
      const uint32_t after = j < kRangesKeys - 1 ? k[j + 2] : next;
      if (p == 0 || k[j] != key) ranges[key].x = p;
      if (p == np - 1 || after != key) ranges[key].y = p + 1;
    }
    return;
  }
  if constexpr (DEG >= 0) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    const uint32_t n_visible = counters->n_visible_kept;
    const uint32_t stride = (gridDim.x - range_blocks) * kRangesColourThreads;
    for (uint32_t k = (blockIdx.x - range_blocks) * kRangesColourThreads + threadIdx.x;
         k < n_visible; k += stride) {
      const uint32_t vi = list[k];
      const int v = (int)(vi / (uint32_t)n);
      const int i = (int)(vi - (uint32_t)v * (uint32_t)n);
      float shc[3 * K];
      load_sh<DEG>(sh, i, shc);
      bool sh_finite = true;
  #pragma unroll
      for (int a = 0; a < 3 * K; ++a) sh_finite = sh_finite && isfinite(shc[a]);
      float4 r2 = rec2[vi];
      if (!sh_finite) {
        atomicAdd(&counters->n_nonfinite, 1u);
        reinterpret_cast<float*>(rec1 + vi)[3] = -INFINITY;
        r2.x = r2.y = r2.z = 0.0f;
        rec2[vi] = r2;
        continue;
      }
      const PoseRef ps = view_pose<kDevPose>(views, v);
      const float m[3] = {__ldg(means + 3 * (size_t)i), __ldg(means + 3 * (size_t)i + 1),
                          __ldg(means + 3 * (size_t)i + 2)};
      float rgb[3];
      sh_colour<DEG>(shc, m, ps, rgb);
      r2.x = rgb[0];
      r2.y = rgb[1];
      r2.z = rgb[2];
      rec2[vi] = r2;
    }
  }
}

// ------------------------------------------------------------------------------------------
// Backward, phase 1: one thread per visible (view, Gaussian) entry (grid-stride over the
// compacted list in (view, Gaussian) order: neighbouring threads read neighbouring Gaussians
// and mostly share a view, whose twist a full warp then sums by shuffles). Chains the entry's screen-space gradients through
// Eq. proj and the colour model to the view-dependent quantities that phase 2 needs, and
// reduces the view's twist gradient over the block. The entry's gradient record is overwritten
// with
//   [0..2] dL/dmu^W (projection and viewing-direction paths), [3..8] dL/dSigma^W (xx, xy, xz,
//   yy, yz, zz; off-diagonal entries hold the sum of both symmetric partners), [9..11] dL/d(raw
//   colour) after the clamp, [12] dL/do.
// ------------------------------------------------------------------------------------------
enum ViewSlot { kVMean = 0, kVSigma = 3, kVRgb = 9, kVOpacity = 12 };

template <int DEG, bool kDevPose>
__global__ void __launch_bounds__(kPreThreads) backward_view_kernel(
    const __grid_constant__ Views views, const Consts c, int n, const float* __restrict__ means,
    const float* __restrict__ log_scales, const float* __restrict__ quats,
    const float* __restrict__ logits, const float* __restrict__ sh,
    const uint32_t* __restrict__ list, const Counters* __restrict__ counters,
    float* __restrict__ g2d, unsigned long long* __restrict__ vis_mask, uint32_t grad_mask,
    float* __restrict__ pose_partial) {
  chain_wait();
  constexpr int K = (DEG + 1) * (DEG + 1);
  __shared__ float s_pose[kMaxViews * 6];
  const int nv = views.n_views;
  for (int t = threadIdx.x; t < nv * 6; t += kPreThreads) s_pose[t] = 0.0f;
  __syncthreads();
  const uint32_t n_visible = counters->n_visible_kept;
  for (uint32_t k = blockIdx.x * kPreThreads + threadIdx.x; k < n_visible;
       k += gridDim.x * kPreThreads) {
    const uint32_t vi = list[k];
    const int v = (int)(vi / (uint32_t)n);
    const int i = (int)(vi - (uint32_t)v * (uint32_t)n);
    float m[3], ls[3], q[4], shc[3 * K];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      m[a] = __ldg(means + 3 * (size_t)i + a);
      ls[a] = __ldg(log_scales + 3 * (size_t)i + a);
    }
    const float4 q4 = __ldg(reinterpret_cast<const float4*>(quats) + i);
    q[0] = q4.x;
    q[1] = q4.y;
    q[2] = q4.z;
    q[3] = q4.w;
    load_sh<DEG>(sh, i, shc);
    // An entry with a non-finite SH coefficient covered no pixel (colour_kernel): its record
    // holds no moments and stays zero, and the view is left out of the Gaussian's mask.
    bool sh_finite = true;
#pragma unroll
    for (int a = 0; a < 3 * K; ++a) sh_finite = sh_finite && isfinite(shc[a]);
    if (!sh_finite) continue;
    GaussianLocal g;
    gaussian_local(m, ls, q, __ldg(logits + i), g);
    const ViewParams& vp = views.v[v];
    const PoseRef ps = view_pose<kDevPose>(views, v);
    float* gp = g2d + (size_t)vi * kG2Stride;
    const float4 ga = *reinterpret_cast<const float4*>(gp);
    const float4 gb = *reinterpret_cast<const float4*>(gp + 4);
    const float2 gc2 = *reinterpret_cast<const float2*>(gp + 8);
    const float m0 = ga.x, wt = ga.y, ws = ga.z, wtt = ga.w;
    const float wts = gb.x, wss = gb.y, g_r = gb.z, g_g = gb.w;
    const float g_b = gc2.x, g_zo = gc2.y;
    ViewProj p;
    project_view(g, vp, ps, c, p);
    const float* R = ps.R;
    // Screen-space gradients from the blend's whitened moments (Section 3.1, Eq. alpha):
    // power = ln o - ln 2 |w|^2 with w = L^T d, d = p - mu^I and L L^T = (log2(e) / 2) Q, so
    //   dpower/dmu^I = Q d = 2 ln 2 L w,
    //   dpower/dSigma^I = 1/2 Q d d^T Q = 2 (ln 2)^2 L w w^T L^T,
    //   dpower/do = 1 / o,
    // and the sums over the covered pixels of dp = dL/dpower times these are linear in
    // sum dp w = (wt, ws) and sum dp w w^T = [[wtt, wts], [wts, wss]].
    const float l11 = p.chol[0], l21 = p.chol[1], l22 = p.chol[2];
    constexpr float c1 = 2.0f * kLn2, c2 = 2.0f * kLn2 * kLn2;
    const float g_mx = c1 * (l11 * wt), g_my = c1 * fmaf(l21, wt, l22 * ws);
    const float g_op = m0 / g.opacity;
    // G_S = c2 L W2 L^T with the lower-triangular L.
    const float r1t = fmaf(l21, wtt, l22 * wts), r1s = fmaf(l21, wts, l22 * wss);
    const float GS00 = c2 * (l11 * (l11 * wtt));
    const float GS01 = c2 * (l11 * r1t);
    const float GS11 = c2 * fmaf(l21, r1t, l22 * r1s);
    // Sigma^I = T Sigma^W T^T: G_T = 2 G_S (T Sigma^W); G_SigmaW = T^T G_S T.
    float GT[6], U[6];
#pragma unroll
    for (int a2 = 0; a2 < 3; ++a2) {
      GT[a2] = 2.0f * (GS00 * p.TS[a2] + GS01 * p.TS[3 + a2]);
      GT[3 + a2] = 2.0f * (GS01 * p.TS[a2] + GS11 * p.TS[3 + a2]);
      U[a2] = GS00 * p.T[a2] + GS01 * p.T[3 + a2];
      U[3 + a2] = GS01 * p.T[a2] + GS11 * p.T[3 + a2];
    }
    float out[13];
    out[kVSigma + 0] = p.T[0] * U[0] + p.T[3] * U[3];
    out[kVSigma + 1] = 2.0f * (p.T[0] * U[1] + p.T[3] * U[4]);
    out[kVSigma + 2] = 2.0f * (p.T[0] * U[2] + p.T[3] * U[5]);
    out[kVSigma + 3] = p.T[1] * U[1] + p.T[4] * U[4];
    out[kVSigma + 4] = 2.0f * (p.T[1] * U[2] + p.T[4] * U[5]);
    out[kVSigma + 5] = p.T[2] * U[2] + p.T[5] * U[5];
    // T = J R: G_J = G_T R^T (all six entries, the structural zeros of J included).
    float GJ[6];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int a2 = 0; a2 < 3; ++a2)
        GJ[3 * r + a2] = GT[3 * r] * R[3 * a2] + GT[3 * r + 1] * R[3 * a2 + 1] +
                         GT[3 * r + 2] * R[3 * a2 + 2];
    // J(mu^C), with no gradient through a clamped x/z or y/z.
    const float z = p.mc[2], rz = 1.0f / z, rz2 = rz * rz;
    const float g_z = -vp.fx * rz2 * GJ[0] - vp.fy * rz2 * GJ[4] + vp.fx * p.uc * rz2 * GJ[2] +
                      vp.fy * p.wc * rz2 * GJ[5];
    float g_u = p.u_cl ? 0.0f : -vp.fx * rz * GJ[2];
    float g_w = p.w_cl ? 0.0f : -vp.fy * rz * GJ[5];
    // mu^I = (fx u + cx, fy w + cy); u = x/z, w = y/z; depth output z.
    g_u += g_mx * vp.fx;
    g_w += g_my * vp.fy;
    float gmc[3];
    gmc[0] = g_u * rz;
    gmc[1] = g_w * rz;
    gmc[2] = g_z - (g_u * p.mc[0] + g_w * p.mc[1]) * rz2 + g_zo;
    // mu^C = R mu^W + t.
#pragma unroll
    for (int a2 = 0; a2 < 3; ++a2)
      out[kVMean + a2] = R[a2] * gmc[0] + R[3 + a2] * gmc[1] + R[6 + a2] * gmc[2];
    // Colour: rgb = max(sum_k sh_k Y_k(dir) + 0.5, 0), dir = normalize(mu^W - c_W).
    float d0 = g.m[0] - ps.c[0], d1 = g.m[1] - ps.c[1],
          d2 = g.m[2] - ps.c[2];
    const float rn = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    d0 *= rn;
    d1 *= rn;
    d2 *= rn;
    float Y[16];
    sh_basis<DEG>(d0, d1, d2, Y);
    float graw[3] = {g_r, g_g, g_b};
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      float acc = 0.5f;
#pragma unroll
      for (int kk = 0; kk < K; ++kk) acc += shc[3 * kk + ch] * Y[kk];
      if (!(acc > 0.0f)) graw[ch] = 0.0f;
      out[kVRgb + ch] = graw[ch];
    }
    float gd[3] = {0.0f, 0.0f, 0.0f};
    if (DEG > 0) {
      float wk[16];
#pragma unroll
      for (int kk = 0; kk < K; ++kk)
        wk[kk] = graw[0] * shc[3 * kk] + graw[1] * shc[3 * kk + 1] + graw[2] * shc[3 * kk + 2];
      float gx, gy, gz;
      sh_basis_vjp<DEG>(d0, d1, d2, wk, gx, gy, gz);
      const float dd = gx * d0 + gy * d1 + gz * d2;
      gd[0] = (gx - d0 * dd) * rn;
      gd[1] = (gy - d1 * dd) * rn;
      gd[2] = (gz - d2 * dd) * rn;
    }
#pragma unroll
    for (int a2 = 0; a2 < 3; ++a2) out[kVMean + a2] += gd[a2];
    out[kVOpacity] = g_op;
    // Overwrite the record for phase 2 (13 of its 16 slots) and mark the view in the
    // Gaussian's visibility mask.
    *reinterpret_cast<float4*>(gp) = make_float4(out[0], out[1], out[2], out[3]);
    *reinterpret_cast<float4*>(gp + 4) = make_float4(out[4], out[5], out[6], out[7]);
    *reinterpret_cast<float4*>(gp + 8) = make_float4(out[8], out[9], out[10], out[11]);
    gp[12] = out[12];
    atomicOr(vis_mask + i, 1ull << v);
    if (grad_mask & RGS_GRAD_POSE) {
      // Twist of the left update (Eq. leftupdate, Eq. muCjac, Eq. sigmaIjac):
      //   rho   = dL/dmu^C + R dL/d(dir-vector)            (the camera centre moves with -R^T t)
      //   omega = mu^C x dL/dmu^C + skew part of J^T G_J   (rotation of Sigma^I, dR = [w]_x R)
      float pose[6];
      pose[0] = gmc[0] + R[0] * gd[0] + R[1] * gd[1] + R[2] * gd[2];
      pose[1] = gmc[1] + R[3] * gd[0] + R[4] * gd[1] + R[5] * gd[2];
      pose[2] = gmc[2] + R[6] * gd[0] + R[7] * gd[1] + R[8] * gd[2];
      pose[3] = p.mc[1] * gmc[2] - p.mc[2] * gmc[1] + p.J02 * GJ[1] + p.J12 * GJ[4] - p.J11 * GJ[5];
      pose[4] = p.mc[2] * gmc[0] - p.mc[0] * gmc[2] + p.J00 * GJ[2] - p.J02 * GJ[0] - p.J12 * GJ[3];
      pose[5] = p.mc[0] * gmc[1] - p.mc[1] * gmc[0] + p.J11 * GJ[3] - p.J00 * GJ[1];
      // A full warp on one view sums its twists by shuffles and adds them once; otherwise each
      // lane adds its own (a shared-memory atomic per lane and component).
      const unsigned active = __activemask();
      const unsigned same = __match_any_sync(active, v);
      if (active == 0xffffffffu && same == 0xffffffffu) {
#pragma unroll
        for (int a2 = 0; a2 < 6; ++a2)
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) pose[a2] += __shfl_xor_sync(0xffffffffu, pose[a2], o);
        if ((threadIdx.x & 31) == 0)
#pragma unroll
          for (int a2 = 0; a2 < 6; ++a2) atomicAdd(&s_pose[v * 6 + a2], pose[a2]);
      } else {
#pragma unroll
        for (int a2 = 0; a2 < 6; ++a2) atomicAdd(&s_pose[v * 6 + a2], pose[a2]);
      }
    }
  }
  if (grad_mask & RGS_GRAD_POSE) {
    __syncthreads();
    for (int t = threadIdx.x; t < nv * 6; t += kPreThreads)
      pose_partial[(size_t)blockIdx.x * nv * 6 + t] = s_pose[t];
  }
}

// ------------------------------------------------------------------------------------------
// Backward, phase 2: one thread per Gaussian. Sums the phase-1 records of the views that see
// the Gaussian (their bits in the visibility mask phase 1 set; records and mask are cleared for
// the next backward), accumulates the SH coefficient gradients view by view, and chains
// dL/dSigma^W to the log-scales and the quaternion once. Every parameter gradient is written
// exactly once.
// ------------------------------------------------------------------------------------------
template <int DEG, bool kReg>
// At most 80 registers (6 blocks of 128 threads per SM): the kernel waits on its gathers, and
// 24 resident warps per SM instead of 16 halve its time despite a few spilled registers (0.98
// -> 0.50 ms over 3M Gaussians; with 64 registers the spills cost more than the warps gain).
__global__ void __launch_bounds__(kPreThreads, 6) backward_gaussian_kernel(
    const __grid_constant__ Views views, int n, const float* __restrict__ means,
    const float* __restrict__ log_scales, const float* __restrict__ quats,
    const float* __restrict__ logits, unsigned long long* __restrict__ vis_mask,
    float* __restrict__ g2d, uint32_t grad_mask, float* __restrict__ d_means,
    float* __restrict__ d_log_scales, float* __restrict__ d_quats, float* __restrict__ d_logits,
    float* __restrict__ d_sh, const MapReg reg, const float* __restrict__ pose_partial,
    int pose_blocks, int n_views, float* __restrict__ d_pose) {
  chain_wait();
  constexpr int K = (DEG + 1) * (DEG + 1);
  __shared__ float s_gsh[3 * K * kPreThreads];
  // Blocks 0 .. 6 V - 1 first finish the twist gradient: d_pose[v, k] = the sum over phase 1's
  // blocks of their partials, in double precision (phase 1 is complete when this kernel runs).
  if (d_pose && (int)blockIdx.x < 6 * n_views) {
    const int vk = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < pose_blocks; b += kPreThreads)
      s += (double)pose_partial[(size_t)b * n_views * 6 + vk];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ double red[kPreThreads / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < kPreThreads / 32; ++w) t += red[w];
      d_pose[vk] = (float)t;
    }
  }
  const int i = blockIdx.x * kPreThreads + threadIdx.x;
  if (i >= n) return;
  // Views that see the Gaussian, as marked by phase 1 (consumed: left zero for the next call).
  uint64_t vis = vis_mask[i];
  if constexpr (!kReg) {
    // Seen by no view: every gradient is zero, and nothing else needs the parameters.
    if (vis == 0) {
      if ((grad_mask & RGS_GRAD_MEANS) && d_means)
#pragma unroll
        for (int k = 0; k < 3; ++k) d_means[3 * (size_t)i + k] = 0.0f;
      if ((grad_mask & RGS_GRAD_SCALES) && d_log_scales)
#pragma unroll
        for (int k = 0; k < 3; ++k) d_log_scales[3 * (size_t)i + k] = 0.0f;
      if ((grad_mask & RGS_GRAD_QUATS) && d_quats)
        reinterpret_cast<float4*>(d_quats)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      if ((grad_mask & RGS_GRAD_OPACITY) && d_logits) d_logits[i] = 0.0f;
      if ((grad_mask & RGS_GRAD_SH) && d_sh) {
        float* p = d_sh + (size_t)i * 3 * K;
        if ((3 * K) % 4 == 0) {
#pragma unroll
          for (int k = 0; k < 3 * K / 4; ++k)
            reinterpret_cast<float4*>(p)[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
#pragma unroll
          for (int k = 0; k < 3 * K; ++k) p[k] = 0.0f;
        }
      }
      return;
    }
  }
  // Every parameter read is issued here, together, ahead of the records' loads.
  float m[3], ls[3], q[4];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    m[a] = __ldg(means + 3 * (size_t)i + a);
    ls[a] = __ldg(log_scales + 3 * (size_t)i + a);
  }
  {
    const float4 q4 = __ldg(reinterpret_cast<const float4*>(quats) + i);
    q[0] = q4.x;
    q[1] = q4.y;
    q[2] = q4.z;
    q[3] = q4.w;
  }
  const float logit = __ldg(logits + i);
  float gm[3] = {0, 0, 0}, gSw[6] = {0, 0, 0, 0, 0, 0}, gop = 0.0f;
  // The SH coefficient gradients accumulate in this thread's column of shared memory (bank =
  // thread), which keeps 3K accumulators out of registers: at 114 registers the kernel held 16
  // warps per SM and waited on its loads.
  float* gsh = s_gsh + threadIdx.x;  // gsh[k * kPreThreads]
#pragma unroll
  for (int k = 0; k < 3 * K; ++k) gsh[k * kPreThreads] = 0.0f;
  if (vis) vis_mask[i] = 0ull;
  const bool any_visible = vis != 0;
  const int n_seen = __popcll(vis);
  (void)n_seen;
  // The records are gathered one view ahead: the next view's loads are issued before the
  // current record is cleared and accumulated.
  struct Rec {
    float4 r0, r1, r2;
    float r3;
  };
  auto load_rec = [&](int v, Rec& r) {
    const float* gp = g2d + ((size_t)v * n + i) * kG2Stride;
    r.r0 = *reinterpret_cast<const float4*>(gp);
    r.r1 = *reinterpret_cast<const float4*>(gp + 4);
    r.r2 = *reinterpret_cast<const float4*>(gp + 8);
    r.r3 = gp[12];
  };
  int v = -1;
  Rec cur{};
  if (vis) {
    v = __ffsll((long long)vis) - 1;
    vis &= vis - 1;
    load_rec(v, cur);
  }
  while (v >= 0) {
    int v_next = -1;
    Rec nxt{};
    if (vis) {
      v_next = __ffsll((long long)vis) - 1;
      vis &= vis - 1;
      load_rec(v_next, nxt);
    }
    // Consume: leave the record zeroed for the next backward.
    float* gp = g2d + ((size_t)v * n + i) * kG2Stride;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    *reinterpret_cast<float4*>(gp) = zero;
    *reinterpret_cast<float4*>(gp + 4) = zero;
    *reinterpret_cast<float4*>(gp + 8) = zero;
    gp[12] = 0.0f;
    gm[0] += cur.r0.x;
    gm[1] += cur.r0.y;
    gm[2] += cur.r0.z;
    gSw[0] += cur.r0.w;
    gSw[1] += cur.r1.x;
    gSw[2] += cur.r1.y;
    gSw[3] += cur.r1.z;
    gSw[4] += cur.r1.w;
    gSw[5] += cur.r2.x;
    gop += cur.r3;
    if (grad_mask & RGS_GRAD_SH) {
      const PoseRef ps = view_pose(views, v);
      float d0 = m[0] - ps.c[0], d1 = m[1] - ps.c[1],
            d2 = m[2] - ps.c[2];
      const float rn = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
      float Y[16];
      sh_basis<DEG>(d0 * rn, d1 * rn, d2 * rn, Y);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        gsh[(3 * k + 0) * kPreThreads] += cur.r2.y * Y[k];
        gsh[(3 * k + 1) * kPreThreads] += cur.r2.z * Y[k];
        gsh[(3 * k + 2) * kPreThreads] += cur.r2.w * Y[k];
      }
    }
    v = v_next;
    cur = nxt;
  }
  float gls[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0}, glogit = 0.0f;
  // A Gaussian culled in every view gets zero gradients; its local quantities may be
  // non-finite and must not enter the chain below.
  if (any_visible) {
    GaussianLocal g;
    gaussian_local(m, ls, q, logit, g);
    glogit = gop * g.opacity * (1.0f - g.opacity);
    if (grad_mask & (RGS_GRAD_SCALES | RGS_GRAD_QUATS)) {
      // Sigma^W = M M^T, M = Rq diag(s): G_M = 2 G_Sym M with G_Sym the symmetric matrix whose
      // off-diagonal entries are half the accumulated off-diagonal gradients.
      const float S00 = gSw[0], S01 = 0.5f * gSw[1], S02 = 0.5f * gSw[2];
      const float S11 = gSw[3], S12 = 0.5f * gSw[4], S22 = gSw[5];
      float GM[9];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        GM[k] = 2.0f * (S00 * g.M[k] + S01 * g.M[3 + k] + S02 * g.M[6 + k]);
        GM[3 + k] = 2.0f * (S01 * g.M[k] + S11 * g.M[3 + k] + S12 * g.M[6 + k]);
        GM[6 + k] = 2.0f * (S02 * g.M[k] + S12 * g.M[3 + k] + S22 * g.M[6 + k]);
      }
#pragma unroll
      for (int k = 0; k < 3; ++k)
        gls[k] = (GM[k] * g.Rq[k] + GM[3 + k] * g.Rq[3 + k] + GM[6 + k] * g.Rq[6 + k]) * g.s[k];
      float G[9];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) G[3 * a + b] = GM[3 * a + b] * g.s[b];
      const float w = g.qn[0], x = g.qn[1], y = g.qn[2], z = g.qn[3];
      const float gw = 2.0f * (-z * G[1] + y * G[2] + z * G[3] - x * G[5] - y * G[6] + x * G[7]);
      const float gx = 2.0f * (y * G[1] + z * G[2] + y * G[3] - 2.0f * x * G[4] - w * G[5] +
                               z * G[6] + w * G[7] - 2.0f * x * G[8]);
      const float gy = 2.0f * (-2.0f * y * G[0] + x * G[1] + w * G[2] + x * G[3] + z * G[5] -
                               w * G[6] + z * G[7] - 2.0f * y * G[8]);
      const float gz = 2.0f * (-2.0f * z * G[0] - w * G[1] + x * G[2] + w * G[3] -
                               2.0f * z * G[4] + y * G[5] + x * G[6] + y * G[7]);
      // Normalisation q / |q|.
      const float dot = gw * w + gx * x + gy * y + gz * z;
      const float iq = 1.0f / g.qnorm;
      gq[0] = (gw - w * dot) * iq;
      gq[1] = (gx - x * dot) * iq;
      gq[2] = (gy - y * dot) * iq;
      gq[3] = (gz - z * dot) * iq;
    }
  }
  if constexpr (kReg) {
    // Eq. reg for this Gaussian, with its gradients added to the rendering ones:
    //   lambda_iso |Sigma - tr(Sigma) / 3 I|_F = lambda_iso sqrt(sum_k (s_k^2 - mean s^2)^2)
    //     (the Frobenius norm is invariant under the rotation, so only the scales enter;
    //     d/d log s_k = 2 s_k^2 (s_k^2 - mean s^2) / norm, 0 at the isotropic kink),
    //   lambda_alpha psi(alpha), psi = -log(alpha) - log(1 - alpha) = |l| + 2 log(1 + e^-|l|)
    //     for the logit l (d psi / d l = 2 alpha - 1),
    //   lambda_mu |mu - mu_bar|^2 (d / d mu = 2 lambda_mu (mu - mu_bar)).
    // Non-finite parameters contribute nothing. The counters add the views that see it.
    const float l = logit;
    float val = 0.0f;
    const bool finite = isfinite(ls[0]) && isfinite(ls[1]) && isfinite(ls[2]) && isfinite(l) &&
                        isfinite(m[0]) && isfinite(m[1]) && isfinite(m[2]);
    const float alpha = 1.0f / (1.0f + expf(-l));
    if (finite) {
      float s2[3], mean = 0.0f;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        s2[a] = expf(2.0f * ls[a]);
        mean += s2[a];
      }
      mean *= (1.0f / 3.0f);
      float nrm2 = 0.0f;
#pragma unroll
      for (int a = 0; a < 3; ++a) nrm2 = fmaf(s2[a] - mean, s2[a] - mean, nrm2);
      const float nrm = sqrtf(nrm2);
      val = reg.lambda_iso * nrm;
      if (nrm > 0.0f)
#pragma unroll
        for (int a = 0; a < 3; ++a) gls[a] += reg.lambda_iso * 2.0f * s2[a] * (s2[a] - mean) / nrm;
      const float al = fabsf(l);
      val += reg.lambda_alpha * (al + 2.0f * log1pf(expf(-al)));
      glogit += reg.lambda_alpha * (2.0f * alpha - 1.0f);
      if (reg.ema_means) {
        float d2 = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const float d = m[a] - __ldg(reg.ema_means + 3 * (size_t)i + a);
          d2 = fmaf(d, d, d2);
          gm[a] += 2.0f * reg.lambda_mu * d;
        }
        val += reg.lambda_mu * d2;
      }
    }
    if (reg.values) reg.values[i] = val;
    if (reg.obs_count) reg.obs_count[i] += (uint32_t)n_seen;
    if (reg.vis_score) reg.vis_score[i] += (float)n_seen * (finite ? alpha : 0.0f);
  }
  if ((grad_mask & RGS_GRAD_MEANS) && d_means)
#pragma unroll
    for (int k = 0; k < 3; ++k) d_means[3 * (size_t)i + k] = gm[k];
  if ((grad_mask & RGS_GRAD_SCALES) && d_log_scales)
#pragma unroll
    for (int k = 0; k < 3; ++k) d_log_scales[3 * (size_t)i + k] = gls[k];
  if ((grad_mask & RGS_GRAD_QUATS) && d_quats)
    reinterpret_cast<float4*>(d_quats)[i] = make_float4(gq[0], gq[1], gq[2], gq[3]);
  if ((grad_mask & RGS_GRAD_OPACITY) && d_logits) d_logits[i] = glogit;
  if ((grad_mask & RGS_GRAD_SH) && d_sh) {
    float* p = d_sh + (size_t)i * 3 * K;
    if ((3 * K) % 4 == 0) {
#pragma unroll
      for (int k = 0; k < 3 * K / 4; ++k)
        reinterpret_cast<float4*>(p)[k] =
            make_float4(gsh[(4 * k) * kPreThreads], gsh[(4 * k + 1) * kPreThreads],
                        gsh[(4 * k + 2) * kPreThreads], gsh[(4 * k + 3) * kPreThreads]);
    } else {
#pragma unroll
      for (int k = 0; k < 3 * K; ++k) p[k] = gsh[k * kPreThreads];
    }
  }
}

// R = sum of the per-Gaussian values, in double precision (grid-stride, one atomic per block).
__global__ void __launch_bounds__(256) reg_sum_kernel(int n, const float* __restrict__ values,
                                                      double* __restrict__ value) {
  chain_wait();
  double s = 0.0;
  for (int i = blockIdx.x * 256 + threadIdx.x; i < n; i += gridDim.x * 256) s += (double)values[i];
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(value, red[0]);
}

}  // namespace

cudaError_t launch_preprocess_forward(const Views& views, const Consts& c,
                                      const rgs_gaussians& g, float4* rec0, float4* rec1,
                                      float4* rec2, uint32_t* ntiles, uint32_t* cand,
                                      uint32_t* vis_bits, bool defer_colour, Counters* counters,
                                      cudaStream_t stream) {
  if (g.n == 0) return cudaSuccess;
  const int bit_words = (int)vis_bit_words_per_view(g.n);
  // Pass 1: one thread per (Gaussian, chunk of views), enough threads to fill every SM a few
  // times over.
  const int blocks_x = (g.n + kPreThreads - 1) / kPreThreads;
  const int target_blocks = 8 * 152;
  const int chunks = max((views.n_views + kCullMaxViewsPerThread - 1) / kCullMaxViewsPerThread,
                         min(views.n_views, (target_blocks + blocks_x - 1) / blocks_x));
  const int per_chunk = (views.n_views + chunks - 1) / chunks;
  const dim3 grid((unsigned)blocks_x, (unsigned)((views.n_views + per_chunk - 1) / per_chunk));
  cudaError_t e = launch_chained(cull_kernel, grid, dim3(kPreThreads), stream, views, c, g.n,
                                 g.means, g.log_scales, g.quats, g.opacity_logits, ntiles, cand,
                                 vis_bits, bit_words, counters, per_chunk);
  RGS_LAUNCHED();
  if (e != cudaSuccess) return e;
  // Pass 2: grid-stride over the candidates.
  const int64_t vn = (int64_t)views.n_views * g.n;
  const int blocks2 = (int)std::min<int64_t>((vn + kPreThreads - 1) / kPreThreads, 16 * 152);
#define RGS_PROJECT(D)                                                                          \
  e = launch_chained(views.pose_dev ? project_kernel<D, true> : project_kernel<D, false>,         \
                     dim3(blocks2), dim3(kPreThreads), stream, views, c, g.n, g.means,            \
                     g.log_scales, g.quats, g.opacity_logits, g.sh, (const uint32_t*)cand, rec0, \
                     rec1, rec2, ntiles, vis_bits, bit_words, counters)
  if (defer_colour) {
    RGS_PROJECT(-1);
  } else {
    switch (g.sh_degree) {
      case 0: RGS_PROJECT(0); break;
      case 1: RGS_PROJECT(1); break;
      case 2: RGS_PROJECT(2); break;
      default: RGS_PROJECT(3); break;
    }
  }
  RGS_LAUNCHED();
#undef RGS_PROJECT
  return e;
}

cudaError_t launch_ranges_colour(const uint32_t* keys, int total_tiles, uint2* ranges,
                                 uint32_t pair_capacity, const Views& views,
                                 const rgs_gaussians& g, const uint32_t* list, int64_t vis_cap,
                                 bool colour, float4* rec1, float4* rec2, Counters* counters,
                                 cudaStream_t stream) {
  const uint32_t range_blocks =
      (uint32_t)(((int64_t)pair_capacity + kRangesKeys * kRangesColourThreads - 1) /
                 (kRangesKeys * kRangesColourThreads));
  const int64_t colour_items = colour && g.n > 0 ? vis_cap : 0;
  const uint32_t colour_blocks = (uint32_t)std::min<int64_t>(
      (colour_items + kRangesColourThreads - 1) / kRangesColourThreads, 4 * 152);
  if (range_blocks + colour_blocks == 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  if (colour_blocks == 0) {
    // Ranges only: the instance without the colour code keeps the registers, and so the
    // occupancy, of a plain scan over the pairs.
    e = launch_chained(ranges_colour_kernel<-1, false>, dim3(range_blocks),
                       dim3(kRangesColourThreads), stream, keys, (uint32_t)total_tiles, ranges,
                       range_blocks, views, g.n, g.means, g.sh, list, rec1, rec2, counters);
    RGS_LAUNCHED();
    return e;
  }
#define RGS_RANGES_COLOUR(D)                                                                   \
  e = launch_chained(views.pose_dev ? ranges_colour_kernel<D, true>                             \
                                    : ranges_colour_kernel<D, false>,                           \
                     dim3(range_blocks + colour_blocks), dim3(kRangesColourThreads), stream,    \
                     keys, (uint32_t)total_tiles, ranges, range_blocks, views, g.n, g.means,    \
                     g.sh, list, rec1, rec2, counters)
  switch (g.sh_degree) {
    case 0: RGS_RANGES_COLOUR(0); break;
    case 1: RGS_RANGES_COLOUR(1); break;
    case 2: RGS_RANGES_COLOUR(2); break;
    default: RGS_RANGES_COLOUR(3); break;
  }
  RGS_LAUNCHED();
#undef RGS_RANGES_COLOUR
  return e;
}

// Phase-1 grid: a fixed number of blocks (grid-stride over the visible entries), so the
// per-block twist partials stay small at any scene size.
int preprocess_backward_blocks(int64_t vn) {
  const int64_t need = (vn + kPreThreads - 1) / kPreThreads;
  return (int)std::min<int64_t>(std::max<int64_t>(need, 1), 8 * 152);
}

cudaError_t launch_preprocess_backward(const Views& views, const Consts& c,
                                       const rgs_gaussians& g, unsigned long long* vis_mask,
                                       const uint32_t* list, const Counters* counters,
                                       int64_t vn, float* g2d, uint32_t grad_mask,
                                       float* d_means, float* d_log_scales, float* d_quats,
                                       float* d_logits, float* d_sh, float* pose_partial,
                                       float* d_pose, const MapReg* reg, cudaStream_t stream) {
  const int blocks1 = preprocess_backward_blocks(vn);
  cudaError_t e = cudaSuccess;
  if (g.n > 0) {
#define RGS_BWD_VIEW(D)                                                                          \
  e = launch_chained(views.pose_dev ? backward_view_kernel<D, true>                               \
                                    : backward_view_kernel<D, false>,                             \
                     dim3(blocks1), dim3(kPreThreads), stream, views, c, g.n, g.means,            \
                     g.log_scales, g.quats, g.opacity_logits, g.sh, list, counters, g2d,          \
                     vis_mask, grad_mask, pose_partial)
    switch (g.sh_degree) {
      case 0: RGS_BWD_VIEW(0); break;
      case 1: RGS_BWD_VIEW(1); break;
      case 2: RGS_BWD_VIEW(2); break;
      default: RGS_BWD_VIEW(3); break;
    }
    RGS_LAUNCHED();
#undef RGS_BWD_VIEW
    if (e != cudaSuccess) return e;
    float* pose_out = ((grad_mask & RGS_GRAD_POSE) && d_pose) ? d_pose : nullptr;
    const int blocks2 = std::max((g.n + kPreThreads - 1) / kPreThreads,
                                 pose_out ? 6 * views.n_views : 1);
    const MapReg no_reg{};
#define RGS_BWD_GAUSS(D)                                                                          \
  e = launch_chained(reg ? backward_gaussian_kernel<D, true> : backward_gaussian_kernel<D, false>, \
                     dim3(blocks2), dim3(kPreThreads), stream, views, g.n, g.means, g.log_scales, \
                     g.quats, g.opacity_logits, vis_mask, g2d, grad_mask, d_means, d_log_scales,  \
                     d_quats, d_logits, d_sh, reg ? *reg : no_reg, (const float*)pose_partial,    \
                     blocks1, views.n_views, pose_out)
    switch (g.sh_degree) {
      case 0: RGS_BWD_GAUSS(0); break;
      case 1: RGS_BWD_GAUSS(1); break;
      case 2: RGS_BWD_GAUSS(2); break;
      default: RGS_BWD_GAUSS(3); break;
    }
    RGS_LAUNCHED();
#undef RGS_BWD_GAUSS
    if (e != cudaSuccess) return e;
  }
  if (reg && reg->value) {
    e = cudaMemsetAsync(reg->value, 0, sizeof(double), stream);
    if (e == cudaSuccess && g.n > 0 && reg->values) {
      const int blocks = std::min((g.n + 255) / 256, 4 * 152);
      e = launch_chained(reg_sum_kernel, dim3(blocks), dim3(256), stream, g.n,
                         (const float*)reg->values, reg->value);
      RGS_LAUNCHED();
    }
    if (e != cudaSuccess) return e;
  }
  // With Gaussians, the per-Gaussian phase above has finished the twist gradient.
  if ((grad_mask & RGS_GRAD_POSE) && d_pose && g.n == 0)
    e = cudaMemsetAsync(d_pose, 0, sizeof(float) * 6 * views.n_views, stream);
  return e;
}

}  // namespace rgs
