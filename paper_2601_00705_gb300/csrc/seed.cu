// seed.cu -- the single-step dense initialisation (Section 3.3 "Multi-view Triangulation" and
// "Gaussian Parameter Initialization"; appendix "Gaussian Initialization and Joint Mapping",
// Eq. app-sigma-init, Eq. app-alpha-init), in FP64 where the paper asks for double precision:
//   triangulate_kernel  one thread per retained reference pixel: for each neighbour the 4x4
//                       linear system of the two-view DLT, its smallest right singular vector by
//                       one-sided Jacobi (Hestenes) in FP64, reprojection error and baseline
//                       angle; the best accepted hypothesis;
//   cell keys + sort    the accepted points grouped by cubic cells of the plane-fit radius
//                       (exact 63-bit cell keys, two stable 32-bit radix sorts);
//   seed_kernel         per accepted point: the points within the radius (27 cells, binary search
//                       in the sorted keys), plane fit by a 3x3 Jacobi eigen-solve, tangent frame,
//                       scales from the reference projection Jacobian, colour as the median of
//                       exposure-corrected bilinear samples, opacity from the confidence;
//   voxel thinning      optional: one seed per cube (highest confidence, then lowest index).
#include <math.h>

#include <algorithm>

#include "rgs_internal.cuh"

namespace rgs {

namespace {

constexpr int kSeedThreads = 128;
constexpr int kMaxNb = 8;      // neighbours per reference pixel
constexpr int kJacobiSweeps = 16;

// Pixel of X in view v and its camera-space depth.
__device__ __forceinline__ void project_pt(const SeedCams& cams, int v, const double X[3],
                                           double& u, double& w, double xc[3]) {
  const double* R = cams.R[v];
  for (int a = 0; a < 3; ++a)
    xc[a] = R[3 * a] * X[0] + R[3 * a + 1] * X[1] + R[3 * a + 2] * X[2] + cams.t[v][a];
  u = cams.fx[v] * xc[0] / xc[2] + cams.cx[v];
  w = cams.fy[v] * xc[1] / xc[2] + cams.cy[v];
}

// Smallest right singular vector of the 4x4 matrix A (row-major), by one-sided Jacobi on its
// columns (Hestenes): plane rotations of column pairs until all pairs are orthogonal to working
// precision; the right singular vectors accumulate in V. At most kJacobiSweeps sweeps.
__device__ void smallest_right_singular_vector(double A[16], double out[4]) {
  double V[16];
  for (int k = 0; k < 16; ++k) V[k] = (k % 5 == 0) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    bool rotated = false;
    for (int p = 0; p < 3; ++p) {
      for (int q = p + 1; q < 4; ++q) {
        double alpha = 0.0, beta = 0.0, gamma = 0.0;
        for (int i = 0; i < 4; ++i) {
          const double ap = A[4 * i + p], aq = A[4 * i + q];
          alpha += ap * ap;
          beta += aq * aq;
          gamma += ap * aq;
        }
        if (gamma == 0.0 || fabs(gamma) <= 1e-15 * sqrt(alpha * beta)) continue;
        rotated = true;
        const double zeta = (beta - alpha) / (2.0 * gamma);
        const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = cs * tt;
        for (int i = 0; i < 4; ++i) {
          const double ap = A[4 * i + p], aq = A[4 * i + q];
          A[4 * i + p] = cs * ap - sn * aq;
          A[4 * i + q] = sn * ap + cs * aq;
          const double vp = V[4 * i + p], vq = V[4 * i + q];
          V[4 * i + p] = cs * vp - sn * vq;
          V[4 * i + q] = sn * vp + cs * vq;
        }
      }
    }
    if (!rotated) break;
  }
  int jmin = 0;
  double smin = 0.0;
  for (int j = 0; j < 4; ++j) {
    double s = 0.0;
    for (int i = 0; i < 4; ++i) s += A[4 * i + j] * A[4 * i + j];
    if (j == 0 || s < smin) {
      smin = s;
      jmin = j;
    }
  }
  for (int i = 0; i < 4; ++i) out[i] = V[4 * i + jmin];
}

__global__ void __launch_bounds__(kSeedThreads) triangulate_kernel(
    const __grid_constant__ SeedCams cams, const SeedConsts c, int64_t m, int k,
    const int32_t* __restrict__ ref_view, const double* __restrict__ ref_xy,
    const int32_t* __restrict__ nb_view, const double* __restrict__ nb_xy,
    const float* __restrict__ nb_conf, uint32_t* __restrict__ valid, double* __restrict__ X_out,
    int32_t* __restrict__ best_out, double* __restrict__ err_out,
    double* __restrict__ angle_out, float* __restrict__ kappa_out) {
  chain_wait();
  const int64_t i = (int64_t)blockIdx.x * kSeedThreads + threadIdx.x;
  if (i >= m) return;
  const int r = ref_view[i];
  if (r < 0 || r >= cams.n_views) {  // not a view of this batch: no hypothesis
    valid[i] = 0u;
    best_out[i] = -1;
    kappa_out[i] = 0.0f;
    return;
  }
  const double xr = ref_xy[2 * i], yr = ref_xy[2 * i + 1];
  double kap = 0.0;
  int n_match = 0;
  // Accepted hypotheses of this pixel (slot order).
  double h_err[kMaxNb], h_ang[kMaxNb], h_X[kMaxNb][3];
  bool h_ok[kMaxNb];
  double emin = 0.0;
  bool any = false;
  for (int s = 0; s < k; ++s) {
    h_ok[s] = false;
    const int n = nb_view[i * k + s];
    if (n < 0 || n >= cams.n_views) continue;
    kap += (double)nb_conf[i * k + s];
    ++n_match;
    const double xn = nb_xy[2 * (i * k + s)], yn = nb_xy[2 * (i * k + s) + 1];
    double A[16];
    const double* Pr = cams.P[r];
    const double* Pn = cams.P[n];
    for (int j = 0; j < 4; ++j) {
      A[j] = xr * Pr[8 + j] - Pr[j];
      A[4 + j] = yr * Pr[8 + j] - Pr[4 + j];
      A[8 + j] = xn * Pn[8 + j] - Pn[j];
      A[12 + j] = yn * Pn[8 + j] - Pn[4 + j];
    }
    double Xh[4];
    smallest_right_singular_vector(A, Xh);
    if (Xh[3] == 0.0) continue;
    const double X[3] = {Xh[0] / Xh[3], Xh[1] / Xh[3], Xh[2] / Xh[3]};
    double ur, wr, un, wn, cr[3], cn[3];
    project_pt(cams, r, X, ur, wr, cr);
    project_pt(cams, n, X, un, wn, cn);
    if (!(cr[2] > 0.0 && cn[2] > 0.0)) continue;
    const double err = sqrt(0.5 * ((ur - xr) * (ur - xr) + (wr - yr) * (wr - yr) +
                                   (un - xn) * (un - xn) + (wn - yn) * (wn - yn)));
    double d1[3], d2[3], dot = 0.0, n1 = 0.0, n2 = 0.0;
    for (int a = 0; a < 3; ++a) {
      d1[a] = X[a] - cams.c[r][a];
      d2[a] = X[a] - cams.c[n][a];
      dot += d1[a] * d2[a];
      n1 += d1[a] * d1[a];
      n2 += d2[a] * d2[a];
    }
    const double cosang = fmin(1.0, fmax(-1.0, dot / (sqrt(n1) * sqrt(n2))));
    const double ang = acos(cosang);
    if (ang < c.min_parallax || err > c.max_reproj) continue;
    h_ok[s] = true;
    h_err[s] = err;
    h_ang[s] = ang;
    h_X[s][0] = X[0];
    h_X[s][1] = X[1];
    h_X[s][2] = X[2];
    emin = any ? fmin(emin, err) : err;
    any = true;
  }
  // The lowest error wins; errors within tie_eps of the lowest are ties, decided by the larger
  // angle, then the earlier slot.
  bool found = false;
  double b_err = 0.0, b_ang = 0.0, bX[3] = {0.0, 0.0, 0.0};
  int b_k = -1;
  for (int s = 0; s < k; ++s) {
    if (!h_ok[s] || h_err[s] > emin + c.tie_eps) continue;
    if (!found || h_ang[s] > b_ang) {
      found = true;
      b_err = h_err[s];
      b_ang = h_ang[s];
      b_k = s;
      bX[0] = h_X[s][0];
      bX[1] = h_X[s][1];
      bX[2] = h_X[s][2];
    }
  }
  valid[i] = found ? 1u : 0u;
  X_out[3 * i] = bX[0];
  X_out[3 * i + 1] = bX[1];
  X_out[3 * i + 2] = bX[2];
  best_out[i] = b_k;
  err_out[i] = b_err;
  angle_out[i] = b_ang;
  kappa_out[i] = n_match ? (float)(kap / n_match) : 0.0f;
}

// Exact cell key of X for cubes of edge h: 21 bits per axis (offset 2^20, clamped).
__device__ __forceinline__ unsigned long long cell_key(const double X[3], double h) {
  unsigned long long key = 0;
  for (int a = 0; a < 3; ++a) {
    double f = floor(X[a] / h) + 1048576.0;
    f = fmin(fmax(f, 0.0), 2097151.0);
    key = (key << 21) | (unsigned long long)f;
  }
  return key;
}

// Entries to seed: valid, with a reference view of this batch.
__global__ void __launch_bounds__(kSeedThreads) seed_flags_kernel(
    int64_t m, int n_views, const uint32_t* __restrict__ valid,
    const int32_t* __restrict__ ref_view, uint32_t* __restrict__ flags) {
  chain_wait();
  const int64_t i = (int64_t)blockIdx.x * kSeedThreads + threadIdx.x;
  if (i < m) flags[i] = (valid[i] && ref_view[i] >= 0 && ref_view[i] < n_views) ? 1u : 0u;
}

__global__ void __launch_bounds__(kSeedThreads) compact_points_kernel(
    int64_t m, const uint32_t* __restrict__ valid, const uint32_t* __restrict__ pos,
    uint32_t* __restrict__ vidx) {
  chain_wait();
  const int64_t i = (int64_t)blockIdx.x * kSeedThreads + threadIdx.x;
  if (i < m && valid[i]) vidx[pos[i]] = (uint32_t)i;
}

// Cell keys of the accepted points: low and high 32-bit words, value = compact slot.
__global__ void __launch_bounds__(kSeedThreads) cell_keys_kernel(
    int s, const uint32_t* __restrict__ vidx, const double* __restrict__ X, double h,
    uint32_t* __restrict__ lo, uint32_t* __restrict__ hi, uint32_t* __restrict__ slot) {
  chain_wait();
  const int j = blockIdx.x * kSeedThreads + threadIdx.x;
  if (j >= s) return;
  const uint32_t i = vidx[j];
  const double P[3] = {X[3 * i], X[3 * i + 1], X[3 * i + 2]};
  const unsigned long long key = cell_key(P, h);
  lo[j] = (uint32_t)key;
  hi[j] = (uint32_t)(key >> 32);
  slot[j] = (uint32_t)j;
}

__global__ void __launch_bounds__(kSeedThreads) gather_u32_kernel(int s,
                                                                  const uint32_t* __restrict__ src,
                                                                  const uint32_t* __restrict__ perm,
                                                                  uint32_t* __restrict__ dst) {
  chain_wait();
  const int j = blockIdx.x * kSeedThreads + threadIdx.x;
  if (j < s) dst[j] = src[perm[j]];
}

// Sorted cell keys (64-bit) and points in sorted order.
__global__ void __launch_bounds__(kSeedThreads) sorted_cells_kernel(
    int s, const uint32_t* __restrict__ perm, const uint32_t* __restrict__ vidx,
    const double* __restrict__ X, double h, unsigned long long* __restrict__ skey,
    double* __restrict__ sX) {
  chain_wait();
  const int j = blockIdx.x * kSeedThreads + threadIdx.x;
  if (j >= s) return;
  const uint32_t i = vidx[perm[j]];
  const double P[3] = {X[3 * i], X[3 * i + 1], X[3 * i + 2]};
  skey[j] = cell_key(P, h);
  sX[3 * j] = P[0];
  sX[3 * j + 1] = P[1];
  sX[3 * j + 2] = P[2];
}

// Eigenvector of the smallest eigenvalue of the symmetric 3x3 matrix S (cyclic Jacobi).
__device__ void smallest_eigenvector3(double S[9], double v[3]) {
  double V[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    const double off = S[1] * S[1] + S[2] * S[2] + S[5] * S[5];
    const double diag = S[0] * S[0] + S[4] * S[4] + S[8] * S[8];
    if (off <= 1e-30 * diag || off == 0.0) break;
    for (int p = 0; p < 2; ++p) {
      for (int q = p + 1; q < 3; ++q) {
        const double apq = S[3 * p + q];
        if (apq == 0.0) continue;
        const double theta = (S[3 * q + q] - S[3 * p + p]) / (2.0 * apq);
        const double tt = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double cs = 1.0 / sqrt(tt * tt + 1.0), sn = tt * cs;
        // S <- J^T S J with J the rotation in the (p, q) plane.
        for (int kk = 0; kk < 3; ++kk) {
          const double skp = S[3 * kk + p], skq = S[3 * kk + q];
          S[3 * kk + p] = cs * skp - sn * skq;
          S[3 * kk + q] = sn * skp + cs * skq;
        }
        for (int kk = 0; kk < 3; ++kk) {
          const double spk = S[3 * p + kk], sqk = S[3 * q + kk];
          S[3 * p + kk] = cs * spk - sn * sqk;
          S[3 * q + kk] = sn * spk + cs * sqk;
        }
        for (int kk = 0; kk < 3; ++kk) {
          const double vkp = V[3 * kk + p], vkq = V[3 * kk + q];
          V[3 * kk + p] = cs * vkp - sn * vkq;
          V[3 * kk + q] = sn * vkp + cs * vkq;
        }
      }
    }
  }
  int j = 0;
  if (S[4] < S[3 * j + j]) j = 1;
  if (S[8] < S[3 * j + j]) j = 2;
  for (int a = 0; a < 3; ++a) v[a] = V[3 * a + j];
}

__device__ __forceinline__ int lower_bound_key(const unsigned long long* __restrict__ keys, int s,
                                               unsigned long long key) {
  int lo = 0, hi = s;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (keys[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Bilinear sample of view v at (x, y) (pixel (i, j) at (i, j)); false if the 2x2 footprint
// leaves the image.
__device__ __forceinline__ bool bilinear(const SeedCams& cams, const float* __restrict__ obs,
                                         int v, double x, double y, double out[3]) {
  const double fx0 = floor(x), fy0 = floor(y);
  const int W = cams.width[v], H = cams.height[v];
  if (!(fx0 >= 0.0 && fy0 >= 0.0 && fx0 + 1.0 <= W - 1 && fy0 + 1.0 <= H - 1)) return false;
  const int x0 = (int)fx0, y0 = (int)fy0;
  const double ax = x - fx0, ay = y - fy0;
  const float* base = obs + 3 * (cams.pixel_offset[v] + (long long)y0 * W + x0);
  for (int ch = 0; ch < 3; ++ch) {
    const double p00 = base[ch], p01 = base[3 + ch];
    const double p10 = base[3 * W + ch], p11 = base[3 * W + 3 + ch];
    out[ch] = (1 - ax) * (1 - ay) * p00 + ax * (1 - ay) * p01 + (1 - ax) * ay * p10 +
              ax * ay * p11;
  }
  return true;
}

__device__ __forceinline__ double median_of(double* a, int n) {
  for (int i = 1; i < n; ++i) {  // insertion sort of at most kMaxNb + 1 values
    const double x = a[i];
    int j = i - 1;
    while (j >= 0 && a[j] > x) {
      a[j + 1] = a[j];
      --j;
    }
    a[j + 1] = x;
  }
  return (n & 1) ? a[n / 2] : 0.5 * (a[n / 2 - 1] + a[n / 2]);
}

// Per accepted point j (compact order): the seed's parameters.
__global__ void __launch_bounds__(kSeedThreads) seed_kernel(
    const __grid_constant__ SeedCams cams, const SeedConsts c, int s, int k, int sh_k,
    const uint32_t* __restrict__ vidx, const int32_t* __restrict__ ref_view,
    const int32_t* __restrict__ nb_view, const double* __restrict__ X_all,
    const double* __restrict__ err_all, const double* __restrict__ ang_all,
    const float* __restrict__ kappa_all, const unsigned long long* __restrict__ skey,
    const double* __restrict__ sX, const float* __restrict__ obs,
    const float* __restrict__ gain_bias, float* __restrict__ means, float* __restrict__ log_scales,
    float* __restrict__ quats, float* __restrict__ logits, float* __restrict__ sh,
    float* __restrict__ normals) {
  chain_wait();
  const int j = blockIdx.x * kSeedThreads + threadIdx.x;
  if (j >= s) return;
  const uint32_t i = vidx[j];
  const double X[3] = {X_all[3 * i], X_all[3 * i + 1], X_all[3 * i + 2]};
  const int r = ref_view[i];
  // Plane fit over the accepted points within the radius (moments about X).
  const double h = c.plane_radius, h2 = h * h;
  const unsigned long long ck = cell_key(X, h);
  double cnt = 0.0, m1[3] = {0, 0, 0}, m2[6] = {0, 0, 0, 0, 0, 0};
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const long long a0 = (long long)((ck >> 42) & 0x1FFFFF) + dx;
        const long long a1 = (long long)((ck >> 21) & 0x1FFFFF) + dy;
        const long long a2 = (long long)(ck & 0x1FFFFF) + dz;
        if (a0 < 0 || a1 < 0 || a2 < 0 || a0 > 0x1FFFFF || a1 > 0x1FFFFF || a2 > 0x1FFFFF)
          continue;
        const unsigned long long key = ((unsigned long long)a0 << 42) |
                                       ((unsigned long long)a1 << 21) | (unsigned long long)a2;
        for (int q = lower_bound_key(skey, s, key); q < s && skey[q] == key; ++q) {
          const double d0 = sX[3 * q] - X[0], d1 = sX[3 * q + 1] - X[1], d2 = sX[3 * q + 2] - X[2];
          if (d0 * d0 + d1 * d1 + d2 * d2 > h2) continue;
          cnt += 1.0;
          m1[0] += d0;
          m1[1] += d1;
          m1[2] += d2;
          m2[0] += d0 * d0;
          m2[1] += d0 * d1;
          m2[2] += d0 * d2;
          m2[3] += d1 * d1;
          m2[4] += d1 * d2;
          m2[5] += d2 * d2;
        }
      }
  const double* cr = cams.c[r];
  double toc[3] = {cr[0] - X[0], cr[1] - X[1], cr[2] - X[2]};
  const double tn = sqrt(toc[0] * toc[0] + toc[1] * toc[1] + toc[2] * toc[2]);
  double v[3];
  if (cnt >= 3.0) {
    const double mu[3] = {m1[0] / cnt, m1[1] / cnt, m1[2] / cnt};
    double S[9];
    S[0] = m2[0] / cnt - mu[0] * mu[0];
    S[1] = S[3] = m2[1] / cnt - mu[0] * mu[1];
    S[2] = S[6] = m2[2] / cnt - mu[0] * mu[2];
    S[4] = m2[3] / cnt - mu[1] * mu[1];
    S[5] = S[7] = m2[4] / cnt - mu[1] * mu[2];
    S[8] = m2[5] / cnt - mu[2] * mu[2];
    smallest_eigenvector3(S, v);
    const double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int a = 0; a < 3; ++a) v[a] /= nv;
    if (v[0] * toc[0] + v[1] * toc[1] + v[2] * toc[2] < 0.0)
      for (int a = 0; a < 3; ++a) v[a] = -v[a];
  } else {
    for (int a = 0; a < 3; ++a) v[a] = toc[a] / tn;
  }
  // Tangent frame (Duff et al., JCGT 2017): [t1, t2, v] is a rotation.
  const double sg = v[2] >= 0.0 ? 1.0 : -1.0;
  const double aa = -1.0 / (sg + v[2]);
  const double bb = v[0] * v[1] * aa;
  const double t1[3] = {1.0 + sg * v[0] * v[0] * aa, sg * bb, -sg * v[0]};
  const double t2[3] = {bb, sg + v[1] * v[1] * aa, -v[1]};
  const double U[9] = {t1[0], t2[0], v[0], t1[1], t2[1], v[1], t1[2], t2[2], v[2]};
  // Quaternion (w, x, y, z), w >= 0 (Shepperd's branches).
  double q[4];
  const double tr = U[0] + U[4] + U[8];
  if (tr > 0.0) {
    const double sq = sqrt(tr + 1.0) * 2.0;
    q[0] = 0.25 * sq;
    q[1] = (U[7] - U[5]) / sq;
    q[2] = (U[2] - U[6]) / sq;
    q[3] = (U[3] - U[1]) / sq;
  } else if (U[0] > U[4] && U[0] > U[8]) {
    const double sq = sqrt(1.0 + U[0] - U[4] - U[8]) * 2.0;
    q[0] = (U[7] - U[5]) / sq;
    q[1] = 0.25 * sq;
    q[2] = (U[1] + U[3]) / sq;
    q[3] = (U[2] + U[6]) / sq;
  } else if (U[4] > U[8]) {
    const double sq = sqrt(1.0 + U[4] - U[0] - U[8]) * 2.0;
    q[0] = (U[2] - U[6]) / sq;
    q[1] = (U[1] + U[3]) / sq;
    q[2] = 0.25 * sq;
    q[3] = (U[5] + U[7]) / sq;
  } else {
    const double sq = sqrt(1.0 + U[8] - U[0] - U[4]) * 2.0;
    q[0] = (U[3] - U[1]) / sq;
    q[1] = (U[2] + U[6]) / sq;
    q[2] = (U[5] + U[7]) / sq;
    q[3] = 0.25 * sq;
  }
  const double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const double qs = (q[0] >= 0.0 ? 1.0 : -1.0) / qn;
  // Scales: s_perp from the reference projection Jacobian, s_par from angle and error.
  double ur, wr, xc[3];
  project_pt(cams, r, X, ur, wr, xc);
  const double z = xc[2];
  const double* R = cams.R[r];
  double Jc[6];
  for (int b = 0; b < 3; ++b) {
    const double j0 = cams.fx[r] / z, j2 = -cams.fx[r] * xc[0] / (z * z);
    const double k1 = cams.fy[r] / z, k2 = -cams.fy[r] * xc[1] / (z * z);
    Jc[b] = j0 * R[b] + j2 * R[6 + b];
    Jc[3 + b] = k1 * R[3 + b] + k2 * R[6 + b];
  }
  const double g00 = Jc[0] * Jc[0] + Jc[1] * Jc[1] + Jc[2] * Jc[2];
  const double g01 = Jc[0] * Jc[3] + Jc[1] * Jc[4] + Jc[2] * Jc[5];
  const double g11 = Jc[3] * Jc[3] + Jc[4] * Jc[4] + Jc[5] * Jc[5];
  const double s_perp = pow(g00 * g11 - g01 * g01, -0.25);
  const double s_par = fmin(s_perp * (1.0 + err_all[i]) / sin(ang_all[i]), c.s_par_cap * s_perp);
  // Colour: median over the supporting views of the exposure-corrected bilinear samples.
  double smp[3][kMaxNb + 1];
  int ns = 0;
  for (int s2 = -1; s2 < k; ++s2) {
    const int vv = s2 < 0 ? r : nb_view[(size_t)i * k + s2];
    if (vv < 0 || vv >= cams.n_views) continue;
    double u, w, xcv[3], col[3];
    project_pt(cams, vv, X, u, w, xcv);
    if (!(xcv[2] > 0.0) || !bilinear(cams, obs, vv, u, w, col)) continue;
    const double g = gain_bias[2 * vv], b = gain_bias[2 * vv + 1];
    for (int ch = 0; ch < 3; ++ch) smp[ch][ns] = (col[ch] - b) / g;
    ++ns;
  }
  double colr[3] = {0.5, 0.5, 0.5};
  if (ns > 0)
    for (int ch = 0; ch < 3; ++ch) colr[ch] = median_of(smp[ch], ns);
  const double alpha = c.alpha_lo + (c.alpha_hi - c.alpha_lo) * (double)kappa_all[i];
  const double Y0 = 0.28209479177387814;
  for (int a = 0; a < 3; ++a) {
    means[3 * j + a] = (float)X[a];
    normals[3 * j + a] = (float)v[a];
  }
  log_scales[3 * j] = (float)log(s_perp);
  log_scales[3 * j + 1] = (float)log(s_perp);
  log_scales[3 * j + 2] = (float)log(s_par);
  for (int a = 0; a < 4; ++a) quats[4 * j + a] = (float)(q[a] * qs);
  logits[j] = (float)log(alpha / (1.0 - alpha));
  for (int b = 0; b < sh_k; ++b)
    for (int ch = 0; ch < 3; ++ch)
      sh[((size_t)j * sh_k + b) * 3 + ch] = b == 0 ? (float)((colr[ch] - 0.5) / Y0) : 0.0f;
}

// Voxel thinning: after sorting by voxel key, the first entry of each run picks the run's best
// seed (highest confidence as float, then lowest reference index) and marks it kept.
__global__ void __launch_bounds__(kSeedThreads) voxel_best_kernel(
    int s, const unsigned long long* __restrict__ skey, const uint32_t* __restrict__ perm,
    const uint32_t* __restrict__ vidx, const float* __restrict__ kappa_all,
    uint32_t* __restrict__ keep) {
  chain_wait();
  const int j = blockIdx.x * kSeedThreads + threadIdx.x;
  if (j >= s || (j > 0 && skey[j - 1] == skey[j])) return;
  int best = perm[j];
  for (int q = j + 1; q < s && skey[q] == skey[j]; ++q) {
    const int cand = perm[q];
    const float kc = kappa_all[vidx[cand]], kb = kappa_all[vidx[best]];
    if (kc > kb || (kc == kb && vidx[cand] < vidx[best])) best = cand;
  }
  keep[best] = 1u;
}

__global__ void __launch_bounds__(kSeedThreads) scatter_seeds_kernel(
    int s, int sh_k, const uint32_t* __restrict__ keep, const uint32_t* __restrict__ pos,
    const uint32_t* __restrict__ vidx, const float* __restrict__ means,
    const float* __restrict__ log_scales, const float* __restrict__ quats,
    const float* __restrict__ logits, const float* __restrict__ sh,
    const float* __restrict__ normals, int32_t* __restrict__ o_index, float* __restrict__ o_means,
    float* __restrict__ o_log_scales, float* __restrict__ o_quats, float* __restrict__ o_logits,
    float* __restrict__ o_sh, float* __restrict__ o_normals) {
  chain_wait();
  const int j = blockIdx.x * kSeedThreads + threadIdx.x;
  if (j >= s || !keep[j]) return;
  const uint32_t o = pos[j];
  o_index[o] = (int32_t)vidx[j];
  for (int a = 0; a < 3; ++a) {
    o_means[3 * o + a] = means[3 * j + a];
    o_log_scales[3 * o + a] = log_scales[3 * j + a];
    o_normals[3 * o + a] = normals[3 * j + a];
  }
  for (int a = 0; a < 4; ++a) o_quats[4 * o + a] = quats[4 * j + a];
  o_logits[o] = logits[j];
  for (int b = 0; b < 3 * sh_k; ++b) o_sh[(size_t)3 * sh_k * o + b] = sh[(size_t)3 * sh_k * j + b];
}

__global__ void fill_u32_kernel(int s, uint32_t value, uint32_t* __restrict__ out) {
  chain_wait();
  const int j = blockIdx.x * kSeedThreads + threadIdx.x;
  if (j < s) out[j] = value;
}

unsigned blocks_for(int64_t n) { return (unsigned)((n + kSeedThreads - 1) / kSeedThreads); }

}  // namespace

cudaError_t launch_triangulate(const SeedCams& cams, const SeedConsts& c, int64_t m, int k,
                               const int32_t* ref_view, const double* ref_xy,
                               const int32_t* nb_view, const double* nb_xy, const float* nb_conf,
                               uint32_t* valid, double* X, int32_t* best, double* err,
                               double* angle, float* kappa, cudaStream_t stream) {
  if (m == 0) return cudaSuccess;
  const cudaError_t e = launch_chained(triangulate_kernel, dim3(blocks_for(m)),
                                       dim3(kSeedThreads), stream, cams, c, m, k, ref_view,
                                       ref_xy, nb_view, nb_xy, nb_conf, valid, X, best, err,
                                       angle, kappa);
  RGS_LAUNCHED();
  return e;
}

// Stable sort of s 63-bit keys (lo, hi words) carrying the compact slots: returns the
// permutation in perm (lo sort, then a stable sort by hi of the gathered high words).
cudaError_t sort_keys64(int s, uint32_t* lo, uint32_t* hi, uint32_t* slot, uint32_t* t0,
                        uint32_t* t1, uint32_t* hist, uint32_t* block_sums, uint32_t** perm,
                        cudaStream_t stream) {
  bool alt = false;
  cudaError_t e = launch_radix_sort(lo, slot, t0, t1, s, nullptr, 0, 32, hist, block_sums, &alt,
                                    stream);
  if (e != cudaSuccess) return e;
  uint32_t* p1 = alt ? t1 : slot;
  uint32_t* spare = alt ? slot : t1;
  // High words in the order of p1.
  uint32_t* hig = alt ? lo : t0;  // the buffer not holding p1's keys
  e = launch_chained(gather_u32_kernel, dim3(blocks_for(s)), dim3(kSeedThreads), stream, s,
                     (const uint32_t*)hi, (const uint32_t*)p1, hig);
  RGS_LAUNCHED();
  if (e != cudaSuccess) return e;
  uint32_t* hig_alt = hi;  // free now
  e = launch_radix_sort(hig, p1, hig_alt, spare, s, nullptr, 0, 31, hist, block_sums, &alt,
                        stream);
  *perm = alt ? spare : p1;
  return e;
}

cudaError_t launch_seed_points(const SeedCams& cams, const SeedConsts& c, int s, int k, int sh_k,
                               const uint32_t* vidx, const int32_t* ref_view,
                               const int32_t* nb_view, const double* X, const double* err,
                               const double* angle, const float* kappa, const float* obs,
                               const float* gain_bias, uint32_t* lo, uint32_t* hi,
                               uint32_t* slot, uint32_t* t0, uint32_t* t1, uint32_t* hist,
                               uint32_t* block_sums, unsigned long long* skey, double* sX,
                               float* means, float* log_scales, float* quats, float* logits,
                               float* sh, float* normals, uint32_t* keep, cudaStream_t stream) {
  if (s == 0) return cudaSuccess;
  const dim3 grid(blocks_for(s)), block(kSeedThreads);
  cudaError_t e = launch_chained(cell_keys_kernel, grid, block, stream, s, vidx, X,
                                 c.plane_radius, lo, hi, slot);
  RGS_LAUNCHED();
  uint32_t* perm = nullptr;
  if (e == cudaSuccess) e = sort_keys64(s, lo, hi, slot, t0, t1, hist, block_sums, &perm, stream);
  if (e == cudaSuccess) {
    e = launch_chained(sorted_cells_kernel, grid, block, stream, s, (const uint32_t*)perm, vidx,
                       X, c.plane_radius, skey, sX);
    RGS_LAUNCHED();
  }
  if (e == cudaSuccess) {
    e = launch_chained(seed_kernel, grid, block, stream, cams, c, s, k, sh_k, vidx, ref_view,
                       nb_view, X, err, angle, kappa, (const unsigned long long*)skey,
                       (const double*)sX, obs, gain_bias, means, log_scales, quats, logits, sh,
                       normals);
    RGS_LAUNCHED();
  }
  if (e != cudaSuccess) return e;
  if (c.voxel > 0.0) {
    e = launch_chained(fill_u32_kernel, grid, block, stream, s, 0u, keep);
    RGS_LAUNCHED();
    if (e == cudaSuccess) {
      e = launch_chained(cell_keys_kernel, grid, block, stream, s, vidx, X, c.voxel, lo, hi,
                         slot);
      RGS_LAUNCHED();
    }
    if (e == cudaSuccess) e = sort_keys64(s, lo, hi, slot, t0, t1, hist, block_sums, &perm, stream);
    if (e == cudaSuccess) {
      e = launch_chained(sorted_cells_kernel, grid, block, stream, s, (const uint32_t*)perm, vidx,
                         X, c.voxel, skey, sX);
      RGS_LAUNCHED();
    }
    if (e == cudaSuccess) {
      e = launch_chained(voxel_best_kernel, grid, block, stream, s,
                         (const unsigned long long*)skey, (const uint32_t*)perm, vidx, kappa,
                         keep);
      RGS_LAUNCHED();
    }
  } else {
    e = launch_chained(fill_u32_kernel, grid, block, stream, s, 1u, keep);
    RGS_LAUNCHED();
  }
  return e;
}

cudaError_t launch_seed_flags(int64_t m, int n_views, const uint32_t* valid,
                              const int32_t* ref_view, uint32_t* flags, cudaStream_t stream) {
  if (m == 0) return cudaSuccess;
  const cudaError_t e = launch_chained(seed_flags_kernel, dim3(blocks_for(m)), dim3(kSeedThreads),
                                       stream, m, n_views, valid, ref_view, flags);
  RGS_LAUNCHED();
  return e;
}

cudaError_t launch_compact_points(int64_t m, const uint32_t* valid, const uint32_t* pos,
                                  uint32_t* vidx, cudaStream_t stream) {
  if (m == 0) return cudaSuccess;
  const cudaError_t e = launch_chained(compact_points_kernel, dim3(blocks_for(m)),
                                       dim3(kSeedThreads), stream, m, valid, pos, vidx);
  RGS_LAUNCHED();
  return e;
}

cudaError_t launch_scatter_seeds(int s, int sh_k, const uint32_t* keep, const uint32_t* pos,
                                 const uint32_t* vidx, const float* means,
                                 const float* log_scales, const float* quats,
                                 const float* logits, const float* sh, const float* normals,
                                 int32_t* o_index, float* o_means, float* o_log_scales,
                                 float* o_quats, float* o_logits, float* o_sh, float* o_normals,
                                 cudaStream_t stream) {
  if (s == 0) return cudaSuccess;
  const cudaError_t e = launch_chained(scatter_seeds_kernel, dim3(blocks_for(s)),
                                       dim3(kSeedThreads), stream, s, sh_k, keep, pos, vidx,
                                       means, log_scales, quats, logits, sh, normals, o_index,
                                       o_means, o_log_scales, o_quats, o_logits, o_sh, o_normals);
  RGS_LAUNCHED();
  return e;
}

}  // namespace rgs
