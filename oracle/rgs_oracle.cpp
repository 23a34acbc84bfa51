/*
 * rgs_oracle.cpp -- plain FP64 CPU oracle of the differentiable Gaussian-splatting rasterizer.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link, import or run this file:
 * only the test suite, the smoke check and the benchmark's CPU-baseline leg use it. It shares no
 * code, header, table or helper with the CUDA library.
 *
 * What it computes (all arithmetic in double precision from the FP32 inputs):
 *   - Section 3.1, Eq. proj: mu^I = pi(R mu^W + t), Sigma^I = J R Sigma^W R^T J^T with J the
 *     Jacobian of the pinhole projection at the camera-space mean.
 *   - Appendix C.1: Sigma^W = R_q diag(s^2) R_q^T, unit quaternion q, s = exp(log-scale); colour
 *     from real spherical harmonics of the viewing direction (Eq. app-sh).
 *   - Section 3.1, Eq. alpha: front-to-back alpha compositing of the Gaussians that cover a pixel,
 *     sorted near to far (Section 3.2.2).
 *   - Gradients of colour, depth and accumulated opacity with respect to every Gaussian parameter
 *     and the camera twist xi of the left update T <- exp(xi^) T (Eq. leftupdate), using
 *     d mu^C / d xi = [I, -[mu^C]_x] (Eq. muCjac), d mu^I / d xi = J_pi [I, -[mu^C]_x] (Eq. muIjac)
 *     and the rotation path of Sigma^I with dR = [d omega]_x R (Eq. sigmaIjac).
 *
 * The paper leaves the following open; the readings used here are:
 *   - a Gaussian covers pixel p iff alpha = min(alpha_max, o G(p)) >= alpha_min (1/255); the
 *     compositing stops before the first Gaussian whose inclusion would drop T below t_min (1e-4);
 *   - pixel (x, y) is sampled at image coordinates (x, y);
 *   - near-to-far order is by camera-space depth z of the Gaussian centre rounded to float32
 *     (the precision of the renderer's sort key), ties by input index;
 *   - Sigma^I gets a low-pass dilation eps2d * I before inversion; J uses x/z, y/z clamped to
 *     +-jac_clamp * (W/2)/fx, +-jac_clamp * (H/2)/fy (no gradient through a clamped component);
 *   - Gaussians with z <= znear, non-finite inputs or det(Sigma^I) <= 0 are culled;
 *   - colour = max(sum_k sh_k Y_k(d) + 0.5, 0), d = normalize(mu^W - c_W), c_W = -R^T t (world frame);
 *   - depth D = sum_i w_i z_i (no background), accumulated opacity A = 1 - T_final, background
 *     colour added as bg * T_final;
 *   - opacity o = sigmoid(opacity logit).
 *
 * Method: per pixel, every Gaussian of the view is a candidate (a padded per-Gaussian bounding box
 * of the alpha >= alpha_min ellipse may be used to skip far-away ones; it never changes a result);
 * the covering set is sorted by (z, index) and composited. The backward pass keeps each pixel's
 * list and uses explicit prefix products T_j = prod_{k<j}(1 - alpha_k) and suffix sums, then
 * chains the per-(view, Gaussian) screen-space gradients through the projection by hand-derived
 * adjoints.
 *
 * Ambiguity flags: where an FP32 implementation may legitimately take the other side of a
 * discrete decision (alpha vs alpha_min / alpha_max, T vs t_min, depth ties, z vs znear, the
 * Jacobian clamp, the colour clamp), the pixel is flagged so that parity tests can leave it out.
 */
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>
#include <limits>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {

constexpr double kPi = 3.14159265358979323846;

struct Config {
  double alpha_min, alpha_max, t_min, znear, eps2d, jac_clamp;
  double bg[3];
  double margin_alpha;  // relative margin around alpha_min and alpha_max
  double margin_t;      // relative margin around t_min
  double margin_z;      // relative slack of this oracle's own depth rounding (see gaussian_forward)
  double margin_g;      // relative margin for per-Gaussian branch points (znear, clamps)
  double margin_effect; // smallest image change a flipped alpha_min decision must be able to
                        // cause for the pixel to be flagged
  double margin_cont;   // largest float32 error bound of a pixel's colour tolerated unflagged
};

struct Camera {
  int width, height;
  double fx, fy, cx, cy;
  double R[3][3];
  double t[3];
};

// Pixel ambiguity bits. 1, 4, 8 and 16 mark decisions whose other outcome changes the image by
// more than margin_effect; 2 and 32 mark kinks that only change gradients.
enum AmbiguityBits {
  kAmbAlphaMin = 1,     // a covering test alpha >= alpha_min within margin_alpha
  kAmbAlphaMax = 2,     // the alpha clamp at alpha_max within margin_alpha (gradient kink)
  kAmbTMin = 4,         // the stop test T' < t_min within margin_t
  kAmbDepthTie = 8,     // a depth key that may round either way next to another key of the list
  kAmbNear = 16,        // a covering Gaussian's depth within margin_g of znear (cull decision)
  kAmbGradKink = 32,    // a covering Gaussian at the Jacobian clamp or colour clamp (gradient kink)
  kAmbCond = 64,        // the float32 evaluation error bound of the pixel exceeds margin_cont
};

// Unit roundoff of float32. The float32 renderer this oracle is compared with evaluates the
// exponent in whitened coordinates: with L L^T = (log2(e) / 2) Q (lower-triangular L, Q the conic),
// log2(o G) = log2 o - (t^2 + s^2), (t, s) = L^T d, where t and s are formed from the products
// l11 dx, l21 dy, l22 dy (dy measured from a tile row at most 8 px away, then moved to the pixel's
// row). Its error is a few units of the roundoff times (|t| + |s|) times the magnitude of those
// products, plus the error of the conic itself. Sigma^I = A A^T + eps I with A = J R M
// (M = R_q diag(s)): rounding J, R, R_q and the scales perturbs A by about the roundoff times
// |J| s_max (the size A would have if the longest axis were not foreshortened), which moves
// ln G by at most 2 |ln G| |dA| / sqrt(lambda_min(Sigma^I)); the oracle carries
// amp = sqrt(max(|J|_F^2 s_max^2, lambda_max) / lambda_min) per (view, Gaussian). It uses this bound,
// with a safety factor of 8, to widen its decision margins and to flag pixels whose float32
// value cannot be expected within the tolerance.
constexpr double kUnitRoundoff32 = 5.9604644775390625e-08;

// ---------------------------------------------------------------------------------------------
// Real spherical harmonics, degree <= 3 (Appendix C.1, Eq. app-sh).
// Basis index k = l*l + l + m, m = -l..l. Y_{l,m} = sqrt(2) Re Y_l^m for m > 0,
// sqrt(2) Im Y_l^{|m|} for m < 0 and Y_l^0 for m = 0, where Y_l^m is the complex harmonic with
// the Condon-Shortley phase. Written out as polynomials of the unit direction (x, y, z), together
// with their gradients with respect to (x, y, z).
// ---------------------------------------------------------------------------------------------
void sh_basis(int degree, const double d[3], double Y[16], double dY[16][3]) {
  const double x = d[0], y = d[1], z = d[2];
  for (int k = 0; k < 16; ++k) {
    Y[k] = 0.0;
    dY[k][0] = dY[k][1] = dY[k][2] = 0.0;
  }
  const double k0 = 0.5 / std::sqrt(kPi);
  Y[0] = k0;
  if (degree < 1) return;
  const double k1 = std::sqrt(3.0 / (4.0 * kPi));
  Y[1] = -k1 * y;  dY[1][1] = -k1;
  Y[2] = k1 * z;   dY[2][2] = k1;
  Y[3] = -k1 * x;  dY[3][0] = -k1;
  if (degree < 2) return;
  const double k2a = 0.5 * std::sqrt(15.0 / kPi);
  const double k2b = 0.25 * std::sqrt(5.0 / kPi);
  const double k2c = 0.25 * std::sqrt(15.0 / kPi);
  Y[4] = k2a * x * y;
  dY[4][0] = k2a * y; dY[4][1] = k2a * x;
  Y[5] = -k2a * y * z;
  dY[5][1] = -k2a * z; dY[5][2] = -k2a * y;
  Y[6] = k2b * (2.0 * z * z - x * x - y * y);
  dY[6][0] = -2.0 * k2b * x; dY[6][1] = -2.0 * k2b * y; dY[6][2] = 4.0 * k2b * z;
  Y[7] = -k2a * x * z;
  dY[7][0] = -k2a * z; dY[7][2] = -k2a * x;
  Y[8] = k2c * (x * x - y * y);
  dY[8][0] = 2.0 * k2c * x; dY[8][1] = -2.0 * k2c * y;
  if (degree < 3) return;
  const double c30 = 0.25 * std::sqrt(35.0 / (2.0 * kPi));
  const double c31 = 0.5 * std::sqrt(105.0 / kPi);
  const double c32 = 0.25 * std::sqrt(21.0 / (2.0 * kPi));
  const double c33 = 0.25 * std::sqrt(7.0 / kPi);
  const double c35 = 0.25 * std::sqrt(105.0 / kPi);
  Y[9] = -c30 * y * (3.0 * x * x - y * y);
  dY[9][0] = -c30 * 6.0 * x * y; dY[9][1] = -c30 * (3.0 * x * x - 3.0 * y * y);
  Y[10] = c31 * x * y * z;
  dY[10][0] = c31 * y * z; dY[10][1] = c31 * x * z; dY[10][2] = c31 * x * y;
  Y[11] = -c32 * y * (4.0 * z * z - x * x - y * y);
  dY[11][0] = -c32 * (-2.0 * x * y);
  dY[11][1] = -c32 * (4.0 * z * z - x * x - 3.0 * y * y);
  dY[11][2] = -c32 * (8.0 * y * z);
  Y[12] = c33 * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
  dY[12][0] = c33 * (-6.0 * x * z); dY[12][1] = c33 * (-6.0 * y * z);
  dY[12][2] = c33 * (6.0 * z * z - 3.0 * x * x - 3.0 * y * y);
  Y[13] = -c32 * x * (4.0 * z * z - x * x - y * y);
  dY[13][0] = -c32 * (4.0 * z * z - 3.0 * x * x - y * y);
  dY[13][1] = -c32 * (-2.0 * x * y);
  dY[13][2] = -c32 * (8.0 * x * z);
  Y[14] = c35 * z * (x * x - y * y);
  dY[14][0] = c35 * 2.0 * x * z; dY[14][1] = -c35 * 2.0 * y * z; dY[14][2] = c35 * (x * x - y * y);
  Y[15] = -c30 * x * (x * x - 3.0 * y * y);
  dY[15][0] = -c30 * (3.0 * x * x - 3.0 * y * y); dY[15][1] = -c30 * (-6.0 * x * y);
}

// Rotation matrix of a unit quaternion (w, x, y, z); Appendix C.1 keeps rotations as quaternions.
void quat_to_rotmat(const double q[4], double R[3][3]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0][0] = 1.0 - 2.0 * (y * y + z * z);
  R[0][1] = 2.0 * (x * y - w * z);
  R[0][2] = 2.0 * (x * z + w * y);
  R[1][0] = 2.0 * (x * y + w * z);
  R[1][1] = 1.0 - 2.0 * (x * x + z * z);
  R[1][2] = 2.0 * (y * z - w * x);
  R[2][0] = 2.0 * (x * z - w * y);
  R[2][1] = 2.0 * (y * z + w * x);
  R[2][2] = 1.0 - 2.0 * (x * x + y * y);
}

// Gradient with respect to the unit quaternion of <G, R(q)>, each entry of R differentiated by hand.
void quat_to_rotmat_vjp(const double q[4], const double G[3][3], double g[4]) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  // dR_ab/dq for each entry, in the order (w, x, y, z).
  const double d[3][3][4] = {
      {{0, 0, -4 * y, -4 * z}, {-2 * z, 2 * y, 2 * x, -2 * w}, {2 * y, 2 * z, 2 * w, 2 * x}},
      {{2 * z, 2 * y, 2 * x, 2 * w}, {0, -4 * x, 0, -4 * z}, {-2 * x, -2 * w, 2 * z, 2 * y}},
      {{-2 * y, 2 * z, -2 * w, 2 * x}, {2 * x, 2 * w, 2 * z, 2 * y}, {0, -4 * x, -4 * y, 0}},
  };
  for (int c = 0; c < 4; ++c) {
    double s = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) s += G[a][b] * d[a][b][c];
    g[c] = s;
  }
}

bool all_finite(const double* v, int n) {
  for (int k = 0; k < n; ++k)
    if (!std::isfinite(v[k])) return false;
  return true;
}

// Everything the forward computes for one (view, Gaussian); the backward re-derives it.
struct GaussFwd {
  bool valid = false;
  int flags = 0;  // near a branch point: 1 znear, 2 Jacobian clamp, 4 colour clamp, 8 depth key
  double q_raw_norm, qn[4], Rq[3][3], s[3], M[3][3], SigW[3][3];
  double mu_c[3], z, u, w, uc, wc;
  float zkey;  // z rounded to float32: the near-to-far sort key
  bool u_clamped, w_clamped;
  double J[2][3], T[2][3], cov2d[2][2], det, conic[3];  // conic = (a, b, c)
  double mean2d[2];
  double opacity;
  double cam_center[3], dvec[3], dnorm, dir[3];
  double Y[16], dY[16][3];
  double rgb_raw[3], rgb[3];
  double kappa;  // dimensionless radius^2 of the alpha >= alpha_min ellipse: 2 ln(o / alpha_min)
};

void gaussian_forward(const double* mean, const double* log_scale, const double* quat, double logit,
                      const double* sh, int degree, const Camera& cam, const Config& cfg,
                      GaussFwd& f) {
  f = GaussFwd();
  const int K = (degree + 1) * (degree + 1);
  if (!all_finite(mean, 3) || !all_finite(log_scale, 3) || !all_finite(quat, 4) ||
      !std::isfinite(logit) || !all_finite(sh, 3 * K))
    return;
  // Camera-space mean, mu^C = R mu^W + t (Section 3.2.3).
  for (int a = 0; a < 3; ++a)
    f.mu_c[a] = cam.R[a][0] * mean[0] + cam.R[a][1] * mean[1] + cam.R[a][2] * mean[2] + cam.t[a];
  f.z = f.mu_c[2];
  if (std::fabs(f.z - cfg.znear) <= cfg.margin_g * cfg.znear) f.flags |= 1;
  if (!(f.z > cfg.znear)) return;
  // Near-to-far order compares depths rounded to float32 (the renderer's key precision). A
  // renderer that evaluates the depth as a compensated dot product (twice the working precision)
  // gets the correctly rounded value unless the exact depth lies within that product's error,
  // about 16 u32^2 (|R_2 . mu^W| summed termwise + |t_2|), of the midpoint between two float32
  // values; such a depth is marked here (plus margin_z * z for this oracle's own rounding), and
  // a pixel is flagged only if another Gaussian of its list has a key within one float32 step.
  f.zkey = static_cast<float>(f.z);
  {
    const double up = std::nextafter(f.zkey, std::numeric_limits<float>::infinity());
    const double dn = std::nextafter(f.zkey, -std::numeric_limits<float>::infinity());
    const double mid_up = 0.5 * (static_cast<double>(f.zkey) + up);
    const double mid_dn = 0.5 * (static_cast<double>(f.zkey) + dn);
    const double sumabs = std::fabs(cam.R[2][0] * mean[0]) + std::fabs(cam.R[2][1] * mean[1]) +
                          std::fabs(cam.R[2][2] * mean[2]) + std::fabs(cam.t[2]);
    const double margin = cfg.margin_z * f.z + 16.0 * kUnitRoundoff32 * kUnitRoundoff32 * sumabs;
    if (std::fabs(f.z - mid_up) <= margin || std::fabs(f.z - mid_dn) <= margin) f.flags |= 8;
  }
  // Unit quaternion and world covariance, Sigma^W = R_q diag(s^2) R_q^T (Appendix C.1).
  f.q_raw_norm = std::sqrt(quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3]);
  if (!(f.q_raw_norm > 0.0)) return;
  for (int c = 0; c < 4; ++c) f.qn[c] = quat[c] / f.q_raw_norm;
  quat_to_rotmat(f.qn, f.Rq);
  for (int a = 0; a < 3; ++a) f.s[a] = std::exp(log_scale[a]);
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) f.M[a][b] = f.Rq[a][b] * f.s[b];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double v = 0.0;
      for (int c = 0; c < 3; ++c) v += f.M[a][c] * f.M[b][c];
      f.SigW[a][b] = v;
    }
  // Projection Jacobian J at mu^C with the guard-band clamp (Eq. proj).
  f.u = f.mu_c[0] / f.z;
  f.w = f.mu_c[1] / f.z;
  f.uc = f.u;
  f.wc = f.w;
  f.u_clamped = f.w_clamped = false;
  if (cfg.jac_clamp > 0.0) {
    const double lim_u = cfg.jac_clamp * 0.5 * cam.width / cam.fx;
    const double lim_w = cfg.jac_clamp * 0.5 * cam.height / cam.fy;
    if (std::fabs(std::fabs(f.u) - lim_u) <= cfg.margin_g * lim_u) f.flags |= 2;
    if (std::fabs(std::fabs(f.w) - lim_w) <= cfg.margin_g * lim_w) f.flags |= 2;
    if (f.u > lim_u) { f.uc = lim_u; f.u_clamped = true; }
    if (f.u < -lim_u) { f.uc = -lim_u; f.u_clamped = true; }
    if (f.w > lim_w) { f.wc = lim_w; f.w_clamped = true; }
    if (f.w < -lim_w) { f.wc = -lim_w; f.w_clamped = true; }
  }
  f.J[0][0] = cam.fx / f.z; f.J[0][1] = 0.0; f.J[0][2] = -cam.fx * f.uc / f.z;
  f.J[1][0] = 0.0; f.J[1][1] = cam.fy / f.z; f.J[1][2] = -cam.fy * f.wc / f.z;
  // T = J R; Sigma^I = T Sigma^W T^T + eps2d I.
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 3; ++b)
      f.T[a][b] = f.J[a][0] * cam.R[0][b] + f.J[a][1] * cam.R[1][b] + f.J[a][2] * cam.R[2][b];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      double v = 0.0;
      for (int c = 0; c < 3; ++c)
        for (int e = 0; e < 3; ++e) v += f.T[a][c] * f.SigW[c][e] * f.T[b][e];
      f.cov2d[a][b] = v;
    }
  f.cov2d[0][0] += cfg.eps2d;
  f.cov2d[1][1] += cfg.eps2d;
  f.det = f.cov2d[0][0] * f.cov2d[1][1] - f.cov2d[0][1] * f.cov2d[1][0];
  if (!(f.det > 0.0)) return;
  f.conic[0] = f.cov2d[1][1] / f.det;
  f.conic[1] = -f.cov2d[0][1] / f.det;
  f.conic[2] = f.cov2d[0][0] / f.det;
  // Projected mean, mu^I = pi(mu^C) (Eq. proj).
  f.mean2d[0] = cam.fx * f.u + cam.cx;
  f.mean2d[1] = cam.fy * f.w + cam.cy;
  // Opacity from its logit.
  f.opacity = 1.0 / (1.0 + std::exp(-logit));
  f.kappa = 2.0 * std::log(f.opacity / cfg.alpha_min);
  // View-dependent colour (Eq. app-sh), direction from the camera centre c_W = -R^T t.
  for (int a = 0; a < 3; ++a)
    f.cam_center[a] = -(cam.R[0][a] * cam.t[0] + cam.R[1][a] * cam.t[1] + cam.R[2][a] * cam.t[2]);
  for (int a = 0; a < 3; ++a) f.dvec[a] = mean[a] - f.cam_center[a];
  f.dnorm = std::sqrt(f.dvec[0] * f.dvec[0] + f.dvec[1] * f.dvec[1] + f.dvec[2] * f.dvec[2]);
  for (int a = 0; a < 3; ++a) f.dir[a] = f.dvec[a] / f.dnorm;
  sh_basis(degree, f.dir, f.Y, f.dY);
  for (int ch = 0; ch < 3; ++ch) {
    double v = 0.0;
    for (int k = 0; k < K; ++k) v += sh[k * 3 + ch] * f.Y[k];
    f.rgb_raw[ch] = v + 0.5;
    f.rgb[ch] = f.rgb_raw[ch] > 0.0 ? f.rgb_raw[ch] : 0.0;
    if (std::fabs(f.rgb_raw[ch]) <= cfg.margin_g) f.flags |= 4;
  }
  f.valid = true;
}

// The per-(view, Gaussian) quantities compositing needs (the backward recomputes the rest).
struct Splat {
  bool valid = false;
  int flags = 0;
  float zkey = 0.0f;
  double mean2d[2], cov2d[3], conic[3], opacity, rgb[3], z;
  double amp;        // float32 error amplification of the conic (see kUnitRoundoff32)
  double chol[3] = {0.0, 0.0, 0.0};  // L L^T = (log2(e) / 2) conic (for the error bound)
};

Splat to_splat(const GaussFwd& f) {
  Splat s;
  s.valid = f.valid;
  s.flags = f.flags;
  s.zkey = f.zkey;
  s.mean2d[0] = f.mean2d[0];
  s.mean2d[1] = f.mean2d[1];
  s.cov2d[0] = f.cov2d[0][0];
  s.cov2d[1] = f.cov2d[0][1];
  s.cov2d[2] = f.cov2d[1][1];
  for (int k = 0; k < 3; ++k) {
    s.conic[k] = f.conic[k];
    s.rgb[k] = f.rgb[k];
  }
  s.opacity = f.opacity;
  s.z = f.z;
  s.amp = 1.0;
  if (f.valid) {
    const double tr = f.cov2d[0][0] + f.cov2d[1][1];
    const double disc = std::sqrt(std::max(0.25 * tr * tr - f.det, 0.0));
    const double lmax = 0.5 * tr + disc;
    const double lmin = f.det / lmax;
    const double jf2 = f.J[0][0] * f.J[0][0] + f.J[0][2] * f.J[0][2] + f.J[1][1] * f.J[1][1] +
                       f.J[1][2] * f.J[1][2];
    const double smax = std::max(f.s[0], std::max(f.s[1], f.s[2]));
    s.amp = std::sqrt(std::max(jf2 * smax * smax, lmax) / lmin);
    // L from the covariance: l11^2 = k a, l11 l21 = k b, l21^2 + l22^2 = k c for the conic
    // (a, b, c) = (Syy, -Sxy, Sxx) / det and k = log2(e) / 2.
    const double k = 0.5 / std::log(2.0);
    s.chol[0] = std::sqrt(k * f.cov2d[1][1] / f.det);
    s.chol[1] = -k * f.cov2d[0][1] / (f.det * s.chol[0]);
    s.chol[2] = std::sqrt(k / f.cov2d[1][1]);
  }
  return s;
}

// ln G = -1/2 d^T Q d at offset d = (dx, dy) from the projected mean (Eq. alpha), and the
// float32 error bound of ln(o G) there (see kUnitRoundoff32): the whitened offsets, the
// magnitude of the products they are formed from, and the conic's own error.
void exponent_and_bound(const Splat& f, double dx, double dy, double& power, double& err) {
  power = -0.5 * (f.conic[0] * dx * dx + f.conic[2] * dy * dy) - f.conic[1] * dx * dy;
  const double t = f.chol[0] * dx + f.chol[1] * dy, u = f.chol[2] * dy;
  const double terms = std::fabs(f.chol[0] * dx) +
                       (std::fabs(f.chol[1]) + std::fabs(f.chol[2])) * (std::fabs(dy) + 8.0);
  const double mag = std::log(2.0) * ((std::fabs(t) + std::fabs(u)) * terms + t * t + u * u);
  err = kUnitRoundoff32 * (8.0 * mag + 8.0 * std::fabs(power) * f.amp + 16.0);
}

// Screen-space gradient slots per (view, Gaussian).
enum G2 { kMx = 0, kMy, kCa, kCb, kCc, kOp, kR, kG, kB, kZ, kG2Count };

// Chains one (view, Gaussian)'s screen-space gradients back to the parameters and the twist.
void gaussian_backward(const GaussFwd& f, const double* mean, const double* sh, int degree,
                       const Camera& cam, const double g2[kG2Count], double g_mean[3],
                       double g_ls[3], double g_q[4], double* g_logit, double* g_sh,
                       double g_pose[6]) {
  const int K = (degree + 1) * (degree + 1);
  // Opacity: o = sigmoid(logit).
  *g_logit += g2[kOp] * f.opacity * (1.0 - f.opacity);
  // Conic = inverse(Sigma^I): G_Sigma = -Q G_Q Q with the symmetric G_Q.
  const double Q[2][2] = {{f.conic[0], f.conic[1]}, {f.conic[1], f.conic[2]}};
  const double GQ[2][2] = {{g2[kCa], 0.5 * g2[kCb]}, {0.5 * g2[kCb], g2[kCc]}};
  double GS[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      double v = 0.0;
      for (int c = 0; c < 2; ++c)
        for (int e = 0; e < 2; ++e) v += Q[a][c] * GQ[c][e] * Q[e][b];
      GS[a][b] = -v;
    }
  // Sigma^I = T Sigma^W T^T (+ eps I): G_T = 2 G_S T Sigma^W, G_SigW = T^T G_S T.
  double GT[2][3], GSigW[3][3];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 3; ++b) {
      double v = 0.0;
      for (int c = 0; c < 2; ++c)
        for (int e = 0; e < 3; ++e) v += GS[a][c] * f.T[c][e] * f.SigW[e][b];
      GT[a][b] = 2.0 * v;
    }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double v = 0.0;
      for (int c = 0; c < 2; ++c)
        for (int e = 0; e < 2; ++e) v += f.T[c][a] * GS[c][e] * f.T[e][b];
      GSigW[a][b] = v;
    }
  // T = J R: G_J = G_T R^T; the rotation's share G_R = J^T G_T.
  double GJ[2][3], GR[3][3];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 3; ++b)
      GJ[a][b] = GT[a][0] * cam.R[b][0] + GT[a][1] * cam.R[b][1] + GT[a][2] * cam.R[b][2];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) GR[a][b] = f.J[0][a] * GT[0][b] + f.J[1][a] * GT[1][b];
  // J(mu^C): J00 = fx/z, J02 = -fx uc/z, J11 = fy/z, J12 = -fy wc/z.
  const double z = f.z, z2 = f.z * f.z;
  double g_z = 0.0, g_u = 0.0, g_w = 0.0;
  g_z += GJ[0][0] * (-cam.fx / z2) + GJ[1][1] * (-cam.fy / z2);
  g_z += GJ[0][2] * (cam.fx * f.uc / z2) + GJ[1][2] * (cam.fy * f.wc / z2);
  if (!f.u_clamped) g_u += GJ[0][2] * (-cam.fx / z);
  if (!f.w_clamped) g_w += GJ[1][2] * (-cam.fy / z);
  // mu^I = (fx u + cx, fy w + cy).
  g_u += g2[kMx] * cam.fx;
  g_w += g2[kMy] * cam.fy;
  // u = x/z, w = y/z; the depth output and sort key z = mu^C_z.
  double g_muc[3];
  g_muc[0] = g_u / z;
  g_muc[1] = g_w / z;
  g_muc[2] = g_z - g_u * f.mu_c[0] / z2 - g_w * f.mu_c[1] / z2 + g2[kZ];
  // mu^C = R mu^W + t.
  for (int a = 0; a < 3; ++a)
    g_mean[a] += cam.R[0][a] * g_muc[0] + cam.R[1][a] * g_muc[1] + cam.R[2][a] * g_muc[2];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) GR[a][b] += g_muc[a] * mean[b];
  double g_t[3] = {g_muc[0], g_muc[1], g_muc[2]};
  // Sigma^W = M M^T, M = R_q diag(s): G_M = 2 G_SigW M; G_Rq = G_M diag(s); g_s_k = sum_a G_M[a][k] Rq[a][k].
  double GM[3][3], GRq[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double v = 0.0;
      for (int c = 0; c < 3; ++c) v += GSigW[a][c] * f.M[c][b];
      GM[a][b] = 2.0 * v;
    }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) GRq[a][b] = GM[a][b] * f.s[b];
  for (int k = 0; k < 3; ++k) {
    double gs = 0.0;
    for (int a = 0; a < 3; ++a) gs += GM[a][k] * f.Rq[a][k];
    g_ls[k] += gs * f.s[k];  // s = exp(log_scale)
  }
  // R_q(q_hat), then q_hat = q / |q|: g_q = (g_hat - q_hat (q_hat . g_hat)) / |q|.
  double g_qn[4];
  quat_to_rotmat_vjp(f.qn, GRq, g_qn);
  const double dotq = g_qn[0] * f.qn[0] + g_qn[1] * f.qn[1] + g_qn[2] * f.qn[2] + g_qn[3] * f.qn[3];
  for (int c = 0; c < 4; ++c) g_q[c] += (g_qn[c] - f.qn[c] * dotq) / f.q_raw_norm;
  // Colour: rgb = max(sum_k sh_k Y_k(dir) + 0.5, 0).
  double g_raw[3];
  for (int ch = 0; ch < 3; ++ch) g_raw[ch] = f.rgb_raw[ch] > 0.0 ? g2[kR + ch] : 0.0;
  double g_dir[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < K; ++k) {
    double coef = 0.0;
    for (int ch = 0; ch < 3; ++ch) {
      g_sh[k * 3 + ch] += g_raw[ch] * f.Y[k];
      coef += g_raw[ch] * sh[k * 3 + ch];
    }
    for (int a = 0; a < 3; ++a) g_dir[a] += coef * f.dY[k][a];
  }
  // dir = dvec / |dvec|, dvec = mu^W - c_W.
  const double dd = g_dir[0] * f.dir[0] + g_dir[1] * f.dir[1] + g_dir[2] * f.dir[2];
  double g_dvec[3];
  for (int a = 0; a < 3; ++a) g_dvec[a] = (g_dir[a] - f.dir[a] * dd) / f.dnorm;
  for (int a = 0; a < 3; ++a) g_mean[a] += g_dvec[a];
  // c_W = -R^T t: G_R += -t g_c^T, g_t += -R g_c with g_c = -g_dvec.
  double g_c[3] = {-g_dvec[0], -g_dvec[1], -g_dvec[2]};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) GR[a][b] += -cam.t[a] * g_c[b];
  for (int a = 0; a < 3; ++a)
    g_t[a] += -(cam.R[a][0] * g_c[0] + cam.R[a][1] * g_c[1] + cam.R[a][2] * g_c[2]);
  // Left twist (Eq. leftupdate): dR = [w]_x R, dt = [w]_x t + rho.
  // dL/drho = g_t; dL/dw from the skew part of M = G_R R^T + g_t t^T.
  double Mx[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double v = 0.0;
      for (int c = 0; c < 3; ++c) v += GR[a][c] * cam.R[b][c];
      Mx[a][b] = v + g_t[a] * cam.t[b];
    }
  g_pose[0] += g_t[0];
  g_pose[1] += g_t[1];
  g_pose[2] += g_t[2];
  g_pose[3] += Mx[2][1] - Mx[1][2];
  g_pose[4] += Mx[0][2] - Mx[2][0];
  g_pose[5] += Mx[1][0] - Mx[0][1];
}

// Per-thread screen-space gradient accumulators (dense array or hash map of touched Gaussians).
struct DenseAcc {
  std::vector<double> data;
  void reset(int n) { data.assign(static_cast<size_t>(n) * kG2Count, 0.0); }
  double* slots(int idx) { return data.data() + static_cast<size_t>(idx) * kG2Count; }
};
struct SparseAcc {
  std::unordered_map<int, std::array<double, kG2Count>> map;
  void reset(int) { map.clear(); }
  double* slots(int idx) {
    auto it = map.find(idx);
    if (it == map.end()) {
      std::array<double, kG2Count> z;
      z.fill(0.0);
      it = map.emplace(idx, z).first;
    }
    return it->second.data();
  }
};

struct PixelOut {
  double color[3], depth, alpha, t_final;
  int n_contrib;
  uint8_t amb;
};

struct Cand {
  double z;
  int idx;
};

// Composites one pixel (Eq. alpha). If `grad` is non-null, accumulates the screen-space gradients
// of <g, outputs> into the accumulator `acc` (slot kG2Count * idx + s).
template <typename Acc>
void shade_pixel(const std::vector<Splat>& F, const std::vector<int>& cands, double px, double py,
                 const Config& cfg, PixelOut& out, const double* g /*5*/, Acc* acc) {
  struct Hit {
    float zkey;
    double z;
    int idx;
    double G, oG, alpha, dx, dy;
    double err;  // float32 error bound of ln(o G) at this pixel
  };
  std::vector<Hit> hits;
  hits.reserve(cands.size());
  const double ln_amin = std::log(cfg.alpha_min), ln_amax = std::log(cfg.alpha_max);
  for (int idx : cands) {
    const Splat& f = F[idx];
    if (!f.valid) continue;
    const double dx = px - f.mean2d[0], dy = py - f.mean2d[1];
    double power, err;
    exponent_and_bound(f, dx, dy, power, err);
    const double G = std::exp(power);
    const double oG = f.opacity * G;
    if (std::log(oG) < ln_amin - cfg.margin_alpha - err) continue;
    hits.push_back({f.zkey, f.z, idx, G, oG, std::min(cfg.alpha_max, oG), dx, dy, err});
  }
  std::sort(hits.begin(), hits.end(), [](const Hit& a, const Hit& b) {
    return a.zkey < b.zkey || (a.zkey == b.zkey && a.idx < b.idx);
  });
  uint8_t amb = 0;
  double T = 1.0;
  double C[3] = {0, 0, 0}, D = 0.0;
  double errT = 0.0;  // float32 error bound of ln T
  double errC = 0.0;  // float32 error bound of the colour
  std::vector<int> inc;  // positions in `hits` of the included Gaussians
  for (size_t k = 0; k < hits.size(); ++k) {
    const Hit& h = hits[k];
    const double* c = F[h.idx].rgb;
    const double cmax = std::max(1.0, std::max(c[0], std::max(c[1], c[2])));
    const double ln_oG = std::log(h.oG);
    // Including or skipping a Gaussian at the threshold changes the image by about alpha_min T c.
    if (std::fabs(ln_oG - ln_amin) <= cfg.margin_alpha + h.err &&
        cfg.alpha_min * T * cmax >= cfg.margin_effect)
      amb |= kAmbAlphaMin;
    if (h.oG < cfg.alpha_min) continue;
    // A depth key that may round the other way only matters next to another key of the list
    // within one float32 step (the pair's order, or their tie-break, could change).
    if (F[h.idx].flags & 8) {
      for (size_t o = 0; o < hits.size(); ++o)
        if (o != k && std::fabs(static_cast<double>(hits[o].zkey) - h.zkey) <=
                          std::fabs(static_cast<double>(
                              std::nextafter(h.zkey, std::numeric_limits<float>::infinity())) -
                          h.zkey))
          amb |= kAmbDepthTie;
    }
    if (F[h.idx].flags & 1) amb |= kAmbNear;
    if (F[h.idx].flags & 6) amb |= kAmbGradKink;
    if (std::fabs(ln_oG - ln_amax) <= cfg.margin_alpha + h.err) amb |= kAmbAlphaMax;
    const double Tn = T * (1.0 - h.alpha);
    // Error bound of ln T': the alpha error through ln(1 - alpha), plus the float32 arithmetic
    // of T' = T - alpha T (two roundings, the first magnified by alpha / (1 - alpha)).
    const double errTn = errT + (h.err + 2.0 * kUnitRoundoff32) * h.alpha / (1.0 - h.alpha) +
                         2.0 * kUnitRoundoff32;
    if (std::fabs(std::log(Tn / cfg.t_min)) <= cfg.margin_t + errTn) amb |= kAmbTMin;
    if (Tn < cfg.t_min) break;
    const double w = h.alpha * T;
    errC += w * cmax * (h.err + errT);
    for (int ch = 0; ch < 3; ++ch) C[ch] += w * F[h.idx].rgb[ch];
    D += w * h.z;
    T = Tn;
    errT = errTn;
    inc.push_back(static_cast<int>(k));
  }
  if (errC > cfg.margin_cont) amb |= kAmbCond;
  for (int ch = 0; ch < 3; ++ch) out.color[ch] = C[ch] + T * cfg.bg[ch];
  out.depth = D;
  out.alpha = 1.0 - T;
  out.t_final = T;
  out.n_contrib = static_cast<int>(inc.size());
  out.amb = amb;
  if (!g || !acc) return;
  // Backward of <g, (C, D, A)> with explicit prefix products and suffix sums.
  const double gC[3] = {g[0], g[1], g[2]}, gD = g[3], gA = g[4];
  const int n = static_cast<int>(inc.size());
  std::vector<double> Tpre(n + 1);
  Tpre[0] = 1.0;
  for (int j = 0; j < n; ++j) Tpre[j + 1] = Tpre[j] * (1.0 - hits[inc[j]].alpha);
  const double TN = Tpre[n];
  double SC[3] = {TN * cfg.bg[0], TN * cfg.bg[1], TN * cfg.bg[2]};  // sum over k > j of w_k c_k + T_N bg
  double SD = 0.0;                                                    // sum over k > j of w_k z_k
  for (int j = n - 1; j >= 0; --j) {
    const Hit& h = hits[inc[j]];
    const Splat& f = F[h.idx];
    const double Tj = Tpre[j];
    const double wj = h.alpha * Tj;
    const double om = 1.0 - h.alpha;
    double dL_dalpha = 0.0;
    for (int ch = 0; ch < 3; ++ch) dL_dalpha += gC[ch] * (f.rgb[ch] * Tj - SC[ch] / om);
    dL_dalpha += gD * (h.z * Tj - SD / om);
    dL_dalpha += gA * TN / om;
    double* a = acc->slots(h.idx);
    a[kR] += gC[0] * wj;
    a[kG] += gC[1] * wj;
    a[kB] += gC[2] * wj;
    a[kZ] += gD * wj;
    if (h.oG < cfg.alpha_max) {  // alpha = o G, not clamped
      a[kOp] += dL_dalpha * h.G;
      const double dL_dpow = dL_dalpha * f.opacity * h.G;
      const double ca = f.conic[0], cb = f.conic[1], cc = f.conic[2];
      // power = -1/2 (a dx^2 + c dy^2) - b dx dy, d = p - mu^I.
      a[kMx] += dL_dpow * (ca * h.dx + cb * h.dy);
      a[kMy] += dL_dpow * (cb * h.dx + cc * h.dy);
      a[kCa] += dL_dpow * (-0.5 * h.dx * h.dx);
      a[kCb] += dL_dpow * (-h.dx * h.dy);
      a[kCc] += dL_dpow * (-0.5 * h.dy * h.dy);
    }
    for (int ch = 0; ch < 3; ++ch) SC[ch] += wj * f.rgb[ch];
    SD += wj * h.z;
  }
}

Config read_config(const double* c) {
  Config cfg;
  cfg.alpha_min = c[0];
  cfg.alpha_max = c[1];
  cfg.t_min = c[2];
  cfg.znear = c[3];
  cfg.eps2d = c[4];
  cfg.jac_clamp = c[5];
  cfg.bg[0] = c[6];
  cfg.bg[1] = c[7];
  cfg.bg[2] = c[8];
  cfg.margin_alpha = c[9];
  cfg.margin_t = c[10];
  cfg.margin_z = c[11];
  cfg.margin_g = c[12];
  cfg.margin_effect = c[13];
  cfg.margin_cont = c[14];
  return cfg;
}

Camera read_camera(const double* c) {
  Camera cam;
  cam.width = static_cast<int>(c[0]);
  cam.height = static_cast<int>(c[1]);
  cam.fx = c[2];
  cam.fy = c[3];
  cam.cx = c[4];
  cam.cy = c[5];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) cam.R[a][b] = c[6 + 3 * a + b];
  for (int a = 0; a < 3; ++a) cam.t[a] = c[15 + a];
  return cam;
}

// Largest total size of the dense per-thread accumulators before the oracle switches to hash
// maps (settable for tests through oracle_set_dense_limit).
double g_dense_limit_bytes = static_cast<double>(1u << 30);

// Runs fn(thread, item) for item in [0, n_items) on n_threads threads (dynamic assignment;
// callers make every result independent of which thread ran an item).
void run_parallel(int n_threads, int n_items, const std::function<void(int, int)>& fn) {
  if (n_threads <= 1) {
    for (int k = 0; k < n_items; ++k) fn(0, k);
    return;
  }
  std::atomic<int> next(0);
  std::vector<std::thread> pool;
  for (int t = 0; t < n_threads; ++t)
    pool.emplace_back([&, t]() {
      for (;;) {
        const int k = next.fetch_add(1);
        if (k >= n_items) break;
        fn(t, k);
      }
    });
  for (auto& th : pool) th.join();
}
}  // namespace

extern "C" {

// Sets the byte limit of the dense per-thread gradient accumulators (results do not depend on it).
void oracle_set_dense_limit(double bytes) { g_dense_limit_bytes = bytes; }

// Real SH basis for n unit directions dirs[n,3] -> Y[n,16] (unused entries zero).
void oracle_sh_basis(int degree, int n, const double* dirs, double* Y) {
  double y[16], dy[16][3];
  for (int i = 0; i < n; ++i) {
    sh_basis(degree, dirs + 3 * i, y, dy);
    for (int k = 0; k < 16; ++k) Y[16 * i + k] = y[k];
  }
}

void oracle_quat_to_rotmat(int n, const double* q, double* R) {
  for (int i = 0; i < n; ++i) {
    double qn[4], r[3][3];
    const double nr = std::sqrt(q[4 * i] * q[4 * i] + q[4 * i + 1] * q[4 * i + 1] +
                                q[4 * i + 2] * q[4 * i + 2] + q[4 * i + 3] * q[4 * i + 3]);
    for (int c = 0; c < 4; ++c) qn[c] = q[4 * i + c] / nr;
    quat_to_rotmat(qn, r);
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) R[9 * i + 3 * a + b] = r[a][b];
  }
}

// Per-(view, Gaussian) screen-space record -> out[V, N, 16]: valid, mean2d[2], cov2d[3]
// (xx, xy, yy), conic[3] (a, b, c), depth z, opacity, rgb[3], kappa, per-Gaussian flags.
void oracle_project(int n, int degree, const double* means, const double* log_scales,
                    const double* quats, const double* logits, const double* sh, int n_views,
                    const double* cams, const double* cfgv, double* out) {
  const Config cfg = read_config(cfgv);
  const int K = (degree + 1) * (degree + 1);
  for (int v = 0; v < n_views; ++v) {
    const Camera cam = read_camera(cams + 18 * v);
    for (int i = 0; i < n; ++i) {
      GaussFwd f;
      gaussian_forward(means + 3 * i, log_scales + 3 * i, quats + 4 * i, logits[i],
                       sh + static_cast<size_t>(3 * K) * i, degree, cam, cfg, f);
      double* o = out + (static_cast<size_t>(v) * n + i) * 16;
      o[0] = f.valid ? 1.0 : 0.0;
      o[1] = f.mean2d[0]; o[2] = f.mean2d[1];
      o[3] = f.cov2d[0][0]; o[4] = f.cov2d[0][1]; o[5] = f.cov2d[1][1];
      o[6] = f.conic[0]; o[7] = f.conic[1]; o[8] = f.conic[2];
      o[9] = f.z; o[10] = f.opacity;
      o[11] = f.rgb[0]; o[12] = f.rgb[1]; o[13] = f.rgb[2];
      o[14] = f.kappa; o[15] = f.flags;
    }
  }
}

// ln(o G) in double precision and its float32 error bound for m (view, Gaussian, pixel) triples:
// items[m, 4] = (view, Gaussian, x, y); out[m, 2] = (ln(o G), bound); a Gaussian culled in the
// view gets (-inf, 0). Used to pin the bound against a float32 evaluation.
void oracle_log_og_bound(int n, int degree, const double* means, const double* log_scales,
                         const double* quats, const double* logits, const double* sh,
                         int n_views, const double* cams, const double* cfgv, int m,
                         const double* items, double* out) {
  const Config cfg = read_config(cfgv);
  const int K = (degree + 1) * (degree + 1);
  for (int k = 0; k < m; ++k) {
    const int v = static_cast<int>(items[4 * k]), i = static_cast<int>(items[4 * k + 1]);
    out[2 * k] = -std::numeric_limits<double>::infinity();
    out[2 * k + 1] = 0.0;
    if (v < 0 || v >= n_views || i < 0 || i >= n) continue;
    const Camera cam = read_camera(cams + 18 * v);
    GaussFwd f;
    gaussian_forward(means + 3 * i, log_scales + 3 * i, quats + 4 * i, logits[i],
                     sh + static_cast<size_t>(3 * K) * i, degree, cam, cfg, f);
    const Splat sp = to_splat(f);
    if (!sp.valid) continue;
    double power, err;
    exponent_and_bound(sp, items[4 * k + 2] - sp.mean2d[0], items[4 * k + 3] - sp.mean2d[1], power,
                       err);
    out[2 * k] = std::log(sp.opacity) + power;
    out[2 * k + 1] = err;
  }
}

/*
 * Renders n_views views and optionally back-propagates upstream image gradients.
 *   cams[V, 18]: width, height, fx, fy, cx, cy, R (row-major 3x3), t (world-to-camera).
 *   cfg[15]: alpha_min, alpha_max, t_min, znear, eps2d, jac_clamp, bg[3], margin_alpha,
 *            margin_t, margin_z, margin_g, margin_effect, margin_cont.
 *   Images are concatenated over views, view v row-major at pixel offset sum_{u<v} W_u H_u.
 *   pixel_mask[P] (nullable): only pixels with a non-zero mask are rendered / back-propagated.
 *   brute_force != 0: every Gaussian is a candidate at every pixel (no bounding-box skip).
 *   d_color[P,3], d_depth[P], d_alpha[P] (all nullable; when all three are null there is no
 *   backward). Gradient outputs are overwritten: g_means[N,3], g_log_scales[N,3], g_quats[N,4],
 *   g_logits[N], g_sh[N,K,3], g_pose[V,6] = (rho, omega); g_2d[V,N,10] (nullable) receives the
 *   screen-space gradients (mean2d x/y, conic a/b/c, opacity, rgb, z).
 * Returns 0 on success.
 */
int oracle_render(int n, int degree, const double* means, const double* log_scales,
                  const double* quats, const double* logits, const double* sh, int n_views,
                  const double* cams, const double* cfgv, const uint8_t* pixel_mask,
                  int brute_force, int n_threads, double* color, double* depth, double* alpha,
                  double* t_final, int32_t* n_contrib, uint8_t* ambiguous, const double* d_color,
                  const double* d_depth, const double* d_alpha, double* g_means,
                  double* g_log_scales, double* g_quats, double* g_logits, double* g_sh,
                  double* g_pose, double* g_2d) {
  if (n < 0 || degree < 0 || degree > 3 || n_views < 0) return 1;
  if (n_threads < 1) n_threads = 1;
  const Config cfg = read_config(cfgv);
  const int K = (degree + 1) * (degree + 1);
  const bool backward = d_color || d_depth || d_alpha;
  if (backward) {
    std::memset(g_means, 0, sizeof(double) * 3 * n);
    std::memset(g_log_scales, 0, sizeof(double) * 3 * n);
    std::memset(g_quats, 0, sizeof(double) * 4 * n);
    std::memset(g_logits, 0, sizeof(double) * n);
    std::memset(g_sh, 0, sizeof(double) * 3 * K * n);
    std::memset(g_pose, 0, sizeof(double) * 6 * n_views);
  }
  std::vector<Splat> F(n);
  // Per-thread screen-space gradient accumulators: dense arrays when they fit in 1 GiB in
  // total, else hash maps of the Gaussians a thread's pixels touch (large scenes, few pixels).
  const bool sparse = backward && static_cast<double>(n) * kG2Count * sizeof(double) * n_threads >
                                      g_dense_limit_bytes;
  std::vector<DenseAcc> dense(backward && !sparse ? n_threads : 0);
  std::vector<SparseAcc> hashed(backward && sparse ? n_threads : 0);
  std::vector<double> g2all(backward ? static_cast<size_t>(n) * kG2Count : 0);
  size_t pix_base = 0;
  for (int v = 0; v < n_views; ++v) {
    const Camera cam = read_camera(cams + 18 * v);
    const int W = cam.width, H = cam.height;
    // Per-Gaussian forward quantities for this view.
    run_parallel(n_threads, (n + 1023) / 1024, [&](int, int blk) {
      const int i0 = blk * 1024, i1 = std::min(n, i0 + 1024);
      GaussFwd f;
      for (int i = i0; i < i1; ++i) {
        gaussian_forward(means + 3 * i, log_scales + 3 * i, quats + 4 * i, logits[i],
                         sh + static_cast<size_t>(3 * K) * i, degree, cam, cfg, f);
        F[i] = to_splat(f);
      }
    });
    // Candidate lists: a 16x16-pixel cell grid over the padded bounding box of the
    // alpha >= alpha_min ellipse (an accelerator only: candidates are tested exactly per pixel).
    const int cell = 16;
    const int gx = (W + cell - 1) / cell, gy = (H + cell - 1) / cell;
    std::vector<std::vector<int>> cells(static_cast<size_t>(gx) * gy);
    std::vector<int> all_valid;
    if (brute_force) {
      for (int i = 0; i < n; ++i)
        if (F[i].valid) all_valid.push_back(i);
    } else {
      for (int i = 0; i < n; ++i) {
        const Splat& f = F[i];
        if (!f.valid) continue;
        const double kap = 2.0 * std::log(f.opacity / (cfg.alpha_min * (1.0 - cfg.margin_alpha)));
        if (!(kap >= 0.0)) continue;
        const double rx = std::sqrt(kap * f.cov2d[0]) + 2.0;
        const double ry = std::sqrt(kap * f.cov2d[2]) + 2.0;
        const double x0 = f.mean2d[0] - rx, x1 = f.mean2d[0] + rx;
        const double y0 = f.mean2d[1] - ry, y1 = f.mean2d[1] + ry;
        if (x1 < 0.0 || y1 < 0.0 || x0 > W - 1.0 || y0 > H - 1.0) continue;
        const int cx0 = std::max(0, static_cast<int>(std::floor(x0 / cell)));
        const int cx1 = std::min(gx - 1, static_cast<int>(std::floor(x1 / cell)));
        const int cy0 = std::max(0, static_cast<int>(std::floor(y0 / cell)));
        const int cy1 = std::min(gy - 1, static_cast<int>(std::floor(y1 / cell)));
        for (int cy = cy0; cy <= cy1; ++cy)
          for (int cx = cx0; cx <= cx1; ++cx) cells[static_cast<size_t>(cy) * gx + cx].push_back(i);
      }
    }
    if (backward) {
      for (auto& a : dense) a.reset(n);
      for (auto& a : hashed) a.reset(n);
    }
    // Pixels. Thread t owns the rows y with y % n_threads == t, so the per-thread gradient
    // sums (and hence the results) do not depend on scheduling.
    run_parallel(n_threads, n_threads, [&](int, int tid) {
      for (int y = tid; y < H; y += n_threads)
      for (int x = 0; x < W; ++x) {
        const size_t p = pix_base + static_cast<size_t>(y) * W + x;
        if (pixel_mask && !pixel_mask[p]) continue;
        const std::vector<int>& cand =
            brute_force ? all_valid : cells[static_cast<size_t>(y / cell) * gx + (x / cell)];
        double g[5] = {0, 0, 0, 0, 0};
        if (backward) {
          if (d_color)
            for (int ch = 0; ch < 3; ++ch) g[ch] = d_color[3 * p + ch];
          if (d_depth) g[3] = d_depth[p];
          if (d_alpha) g[4] = d_alpha[p];
        }
        PixelOut po;
        if (!backward)
          shade_pixel<DenseAcc>(F, cand, x, y, cfg, po, nullptr, nullptr);
        else if (sparse)
          shade_pixel(F, cand, x, y, cfg, po, g, &hashed[tid]);
        else
          shade_pixel(F, cand, x, y, cfg, po, g, &dense[tid]);
        for (int ch = 0; ch < 3; ++ch) color[3 * p + ch] = po.color[ch];
        depth[p] = po.depth;
        alpha[p] = po.alpha;
        t_final[p] = po.t_final;
        n_contrib[p] = po.n_contrib;
        ambiguous[p] = po.amb;
      }
    });
    if (backward) {
      // Sum the per-thread screen-space gradients in thread order.
      std::fill(g2all.begin(), g2all.end(), 0.0);
      if (sparse) {
        for (int t = 0; t < n_threads; ++t)
          for (const auto& kv : hashed[t].map)
            for (int s = 0; s < kG2Count; ++s)
              g2all[static_cast<size_t>(kv.first) * kG2Count + s] += kv.second[s];
      } else {
        run_parallel(n_threads, (n + 1023) / 1024, [&](int, int blk) {
          const size_t i0 = static_cast<size_t>(blk) * 1024;
          const size_t i1 = std::min(static_cast<size_t>(n), i0 + 1024);
          for (int t = 0; t < n_threads; ++t)
            for (size_t j = i0 * kG2Count; j < i1 * kG2Count; ++j) g2all[j] += dense[t].data[j];
        });
      }
      // Chain each touched Gaussian (forward quantities recomputed in full).
      const int n_blk = (n + 1023) / 1024;
      std::vector<double> pose_part(static_cast<size_t>(n_blk) * 6, 0.0);
      run_parallel(n_threads, n_blk, [&](int, int blk) {
        const int i0 = blk * 1024, i1 = std::min(n, i0 + 1024);
        GaussFwd f;
        for (int i = i0; i < i1; ++i) {
          const double* g2 = g2all.data() + static_cast<size_t>(i) * kG2Count;
          bool any = false;
          for (int s = 0; s < kG2Count; ++s) any = any || g2[s] != 0.0;
          if (g_2d)
            for (int s = 0; s < kG2Count; ++s)
              g_2d[(static_cast<size_t>(v) * n + i) * kG2Count + s] = g2[s];
          if (!any || !F[i].valid) continue;
          gaussian_forward(means + 3 * i, log_scales + 3 * i, quats + 4 * i, logits[i],
                           sh + static_cast<size_t>(3 * K) * i, degree, cam, cfg, f);
          gaussian_backward(f, means + 3 * i, sh + static_cast<size_t>(3 * K) * i, degree, cam,
                            g2, g_means + 3 * i, g_log_scales + 3 * i, g_quats + 4 * i,
                            g_logits + i, g_sh + static_cast<size_t>(3 * K) * i,
                            pose_part.data() + 6 * blk);
        }
      });
      for (int b = 0; b < n_blk; ++b)
        for (int s = 0; s < 6; ++s) g_pose[6 * v + s] += pose_part[6 * b + s];
    }
    pix_base += static_cast<size_t>(W) * H;
  }
  return 0;
}

}  // extern "C"
