"""Pin of the oracle's float32 error bound of ln(o G) (the bound its ambiguity flags use).

The oracle flags a pixel when a discrete decision (alpha against 1/255, T against 1e-4) lies
within the float32 evaluation error of its threshold, using a modelled bound of that error. A
bound that is too narrow would let a legitimate float32 result fail parity; one far too wide
would flag pixels for nothing. This test evaluates ln(o G) in float32, step by step as a float32
renderer of Eq. proj and Eq. alpha does (covariance from the rounded Jacobian, rotation and scales,
the whitened exponent log2 o - |L^T d|^2 from a tile anchor row), for more than 1e5 (Gaussian,
pixel) cases inside the alpha >= 1/255 footprints: small and large Gaussians, thin ones whose projected
condition number reaches 1e5, centres thousands of pixels off the image and just beyond the near
plane. Every float32 value must lie within the bound of the double-precision one, and the bound
must not exceed the observed worst error by more than its stated safety factor's margin.
"""
import numpy as np

import oracle

F = np.float32
LN2 = np.log(2.0)


def _fma(a, b, c):
    """float32 fused multiply-add: the double product of two floats is exact."""
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(F)


def _scene(rng, n):
    """Gaussians in front of a 1920x1080 camera (f = 960), mixing ordinary, large and thin ones,
    some centred far outside the image and some just beyond the near plane."""
    z = np.exp(rng.uniform(np.log(0.21), np.log(12.0), n))
    # |x/z| up to 6 (the Jacobian clamp is at 1.3 W / 2 / f), most inside the view.
    u = np.where(rng.random(n) < 0.7, rng.uniform(-1.1, 1.1, n), rng.uniform(-6.0, 6.0, n))
    w = np.where(rng.random(n) < 0.7, rng.uniform(-0.6, 0.6, n), rng.uniform(-4.0, 4.0, n))
    means = np.stack([u * z, w * z, z], 1)
    ls = rng.normal(-4.0, 1.0, (n, 3))
    thin = rng.random(n) < 0.4
    ls[thin, 0] = rng.uniform(-2.0, -0.5, thin.sum())       # one long axis
    ls[thin, 1:] = rng.uniform(-7.0, -4.5, (thin.sum(), 2))  # two thin ones
    q = rng.standard_normal((n, 4))
    logit = rng.normal(1.0, 1.5, n)
    return dict(means=means.astype(F), log_scales=ls.astype(F), quats=q.astype(F),
                opacity_logits=logit.astype(F), sh=np.zeros((n, 1, 3), F))


CAM = dict(width=1920, height=1080, fx=960.0, fy=960.0, cx=959.5, cy=539.5,
           R=np.eye(3), t=np.zeros(3))


def _float32_log_og(g, items, eps2d=0.3, jac_clamp=1.3):
    """ln(o G) as a float32 renderer evaluates it (every operation rounded to float32)."""
    i = items[:, 1].astype(np.int64)
    m = g["means"][i].astype(F)
    ls = g["log_scales"][i].astype(F)
    q = g["quats"][i].astype(F)
    logit = g["opacity_logits"][i].astype(F)
    px, py = items[:, 2].astype(F), items[:, 3].astype(F)
    qn = np.sqrt(np.sum(q * q, 1, dtype=F)).astype(F)
    qq = q * (F(1) / qn)[:, None]
    w_, x, y, z = qq[:, 0], qq[:, 1], qq[:, 2], qq[:, 3]
    one, two = F(1), F(2)
    Rq = np.stack([one - two * (y * y + z * z), two * (x * y - w_ * z), two * (x * z + w_ * y),
                   two * (x * y + w_ * z), one - two * (x * x + z * z), two * (y * z - w_ * x),
                   two * (x * z - w_ * y), two * (y * z + w_ * x), one - two * (x * x + y * y)],
                  1).reshape(-1, 3, 3).astype(F)
    s = np.exp(ls).astype(F)
    M = (Rq * s[:, None, :]).astype(F)
    opacity = (one / (one + np.exp(-logit))).astype(F)
    # Camera-space mean: the float32 rounding of the exact value (identity pose here).
    mc = m.astype(np.float64)
    zz = mc[:, 2].astype(F)
    rz = (one / zz).astype(F)
    u = (mc[:, 0].astype(F) / zz).astype(F)
    v = (mc[:, 1].astype(F) / zz).astype(F)
    fx, fy, cx, cy = F(CAM["fx"]), F(CAM["fy"]), F(CAM["cx"]), F(CAM["cy"])
    lim_u = F(jac_clamp * 0.5 * CAM["width"] / CAM["fx"])
    lim_w = F(jac_clamp * 0.5 * CAM["height"] / CAM["fy"])
    uc, wc = np.clip(u, -lim_u, lim_u), np.clip(v, -lim_w, lim_w)
    J00, J11 = fx * rz, fy * rz
    J02, J12 = -fx * uc * rz, -fy * wc * rz
    # T = J R with R = I: rows (J00, 0, J02), (0, J11, J12).
    T = np.zeros((len(i), 2, 3), F)
    T[:, 0, 0], T[:, 0, 2], T[:, 1, 1], T[:, 1, 2] = J00, J02, J11, J12
    A = np.einsum("nrc,nck->nrk", T, M).astype(F)
    sxx = np.sum(A[:, 0] * A[:, 0], 1, dtype=F)
    syy = np.sum(A[:, 1] * A[:, 1], 1, dtype=F)
    sxy = np.sum(A[:, 0] * A[:, 1], 1, dtype=F)
    e = F(eps2d)
    cov0, cov2 = sxx + e, syy + e
    A64 = A.astype(np.float64)
    minors = [(A64[:, 0, a] * A64[:, 1, b] - A64[:, 0, b] * A64[:, 1, a]).astype(F)
              for a, b in ((0, 1), (0, 2), (1, 2))]
    det = (minors[0] * minors[0] + minors[1] * minors[1] + minors[2] * minors[2]
           + e * (sxx + syy) + e * e).astype(F)
    k = F(0.5 / LN2)
    idet = (one / det).astype(F)
    l11 = np.sqrt(k * cov2 * idet).astype(F)
    l21 = (-k * sxy * idet / l11).astype(F)
    l22 = np.sqrt(k / cov2).astype(F)
    lg2o = np.log2(opacity).astype(F)
    # Projected mean as an unevaluated double-float sum.
    mx = CAM["fx"] * (mc[:, 0] / mc[:, 2]) + CAM["cx"]
    my = CAM["fy"] * (mc[:, 1] / mc[:, 2]) + CAM["cy"]
    mx_hi, my_hi = mx.astype(F), my.astype(F)
    mx_lo, my_lo = (mx - mx_hi).astype(F), (my - my_hi).astype(F)
    # The blend's evaluation at pixel (px, py) of a 16x16 tile anchored at its middle row.
    y_a = (F(16) * np.floor(py / F(16)) + F(8)).astype(F)
    dya = ((y_a - my_hi) - my_lo).astype(F)
    c21, s_a = (l21 * dya).astype(F), (l22 * dya).astype(F)
    dx = ((px - mx_hi) - mx_lo).astype(F)
    ta = _fma(l11, dx, c21)
    r = (py - y_a).astype(F)
    t = _fma(r, l21, ta)
    sv = _fma(r, l22, s_a)
    nq = _fma(t, t, _fma(sv, sv, -lg2o))
    return -nq.astype(np.float64) * LN2


def test_float32_exponent_stays_within_the_oracle_bound():
    rng = np.random.default_rng(4242)
    n = 12000
    g = _scene(rng, n)
    pr = oracle.project(g, [CAM])
    valid = pr["valid"][0]
    mean2d, cov, kappa = pr["mean2d"][0], pr["cov2d"][0], pr["kappa"][0]
    items = []
    for i in np.nonzero(valid & (kappa > 0))[0]:
        S = np.array([[cov[i, 0], cov[i, 1]], [cov[i, 1], cov[i, 2]]])
        Lc = np.linalg.cholesky(S)
        # Points of the alpha >= 1/255 ellipse: d = Lc w with |w|^2 <= kappa, then the pixel.
        wv = rng.standard_normal((64, 2))
        wv *= (np.sqrt(kappa[i]) * np.sqrt(rng.random(64)) / np.linalg.norm(wv, axis=1))[:, None]
        p = np.rint(mean2d[i] + wv @ Lc.T)
        ok = (p[:, 0] >= 0) & (p[:, 0] < 1920) & (p[:, 1] >= 0) & (p[:, 1] < 1080)
        for xy in p[ok][:20]:
            items.append((0, i, xy[0], xy[1]))
    items = np.array(items, np.float64)
    assert len(items) > 100_000, len(items)
    ln64, bound = oracle.log_og_bound(g, [CAM], items)
    ln32 = _float32_log_og(g, items)
    c = cov[items[:, 1].astype(np.int64)]
    tr, det = c[:, 0] + c[:, 2], c[:, 0] * c[:, 2] - c[:, 1] ** 2
    lmax = 0.5 * tr + np.sqrt(np.maximum(0.25 * tr * tr - det, 0.0))
    cond = lmax * lmax / det
    keep = ln64 >= np.log(1.0 / 255.0) - 1.0
    err = np.abs(ln32 - ln64)[keep]
    b = bound[keep]
    ratio = err / b
    worst = np.argsort(-ratio)[:5]
    info = dict(cases=int(keep.sum()), max_ratio=float(ratio.max()),
                median_ratio=float(np.median(ratio)), max_err=float(err.max()),
                worst=[(float(err[w]), float(b[w])) for w in worst])
    print(info)
    assert (err <= b).all(), info
    # The bound carries a safety factor of 8 on its leading terms; the worst case must come
    # within a factor 100 of it, or the bound flags pixels for nothing.
    assert ratio.max() >= 0.01, info
    # Thin footprints are in the sample.
    assert (cond[keep] > 1e3).sum() > 1000, np.quantile(cond[keep], [0.5, 0.99, 1.0])
