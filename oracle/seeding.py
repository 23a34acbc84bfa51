"""FP64 CPU oracle of the single-step dense initialisation (Section 3.3 "Multi-view
Triangulation" and "Gaussian Parameter Initialization"; appendix "Gaussian Initialization and
Joint Mapping": Eq. app-sigma-init, Eq. app-alpha-init).

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this module. The product path never imports it, and it imports
nothing from the product package.

Plain numpy in float64, one reference pixel at a time; the SVD is numpy's (LAPACK).

Inputs (M retained reference pixels, up to K neighbours each):
  cameras: V camera dicts (width, height, fx, fy, cx, cy, R [3,3], t [3]; world-to-camera);
  ref_view [M] int, ref_xy [M,2] pixel coordinates in the reference view;
  nb_view [M,K] int (-1: no neighbour), nb_xy [M,K,2] matched coordinates, nb_conf [M,K] the
  per-neighbour confidences kappa_{r->n}(p) in [0, 1];
  observed [P,3] frames (views concatenated, row-major), gain_bias [V,2] exposure of each view.

Readings where the paper is silent (the CUDA path takes the same ones):
  * A hypothesis (r, n) is rejected unless the point lies in front of both cameras, the angle
    between the two rays reaching it is at least min_parallax (radians), and its reprojection
    error, the RMS over the two views of |pi(X) - x| in pixels, is at most max_reproj.
  * Among the accepted hypotheses the lowest error wins; errors within tie_eps pixels of the
    lowest count as ties, decided by the larger baseline angle, then the lower neighbour slot.
  * kappa_bar(p) is the mean confidence over the neighbours that have a match (Eq. conf).
  * Normal: the eigenvector of the smallest eigenvalue of the covariance of the accepted points
    within radius plane_radius of X (X included), turned towards the reference camera; with
    fewer than 3 such points, the unit vector from X to the reference camera centre.
  * Tangent frame: t1, t2 from the normal by the branchless construction of Duff et al. (JCGT
    2017), so that [t1, t2, v] is a rotation; its quaternion (w, x, y, z) with w >= 0.
  * s_perp = det(J J^T)^(-1/4): the geometric mean of the two back-projected extents of one
    pixel through the projection Jacobian J at X in the reference view.
    s_par = min(s_perp (1 + err / 1 px) / sin(theta), s_par_cap s_perp) for the chosen
    hypothesis' error err and baseline angle theta.
  * Colour: per channel the median (mean of the two middle values for an even count) of the
    exposure-corrected bilinear samples (I - b) / g over the supporting views: the reference and
    every neighbour view with a match, where X projects in front of the camera with its
    bilinear footprint inside the image (pixel (x, y) is sampled at (x, y)). SH DC
    (c - 0.5) / Y_0, higher orders 0.
  * Opacity: alpha = alpha_lo + (alpha_hi - alpha_lo) kappa_bar (Eq. app-alpha-init), stored as
    a logit.
  * Subsampling for uniform coverage: at most one seed per cube of edge voxel (world space,
    cubes at integer multiples of voxel), the one with the highest kappa_bar as stored (rounded
    to float32), ties by the lower reference-pixel index; voxel = 0 keeps every seed.
"""
from __future__ import annotations

import math

import numpy as np

Y0 = 0.28209479177387814

DEFAULTS = dict(min_parallax=math.radians(1.0), max_reproj=2.0, tie_eps=1e-3, plane_radius=0.05,
                s_par_cap=10.0, alpha_lo=0.1, alpha_hi=0.9, voxel=0.0)


def _proj_matrix(cam):
    Kc = np.array([[cam["fx"], 0.0, cam["cx"]], [0.0, cam["fy"], cam["cy"]], [0.0, 0.0, 1.0]])
    Rt = np.c_[np.asarray(cam["R"], np.float64).reshape(3, 3),
               np.asarray(cam["t"], np.float64).reshape(3)]
    return Kc @ Rt


def _center(cam):
    R = np.asarray(cam["R"], np.float64).reshape(3, 3)
    return -R.T @ np.asarray(cam["t"], np.float64).reshape(3)


def _project(cam, X):
    R = np.asarray(cam["R"], np.float64).reshape(3, 3)
    xc = R @ X + np.asarray(cam["t"], np.float64).reshape(3)
    with np.errstate(divide="ignore", invalid="ignore"):  # a point at depth 0 is rejected later
        return np.array([cam["fx"] * xc[0] / xc[2] + cam["cx"],
                         cam["fy"] * xc[1] / xc[2] + cam["cy"]]), xc


def triangulate_pair(Pr, Pn, xr, xn):
    """Two-view DLT: the right singular vector of A for the smallest singular value, X = X~[:3] /
    X~[3] (Section 3.3). Returns X (or None when X~[3] = 0)."""
    A = np.stack([xr[0] * Pr[2] - Pr[0], xr[1] * Pr[2] - Pr[1],
                  xn[0] * Pn[2] - Pn[0], xn[1] * Pn[2] - Pn[1]])
    _, _, Vt = np.linalg.svd(A)
    Xh = Vt[-1]
    if Xh[3] == 0.0:
        return None
    return Xh[:3] / Xh[3]


def triangulate(cameras, ref_view, ref_xy, nb_view, nb_xy, nb_conf, config=None):
    """Best hypothesis per reference pixel. Returns dict: valid [M] bool, X [M,3], best [M]
    (neighbour slot, -1), err [M], angle [M], kappa [M], n_hyp [M] (hypotheses formed)."""
    c = dict(DEFAULTS, **(config or {}))
    M, K = np.asarray(nb_view).shape
    P = [_proj_matrix(cam) for cam in cameras]
    C = [_center(cam) for cam in cameras]
    out = dict(valid=np.zeros(M, bool), X=np.zeros((M, 3)), best=np.full(M, -1),
               err=np.zeros(M), angle=np.zeros(M), kappa=np.zeros(M), n_hyp=np.zeros(M, int))
    for m in range(M):
        r = int(ref_view[m])
        xr = np.asarray(ref_xy[m], np.float64)
        confs = [float(nb_conf[m][k]) for k in range(K) if nb_view[m][k] >= 0]
        out["kappa"][m] = float(np.mean(confs)) if confs else 0.0
        cands = []
        for k in range(K):
            n = int(nb_view[m][k])
            if n < 0:
                continue
            out["n_hyp"][m] += 1
            xn = np.asarray(nb_xy[m][k], np.float64)
            X = triangulate_pair(P[r], P[n], xr, xn)
            if X is None:
                continue
            pr, cr = _project(cameras[r], X)
            pn, cn = _project(cameras[n], X)
            if not (cr[2] > 0 and cn[2] > 0):
                continue
            err = math.sqrt(0.5 * (np.sum((pr - xr) ** 2) + np.sum((pn - xn) ** 2)))
            d1, d2 = X - C[r], X - C[n]
            cosang = float(d1 @ d2) / (np.linalg.norm(d1) * np.linalg.norm(d2))
            ang = math.acos(max(-1.0, min(1.0, cosang)))
            if ang < c["min_parallax"] or err > c["max_reproj"]:
                continue
            cands.append((err, ang, k, X))
        if not cands:
            continue
        emin = min(e for e, _, _, _ in cands)
        ties = [t for t in cands if t[0] <= emin + c["tie_eps"]]
        ties.sort(key=lambda t: (-t[1], t[2]))
        err, ang, k, X = ties[0]
        out["valid"][m] = True
        out["X"][m], out["best"][m], out["err"][m], out["angle"][m] = X, k, err, ang
    return out


def _frame(v):
    """Orthonormal t1, t2 with [t1, t2, v] a rotation (Duff et al., JCGT 6(1), 2017)."""
    s = 1.0 if v[2] >= 0.0 else -1.0
    a = -1.0 / (s + v[2])
    b = v[0] * v[1] * a
    t1 = np.array([1.0 + s * v[0] * v[0] * a, s * b, -s * v[0]])
    t2 = np.array([b, s + v[1] * v[1] * a, -v[1]])
    return t1, t2


def _quat_of(U):
    """(w, x, y, z), w >= 0, of the rotation U (Shepperd's method)."""
    tr = U[0, 0] + U[1, 1] + U[2, 2]
    if tr > 0:
        s = math.sqrt(tr + 1.0) * 2
        q = np.array([0.25 * s, (U[2, 1] - U[1, 2]) / s, (U[0, 2] - U[2, 0]) / s,
                      (U[1, 0] - U[0, 1]) / s])
    elif U[0, 0] > U[1, 1] and U[0, 0] > U[2, 2]:
        s = math.sqrt(1.0 + U[0, 0] - U[1, 1] - U[2, 2]) * 2
        q = np.array([(U[2, 1] - U[1, 2]) / s, 0.25 * s, (U[0, 1] + U[1, 0]) / s,
                      (U[0, 2] + U[2, 0]) / s])
    elif U[1, 1] > U[2, 2]:
        s = math.sqrt(1.0 + U[1, 1] - U[0, 0] - U[2, 2]) * 2
        q = np.array([(U[0, 2] - U[2, 0]) / s, (U[0, 1] + U[1, 0]) / s, 0.25 * s,
                      (U[1, 2] + U[2, 1]) / s])
    else:
        s = math.sqrt(1.0 + U[2, 2] - U[0, 0] - U[1, 1]) * 2
        q = np.array([(U[1, 0] - U[0, 1]) / s, (U[0, 2] + U[2, 0]) / s, (U[1, 2] + U[2, 1]) / s,
                      0.25 * s])
    q /= np.linalg.norm(q)
    return q if q[0] >= 0 else -q


def _bilinear(img, W, H, x, y):
    """Sample at (x, y) with pixel (i, j) at (i, j); None if the footprint leaves the image."""
    x0, y0 = math.floor(x), math.floor(y)
    if x0 < 0 or y0 < 0 or x0 + 1 > W - 1 or y0 + 1 > H - 1:
        return None
    fx, fy = x - x0, y - y0
    p = img.reshape(H, W, 3)
    return ((1 - fx) * (1 - fy) * p[y0, x0] + fx * (1 - fy) * p[y0, x0 + 1]
            + (1 - fx) * fy * p[y0 + 1, x0] + fx * fy * p[y0 + 1, x0 + 1])


def init_seeds(cameras, tri, ref_view, nb_view, observed, gain_bias, sh_degree=0, config=None):
    """Gaussian seeds of the accepted points (Eq. app-sigma-init, Eq. app-alpha-init).

    Returns dict with index [S] (reference-pixel index of each seed, increasing), means [S,3],
    log_scales [S,3], quats [S,4], opacity_logits [S], sh [S,K,3], normals [S,3]."""
    c = dict(DEFAULTS, **(config or {}))
    K = (sh_degree + 1) ** 2
    obs = np.asarray(observed, np.float64).reshape(-1, 3)
    offs = np.cumsum([0] + [int(cm["width"]) * int(cm["height"]) for cm in cameras])
    valid = np.nonzero(tri["valid"])[0]
    pts = tri["X"][valid]
    rows = []
    for j, m in enumerate(valid):
        X = pts[j]
        r = int(ref_view[m])
        cam = cameras[r]
        d = np.linalg.norm(pts - X, axis=1)
        nb = pts[d <= c["plane_radius"]]
        cr = _center(cam)
        if nb.shape[0] >= 3:
            cov = np.cov(nb.T, bias=True)
            w, V = np.linalg.eigh(cov)
            v = V[:, 0]
            if v @ (cr - X) < 0:
                v = -v
        else:
            v = (cr - X) / np.linalg.norm(cr - X)
        t1, t2 = _frame(v)
        U = np.stack([t1, t2, v], 1)
        # s_perp from the projection Jacobian at X in the reference view.
        _, xc = _project(cam, X)
        R = np.asarray(cam["R"], np.float64).reshape(3, 3)
        z = xc[2]
        Jc = np.array([[cam["fx"] / z, 0.0, -cam["fx"] * xc[0] / z ** 2],
                       [0.0, cam["fy"] / z, -cam["fy"] * xc[1] / z ** 2]]) @ R
        s_perp = np.linalg.det(Jc @ Jc.T) ** -0.25
        s_par = min(s_perp * (1.0 + tri["err"][m]) / math.sin(tri["angle"][m]),
                    c["s_par_cap"] * s_perp)
        # Colour: exposure-corrected bilinear samples over the supporting views.
        views = [r] + [int(n) for n in nb_view[m] if n >= 0]
        samples = []
        for vv in views:
            cmv = cameras[vv]
            p, xcv = _project(cmv, X)
            if not xcv[2] > 0:
                continue
            W, H = int(cmv["width"]), int(cmv["height"])
            s = _bilinear(obs[offs[vv]:offs[vv + 1]], W, H, p[0], p[1])
            if s is None:
                continue
            g, b = gain_bias[vv]
            samples.append((s - b) / g)
        col = np.median(np.array(samples), axis=0) if samples else np.full(3, 0.5)
        alpha = c["alpha_lo"] + (c["alpha_hi"] - c["alpha_lo"]) * tri["kappa"][m]
        sh = np.zeros((K, 3))
        sh[0] = (col - 0.5) / Y0
        rows.append(dict(index=m, mean=X, log_scales=np.log([s_perp, s_perp, s_par]),
                         quat=_quat_of(U), logit=math.log(alpha / (1.0 - alpha)), sh=sh,
                         normal=v, kappa=float(np.float32(tri["kappa"][m]))))
    if c["voxel"] > 0 and rows:
        best = {}
        for row in rows:
            key = tuple(np.floor(row["mean"] / c["voxel"]).astype(np.int64))
            cur = best.get(key)
            if cur is None or (row["kappa"], -row["index"]) > (cur["kappa"], -cur["index"]):
                best[key] = row
        rows = sorted(best.values(), key=lambda r_: r_["index"])
    S = len(rows)
    return dict(index=np.array([r_["index"] for r_ in rows], dtype=np.int64),
                means=np.array([r_["mean"] for r_ in rows]).reshape(S, 3),
                log_scales=np.array([r_["log_scales"] for r_ in rows]).reshape(S, 3),
                quats=np.array([r_["quat"] for r_ in rows]).reshape(S, 4),
                opacity_logits=np.array([r_["logit"] for r_ in rows]).reshape(S),
                sh=np.array([r_["sh"] for r_ in rows]).reshape(S, K, 3),
                normals=np.array([r_["normal"] for r_ in rows]).reshape(S, 3))
