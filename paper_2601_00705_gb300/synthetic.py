"""Seeded synthetic scenes, cameras and upstream gradients for the rasterizer.

This module only draws inputs; it holds none of the renderer's arithmetic (no projection, no
compositing, no gradients). Both the CUDA path and the FP64 oracle are fed from it, so it must
stay free of either side's code.

Scenes stand in for the paper's Replica and TUM RGB-D sequences (Section 4), which are not
available: Gaussians are seeded on the surfaces of a 6 x 5 x 3 m room (six walls) plus spheres,
jittered along the surface normal, with random orientations, a spacing-derived scale, constant or
random opacity and SH colour coefficients. Cameras follow the five workload shapes:

  tiny      2,000 Gaussians in a slab in front of one 160x120 camera (identity pose), SH degree 0.
  replica   300k Gaussians on the room plus 20 spheres, one 1200x680 camera (f = 600), SH degree 0.
  tum       150k Gaussians, SH degree 3, a window of 10 keyframes at 640x480 (TUM intrinsics) on a
            1 m random walk through the room.
  uneven    1M Gaussians (room plus 200 clutter spheres), SH degree 3, 24 views whose resolution
            is drawn from {320x240, 640x480, 1200x680, 1920x1080}.
  large     3M Gaussians, log-scales N(-4, 0.7), SH degree 3, 16 views at 1920x1080 on a loop
            of radius 1.5 m around the room centre, looking outward.

Camera frames are x right, y down, z forward; a camera is a dict with width, height, fx, fy, cx,
cy and the world-to-camera rotation R [3,3] and translation t [3] (mu^C = R mu^W + t).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

ROOM = np.array([6.0, 5.0, 3.0])

WORKLOADS = ("tiny", "replica", "tum", "uneven", "large")
SEEDS = dict(tiny=1001, replica=1002, tum=1003, uneven=1004, large=1005, crowded=1006,
             seeding=1007)

# Intrinsics per resolution: TUM RGB-D (640x480) and half of it, Replica (1200x680), 1080p.
INTRINSICS = {
    (320, 240): (258.65, 258.25, 159.3, 127.65),
    (640, 480): (517.3, 516.5, 318.6, 255.3),
    (1200, 680): (600.0, 600.0, 599.5, 339.5),
    (1920, 1080): (960.0, 960.0, 959.5, 539.5),
}


@dataclass
class Gaussians:
    means: np.ndarray           # [N,3] float32, world frame
    log_scales: np.ndarray      # [N,3] float32
    quats: np.ndarray           # [N,4] float32, (w, x, y, z), not necessarily unit
    opacity_logits: np.ndarray  # [N] float32
    sh: np.ndarray              # [N,K,3] float32, K = (degree+1)^2

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def sh_degree(self) -> int:
        return int(round(self.sh.shape[1] ** 0.5)) - 1

    def as_dict(self) -> dict:
        return dict(means=self.means, log_scales=self.log_scales, quats=self.quats,
                    opacity_logits=self.opacity_logits, sh=self.sh)


@dataclass
class Workload:
    name: str
    gaussians: Gaussians
    cameras: list               # list of camera dicts
    grad_mask: str              # "all" or "pose"
    depth_weight: float         # weight of the depth L1 term in the upstream gradient

    @property
    def n_pixels(self) -> int:
        return int(sum(c["width"] * c["height"] for c in self.cameras))


def camera(width, height, fx, fy, cx, cy, R, t) -> dict:
    return dict(width=int(width), height=int(height), fx=float(fx), fy=float(fy), cx=float(cx),
                cy=float(cy), R=np.asarray(R, dtype=np.float32).reshape(3, 3),
                t=np.asarray(t, dtype=np.float32).reshape(3))


def camera_for(width, height, R, t) -> dict:
    fx, fy, cx, cy = INTRINSICS[(width, height)]
    return camera(width, height, fx, fy, cx, cy, R, t)


def look_pose(position, yaw, pitch):
    """World-to-camera (R, t) of a camera at `position` looking along (yaw, pitch), roll 0, z up."""
    fwd = np.array([math.cos(pitch) * math.cos(yaw), math.cos(pitch) * math.sin(yaw),
                    math.sin(pitch)])
    right = np.cross(fwd, np.array([0.0, 0.0, 1.0]))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])  # rows: camera axes in world coordinates
    t = -R @ np.asarray(position, dtype=np.float64)
    return R, t


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def _dc_from_rgb(rgb):
    # SH degree-0 basis value 1 / (2 sqrt(pi)); colour = dc * Y_0 + 0.5.
    return (rgb - 0.5) / (0.5 / math.sqrt(math.pi))


def _sample_spheres(rng, count, rmin, rmax, keep_clear=()):
    centres, radii = [], []
    while len(radii) < count:
        r = rng.uniform(rmin, rmax)
        lo = np.full(3, r + 0.3)
        c = rng.uniform(lo, ROOM - lo)
        if any(np.linalg.norm(c - p) - r < 0.4 for p in keep_clear):
            continue
        centres.append(c)
        radii.append(r)
    return np.array(centres), np.array(radii)


def _surface_points(rng, n, centres, radii, jitter=0.01):
    """n points on the room's six walls and the given spheres, uniform by area."""
    X, Y, Z = ROOM
    walls = [  # (origin, u-axis, v-axis, inward normal)
        ((0, 0, 0), (X, 0, 0), (0, Y, 0), (0, 0, 1)),
        ((0, 0, Z), (X, 0, 0), (0, Y, 0), (0, 0, -1)),
        ((0, 0, 0), (0, Y, 0), (0, 0, Z), (1, 0, 0)),
        ((X, 0, 0), (0, Y, 0), (0, 0, Z), (-1, 0, 0)),
        ((0, 0, 0), (X, 0, 0), (0, 0, Z), (0, 1, 0)),
        ((0, Y, 0), (X, 0, 0), (0, 0, Z), (0, -1, 0)),
    ]
    areas = [np.linalg.norm(np.cross(u, v)) for _, u, v, _ in walls]
    areas += list(4.0 * math.pi * radii ** 2)
    areas = np.array(areas)
    counts = rng.multinomial(n, areas / areas.sum())
    pts, nrm = [], []
    for k, (o, u, v, nn) in enumerate(walls):
        m = counts[k]
        a, b = rng.random(m), rng.random(m)
        pts.append(np.asarray(o) + a[:, None] * np.asarray(u) + b[:, None] * np.asarray(v))
        nrm.append(np.tile(np.asarray(nn, dtype=np.float64), (m, 1)))
    for s in range(len(radii)):
        m = counts[6 + s]
        d = rng.standard_normal((m, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        pts.append(centres[s] + radii[s] * d)
        nrm.append(d)
    P = np.concatenate(pts)
    Nn = np.concatenate(nrm)
    P = P + rng.normal(0.0, jitter, size=(P.shape[0], 1)) * Nn
    perm = rng.permutation(P.shape[0])
    return P[perm], float(areas.sum())


def _surface_gaussians(rng, n, degree, centres, radii, log_scale=None, opacity=0.9):
    means, area = _surface_points(rng, n, centres, radii)
    if log_scale is None:
        ls = math.log(math.sqrt(area / n)) + rng.normal(0.0, 0.1, size=(n, 3))
    else:
        ls = rng.normal(log_scale[0], log_scale[1], size=(n, 3))
    K = (degree + 1) ** 2
    sh = np.zeros((n, K, 3))
    sh[:, 0, :] = _dc_from_rgb(rng.random((n, 3)))
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.1, size=(n, K - 1, 3))
    logit = math.log(opacity / (1.0 - opacity))
    return Gaussians(means=means.astype(np.float32), log_scales=ls.astype(np.float32),
                     quats=_unit_quats(rng, n).astype(np.float32),
                     opacity_logits=np.full(n, logit, dtype=np.float32),
                     sh=sh.astype(np.float32))


def _position_ok(p, centres, radii, wall_margin=0.3, clearance=0.3):
    if np.any(p < wall_margin) or np.any(p > ROOM - wall_margin):
        return False
    if len(radii) and np.any(np.linalg.norm(centres - p, axis=1) - radii < clearance):
        return False
    return True


def _random_pose(rng, centres, radii):
    while True:
        p = rng.uniform([1.0, 1.0, 1.0], ROOM - 1.0)
        if _position_ok(p, centres, radii):
            return p, rng.uniform(0.0, 2.0 * math.pi), math.radians(rng.normal(0.0, 10.0))


def tiny(seed=SEEDS["tiny"], n=2000, width=160, height=120) -> Workload:
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(2, 5, n)], axis=1)
    g = Gaussians(
        means=means.astype(np.float32),
        log_scales=rng.normal(-3.5, 0.5, size=(n, 3)).astype(np.float32),
        quats=_unit_quats(rng, n).astype(np.float32),
        opacity_logits=rng.normal(0.0, 1.0, size=n).astype(np.float32),
        sh=_dc_from_rgb(rng.random((n, 1, 3))).astype(np.float32))
    cam = camera(width, height, 150.0, 150.0, (width - 1) / 2.0, (height - 1) / 2.0, np.eye(3),
                 np.zeros(3))
    return Workload("tiny", g, [cam], grad_mask="all", depth_weight=0.0)


def replica(seed=SEEDS["replica"], n=300_000) -> Workload:
    rng = np.random.default_rng(seed)
    centres, radii = _sample_spheres(rng, 20, 0.2, 0.6)
    g = _surface_gaussians(rng, n, 0, centres, radii)
    p, yaw, pitch = _random_pose(rng, centres, radii)
    R, t = look_pose(p, yaw, pitch)
    return Workload("replica", g, [camera_for(1200, 680, R, t)], grad_mask="pose",
                    depth_weight=0.1)


def tum(seed=SEEDS["tum"], n=150_000, n_views=10) -> Workload:
    rng = np.random.default_rng(seed)
    centres, radii = _sample_spheres(rng, 20, 0.2, 0.6)
    g = _surface_gaussians(rng, n, 3, centres, radii)
    p, yaw, pitch = _random_pose(rng, centres, radii)
    cams = []
    for _ in range(n_views):
        R, t = look_pose(p, yaw, pitch)
        cams.append(camera_for(640, 480, R, t))
        for _attempt in range(64):
            yaw += math.radians(rng.normal(0.0, 3.0))
            pitch = float(np.clip(pitch + math.radians(rng.normal(0.0, 3.0)), -0.5, 0.5))
            step = 0.1 * np.array([math.cos(yaw), math.sin(yaw), 0.0])
            if _position_ok(p + step, centres, radii, wall_margin=0.5):
                p = p + step
                break
            yaw += math.pi
    return Workload("tum", g, cams, grad_mask="all", depth_weight=0.0)


def uneven(seed=SEEDS["uneven"], n=1_000_000, n_views=24) -> Workload:
    rng = np.random.default_rng(seed)
    centres, radii = _sample_spheres(rng, 200, 0.05, 0.3)
    g = _surface_gaussians(rng, n, 3, centres, radii)
    sizes = [(320, 240), (640, 480), (1200, 680), (1920, 1080)]
    picks = rng.integers(0, 4, size=n_views)
    cams = []
    for k in picks:
        p, yaw, pitch = _random_pose(rng, centres, radii)
        R, t = look_pose(p, yaw, pitch)
        cams.append(camera_for(*sizes[k], R, t))
    return Workload("uneven", g, cams, grad_mask="all", depth_weight=0.0)


def large(seed=SEEDS["large"], n=3_000_000, n_views=16) -> Workload:
    rng = np.random.default_rng(seed)
    centre = ROOM / 2.0
    positions, yaws = [], []
    for k in range(n_views):
        th = 2.0 * math.pi * k / n_views
        positions.append(centre + 1.5 * np.array([math.cos(th), math.sin(th), 0.0]))
        yaws.append(th)
    centres, radii = _sample_spheres(rng, 200, 0.05, 0.3, keep_clear=positions)
    g = _surface_gaussians(rng, n, 3, centres, radii, log_scale=(-4.0, 0.7))
    cams = []
    for p, yaw in zip(positions, yaws):
        R, t = look_pose(p, yaw, 0.0)
        cams.append(camera_for(1920, 1080, R, t))
    return Workload("large", g, cams, grad_mask="all", depth_weight=0.0)


def crowded(seed=SEEDS["crowded"], n=12000, depth_levels=300) -> Workload:
    """A test scene for long tile lists: n small, faint Gaussians crowded in front of the centre
    of a 160x120 view (identity pose), so that a few tiles are each covered by thousands of
    them, and on only `depth_levels` distinct float32 depths, so that equal depths are common."""
    rng = np.random.default_rng(seed)
    z = (2.0 + 0.01 * rng.integers(0, depth_levels, size=n)).astype(np.float32)
    xy = rng.uniform(-0.01, 0.01, size=(n, 2)) * z[:, None]
    g = Gaussians(
        means=np.concatenate([xy, z[:, None]], axis=1).astype(np.float32),
        log_scales=(math.log(0.004) + rng.normal(0.0, 0.2, size=(n, 3))).astype(np.float32),
        quats=_unit_quats(rng, n).astype(np.float32),
        opacity_logits=np.full(n, -3.0, dtype=np.float32),
        sh=_dc_from_rgb(rng.random((n, 1, 3))).astype(np.float32))
    cam = camera(160, 120, 150.0, 150.0, 79.5, 59.5, np.eye(3), np.zeros(3))
    return Workload("crowded", g, [cam], grad_mask="all", depth_weight=0.0)


def make(name: str, **kw) -> Workload:
    return dict(tiny=tiny, replica=replica, tum=tum, uneven=uneven, large=large,
                crowded=crowded)[name](**kw)


def upstream(workload: Workload, seed: int = 2001):
    """Seeded upstream image gradients shaped like an L1 loss: +-1/P per colour channel, and
    +-depth_weight/P on depth; no gradient on accumulated opacity."""
    rng = np.random.default_rng(seed)
    P = workload.n_pixels
    d_color = (rng.integers(0, 2, size=(P, 3)) * 2 - 1).astype(np.float32) / P
    d_depth = ((rng.integers(0, 2, size=P) * 2 - 1).astype(np.float32) * workload.depth_weight / P
               if workload.depth_weight else np.zeros(P, dtype=np.float32))
    d_alpha = np.zeros(P, dtype=np.float32)
    return d_color, d_depth, d_alpha


def patch_mask(cameras, fraction=0.1, patch=16, seed=3001) -> np.ndarray:
    """Seeded mask of whole patch x patch pixel blocks, `fraction` of the blocks of every view."""
    rng = np.random.default_rng(seed)
    masks = []
    for c in cameras:
        W, H = c["width"], c["height"]
        px, py = (W + patch - 1) // patch, (H + patch - 1) // patch
        sel = rng.random((py, px)) < fraction
        m = np.kron(sel, np.ones((patch, patch), dtype=bool))[:H, :W]
        masks.append(m.reshape(-1))
    return np.concatenate(masks)


# ------------------------------------------------------------------------------------------
# Correspondences for the dense initialisation (the stand-in for matched keyframes): ground-truth
# surface points of the TUM-shaped room seen from a window of keyframes, their pixels in a
# reference view and in up to K neighbour views with Gaussian pixel noise, a share of outlier
# matches at random pixels, per-match confidences (inliers high, outliers low), observed frames
# with a smooth colour pattern per view and a per-view exposure (gain, bias).
# ------------------------------------------------------------------------------------------
@dataclass
class Correspondences:
    cameras: list
    ref_view: np.ndarray      # [M] int32
    ref_xy: np.ndarray        # [M,2] float64
    nb_view: np.ndarray       # [M,K] int32, -1: no match
    nb_xy: np.ndarray         # [M,K,2] float64
    nb_conf: np.ndarray       # [M,K] float32
    observed: np.ndarray      # [P,3] float32
    gain_bias: np.ndarray     # [V,2] float32
    points: np.ndarray        # [M,3] ground truth


def correspondences(seed=SEEDS["seeding"], m=2048, k=4, n_views=10, noise_px=0.3,
                    outlier_frac=0.05, width=640, height=480) -> Correspondences:
    rng = np.random.default_rng(seed)
    cams = tum(seed=SEEDS["tum"], n=16, n_views=n_views).cameras
    cams = [camera(width, height, *INTRINSICS[(640, 480)][:2],
                   (width - 1) / 2.0, (height - 1) / 2.0, c["R"], c["t"]) for c in cams]
    centres, radii = _sample_spheres(np.random.default_rng(SEEDS["tum"]), 20, 0.2, 0.6)

    def pix(v, X):  # pixels of points X [N,3] in view v and whether they are usable
        cam = cams[v]
        xc = X @ cam["R"].astype(np.float64).T + cam["t"].astype(np.float64)
        z = np.where(xc[:, 2] > 0.05, xc[:, 2], 1.0)
        uv = np.stack([cam["fx"] * xc[:, 0] / z + cam["cx"], cam["fy"] * xc[:, 1] / z + cam["cy"]], 1)
        ok = ((xc[:, 2] > 0.05) & (uv[:, 0] >= 1.0) & (uv[:, 0] <= width - 2.0)
              & (uv[:, 1] >= 1.0) & (uv[:, 1] <= height - 2.0))
        return uv, ok

    chunks = []
    have = 0
    while have < m:
        N = 4 * (m - have) + 64
        X = _surface_points(rng, N, centres, radii, jitter=0.0)[0].astype(np.float64)
        r = rng.integers(n_views, size=N)
        xr = np.zeros((N, 2))
        okr = np.zeros(N, bool)
        for v in range(n_views):
            sel = r == v
            uv, ok = pix(v, X[sel])
            xr[sel], okr[sel] = uv, ok
        nbv = np.full((N, k), -1, np.int64)
        nbx = np.zeros((N, k, 2))
        nbc = np.zeros((N, k))
        fill = np.zeros(N, np.int64)
        for j in range(k):  # the j-th nearest other view by index distance
            for v in range(n_views):
                sel = np.nonzero((r == v) & okr)[0]
                order = sorted([u for u in range(n_views) if u != v], key=lambda u: (abs(u - v), u))
                if j >= len(order) or sel.size == 0:
                    continue
                n = order[j]
                uv, ok = pix(n, X[sel])
                sel, uv = sel[ok], uv[ok]
                out = rng.random(sel.size) < outlier_frac
                noisy = uv + rng.normal(0.0, noise_px, uv.shape)
                rand = np.stack([rng.uniform(1, width - 2, sel.size), rng.uniform(1, height - 2, sel.size)], 1)
                slot = fill[sel]
                nbv[sel, slot] = n
                nbx[sel, slot] = np.where(out[:, None], rand, noisy)
                nbc[sel, slot] = np.where(out, rng.uniform(0.0, 0.4, sel.size), rng.uniform(0.6, 1.0, sel.size))
                fill[sel] += 1
        keep = np.nonzero(okr & (fill > 0))[0][:m - have]
        xr_noisy = xr[keep] + rng.normal(0.0, noise_px, (keep.size, 2))
        chunks.append((r[keep], xr_noisy, nbv[keep], nbx[keep], nbc[keep], X[keep]))
        have += keep.size
    ref_view = np.concatenate([c[0] for c in chunks]).astype(np.int32)
    ref_xy = np.concatenate([c[1] for c in chunks])
    nb_view = np.concatenate([c[2] for c in chunks]).astype(np.int32)
    nb_xy = np.concatenate([c[3] for c in chunks])
    nb_conf = np.concatenate([c[4] for c in chunks]).astype(np.float32)
    points = np.concatenate([c[5] for c in chunks])
    P = width * height
    obs = np.zeros((n_views * P, 3), np.float32)
    yy, xx = np.mgrid[0:height, 0:width].astype(np.float32)
    for v in range(n_views):
        f = rng.uniform(0.01, 0.05, size=(3, 2)).astype(np.float32)
        ph = rng.uniform(0, 2 * math.pi, size=3).astype(np.float32)
        for c in range(3):
            obs[v * P:(v + 1) * P, c] = (0.5 + 0.4 * np.sin(f[c, 0] * xx + f[c, 1] * yy + ph[c])).ravel()
    gain_bias = np.stack([rng.uniform(0.8, 1.2, n_views), rng.uniform(-0.05, 0.05, n_views)],
                         1).astype(np.float32)
    return Correspondences(cams, ref_view, ref_xy, nb_view, nb_xy, nb_conf, obs, gain_bias, points)
