"""Pins of the dense-initialisation oracle (oracle/seeding.py) to things other than itself.

  * two-view DLT: noise-free points are recovered exactly; swapping the two views gives the same
    point; the result is invariant to scaling the homogeneous system;
  * hypothesis selection: a planted case whose errors and angles are known by construction
    (a noisy neighbour loses to exact ones, a tie goes to the larger baseline angle, a neighbour
    at the reference camera's centre is rejected for parallax, an outlier for its error);
  * kappa_bar is the mean of the matched confidences;
  * seeds: points on a known plane give its normal (towards the camera); a point on the optical
    axis of a camera with f = fx = fy gives s_perp = z / f exactly; s_par by its formula and its
    cap; constant observed frames give colour (I - b) / g and the SH DC term; an even number of
    samples gives the mean of the middle two; the quaternion maps to [t1, t2, v] through the
    rasterizer oracle's quaternion convention; the opacity logit of Eq. app-alpha-init; voxel
    thinning keeps the highest confidence, then the lowest index.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import seeding


def _cam(R=np.eye(3), t=np.zeros(3), f=500.0, W=640, H=480):
    return dict(width=W, height=H, fx=f, fy=f, cx=(W - 1) / 2, cy=(H - 1) / 2,
                R=np.asarray(R, float), t=np.asarray(t, float))


def _rot(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def _px(cam, X):
    return seeding._project(cam, np.asarray(X, float))[0]


def _pose_at(center, R):
    return dict(R=R, t=-R @ np.asarray(center, float))


def test_dlt_recovers_noise_free_points_and_is_symmetric():
    rng = np.random.default_rng(0)
    for _ in range(20):
        c1 = _cam(**_pose_at(rng.normal(size=3) * 0.2, _rot(rng.normal(size=3), 0.1)))
        c2 = _cam(**_pose_at(rng.normal(size=3) * 0.2 + [0.3, 0, 0], _rot(rng.normal(size=3), 0.1)))
        X = np.array([0.0, 0.0, 3.0]) + rng.normal(size=3) * 0.5
        P1, P2 = seeding._proj_matrix(c1), seeding._proj_matrix(c2)
        x1, x2 = _px(c1, X), _px(c2, X)
        Xa = seeding.triangulate_pair(P1, P2, x1, x2)
        Xb = seeding.triangulate_pair(P2, P1, x2, x1)
        np.testing.assert_allclose(Xa, X, rtol=0, atol=1e-9)
        np.testing.assert_allclose(Xb, Xa, rtol=0, atol=1e-9)
        np.testing.assert_allclose(seeding.triangulate_pair(3.0 * P1, 0.5 * P2, x1, x2), Xa,
                                   rtol=0, atol=1e-9)


def test_hypothesis_selection_on_a_planted_case():
    X = np.array([0.2, -0.1, 3.0])
    ref = _cam()
    near = _cam(**_pose_at([0.1, 0.0, 0.0], np.eye(3)))   # small baseline
    far = _cam(**_pose_at([0.3, 0.0, 0.0], np.eye(3)))    # larger baseline
    same = _cam(**_pose_at([0.0, 0.0, 0.0], _rot([0, 1, 0], 0.05)))  # same centre: no parallax
    cams = [ref, near, far, same]
    xr = _px(ref, X)
    nb_view = np.array([[1, 2, 3, 2]])
    # Offsets across the epipolar lines (the baselines are along x): along them a wrong match
    # only moves the depth and reprojects exactly.
    nb_xy = np.array([[_px(near, X), _px(far, X), _px(same, X), _px(far, X) + [0.0, 5.0]]])
    conf = np.array([[0.9, 0.7, 0.8, 0.2]], np.float32)
    tri = seeding.triangulate(cams, np.array([0]), xr[None], nb_view, nb_xy, conf)
    # Exact neighbours 1 and 2 tie (error ~0); the larger baseline (view 2, slot 1) wins; the
    # same-centre view has no parallax; slot 3 is 5 px off its epipolar line (RMS 2.5 > 2).
    assert tri["valid"][0] and tri["best"][0] == 1
    np.testing.assert_allclose(tri["X"][0], X, atol=1e-9)
    assert tri["err"][0] < 1e-6
    assert tri["kappa"][0] == pytest.approx(np.mean(conf.astype(np.float64)))
    # With the exact far neighbour removed, the near one wins; with only the bad ones, nothing.
    tri2 = seeding.triangulate(cams, np.array([0]), xr[None], np.array([[1, -1, 3, 2]]), nb_xy, conf)
    assert tri2["best"][0] == 0
    tri3 = seeding.triangulate(cams, np.array([0]), xr[None], np.array([[-1, -1, 3, 2]]), nb_xy, conf)
    assert not tri3["valid"][0]
    # A 1 px error on the far neighbour: accepted, and it loses the tie to the exact near one.
    nb_xy4 = nb_xy.copy()
    nb_xy4[0, 1] += [0.0, 1.0]
    tri4 = seeding.triangulate(cams, np.array([0]), xr[None], nb_view, nb_xy4, conf)
    assert tri4["best"][0] == 0


def _seed_case(points, cams, ref=0, nb=1):
    M = len(points)
    ref_view = np.full(M, ref)
    ref_xy = np.array([_px(cams[ref], X) for X in points])
    nb_view = np.full((M, 1), nb)
    nb_xy = np.array([[_px(cams[nb], X)] for X in points])
    conf = np.full((M, 1), 0.75, np.float32)
    tri = seeding.triangulate(cams, ref_view, ref_xy, nb_view, nb_xy, conf,
                              config=dict(min_parallax=0.0))
    return tri, ref_view, nb_view


def test_plane_normal_axis_scale_and_frame():
    cams = [_cam(), _cam(**_pose_at([0.4, 0.0, 0.0], np.eye(3)))]
    rng = np.random.default_rng(1)
    n = np.array([0.2, -0.3, -1.0])
    n /= np.linalg.norm(n)
    base = np.array([0.0, 0.0, 3.0])
    t1 = np.cross(n, [1.0, 0.0, 0.0])
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(n, t1)
    pts = [base + a * t1 + b * t2 for a, b in rng.uniform(-0.04, 0.04, size=(30, 2))]
    pts[0] = base.copy()  # on the optical axis of the reference camera
    tri, rv, nv = _seed_case(pts, cams)
    obs = np.full((2 * 640 * 480, 3), 0.6)
    gb = np.array([[1.2, 0.05], [0.8, -0.02]])
    seeds = seeding.init_seeds(cams, tri, rv, nv, obs, gb, config=dict(plane_radius=0.2))
    assert list(seeds["index"]) == list(range(30))
    # Normal of the plane, turned towards the reference camera at the origin (n already faces it:
    # n . (0 - X) > 0).
    np.testing.assert_allclose(seeds["normals"], np.tile(n, (30, 1)), atol=1e-9)
    # On the axis of a camera with f = 500: s_perp = z / f.
    assert math.exp(seeds["log_scales"][0, 0]) == pytest.approx(3.0 / 500.0, rel=1e-9)
    s_perp, err, ang = 3.0 / 500.0, tri["err"][0], tri["angle"][0]
    assert math.exp(seeds["log_scales"][0, 2]) == pytest.approx(
        min(s_perp * (1 + err) / math.sin(ang), 10 * s_perp), rel=1e-9)
    # Rotation of the quaternion (rasterizer oracle's convention) is [t1, t2, v].
    for i in range(30):
        R = oracle.quat_to_rotmat(seeds["quats"][i][None])[0]
        np.testing.assert_allclose(R[:, 2], seeds["normals"][i], atol=1e-12)
        np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-12)
        assert np.linalg.det(R) == pytest.approx(1.0)
        assert seeds["quats"][i][0] >= 0
    # Median of (0.6 - b) / g over the two views: the mean of the two middle values.
    col = np.mean([(0.6 - 0.05) / 1.2, (0.6 + 0.02) / 0.8])
    np.testing.assert_allclose(seeds["sh"][:, 0], (col - 0.5) / seeding.Y0, rtol=1e-12)
    a = 0.1 + 0.8 * 0.75
    np.testing.assert_allclose(seeds["opacity_logits"], math.log(a / (1 - a)), rtol=1e-6)


def test_normal_without_neighbours_faces_the_camera_and_s_par_cap():
    cams = [_cam(), _cam(**_pose_at([0.05, 0.0, 0.0], np.eye(3)))]
    X = np.array([0.3, 0.2, 4.0])
    tri, rv, nv = _seed_case([X], cams)
    seeds = seeding.init_seeds(cams, tri, rv, nv, np.full((2 * 640 * 480, 3), 0.5),
                               np.array([[1.0, 0.0], [1.0, 0.0]]))
    np.testing.assert_allclose(seeds["normals"][0], -X / np.linalg.norm(X), atol=1e-12)
    # Baseline angle ~0.7 degrees: 1 / sin is above 10, so the cap holds.
    assert seeds["log_scales"][0, 2] - seeds["log_scales"][0, 0] == pytest.approx(math.log(10.0))


def test_voxel_thinning_keeps_highest_confidence_then_lowest_index():
    cams = [_cam(), _cam(**_pose_at([0.4, 0.0, 0.0], np.eye(3)))]
    pts = [np.array([0.01, 0.01, 3.01]), np.array([0.02, 0.03, 3.02]),
           np.array([0.03, 0.02, 3.03]), np.array([0.55, 0.5, 3.3])]
    tri, rv, nv = _seed_case(pts, cams)
    tri["kappa"][:] = [0.5, 0.9, 0.9, 0.1]
    obs = np.full((2 * 640 * 480, 3), 0.5)
    gb = np.array([[1.0, 0.0], [1.0, 0.0]])
    seeds = seeding.init_seeds(cams, tri, rv, nv, obs, gb, config=dict(voxel=0.1))
    # Points 0-2 share the cube [0, 0.1)^2 x [3.0, 3.1); 1 and 2 tie on confidence: 1 is kept.
    assert list(seeds["index"]) == [1, 3]
