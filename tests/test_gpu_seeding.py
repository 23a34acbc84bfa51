"""GPU tests of the dense initialisation (Section 3.3; Eq. app-sigma-init, Eq. app-alpha-init)
against the FP64 oracle in oracle/seeding.py, through the C ABI, on seeded synthetic matches of
a TUM-shaped keyframe window (noise 0.3 px, 5 % outliers):
  * triangulation: acceptance and chosen neighbour equal; point max-abs 1e-6 x (1 + |X|) (the
    smallest singular vector of a small-baseline system is determined only to about 3e-8
    relative, by LAPACK and by one-sided Jacobi alike: measured differences up to 1.3e-7 at
    |X| ~ 5); reprojection error 1e-4 px and angle 1e-7 rad, what that point difference moves
    them by; kappa exact;
  * seeds from the same accepted points: the same seeds; means, tangential log-scales, opacity
    logits max-abs 1e-6; axial log-scale 2e-4 (it moves with the error and angle above);
    normals and the quaternion's rotation max-abs 1e-5; SH DC max-abs 1e-5;
    with voxel thinning, the same kept set;
  * edge cases: m = 0, reference or neighbour views out of range;
  * the seeding scratch the context keeps, across calls that grow it and calls that reuse it.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import seeding as oseed
from paper_2601_00705_gb300 import binding, seeding, synthetic
from gpu_common import renderer

pytestmark = pytest.mark.gpu

F32 = lambda x: float(np.float32(x))  # noqa: E731  the C config holds FP32 constants


def _cfg(**kw):
    c = dict(oseed.DEFAULTS, **kw)
    return {k: F32(v) for k, v in c.items()}


def _case(m=4096, seed=1007):
    return synthetic.correspondences(seed=seed, m=m)


def _run_tri(c, cfg):
    r = renderer()
    tri = seeding.triangulate(r.ctx, c.cameras, c.ref_view, c.ref_xy, c.nb_view, c.nb_xy,
                              c.nb_conf, r.device, r.stream_handle(), **cfg)
    torch.cuda.synchronize()
    return r, tri


@pytest.mark.parametrize("m", [1, 777, 4096])
def test_triangulation_matches_oracle(m):
    c = _case(m=m)
    cfg = _cfg()
    r, tri = _run_tri(c, cfg)
    ref = oseed.triangulate(c.cameras, c.ref_view, c.ref_xy, c.nb_view, c.nb_xy, c.nb_conf,
                            config=cfg)
    valid = tri["valid"].cpu().numpy().astype(bool)
    np.testing.assert_array_equal(valid, ref["valid"])
    np.testing.assert_array_equal(tri["best"].cpu().numpy(), ref["best"])
    v = ref["valid"]
    X = tri["X"].cpu().numpy()
    assert np.all(np.abs(X[v] - ref["X"][v]) <= 1e-6 * (1 + np.abs(ref["X"][v])))
    np.testing.assert_allclose(tri["err"].cpu().numpy()[v], ref["err"][v], rtol=0, atol=1e-4)
    np.testing.assert_allclose(tri["angle"].cpu().numpy()[v], ref["angle"][v], rtol=0, atol=1e-7)
    np.testing.assert_array_equal(tri["kappa"].cpu().numpy(), ref["kappa"].astype(np.float32))
    if m > 100:
        assert 0.5 < v.mean() < 0.99


def _seed_both(c, cfg, sh_degree=0):
    r, tri = _run_tri(c, cfg)
    host_tri = dict(valid=tri["valid"].cpu().numpy().astype(bool), X=tri["X"].cpu().numpy(),
                    err=tri["err"].cpu().numpy(), angle=tri["angle"].cpu().numpy(),
                    kappa=tri["kappa"].cpu().numpy().astype(np.float64))
    gpu = seeding.init_seeds(r.ctx, c.cameras, tri, c.observed, c.gain_bias, r.device,
                             sh_degree=sh_degree, **cfg)
    gpu = {k: v.cpu().numpy() for k, v in gpu.items()}
    ref = oseed.init_seeds(c.cameras, host_tri, c.ref_view, c.nb_view, c.observed, c.gain_bias,
                           sh_degree=sh_degree, config=cfg)
    return gpu, ref


@pytest.mark.parametrize("voxel,sh_degree", [(0.0, 0), (0.0, 3), (0.15, 0)])
def test_seeds_match_oracle(voxel, sh_degree):
    c = _case(m=4096, seed=1008)
    cfg = _cfg(plane_radius=0.25, voxel=voxel)
    gpu, ref = _seed_both(c, cfg, sh_degree)
    np.testing.assert_array_equal(gpu["index"], ref["index"])
    assert len(ref["index"]) > 100
    for k in ("means", "opacity_logits"):
        np.testing.assert_allclose(gpu[k], ref[k], rtol=0, atol=1e-6, err_msg=k)
    np.testing.assert_allclose(gpu["log_scales"][:, :2], ref["log_scales"][:, :2], rtol=0,
                               atol=1e-6)
    # log s_par moves with the hypothesis' error and angle (1e-4 px, 1e-7 rad above).
    np.testing.assert_allclose(gpu["log_scales"][:, 2], ref["log_scales"][:, 2], rtol=0,
                               atol=2e-4)
    np.testing.assert_allclose(gpu["normals"], ref["normals"], rtol=0, atol=1e-5)
    Rg = oracle.quat_to_rotmat(gpu["quats"].astype(np.float64))
    Rr = oracle.quat_to_rotmat(ref["quats"])
    np.testing.assert_allclose(Rg, Rr, rtol=0, atol=1e-5)
    np.testing.assert_allclose(gpu["sh"], ref["sh"], rtol=0, atol=1e-5)
    if voxel:
        assert len(ref["index"]) < 0.9 * int(np.sum(_run_tri(c, cfg)[1]["valid"].cpu().numpy()))


def test_seeding_edge_cases():
    r = renderer()
    c = _case(m=64, seed=1009)
    cfg = _cfg()
    # m = 0: nothing to do.
    e = seeding.triangulate(r.ctx, c.cameras, c.ref_view[:0], c.ref_xy[:0], c.nb_view[:0],
                            c.nb_xy[:0], c.nb_conf[:0], r.device, r.stream_handle(), **cfg)
    assert e["valid"].numel() == 0
    # Out-of-range views: the pixel (reference) or the match (neighbour) is ignored.
    rv = c.ref_view.copy()
    nv = c.nb_view.copy()
    rv[0] = len(c.cameras)
    nv[1, :] = 99
    nv[2, 0] = -7
    tri = seeding.triangulate(r.ctx, c.cameras, rv, c.ref_xy, nv, c.nb_xy, c.nb_conf, r.device,
                              r.stream_handle(), **cfg)
    torch.cuda.synchronize()
    ref = oseed.triangulate(c.cameras, np.where(rv < len(c.cameras), rv, 0), c.ref_xy,
                            np.where((nv >= 0) & (nv < len(c.cameras)), nv, -1), c.nb_xy,
                            c.nb_conf, config=cfg)
    valid = tri["valid"].cpu().numpy().astype(bool)
    assert not valid[0] and not valid[1]
    np.testing.assert_array_equal(valid[2:], ref["valid"][2:])
    seeds = seeding.init_seeds(r.ctx, c.cameras, tri, c.observed, c.gain_bias, r.device, **cfg)
    assert 0 not in seeds["index"].cpu().numpy()
    with pytest.raises(binding.RGSError):
        seeding.triangulate(r.ctx, c.cameras, c.ref_view, c.ref_xy,
                            np.zeros((64, 9), np.int32), np.zeros((64, 9, 2)),
                            np.zeros((64, 9), np.float32), r.device, r.stream_handle(), **cfg)


def test_seed_scratch_grows_and_is_reused():
    # The context keeps the seeding scratch between calls: a small call, a larger one (the
    # scratch grows) and a small one again (reused) each match the oracle.
    cfg = _cfg(plane_radius=0.25)
    for m, seed in ((300, 1010), (4096, 1011), (300, 1012)):
        gpu, ref = _seed_both(_case(m=m, seed=seed), cfg)
        np.testing.assert_array_equal(gpu["index"], ref["index"], err_msg=str(m))
        np.testing.assert_allclose(gpu["means"], ref["means"], rtol=0, atol=1e-6, err_msg=str(m))
