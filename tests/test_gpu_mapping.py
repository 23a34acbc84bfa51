"""GPU tests of the mapping regulariser and maintenance (Eq. reg, Eq. app-ema, pruning bounds)
against oracle/mapping.py, through the C ABI, on a three-view scene:
  * the backward with the regulariser equals the plain backward plus the oracle's regulariser
    gradients (log-scales, logits, means; max-abs 1e-5 x (1 + |g|), the rest within atomics-order
    rounding), and the other gradients are unchanged; the value R within relative 1e-5;
  * observation counts equal the number of views in which each Gaussian has a touched tile (from
    the state's own records); visibility scores that number times alpha (relative 1e-6);
  * the anchor update and the prune mask equal the oracle's.
"""
import numpy as np
import pytest
import torch

from oracle import mapping as omap
from paper_2601_00705_gb300 import binding, synthetic
from paper_2601_00705_gb300.mapping import MapRegularizer
from gpu_common import renderer, to_dev

pytestmark = pytest.mark.gpu


def _scene():
    wl = synthetic.tiny(seed=31)
    base = wl.cameras[0]
    cams = [base,
            synthetic.camera(64, 48, 80.0, 80.0, 31.5, 23.5, np.eye(3), np.zeros(3)),
            synthetic.camera(120, 90, 110.0, 110.0, 59.5, 44.5, np.eye(3), [0.3, 0.0, 0.2])]
    return wl.gaussians.as_dict(), cams


def test_backward_with_regularizer_and_counters():
    g, cams = _scene()
    r = renderer()
    p = [to_dev(g[k]) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")]
    n, K, V = int(p[0].shape[0]), int(p[4].shape[1]), len(cams)
    color, depth, alpha, state = r.forward_raw(*p, cams)
    rng = np.random.default_rng(2)
    up = to_dev(rng.normal(0, 1e-3, size=tuple(color.shape)))
    base = r.backward_raw(state, n, K, V, up, None, None, binding.GRAD_ALL)
    ema = g["means"] + rng.normal(0, 0.05, size=g["means"].shape).astype(np.float32)
    mr = MapRegularizer(r.ctx, p[0], lambda_iso=10.0, lambda_alpha=0.1, lambda_mu=1.0)
    mr.ema_means.copy_(to_dev(ema))
    mr.obs_count.fill_(3)
    mr.vis_score.fill_(0.5)
    withreg = r.backward_raw(state, n, K, V, up, None, None, binding.GRAD_ALL, reg=mr.reg())
    torch.cuda.synchronize()
    val, d_ls, d_lg, d_mu = omap.regularizer(g["log_scales"], g["opacity_logits"], g["means"], ema,
                                             10.0, 0.1, 1.0)
    assert float(mr.value.item()) == pytest.approx(val, rel=1e-5)
    for key, ref in (("log_scales", d_ls), ("opacity_logits", d_lg), ("means", d_mu)):
        diff = (withreg[key] - base[key]).cpu().numpy().astype(np.float64)
        scale = 1.0 + np.abs(base[key].cpu().numpy())
        assert np.all(np.abs(diff - ref) <= 1e-5 * scale), key
    for key in ("quats", "sh", "pose"):
        a, b = withreg[key].cpu().numpy(), base[key].cpu().numpy()
        assert np.abs(a - b).max() <= 1e-5 * max(np.abs(b).max(), 1e-12), key
    # Counters: views in which each Gaussian has a touched tile, from the state's records.
    _, ntiles = r.ctx.records(state, V * n)
    seen = (np.asarray(ntiles).reshape(V, n) > 0).sum(0)
    assert seen.max() >= 2
    obs, vis = omap.counters(np.full(n, 3), np.full(n, 0.5), seen, g["opacity_logits"])
    np.testing.assert_array_equal(mr.obs_count.cpu().numpy(), obs)
    np.testing.assert_allclose(mr.vis_score.cpu().numpy(), vis, rtol=1e-6)
    r.release(state)


def test_anchor_update_and_prune_mask():
    rng = np.random.default_rng(5)
    n = 10007
    means = rng.normal(size=(n, 3)).astype(np.float32)
    ema = rng.normal(size=(n, 3)).astype(np.float32)
    r = renderer()
    mr = MapRegularizer(r.ctx, to_dev(ema), eta=0.2)
    mr.update_anchor(to_dev(means), r.stream_handle())
    torch.cuda.synchronize()
    np.testing.assert_allclose(mr.ema_means.cpu().numpy(), omap.ema(means, ema, np.float32(0.2)),
                               rtol=0, atol=1e-6)
    ls = rng.normal(-1.5, 1.0, size=(n, 3)).astype(np.float32)
    lg = rng.normal(-2.0, 3.0, size=n).astype(np.float32)
    obs = rng.integers(0, 10, size=n).astype(np.int32)
    vis = rng.uniform(0, 3, size=n).astype(np.float32)
    mr.obs_count.copy_(torch.from_numpy(obs).cuda())
    mr.vis_score.copy_(torch.from_numpy(vis).cuda())
    keep, n_keep = mr.prune_mask(to_dev(ls), to_dev(lg), r.stream_handle())
    torch.cuda.synchronize()
    ref = omap.prune_mask(ls, lg, obs, vis, min_opacity=np.float32(0.005), max_trace=1.0,
                          min_observations=5, min_visibility=1.0)
    got = keep.cpu().numpy().astype(bool)
    # Decisions within FP32 rounding of a bound may differ; there are none at these values.
    np.testing.assert_array_equal(got, ref)
    assert int(n_keep.item()) == int(ref.sum())
    assert 0 < ref.sum() < n
