"""The PyTorch front end and the library's failure paths, on the GPU.

* autograd: the torch.autograd.Function wrapper returns the library's gradients, which match
  the FP64 oracle and central finite differences of the GPU forward (the twist included);
* CUDA graphs: a captured forward + backward replays to the eager results;
* capacity: a pair list that outgrows its capacity during stream capture is reported through the
  status word, not written out of bounds, and the next eager call grows it and succeeds;
* argument validation: bad arguments and unknown handles come back as error codes.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2601_00705_gb300 import binding, synthetic
from paper_2601_00705_gb300.render import Renderer, render

from gpu_common import GRAD_REL_L2, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _scene(n=80, W=48, H=40, seed=5):
    wl = synthetic.tiny(seed=seed, n=n, width=W, height=H)
    # A rotated, translated camera so that every pose component matters.
    ang = 0.1
    R = np.array([[np.cos(ang), 0, np.sin(ang)], [0, 1, 0], [-np.sin(ang), 0, np.cos(ang)]])
    cam = dict(wl.cameras[0])
    cam["R"] = R.astype(np.float32)
    cam["t"] = np.array([0.05, -0.03, 0.1], np.float32)
    wl.cameras[0] = cam
    return wl


# Wide margins: pixels where a perturbation of the finite-difference size could flip a discrete
# decision (coverage, transmittance stop, clamps) get zero loss weight, so the loss is smooth
# in every parameter over the step.
FD_MARGINS = dict(margin_alpha=0.1, margin_t=0.1, margin_g=0.05, margin_effect=0.0,
                  margin_cont=1.0)


def _weights(orc, P, seed=0):
    rng = np.random.default_rng(seed)
    keep = (orc["ambiguous"] & oracle.BACKWARD_AMBIGUOUS) == 0
    wc = (rng.standard_normal((P, 3)) / P).astype(np.float32) * keep[:, None]
    wd = (rng.standard_normal(P) / P).astype(np.float32) * keep
    wa = (rng.standard_normal(P) / P).astype(np.float32) * keep
    return wc, wd, wa


def test_autograd_gradients_match_oracle_and_finite_differences():
    wl = _scene()
    g = wl.gaussians.as_dict()
    P = wl.n_pixels
    orc0 = oracle.render(g, wl.cameras, FD_MARGINS)
    wc, wd, wa = _weights(orc0, P)
    assert (wc != 0).any(axis=1).mean() > 0.5
    orc = oracle.render(g, wl.cameras, d_color=wc, d_depth=wd, d_alpha=wa)
    r = Renderer(0)
    params = {k: to_dev(v).requires_grad_(True) for k, v in g.items()}
    twist = torch.zeros((1, 6), device="cuda", requires_grad=True)
    wc_t, wd_t, wa_t = to_dev(wc), to_dev(wd), to_dev(wa)

    def loss_fn(p, cams, tw):
        c, d, a = render(r, cams, p["means"], p["log_scales"], p["quats"], p["opacity_logits"],
                         p["sh"], tw)
        if torch.is_grad_enabled():
            return (c * wc_t).sum() + (d * wd_t).sum() + (a * wa_t).sum()
        # Finite differences: sum in double so that the difference is not lost to rounding.
        return ((c.double() * wc_t.double()).sum() + (d.double() * wd_t.double()).sum() +
                (a.double() * wa_t.double()).sum())

    loss = loss_fn(params, wl.cameras, twist)
    loss.backward()
    pairs = [("means", "g_means"), ("log_scales", "g_log_scales"), ("quats", "g_quats"),
             ("opacity_logits", "g_opacity_logits"), ("sh", "g_sh")]
    for k, ok in pairs:
        assert rel_l2(params[k].grad.cpu().numpy(), orc[ok]) <= GRAD_REL_L2, k
    assert rel_l2(twist.grad.cpu().numpy(), orc["g_pose"]) <= GRAD_REL_L2

    # Central differences of the GPU forward (float32; h large enough to beat rounding) on
    # the largest-gradient coordinates of the means and on every twist component.
    with torch.no_grad():
        gm = params["means"].grad.abs().flatten()
        idx = torch.topk(gm, 6).indices.tolist()
        for flat in idx:
            h = 2e-4
            base = {k: v.detach().clone() for k, v in params.items()}
            plus = {k: v.clone() for k, v in base.items()}
            minus = {k: v.clone() for k, v in base.items()}
            plus["means"].view(-1)[flat] += h
            minus["means"].view(-1)[flat] -= h
            fd = (loss_fn(plus, wl.cameras, None) - loss_fn(minus, wl.cameras, None)) / (2 * h)
            an = params["means"].grad.view(-1)[flat]
            assert abs(float(fd - an)) <= 3e-2 * abs(float(an)) + 1e-7, (flat, float(fd), float(an))
        import scipy.linalg
        cam = wl.cameras[0]
        T = np.eye(4)
        T[:3, :3], T[:3, 3] = cam["R"], cam["t"]
        for k in range(6):
            vals = []
            for sgn in (1.0, -1.0):
                xi = np.zeros(6)
                xi[k] = sgn * 2e-4
                M = np.zeros((4, 4))
                w = xi[3:]
                M[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
                M[:3, 3] = xi[:3]
                Tn = scipy.linalg.expm(M) @ T
                c2 = dict(cam)
                c2["R"], c2["t"] = Tn[:3, :3].astype(np.float32), Tn[:3, 3].astype(np.float32)
                vals.append(float(loss_fn(params, [c2], None)))
            fd = (vals[0] - vals[1]) / 4e-4
            an = float(twist.grad[0, k])
            assert abs(fd - an) <= 3e-2 * abs(an) + 2e-6, (k, fd, an)


@pytest.mark.parametrize("scene,tile", [
    ("tum3", (16, 16, 4)), ("tiny", (8, 8, 1)), ("tiny", (16, 16, 4)), ("tiny", (32, 8, 2)),
    ("tiny", (16, 16, 8))])
def test_cuda_graph_replay_matches_eager(scene, tile):
    # Small scenes keep every sort and scan short, so the whole launch chain of a step is made of
    # brief kernels; the 3-view window has sorts of 10^5 keys and more.
    wl = synthetic.tum(n=20_000, n_views=3) if scene == "tum3" else synthetic.tiny()
    g = wl.gaussians.as_dict()
    n, K, V = g["means"].shape[0], g["sh"].shape[1], len(wl.cameras)
    P = wl.n_pixels
    r = Renderer(0, tile_w=tile[0], tile_h=tile[1], pixels_per_thread=tile[2])
    params = [to_dev(g[k]) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")]
    up = to_dev(np.random.default_rng(1).standard_normal((P, 3)).astype(np.float32) / P)
    cams = binding.make_cameras(wl.cameras)
    imgs = (torch.empty((P, 3), device="cuda"), torch.empty(P, device="cuda"),
            torch.empty(P, device="cuda"))
    shapes = dict(means=(n, 3), log_scales=(n, 3), quats=(n, 4), opacity_logits=(n,),
                  sh=(n, K, 3), pose=(V, 6))
    grads = {k: torch.empty(s, device="cuda") for k, s in shapes.items()}

    def step(state):
        _, _, _, state = r.forward_raw(*params, cams, state=state, out=imgs)
        r.backward_raw(state, n, K, V, up, None, None, binding.GRAD_ALL, out=grads)
        return state

    state = step(0)
    torch.cuda.synchronize()
    eager_img = [t.clone() for t in imgs]
    eager_grad = {k: v.clone() for k, v in grads.items()}
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            step(state)
    torch.cuda.current_stream().wait_stream(s)
    for t in list(imgs) + list(grads.values()):
        t.zero_()
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    for a, b in zip(imgs, eager_img):
        assert torch.equal(a, b)
    for k in grads:
        assert rel_l2(grads[k].cpu().numpy(), eager_grad[k].cpu().numpy()) <= 1e-5, k
    st = r.stats(state)
    assert st["n_eval"] > 0, st
    r.release(state)


def test_pair_overflow_under_capture_is_reported_then_recovered():
    wl = synthetic.tiny(n=3000, width=128, height=96)
    g = wl.gaussians.as_dict()
    P = wl.n_pixels
    r = Renderer(0)
    small = {k: to_dev(v) for k, v in g.items()}
    big = dict(small)
    big["log_scales"] = small["log_scales"] + 2.5  # much larger footprints: many more pairs
    imgs = (torch.empty((P, 3), device="cuda"), torch.empty(P, device="cuda"),
            torch.empty(P, device="cuda"))
    keys = ("means", "log_scales", "quats", "opacity_logits", "sh")
    _, _, _, state = r.forward_raw(*[small[k] for k in keys], wl.cameras, out=imgs)
    torch.cuda.synchronize()
    cap = r.stats(state)["pair_capacity"]
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            r.forward_raw(*[big[k] for k in keys], wl.cameras, state=state, out=imgs)
    torch.cuda.current_stream().wait_stream(s)
    graph.replay()
    torch.cuda.synchronize()
    st = r.stats(state)
    assert st["n_pairs"] > cap and st["status"] & 1, st
    # Outside capture the same call grows the list and renders completely.
    _, _, _, state = r.forward_raw(*[big[k] for k in keys], wl.cameras, state=state, out=imgs)
    torch.cuda.synchronize()
    st2 = r.stats(state)
    assert st2["status"] == 0 and st2["pair_capacity"] >= st2["n_pairs"] == st["n_pairs"]
    r.release(state)


def test_visible_overflow_under_capture_is_reported_then_recovered():
    wl = synthetic.tiny(n=20000, width=128, height=96)
    g = wl.gaussians.as_dict()
    P = wl.n_pixels
    r = Renderer(0)
    keys = ("means", "log_scales", "quats", "opacity_logits", "sh")
    full = {k: to_dev(v) for k, v in g.items()}
    few = dict(full)
    means = g["means"].copy()
    means[2000:, 0] += 100.0  # all but 2000 Gaussians far outside the view
    few["means"] = to_dev(means)
    imgs = (torch.empty((P, 3), device="cuda"), torch.empty(P, device="cuda"),
            torch.empty(P, device="cuda"))
    _, _, _, state = r.forward_raw(*[few[k] for k in keys], wl.cameras, out=imgs)
    torch.cuda.synchronize()
    seen = r.stats(state)["n_visible"]
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            r.forward_raw(*[full[k] for k in keys], wl.cameras, state=state, out=imgs)
    torch.cuda.current_stream().wait_stream(s)
    graph.replay()
    torch.cuda.synchronize()
    st = r.stats(state)
    # The stats give the true visible count; the entries beyond the capacity were dropped.
    assert st["status"] & 2 and st["n_visible"] > 5 * seen, (seen, st)
    # Outside capture the same call sizes the list from the true count and renders completely,
    # exactly as a fresh state does.
    _, _, _, state = r.forward_raw(*[full[k] for k in keys], wl.cameras, state=state, out=imgs)
    torch.cuda.synchronize()
    st2 = r.stats(state)
    assert st2["status"] == 0 and st2["n_visible"] == st["n_visible"], st2
    assert st2["n_pairs"] > st["n_pairs"], (st, st2)
    got = [t.clone() for t in imgs]
    r2 = Renderer(0)
    ref = r2.forward_raw(*[full[k] for k in keys], wl.cameras)
    torch.cuda.synchronize()
    for a, b in zip(got, ref[:3]):
        assert torch.equal(a, b)
    r.release(state)
    r2.release(ref[3])


def test_invalid_arguments_and_handles_return_error_codes():
    lib = binding.load()
    r = Renderer(0)
    ctx = r.ctx
    wl = synthetic.tiny(n=10)
    g = {k: to_dev(v) for k, v in wl.gaussians.as_dict().items()}
    cams = binding.make_cameras(wl.cameras)
    P = wl.n_pixels
    out = binding.Images(torch.empty((P, 3), device="cuda").data_ptr(),
                         torch.empty(P, device="cuda").data_ptr(),
                         torch.empty(P, device="cuda").data_ptr())

    def gauss(**kw):
        d = dict(n=10, deg=0, means=g["means"].data_ptr(), ls=g["log_scales"].data_ptr(),
                 q=g["quats"].data_ptr(), o=g["opacity_logits"].data_ptr(), sh=g["sh"].data_ptr())
        d.update(kw)
        return binding.Gaussians(d["n"], d["deg"], d["means"], d["ls"], d["q"], d["o"], d["sh"])

    def fwd(gs, n_views=1, cfg=None):
        h = ctypes.c_uint64(0)
        return lib.rgs_render_forward(ctx.handle, ctypes.byref(gs), cams, n_views,
                                      ctypes.byref(cfg or r.config), ctypes.byref(out),
                                      ctypes.byref(h), None)

    assert fwd(gauss(), n_views=0) == binding.RGS_ERR_INVALID_ARG
    assert fwd(gauss(), n_views=binding.RGS_MAX_VIEWS + 1) == binding.RGS_ERR_INVALID_ARG
    assert fwd(gauss(deg=4)) == binding.RGS_ERR_INVALID_ARG
    assert fwd(gauss(n=-1)) == binding.RGS_ERR_INVALID_ARG
    assert fwd(gauss(means=g["means"].data_ptr() + 4)) == binding.RGS_ERR_INVALID_ARG
    assert fwd(gauss(q=0)) == binding.RGS_ERR_INVALID_ARG
    bad = binding.default_config(tile_w=12, tile_h=12)
    assert fwd(gauss(), cfg=bad) == binding.RGS_ERR_INVALID_ARG
    bad = binding.default_config(tile_w=8, tile_h=8, pixels_per_thread=4)
    assert fwd(gauss(), cfg=bad) == binding.RGS_ERR_INVALID_ARG
    bad = binding.default_config(tile_w=8, tile_h=8, pixels_per_thread=2,
                                 backward_pixels_per_thread=8)
    assert fwd(gauss(), cfg=bad) == binding.RGS_ERR_INVALID_ARG
    bad = binding.default_config(backward_pixels_per_thread=3)
    assert fwd(gauss(), cfg=bad) == binding.RGS_ERR_INVALID_ARG
    bad = binding.default_config(znear=-1.0)
    assert fwd(gauss(), cfg=bad) == binding.RGS_ERR_INVALID_ARG
    grads = binding.ImageGrads(None, None, None)
    st = lib.rgs_render_backward(ctx.handle, ctypes.c_uint64(987654), ctypes.byref(grads), 63,
                                 None, None, None, None, None, None, None)
    assert st == binding.RGS_ERR_STATE
    assert lib.rgs_release_state(ctx.handle, ctypes.c_uint64(987654)) == binding.RGS_ERR_STATE
    # A valid forward, then a backward asking for a gradient it gives no buffer for.
    h = ctypes.c_uint64(0)
    assert lib.rgs_render_forward(ctx.handle, ctypes.byref(gauss()), cams, 1,
                                  ctypes.byref(r.config), ctypes.byref(out), ctypes.byref(h),
                                  None) == binding.RGS_OK
    st = lib.rgs_render_backward(ctx.handle, h, ctypes.byref(grads), binding.GRAD_MEANS,
                                 None, None, None, None, None, None, None)
    assert st == binding.RGS_ERR_INVALID_ARG
    assert lib.rgs_release_state(ctx.handle, h) == binding.RGS_OK
    assert lib.rgs_release_state(ctx.handle, h) == binding.RGS_ERR_STATE


def test_sh_event_defers_the_wait_for_the_coefficients():
    # The coefficients reach the device only after a long wait on a side stream; the forward,
    # given the event, must wait for them where it first reads them and render exactly what a
    # forward on resident coefficients renders (a forward that read them early would see
    # zeros). The backward then runs on the same stream.
    wl = synthetic.tiny(seed=5)
    g = wl.gaussians.as_dict()
    rng = np.random.default_rng(5)
    sh3 = np.concatenate([g["sh"], rng.normal(0, 0.1, size=(g["sh"].shape[0], 15, 3))],
                         axis=1).astype(np.float32)
    keys = ("means", "log_scales", "quats", "opacity_logits")
    p = [to_dev(g[k]) for k in keys]
    sh = to_dev(sh3)
    n, K, V = int(p[0].shape[0]), 16, len(wl.cameras)
    P = wl.n_pixels
    up = to_dev(rng.normal(0, 1e-3, size=(P, 3)))
    r = Renderer(0)
    ref = r.forward_raw(*p, sh, wl.cameras)
    ref_g = r.backward_raw(ref[3], n, K, V, up, None, None, binding.GRAD_ALL)
    torch.cuda.synchronize()
    r2 = Renderer(0)
    late = torch.zeros_like(sh)
    side = torch.cuda.Stream()
    ev = torch.cuda.Event()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        torch.cuda._sleep(100_000_000)  # ~50 ms of GPU cycles before the copy
        late.copy_(sh)
        ev.record(side)
    got = r2.forward_raw(*p, late, wl.cameras, sh_event=ev)
    got_g = r2.backward_raw(got[3], n, K, V, up, None, None, binding.GRAD_ALL)
    torch.cuda.synchronize()
    for a, b in zip(got[:3], ref[:3]):
        assert torch.equal(a, b)
    # Gradients are sums of float atomics whose order varies from run to run: equal to about
    # 1e-6 of the largest entry, not bit for bit.
    for k in ("means", "sh", "pose"):
        np.testing.assert_allclose(got_g[k].cpu().numpy(), ref_g[k].cpu().numpy(), rtol=1e-5,
                                   atol=1e-6 * float(ref_g[k].abs().max()))
    assert r2.stats(got[3])["status"] == 0
    r.release(ref[3])
    r2.release(got[3])


def test_deferred_colours_treat_nonfinite_sh_like_the_projection():
    # With an SH event the colours are evaluated after the sorts, and an entry with a non-finite
    # coefficient is kept in the lists but covers no pixel; without one the projection culls it.
    # Images are identical and gradients agree; both count the entry as culled.
    wl = synthetic.tiny(n=300)
    g = {k: v.copy() for k, v in wl.gaussians.as_dict().items()}
    proj = oracle.project(g, wl.cameras)
    m2 = proj["mean2d"][0]
    on = np.nonzero(proj["valid"][0] & (m2[:, 0] > 10) & (m2[:, 0] < 150) & (m2[:, 1] > 10) &
                    (m2[:, 1] < 110))[0]
    bad = int(on[5])
    g["sh"][bad, 0, 1] = np.nan
    keys = ("means", "log_scales", "quats", "opacity_logits", "sh")
    p = [to_dev(g[k]) for k in keys]
    n, K, V, P = 300, int(g["sh"].shape[1]), len(wl.cameras), wl.n_pixels
    up = to_dev(np.random.default_rng(7).normal(0, 1e-3, size=(P, 3)))
    ev = torch.cuda.Event()
    ev.record()
    outs = []
    for kw in ({}, {"sh_event": ev}):
        r = Renderer(0)
        c, d, a, st = r.forward_raw(*p, wl.cameras, **kw)
        gr = r.backward_raw(st, n, K, V, up, None, None, binding.GRAD_ALL)
        torch.cuda.synchronize()
        outs.append(((c, d, a), gr, r.stats(st)))
        r.release(st)
    (img0, g0, s0), (img1, g1, s1) = outs
    for x, y in zip(img0, img1):
        assert torch.equal(x, y)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "pose"):
        a0, a1 = g0[k].cpu().numpy(), g1[k].cpu().numpy()
        assert np.isfinite(a1).all(), k
        # Sums of float atomics in a run-dependent order (see above).
        np.testing.assert_allclose(a1, a0, rtol=1e-5, atol=1e-6 * float(np.abs(a0).max()))
    assert not g1["means"][bad].any() and not g1["sh"][bad].any()
    assert s0["n_nonfinite"] == 1 and s1["n_nonfinite"] == 1
    assert s0["status"] == 0 and s1["status"] == 0
