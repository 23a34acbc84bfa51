"""Eager forward + backward steps of a synthetic workload in a fixed tile configuration, or
eager runs of the dense initialisation.

A driver for kernel profilers: it runs ``--steps`` batched steps through ``Renderer`` (the
library's public path) with no autotuning, no CUDA graph and no timing, so that a profiler's
launch filter (``-k`` / ``-s`` / ``-c``) sees exactly ``--steps`` launches of each kernel in
the order forward, backward. Prints the counters of the last forward. With ``--seeding M`` it
instead runs ``--steps`` triangulations and seed initialisations of M synthetic matched pixels
(up to 4 neighbours each, ten 640x480 keyframes).

    python -m paper_2601_00705_gb300.profile_step --workload tum --tile 16x16x8 --steps 2
    python -m paper_2601_00705_gb300.profile_step --seeding 131072 --steps 2
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import binding, synthetic
from .render import Renderer


def main(argv: list[str] | None = None) -> None:
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--workload", default="tum", choices=sorted(synthetic.WORKLOADS))
    p.add_argument("--tile", default="16x16x8", help="tile_w x tile_h x pixels per thread")
    p.add_argument("--backward-ppt", type=int, default=0,
                   help="pixels per thread of the backward blend (0: as the forward)")
    p.add_argument("--steps", type=int, default=2)
    p.add_argument("--seeding", type=int, default=0,
                   help="run the dense initialisation on this many matched pixels instead")
    args = p.parse_args(argv)
    if args.seeding:
        from . import seeding
        r = Renderer(torch.device("cuda", 0))
        c = synthetic.correspondences(m=args.seeding, k=4)
        for _ in range(args.steps):
            tri = seeding.triangulate(r.ctx, c.cameras, c.ref_view, c.ref_xy, c.nb_view, c.nb_xy,
                                      c.nb_conf, r.device, r.stream_handle())
            seeds = seeding.init_seeds(r.ctx, c.cameras, tri, c.observed, c.gain_bias, r.device)
        torch.cuda.synchronize()
        print(json.dumps({"seeding": args.seeding, "steps": args.steps,
                          "hypotheses": int((c.nb_view >= 0).sum()),
                          "accepted": int(tri["valid"].sum().item()),
                          "seeds": int(seeds["index"].numel())}))
        return
    tw, th, ppt = (int(x) for x in args.tile.split("x"))

    wl = synthetic.make(args.workload)
    g = wl.gaussians.as_dict()
    n, K, V = g["means"].shape[0], g["sh"].shape[1], len(wl.cameras)
    dev = torch.device("cuda", 0)

    def up(a):
        return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev)

    params = [up(g[k]) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")]
    d_color, d_depth, _ = synthetic.upstream(wl)
    d_color = up(d_color)
    d_depth = up(d_depth) if wl.depth_weight else None
    mask = binding.GRAD_POSE if wl.grad_mask == "pose" else binding.GRAD_ALL
    r = Renderer(dev, tile_w=tw, tile_h=th, pixels_per_thread=ppt,
                 backward_pixels_per_thread=args.backward_ppt)
    cams = binding.make_cameras(wl.cameras)
    state = 0
    for _ in range(args.steps):
        _, _, _, state = r.forward_raw(*params, cams, state=state)
        r.backward_raw(state, n, K, V, d_color, d_depth, None, mask)
    torch.cuda.synchronize(dev)
    print(json.dumps({"workload": args.workload, "tile": args.tile,
                      "backward_ppt": args.backward_ppt or ppt, "steps": args.steps,
                      "counters": r.stats(state)}))


if __name__ == "__main__":
    main()
