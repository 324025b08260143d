"""Render a camera sequence of one of the benchmark's workloads with the
product configuration (persistent passes, fused tensor-core resolve, pass 2
merged above half size, 64-pixel quadtree base tiles), or with per-leaf pass
scales (--leaf), without timing: the command to put under a profiler.

    python -m paper_2606_16747_b300.render --workload hd --steps 8
"""
from __future__ import annotations

import argparse
import os

import numpy as np
import torch

from . import build, scenes
from . import star_nt as sn
from .pipeline import Renderer

HERE = os.path.dirname(os.path.abspath(__file__))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", default="hd", choices=["hd", "uhd"])
    ap.add_argument("--steps", type=int, default=8, help="real + interpolated frame pairs")
    ap.add_argument("--mlp", default="bf16", choices=["bf16", "fp8", "fp8x2"])
    ap.add_argument("--merge-scale2", type=float, default=0.5)
    ap.add_argument("--merge-scale3", type=float, default=0.7)
    ap.add_argument("--block-w", type=int, default=8, choices=[4, 8, 16])
    ap.add_argument("--base-tile", type=int, default=64, choices=[16, 64])
    ap.add_argument("--leaf", action="store_true", help="passes 2 and 3 at each leaf's Eq. 2 scale")
    args = ap.parse_args(argv)
    build.build()
    sc = scenes.hd_scene() if args.workload == "hd" else scenes.uhd_scene()
    W, H = sc.width, sc.height
    w = dict(np.load(os.path.join(HERE, "weights", "tail_mlp.npz")))
    r = Renderer(sc.verts, sc.rgba8, W, H, mlp=w, x_dtype=sn.BF16,
                 fused=args.mlp if args.mlp in ("fp8", "fp8x2") else True, persistent=True,
                 tuning=(args.block_w, 0, 0), merge_scale2=args.merge_scale2,
                 merge_scale3=args.merge_scale3, base_tile=args.base_tile,
                 leaf=args.leaf)
    cams = scenes.orbit_cameras(W, H, 2 * args.steps)
    vp32 = torch.tensor(np.stack([c.vp32 for c in cams]), device="cuda")
    vp64 = torch.tensor(np.stack([c.vp64.reshape(16) for c in cams]), device="cuda")
    for k in range(args.steps):
        r.set_cameras(vp32[2 * k], vp64[2 * k], vp64[2 * k + 1])
        r.step()
    torch.cuda.synchronize()
    r.check_status()
    if args.leaf:
        print("rendered", args.steps, "steps; targets", r.plan.sizes())
    else:
        print("rendered", args.steps, "steps; pass state", r.pass_state())


if __name__ == "__main__":
    main()
