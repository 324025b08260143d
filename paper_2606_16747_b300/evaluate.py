"""Quality of a camera sequence against the exact A-buffer (the evaluation of
Sec. 4 on the synthetic workloads): every frame of an orbit rendered by
STAR-NT (real and interpolated frames alternating; pass scales from Eq. 2
over the frame, and per quadtree leaf), by the plain
full-resolution neural pipeline, by weighted blended OIT and by naive
unsorted blending, each compared with the exact A-buffer of its camera.

    python -m paper_2606_16747_b300.evaluate --workload hd --frames 120
"""
from __future__ import annotations

import argparse
import json
import math
import os

import numpy as np
import torch

from . import build, scenes
from . import star_nt as sn
from .pipeline import Renderer

HERE = os.path.dirname(os.path.abspath(__file__))


def exact_and_frags(r: Renderer, vp32):
    """Exact A-buffer colour of camera vp32 (and its fragment lists)."""
    W, H, P = r.W, r.H, r.P
    r.set_camera(vp32)
    cnt = torch.zeros(P, dtype=torch.int32, device="cuda")
    off = torch.zeros(P + 1, dtype=torch.int32, device="cuda")
    tot = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    probe = dict(count=cnt, offset=off, z=torch.zeros(1, device="cuda"),
                 prim=torch.zeros(1, dtype=torch.int32, device="cuda"), total=tot)
    sn.raster(r.scene, r.vp, r.full_size, W, H, r.bins[0], probe, st)
    torch.cuda.synchronize()
    F = int(tot.cpu().numpy().view(np.uint32)[0])
    frags = dict(count=cnt, offset=off, z=torch.empty(max(F, 1), device="cuda"),
                 prim=torch.empty(max(F, 1), dtype=torch.int32, device="cuda"), total=tot)
    st.zero_()  # the sizing call above reports the probe's capacity overflow
    sn.raster(r.scene, r.vp, r.full_size, W, H, r.bins[0], frags, st)
    out = torch.empty(P * 4, device="cuda")
    sn.abuffer(frags, r.rgba8, W, H, tuple(r.params.bg), out, None)
    torch.cuda.synchronize()
    if int(st.item()) != 0:
        raise sn.StarNTError("star_nt_raster", int(st.item()))
    return out.view(P, 4)[:, :3].clone(), frags


def leaf_active(r: Renderer):
    """Per target of a per-leaf renderer: the fraction of its tiles that ran
    pass 2 and/or 3 in the last frame."""
    modes = r.leaf_ws.cpu().numpy()
    out, o = [], 0
    for w, h in r.plan.sizes():
        n = ((w + 15) // 16) * ((h + 15) // 16)
        out.append(float(np.mean(modes[o:o + n] != 0)))
        o += n
    return out


def mse(a, b) -> float:
    return float(torch.mean((a - b) ** 2).item())


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--workload", default="hd", choices=["hd", "uhd", "small"])
    ap.add_argument("--frames", type=int, default=120)
    ap.add_argument("--base-tile", type=int, default=64, choices=[16, 64])
    ap.add_argument("--merge-scale2", type=float, default=0.5)
    ap.add_argument("--merge-scale3", type=float, default=0.7)
    ap.add_argument("--mlp", default="bf16", choices=["bf16", "fp8", "fp8x2"])
    ap.add_argument("--tau", default=None, help="SPLIT,MERGE quadtree thresholds (8-bit units)")
    args = ap.parse_args(argv)
    build.build()
    sc = {"hd": scenes.hd_scene, "uhd": scenes.uhd_scene, "small": scenes.small_scene}[args.workload]()
    W, H = sc.width, sc.height
    w = dict(np.load(os.path.join(HERE, "weights", "tail_mlp.npz")))
    tau = {}
    if args.tau:
        ts, tm = (float(v) for v in args.tau.split(","))
        tau = {"tau_split": ts, "tau_merge": tm}
    star = Renderer(sc.verts, sc.rgba8, W, H, params=sn.default_params(**tau), mlp=w, x_dtype=sn.BF16,
                    fused=args.mlp if args.mlp in ("fp8", "fp8x2") else True, persistent=True,
                    base_tile=args.base_tile, merge_scale2=args.merge_scale2,
                    merge_scale3=args.merge_scale3)
    leaf = Renderer(sc.verts, sc.rgba8, W, H, params=sn.default_params(**tau), mlp=w, x_dtype=sn.BF16,
                    fused=args.mlp if args.mlp in ("fp8", "fp8x2") else True, base_tile=args.base_tile, leaf=True)
    ref = Renderer(sc.verts, sc.rgba8, W, H, mlp=w, x_dtype=sn.F32)
    cams = scenes.orbit_cameras(W, H, args.frames + 1)
    bg = tuple(ref.params.bg)
    err = {k: [] for k in ("star", "star_real", "star_interpolated", "leaf", "leaf_real", "leaf_interpolated",
                           "plain", "wboit", "unsorted_over")}
    active = []
    for f in range(0, args.frames, 2):   # real frame f, interpolated frame f + 1
        c_real, c_int = cams[f], cams[f + 1]
        star.set_cameras(c_real.vp32, c_real.vp64.reshape(16), c_int.vp64.reshape(16))
        star.step()
        leaf.set_cameras(c_real.vp32, c_real.vp64.reshape(16), c_int.vp64.reshape(16))
        leaf.step()
        torch.cuda.synchronize()
        real = star.rgba32f.view(-1, 4)[:, :3].clone()
        interp = star.interp_out.view(-1, 4)[:, :3].clone()
        l_real = leaf.rgba32f.view(-1, 4)[:, :3].clone()
        l_interp = leaf.interp_out.view(-1, 4)[:, :3].clone()
        active.append(leaf_active(leaf))
        ex, frags = exact_and_frags(ref, c_real.vp32)
        ref.set_cameras(c_real.vp32)
        ref.plain_frame()
        plain = ref.rgba32f.view(-1, 4)[:, :3].clone()
        wb = torch.empty(W * H * 4, device="cuda")
        sn.raster(ref.scene, ref.vp, ref.full_size, W, H, ref.bins[0], None, ref.status)
        sn.wboit(ref.bins[0], scenes.NEAR, scenes.FAR, bg, wb)
        un = torch.empty(W * H * 4, device="cuda")
        sn.unsorted_over(frags, ref.rgba8, W, H, bg, un)
        torch.cuda.synchronize()
        e_real = mse(real, ex)
        err["star_real"].append(e_real)
        err["star"].append(e_real)
        e_lr = mse(l_real, ex)
        err["leaf_real"].append(e_lr)
        err["leaf"].append(e_lr)
        err["plain"].append(mse(plain, ex))
        err["wboit"].append(mse(wb.view(-1, 4)[:, :3], ex))
        err["unsorted_over"].append(mse(un.view(-1, 4)[:, :3], ex))
        if f + 1 < args.frames:
            ex_i, _ = exact_and_frags(ref, c_int.vp32)
            e_int = mse(interp, ex_i)
            err["star_interpolated"].append(e_int)
            err["star"].append(e_int)
            e_li = mse(l_interp, ex_i)
            err["leaf_interpolated"].append(e_li)
            err["leaf"].append(e_li)
    star.check_status()
    leaf.check_status()
    ref.check_status()
    mean = {k: float(np.mean(v)) for k, v in err.items()}
    e_rand = mean["unsorted_over"]
    out = {"workload": f"{args.workload} {W}x{H}, {sc.verts.shape[0]} triangles", "frames": args.frames,
           "base_tile": args.base_tile, "tau_split_merge": [star.params.tau_split, star.params.tau_merge], "pass2_merge_scale": args.merge_scale2,
           "pass3_merge_scale": args.merge_scale3, "mlp": args.mlp,
           "mean_mse": {k: float(f"{v:.4e}") for k, v in mean.items()},
           "psnr_of_mean_mse_db": {k: round(10 * math.log10(1 / v), 3) for k, v in mean.items()},
           "mse_reduction_vs_wboit_pct": {k: round(100 * (mean["wboit"] - v) / mean["wboit"], 2)
                                          for k, v in mean.items() if k != "wboit"},
           "error_reduction_vs_unsorted_pct": {k: round(100 * (e_rand - v) / e_rand, 2)
                                               for k, v in mean.items() if k != "unsorted_over"},
           "final_pass_state": star.pass_state(),
           "leaf_targets": [list(t) for t in leaf.plan.sizes()],
           "leaf_active_tile_fraction_mean": [round(float(v), 4) for v in np.mean(np.array(active), axis=0)]}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
