"""Benchmark of the STAR-NT per-frame hot path on B300.

Default workload: 1920x1080, 20k seeded transparent triangles (mean depth
complexity ~8), camera orbiting at 5 deg/s, 60 fps.  One step = one real
STAR-NT frame (pass 1 at full resolution, passes 2 and 3 at the quadtree's
scales, upscale, MLP, composite, quadtree update) plus one interpolated
frame (depth reprojection): every stage of the hot path.  The metric is
ms/frame = step time / 2.  The plain full-resolution neural OIT pipeline on
the same scene is timed alongside (``plain_ms_per_frame``), and the step is
decomposed into what the fused kernels, the quadtree's reduced passes and the
interpolated frames each save (``decomposition_ms``).  The metric is quoted
at 1080p and 4K: the default run adds the same measurements at 3840x2160
(80k triangles) as the ``uhd`` record.  ``e2e`` runs the step through the
context call of the C ABI from host memory, copies included.

``--impl reference`` times the CPU oracle (float64, host cores) on the same
workload instead.  Multi-GPU runs are independent replicas (the frame path
has no exchange step): each rank renders its own sequence.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_PEAKS = {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0,
                  "sm_max_mhz": 2032.0}
N_SM = 148
ALU_LANES_PER_SM = 128
OPS_PER_FRAGMENT = 31     # algorithmic integer/fp operations per fragment (see design notes)


def kernels_per_step(r) -> int:
    """Kernel launches of one real + interpolated step of renderer r: raster of
    the passes (set-up/count, tile scan, fill); the geometry passes (the fused
    pass launch and the persistent launch, or the persistent launch alone, or
    three launches); the resolve (one launch, or features + MLP + composite);
    the quadtree (decide, relax, relax + histogram + Eq. 2); the reprojection
    (matrix, pixels)."""
    if r.persistent:
        passes = 2 if (r.fused and not r.fused_fp8 and r.fuse_passes) else 1
    else:
        passes = 3
    return 3 + passes + (1 if r.fused else 3) + 3 + 2
STAGE_REPS = 20
# DRAM bytes (read + write) of one launch of the dominant kernel, from one ncu
# capture of the benchmark's workload (dram__bytes_read.sum +
# dram__bytes_write.sum); per workload, None where no capture of the current
# kernel exists.  k_passes2: the persistent passes with pass 3 separate;
# k_passes_resolve: every pass at full size, with the network and composite.
PASSES_DRAM_BYTES = {"hd": 14934272, "uhd": 172245504}
FUSED_DRAM_BYTES = {"hd": 8356864, "uhd": 191712000}


def stage_rooflines(star, torch, stage_state, stage_mean, hbm_gbs):
    """Each stage's achieved fraction of the HBM roofline: the algorithmic bytes
    of its launches at the sizes in force when the stage graphs ran, over the
    stage's measured time.  Per unit:
      raster   (bin count, tile scan, bin fill; per pass that is binned): 52 B of
               vertices and colour + 112 B of set-up written and 112 B read back
               per triangle, 8 B per (triangle, tile) pair (count, list entry),
               16 B per tile (count, offset, cursor, cleared count);
      passes   id1, z1 per full-resolution pixel (8 B), id2 (4 B) per pixel of
               pass 2, n, tail, t_tail (24 B) per pixel of pass 3 (merged passes
               at the full size), 20 B of frame per pixel when the launch also
               resolves the frame; set-ups and pair lists read once;
      resolve  id1 4 B + frame 20 B per pixel, id2 4 B per pixel of pass 2 and
               24 B per pixel of pass 3 (the bilinear taps' planes read once);
      quadtree id1 4 B per pixel, 256 corner samples of 4 B and the mask per
               base tile;
      reproject z1 4 B + previous frame 16 B + 8-bit frame 4 B per pixel, + 16 B
               when the float copy of the interpolated frame is kept.
    The passes are ALU-bound (the headline roofline), the resolve issue-bound;
    their HBM fractions say how far from the memory bound they are."""
    W, H, T = star.W, star.H, star.T
    P = W * H
    hdr = [star.bins[k].mem[:64].view(torch.int32).cpu().numpy() for k in range(3)]
    binned = [h for h in hdr if int(h[8]) == 0 and int(h[4]) > 0]
    pairs = sum(int(np.uint32(h[6])) for h in binned)
    tiles = sum(int(h[4]) for h in binned)
    P2 = P if int(hdr[1][8]) else stage_state["W2"] * stage_state["H2"]
    P3 = P if int(hdr[2][8]) else stage_state["W3"] * stage_state["H3"]
    resolved = bool(int(hdr[1][11]))
    B = star.params.base_tile
    qt_tiles = ((W + B - 1) // B) * ((H + B - 1) // B)
    work = {
        "raster": len(binned) * T * 276 + 8 * pairs + 16 * tiles,
        "passes": 8 * P + 4 * P2 + 24 * P3 + (20 * P if resolved else 0) + len(binned) * T * 112
                  + 4 * pairs,
        "resolve": None if resolved else 24 * P + 4 * P2 + 24 * P3,
        "quadtree": 4 * P + qt_tiles * (1024 + 8),
        "reproject": P * (24 + (16 if star.interp_float else 0)),
    }
    out = {}
    for name, b in work.items():
        ms = stage_mean.get(name)
        if ms is None:
            continue
        if b is None:
            out[name] = {"bytes": None, "ms": round(ms, 5),
                         "note": "the pass launch produced the frame; this launch returns at once"}
            continue
        gbs = b / (ms * 1e-3) / 1e9
        out[name] = {"bytes": int(b), "ms": round(ms, 5), "achieved_gbs": round(gbs, 1),
                     "frac": round(gbs / hbm_gbs, 4)}
    return out


def load_peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return dict(FALLBACK_PEAKS), "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._thr = None

    def start(self):
        self._thr = threading.Thread(target=self._run, daemon=True)
        self._thr.start()
        return self

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                if out:
                    self.samples.append([v.strip() for v in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def stop(self):
        self._stop.set()
        if self._thr:
            self._thr.join(timeout=6)
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 2 + i and s[2 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons}


def workload_scene(name):
    from paper_2606_16747_b300 import scenes
    if name == "hd":
        return scenes.hd_scene(), "1920x1080, 20k triangles, mean depth complexity ~8"
    if name == "uhd":
        return scenes.uhd_scene(), "3840x2160, 80k triangles, mean depth complexity ~16"
    if name == "small":
        return scenes.small_scene(), "256x256, 32 triangles, mean depth complexity ~4"
    raise ValueError(name)


def mlp_weights():
    """Trained tail-colour weights when present, seeded Xavier weights otherwise."""
    from paper_2606_16747_b300 import scenes
    path = os.path.join(ROOT, "paper_2606_16747_b300", "weights", "tail_mlp.npz")
    if os.path.exists(path):
        d = np.load(path)
        return {k: d[k].astype(np.float32) for k, _ in scenes.MLP_SHAPES}, "trained"
    return scenes.mlp_xavier(2), "xavier_seed2"


# ---------------------------------------------------------------------------
def head_start(torch, ms):
    """Holds the current stream for about `ms` milliseconds with torch's own
    fixed-length spin kernel (it counts clock cycles and waits on nothing),
    so that the launches the host enqueues next are queued before the GPU
    reaches them.  A timed step then measures its own work: without it, a
    host slower than the GPU leaves the device idle between a step's start
    event and its graph launch, and that gap would count as step time."""
    torch.cuda._sleep(int(ms * 2.1e6))   # cycles, at up to 2.1 GHz


def timed_graph_ms(torch, g, flush, set_cams, k0, steps, warmup):
    """Mean ms of `steps` replays of graph g (after `warmup`), L2 flushed and
    the cameras of step k set before each; returns (ms, next step index)."""
    k = k0
    for _ in range(warmup):
        set_cams(k)
        g.replay()
        k += 1
    ev = []
    head_start(torch, 0.3 * steps + 0.5)
    for _ in range(steps):
        flush.fill_(1)
        set_cams(k)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        ev.append((e0, e1))
        k += 1
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in ev])), k


def measure(args, workload, steps, warmup, rank, world, leaf_variant=True, main=True):
    """The STAR-NT step on one workload: the timed step, per-stage times, the
    decomposition into what the quadtree and the reprojection each buy, the
    plain full-resolution pipeline, quality against the exact A-buffer, e2e
    through the context API, and the rooflines.  main: the headline line (all
    fields); otherwise a sub-record of the same measurements."""
    import torch

    from paper_2606_16747_b300 import build, scenes
    from paper_2606_16747_b300 import star_nt as sn
    from paper_2606_16747_b300.pipeline import Renderer

    build.build()
    torch.cuda.set_device(rank % max(1, torch.cuda.device_count()))
    dev = torch.device("cuda")
    sc, desc = workload_scene(workload)
    W, H = sc.width, sc.height
    w, wname = mlp_weights()
    x_dtype = sn.F32 if args.mlp == "f32" else sn.BF16
    # fused resolve: bf16 or fp8 operands on tcgen05 (f32 runs the separate kernels)
    fused_kind = (args.mlp if args.mlp != "bf16" else True) if args.fused and x_dtype == sn.BF16 else False
    params = sn.default_params(**({"tau_split": args.tau[0], "tau_merge": args.tau[1]} if args.tau else {}))
    star = Renderer(sc.verts, sc.rgba8, W, H, params=params, mlp=w, x_dtype=x_dtype, base_tile=args.base_tile,
                    fused=fused_kind, persistent=args.persistent,
                    merge_scale2=args.merge_scale2, merge_scale3=args.merge_scale3,
                    fixed_scales=args.fixed_scales, fuse_passes=args.fuse_passes)
    star.interp_float = False   # a display takes the 8-bit interpolated frame
    plain = Renderer(sc.verts, sc.rgba8, W, H, mlp=w, x_dtype=sn.F32)
    n_frames = 2 * (40 + 4 * warmup + 4 * steps)
    cams = scenes.orbit_cameras(W, H, n_frames)
    vp32 = torch.tensor(np.stack([c.vp32 for c in cams]), device=dev)
    vp64 = torch.tensor(np.stack([c.vp64.reshape(16) for c in cams]), device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 126 MB L2
    head_start(torch, 0.01)   # loads the spin kernel before any timed region

    def set_cams(k):            # step k: real frame 2k, interpolated frame 2k + 1
        star.set_cameras(vp32[2 * k], vp64[2 * k], vp64[2 * k + 1])

    # settle the tile hierarchy on the first frames, tune the pass launch on
    # this workload, then capture one step
    for k in range(4):
        set_cams(k)
        star.step()
    tuned = None
    if args.persistent and not args.no_tune:
        from paper_2606_16747_b300 import autotune
        tuned = autotune.tune(star)
        star.tuning = (tuned["block_w"], tuned["ctas_per_sm"], tuned["pixels_per_thread"])
        if "fuse_passes" in tuned and args.fuse_passes:
            star.fuse_passes = tuned["fuse_passes"]
    stages = star.star_stages() + [("reproject", star.interp_frame)]
    g_step = star.capture(star.step)
    g_stage = [(name, star.capture(fn)) for name, fn in stages]
    step = 4
    for _ in range(warmup):
        set_cams(step)
        g_step.replay()
        step += 1
    torch.cuda.synchronize()
    star.check_status()

    def timed(replay, k):
        flush.fill_(1)
        set_cams(k)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        replay()
        e1.record()
        return e0, e1

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device()).start()
    wall0 = time.perf_counter()
    events = []
    # per timed step, whether the pass launch produced the frame (bins2 header
    # word 11), copied on the device after the step's end event
    resolved_log = torch.zeros(steps, dtype=torch.int32, device=dev)
    head_start(torch, 0.3 * steps + 0.5)
    for k in range(steps):
        events.append(timed(g_step.replay, step))
        resolved_log[k:k + 1].copy_(star.bins[1].mem[44:48].view(torch.int32))
        step += 1
    torch.cuda.synchronize()
    resolved_steps = resolved_log.cpu().numpy().astype(bool)
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in events]
    # full-resolution fragments of the timed real frames (counted afterwards)
    Fcount = float(np.mean([fragment_count(sn, star, vp32[2 * k], W, H)
                            for k in range(step - steps, step)]))
    if world > 1:
        torch.distributed.barrier()
    star.check_status()
    state = star.pass_state()

    q_step = step
    step += 1
    # per-stage times: each stage graph replayed REPS times back to back (the
    # host enqueues faster than a stage runs, so the device never waits) after
    # one warm-up replay; the average is that stage's duration
    stage_ms = {}
    set_cams(step)
    step += 1
    g_step.replay()
    stage_state = star.pass_state()
    for name, g in g_stage:
        g.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        head_start(torch, 0.05 * STAGE_REPS + 0.5)
        e0.record()
        for _ in range(STAGE_REPS):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        stage_ms[name] = [e0.elapsed_time(e1) / STAGE_REPS]

    # the real frame alone (raster, passes, resolve, quadtree update), timed
    # as the step is: what the interpolated frames save is the difference
    g_real = star.capture(lambda: star.star_frame())
    real_ms, step = timed_graph_ms(torch, g_real, flush, set_cams, step, steps, warmup)
    # and without the quadtree update (inside the step it runs beside the
    # interpolated frame)
    g_real_nq = star.capture(lambda: star.star_frame(update_tiles=False))
    real_nq_ms, step = timed_graph_ms(torch, g_real_nq, flush, set_cams, step, steps, warmup)
    star.check_status()

    # the same step with passes 2 and 3 at the sizes Eq. 2 gives (no merge below full size)
    eq2_ms = None
    if star.merge_scale2 < 1.0 or star.merge_scale3 < 1.0:
        star.merge_scale2 = star.merge_scale3 = 1.0
        g_eq2 = star.capture(star.step)
        eq2_step_ms, step = timed_graph_ms(torch, g_eq2, flush, set_cams, step, steps, warmup)
        eq2_ms = eq2_step_ms / 2.0
        star.merge_scale2, star.merge_scale3 = args.merge_scale2, args.merge_scale3
        star.check_status()

    # the same fused pass launch and resolve with every pass at full size and
    # no quadtree: what the quadtree's reduced passes buy is the difference
    # to the real frame
    plain_fused_ms = None
    if star.fused and star.persistent:
        pf = Renderer(sc.verts, sc.rgba8, W, H, params=params, mlp=w, x_dtype=x_dtype, base_tile=args.base_tile,
                      fused=fused_kind, persistent=True, tuning=star.tuning, fuse_passes=star.fuse_passes,
                      fixed_scales=(1.0, 1.0))
        g_pf = pf.capture(lambda: pf.star_frame(update_tiles=False))

        def set_pf(k):
            pf.set_cameras(vp32[2 * k])
        plain_fused_ms, _ = timed_graph_ms(torch, g_pf, flush, set_pf, 4, steps, warmup)
        pf.check_status()
        del pf, g_pf

    # the per-leaf variant: passes 2 and 3 at the Eq. 2 scale of each pixel's
    # own leaf level, on the same cameras
    leaf = None
    leaf_info = None
    if star.fused and leaf_variant:
        leaf = Renderer(sc.verts, sc.rgba8, W, H, params=sn.default_params(
                            **({"tau_split": args.tau[0], "tau_merge": args.tau[1]} if args.tau else {})),
                        mlp=w, x_dtype=x_dtype, base_tile=args.base_tile, fused=fused_kind, leaf=True)
        leaf.interp_float = False

        def set_leaf_cams(k):
            leaf.set_cameras(vp32[2 * k], vp64[2 * k], vp64[2 * k + 1])

        for k in range(4):
            set_leaf_cams(k)
            leaf.step()
        leaf_tuned = None
        if not args.no_tune:
            from paper_2606_16747_b300 import autotune
            leaf_tuned = autotune.tune(leaf)
            leaf.tuning = (leaf_tuned["block_w"], leaf_tuned["ctas_per_sm"],
                           leaf_tuned["pixels_per_thread"])
        g_leaf = leaf.capture(leaf.step)
        leaf_step_ms, _ = timed_graph_ms(torch, g_leaf, flush, set_leaf_cams, 4, steps, warmup)
        leaf.check_status()
        leaf_ms = leaf_step_ms / 2.0
        active = leaf_active_tiles(leaf)
        leaf_stage_ms = {}
        for name, fn in leaf.star_stages() + [("reproject", leaf.interp_frame)]:
            g = leaf.capture(fn)
            g.replay()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            head_start(torch, 0.05 * STAGE_REPS + 0.5)
            e0.record()
            for _ in range(STAGE_REPS):
                g.replay()
            e1.record()
            torch.cuda.synchronize()
            leaf_stage_ms[name] = round(e0.elapsed_time(e1) / STAGE_REPS, 5)
        leaf.check_status()
        leaf_info = {"ms_per_frame": round(leaf_ms, 5), "stages_ms": leaf_stage_ms,
                     "targets": [list(t) for t in leaf.plan.sizes()],
                     "pass2_target_by_level": leaf.plan.targets(2),
                     "pass3_target_by_level": leaf.plan.targets(3),
                     "active_tile_fraction": active, "pass_tuning": leaf_tuned,
                     "leaf_level_area_fraction": leaf_level_fractions(leaf),
                     "note": "Eq. 2 per quadtree leaf (scene index replaced by the leaf level); "
                             "same cameras, same step structure (real + interpolated frame)"}

    # plain full-resolution FP32 pipeline on the same scene and cameras
    plain.set_cameras(vp32[0])
    g_plain = plain.capture(plain.plain_frame)
    plain_ms = []
    for k in range(warmup + steps):
        head_start(torch, 0.3)
        flush.fill_(1)
        plain.set_cameras(vp32[2 * k])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g_plain.replay()
        e1.record()
        torch.cuda.synchronize()
        if k >= warmup:
            plain_ms.append(e0.elapsed_time(e1))
    plain.check_status()

    # weighted blended OIT (the evaluation's baseline OIT method): raster + one pass
    def wboit_frame():
        sn.raster(plain.scene, plain.vp, plain.full_size, W, H, plain.bins[0], None, plain.status)
        sn.wboit(plain.bins[0], scenes.NEAR, scenes.FAR, tuple(plain.params.bg), plain.rgba32f,
                 plain.rgba8_out)
    g_wb = plain.capture(wboit_frame)
    wboit_ms = []
    for k in range(warmup + steps):
        head_start(torch, 0.3)
        flush.fill_(1)
        plain.set_cameras(vp32[2 * k])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g_wb.replay()
        e1.record()
        torch.cuda.synchronize()
        if k >= warmup:
            wboit_ms.append(e0.elapsed_time(e1))
    plain.check_status()

    psnr_measured = quality(sn, star, plain, W, H, cams, q_step, leaf)
    del leaf
    precision = (precision_record(sn, torch, star, sc, w, W, H, vp32[2 * q_step])
                 if star.fused and star.persistent and x_dtype == sn.BF16 else None)
    dfaoit = dfaoit_record(sn, torch, plain, sc, W, H, vp32[2 * q_step], flush)

    # end to end through the public API: the context call, host inputs in and
    # both 8-bit frames out every step
    e2e = end_to_end(sn, torch, sc, w, W, H, cams, args, params, star.tuning, star.fuse_passes, steps, warmup)

    t_max, ms_frame, ms_frame_job = job_timing(float(np.mean(step_ms)), world, dev)
    stage_mean = {k: float(np.mean(v)) for k, v in stage_ms.items()}
    peaks, peaks_kind = load_peaks()
    # dominant kernel: the geometry passes (one persistent launch, or pass 1)
    alu_peak = N_SM * ALU_LANES_PER_SM * peaks.get("sm_max_mhz", 2032.0) * 1e6 / 1e12  # Tops/s
    if "passes" in stage_mean:
        # fragments the timed launch processed: the stage graphs ran on the
        # cameras of the last step, at the pass sizes in force then
        dom_ms = stage_mean["passes"]
        vp_last = vp32[2 * (q_step + 1)]
        dom_frags = fragment_count(sn, star, vp_last, W, H)
        # a pass merged into pass 1 shares pass 1's traversal (its fragments are
        # pass 1's); a separate pass traverses the fragments at its own size
        merged = [int(star.bins[k].mem[32:36].view(torch.int32).item()) for k in (1, 2)]
        for (wp, hp), m in zip(((stage_state["W2"], stage_state["H2"]),
                                (stage_state["W3"], stage_state["H3"])), merged):
            if not m:
                dom_frags += fragment_count(sn, star, vp_last, W, H, (wp, hp))
        pix = star.tuning[2] if star.tuning is not None and len(star.tuning) > 2 and star.tuning[2] else 2
        if all(merged) and star.persistent and star.fused and not star.fused_fp8 and star.fuse_passes:
            dom_name = (f"k_passes_resolve ({pix} pixel(s) per thread; passes 1-3 at full size with the "
                        "network input, tcgen05 MLP and composite of every pixel; only the traversal ops "
                        "are counted)")
            traffic = FUSED_DRAM_BYTES.get(workload)
        else:
            dom_name = (f"{'k_passes2' if pix == 2 else 'k_passes'} (passes 1-3, one persistent launch, "
                        f"{pix} pixel(s) per thread)")
            traffic = PASSES_DRAM_BYTES.get(workload)
    else:
        dom_ms = stage_mean["pass1"]
        dom_frags = Fcount
        dom_name = "k_pass_merged (pass 1, full resolution)"
        traffic = None
    achieved = OPS_PER_FRAGMENT * dom_frags / (dom_ms * 1e-3) / 1e12
    psnr = psnr_measured
    plain_mean = float(np.mean(plain_ms))
    line = {
        "metric": "ms/frame (STAR-NT, 1080p)" if workload == "hd" else f"ms/frame (STAR-NT, {workload})",
        "value": round(ms_frame_job, 5),
        "value_note": "ms per frame of the whole job: N replicas each render 2 frames per step, "
                      "timed by the slowest rank (equals the per-rank ms/frame at N = 1)",
        "ms_per_frame_per_rank": round(ms_frame, 5),
        "unit": "ms/frame",
        "n_gpus": world,
        "steps": steps,
        "warmup": warmup,
        "ms_per_step": round(t_max, 5),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"bf16": "f32+bf16", "fp8": "f32+e4m3", "fp8x2": "f32+e4m3x2", "fp8t": "f32+e4m3",
                  "fp8x2t": "f32+e4m3x2", "f32": "f32"}[args.mlp],
        "data": "synthetic seeded triangle soup, orbit camera",
        "config": {"workload": desc, "frames_per_step": 2, "mlp": args.mlp, "weights": wname,
                   "resolve": "fused" if star.fused else "separate",
                   "pass_launch_resolves": bool(star.fuse_passes and star.fused and not star.fused_fp8
                                                and star.persistent),
                   "passes": "persistent" if star.persistent else "separate",
                   "pass2_merge_scale": star.merge_scale2,
                   "pass3_merge_scale": star.merge_scale3,
                   "fixed_scales": list(args.fixed_scales) if args.fixed_scales else None,
                   "pass_tuning": tuned,
                   "base_tile": args.base_tile, "tau_split_merge": [star.params.tau_split, star.params.tau_merge],
                   "l2": "flushed between steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "fragments_per_s": round(world * Fcount / (ms_frame * 1e-3), 1),
        "fragments_full_res": int(Fcount),
        "fragments_note": "mean full-resolution fragment count of the timed real frames",
        "eq2_sizes_ms_per_frame": round(eq2_ms, 5) if eq2_ms is not None else None,
        "eq2_sizes_note": "the same step with passes 2 and 3 always at their Eq. 2 sizes (merge scales 1.0)",
        "plain_ms_per_frame": round(plain_mean, 5),
        "wboit_ms_per_frame": round(float(np.mean(wboit_ms)), 5),
        "speedup_vs_plain": round(plain_mean / ms_frame, 4),
        "decomposition_ms": decomposition(plain_mean, plain_fused_ms, real_ms, real_nq_ms, ms_frame,
                                          stage_mean),
        "stages_ms": {k: round(v, 5) for k, v in stage_mean.items()},
        "pass_state": {k: state[k] for k in ("W2", "H2", "W3", "H3", "s2", "s3", "wbar", "hist")},
        "wall_s": round(wall, 3),
        "graph": "one CUDA graph per step (real + interpolated frame), replayed",
        "gpu_launches": kernels_per_step(star) * steps,
        "frames_resolved_by_pass_launch": int(resolved_steps.sum()),
        "clocks": clocks,
        "e2e": e2e,
        "roofline": {"bound": "alu", "kernel": dom_name, "fragments": int(dom_frags),
                     "achieved": round(achieved, 4), "peak": round(alu_peak, 3), "unit": "Tops/s",
                     "frac": round(achieved / alu_peak, 5),
                     "traffic": traffic,
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of the "
                                       "dominant kernel on this workload (build of the profile summaries)"
                                       if traffic is not None else "no capture for this configuration",
                     "peak_source": f"{N_SM} SM x {ALU_LANES_PER_SM} lanes x sm_max_mhz ({peaks_kind})",
                     "ops_per_fragment": OPS_PER_FRAGMENT, "launch_ms": round(dom_ms, 5)},
    }
    line["stage_roofline"] = {"bound": "hbm", "peak": peaks.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"]),
                              "unit": "GB/s", "peak_source": f"hbm_gbs ({peaks_kind})",
                              "stages": stage_rooflines(star, torch, stage_state, stage_mean,
                                                        peaks.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"]))}
    line["per_leaf"] = leaf_info
    line["precision"] = precision
    line["dfaoit"] = dfaoit
    line["psnr_db_vs_exact_abuffer"] = psnr["psnr_db"]
    line["quality"] = {"mse_vs_exact_abuffer": psnr["mse"],
                       "error_reduction_vs_unsorted_pct": psnr["error_reduction_vs_unsorted_pct"],
                       "note": "one real frame and the following interpolated frame after the timed "
                               "steps; unsorted_over = naive blending in submission order (E_random "
                               "of the Q measure); wboit = weighted blended OIT, one pass"}
    if not main:
        for k in ("value_note", "n_gpus", "higher_is_better", "scaling", "vs_baseline", "data", "graph"):
            line.pop(k, None)
    return line


def precision_record(sn, torch, star, sc, w, W, H, vp, reps=20):
    """The resolve with every MLP operand type on the same pass planes (the
    state and camera of the measured frame): its time, and the frame's error
    against the float32 MLP path on those planes (separate feature, float32
    MLP and composite kernels, within 1e-5 of the float64 oracle by the parity
    tests), in 8-bit units: max and 99.9th percentile over pixels and
    channels."""
    from paper_2606_16747_b300.pipeline import MLP_TYPES, Renderer
    r = Renderer(sc.verts, sc.rgba8, W, H, params=star.params, mlp=w, x_dtype=sn.BF16, fused=True,
                 persistent=True, fuse_passes=False, tuning=star.tuning, merge_scale2=star.merge_scale2,
                 merge_scale3=star.merge_scale3)
    r.state.copy_(star.state)
    r.set_cameras(vp)
    stages = dict(r.star_stages(update_tiles=False))
    stages["raster"]()
    stages["passes"]()
    P = W * H
    x32 = torch.empty(P * 8, device="cuda")
    front = torch.empty(P * 4, device="cuda")
    f = torch.empty(P * 4, device="cuda")
    ref = torch.empty(P * 4, device="cuda")
    b2, b3 = r.bins[1], r.bins[2]
    sn.upscale_features(r.scene, b2, b3, r.l1, r.l2, r.l3, W, H, r.params, x32, sn.F32, front)
    sn.infer(r.mlp, sn.F32, x32, f, P, r.status)
    sn.composite(front, f, P, ref, None)
    out = torch.empty(P * 4, device="cuda")
    rec = {}
    for name, t in MLP_TYPES.items():
        def call():
            sn.resolve_mlp(r.scene, b2, b3, r.l1, r.l2, r.l3, W, H, r.params, r.mlp, t, out, None, r.status)
        g = r.capture(call)
        g.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        head_start(torch, 0.05 * reps + 0.5)
        e0.record()
        for _ in range(reps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        r.check_status()
        err = (out.view(P, 4)[:, :3] - ref.view(P, 4)[:, :3]).abs().flatten()
        k = max(1, int(round(0.001 * err.numel())))
        rec[name] = {"resolve_ms": round(e0.elapsed_time(e1) / reps, 5),
                     "max_err_255": round(float(err.max()) * 255.0, 4),
                     "p999_err_255": round(float(torch.topk(err, k).values[-1]) * 255.0, 4)}
    rec["reference"] = ("frame of the float32 MLP path on the same planes (separate kernels; within 1e-5 "
                        "of the float64 oracle by the parity tests); bar 2/255")
    return rec


def dfaoit_record(sn, torch, plain, sc, W, H, vp, flush, reps=20):
    """The DFAOIT comparison network (Sec. 3.3; Table 2's inference columns)
    beside STAR-NT's tail network on the same frame: the bf16 tensor-core
    inference of each on every pixel (5 inputs, 16 B per pixel, against 11
    inputs, 32 B per pixel), the DFAOIT frame (raster, 11-feature pass,
    network, composite) and, with trained weights, its PSNR against the exact
    A-buffer."""
    from paper_2606_16747_b300 import train as tr
    P = W * H
    path = os.path.join(ROOT, "paper_2606_16747_b300", "weights", "dfaoit_mlp.npz")
    trained = os.path.exists(path)
    wd = dict(np.load(path)) if trained else tr.dfaoit_initial_weights(0)
    wt = {k: torch.as_tensor(np.asarray(v, np.float32)).cuda() for k, v in wd.items()}
    mlp10 = sn.mlp_struct(wt)
    x5 = torch.zeros(P * 8, dtype=torch.bfloat16, device="cuda")
    x10 = torch.zeros(P * 16, dtype=torch.bfloat16, device="cuda")
    front5 = torch.empty(P * 4, device="cuda")
    front10 = torch.empty(P * 4, device="cuda")
    f = torch.empty(P * 4, device="cuda")
    out = torch.empty(P * 4, device="cuda")
    plain.set_cameras(vp)
    b = plain.bins[0]
    sn.raster(plain.scene, plain.vp, plain.full_size, W, H, b, None, plain.status)
    sn.build_inputs(plain.scene, b, b, b, plain.l1, None, None, W, H, plain.params, x5, sn.BF16, front5,
                    plain.status)
    sn.build_inputs_dfaoit(plain.scene, b, None, W, H, plain.params, x10, sn.BF16, front10, plain.status)
    torch.cuda.synchronize()
    plain.check_status()

    def time_graph(fn):
        g = plain.capture(fn)
        g.replay()
        ev = []
        head_start(torch, 0.3 * reps + 0.5)
        for _ in range(reps):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            ev.append((e0, e1))
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(c) for a, c in ev]))

    ms5 = time_graph(lambda: sn.infer(plain.mlp, sn.BF16, x5, f, P, plain.status))
    ms10 = time_graph(lambda: sn.infer_dfaoit(mlp10, sn.BF16, x10, f, P, plain.status))

    def dfaoit_frame():
        sn.raster(plain.scene, plain.vp, plain.full_size, W, H, b, None, plain.status)
        sn.build_inputs_dfaoit(plain.scene, b, None, W, H, plain.params, x10, sn.BF16, front10, plain.status)
        sn.infer_dfaoit(mlp10, sn.BF16, x10, f, P, plain.status)
        sn.composite(front10, f, P, out, None)
    frame_ms = time_graph(dfaoit_frame)
    plain.check_status()
    rec = {"inference_ms_5f": round(ms5, 5), "inference_ms_10f": round(ms10, 5),
           "inference_speedup_10_to_5": round(ms10 / ms5, 4),
           "input_bytes_per_pixel": {"5f": 16, "10f": 32},
           "dfaoit_frame_ms": round(frame_ms, 5), "weights": "trained" if trained else "xavier_seed0",
           "note": "bf16 tensor-core inference over every pixel of the frame (L2 flushed before each); "
                   "the paper's ten features are eleven listed scalars, all eleven are inputs"}
    if trained:
        dfaoit_frame()
        ex = exact_frame(sn, plain, vp, W, H)
        rec["psnr_db_vs_exact_abuffer"] = psnr_db(out.view(P, 4)[:, :3], ex)
    return rec


def decomposition(plain_ms, plain_fused_ms, real_ms, real_nq_ms, ms_frame, stage_mean):
    """Where the STAR-NT frame time comes from, per frame (ms):
      gain_kernels:  the plain full-resolution pipeline (FP32, separate
                     kernels) minus the fused BF16 pass launch and resolve
                     with every pass at full size (no quadtree);
      gain_spatial:  that fused full-size frame minus the real STAR-NT frame
                     without the quadtree update (passes 2 and 3 at the sizes
                     the quadtree chose: merged into pass 1 above the merge
                     scales, reduced below);
      quadtree:      the quadtree update's own time (it runs beside the
                     interpolated frame inside the step);
      gain_temporal: the real frame (with the update) minus the STAR-NT
                     ms/frame (every other frame is an interpolated frame)."""
    out = {"plain_fp32": round(plain_ms, 5),
           "plain_fused_full_size": round(plain_fused_ms, 5) if plain_fused_ms is not None else None,
           "star_real_frame": round(real_ms, 5),
           "star_real_frame_without_quadtree": round(real_nq_ms, 5),
           "star_per_frame": round(ms_frame, 5),
           "quadtree_stage": round(stage_mean.get("quadtree", float("nan")), 5),
           "interpolated_frame_stage": round(stage_mean.get("reproject", float("nan")), 5)}
    if plain_fused_ms is not None:
        out["gain_kernels"] = round(plain_ms - plain_fused_ms, 5)
        out["gain_spatial"] = round(plain_fused_ms - real_nq_ms, 5)
    out["gain_temporal"] = round(real_ms - ms_frame, 5)
    return out


def run_ours(args, rank, world):
    line = measure(args, args.workload, args.steps, args.warmup, rank, world, leaf_variant=not args.no_leaf)
    if args.workload == "hd" and not args.no_uhd:
        # the metric is quoted at 1080p and 4K: the same measurements at
        # 3840x2160 (80k triangles), fewer steps
        line["uhd"] = measure(args, "uhd", max(5, args.steps // 2), args.warmup, rank, world,
                              leaf_variant=False, main=False)
    return line


def job_timing(t_step_ms, world, device, frames_per_step=2):
    """(slowest rank's ms per step, its ms per frame, the whole job's ms per
    frame): every rank renders its own replica of the sequence, so the job
    renders world x frames_per_step frames per step in the slowest rank's
    time.  Collective only for world > 1 (MAX over ranks, on the group's
    backend: NCCL for the benchmark, gloo in the CPU tests)."""
    import torch
    t_max = float(t_step_ms)
    if world > 1:
        t = torch.tensor([t_max], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        t_max = float(t.item())
    ms_frame = t_max / frames_per_step
    return t_max, ms_frame, ms_frame / world


def leaf_active_tiles(r):
    """Per plan target: the fraction of its tiles that ran pass 2 and/or 3 in
    the last frame (target 0 always runs pass 1)."""
    modes = r.leaf_ws.cpu().numpy()
    out, o = [], 0
    for w, h in r.plan.sizes():
        n = ((w + 15) // 16) * ((h + 15) // 16)
        out.append(round(float(np.mean(modes[o:o + n] != 0)), 4))
        o += n
    return out


def leaf_level_fractions(r):
    """Fraction of the base tiles' area per leaf level under the current
    masks (bit 0 root split, bits 1..4 level-1 splits, bits 5..20 level-2)."""
    m = r.mask[0].cpu().numpy().view(np.uint32).astype(np.int64)
    root = (m & 1) != 0
    a = [float(np.sum(~root)), 0.0, 0.0, 0.0]
    for c1 in range(4):
        s1 = root & (((m >> (1 + c1)) & 1) != 0)
        a[1] += float(np.sum(root & ~s1)) / 4
        for c2 in range(4):
            s2 = s1 & (((m >> (5 + 4 * c1 + c2)) & 1) != 0)
            a[2] += float(np.sum(s1 & ~s2)) / 16
            a[3] += float(np.sum(s2)) / 16
    return [round(v / m.size, 4) for v in a]


def fragment_count(sn, r, vp, W, H, size=None):
    """Fragments of the scene under camera vp at W x H (or at ``size``)."""
    import torch
    P = W * H
    size_t = r.full_size if size is None else torch.tensor(list(size), dtype=torch.int32, device="cuda")
    frags = dict(count=torch.zeros(P, dtype=torch.int32, device="cuda"),
                 offset=torch.zeros(P + 1, dtype=torch.int32, device="cuda"),
                 z=torch.zeros(1, dtype=torch.float32, device="cuda"),
                 prim=torch.zeros(1, dtype=torch.int32, device="cuda"),
                 total=torch.zeros(1, dtype=torch.int32, device="cuda"))
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    sn.raster(r.scene, vp, size_t, W, H, r.bins[0], frags, st)
    torch.cuda.synchronize()
    return int(frags["total"].cpu().numpy().view(np.uint32)[0])


def end_to_end(sn, torch, sc, w, W, H, cams, args, params, tuning, fuse_passes, steps, warmup):
    """The same metric through the public API: the context call
    (star_nt_frame) from host memory.  Every step copies the triangle soup and
    the cameras host->device from pinned memory (two copies), renders one real
    and one interpolated frame, and reads both 8-bit frames back into pinned
    memory (one copy).
    Inputs and outputs are triple-buffered (one captured graph per buffer
    set): step k+1's inputs copy in and step k's frames copy out on their own
    streams while step k+1 renders; a buffer set is reused only once its
    previous copy-out has landed.  With two sets the render of step k waited
    for the copy-out of step k-2 and the link idled between copies (0.168
    against 0.155 ms/frame at 1080p); with three the device-to-host link, the
    bound of this leg, stays busy.  The time is the host's wall clock from the
    first copy-in to the last frame on the host, over 2 x steps frames."""
    mlp_type = {"bf16": sn.BF16, "fp8": sn.E4M3, "fp8x2": sn.E4M3X2, "fp8t": sn.E4M3_TENSOR,
                "fp8x2t": sn.E4M3X2_TENSOR}.get(args.mlp)
    if mlp_type is None or not args.fused or not args.persistent or args.fixed_scales:
        return None   # the context runs the fused, persistent product path only
    T = int(sc.rgba8.shape[0])
    P = W * H
    ctx = sn.Context(params=params, mlp_type=mlp_type, merge_scale2=args.merge_scale2,
                     merge_scale3=args.merge_scale3, fuse_passes=fuse_passes)
    if tuning is not None:
        ctx.set_tuning(tuning, fuse_passes)
    ctx.bind(W, H, T)
    wt = {k: torch.as_tensor(np.ascontiguousarray(v, np.float32)).cuda() for k, v in w.items()}
    mlp = sn.mlp_struct(wt)
    # the scene in one pinned block (triangle vertices, then colours at a
    # 256-byte boundary), and per step one 320-byte block of cameras (vp32
    # [16] f32, then vp64 of the real and the interpolated frame [2][16]
    # f64): two host-to-device copies per step
    vb = np.ascontiguousarray(sc.verts).view(np.uint8).reshape(-1)
    cb = np.ascontiguousarray(sc.rgba8).view(np.uint8).reshape(-1)
    c_off = (vb.size + 255) // 256 * 256
    hscene = torch.zeros(c_off + cb.size, dtype=torch.uint8).pin_memory()
    hscene[:vb.size] = torch.from_numpy(vb)
    hscene[c_off:] = torch.from_numpy(cb)
    ncam = 4 + warmup + steps + 2
    cam_blocks = [np.concatenate([cams[2 * k].vp32.astype(np.float32).view(np.uint8).reshape(-1),
                                  np.stack([cams[2 * k].vp64.reshape(16), cams[2 * k + 1].vp64.reshape(16)])
                                  .astype(np.float64).view(np.uint8).reshape(-1)]) for k in range(ncam)]
    hcam = torch.from_numpy(np.stack(cam_blocks)).pin_memory()          # [ncam][320] bytes
    sets = []
    for b in range(3):
        dscene = torch.empty_like(hscene, device="cuda")
        dcam = torch.empty(320, dtype=torch.uint8, device="cuda")
        frames8 = torch.empty(2, P, dtype=torch.int32, device="cuda")  # real, interpolated
        d = dict(dscene=dscene, dcam=dcam, vp=dcam[:64].view(torch.float32),
                 v64=dcam[64:].view(torch.float64).view(2, 16), rgba32f=torch.empty(P * 4, device="cuda"),
                 frames8=frames8, host8=torch.empty(2, P, dtype=torch.int32).pin_memory(),
                 copied_in=torch.cuda.Event(), rendered=torch.cuda.Event(), copied_out=torch.cuda.Event(),
                 out_pending=False)
        d["scene"] = sn.Scene(dscene.data_ptr(), dscene.data_ptr() + c_off, T)
        sets.append(d)
    # one copy-out stream: one DMA stream reads back 57 GB/s on the B300, as
    # many as eight do
    main, cin, cout = torch.cuda.current_stream(), torch.cuda.Stream(), torch.cuda.Stream()

    status = torch.zeros(1, dtype=torch.int32, device="cuda")

    def render(d):
        ctx.frame(d["scene"], mlp, d["vp"], d["v64"][0], d["v64"][1], d["rgba32f"], d["frames8"][0], None,
                  d["frames8"][1], status=status)

    def copy_in(d, k):
        with torch.cuda.stream(cin):
            if d["out_pending"]:         # its last frames were read back already
                cin.wait_event(d["copied_out"])
            d["dscene"].copy_(hscene, non_blocking=True)
            d["dcam"].copy_(hcam[k], non_blocking=True)
            d["copied_in"].record(cin)

    # settle the tiles, then capture one graph per buffer set
    for k in range(4):
        d = sets[k % len(sets)]
        copy_in(d, k)
        main.wait_event(d["copied_in"])
        render(d)
    torch.cuda.synchronize()
    graphs = []
    for d in sets:
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(main)
        with torch.cuda.stream(s):
            with torch.cuda.graph(g):
                render(d)
        main.wait_stream(s)
        graphs.append(g)
    torch.cuda.synchronize()

    def run(k0, n):
        for i in range(n):
            k = k0 + i
            d, g = sets[k % len(sets)], graphs[k % len(sets)]
            copy_in(d, k)
            main.wait_event(d["copied_in"])
            g.replay()
            d["rendered"].record(main)
            with torch.cuda.stream(cout):
                cout.wait_event(d["rendered"])
                d["host8"].copy_(d["frames8"], non_blocking=True)
                d["copied_out"].record(cout)
            d["out_pending"] = True
        torch.cuda.synchronize()

    run(4, warmup)
    t0 = time.perf_counter()
    run(4 + warmup, steps)
    dt = time.perf_counter() - t0
    if int(status.item()) != sn.OK:
        raise sn.StarNTError("star_nt_frame (device)", int(status.item()))
    # the leg's bound: the same copies alone (both frames out, inputs in),
    # no rendering, timed the same way
    torch.cuda.synchronize()
    l0 = time.perf_counter()
    for i in range(steps):
        d = sets[i % len(sets)]
        with torch.cuda.stream(cin):
            d["dscene"].copy_(hscene, non_blocking=True)
            d["dcam"].copy_(hcam[i], non_blocking=True)
        with torch.cuda.stream(cout):
            d["host8"].copy_(d["frames8"], non_blocking=True)
    torch.cuda.synchronize()
    ldt = time.perf_counter() - l0
    ctx.close()
    h2d = hscene.numel() + 320
    link_ms = ldt * 1e3 / (2.0 * steps)
    return {"value": round(dt * 1e3 / (2.0 * steps), 5), "unit": "ms/frame",
            "link_floor": {"value": round(link_ms, 5), "unit": "ms/frame",
                           "d2h_gbs": round(2 * P * 4 * steps / ldt / 1e9, 1),
                           "what": "the step's copies alone (triangles in, both 8-bit frames out), no rendering"},
            "frac_of_link": round(link_ms / (dt * 1e3 / (2.0 * steps)), 3),
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(2 * P * 4),
            "api": "star_nt_frame (context): host triangles and cameras in, both 8-bit frames out, "
                   "every step; inputs and outputs triple-buffered so copies overlap rendering",
            "copies_declared": True}


def exact_frame(sn, r, vp32, W, H, keep_frags=False):
    """Exact A-buffer of the scene under camera vp32 (GPU, sorted fragments);
    with keep_frags also the fragment lists (bins of r hold the raster)."""
    import torch
    P = W * H
    r.set_cameras(vp32)
    cnt = torch.zeros(P, dtype=torch.int32, device="cuda")
    off = torch.zeros(P + 1, dtype=torch.int32, device="cuda")
    tot = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    probe = dict(count=cnt, offset=off, z=torch.zeros(1, device="cuda"),
                 prim=torch.zeros(1, dtype=torch.int32, device="cuda"), total=tot)
    sn.raster(r.scene, r.vp, r.full_size, W, H, r.bins[0], probe, st)
    torch.cuda.synchronize()
    F = int(tot.cpu().numpy().view(np.uint32)[0])
    frags = dict(count=cnt, offset=off, z=torch.empty(F, device="cuda"),
                 prim=torch.empty(F, dtype=torch.int32, device="cuda"), total=tot)
    sn.raster(r.scene, r.vp, r.full_size, W, H, r.bins[0], frags, st)
    out = torch.empty(P * 4, device="cuda")
    sn.abuffer(frags, r.rgba8, W, H, tuple(r.params.bg), out, None)
    torch.cuda.synchronize()
    if keep_frags:
        return out.view(P, 4)[:, :3], frags
    return out.view(P, 4)[:, :3]


def psnr_db(a, b):
    import torch
    mse = float(torch.mean((a - b) ** 2).item())
    return round(10.0 * math.log10(1.0 / max(mse, 1e-30)), 3)


def quality(sn, star, plain, W, H, cams, k, leaf=None):
    """PSNR against the exact A-buffer: STAR-NT real frame 2k and interpolated
    frame 2k + 1 (global and, when given, per-leaf pass scales), and the plain
    pipeline at frame 2k (after the timed runs)."""
    import torch

    def star_pair(r):
        r.set_cameras(cams[2 * k].vp32, cams[2 * k].vp64.reshape(16), cams[2 * k + 1].vp64.reshape(16))
        keep = r.interp_float
        r.interp_float = True
        r.step()
        r.interp_float = keep
        return r.rgba32f.view(-1, 4)[:, :3].clone(), r.interp_out.view(-1, 4)[:, :3].clone()

    real, interp = star_pair(star)
    leaf_pair = star_pair(leaf) if leaf is not None else None
    plain.set_cameras(cams[2 * k].vp32)
    plain.plain_frame()
    pl = plain.rgba32f.view(-1, 4)[:, :3].clone()
    ex_real, frags = exact_frame(sn, plain, cams[2 * k].vp32, W, H, keep_frags=True)
    # comparison renderers of the evaluation: naive unsorted blending (E_random)
    # and weighted blended OIT, on the same frame
    from paper_2606_16747_b300 import scenes
    bg = tuple(plain.params.bg)
    un = torch.empty(W * H * 4, device="cuda")
    sn.unsorted_over(frags, plain.rgba8, W, H, bg, un)
    wb = torch.empty(W * H * 4, device="cuda")
    sn.wboit(plain.bins[0], scenes.NEAR, scenes.FAR, bg, wb)
    torch.cuda.synchronize()
    un, wb = un.view(-1, 4)[:, :3], wb.view(-1, 4)[:, :3]
    ex_interp = exact_frame(sn, plain, cams[2 * k + 1].vp32, W, H)
    frames = {"star_real": (real, ex_real), "star_interpolated": (interp, ex_interp),
              "plain": (pl, ex_real), "wboit": (wb, ex_real), "unsorted_over": (un, ex_real)}
    if leaf_pair is not None:
        frames["leaf_real"] = (leaf_pair[0], ex_real)
        frames["leaf_interpolated"] = (leaf_pair[1], ex_interp)
    mse = {k: float(torch.mean((a - b) ** 2).item()) for k, (a, b) in frames.items()}
    e_random = mse["unsorted_over"]
    return {"psnr_db": {k: round(10.0 * math.log10(1.0 / max(v, 1e-30)), 3) for k, v in mse.items()},
            "mse": {k: float(f"{v:.4e}") for k, v in mse.items()},
            "error_reduction_vs_unsorted_pct": {k: round(100.0 * (e_random - v) / e_random, 2)
                                                for k, v in mse.items() if k != "unsorted_over"}}


# ---------------------------------------------------------------------------
def cpu_oracle_frame(sc, w, cam, threads):
    import oracle
    from paper_2606_16747_b300 import scenes
    return oracle.frame_full(sc.verts, sc.rgba8, cam.vp32, sc.width, sc.height, scenes.mlp_flat(w),
                             threads=threads)


def cpu_phases(sc, w, cam, threads, rows=None):
    """Oracle time per phase of one plain full-resolution frame (ms): raster,
    per-pixel sort + A-buffer + layer terms, and the neural path (features,
    MLP, composite).  rows: only the first rows of the frame (a sample)."""
    import oracle
    from paper_2606_16747_b300 import scenes
    W, H = sc.width, sc.height
    t0 = time.perf_counter()
    fr = oracle.raster(sc.verts, cam.vp32, W, H, threads)
    t1 = time.perf_counter()
    if rows is not None:   # keep the first rows' fragment lists only
        P = W * rows
        end = int(fr.offsets[P])
        fr = oracle.Frags(W, rows, fr.counts[:P], fr.offsets[:P + 1], fr.z[:end], fr.prim[:end])
    r = oracle.resolve(fr, sc.rgba8, (1.0, 1.0, 1.0), threads)
    t2 = time.perf_counter()
    flag = (r["n"] > 2).astype(np.uint8)
    x, front = oracle.features(r["id1"], sc.rgba8, r["layer2"], r["n"].astype(np.float64),
                               r["a_tail"].astype(np.float64), r["s_tail"].astype(np.float64),
                               r["t_tail"], (1.0, 1.0, 1.0))
    f = oracle.mlp_forward(oracle.params64(scenes.mlp_flat(w)), x, flag)
    oracle.composite(front, f)
    t3 = time.perf_counter()
    return {"raster_ms": round((t1 - t0) * 1e3, 1), "sort_abuffer_layers_ms": round((t2 - t1) * 1e3, 1),
            "neural_path_ms": round((t3 - t2) * 1e3, 1)}


def run_cpu_baseline(args):
    """The oracle as it stands on the host cores, bounded sample of the workload."""
    from paper_2606_16747_b300 import scenes
    sc, desc = workload_scene(args.workload)
    w, _ = mlp_weights()
    cams = scenes.orbit_cameras(sc.width, sc.height, 4)
    threads = os.cpu_count() or 1
    cpu_oracle_frame(sc, w, cams[0], threads)          # build / page in
    t0 = time.perf_counter()
    n = 0
    while n < 2 or (time.perf_counter() - t0 < 10.0 and n < 8):
        cpu_oracle_frame(sc, w, cams[n % 4], threads)
        n += 1
    dt = (time.perf_counter() - t0) / n
    # phases on all cores, and on one core over the first 1/16 of the rows
    # (raster of the whole frame, the rest on the sample)
    phases = cpu_phases(sc, w, cams[0], threads)
    rows = max(1, sc.height // 16)
    single = cpu_phases(sc, w, cams[0], 1, rows=rows)
    return {"value": round(dt * 1e3, 3), "unit": "ms/frame", "cores": threads, "kind": "oracle",
            "sample": f"{n} full frames of the plain full-resolution neural pipeline ({desc}), "
                      "float64 oracle, threads over rows",
            "phases_all_cores_ms": phases,
            "phases_one_core_ms": single,
            "phases_one_core_sample": f"raster of the full frame; the other phases on the first {rows} "
                                      f"of {sc.height} rows"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    cb = run_cpu_baseline_steps(args)
    return cb


def run_cpu_baseline_steps(args):
    from paper_2606_16747_b300 import scenes
    sc, desc = workload_scene(args.workload)
    w, _ = mlp_weights()
    cams = scenes.orbit_cameras(sc.width, sc.height, 2 * (args.warmup + args.steps) + 2)
    threads = os.cpu_count() or 1
    for k in range(args.warmup):
        cpu_oracle_frame(sc, w, cams[k], threads)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        cpu_oracle_frame(sc, w, cams[args.warmup + k], threads)
        times.append(time.perf_counter() - t0)
    v = float(np.mean(times)) * 1e3
    return {"impl": "reference", "metric": "ms/frame (STAR-NT, 1080p)" if args.workload == "hd" else
            f"ms/frame (STAR-NT, {args.workload})", "value": round(v, 3), "unit": "ms/frame",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v, 3),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic seeded triangle soup",
            "config": {"workload": desc, "frames_per_step": 1},
            "cpu_baseline": {"value": round(v, 3), "unit": "ms/frame", "cores": threads, "kind": "oracle",
                             "sample": "one full frame per step (plain full-resolution pipeline), "
                                       "float64 oracle"},
            "e2e": {"value": round(v, 3), "unit": "ms/frame", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="hd", choices=["hd", "uhd", "small"])
    ap.add_argument("--mlp", default="bf16", choices=["bf16", "fp8", "fp8x2", "fp8t", "fp8x2t", "f32"])
    ap.add_argument("--base-tile", type=int, default=64, choices=[16, 64],
                    help="quadtree base tile (64: leaves of 8 to 64 pixels)")
    ap.add_argument("--separate-passes", dest="persistent", action="store_false",
                    help="three geometry-pass launches instead of one persistent launch")
    ap.add_argument("--no-tune", action="store_true", help="skip the pass-launch autotuner")
    ap.add_argument("--merge-scale2", type=float, default=0.5,
                    help="pass 2 at least this fraction of the full size runs inside pass 1 at full "
                         "size (1.0: only at full size, as Eq. 2 sizes it)")
    ap.add_argument("--merge-scale3", type=float, default=0.7,
                    help="the same for pass 3 (1.0: only at full size)")
    ap.add_argument("--no-fuse-passes", dest="fuse_passes", action="store_false",
                    help="never let the pass launch produce the frame (always the separate resolve)")
    ap.add_argument("--unfused", dest="fused", action="store_false",
                    help="separate upscale/features, MLP and composite kernels")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-leaf", action="store_true", help="skip the per-leaf pass-resolution variant")
    ap.add_argument("--no-uhd", action="store_true", help="1080p only (no 3840x2160 sub-record)")
    ap.add_argument("--tau", default=None,
                    help="SPLIT,MERGE: quadtree thresholds (8-bit units) instead of the library's defaults")
    ap.add_argument("--fixed-scales", default=None,
                    help="S2,S3: passes 2 and 3 at these fixed scales instead of Eq. 2's (the paper's "
                         "ablation settings, e.g. 0.5,0.5 or 0.5,0.25); merges only at full size")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.tau:
        args.tau = tuple(float(v) for v in args.tau.split(","))
        if len(args.tau) != 2 or not args.tau[1] < args.tau[0]:
            raise SystemExit("--tau wants SPLIT,MERGE with MERGE < SPLIT")
    if args.fixed_scales:
        args.fixed_scales = tuple(float(v) for v in args.fixed_scales.split(","))
        if len(args.fixed_scales) != 2 or not all(0.25 <= v <= 1.0 for v in args.fixed_scales):
            raise SystemExit("--fixed-scales wants two scales in [0.25, 1]")
        args.merge_scale2 = args.merge_scale3 = 1.0   # the passes run at the fixed sizes
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if rank == 0 and line is not None:
            print(json.dumps(line))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    line = run_ours(args, rank, world)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = run_cpu_baseline(args)
        print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
