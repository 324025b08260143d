"""Frame driver of the STAR-NT hot path on one GPU.

Owns the device buffers (torch allocations) and sequences the C-ABI calls:

  plain frame     raster (full res) -> fused build_inputs -> infer -> composite
  STAR-NT frame   raster x3 (full, s2, s3) -> geometry passes 1-3 -> upscale /
                  features -> infer -> composite -> quadtree (next s2, s3)
  per-leaf frame  raster of the plan's targets -> pass modes + passes -> resolve
                  (each pixel's passes 2, 3 at its leaf's scale) -> quadtree
  interpolated    reproject from the last real frame (Sec. 3.3, last paragraph)

Pass resolutions and cameras live in device buffers with fixed addresses, so
one captured CUDA graph replays every frame of a sequence.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import star_nt as sn

STATE_W2, STATE_W3 = 8, 16   # byte offsets of {W2, H2} and {W3, H3} in star_nt_pass_state
# MLP operand types of the fused resolve
MLP_TYPES = {"bf16": sn.BF16, "fp8": sn.E4M3, "fp8x2": sn.E4M3X2, "fp8t": sn.E4M3_TENSOR,
             "fp8x2t": sn.E4M3X2_TENSOR}


def _i32(vals, device):
    return torch.tensor(vals, dtype=torch.int32, device=device)


class Renderer:
    def __init__(self, verts, rgba8, W, H, params=None, x_dtype=sn.F32, mlp=None,
                 pair_capacity=None, device="cuda", base_tile=None, fused=False,
                 persistent=False, tuning=None, merge_scale2=1.0, merge_scale3=1.0, leaf=False,
                 fuse_passes=True, fixed_scales=None):
        self.device = device
        sn.preload(torch.device(device).index)
        self.W, self.H = int(W), int(H)
        self.P = self.W * self.H
        self.verts = torch.as_tensor(np.ascontiguousarray(verts, np.float32)).to(device)
        self.rgba8 = torch.as_tensor(np.ascontiguousarray(rgba8, np.uint32).view(np.int32)).to(device)
        self.T = int(self.rgba8.shape[0])
        self.scene = sn.scene_struct(self.verts, self.rgba8)
        self.params = params if params is not None else sn.default_params()
        if base_tile is not None:
            self.params.base_tile = base_tile
        self.x_dtype = x_dtype
        # fused: upscale + features + MLP on tcgen05 + composite in one kernel
        # (True or "bf16": bf16 operands; "fp8": e4m3 operands; "fp8x2":
        # compensated e4m3 pairs; "fp8t", "fp8x2t": the same with per-tensor
        # scales)
        if fused not in (False, None, True) and fused not in MLP_TYPES:
            raise ValueError(f"fused: {fused!r}")
        self.fused = bool(fused)
        self.fused_fp8 = fused in MLP_TYPES and fused != "bf16"
        self.mlp_kind = fused if self.fused_fp8 else "bf16"
        # persistent: the three geometry passes in one launch (tuning: star_nt_tuning's
        # (block_w, ctas_per_sm, pixels_per_thread))
        self.persistent = bool(persistent)
        self.tuning = tuning
        # persistent + fused bf16 resolve: when every pass runs at full size the
        # pass launch also runs the network and the composite (the resolve
        # launch then returns at once)
        self.fuse_passes = bool(fuse_passes)
        # a reduced pass at least this fraction of the full size (both axes)
        # is produced by pass 1 at the full size instead (1.0: only at full size)
        self.merge_scale2 = float(merge_scale2)
        self.merge_scale3 = float(merge_scale3)
        if self.fused and x_dtype != sn.BF16:
            raise ValueError("the fused resolve runs the BF16 tensor-core MLP")
        # leaf: passes 2 and 3 per quadtree leaf (Eq. 2 at the leaf's level)
        # instead of one scale per frame; runs the fused resolve
        self.leaf = bool(leaf)
        if self.leaf and not self.fused:
            raise ValueError("the per-leaf frame runs the fused resolve (fused=True, 'fp8' or 'fp8x2')")
        cap = pair_capacity if pair_capacity is not None else max(1 << 20, 96 * self.T)
        self.bins = [sn.BinsBuffer(self.W, self.H, self.T, cap, device) for _ in range(3)]
        P = self.P
        f32 = dict(dtype=torch.float32, device=device)
        i32 = dict(dtype=torch.int32, device=device)
        self.status = torch.zeros(1, **i32)
        self.side = torch.cuda.Stream(device=device)  # interpolated frame beside the quadtree
        self.vp = torch.zeros(16, **f32)
        self.full_size = _i32([self.W, self.H], device)
        # per-pass planes (sized for full resolution)
        self.l1 = dict(id1=torch.empty(P, **i32), z1=torch.empty(P, **f32))
        self.l2 = dict(id2=torch.empty(P, **i32))
        self.l3 = dict(n=torch.empty(P, **i32), tail=torch.empty(P * 4, **i32),
                       t_tail=torch.empty(P, **f32))
        xdt = torch.float32 if x_dtype == sn.F32 else torch.bfloat16
        self.x = torch.empty(P * 8, dtype=xdt, device=device)
        self.front = torch.empty(P * 4, **f32)
        self.f = torch.empty(P * 4, **f32)
        self.rgba32f = torch.empty(P * 4, **f32)
        self.rgba8_out = torch.empty(P, **i32)
        # quadtree state: pass sizes live in ``state`` on the device
        self.state = torch.zeros(64, dtype=torch.uint8, device=device)
        self.state.view(torch.int32)[:6] = torch.tensor([self.W, self.H] * 3, dtype=torch.int32)
        # fixed_scales (s2, s3): the pass sizes of every frame are ceil(s W) x
        # ceil(s H) (the fixed settings of the paper's ablation) instead of
        # Eq. 2's; the quadtree still runs and reports its histogram and w-bar
        self.fixed_sizes = None
        if fixed_scales is not None:
            self.fixed_sizes = {p: _i32([math.ceil(s * self.W), math.ceil(s * self.H)], device)
                                for p, s in zip((2, 3), fixed_scales)}
        B = self.params.base_tile
        self.n_tiles = math.ceil(self.W / B) * math.ceil(self.H / B)
        self.mask = [torch.zeros(self.n_tiles, **i32), torch.zeros(self.n_tiles, **i32)]
        self.qt_ws = torch.zeros(sn.quadtree_ws_bytes(self.W, self.H, B), dtype=torch.uint8, device=device)
        if self.leaf:
            self._init_leaf(cap)
        self.mlp_tensors = None
        if mlp is not None:
            self.set_mlp(mlp)
        # reprojection
        self.interp_out = torch.zeros(P * 4, **f32)
        self.interp_float = True   # float copy of interpolated frames (analysis; displays use 8-bit)
        self.interp_rgba8 = torch.zeros(P, **i32)
        self.vp64_prev = torch.zeros(16, dtype=torch.float64, device=device)
        self.vp64_cur = torch.zeros(16, dtype=torch.float64, device=device)
        self.reproj_ws = torch.zeros(sn.REPROJECT_WS_BYTES, dtype=torch.uint8, device=device)

    def _init_leaf(self, cap):
        """Targets of the per-leaf plan: target 0 is the full resolution (its
        bins and planes are those of pass 1 and the full-size pass 2 / 3
        planes); the others get their own bins and planes.  The masks start
        fully split (every leaf at level 3), so the first frame runs passes 2
        and 3 at the scale of the finest leaves."""
        dev = self.device
        self.plan = sn.leaf_plan(self.W, self.H, self.params)
        sizes = self.plan.sizes()
        t2, t3 = set(self.plan.targets(2)), set(self.plan.targets(3))
        self.leaf_sizes = [_i32([w, h], dev) for w, h in sizes]
        self.leaf_bins = [self.bins[0]] + [sn.BinsBuffer(w, h, self.T, cap, dev) for w, h in sizes[1:]]
        self.leaf_layers = []
        for k, (w, h) in enumerate(sizes):
            if k == 0:
                d = dict(self.l1)
                if 0 in t2:
                    d["id2"] = self.l2["id2"]
                if 0 in t3:
                    d.update(self.l3)
            else:
                n = w * h
                d = {}
                if k in t2:
                    d["id2"] = torch.full((n,), -1, dtype=torch.int32, device=dev)
                if k in t3:
                    d.update(n=torch.zeros(n, dtype=torch.int32, device=dev),
                             tail=torch.zeros(4 * n, dtype=torch.int32, device=dev),
                             t_tail=torch.ones(n, dtype=torch.float32, device=dev))
            self.leaf_layers.append(d)
        self.leaf_ws = torch.zeros(sn.leaf_ws_bytes(self.plan), dtype=torch.uint8, device=dev)
        self.mask[0].fill_((1 << 21) - 1)

    # -- inputs -------------------------------------------------------------
    def set_mlp(self, w: dict):
        self.mlp_tensors = {k: torch.as_tensor(np.ascontiguousarray(v, np.float32)).to(self.device)
                            for k, v in w.items()}
        self.mlp = sn.mlp_struct(self.mlp_tensors)

    def set_camera(self, vp32):
        self.vp.copy_(torch.as_tensor(np.asarray(vp32, np.float32).reshape(16)))

    def state_size(self, which):
        off = {1: None, 2: STATE_W2, 3: STATE_W3}[which]
        if off is None:
            return self.full_size
        if self.fixed_sizes is not None:
            return self.fixed_sizes[which]
        return self.state[off:off + 8].view(torch.int32)

    # -- frames -------------------------------------------------------------
    def plain_stages(self, stream=None):
        """The plain neural OIT pipeline: every pass at full resolution, fused."""
        b = self.bins[0]
        return [("raster", lambda: sn.raster(self.scene, self.vp, self.full_size, self.W, self.H, b,
                                            None, self.status, stream)),
                ("pass_fused", lambda: sn.build_inputs(self.scene, b, b, b, self.l1, None, None,
                                                       self.W, self.H, self.params, self.x,
                                                       self.x_dtype, self.front, self.status,
                                                       stream)),
                ("infer", lambda: sn.infer(self.mlp, self.x_dtype, self.x, self.f, self.P,
                                           self.status, stream)),
                ("composite", lambda: sn.composite(self.front, self.f, self.P, self.rgba32f,
                                                   self.rgba8_out, stream))]

    def plain_frame(self, stream=None):
        for _, fn in self.plain_stages(stream):
            fn()

    def leaf_stages(self, stream=None, update_tiles=True):
        """The stages of one real frame with per-leaf pass resolution."""
        def raster():
            sn.raster_passes(self.scene, [(self.vp, self.leaf_sizes[k], w, h, self.leaf_bins[k], None)
                                          for k, (w, h) in enumerate(self.plan.sizes())],
                             self.status, stream)

        st = [("raster", raster),
              ("passes", lambda: sn.geometry_passes_leaf(self.scene, self.plan, self.leaf_bins,
                                                         self.leaf_layers, self.mask[0], self.leaf_ws,
                                                         self.tuning, self.status, stream)),
              ("resolve", lambda: sn.resolve_leaf(self.scene, self.plan, self.leaf_layers, self.mask[0],
                                                  self.params, self.mlp, MLP_TYPES[self.mlp_kind],
                                                  self.rgba32f, self.rgba8_out, self.status, stream))]
        if update_tiles:
            st.append(("quadtree", lambda: self.update_tiles(stream)))
        return st

    def star_stages(self, stream=None, update_tiles=True):
        """The stages of one real STAR-NT frame as (name, callable) pairs:
        pass 1 at full resolution, passes 2 and 3 at the device-held sizes
        (or per leaf, for a per-leaf renderer)."""
        if self.leaf:
            return self.leaf_stages(stream, update_tiles)
        b1, b2, b3 = self.bins

        def raster():
            # the three passes share the binning launches; passes 2 and 3 at
            # full size are taken over by pass 1 (merged)
            sn.raster_passes(self.scene, [
                (self.vp, self.full_size, self.W, self.H, b1, None),
                (self.vp, self.state_size(2), self.W, self.H, b2, self.full_size, self.merge_scale2),
                (self.vp, self.state_size(3), self.W, self.H, b3, self.full_size, self.merge_scale3)],
                self.status, stream)

        st = [("raster", raster)]
        if self.persistent and self.fused and not self.fused_fp8 and self.fuse_passes:
            st.append(("passes", lambda: sn.geometry_passes_resolve(
                self.scene, b1, b2, b3, self.l1, self.l2, self.l3, self.params, self.mlp, self.rgba32f,
                self.rgba8_out, self.tuning, self.status, stream)))
        elif self.persistent:
            st.append(("passes", lambda: sn.geometry_passes(self.scene, b1, b2, b3, self.l1, self.l2,
                                                            self.l3, self.tuning, self.status,
                                                            stream)))
        else:
            st += [("pass1", lambda: sn.geometry_pass_merged(self.scene, b1, b2, b3, self.l1,
                                                             self.l2, self.l3, self.status,
                                                             stream)),
                   ("pass2", lambda: sn.geometry_pass(self.scene, b2, 2, self.l2, self.status,
                                                      stream)),
                   ("pass3", lambda: sn.geometry_pass(self.scene, b3, 3, self.l3, self.status,
                                                      stream))]
        if self.fused:
            res = {"bf16": sn.resolve, "fp8": sn.resolve_fp8, "fp8x2": sn.resolve_fp8x2}.get(self.mlp_kind)
            if res is None:
                t = MLP_TYPES[self.mlp_kind]
                res = lambda *a: sn.resolve_mlp(*a[:10], t, *a[10:])
            st.append(("resolve", lambda: res(self.scene, b2, b3, self.l1, self.l2, self.l3,
                                              self.W, self.H, self.params, self.mlp,
                                              self.rgba32f, self.rgba8_out, self.status, stream)))
        else:
            st += [("features", lambda: sn.upscale_features(self.scene, b2, b3, self.l1, self.l2,
                                                            self.l3, self.W, self.H, self.params,
                                                            self.x, self.x_dtype, self.front,
                                                            stream)),
                   ("infer", lambda: sn.infer(self.mlp, self.x_dtype, self.x, self.f, self.P,
                                              self.status, stream)),
                   ("composite", lambda: sn.composite(self.front, self.f, self.P, self.rgba32f,
                                                      self.rgba8_out, stream))]
        if update_tiles:
            st.append(("quadtree", lambda: self.update_tiles(stream)))
        return st

    def star_frame(self, stream=None, update_tiles=True):
        for _, fn in self.star_stages(stream, update_tiles):
            fn()

    def update_tiles(self, stream=None):
        """Quadtree update from this frame, in place: the masks keep one
        buffer, so one captured graph serves every frame."""
        sn.quadtree(self.rgba8_out, self.l1["id1"], self.W, self.H, self.params, self.mask[0],
                    self.mask[0], self.state, self.qt_ws, stream)

    def _infer_composite(self, stream):
        if self.mlp_tensors is None:
            raise RuntimeError("no MLP weights: call set_mlp first")
        sn.infer(self.mlp, self.x_dtype, self.x, self.f, self.P, self.status, stream)
        sn.composite(self.front, self.f, self.P, self.rgba32f, self.rgba8_out, stream)

    def set_cameras(self, vp32=None, vp64_real=None, vp64_interp=None):
        """Copy camera matrices into the device buffers the frames read
        (arrays or device tensors)."""
        for dst, src, dt in ((self.vp, vp32, np.float32), (self.vp64_prev, vp64_real, np.float64),
                             (self.vp64_cur, vp64_interp, np.float64)):
            if src is None:
                continue
            if isinstance(src, torch.Tensor):
                dst.copy_(src, non_blocking=True)
            else:
                dst.copy_(torch.as_tensor(np.asarray(src, dt).reshape(16)))

    def interp_frame(self, stream=None):
        """Interpolated frame from the last real frame (its colour and pass-1
        depth stay in ``rgba32f`` and ``l1['z1']`` until the next real frame);
        camera matrices from ``vp64_prev`` (real) and ``vp64_cur``.  The
        8-bit frame always, the float frame (``interp_out``) when
        ``interp_float`` is set."""
        sn.reproject(self.rgba32f, self.l1["z1"], self.vp64_prev, self.vp64_cur, self.W, self.H,
                     self.interp_out if self.interp_float else None, self.reproj_ws, stream,
                     out_rgba8=self.interp_rgba8)

    def step(self, stream=None):
        """One real STAR-NT frame followed by one interpolated frame.  The
        interpolated frame needs only the real frame's colour and depth, so it
        runs on a second stream beside the quadtree update; the step ends when
        both are done (both branches land in one captured graph)."""
        main = stream if stream is not None else torch.cuda.current_stream()
        self.star_frame(main, update_tiles=False)
        self.side.wait_stream(main)
        self.interp_frame(self.side)
        with torch.cuda.stream(main):
            self.update_tiles(main)
        main.wait_stream(self.side)

    def capture(self, fn):
        """Capture ``fn`` (enqueueing work on the current stream) as a CUDA
        graph after one eager warm-up run."""
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            fn()
        torch.cuda.current_stream().wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        return g

    def pass_state(self):
        return sn.read_pass_state(self.state)

    def check_status(self):
        s = int(self.status.item())
        if s != sn.OK:
            raise sn.StarNTError("device", s)


class AdaptiveInterval:
    """Interpolation interval of Sec. 3.3 (last paragraph): the number n of
    interpolated frames after each real frame, adapted to the measured frame
    times and capped at four; below the target frame rate it falls back to
    real frames only.

    Reading: a real frame must still arrive at least at the target rate, so
    one real frame and its n interpolated frames share the budget 1 / target:
    n = floor((1/target - t_real) / t_interp), clamped to [0, max_interp],
    with t_real and t_interp exponential moving averages of measured frame
    times.  When t_real alone exceeds the budget, n = 0 (standard rendering)."""

    def __init__(self, target_fps: float = 60.0, max_interp: int = 4, smoothing: float = 0.25):
        if target_fps <= 0 or not 0 <= max_interp <= 4 or not 0 < smoothing <= 1:
            raise ValueError("target_fps > 0, max_interp in [0, 4], smoothing in (0, 1]")
        self.budget_ms = 1000.0 / target_fps
        self.max_interp = max_interp
        self.smoothing = smoothing
        self.t_real = None
        self.t_interp = None

    def _ema(self, old, new):
        return new if old is None else old + self.smoothing * (new - old)

    def observe(self, real_ms=None, interp_ms=None):
        if real_ms is not None:
            self.t_real = self._ema(self.t_real, float(real_ms))
        if interp_ms is not None:
            self.t_interp = self._ema(self.t_interp, float(interp_ms))

    def interval(self) -> int:
        if self.t_real is None:
            return 0
        spare = self.budget_ms - self.t_real
        if spare <= 0.0:
            return 0
        if self.t_interp is None or self.t_interp <= 0.0:
            return 1 if self.max_interp > 0 else 0  # one interpolated frame to measure it
        return int(min(self.max_interp, max(0, math.floor(spare / self.t_interp))))


class Sequence:
    """Renders a camera sequence with real and interpolated frames: each real
    frame is followed by n interpolated frames reprojected from it (n from an
    AdaptiveInterval, or fixed), every frame timed with CUDA events.  Frame
    times are read back one frame late (event queries, no synchronisation on
    the frame path), so decisions use the previous measurements."""

    def __init__(self, renderer: Renderer, controller: AdaptiveInterval = None, fixed_interval=None):
        self.r = renderer
        self.ctl = controller
        self.fixed = fixed_interval
        self.left = 0          # interpolated frames left before the next real frame
        self.pending = []      # (kind, start event, end event) not yet read back
        self.kinds = []        # "real" / "interp" per rendered frame
        self.real_graph = renderer.capture(lambda: renderer.star_frame())
        self.interp_graph = renderer.capture(renderer.interp_frame)

    def _collect(self):
        keep = []
        for kind, e0, e1 in self.pending:
            if e1.query():
                ms = e0.elapsed_time(e1)
                if self.ctl is not None:
                    self.ctl.observe(real_ms=ms if kind == "real" else None,
                                     interp_ms=ms if kind == "interp" else None)
            else:
                keep.append((kind, e0, e1))
        self.pending = keep

    def frame(self, vp32, vp64):
        """Render the next frame for camera (vp32, vp64); returns "real" or
        "interp".  The frame is in renderer.rgba32f / rgba8_out (real) or
        renderer.interp_out / interp_rgba8 (interpolated)."""
        self._collect()
        r = self.r
        kind = "interp" if self.left > 0 else "real"
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if kind == "real":
            r.set_cameras(vp32=vp32, vp64_real=vp64)
            e0.record()
            self.real_graph.replay()
            e1.record()
            n = self.fixed if self.fixed is not None else (self.ctl.interval() if self.ctl else 0)
            self.left = int(n)
        else:
            r.set_cameras(vp64_interp=vp64)
            e0.record()
            self.interp_graph.replay()
            e1.record()
            self.left -= 1
        self.pending.append((kind, e0, e1))
        self.kinds.append(kind)
        return kind
