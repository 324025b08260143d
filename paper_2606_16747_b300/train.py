"""Training of the tail-colour MLP (Sec. 3.3: MSE loss, Adam) on data the
method generates itself: exact tail colours from the A-buffer of seeded
scenes, with the network inputs of the plain full-resolution pipeline.

The forward and backward passes are the library's CUDA kernels wrapped in
``torch.autograd.Function``s; Adam updates float32 master weights and keeps
their bfloat16-rounded copy for the forward pass.

    python -m paper_2606_16747_b300.train --out paper_2606_16747_b300/weights
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import scenes
from . import star_nt as sn
from .pipeline import Renderer

N_PARAMS = scenes.MLP_PARAM_COUNT
# the DFAOIT comparison network (Sec. 3.3): 11 inputs, sigmoid output
DFAOIT_SHAPES = (("w1", (32, 11)), ("b1", (32,)), ("w2", (16, 32)), ("b2", (16,)), ("w3", (3, 16)),
                 ("b3", (3,)))
DFAOIT_PARAMS = 963


def _slices(shapes):
    out, o = {}, 0
    for name, shape in shapes:
        n = int(np.prod(shape))
        out[name] = (o, o + n)
        o += n
    return out


def mlp_from_flat(flat: torch.Tensor, shapes=scenes.MLP_SHAPES) -> sn.Mlp:
    """C-ABI weight struct pointing into a flat float32 device tensor
    ([771] for the tail MLP, [963] for the DFAOIT network)."""
    base = flat.data_ptr()
    sl = _slices(shapes)
    return sn.Mlp(*[base + 4 * sl[k][0] for k in ("w1", "b1", "w2", "b2", "w3", "b3")])


def flat_to_dict(flat, shapes=scenes.MLP_SHAPES) -> dict:
    a = flat.detach().cpu().numpy() if isinstance(flat, torch.Tensor) else np.asarray(flat)
    sl = _slices(shapes)
    return {k: a[sl[k][0]:sl[k][1]].reshape(shape).astype(np.float32) for k, shape in shapes}


class _Workspace:
    def __init__(self):
        self.buf = None

    def get(self, B, device):
        n = sn.train_ws_bytes(B)
        if self.buf is None or self.buf.numel() < n:
            self.buf = torch.empty(n, dtype=torch.uint8, device=device)
        return self.buf


_WS = _Workspace()


class TailMLPFunction(torch.autograd.Function):
    """f = MLP(x) with the library's float32 forward kernel; the backward pass
    is the library's backpropagation kernel (gradient for the 771 weights)."""

    @staticmethod
    def forward(ctx, x, params):
        B = x.numel() // 8
        f = torch.empty(B * 4, dtype=torch.float32, device=x.device)
        sn.infer(mlp_from_flat(params), sn.F32, x, f, B)
        ctx.save_for_backward(x, params)
        return f

    @staticmethod
    def backward(ctx, grad_f):
        x, params = ctx.saved_tensors
        B = x.numel() // 8
        grad = torch.empty(N_PARAMS, dtype=torch.float32, device=x.device)
        sn.mlp_backward(mlp_from_flat(params), x, grad_f.contiguous(), B, grad, _WS.get(B, x.device))
        return None, grad


class DfaoitMLPFunction(torch.autograd.Function):
    """The DFAOIT comparison network, C_t = MLP(x) (x [B][16]), with the
    library's float32 forward and its backpropagation kernel (963 weights)."""

    @staticmethod
    def forward(ctx, x, params):
        B = x.numel() // 16
        f = torch.empty(B * 4, dtype=torch.float32, device=x.device)
        sn.infer_dfaoit(mlp_from_flat(params, DFAOIT_SHAPES), sn.F32, x, f, B)
        ctx.save_for_backward(x, params)
        return f

    @staticmethod
    def backward(ctx, grad_f):
        x, params = ctx.saved_tensors
        B = x.numel() // 16
        grad = torch.empty(DFAOIT_PARAMS, dtype=torch.float32, device=x.device)
        sn.dfaoit_backward(mlp_from_flat(params, DFAOIT_SHAPES), x, grad_f.contiguous(), B, grad,
                           _WS.get(B, x.device))
        return None, grad


class MSEFunction(torch.autograd.Function):
    """Mean squared error over B samples x 3 channels with the library's
    kernel, optionally weighted per sample (w [B]); its backward is the
    kernel's dL/df."""

    @staticmethod
    def forward(ctx, f, y, w=None):
        B = f.numel() // 4
        dy = torch.empty_like(f)
        loss = torch.empty(1, dtype=torch.float32, device=f.device)
        sn.mse_grad(f, y, B, dy, loss, _WS.get(B, f.device), w=w)
        ctx.save_for_backward(dy)
        return loss

    @staticmethod
    def backward(ctx, grad_loss):
        (dy,) = ctx.saved_tensors
        return dy * grad_loss, None, None


# ---------------------------------------------------------------------------
# data

def render_samples(scene: scenes.Scene, device="cuda"):
    """Network inputs (plain full-resolution pipeline, float32 layout), exact
    tail colours, front terms and the exact A-buffer colour of one scene."""
    W, H = scene.width, scene.height
    r = Renderer(scene.verts, scene.rgba8, W, H, x_dtype=sn.F32, device=device)
    r.set_camera(scene.cam.vp32)
    b = r.bins[0]
    sn.raster(r.scene, r.vp, r.full_size, W, H, b, None, r.status)
    sn.build_inputs(r.scene, b, b, b, r.l1, None, None, W, H, r.params, r.x, sn.F32, r.front, r.status)
    # fragment lists of the same pass for the exact resolve
    P = W * H
    cnt = torch.zeros(P, dtype=torch.int32, device=device)
    off = torch.zeros(P + 1, dtype=torch.int32, device=device)
    tot = torch.zeros(1, dtype=torch.int32, device=device)
    probe = dict(count=cnt, offset=off, z=torch.zeros(1, device=device),
                 prim=torch.zeros(1, dtype=torch.int32, device=device), total=tot)
    probe_status = torch.zeros(1, dtype=torch.int32, device=device)   # expected: capacity exceeded
    sn.raster(r.scene, r.vp, r.full_size, W, H, b, probe, probe_status)
    torch.cuda.synchronize()
    F = int(tot.cpu().numpy().view(np.uint32)[0])
    frags = dict(count=cnt, offset=off, z=torch.empty(max(F, 1), device=device),
                 prim=torch.empty(max(F, 1), dtype=torch.int32, device=device), total=tot)
    sn.raster(r.scene, r.vp, r.full_size, W, H, b, frags, r.status)
    abuf = torch.empty(P * 4, device=device)
    tail = torch.empty(P * 4, device=device)
    sn.abuffer(frags, r.rgba8, W, H, tuple(r.params.bg), abuf, tail)
    torch.cuda.synchronize()
    r.check_status()
    return dict(x=r.x.view(P, 8).clone(), tail=tail.view(P, 4), front=r.front.view(P, 4).clone(),
                abuf=abuf.view(P, 4), fragments=F)


def render_dfaoit_samples(scene: scenes.Scene, device="cuda", x_dtype=sn.F32):
    """The DFAOIT network's inputs ([P][16]), its composite terms (T_all C_b,
    1), the target transparency colour C_t = A-buffer - T_all C_b, and the
    exact A-buffer of one scene."""
    W, H = scene.width, scene.height
    d = render_samples(scene, device)
    r = Renderer(scene.verts, scene.rgba8, W, H, x_dtype=sn.F32, device=device)
    r.set_camera(scene.cam.vp32)
    P = W * H
    b = r.bins[0]
    sn.raster(r.scene, r.vp, r.full_size, W, H, b, None, r.status)
    x = torch.empty(P * 16, dtype=torch.float32 if x_dtype == sn.F32 else torch.bfloat16, device=device)
    front = torch.empty(P * 4, device=device)
    sn.build_inputs_dfaoit(r.scene, b, None, W, H, r.params, x, x_dtype, front, r.status)
    torch.cuda.synchronize()
    r.check_status()
    abuf = d["abuf"]
    ct = torch.zeros(P, 4, device=device)
    ct[:, :3] = abuf[:, :3] - front.view(P, 4)[:, :3]
    return dict(x=x.view(P, 16), front=front.view(P, 4), target=ct, abuf=abuf)


def build_dfaoit_dataset(seeds, width=512, height=512, device="cuda", log=print):
    """Inputs and target transparency colours of the pixels with a fragment."""
    xs, ys = [], []
    for i, seed in enumerate(seeds):
        d = render_dfaoit_samples(scenes.training_scene(seed, width, height), device)
        keep = d["x"][:, 11] == 1.0
        xs.append(d["x"][keep].contiguous())
        ys.append(d["target"][keep].contiguous())
        if log and (i + 1) % 50 == 0:
            log(f"  scene {i + 1}/{len(seeds)}: {sum(x.shape[0] for x in xs)} samples")
    return torch.cat(xs), torch.cat(ys)


def build_dataset(seeds, width=512, height=512, device="cuda", log=print, with_t2=False):
    """Network inputs and exact tail colours of the pixels with a tail; with
    with_t2 also each pixel's T_2 (the factor of f in Eq. 4)."""
    xs, ys, ts, n_frag = [], [], [], 0
    t0 = time.time()
    for i, seed in enumerate(seeds):
        d = render_samples(scenes.training_scene(seed, width, height), device)
        keep = d["x"][:, 5] == 1.0                   # pixels with a tail (N > 2)
        xs.append(d["x"][keep].contiguous())
        ys.append(d["tail"][keep].contiguous())
        ts.append(d["front"][keep, 3].contiguous())
        n_frag += d["fragments"]
        if log and (i + 1) % 50 == 0:
            log(f"  scene {i + 1}/{len(seeds)}: {sum(x.shape[0] for x in xs)} samples, {time.time() - t0:.1f} s")
    if with_t2:
        return torch.cat(xs), torch.cat(ys), n_frag, torch.cat(ts)
    return torch.cat(xs), torch.cat(ys), n_frag


# ---------------------------------------------------------------------------
# training

def initial_weights(seed=0):
    """Xavier-uniform weights; hidden biases 0.1 and output biases 0.5 (about
    the mean tail colour) so that no ReLU unit starts dead: with zero biases an
    output unit that starts negative on every sample never receives a
    gradient and the loss stalls far above its floor."""
    w = scenes.mlp_xavier(seed + 2)
    w["b1"][:] = 0.1
    w["b2"][:] = 0.1
    w["b3"][:] = 0.5
    return w


def train(x, y, steps=3000, batch=65536, lr=3e-3, seed=0, init=None, log=print, every=500, w=None,
          net="tail"):
    """Adam on float32 master weights (cosine-decayed learning rate); the
    forward uses the bf16-rounded copy.  w [N]: per-sample loss weights.
    net: "tail" (the 5-input tail MLP) or "dfaoit" (the comparison network)."""
    device = x.device
    g = torch.Generator(device=device).manual_seed(seed)   # indices drawn on the device: no host sync
    fn = TailMLPFunction if net == "tail" else DfaoitMLPFunction
    if net == "tail":
        flat0 = scenes.mlp_flat(init if init is not None else initial_weights(seed))
    else:
        flat0 = np.concatenate([v.ravel() for v in (init or dfaoit_initial_weights(seed)).values()]
                               ).astype(np.float32)
    master = torch.tensor(flat0, device=device)
    rounded = master.to(torch.bfloat16).to(torch.float32)
    m = torch.zeros_like(master)
    v = torch.zeros_like(master)
    N = x.shape[0]
    xb = torch.empty((batch,) + tuple(x.shape[1:]), dtype=x.dtype, device=device)
    yb = torch.empty((batch,) + tuple(y.shape[1:]), dtype=y.dtype, device=device)
    wb = torch.empty((batch, 1), dtype=w.dtype, device=device) if w is not None else None
    history = []
    t0 = time.time()
    for step in range(1, steps + 1):
        idx = torch.randint(0, N, (batch,), generator=g, device=device)
        sn.gather_rows(x, idx, xb)          # the library's row gather (one launch per array)
        sn.gather_rows(y, idx, yb)
        if w is not None:
            sn.gather_rows(w.view(-1, 1), idx, wb)
        p = rounded.clone().requires_grad_(True)
        f = fn.apply(xb.reshape(-1), p)
        loss = MSEFunction.apply(f, yb.reshape(-1), wb.reshape(-1) if w is not None else None)
        loss.backward()
        lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * (step - 1) / steps))
        sn.adam(master, p.grad, m, v, step, lr=lr_t, bf16_rounded=rounded)
        if step % every == 0 or step == 1 or step == steps:
            lv = float(loss.item())
            history.append((step, lv))
            if log:
                log(f"  step {step:5d}  loss {lv:.6f}  ({time.time() - t0:.1f} s)")
    return dict(master=master, rounded=rounded, m=m, v=v, step=steps, seed=seed, history=history)


def dfaoit_initial_weights(seed=0):
    """Xavier-uniform weights of the comparison network, hidden biases 0.1."""
    rng = np.random.Generator(np.random.PCG64(seed + 7))
    w = {}
    for name, shape in DFAOIT_SHAPES:
        if name.startswith("w"):
            lim = math.sqrt(6.0 / (shape[0] + shape[1]))
            w[name] = rng.uniform(-lim, lim, shape).astype(np.float32)
        else:
            w[name] = np.full(shape, 0.1 if name != "b3" else 0.0, np.float32)
    return w


def save_checkpoint(state, path_dir):
    os.makedirs(path_dir, exist_ok=True)
    w = flat_to_dict(state["master"])
    np.savez(os.path.join(path_dir, "tail_mlp.npz"), **w)
    np.savez(os.path.join(path_dir, "tail_mlp_checkpoint.npz"),
             master=state["master"].cpu().numpy(), m=state["m"].cpu().numpy(),
             v=state["v"].cpu().numpy(), step=state["step"], seed=state["seed"])


# ---------------------------------------------------------------------------
# evaluation: PSNR against the exact A-buffer

def psnr(a, b):
    mse = float(torch.mean((a[:, :3] - b[:, :3]) ** 2).item())
    return 10.0 * math.log10(1.0 / max(mse, 1e-30))


def evaluate(weights: dict, seeds, width=512, height=512, device="cuda"):
    """PSNR (dB, averaged over scenes) of Eq. 4 with f = 0, with the heuristic
    tail f = C~ (1 - t_tail), and with the network (bf16 tensor cores)."""
    res = {"zero": [], "heuristic": [], "mlp_bf16": [], "mlp_f32": []}
    wt = {k: torch.tensor(np.asarray(v, np.float32), device=device) for k, v in weights.items()}
    mlp = sn.mlp_struct(wt)
    for seed in seeds:
        d = render_samples(scenes.training_scene(seed, width, height), device)
        P = d["x"].shape[0]
        out = torch.empty(P * 4, device=device)

        def comp(fv):
            sn.composite(d["front"].reshape(-1), fv.reshape(-1).contiguous(), P, out, None)
            return out.view(P, 4)

        res["zero"].append(psnr(comp(torch.zeros(P, 4, device=device)), d["abuf"]))
        x = d["x"]
        heur = torch.zeros(P, 4, device=device)
        heur[:, :3] = x[:, 2:5] * (1.0 - x[:, 1:2]) * x[:, 5:6]
        res["heuristic"].append(psnr(comp(heur), d["abuf"]))
        f32 = torch.empty(P * 4, device=device)
        sn.infer(mlp, sn.F32, x.reshape(-1), f32, P)
        res["mlp_f32"].append(psnr(comp(f32), d["abuf"]))
        xb = torch.zeros(P, 8, dtype=torch.bfloat16, device=device)
        xb[:, :6] = x[:, :6].to(torch.bfloat16)
        fb = torch.empty(P * 4, device=device)
        sn.infer(mlp, sn.BF16, xb.reshape(-1), fb, P)
        res["mlp_bf16"].append(psnr(comp(fb), d["abuf"]))
    torch.cuda.synchronize()
    return {k: float(np.mean(v)) for k, v in res.items()}


def evaluate_dfaoit(weights: dict, seeds, width=512, height=512, device="cuda"):
    """PSNR (dB, mean over scenes) of the DFAOIT frame C_t + T_all C_b against
    the exact A-buffer, network on the bf16 tensor cores and in float32."""
    wt = {k: torch.tensor(np.asarray(v, np.float32), device=device) for k, v in weights.items()}
    mlp = sn.mlp_struct(wt)
    res = {"dfaoit_bf16": [], "dfaoit_f32": []}
    for seed in seeds:
        sc = scenes.training_scene(seed, width, height)
        for key, dt in (("dfaoit_f32", sn.F32), ("dfaoit_bf16", sn.BF16)):
            d = render_dfaoit_samples(sc, device, dt)
            P = d["x"].shape[0]
            f = torch.empty(P * 4, device=device)
            out = torch.empty(P * 4, device=device)
            sn.infer_dfaoit(mlp, dt, d["x"].reshape(-1), f, P)
            sn.composite(d["front"].reshape(-1), f, P, out, None)
            res[key].append(psnr(out.view(P, 4), d["abuf"]))
    torch.cuda.synchronize()
    return {k: float(np.mean(v)) for k, v in res.items()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--scenes", type=int, default=200)
    ap.add_argument("--first-seed", type=int, default=1000)
    ap.add_argument("--heldout", type=int, default=20)
    ap.add_argument("--heldout-seed", type=int, default=2000)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=65536)
    ap.add_argument("--lr", type=float, default=3e-3)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(__file__), "weights"))
    ap.add_argument("--report", default=None)
    ap.add_argument("--net", default="tail", choices=["tail", "dfaoit"],
                    help="tail: the STAR-NT tail MLP; dfaoit: the 11-input comparison network")
    ap.add_argument("--loss", default="frame", choices=["frame", "tail"],
                    help="frame: squared error of the composited frame (weights T_2^2); "
                         "tail: squared error of the tail colour")
    args = ap.parse_args()
    torch.cuda.set_device(0)
    t0 = time.time()
    heldout = range(args.heldout_seed, args.heldout_seed + args.heldout)
    if args.net == "dfaoit":
        x, y = build_dfaoit_dataset(range(args.first_seed, args.first_seed + args.scenes))
        print(f"dataset: {x.shape[0]} samples from {args.scenes} scenes, {time.time() - t0:.1f} s")
        state = train(x, y, steps=args.steps, batch=args.batch, lr=args.lr, net="dfaoit")
        w = flat_to_dict(state["master"], DFAOIT_SHAPES)
        os.makedirs(args.out, exist_ok=True)
        np.savez(os.path.join(args.out, "dfaoit_mlp.npz"), **w)
        report = {"net": "dfaoit", "samples": int(x.shape[0]), "scenes": args.scenes, "steps": args.steps,
                  "batch": args.batch, "lr": args.lr, "loss_history": state["history"],
                  "heldout_psnr_db": evaluate_dfaoit(w, heldout), "seconds": round(time.time() - t0, 1)}
        print(json.dumps(report))
        if args.report:
            with open(args.report, "w") as f:
                json.dump(report, f, indent=1)
        return
    x, y, nf, t2 = build_dataset(range(args.first_seed, args.first_seed + args.scenes), with_t2=True)
    print(f"dataset: {x.shape[0]} samples from {args.scenes} scenes ({nf} fragments), {time.time() - t0:.1f} s")
    state = train(x, y, steps=args.steps, batch=args.batch, lr=args.lr,
                  w=(t2 * t2).contiguous() if args.loss == "frame" else None)
    save_checkpoint(state, args.out)
    ev = evaluate(flat_to_dict(state["master"]), heldout)
    ev_init = evaluate(scenes.mlp_xavier(2), heldout)
    report = {"samples": int(x.shape[0]), "scenes": args.scenes, "steps": args.steps, "batch": args.batch,
              "lr": args.lr, "loss": args.loss, "loss_history": state["history"], "heldout_psnr_db": ev,
              "heldout_psnr_db_untrained_xavier": ev_init, "seconds": round(time.time() - t0, 1)}
    print(json.dumps(report))
    if args.report:
        with open(args.report, "w") as f:
            json.dump(report, f, indent=1)


if __name__ == "__main__":
    main()
