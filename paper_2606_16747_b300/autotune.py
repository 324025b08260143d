"""Autotuner of the persistent geometry-pass launch: tries tile shapes (the
pixel block a warp owns inside a 16 x 16 tile), one or two pixels per thread
and resident CTAs per SM on the renderer's own workload, and keeps the
fastest; then, with that shape,
whether the pass launch should also produce the frame when every pass runs at
full size (the network inside the pass launch against the separate resolve).
Results are stored per workload key in a JSON file next to this module."""
from __future__ import annotations

import json
import os

import torch

TUNED_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")
# (block_w, ctas_per_sm, pixels_per_thread) of star_nt_tuning
CANDIDATES = [(8, 0, 2), (4, 0, 2), (16, 0, 2), (8, 10, 2), (4, 10, 2), (8, 0, 1), (4, 0, 1), (8, 6, 1),
              (4, 6, 1)]


def candidate_key(c) -> str:
    bw, k, pix = c
    return f"{bw}x{32 // bw}/{k}/{pix}px"


def workload_key(renderer) -> str:
    return f"{renderer.W}x{renderer.H}_T{renderer.T}"


def time_stages(renderer, names, reps=10) -> float:
    """Average ms of the named stages of one real frame, replayed back to back
    as one graph."""
    stages = dict(renderer.star_stages())
    fns = [stages[n] for n in names]

    def run():
        for fn in fns:
            fn()

    g = renderer.capture(run)
    g.replay()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def time_passes(renderer, tuning, reps=10) -> float:
    """Average ms of one persistent pass launch (graph replays back to back)."""
    old = renderer.tuning, renderer.persistent
    renderer.tuning, renderer.persistent = tuning, True
    try:
        return time_stages(renderer, ["passes"], reps)
    finally:
        renderer.tuning, renderer.persistent = old


def all_merged(renderer) -> bool:
    """Whether the renderer's last raster took both reduced passes over into
    pass 1 (the merged word of the pass-2 and pass-3 bins headers)."""
    return all(int(renderer.bins[k].mem[32:36].view(torch.int32).item()) != 0 for k in (1, 2))


def tune(renderer, candidates=CANDIDATES, reps=10) -> dict:
    """Time every candidate on the renderer's current frame state (bins and
    pass sizes must be those of a real frame) and return the fastest, with the
    fused-resolve choice when the renderer can make it.  That choice is only
    measured on a frame whose reduced passes are both merged: otherwise the
    pass launch returns at once in either setting and the comparison says
    nothing, so the launch that resolves stays on."""
    times = {candidate_key(c): time_passes(renderer, tuple(c), reps) for c in candidates}
    best = tuple(min(candidates, key=lambda c: times[candidate_key(c)]))
    out = {"block_w": best[0], "ctas_per_sm": best[1], "pixels_per_thread": best[2], "ms": times}
    if getattr(renderer, "leaf", False) or not (renderer.fused and not renderer.fused_fp8):
        return out
    old = renderer.tuning, renderer.persistent, renderer.fuse_passes
    renderer.tuning, renderer.persistent = best, True
    try:
        both = {}
        for fuse in (True, False):
            renderer.fuse_passes = fuse
            # the raster resets the frame's resolved mark, so both settings
            # start every replay from the same state
            both[fuse] = time_stages(renderer, ["raster", "passes", "resolve"], reps)
    finally:
        renderer.tuning, renderer.persistent, renderer.fuse_passes = old
    merged = all_merged(renderer)
    out["fuse_passes"] = both[True] <= both[False] or not merged
    out["raster_passes_resolve_ms"] = {"pass launch resolves": both[True], "separate resolve": both[False],
                                       "frame merged": merged}
    return out


def load(key: str):
    try:
        with open(TUNED_PATH) as f:
            d = json.load(f).get(key)
        return (d["block_w"], d["ctas_per_sm"], d.get("pixels_per_thread", 1)) if d else None
    except (OSError, ValueError, KeyError):
        return None


def save(key: str, result: dict) -> None:
    try:
        with open(TUNED_PATH) as f:
            d = json.load(f)
    except (OSError, ValueError):
        d = {}
    d[key] = result
    with open(TUNED_PATH, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
