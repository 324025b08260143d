"""Autotuner of the persistent geometry-pass launch: tries tile shapes (the
pixel block a warp owns inside a 16 x 16 tile) and resident CTAs per SM on
the renderer's own workload, and keeps the fastest.  Results are stored per
workload key in a JSON file next to this module."""
from __future__ import annotations

import json
import os

import torch

TUNED_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")
CANDIDATES = [(8, 0), (16, 0), (4, 0), (8, 6), (16, 6), (4, 6)]


def workload_key(renderer) -> str:
    return f"{renderer.W}x{renderer.H}_T{renderer.T}"


def time_passes(renderer, tuning, reps=10) -> float:
    """Average ms of one persistent pass launch (graph replays back to back)."""
    old = renderer.tuning, renderer.persistent
    renderer.tuning, renderer.persistent = tuning, True
    try:
        fn = dict(renderer.star_stages())["passes"]
        g = renderer.capture(fn)
        g.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps
    finally:
        renderer.tuning, renderer.persistent = old


def tune(renderer, candidates=CANDIDATES, reps=10) -> dict:
    """Time every candidate on the renderer's current frame state (bins and
    pass sizes must be those of a real frame) and return the fastest."""
    times = {f"{bw}x{32 // bw}/{k}": time_passes(renderer, (bw, k), reps) for bw, k in candidates}
    best = min(candidates, key=lambda c: times[f"{c[0]}x{32 // c[0]}/{c[1]}"])
    return {"block_w": best[0], "ctas_per_sm": best[1], "ms": times}


def load(key: str):
    try:
        with open(TUNED_PATH) as f:
            d = json.load(f).get(key)
        return (d["block_w"], d["ctas_per_sm"]) if d else None
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
