"""Adaptive interpolation interval (Sec. 3.3, last paragraph): host logic on
the CPU, the frame sequence on the GPU."""
import numpy as np
import pytest
import torch

from paper_2606_16747_b300 import scenes
from paper_2606_16747_b300.pipeline import AdaptiveInterval


@pytest.fixture(scope="module")
def sn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_16747_b300 import build, star_nt
    build.build()
    return star_nt


def test_interval_budget_rule():
    c = AdaptiveInterval(target_fps=60.0)          # budget 16.67 ms per real frame + its interpolations
    assert c.interval() == 0                       # nothing measured: real frames
    c.observe(real_ms=10.0)
    assert c.interval() == 1                       # one interpolated frame to measure it
    c.observe(interp_ms=3.0)
    assert c.interval() == 2                       # floor((16.67 - 10) / 3)
    c = AdaptiveInterval(target_fps=60.0)
    c.observe(real_ms=4.0, interp_ms=1.0)
    assert c.interval() == 4                       # capped at four (Sec. 3.3)
    c = AdaptiveInterval(target_fps=60.0, max_interp=2)
    c.observe(real_ms=4.0, interp_ms=1.0)
    assert c.interval() == 2


def test_interval_reverts_below_target():
    c = AdaptiveInterval(target_fps=60.0, smoothing=1.0)
    c.observe(real_ms=16.0, interp_ms=1.0)
    assert c.interval() == 0                       # 0.67 ms left: no room for a 1 ms frame
    c.observe(real_ms=20.0)
    assert c.interval() == 0                       # below the target frame rate: standard rendering
    c.observe(real_ms=5.0)
    assert c.interval() == 4                       # recovers when the real frame is fast again


def test_interval_smoothing():
    c = AdaptiveInterval(target_fps=100.0, smoothing=0.25)
    c.observe(real_ms=4.0, interp_ms=2.0)
    c.observe(real_ms=8.0)                         # EMA: 4 + 0.25 * (8 - 4) = 5
    assert c.t_real == pytest.approx(5.0)
    assert c.interval() == 2                       # floor((10 - 5) / 2)
    for bad in (dict(target_fps=0), dict(max_interp=5), dict(smoothing=0.0)):
        with pytest.raises(ValueError):
            AdaptiveInterval(**bad)


@pytest.mark.gpu
def test_sequence_interpolates_from_last_real_frame(sn):
    from paper_2606_16747_b300.pipeline import Renderer, Sequence
    sc = scenes.screen_scene(7, 1500, 192, 128, size_scale=0.7, colours="coherent")
    W, H = sc.width, sc.height
    r = Renderer(sc.verts, sc.rgba8, W, H, mlp=scenes.mlp_xavier(4), x_dtype=sn.BF16, fused=True,
                 persistent=True)
    cams = scenes.orbit_cameras(W, H, 8)
    seq = Sequence(r, fixed_interval=2)
    kinds = []
    last = None
    for c in cams[:7]:
        vp64 = torch.tensor(c.vp64.reshape(16), device="cuda")
        k = seq.frame(c.vp32, vp64)
        kinds.append(k)
        torch.cuda.synchronize()
        r.check_status()
        if k == "real":
            last = (r.rgba32f.clone(), r.l1["z1"].clone(), vp64.clone())
        else:
            out = torch.zeros_like(r.interp_out)
            ws = torch.zeros(sn.REPROJECT_WS_BYTES, dtype=torch.uint8, device="cuda")
            sn.reproject(last[0], last[1], last[2], vp64, W, H, out, ws)
            torch.cuda.synchronize()
            assert torch.equal(out, r.interp_out)
    assert kinds == ["real", "interp", "interp", "real", "interp", "interp", "real"]


@pytest.mark.gpu
def test_sequence_adaptive(sn):
    from paper_2606_16747_b300.pipeline import Renderer, Sequence
    sc = scenes.screen_scene(8, 1500, 192, 128, size_scale=0.7)
    W, H = sc.width, sc.height
    r = Renderer(sc.verts, sc.rgba8, W, H, mlp=scenes.mlp_xavier(4), x_dtype=sn.BF16, fused=True)
    seq = Sequence(r, controller=AdaptiveInterval(target_fps=60.0))
    cams = scenes.orbit_cameras(W, H, 24)
    for c in cams:
        seq.frame(c.vp32, torch.tensor(c.vp64.reshape(16), device="cuda"))
        torch.cuda.synchronize()
    r.check_status()
    # sub-millisecond frames against a 16.7 ms budget: the interval opens up to four
    assert seq.kinds[0] == "real"
    assert "interp" in seq.kinds
    assert seq.ctl.interval() == 4
    runs = "".join("r" if k == "real" else "i" for k in seq.kinds).split("r")
    assert max(len(x) for x in runs) <= 4
