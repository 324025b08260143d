"""Run-to-run determinism of the product path.  The binning ranks a tile's
pairs by atomics and the persistent pass launches take tiles from a work
counter, so the order in which fragments and tiles are processed changes from
run to run; every output must not.  The same real frame rendered ten times
from the same state, through the pass launch that resolves the frame and
through the separate passes and resolve, and the interpolated frame from it,
must agree bit for bit: ids, depths, tail planes, float and 8-bit frames."""
import numpy as np
import pytest
import torch

from paper_2606_16747_b300 import scenes

pytestmark = pytest.mark.gpu

REPEATS = 10


@pytest.fixture(scope="module")
def sn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_16747_b300 import build, star_nt
    build.build()
    return star_nt


def _renderer(sn, merge3, tuning):
    from paper_2606_16747_b300.pipeline import Renderer
    W, H = 640, 384
    sc = scenes.screen_scene(41, 6000, W, H, size_scale=0.8, colours="coherent")
    r = Renderer(sc.verts, sc.rgba8, W, H, params=sn.default_params(base_tile=64), mlp=scenes.mlp_xavier(5),
                 x_dtype=sn.BF16, fused=True, persistent=True, tuning=tuning, merge_scale2=0.5,
                 merge_scale3=merge3)
    cams = scenes.orbit_cameras(W, H, 8, deg_per_s=30.0)
    for k in range(3):   # settle the quadtree's pass sizes
        r.set_cameras(cams[2 * k].vp32, cams[2 * k].vp64.reshape(16), cams[2 * k + 1].vp64.reshape(16))
        r.step()
    r.set_cameras(cams[6].vp32, cams[6].vp64.reshape(16), cams[7].vp64.reshape(16))
    torch.cuda.synchronize()
    return r


def _snapshot(r):
    """The planes as raw 32-bit words (bit-for-bit comparison, NaN included:
    a plane's entries beyond a reduced pass's size are never written)."""
    planes = [r.rgba32f, r.rgba8_out, r.l1["id1"], r.l1["z1"], r.interp_out, r.interp_rgba8]
    planes += [r.l2["id2"], r.l3["n"], r.l3["tail"], r.l3["t_tail"]]
    return [p.view(torch.int32).clone() for p in planes]


@pytest.mark.parametrize("merge3,tuning", [(0.7, (8, 0, 2)), (1.0, (8, 0, 2)), (0.7, (4, 10, 2)),
                                           (1.0, (8, 0, 1))])
def test_real_and_interpolated_frames_repeat_bit_for_bit(sn, merge3, tuning):
    """merge3 0.7: every pass merged, the pass launch produces the frame;
    1.0: pass 3 at its own size, the separate passes and resolve run."""
    r = _renderer(sn, merge3, tuning)
    first = None
    for rep in range(REPEATS):
        r.star_frame(update_tiles=False)   # the quadtree state stays as it is
        r.interp_frame()
        torch.cuda.synchronize()
        r.check_status()
        snap = _snapshot(r)
        if first is None:
            first = snap
            continue
        for k, (a, b) in enumerate(zip(first, snap)):
            assert torch.equal(a, b), f"plane {k} differs on repeat {rep}"
    # the frame is not trivially empty
    ids = first[2].cpu().numpy()
    assert (ids >= 0).mean() > 0.5
    assert int(r.bins[0].mem[24:28].view(torch.int32).item()) > 1000   # (triangle, tile) pairs binned
