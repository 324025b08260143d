"""Per-leaf pass resolution on the GPU (Eq. 2 with the scene index replaced
by the level of each pixel's quadtree leaf): the frame against the oracle's
per-leaf frame, the per-tile pass modes against the tiles the pixels' bilinear
footprints touch, and uniform levels against the global-scale renderer."""
import numpy as np
import pytest
import torch

from paper_2606_16747_b300 import scenes

pytestmark = pytest.mark.gpu

TOL_BF16 = 2.0 / 255.0   # bf16 MLP, frame error <= MLP error (scaled by T_2 <= 1)


@pytest.fixture(scope="module")
def sn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_16747_b300 import build, star_nt
    build.build()
    return star_nt


def random_masks(rng, n, p_root=0.8, p1=0.6, p2=0.5):
    m = np.zeros(n, np.uint32)
    for t in range(n):
        v = 0
        if rng.random() < p_root:
            v |= 1
            for c1 in range(4):
                if rng.random() < p1:
                    v |= 1 << (1 + c1)
                    for c2 in range(4):
                        if rng.random() < p2:
                            v |= 1 << (5 + 4 * c1 + c2)
        m[t] = v
    return m


def leaf_renderer(sn, sc, masks, B=16, fused=True, mlp=None, tuning=None):
    from paper_2606_16747_b300.pipeline import Renderer
    r = Renderer(sc.verts, sc.rgba8, sc.width, sc.height, mlp=mlp or scenes.mlp_xavier(4), x_dtype=sn.BF16,
                 fused=fused, leaf=True, base_tile=B, tuning=tuning)
    r.set_camera(sc.cam.vp32)
    if masks is not None:
        r.mask[0].copy_(torch.as_tensor(masks.view(np.int32)))
    return r


def axis_taps(n_full, n_target):
    """Per full-resolution pixel: the target samples of nonzero bilinear
    weight (half-pixel centres, clamp to edge), as (i0, i1 or -1)."""
    x = np.arange(n_full, dtype=np.int64)
    num = (2 * x + 1) * n_target - n_full
    q = np.floor_divide(num, 2 * n_full)
    rem = num - q * 2 * n_full
    i0 = np.clip(q, 0, n_target - 1)
    i1 = np.where(rem > 0, np.clip(q + 1, 0, n_target - 1), -1)
    return i0, i1


def expected_modes(plan, levels, W, H):
    """Mode byte of every target tile: bit 0 when a pixel whose level maps
    pass 2 to the target has a nonzero-weight sample in the tile, bit 1 the
    same for pass 3."""
    lv = levels.reshape(H, W)
    out = []
    for k, (Wk, Hk) in enumerate(plan.sizes()):
        tx_n, ty_n = (Wk + 15) // 16, (Hk + 15) // 16
        mode = np.zeros((ty_n, tx_n), np.uint8)
        x0, x1 = axis_taps(W, Wk)
        y0, y1 = axis_taps(H, Hk)
        for bit, p in ((1, 2), (2, 3)):
            lmask = np.isin(lv, [l for l, t in enumerate(plan.targets(p)) if t == k])
            ys, xs = np.nonzero(lmask)
            for sy in (y0[ys], y1[ys]):
                for sx in (x0[xs], x1[xs]):
                    ok = (sx >= 0) & (sy >= 0)
                    mode[sy[ok] // 16, sx[ok] // 16] |= bit
        out.append(mode.reshape(-1))
    return np.concatenate(out)


@pytest.mark.parametrize("B", [16, 64])
def test_leaf_frame_matches_oracle(orc, sn, B):
    sc = scenes.screen_scene(29, 3000, 333, 197, size_scale=0.7)   # ragged: partial tiles
    W, H = sc.width, sc.height
    rng = np.random.default_rng(B)
    masks = random_masks(rng, ((W + B - 1) // B) * ((H + B - 1) // B))
    mlp = scenes.mlp_xavier(4)
    r = leaf_renderer(sn, sc, masks, B, mlp=mlp)
    r.star_frame(update_tiles=False)
    torch.cuda.synchronize()
    r.check_status()
    lv = orc.leaf_levels(masks, W, H, B)
    assert len(set(lv.tolist())) == 4
    o = orc.frame_star_leaf(sc.verts, sc.rgba8, sc.cam.vp32, W, H, lv, scenes.mlp_flat(mlp), threads=4)
    # pass 1 is exact; the modes are exactly the tiles some pixel samples
    assert np.array_equal(r.l1["id1"].cpu().numpy(), o["res"][(W, H)]["id1"])
    modes = r.leaf_ws.cpu().numpy()[:sum(((w + 15) // 16) * ((h + 15) // 16) for w, h in r.plan.sizes())]
    assert np.array_equal(modes, expected_modes(r.plan, lv, W, H))
    # every needed sample of every target equals the oracle's planes
    for k, (Wk, Hk) in enumerate(r.plan.sizes()):
        ref = o["res"].get((Wk, Hk))
        if ref is None:
            continue
        m = modes[sum(((w + 15) // 16) * ((h + 15) // 16) for w, h in r.plan.sizes()[:k]):][
            :((Wk + 15) // 16) * ((Hk + 15) // 16)].reshape((Hk + 15) // 16, (Wk + 15) // 16)
        yy, xx = np.divmod(np.arange(Wk * Hk), Wk)
        tm = m[yy // 16, xx // 16]
        L = r.leaf_layers[k]
        if "id2" in L and (tm & 1).any():
            sel = (tm & 1) != 0
            assert np.array_equal(L["id2"][:Wk * Hk].cpu().numpy()[sel], ref["id2"][sel])
        if "n" in L and (tm & 2).any():
            sel = (tm & 2) != 0
            assert np.array_equal(L["n"][:Wk * Hk].cpu().numpy()[sel], ref["n"].astype(np.int32)[sel])
    rgb = r.rgba32f.cpu().numpy().reshape(-1, 4)[:, :3]
    err = np.abs(rgb - o["rgb"])
    assert err.max() <= TOL_BF16, err.max() * 255
    no_tail = o["flag"] == 0
    if no_tail.any():   # f = 0: exact up to the float32 front terms
        assert err[no_tail].max() <= 1e-5


@pytest.mark.parametrize("level", [0, 1, 2, 3])
@pytest.mark.parametrize("fused", [True, "fp8", "fp8x2", "fp8t", "fp8x2t"])
def test_uniform_levels_equal_global_renderer(sn, level, fused):
    """All leaves at one level: the per-leaf frame is the global-scale frame
    at that level's sizes, bit for bit (same planes, same resolve arithmetic)."""
    from paper_2606_16747_b300.pipeline import Renderer
    sc = scenes.screen_scene(37, 2500, 208, 144, size_scale=0.7)
    W, H = sc.width, sc.height
    n = (W // 16) * (H // 16)
    full = [0, 1, (1 << 5) - 1, (1 << 21) - 1][level]
    r = leaf_renderer(sn, sc, np.full(n, full, np.uint32), fused=fused)
    r.star_frame(update_tiles=False)
    torch.cuda.synchronize()
    r.check_status()
    s2 = r.plan.sizes()[r.plan.targets(2)[level]]
    s3 = r.plan.sizes()[r.plan.targets(3)[level]]
    g = Renderer(sc.verts, sc.rgba8, W, H, mlp=scenes.mlp_xavier(4), x_dtype=sn.BF16, fused=fused,
                 persistent=True)
    g.set_camera(sc.cam.vp32)
    g.state.view(torch.int32)[:6] = torch.tensor([W, H, *s2, *s3], dtype=torch.int32)
    g.star_frame(update_tiles=False)
    torch.cuda.synchronize()
    g.check_status()
    assert torch.equal(r.rgba32f, g.rgba32f) and torch.equal(r.rgba8_out, g.rgba8_out)


def test_leaf_frames_repeat_and_graph_replay(sn):
    """The persistent launch's work counter resets itself: eager frames and
    graph replays give the same frame; the quadtree then updates the masks in
    place and the next frame follows them."""
    sc = scenes.screen_scene(41, 2500, 208, 144, size_scale=0.7, colours="coherent")
    r = leaf_renderer(sn, sc, None, tuning=(16, 6, 1))
    r.star_frame(update_tiles=False)
    torch.cuda.synchronize()
    first = r.rgba32f.clone()
    g = r.capture(lambda: r.star_frame(update_tiles=False))
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    r.check_status()
    assert torch.equal(first, r.rgba32f)
    for _ in range(4):
        r.star_frame()
    torch.cuda.synchronize()
    r.check_status()
    m = r.mask[0].cpu().numpy().view(np.uint32)
    assert (m != (1 << 21) - 1).any()   # uniform regions merged
