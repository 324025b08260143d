"""Pins of the per-tile resolution variant (Eq. 2 per base tile): the grid
rule, the per-tile histograms, and the tiled frame against the global-scale
frames it selects from."""
import numpy as np
import pytest

from paper_2606_16747_b300 import scenes


def test_tile_grid_rule(orc):
    th = np.array([[0, 0, 0, 5],     # only level-3 leaves: wbar 3
                   [7, 0, 0, 0],     # only level 0: wbar 0
                   [0, 3, 0, 0],     # wbar 1
                   [0, 1, 4, 0],     # wbar 1.8
                   [0, 0, 0, 0],     # no occupied leaf
                   [1, 1, 1, 1]],    # wbar 1.5
                  np.uint32)
    # delta - wbar < 1/2 -> 1, < 3/2 -> 2, else 4
    assert orc.tile_grid(th, 2.2).tolist() == [1, 4, 2, 1, 4, 2]   # -0.8, 2.2, 1.2, 0.4, -, 0.7
    assert orc.tile_grid(th, 3.0).tolist() == [1, 4, 4, 2, 4, 4]   # 0, 3, 2, 1.2, -, 1.5


def test_tile_histograms_sum_to_global(orc):
    rng = np.random.default_rng(3)
    W, H, B = 96, 64, 16
    img = rng.integers(0, 1 << 24, size=W * H, dtype=np.uint32) | np.uint32(0xFF000000)
    id1 = np.where(rng.random(W * H) < 0.7, 0, -1).astype(np.int32)
    mprev = np.zeros((W // B) * (H // B), np.uint32)
    mask, hist, th = orc.quadtree(img, id1, W, H, B, 20.0, 9.0, mprev, per_tile=True)
    assert np.array_equal(th.sum(axis=0), hist)
    mask2, hist2 = orc.quadtree(img, id1, W, H, B, 20.0, 9.0, mprev)
    assert np.array_equal(mask, mask2) and np.array_equal(hist, hist2)


@pytest.fixture(scope="module")
def tiled_case():
    sc = scenes.screen_scene(21, 700, 96, 64, size_scale=0.6)
    return sc, scenes.mlp_flat(scenes.mlp_xavier(5))


def test_tiled_uniform_grids_equal_global_frames(orc, tiled_case):
    """Every tile at one spacing is the global frame at that resolution."""
    sc, w = tiled_case
    W, H = sc.width, sc.height
    nt = (W // 16) * (H // 16)
    for g2, g3 in ((1, 1), (2, 4), (4, 2)):
        t = orc.frame_star_tiled(sc.verts, sc.rgba8, sc.cam.vp32, W, H, np.full(nt, g2), np.full(nt, g3), w)
        ref = orc.frame_star(sc.verts, sc.rgba8, sc.cam.vp32, W, H, (W // g2, H // g2), (W // g3, H // g3), w)
        assert np.array_equal(t["rgb"], ref["rgb"])


def test_tiled_mixed_grids_select_per_pixel(orc, tiled_case):
    """With grids mixed over the tiles, each pixel equals the global frame of
    its own tile's spacings (the upscale of one target does not depend on the
    other tiles' choice)."""
    sc, w = tiled_case
    W, H = sc.width, sc.height
    TX, TY = W // 16, H // 16
    rng = np.random.default_rng(8)
    g2 = rng.choice([1, 2, 4], size=TX * TY).astype(np.uint8)
    g3 = rng.choice([1, 2, 4], size=TX * TY).astype(np.uint8)
    t = orc.frame_star_tiled(sc.verts, sc.rgba8, sc.cam.vp32, W, H, g2, g3, w)
    yy, xx = np.divmod(np.arange(W * H), W)
    tile = (yy // 16) * TX + xx // 16
    for a in (1, 2, 4):
        for b in (1, 2, 4):
            sel = (g2[tile] == a) & (g3[tile] == b)
            if not sel.any():
                continue
            ref = orc.frame_star(sc.verts, sc.rgba8, sc.cam.vp32, W, H, (W // a, H // a), (W // b, H // b), w)
            assert np.array_equal(t["rgb"][sel], ref["rgb"][sel])
