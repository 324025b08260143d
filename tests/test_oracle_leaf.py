"""Pins of the per-leaf resolution variant (Eq. 2 with the scene index
replaced by the level of the pixel's own quadtree leaf): the per-pixel levels
read from the split masks, the per-level pass sizes, and the frame against the
global-scale frames it selects from."""
import numpy as np
import pytest

from paper_2606_16747_b300 import scenes


def paint_levels(mask, W, H, B):
    """Levels by painting every leaf node's square (a second formulation:
    walk the nodes the mask creates instead of descending per pixel)."""
    TX = (W + B - 1) // B
    out = np.full((H, W), 255, np.uint8)
    for t, m in enumerate(np.asarray(mask, np.uint32).tolist()):
        x0, y0 = (t % TX) * B, (t // TX) * B

        def paint(l, i, j):
            S = B >> l
            out[y0 + j * S:y0 + (j + 1) * S, x0 + i * S:x0 + (i + 1) * S] = l

        if not m & 1:
            paint(0, 0, 0)
            continue
        for c1 in range(4):
            i1, j1 = c1 & 1, c1 >> 1
            if not (m >> (1 + c1)) & 1:
                paint(1, i1, j1)
                continue
            for c2 in range(4):
                i2, j2 = 2 * i1 + (c2 & 1), 2 * j1 + (c2 >> 1)
                if not (m >> (5 + 4 * c1 + c2)) & 1:
                    paint(2, i2, j2)
                    continue
                for c3 in range(4):
                    paint(3, 2 * i2 + (c3 & 1), 2 * j2 + (c3 >> 1))
    return out.reshape(-1)


def test_leaf_levels_hand_cases(orc):
    B = 16
    lv = orc.leaf_levels(np.array([0], np.uint32), B, B, B)
    assert (lv == 0).all()
    lv = orc.leaf_levels(np.array([1], np.uint32), B, B, B).reshape(B, B)
    assert (lv == 1).all()
    # root split, level-1 child 1 (right half, top) split, its level-2 child 3 split
    m = 1 | (1 << 2) | (1 << (5 + 4 * 1 + 3))
    lv = orc.leaf_levels(np.array([m], np.uint32), B, B, B).reshape(B, B)
    assert (lv[8:, :] == 1).all() and (lv[:8, :8] == 1).all()
    assert (lv[4:8, 12:16] == 3).all()
    assert (lv[:4, 8:16] == 2).all() and (lv[4:8, 8:12] == 2).all()


@pytest.mark.parametrize("B", [16, 64])
def test_leaf_levels_match_painted_nodes(orc, B):
    rng = np.random.default_rng(B)
    W, H = 3 * B, 2 * B
    masks = []
    for _ in range(6):
        m = 0
        if rng.random() < 0.8:
            m |= 1
            for c1 in range(4):
                if rng.random() < 0.6:
                    m |= 1 << (1 + c1)
                    for c2 in range(4):
                        if rng.random() < 0.5:
                            m |= 1 << (5 + 4 * c1 + c2)
        masks.append(m)
    masks = np.array(masks, np.uint32)
    assert np.array_equal(orc.leaf_levels(masks, W, H, B), paint_levels(masks, W, H, B))


def test_leaf_levels_reproduce_the_leaf_histogram(orc):
    """Occupied leaves counted from the per-pixel levels equal the quadtree's
    histogram (Sec. 3.2), computed by the C oracle from the masks directly."""
    rng = np.random.default_rng(11)
    W, H, B = 96, 80, 16
    yy, xx = np.divmod(np.arange(W * H), W)
    # flat left part, a hard vertical edge, noise in the lower right corner
    img = np.where(xx < 40, 0x202020, 0xC0C0C0).astype(np.uint32)
    noisy = (xx >= 64) & (yy >= 48)
    img[noisy] = rng.integers(0, 1 << 24, size=int(noisy.sum()), dtype=np.uint32)
    img |= np.uint32(0xFF000000)
    id1 = np.where(rng.random(W * H) < 0.05, 0, -1).astype(np.int32)
    mask = np.zeros((W // B) * (H // B), np.uint32)
    for _ in range(4):  # a few frames: mixed levels
        mask, hist = orc.quadtree(img, id1, W, H, B, 150.0, 60.0, mask)
    lv = orc.leaf_levels(mask, W, H, B)
    assert len(set(lv.tolist())) >= 3
    counts = []
    for l in range(4):
        S = B >> l
        sel = (lv == l) & (id1 >= 0)
        counts.append(len(set(zip((yy[sel] // S).tolist(), (xx[sel] // S).tolist()))))
    assert counts == hist.tolist()


def test_leaf_sizes_closed_form(orc):
    # s_p(l) = clamp(2^(l - delta_p), 1/4, 1): pass 2 (delta 2.2) 1/4, 2^-1.2,
    # 2^-0.2, 1; pass 3 (delta 3) 1/4, 1/4, 1/2, 1
    sz = orc.leaf_sizes(96, 64)
    assert [sz[(2, l)] for l in range(4)] == [(24, 16), (42, 28), (84, 56), (96, 64)]
    assert [sz[(3, l)] for l in range(4)] == [(24, 16), (24, 16), (48, 32), (96, 64)]
    assert 96 * 2 ** -1.2 == pytest.approx(41.786, abs=1e-3) and 64 * 2 ** -0.2 == pytest.approx(55.716, abs=1e-3)


@pytest.fixture(scope="module")
def leaf_case():
    sc = scenes.screen_scene(21, 700, 96, 64, size_scale=0.6)
    return sc, scenes.mlp_flat(scenes.mlp_xavier(5))


def test_uniform_levels_equal_global_frames(orc, leaf_case):
    """Every leaf at one level is the global frame at that level's sizes."""
    sc, w = leaf_case
    W, H = sc.width, sc.height
    sz = orc.leaf_sizes(W, H)
    for l in range(4):
        t = orc.frame_star_leaf(sc.verts, sc.rgba8, sc.cam.vp32, W, H, np.full(W * H, l, np.uint8), w)
        ref = orc.frame_star(sc.verts, sc.rgba8, sc.cam.vp32, W, H, sz[(2, l)], sz[(3, l)], w)
        assert np.array_equal(t["rgb"], ref["rgb"])


def test_mixed_levels_select_per_pixel(orc, leaf_case):
    """With levels mixed over the frame, each pixel equals the global frame at
    its own leaf's sizes (one target's upscale does not depend on the other
    pixels' levels)."""
    sc, w = leaf_case
    W, H, B = sc.width, sc.height, 16
    rng = np.random.default_rng(8)
    mask = rng.integers(0, 1 << 21, size=(W // B) * (H // B)).astype(np.uint32)
    lv = orc.leaf_levels(mask, W, H, B)
    t = orc.frame_star_leaf(sc.verts, sc.rgba8, sc.cam.vp32, W, H, lv, w)
    sz = orc.leaf_sizes(W, H)
    for l in range(4):
        sel = lv == l
        if sel.any():
            ref = orc.frame_star(sc.verts, sc.rgba8, sc.cam.vp32, W, H, sz[(2, l)], sz[(3, l)], w)
            assert np.array_equal(t["rgb"][sel], ref["rgb"][sel])
