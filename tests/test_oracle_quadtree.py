"""Pins of the oracle's adaptive tiles (Sec. 3.1) and tile-guided resolution
(Sec. 3.2, Eq. 2): the printed Eq. 2 values, hand-built corner colours,
quadtree invariants and brute-force leaf histograms."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "eq2_scales.txt")


def _rows():
    out = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            out.append([float(v) for v in line.split()])
    return out


def test_eq2_golden(orc):
    for wbar, s2, s3 in _rows():
        assert orc.pass_scale(wbar, 2.2) == pytest.approx(s2, abs=1e-12)
        assert orc.pass_scale(wbar, 3.0) == pytest.approx(s3, abs=1e-12)


def test_eq2_doubling_and_clamp(orc):
    for w in (1.5, 1.9, 2.0):
        assert orc.pass_scale(w + 0.2 - 1, 2.2) * 2 == pytest.approx(orc.pass_scale(w + 0.2, 2.2), rel=1e-14)
    assert orc.pass_scale(-5, 2.2) == 0.25 and orc.pass_scale(10, 3.0) == 1.0
    assert orc.pass_size(0.25, 1080) == 270 and orc.pass_size(0.4, 1921) == 769


def test_wbar_definition(orc):
    assert orc.wbar([4, 0, 0, 0]) == 0.0
    assert orc.wbar([0, 0, 0, 7]) == 3.0
    assert orc.wbar([1, 1, 1, 1]) == 1.5
    assert orc.wbar([0, 0, 0, 0]) == 0.0


# --- mask helpers written independently of the oracle (recursive descent) ---

def leaves(mask):
    """All leaves (level, i, j) of one tile by recursive descent."""
    out = []

    def bit(l, i, j):
        if l == 0:
            return 0
        if l == 1:
            return 1 + (j << 1 | i)
        return 5 + 4 * (((j >> 1) << 1) | (i >> 1)) + ((j & 1) << 1 | (i & 1))

    def rec(l, i, j):
        if l < 3 and (mask >> bit(l, i, j)) & 1:
            for c in range(4):
                rec(l + 1, 2 * i + (c & 1), 2 * j + (c >> 1))
        else:
            out.append((l, i, j))
    rec(0, 0, 0)
    return out


def level_grid(masks, TX, TY):
    g = np.zeros((TY * 8, TX * 8), np.int32)
    for t, m in enumerate(masks):
        tx, ty = t % TX, t // TX
        for l, i, j in leaves(int(m)):
            s = 8 >> l
            g[ty * 8 + j * s: ty * 8 + (j + 1) * s, tx * 8 + i * s: tx * 8 + (i + 1) * s] = l
    return g


def max_neighbour_gap(g):
    return max(np.abs(np.diff(g, axis=0)).max(initial=0), np.abs(np.diff(g, axis=1)).max(initial=0))


def test_corner_distance_mean_and_strictness(orc):
    """Only the four corner pixels of the root node carry colour; one corner is
    (0, 0, 6) and the rest black, so D = (6 + 6 + 6) / 6 = 3.  The node splits
    for tau_split < 3 and not for tau_split = 3 (strict inequality)."""
    W = H = 16
    img = np.full(W * H, 0xFF000000, np.uint32)
    img[15 * W + 15] = 0xFF000000 | (6 << 16)
    id1 = np.zeros(W * H, np.int32)
    m, _ = orc.quadtree(img, id1, W, H, 16, 3.0, -1.0, np.zeros(1, np.uint32), relax_iters=0)
    assert m[0] == 0
    m, _ = orc.quadtree(img, id1, W, H, 16, 2.999, -1.0, np.zeros(1, np.uint32), relax_iters=0)
    assert m[0] == 1
    # colour at a non-corner pixel is invisible to the root node
    img2 = np.full(W * H, 0xFF000000, np.uint32)
    img2[7 * W + 9] = 0xFFFFFFFF
    m, _ = orc.quadtree(img2, id1, W, H, 16, 1.0, -1.0, np.zeros(1, np.uint32), relax_iters=0)
    assert m[0] == 0


def test_constant_image_merges_one_level_per_frame(orc):
    W, H, B = 64, 48, 16
    TX, TY = 4, 3
    img = np.full(W * H, 0xFF336699, np.uint32)
    id1 = np.zeros(W * H, np.int32)
    mask = np.full(TX * TY, (1 << 21) - 1, np.uint32)
    prev_g = level_grid(mask, TX, TY)
    for frame in range(3):
        mask, hist = orc.quadtree(img, id1, W, H, B, 24, 12, mask)
        g = level_grid(mask, TX, TY)
        assert np.abs(g - prev_g).max() == 1 and np.all(g == 2 - frame)
        prev_g = g
    assert np.all(mask == 0) and hist.tolist() == [TX * TY, 0, 0, 0]


def test_edge_refines_and_stays_balanced(orc):
    """A hard colour edge refines the leaves it crosses down to level 3, one
    level per frame; neighbours never differ by more than one level; a static
    image converges and then stays fixed."""
    W, H, B = 96, 64, 16
    TX, TY = 6, 4
    yy, xx = np.mgrid[0:H, 0:W]
    img = np.where(xx < 37, 0xFF000000, 0xFFFFFFFF).astype(np.uint32).reshape(-1)
    id1 = np.zeros(W * H, np.int32)
    mask = np.zeros(TX * TY, np.uint32)
    prev_g = level_grid(mask, TX, TY)
    history = []
    for frame in range(6):
        mask, hist = orc.quadtree(img, id1, W, H, B, 24, 12, mask)
        g = level_grid(mask, TX, TY)
        assert max_neighbour_gap(g) <= 1
        history.append(mask.copy())
        prev_g = g
    assert np.array_equal(history[-1], history[-2]) and np.array_equal(history[-2], history[-3])
    g = level_grid(history[-1], TX, TY)
    # the cells containing the edge pixels (x = 36 | 37) are finest
    assert np.all(g[:, 36 * 8 // B] == 3) and np.all(g[:, 37 * 8 // B] == 3)
    # far from the edge the tiles stay coarse
    assert np.all(g[:, -8:] <= 1)


def test_level_change_at_most_one_without_relaxation(orc):
    rng = np.random.default_rng(0)
    W, H, B = 64, 64, 16
    TX = TY = 4
    mask = np.zeros(TX * TY, np.uint32)
    for frame in range(5):
        img = rng.integers(0, 2 ** 32, W * H, dtype=np.uint64).astype(np.uint32) | np.uint32(0xFF000000)
        if frame % 2:
            img[:] = img[0]
        new, _ = orc.quadtree(img, np.zeros(W * H, np.int32), W, H, B, 60, 30, mask, relax_iters=0)
        assert np.abs(level_grid(new, TX, TY) - level_grid(mask, TX, TY)).max() <= 1
        for m in new:   # a set child bit implies a set parent bit
            m = int(m)
            for c1 in range(4):
                if (m >> (1 + c1)) & 1:
                    assert m & 1
                for c2 in range(4):
                    if (m >> (5 + 4 * c1 + c2)) & 1:
                        assert (m >> (1 + c1)) & 1
        mask = new


def test_relaxation_exact_masks(orc):
    """Tile A fully refined (level 3) left of tile B at level 0, thresholds
    inert: relaxation splits B's root, then B's two level-1 children that
    touch A (children 0 and 2): mask_B = 1 | 2 | 8."""
    W, H, B = 32, 16, 16
    img = np.full(W * H, 0xFF000000, np.uint32)
    id1 = np.full(W * H, -1, np.int32)
    mp = np.array([(1 << 21) - 1, 0], np.uint32)
    m1, _ = orc.quadtree(img, id1, W, H, B, 1e9, -1.0, mp, relax_iters=1)
    assert m1.tolist() == [(1 << 21) - 1, 1]
    m2, _ = orc.quadtree(img, id1, W, H, B, 1e9, -1.0, mp, relax_iters=2)
    assert m2.tolist() == [(1 << 21) - 1, 1 | 2 | 8]
    assert max_neighbour_gap(level_grid(m2, 2, 1)) == 1


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_histogram_brute_force(orc, seed):
    """With inert thresholds and no relaxation the mask is kept, and the
    histogram counts leaves with at least one covered pixel, per level."""
    rng = np.random.default_rng(seed)
    W, H, B = 80, 56, 16           # partial tiles on the right and bottom
    TX, TY = 5, 4
    masks = []
    for _ in range(TX * TY):       # random consistent masks
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
    id1 = np.where(rng.random(W * H) < 0.02, 0, -1).astype(np.int32)
    img = np.zeros(W * H, np.uint32)
    out, hist = orc.quadtree(img, id1, W, H, B, 1e9, -1.0, masks, relax_iters=0)
    assert np.array_equal(out, masks)
    exp = [0, 0, 0, 0]
    cov = id1.reshape(H, W) >= 0
    for t, m in enumerate(masks):
        tx, ty = t % TX, t // TX
        for l, i, j in leaves(int(m)):
            s = B >> l
            x0, y0 = tx * B + i * s, ty * B + j * s
            if cov[y0:min(y0 + s, H), x0:min(x0 + s, W)].any():
                exp[l] += 1
    assert hist.tolist() == exp
