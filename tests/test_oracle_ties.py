"""Pins of the depth-tie rule: fragments are ordered by the key (depth,
primitive id), so among fragments of equal depth the lower primitive id is
nearer (Sec. 3.3 orders the layers by depth; the id breaks ties).

The scenes stack axis-aligned rectangles at a handful of shared, exactly
representable depths, their triangles submitted in shuffled order.  Which
triangles cover a pixel centre follows from the rectangle geometry alone (no
centre lies on a border or a diagonal), and the expected layers are written
from the rule itself: the nearest fragment is the lowest id among those at
the minimum depth; the second is the next-lowest id at that depth when there
is one, else the lowest id at the next depth.  A reversed or missing tie rule
fails these tests."""
import numpy as np
import pytest

from tests.helpers import TIE_DEPTHS, pixel_vp, rgba, tied_rect_scene, quad

BG = (0.25, 0.5, 1.0)


def covering(meta, W, H):
    """Per pixel, the (depth, id) of the triangles whose interior holds the
    pixel centre, from the rectangle geometry."""
    out = [[] for _ in range(W * H)]
    for (x0, y0, x1, y1, z, ida, idb) in meta:
        for y in range(max(0, y0), min(H, y1)):
            cy = y + 0.5
            for x in range(max(0, x0), min(W, x1)):
                cx = x + 0.5
                # below the diagonal (x0, y0) -> (x1, y1) in y-down screen
                # coordinates is triangle a, which holds the corner (x1, y0)
                below = (cx - x0) * (y1 - y0) > (cy - y0) * (x1 - x0)
                out[y * W + x].append((z, ida if below else idb))
    return out


def expected_layers(frags):
    """(id1, z1, id2) of one pixel from the tie rule, without sorting keys."""
    if not frags:
        return -1, 1.0, -1
    zmin = min(z for z, _ in frags)
    at_min = sorted(i for z, i in frags if z == zmin)
    if len(at_min) >= 2:
        return at_min[0], zmin, at_min[1]
    rest = [(z, i) for z, i in frags if z != zmin]
    if not rest:
        return at_min[0], zmin, -1
    znext = min(z for z, _ in rest)
    return at_min[0], zmin, min(i for z, i in rest if z == znext)


def composite_order(frags):
    """Fragments front to back: depth levels ascending, ids ascending within
    a level."""
    out = []
    for z in sorted({z for z, _ in frags}):
        out += [(z, i) for i in sorted(i for zz, i in frags if zz == z)]
    return out


def check_scene(orc, verts, rgba8, meta, W, H):
    fr = orc.raster(verts, pixel_vp(W, H), W, H)
    r = orc.resolve(fr, rgba8, BG)
    cov = covering(meta, W, H)
    c64 = rgba8.astype(np.int64)
    ties1 = ties2 = tail_ties = 0
    for p in range(W * H):
        frags = cov[p]
        a, b = fr.offsets[p], fr.offsets[p + 1]
        # the rasteriser produced exactly the covering set
        assert sorted(zip(fr.z[a:b].tolist(), fr.prim[a:b].tolist())) == sorted(frags)
        id1, z1, id2 = expected_layers(frags)
        assert (r["id1"][p], r["id2"][p]) == (id1, id2), p
        assert r["z1"][p] == np.float32(z1)
        assert r["n"][p] == len(frags)
        tail = [i for _, i in frags if i not in (id1, id2)]
        a8 = [int(c64[i] >> 24) for i in tail]
        assert r["a_tail"][p] == sum(a8)
        for k in range(3):
            assert r["s_tail"][p, k] == sum(int((c64[i] >> (8 * k)) & 255) * int(c64[i] >> 24) for i in tail)
        assert r["t_tail"][p] == pytest.approx(np.prod([1.0 - v / 255.0 for v in a8]), rel=1e-13, abs=0)
        # the A-buffer composites in the same order
        C, T = np.zeros(3), 1.0
        for _, i in composite_order(frags):
            al = int(c64[i] >> 24) / 255.0
            C += T * al * np.array([int((c64[i] >> (8 * k)) & 255) for k in range(3)]) / 255.0
            T *= 1.0 - al
        assert np.allclose(r["abuf"][p], C + T * np.array(BG), rtol=0, atol=1e-13)
        zs = [z for z, _ in frags]
        if len(frags) >= 2:
            ties1 += zs.count(z1) >= 2
            ties2 += zs.count(z1) == 1 and len(frags) >= 3 and sorted(zs)[1] == sorted(zs)[2]
            tail_ties += len(frags) >= 4 and len(set(sorted(zs)[2:])) < len(zs) - 2
    return ties1, ties2, tail_ties


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_ties_follow_primitive_id(orc, seed):
    W, H = 32, 16
    rng = np.random.default_rng(100 + seed)
    verts, rgba8, meta = tied_rect_scene(rng, W, H, 14)
    t1, t2, tt = check_scene(orc, verts, rgba8, meta, W, H)
    # the scenes exercise ties at the nearest layer, at the second layer and
    # inside the tail
    assert t1 > 50 and t2 > 5 and tt > 5, (t1, t2, tt)


def test_ties_under_every_submission_order(orc):
    """The same rectangles submitted in several orders: each order's layers
    follow the rule for its own ids."""
    W, H = 16, 16
    for perm_seed in range(6):
        rng = np.random.default_rng(7)          # same rectangles and colours ...
        verts, rgba8, meta = tied_rect_scene(rng, W, H, 10)
        order = np.random.default_rng(1000 + perm_seed).permutation(len(rgba8))
        new_pos = np.empty_like(order)
        new_pos[order] = np.arange(len(order))  # ... submitted in another order
        m2 = [(x0, y0, x1, y1, z, int(new_pos[a]), int(new_pos[b])) for (x0, y0, x1, y1, z, a, b) in meta]
        check_scene(orc, np.ascontiguousarray(verts[order]), np.ascontiguousarray(rgba8[order]), m2, W, H)


def test_all_fragments_at_one_depth(orc):
    """Full-screen quads all at one depth, submitted out of id order: layer 1
    and layer 2 are the two lowest ids, everything else is tail."""
    W, H = 16, 16
    cols = [rgba(10 * k, 255 - 10 * k, 7 * k, 40 + 9 * k) for k in range(10)]
    order = [7, 3, 9, 0, 5, 1, 8, 2, 6, 4]      # quad order of submission
    v, c = [], []
    for q in order:
        for t in quad(0, 0, W, H, 0.5):
            v.append(t)
            c.append(cols[q])
    v, c = np.stack(v), np.array(c, np.uint32)
    fr = orc.raster(v, pixel_vp(W, H), W, H)
    r = orc.resolve(fr, c, BG)
    # every pixel is covered by one triangle of each quad; the two quads
    # submitted first (positions 0 and 1) hold ids 0..3
    assert np.all(r["n"] == 10)
    assert np.all(r["id1"] < 2) and np.all((r["id2"] >= 2) & (r["id2"] < 4))
    a8 = np.array([int(x) >> 24 for x in c], np.int64)
    for p in range(W * H):
        ids = fr.prim[fr.offsets[p]:fr.offsets[p + 1]]
        assert r["id1"][p] == ids.min() and r["id2"][p] == np.sort(ids)[1]
        assert r["a_tail"][p] == a8[ids].sum() - a8[r["id1"][p]] - a8[r["id2"][p]]


def test_tie_depth_levels_are_exact():
    """The tie scenes rely on depths that float32 holds exactly, and on
    0.5 + 2^-16 minus the 2^-16 depth margin being exactly 0.5."""
    for z in TIE_DEPTHS:
        assert float(np.float32(z)) == z
    assert np.float32(TIE_DEPTHS[1]) - np.float32(2.0 ** -16) == np.float32(0.5)
