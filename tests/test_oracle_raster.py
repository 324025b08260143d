"""Pins of the oracle's rasteriser (the geometry passes of Sec. 3) against
exact rational geometry, watertightness and permutation invariance."""
from fractions import Fraction

import numpy as np
import pytest

from tests.helpers import pixel_vp, random_dyadic_scene, tri, watertight_mesh


def _barycentric(v, px, py):
    """Exact barycentric coordinates by Cramer's rule (Fractions)."""
    (x0, y0), (x1, y1), (x2, y2) = [(Fraction(float(a[0])), Fraction(float(a[1]))) for a in v]
    den = (y1 - y2) * (x0 - x2) + (x2 - x1) * (y0 - y2)
    if den == 0:
        return None
    l0 = ((y1 - y2) * (px - x2) + (x2 - x1) * (py - y2)) / den
    l1 = ((y2 - y0) * (px - x2) + (x0 - x2) * (py - y2)) / den
    return l0, l1, 1 - l0 - l1


def _pixel_frags(fr, p):
    a, b = fr.offsets[p], fr.offsets[p + 1]
    return sorted(zip(fr.prim[a:b].tolist(), fr.z[a:b].tolist()))


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_coverage_and_depth_match_exact_geometry(orc, seed):
    """Every pixel centre strictly inside a triangle is covered exactly once by
    it, strictly outside never, and its depth is the exact affine interpolation
    of the vertex depths to float32 accuracy."""
    W, H = 32, 16
    rng = np.random.default_rng(seed)
    verts, _ = random_dyadic_scene(rng, 12, W, H, grid=4)
    fr = orc.raster(verts, pixel_vp(W, H), W, H)
    n_strict = 0
    for t in range(verts.shape[0]):
        v = verts[t, :, :2]
        for y in range(H):
            for x in range(W):
                lam = _barycentric(v, Fraction(2 * x + 1, 2), Fraction(2 * y + 1, 2))
                p = y * W + x
                hits = [z for (pr, z) in _pixel_frags(fr, p) if pr == t]
                if lam is None or min(lam) < 0:
                    assert hits == [], (t, x, y)
                elif min(lam) > 0:
                    n_strict += 1
                    assert len(hits) == 1, (t, x, y)
                    zex = sum(l * Fraction(float(verts[t, k, 2])) for k, l in enumerate(lam))
                    assert abs(hits[0] - float(zex)) <= 4e-7, (t, x, y)
                else:
                    assert len(hits) <= 1
    assert n_strict > 100


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_watertight_shared_edges_and_vertices(orc, seed):
    """A mesh that tiles the screen covers every pixel centre exactly once,
    whatever the triangle orientation: the tie rule owns each shared edge and
    vertex once (pins the fill convention)."""
    W, H = 32, 16
    rng = np.random.default_rng(seed)
    mesh = watertight_mesh(rng, W, H, 9, 5)
    fr = orc.raster(mesh, pixel_vp(W, H), W, H)
    assert fr.counts.min() == 1 and fr.counts.max() == 1


def test_fan_around_pixel_centre(orc):
    """Eight triangles meeting at a pixel centre: that centre, and every centre
    on the spokes, belongs to exactly one of them."""
    W, H = 16, 16
    c = (8.5, 8.5)
    ring = [(2.5, 2.5), (8.5, 0.5), (15.5, 2.5), (15.5, 8.5), (15.5, 15.5), (8.5, 15.5),
            (0.5, 15.5), (0.5, 8.5)]
    tris = np.stack([tri(c, ring[i], ring[(i + 1) % 8]) for i in range(8)])
    fr = orc.raster(tris, pixel_vp(W, H), W, H)
    cnt = fr.counts.reshape(H, W)
    assert cnt[8, 8] == 1
    assert cnt[8, 2:15].tolist() == [1] * 13 and cnt[2:15, 8].tolist() == [1] * 13


def test_large_triangle_area(orc):
    """Pixel count of a large triangle equals its area up to the boundary."""
    W, H = 256, 256
    v = np.stack([tri((10.3, 7.9), (240.1, 31.7), (60.6, 250.2))])
    fr = orc.raster(v, pixel_vp(W, H), W, H)
    x0, y0, x1, y1, x2, y2 = 10.3, 7.9, 240.1, 31.7, 60.6, 250.2
    area = abs((x1 - x0) * (y2 - y0) - (y1 - y0) * (x2 - x0)) / 2
    perim = sum(np.hypot(a - c, b - d) for a, b, c, d in [(x0, y0, x1, y1), (x1, y1, x2, y2), (x2, y2, x0, y0)])
    assert abs(fr.total - area) <= perim


def test_permutation_invariance(orc):
    """The per-pixel fragment multiset does not depend on submission order."""
    W, H = 32, 32
    rng = np.random.default_rng(7)
    verts, _ = random_dyadic_scene(rng, 20, W, H, grid=8)
    perm = rng.permutation(20)
    a = orc.raster(verts, pixel_vp(W, H), W, H)
    b = orc.raster(verts[perm], pixel_vp(W, H), W, H)
    assert np.array_equal(a.counts, b.counts)
    for p in range(W * H):
        fa = _pixel_frags(a, p)
        fb = sorted((int(perm[pr]), z) for pr, z in _pixel_frags(b, p))
        assert fa == fb


def test_drop_rules(orc):
    """Degenerate triangles and triangles with a vertex behind the near plane
    or outside the depth range produce no fragments."""
    W, H = 16, 16
    vp = pixel_vp(W, H)
    good = tri((1, 1), (14, 2), (3, 13))
    degenerate = tri((1, 1), (5, 5), (9, 9))
    far = tri((1, 1), (14, 2), (3, 13), (0.5, 0.5, 1.5))
    near = tri((1, 1), (14, 2), (3, 13), (-0.25, 0.5, 0.5))
    fr = orc.raster(np.stack([degenerate, far, near]), vp, W, H)
    assert fr.total == 0
    fr = orc.raster(np.stack([good]), vp, W, H)
    assert fr.total > 50


def test_perspective_scene_counts_stable(orc):
    """Frustum scene of 32 triangles at 256x256: the mean depth complexity of
    covered pixels matches the workload description (~4)."""
    from paper_2606_16747_b300 import scenes
    sc = scenes.small_scene()
    fr = orc.raster(sc.verts, sc.cam.vp32, sc.width, sc.height)
    c = fr.counts
    assert 3.0 < c[c > 0].mean() < 5.0
