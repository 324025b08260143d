"""Pins of the oracle's comparison renderers (Sec. 4): the naive unsorted
"over" blend and weighted blended OIT."""
import numpy as np
import pytest

from tests.helpers import pixel_vp, quad


def frags_of(lists, W=1, H=None):
    """CSR fragment lists from per-pixel [(z, prim), ...]."""
    import oracle
    H = H if H is not None else len(lists)
    counts = np.array([len(l) for l in lists], np.uint32)
    offsets = np.zeros(len(lists) + 1, np.int64)
    offsets[1:] = np.cumsum(counts)
    z = np.array([f[0] for l in lists for f in l], np.float32)
    prim = np.array([f[1] for l in lists for f in l], np.int32)
    return oracle.Frags(W, H, counts, offsets, z, prim)


def rgba(r, g, b, a):
    return np.uint32(r | (g << 8) | (b << 16) | (a << 24))


BG = (0.2, 0.5, 1.0)
NEAR, FAR = 0.5, 20.0


def ndc(d):  # view depth -> NDC z in [0, 1]
    return FAR * (d - NEAR) / (d * (FAR - NEAR))


def test_wboit_single_fragment_is_over(orc):
    cols = np.array([rgba(200, 100, 50, 128)], np.uint32)
    fr = frags_of([[(ndc(3.0), 0)]])
    out = orc.wboit(fr, cols, NEAR, FAR, BG)
    a = 128 / 255
    c = np.array([200, 100, 50]) / 255
    assert np.allclose(out[0], a * c + (1 - a) * np.array(BG), atol=1e-12)


def test_wboit_equal_colours_is_over(orc):
    """Fragments of one colour: the weighted average is that colour, and the
    coverage 1 - prod(1 - a) is exact, so WBOIT equals the sorted blend."""
    cols = np.array([rgba(10, 200, 90, 60), rgba(10, 200, 90, 200), rgba(10, 200, 90, 255)], np.uint32)
    fr = frags_of([[(ndc(2.0), 0), (ndc(9.0), 1)], [(ndc(15.0), 2), (ndc(1.0), 0), (ndc(4.0), 1)]])
    out = orc.wboit(fr, cols, NEAR, FAR, BG)
    c = np.array([10, 200, 90]) / 255
    T0 = (1 - 60 / 255) * (1 - 200 / 255)
    assert np.allclose(out[0], c * (1 - T0) + T0 * np.array(BG), atol=1e-12)
    assert np.allclose(out[1], c, atol=1e-12)   # an opaque fragment: T = 0


def test_wboit_weight_regions(orc):
    """Near fragments (d below 0.28, weight capped at 3e3 a) weigh by opacity
    only; a near fragment against a far one (d above 640, weight floored at
    1e-2 a) dominates by the ratio 3e5 of the clamps."""
    red, blue = rgba(255, 0, 0, 100), rgba(0, 0, 255, 50)
    cols = np.array([red, blue], np.uint32)
    # NEAR = 0.5 bounds the view depth from below; use a projection with near 0.1 for the cap
    n, f = 0.1, 1000.0
    z = lambda d: f * (d - n) / (d * (f - n))
    fr = frags_of([[(z(0.2), 0), (z(0.25), 1)], [(z(0.2), 0), (z(900.0), 1)]])
    out = orc.wboit(fr, cols, n, f, (0.0, 0.0, 0.0))
    a0, a1 = 100 / 255, 50 / 255
    cov = 1 - (1 - a0) * (1 - a1)
    # equal weights per unit opacity: colour = sum a^2 c / sum a^2
    r = a0 * a0 / (a0 * a0 + a1 * a1)
    assert np.allclose(out[0], np.array([r, 0, 1 - r]) * cov, atol=1e-12)
    r = a0 * a0 * 3e3 / (a0 * a0 * 3e3 + a1 * a1 * 1e-2)
    assert np.allclose(out[1], np.array([r, 0, 1 - r]) * cov, atol=1e-12)


def test_wboit_order_free(orc):
    rng = np.random.default_rng(5)
    cols = (rng.integers(0, 256, size=(6, 4)) * np.array([1, 256, 65536, 16777216])).sum(1).astype(np.uint32)
    frs = [(float(ndc(rng.uniform(1, 15))), k) for k in range(6)]
    a = orc.wboit(frags_of([frs]), cols, NEAR, FAR, BG)
    b = orc.wboit(frags_of([frs[::-1]]), cols, NEAR, FAR, BG)
    assert np.allclose(a, b, atol=1e-13)


def test_unsorted_over_in_depth_order_is_abuffer(orc):
    """Submission order that happens to be front to back gives the A-buffer;
    the reverse order does not."""
    W, H = 16, 16
    # three overlapping quads, primitive id increasing with depth
    tris = np.concatenate([quad(0, 0, 16, 16, 0.2), quad(2, 2, 14, 14, 0.5), quad(4, 4, 12, 12, 0.8)])
    cols = np.array([rgba(255, 0, 0, 120)] * 2 + [rgba(0, 255, 0, 90)] * 2 + [rgba(0, 0, 255, 200)] * 2,
                    np.uint32)
    fr = orc.raster(tris, pixel_vp(W, H), W, H)
    res = orc.resolve(fr, cols, BG)
    assert np.allclose(orc.unsorted_over(fr, cols, BG), res["abuf"], atol=1e-12)
    rev = tris[::-1].copy()
    fr2 = orc.raster(rev, pixel_vp(W, H), W, H)
    out = orc.unsorted_over(fr2, cols[::-1].copy(), BG)
    centre = 8 * W + 8
    assert not np.allclose(out[centre], res["abuf"][centre], atol=1e-3)
