"""Pins of the oracle's per-pixel resolve: the A-buffer (Eq. 1), the two
nearest layers, the tail statistics of Sec. 3.3 and the decomposition of
Eq. 4, against closed forms, brute force and an independent back-to-front
evaluation."""
import numpy as np
import pytest

from tests.helpers import pixel_vp, quad, random_dyadic_scene, rgba

W, H = 16, 16
BG = (0.25, 0.5, 1.0)


def _scene(layers):
    """layers: list of (depth, rgba8); each a full-screen quad."""
    v, c = [], []
    for z, col in layers:
        for t in quad(0, 0, W, H, z):
            v.append(t)
            c.append(col)
    return np.stack(v) if v else np.zeros((0, 3, 4), np.float32), np.array(c, dtype=np.uint32)


def _run(orc, layers, bg=BG):
    v, c = _scene(layers)
    fr = orc.raster(v, pixel_vp(W, H), W, H)
    return orc.resolve(fr, c, bg), c


def test_empty_pixel_is_background(orc):
    r, _ = _run(orc, [])
    assert np.all(r["abuf"] == np.array(BG))
    assert np.all(r["n"] == 0) and np.all(r["id1"] == -1) and np.all(r["id2"] == -1)
    assert np.all(r["z1"] == 1.0) and np.all(r["t_all"] == 1.0)


def test_single_fragment_closed_form(orc):
    col = rgba(200, 100, 50, 77)
    r, _ = _run(orc, [(0.3, col)])
    a = 77 / 255
    exp = np.array([200, 100, 50]) / 255 * a + (1 - a) * np.array(BG)
    assert np.allclose(r["abuf"], exp, rtol=0, atol=1e-15)
    assert np.all(r["n"] == 1) and np.all(r["id2"] == -1)


def test_two_fragments_textbook_over(orc):
    c1, c2 = rgba(10, 20, 30, 100), rgba(250, 128, 3, 200)
    r, _ = _run(orc, [(0.7, c2), (0.2, c1)])   # submitted back first
    a1, a2 = 100 / 255, 200 / 255
    C1, C2 = np.array([10, 20, 30]) / 255, np.array([250, 128, 3]) / 255
    exp = a1 * C1 + (1 - a1) * (a2 * C2 + (1 - a2) * np.array(BG))
    assert np.allclose(r["abuf"], exp, rtol=0, atol=1e-15)


def test_opaque_front_occludes_everything(orc):
    front = rgba(17, 34, 51, 255)
    layers = [(0.9, rgba(255, 0, 0, 128)), (0.05, front), (0.5, rgba(0, 255, 0, 30)),
              (0.6, rgba(0, 0, 255, 250))]
    r, _ = _run(orc, layers)
    assert np.all(r["abuf"] == np.array([17, 34, 51]) / 255)
    assert np.all(r["t_all"] == 0.0)


def _back_to_front(orc, verts, rgba8, bg):
    """Independent evaluation: gather each pixel's fragments, sort them with
    Python's sort and composite from the back with C <- a c + (1 - a) C."""
    fr = orc.raster(verts, pixel_vp(W, H), W, H)
    out = np.zeros((W * H, 3))
    for p in range(W * H):
        a, b = fr.offsets[p], fr.offsets[p + 1]
        frags = sorted(zip(fr.z[a:b].tolist(), fr.prim[a:b].tolist()))
        C = np.array(bg, dtype=np.float64)
        for z, pr in reversed(frags):
            col = int(rgba8[pr])
            al = (col >> 24) / 255
            c = np.array([(col >> (8 * k)) & 255 for k in range(3)]) / 255
            C = al * c + (1 - al) * C
        out[p] = C
    return fr, out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_abuffer_equals_back_to_front(orc, seed):
    rng = np.random.default_rng(seed)
    v, c = random_dyadic_scene(rng, 24, W, H)
    fr, exp = _back_to_front(orc, v, c, BG)
    r = orc.resolve(fr, c, BG)
    assert np.allclose(r["abuf"], exp, rtol=0, atol=1e-12)
    assert fr.counts.max() >= 4


@pytest.mark.parametrize("seed", [0, 1])
def test_layers_and_tail_sums_brute_force(orc, seed):
    rng = np.random.default_rng(seed)
    v, c = random_dyadic_scene(rng, 24, W, H)
    fr = orc.raster(v, pixel_vp(W, H), W, H)
    r = orc.resolve(fr, c, BG)
    for p in range(W * H):
        a, b = fr.offsets[p], fr.offsets[p + 1]
        frags = sorted(zip(fr.z[a:b].tolist(), fr.prim[a:b].tolist()))
        ids = [pr for _, pr in frags]
        assert r["n"][p] == len(ids)
        assert r["id1"][p] == (ids[0] if ids else -1)
        assert r["id2"][p] == (ids[1] if len(ids) > 1 else -1)
        tail = ids[2:]
        a8 = [int(c[i]) >> 24 for i in tail]
        assert r["a_tail"][p] == sum(a8)
        for k in range(3):
            assert r["s_tail"][p, k] == sum(((int(c[i]) >> (8 * k)) & 255) * (int(c[i]) >> 24) for i in tail)
        assert r["t_tail"][p] == pytest.approx(np.prod([1 - x / 255 for x in a8]), rel=1e-13, abs=0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_eq4_with_exact_tail_equals_abuffer(orc, seed):
    """Eq. 4 with f(x) replaced by the exact tail colour reproduces the A-buffer:
    C_exact,2 + T_2 C_tail + prod(1 - a_i) C_b."""
    rng = np.random.default_rng(seed)
    v, c = random_dyadic_scene(rng, 30, W, H)
    fr = orc.raster(v, pixel_vp(W, H), W, H)
    r = orc.resolve(fr, c, BG)
    rec = r["front2"][:, :3] + r["front2"][:, 3:4] * r["tail_rgb"] + r["t_all"][:, None] * np.array(BG)
    assert np.max(np.abs(rec - r["abuf"])) <= 1e-12
    # the background transmittance factors through the two layers and the tail
    assert np.allclose(r["front2"][:, 3] * r["t_tail"], r["t_all"], rtol=1e-13, atol=0)


def test_integer_identity_of_tail_sums(orc):
    """sum over all fragments of a8 c8 = layer-1 term + layer-2 term + S."""
    rng = np.random.default_rng(5)
    v, c = random_dyadic_scene(rng, 30, W, H)
    fr = orc.raster(v, pixel_vp(W, H), W, H)
    r = orc.resolve(fr, c, BG)
    cc = c.astype(np.int64)
    for p in range(W * H):
        a, b = fr.offsets[p], fr.offsets[p + 1]
        allsum = [sum(((cc[i] >> (8 * k)) & 255) * (cc[i] >> 24) for i in fr.prim[a:b]) for k in range(3)]
        for k in range(3):
            part = r["s_tail"][p, k]
            for idx in (r["id1"][p], r["id2"][p]):
                if idx >= 0:
                    part += ((cc[idx] >> (8 * k)) & 255) * (cc[idx] >> 24)
            assert part == allsum[k]


def test_resolve_permutation_invariant_bitwise(orc):
    rng = np.random.default_rng(11)
    v, c = random_dyadic_scene(rng, 30, W, H, zgrid=1 << 20)
    perm = rng.permutation(30)
    ra = orc.resolve(orc.raster(v, pixel_vp(W, H), W, H), c, BG)
    rb = orc.resolve(orc.raster(v[perm], pixel_vp(W, H), W, H), c[perm], BG)
    for k in ("abuf", "n", "a_tail", "s_tail", "t_tail", "tail_rgb", "front2", "t_all", "z1"):
        assert np.array_equal(ra[k], rb[k]), k
    inv = np.argsort(perm)
    assert np.array_equal(np.where(rb["id1"] >= 0, perm[rb["id1"]], -1), ra["id1"])


def test_unsorted_over_differs_and_matches_in_order(orc):
    """The naive renderer equals the A-buffer when submission is already
    front-to-back and differs otherwise."""
    layers = [(0.1, rgba(255, 0, 0, 128)), (0.5, rgba(0, 255, 0, 128)), (0.9, rgba(0, 0, 255, 128))]
    v, c = _scene(layers)
    fr = orc.raster(v, pixel_vp(W, H), W, H)
    r = orc.resolve(fr, c, BG)
    assert np.allclose(orc.unsorted_over(fr, c, BG), r["abuf"], atol=1e-15)
    v2, c2 = _scene(layers[::-1])
    fr2 = orc.raster(v2, pixel_vp(W, H), W, H)
    assert np.max(np.abs(orc.unsorted_over(fr2, c2, BG) - r["abuf"])) > 0.05


# ---------------------------------------------------------------------------
# Bilinear upscale (Sec. 3.2)

def test_upscale_identity_and_constant(orc):
    rng = np.random.default_rng(0)
    src = rng.random((12 * 10, 3))
    assert np.array_equal(orc.upscale(src, 12, 10, 12, 10), src)
    const = np.full((5 * 4, 2), 0.375)
    assert np.allclose(orc.upscale(const, 5, 4, 23, 17), 0.375, rtol=0, atol=1e-15)


def test_upscale_reproduces_affine_fields(orc):
    """Bilinear interpolation is exact on affine functions away from the
    clamped border; the sample coordinate is u = (x + 0.5) Wp / W - 0.5."""
    Wp, Hp, Wo, Ho = 7, 5, 29, 19
    jj, ii = np.mgrid[0:Hp, 0:Wp]
    src = (3.0 * ii + 5.0 * jj + 1.0).reshape(-1)
    out = orc.upscale(src, Wp, Hp, Wo, Ho).reshape(Ho, Wo)
    for y in range(Ho):
        v = (y + 0.5) * Hp / Ho - 0.5
        for x in range(Wo):
            u = (x + 0.5) * Wp / Wo - 0.5
            if 0 <= u <= Wp - 1 and 0 <= v <= Hp - 1:
                assert out[y, x] == pytest.approx(3 * u + 5 * v + 1, abs=1e-12)
            else:
                uc, vc = min(max(u, 0), Wp - 1), min(max(v, 0), Hp - 1)
                assert out[y, x] == pytest.approx(3 * uc + 5 * vc + 1, abs=1e-12)


def test_tail_flag_exact_threshold(orc):
    """The tail-present flag is the exact predicate 'upscaled N > 2'."""
    from fractions import Fraction
    rng = np.random.default_rng(3)
    Wp, Hp, Wo, Ho = 5, 4, 13, 11
    n = rng.integers(0, 5, size=Wp * Hp).astype(np.uint32)
    flag = orc.tail_flag(n, Wp, Hp, Wo, Ho)
    N = n.reshape(Hp, Wp)
    for y in range(Ho):
        v = Fraction(2 * y + 1, 2) * Fraction(Hp, Ho) - Fraction(1, 2)
        for x in range(Wo):
            u = Fraction(2 * x + 1, 2) * Fraction(Wp, Wo) - Fraction(1, 2)
            i0, j0 = int(np.floor(u)), int(np.floor(v))
            fx, fy = u - i0, v - j0
            cl = lambda a, m: min(max(a, 0), m - 1)
            val = ((1 - fy) * ((1 - fx) * int(N[cl(j0, Hp), cl(i0, Wp)]) + fx * int(N[cl(j0, Hp), cl(i0 + 1, Wp)]))
                   + fy * ((1 - fx) * int(N[cl(j0 + 1, Hp), cl(i0, Wp)]) + fx * int(N[cl(j0 + 1, Hp), cl(i0 + 1, Wp)])))
            assert flag[y * Wo + x] == (val > 2)


# ---------------------------------------------------------------------------
# Network input and front terms (Sec. 3.3)

def test_features_hand_example(orc):
    col1 = rgba(255, 0, 0, 51)      # alpha 0.2
    rgba8 = np.array([col1], dtype=np.uint32)
    layer2 = np.array([[0.1, 0.2, 0.3, 0.5]])
    x, front = orc.features(np.array([0]), rgba8, layer2, np.array([5.0]), np.array([20.0]),
                            np.array([[2550.0, 0.0, 1275.0]]), np.array([0.5]), (1.0, 1.0, 1.0))
    assert x[0].tolist() == pytest.approx([5 / 64, 0.5, 0.5, 0.0, 0.25], abs=1e-15)
    T2 = 0.8 * 0.5
    exp = [0.2 * 1 + 0.8 * 0.1 + T2 * 0.5, 0.8 * 0.2 + T2 * 0.5, 0.8 * 0.3 + T2 * 0.5, T2]
    assert front[0].tolist() == pytest.approx(exp, abs=1e-15)


def test_features_empty_tail_has_zero_colour(orc):
    x, _ = orc.features(np.array([-1]), np.zeros(1, np.uint32), np.zeros((1, 4)), np.array([2.0]),
                        np.array([0.0]), np.zeros((1, 3)), np.array([1.0]))
    assert x[0].tolist() == [2 / 64, 1.0, 0.0, 0.0, 0.0]


def test_composite_and_quantize(orc):
    front = np.array([[0.1, 0.2, 0.3, 0.5], [0.0, 0.0, 0.0, 1.0]])
    f = np.array([[0.2, 0.4, 0.6], [1.5 / 255, 2.5 / 255, 2.0]])
    out = orc.composite(front, f)
    assert out[0].tolist() == pytest.approx([0.2, 0.4, 0.6], abs=1e-15)
    q = orc.quantize(out)
    # round half to even: 1.5 -> 2, 2.5 -> 2, values above 1 clamp to 255
    assert [(int(q[1]) >> (8 * k)) & 255 for k in range(4)] == [2, 2, 255, 255]
    assert [(int(q[0]) >> (8 * k)) & 255 for k in range(3)] == [51, 102, 153]
