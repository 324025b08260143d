"""Pins of the oracle's DFAOIT comparison network (Sec. 3.3): its eleven
listed features (the exact blend of the two front fragments, the tail's
average colour and opacity, the tail's accumulated premultiplied colour, the
fragment count) on hand-built scenes, the network with a sigmoid output on
weights whose result is known in closed form, its gradient by finite
differences, and the composite C = C_t + C_b prod(1 - a_i) against the
exact A-buffer when the network is replaced by the exact C_t."""
import numpy as np
import pytest

from tests.helpers import pixel_vp, quad, random_dyadic_scene, rgba

W, H = 16, 16
KAPPA = 1.0 / 64.0


def _scene(layers):
    v, c = [], []
    for z, col in layers:
        for t in quad(0, 0, W, H, z):
            v.append(t)
            c.append(col)
    return np.stack(v), np.array(c, dtype=np.uint32)


def _features(orc, layers):
    v, c = _scene(layers)
    fr = orc.raster(v, pixel_vp(W, H), W, H)
    return orc.dfaoit_features(fr, c), fr


def _rgb(col):
    return np.array([(col >> (8 * k)) & 255 for k in range(3)], np.float64) / 255.0


def _a(col):
    return (col >> 24) / 255.0


def test_no_fragment(orc):
    fr = orc.raster(np.zeros((0, 3, 4), np.float32), pixel_vp(W, H), W, H)
    x, t = orc.dfaoit_features(fr, np.zeros(0, np.uint32))
    assert np.all(x == 0.0) and np.all(t == 1.0)


def test_one_and_two_fragments(orc):
    c1, c2 = int(rgba(200, 100, 50, 77)), int(rgba(10, 250, 128, 200))
    (x, t), _ = _features(orc, [(0.3, c1)])
    assert np.allclose(x[:, 0:3], _a(c1) * _rgb(c1), rtol=0, atol=1e-15)
    assert np.all(x[:, 3:10] == 0.0) and np.all(x[:, 10] == KAPPA)
    assert np.allclose(t, 1.0 - _a(c1), rtol=0, atol=1e-15)
    (x, t), _ = _features(orc, [(0.7, c2), (0.2, c1)])          # submitted back first
    front = _a(c1) * _rgb(c1) + (1.0 - _a(c1)) * _a(c2) * _rgb(c2)
    assert np.allclose(x[:, 0:3], front, rtol=0, atol=1e-15)
    assert np.all(x[:, 3:10] == 0.0) and np.all(x[:, 10] == 2 * KAPPA)


def test_tail_statistics_by_hand(orc):
    """Five stacked quads at distinct depths, submitted out of depth order:
    the two nearest give the front blend, the three others the tail means
    and the premultiplied sum."""
    cols = [int(rgba(255, 0, 0, 60)), int(rgba(0, 255, 0, 120)), int(rgba(0, 0, 255, 180)),
            int(rgba(40, 80, 120, 30)), int(rgba(250, 200, 150, 255))]
    depths = [0.1, 0.3, 0.5, 0.7, 0.9]
    order = [3, 0, 4, 2, 1]
    (x, t), _ = _features(orc, [(depths[i], cols[i]) for i in order])
    front = _a(cols[0]) * _rgb(cols[0]) + (1.0 - _a(cols[0])) * _a(cols[1]) * _rgb(cols[1])
    tail = cols[2:]
    avg_c = sum(_rgb(c) for c in tail) / 3.0
    avg_a = sum(_a(c) for c in tail) / 3.0
    acc = sum(_a(c) * _rgb(c) for c in tail)
    T = np.prod([1.0 - _a(c) for c in cols])
    exp = np.concatenate([front, avg_c, [avg_a], acc, [5 * KAPPA]])
    assert np.allclose(x, exp[None, :], rtol=0, atol=1e-14)
    assert np.allclose(t, T, rtol=0, atol=1e-15) and T == 0.0   # an opaque fragment in the tail


@pytest.mark.parametrize("seed", [0, 1])
def test_features_agree_with_the_layer_terms(orc, seed):
    """On random scenes: the front blend is the resolve's exact two-layer
    composite, the premultiplied tail sum its integer tail sums / 255^2, the
    mean opacity its alpha sum / (255 (n - 2)), and t_all its total
    transmittance."""
    rng = np.random.default_rng(seed)
    v, c = random_dyadic_scene(rng, 30, W, H)
    fr = orc.raster(v, pixel_vp(W, H), W, H)
    x, t = orc.dfaoit_features(fr, c)
    r = orc.resolve(fr, c)
    n = r["n"].astype(np.float64)
    assert np.allclose(x[:, 0:3], r["front2"][:, :3], rtol=0, atol=1e-14)
    assert np.allclose(x[:, 7:10], r["s_tail"] / 255.0 ** 2, rtol=0, atol=1e-12)
    tail = n > 2
    assert np.allclose(x[tail, 6], r["a_tail"][tail] / (255.0 * (n[tail] - 2)), rtol=0, atol=1e-14)
    assert np.all(x[~tail, 3:10] == 0.0)
    assert np.allclose(x[:, 10], n * KAPPA, rtol=0, atol=0)
    assert np.allclose(t, r["t_all"], rtol=0, atol=1e-14)
    assert tail.sum() > 50


def test_exact_transparency_colour_composites_to_the_abuffer(orc):
    """With the network replaced by the exact C_t (the A-buffer minus the
    background term), C_t + t_all C_b is the A-buffer; the front blend plus
    T_2 times the exact tail colour is C_t (the decomposition of Eq. 4)."""
    rng = np.random.default_rng(4)
    v, c = random_dyadic_scene(rng, 30, W, H)
    bg = np.array([0.25, 0.5, 1.0])
    fr = orc.raster(v, pixel_vp(W, H), W, H)
    x, t = orc.dfaoit_features(fr, c)
    r = orc.resolve(fr, c, tuple(bg))
    ct = r["abuf"] - t[:, None] * bg[None, :]
    assert np.allclose(ct, x[:, 0:3] + r["front2"][:, 3:4] * r["tail_rgb"], rtol=0, atol=1e-12)


def _ident_params():
    """w1 copies inputs 0..10 to hidden units 0..10, w2 units 0..10 to units
    0..10, w3 units 0..2 to the outputs, every bias 0: f = sigmoid(relu(x[0..2]))."""
    p = np.zeros(963)
    w1 = np.zeros((32, 11))
    w1[np.arange(11), np.arange(11)] = 1.0
    w2 = np.zeros((16, 32))
    w2[np.arange(11), np.arange(11)] = 1.0
    w3 = np.zeros((3, 16))
    w3[np.arange(3), np.arange(3)] = 1.0
    p[0:352] = w1.ravel()
    p[384:896] = w2.ravel()
    p[912:960] = w3.ravel()
    return p


def test_forward_closed_form(orc):
    rng = np.random.default_rng(2)
    x = rng.uniform(-2.0, 2.0, (200, 11))
    flag = (rng.random(200) < 0.8).astype(np.uint8)
    f = orc.mlp_dfaoit_forward(_ident_params(), x, flag)
    exp = 1.0 / (1.0 + np.exp(-np.maximum(x[:, :3], 0.0)))
    assert np.allclose(f[flag == 1], exp[flag == 1], rtol=0, atol=1e-15)
    assert np.all(f[flag == 0] == 0.0)
    # biases only: sigmoid(b3)
    p = np.zeros(963)
    p[960:963] = [-1.0, 0.0, 2.0]
    f = orc.mlp_dfaoit_forward(p, x[:3], None)
    assert np.allclose(f, 1.0 / (1.0 + np.exp(-np.array([-1.0, 0.0, 2.0])))[None, :], rtol=0, atol=1e-15)


def test_gradient_by_finite_differences(orc):
    rng = np.random.default_rng(5)
    p = rng.normal(0.0, 0.4, 963)
    x = rng.uniform(0.0, 1.0, (64, 11))
    y = rng.uniform(0.0, 1.0, (64, 3))
    loss, g = orc.mlp_dfaoit_mse_grad(p, x, y)
    f = orc.mlp_dfaoit_forward(p, x)
    assert loss == pytest.approx(np.mean((f - y) ** 2), rel=1e-13)
    h = 1e-6
    for i in rng.choice(963, 60, replace=False):
        q = p.copy()
        q[i] += h
        lp, _ = orc.mlp_dfaoit_mse_grad(q, x, y)
        q[i] -= 2 * h
        lm, _ = orc.mlp_dfaoit_mse_grad(q, x, y)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), i
