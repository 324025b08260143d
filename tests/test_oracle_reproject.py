"""Pins of the oracle's depth-based reprojection (Sec. 3.3, last paragraph):
identity camera, a pure screen-space translation and an orbit step checked
against hand-derived geometry."""
import math

import numpy as np
import pytest

from paper_2606_16747_b300 import scenes


def test_inverse4(orc):
    rng = np.random.default_rng(0)
    a = rng.normal(size=(4, 4))
    assert np.allclose(orc.inverse4(a) @ a, np.eye(4), atol=1e-12)
    with pytest.raises(ValueError):
        orc.inverse4(np.zeros((4, 4)))


def test_identity_camera_returns_previous_frame(orc):
    W, H = 40, 24
    rng = np.random.default_rng(1)
    prev = rng.random((W * H, 4)).astype(np.float32)
    z1 = rng.uniform(0.2, 1.0, W * H).astype(np.float32)
    vp = scenes.camera(W, H, 0.0).vp64
    out = orc.reproject(prev, z1, vp, vp, W, H)
    assert np.max(np.abs(out - prev)) < 1e-9


@pytest.mark.parametrize("k,m", [(3, 0), (-2, 5), (7, -4)])
def test_screen_translation_shifts_by_whole_pixels(orc, k, m):
    """VP_prev = S VP_cur with S translating NDC by (2k/W, -2m/H): pixel
    (x, y) samples the previous frame at (x + k, y + m), clamped to the edge."""
    W, H = 32, 20
    rng = np.random.default_rng(2)
    prev = rng.random((W * H, 4)).astype(np.float32)
    z1 = rng.uniform(0.3, 0.9, W * H).astype(np.float32)
    cur = scenes.camera(W, H, 0.0).vp64
    S = np.eye(4)
    S[0, 3] = 2.0 * k / W
    S[1, 3] = -2.0 * m / H
    out = orc.reproject(prev, z1, S @ cur, cur, W, H).reshape(H, W, 4)
    P = prev.reshape(H, W, 4)
    for y in range(H):
        for x in range(W):
            xs, ys = min(max(x + k, 0), W - 1), min(max(y + m, 0), H - 1)
            assert np.max(np.abs(out[y, x] - P[ys, xs])) < 1e-9


def test_orbit_step_matches_geometry(orc):
    """The previous frame is a horizontal ramp r = px / W so the sampled value
    reveals the sampled column.  A pixel at NDC depth d is unprojected by hand
    (perspective with vertical FOV 60, near 0.5, far 20), rotated about the
    orbit centre and projected again; the ramp value must match."""
    W, H = 64, 48
    theta = 2.0
    cur = scenes.camera(W, H, theta).vp64     # current camera: orbit angle theta
    prv = scenes.camera(W, H, 0.0).vp64       # previous camera: identity view
    xs = np.arange(W, dtype=np.float64)
    prev = np.zeros((H, W, 4), np.float32)
    prev[..., 0] = (xs / W)[None, :]
    prev = prev.reshape(-1, 4)
    d = np.float32(0.97)
    z1 = np.full(W * H, d, np.float32)
    out = orc.reproject(prev, z1, prv, cur, W, H).reshape(H, W, 4)
    n, f = scenes.NEAR, scenes.FAR
    th = math.tan(math.radians(30.0))
    asp = W / H
    # NDC depth d = (f/(n-f) (-D) + n f/(n-f)) / D  ->  view distance D
    D = (n * f / (n - f)) / (float(d) + f / (n - f))
    c = np.array(scenes.ORBIT_CENTRE)
    t = math.radians(theta)
    for y in (5, 20, 40):
        for x in (10, 31, 50):
            nx, ny = (2 * x + 1) / W - 1, 1 - (2 * y + 1) / H
            pv = np.array([nx * D * th * asp, ny * D * th, -D])     # point in current view space
            # current view = world rotated by -theta about the centre: undo it
            q = pv - c
            world = c + np.array([math.cos(t) * q[0] + math.sin(t) * q[2], q[1],
                                  -math.sin(t) * q[0] + math.cos(t) * q[2]])
            u = world[0] / (-world[2] * th * asp)                   # previous NDC x
            px = (u + 1) * 0.5 * W - 0.5
            assert 1 <= px <= W - 2
            assert out[y, x, 0] == pytest.approx(px / W, abs=1e-9)
