"""Input builders shared by the tests (no method arithmetic here)."""
from __future__ import annotations

import numpy as np


def pixel_vp(W: int, H: int) -> np.ndarray:
    """float32 view-projection that maps world (x, y, z, 1), x and y in pixels,
    z in [0, 1], to screen position (x, y) and NDC depth z.  With W and H powers
    of two and dyadic coordinates every float32 operation of the transform is
    exact, so tests can place vertices on the 1/256-pixel grid exactly."""
    m = np.array([[2.0 / W, 0, 0, -1.0],
                  [0, -2.0 / H, 0, 1.0],
                  [0, 0, 1.0, 0],
                  [0, 0, 0, 1.0]], dtype=np.float64)
    return m.astype(np.float32).reshape(16)


def tri(p0, p1, p2, z=(0.5, 0.5, 0.5)):
    return np.array([[p0[0], p0[1], z[0], 1.0], [p1[0], p1[1], z[1], 1.0],
                     [p2[0], p2[1], z[2], 1.0]], dtype=np.float32)


def rgba(r, g, b, a):
    return np.uint32(r | (g << 8) | (b << 16) | (a << 24))


def quad(x0, y0, x1, y1, z):
    """Two triangles covering [x0, x1] x [y0, y1] at constant depth z."""
    return [tri((x0, y0), (x1, y0), (x1, y1), (z, z, z)), tri((x0, y0), (x1, y1), (x0, y1), (z, z, z))]


def random_dyadic_scene(rng, n, W, H, grid=4, margin=2.0, zgrid=1024):
    """n random triangles with vertices on a 1/grid pixel lattice and depths on
    a 1/zgrid lattice in [0, 1] (exactly representable in float32)."""
    xs = rng.integers(int(-margin * grid), int((W + margin) * grid) + 1, size=(n, 3)) / grid
    ys = rng.integers(int(-margin * grid), int((H + margin) * grid) + 1, size=(n, 3)) / grid
    zs = rng.integers(0, zgrid + 1, size=(n, 3)) / zgrid
    v = np.stack([xs, ys, zs, np.ones_like(xs)], axis=-1).astype(np.float32)
    cols = rng.integers(0, 256, size=(n, 4)).astype(np.uint32)
    cols[:, 3] = rng.integers(1, 256, size=n)
    rgba8 = (cols[:, 0] | (cols[:, 1] << 8) | (cols[:, 2] << 16) | (cols[:, 3] << 24)).astype(np.uint32)
    return v, rgba8


def watertight_mesh(rng, W, H, gx, gy, jitter_grid=4, shuffle=True):
    """A grid mesh over [-2, W+2] x [-2, H+2]: interior vertices jittered on a
    1/jitter_grid lattice, each cell cut along a random diagonal, vertex order
    and triangle order randomised.  Every pixel centre lies in exactly one
    triangle's closure; ties on shared edges and vertices are frequent."""
    xs = np.linspace(-2, W + 2, gx + 1)
    ys = np.linspace(-2, H + 2, gy + 1)
    P = np.zeros((gy + 1, gx + 1, 2))
    for j in range(gy + 1):
        for i in range(gx + 1):
            x, y = xs[i], ys[j]
            if 0 < i < gx and 0 < j < gy:
                x += rng.integers(-jitter_grid, jitter_grid + 1) / jitter_grid * 0.75
                y += rng.integers(-jitter_grid, jitter_grid + 1) / jitter_grid * 0.75
            P[j, i] = (np.round(x * jitter_grid) / jitter_grid, np.round(y * jitter_grid) / jitter_grid)
    tris = []
    for j in range(gy):
        for i in range(gx):
            a, b, c, d = P[j, i], P[j, i + 1], P[j + 1, i + 1], P[j + 1, i]
            pair = [(a, b, c), (a, c, d)] if rng.random() < 0.5 else [(a, b, d), (b, c, d)]
            for t in pair:
                t = list(t)
                if rng.random() < 0.5:
                    t = [t[0], t[2], t[1]]
                tris.append(tri(t[0], t[1], t[2], tuple(rng.integers(0, 1025, 3) / 1024)))
    tris = np.stack(tris)
    if shuffle:
        tris = tris[rng.permutation(len(tris))]
    return np.ascontiguousarray(tris)


# depth levels of the tie scenes: exact in float32, and 0.5 + 2^-16 sits exactly
# one depth margin (2^-16) behind 0.5, the edge case of a triangle whose depth
# lower bound equals another fragment's depth
TIE_DEPTHS = (0.5, 0.5 + 2.0 ** -16, 0.5 + 2.0 ** -15, 0.75)


def tied_rect_scene(rng, W, H, n_rects, depths=TIE_DEPTHS, alpha=(20, 235)):
    """Axis-aligned rectangles at a few shared depths, each split along its
    main diagonal into two triangles, the triangles submitted in a random
    order (primitive id = position in the returned arrays).  Rectangle corners
    are whole pixels, widths odd and heights even, so no pixel centre lies on
    a rectangle's border or on its diagonal: each centre inside a rectangle is
    covered by exactly one of its two triangles, whatever the tie rule.

    Returns verts [2n][3][4], rgba8 [2n], and per rectangle (x0, y0, x1, y1, z,
    id_a, id_b), where id_a is the triangle (x0,y0) (x1,y0) (x1,y1) and id_b the
    triangle (x0,y0) (x1,y1) (x0,y1)."""
    rects, tris, cols = [], [], []
    for _ in range(n_rects):
        w = 2 * int(rng.integers(1, max(2, W // 2))) + 1
        h = 2 * int(rng.integers(1, max(2, H // 2)))
        x0 = int(rng.integers(-w // 2, W - w // 2))
        y0 = int(rng.integers(-h // 2, H - h // 2))
        z = float(depths[int(rng.integers(0, len(depths)))])
        rects.append((x0, y0, x0 + w, y0 + h, z))
        for _t in range(2):
            cols.append(rgba(*[int(v) for v in rng.integers(0, 256, 3)], int(rng.integers(alpha[0], alpha[1] + 1))))
    for (x0, y0, x1, y1, z) in rects:
        tris += [tri((x0, y0), (x1, y0), (x1, y1), (z, z, z)), tri((x0, y0), (x1, y1), (x0, y1), (z, z, z))]
    perm = rng.permutation(len(tris))          # new position of each triangle
    verts = np.zeros((len(tris), 3, 4), np.float32)
    rgba8 = np.zeros(len(tris), np.uint32)
    for k, pos in enumerate(perm):
        verts[pos] = tris[k]
        rgba8[pos] = cols[k]
    meta = [(x0, y0, x1, y1, z, int(perm[2 * i]), int(perm[2 * i + 1]))
            for i, (x0, y0, x1, y1, z) in enumerate(rects)]
    return verts, rgba8, meta
