"""GPU parity on scenes with large triangles (Sec. 3, Sec. 3.3).  A triangle
whose doubled area in 1/256-pixel units does not fit int32 (more than
16,384 square pixels) takes its fragment depths from the int64 edge
functions, the others from the 32-bit tile-relative values; the scene mixes
both kinds, with depth planes that vary across each triangle, so that the
layer ids, depths, counts and tail sums of the two-pixel traversal are
checked bit for bit against the oracle on both paths, in the persistent pass
launch under every two-pixel tile shape and in the pass launch that also
produces the frame."""
import numpy as np
import pytest
import torch

from paper_2606_16747_b300 import scenes
from tests.helpers import pixel_vp, tri
from tests.test_gpu_parity import TOL_BF16
from tests.test_gpu_ties import Passes, check_planes

pytestmark = pytest.mark.gpu

W, H = 600, 400          # ragged: 37.5 x 25 tiles of 16 pixels


@pytest.fixture(scope="module")
def sn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_16747_b300 import build, star_nt
    build.build()
    return star_nt


def large_tri_scene(seed, n_large=14, n_small=80):
    """Seeded triangles: n_large spanning most of the frame (areas of
    20,000-150,000 square pixels), n_small of 4-40 pixels; per-vertex depths
    in [0.05, 0.95] on a 1/1024 grid, straight RGBA8 with alpha 20-235."""
    rng = np.random.default_rng(900 + seed)
    tris, areas = [], []

    def add(p, z):
        tris.append(tri(p[0], p[1], p[2], z))
        (x0, y0), (x1, y1), (x2, y2) = p
        areas.append(abs((x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0)) / 2)

    while len(tris) < n_large:
        p = [(float(rng.integers(-60, W + 60)) + rng.integers(0, 256) / 256.0,
              float(rng.integers(-60, H + 60)) + rng.integers(0, 256) / 256.0) for _ in range(3)]
        (x0, y0), (x1, y1), (x2, y2) = p
        a = abs((x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0)) / 2
        if 20000 <= a <= 150000:
            add(p, rng.integers(51, 973, 3) / 1024.0)
    for _ in range(n_small):
        cx, cy = rng.uniform(0, W), rng.uniform(0, H)
        s = rng.uniform(4, 40)
        p = [(cx + s * np.cos(t), cy + s * np.sin(t)) for t in rng.uniform(0, 2 * np.pi, 3)]
        p = [(np.round(x * 256) / 256, np.round(y * 256) / 256) for x, y in p]
        add(p, rng.integers(51, 973, 3) / 1024.0)
    order = rng.permutation(len(tris))
    verts = np.stack([tris[i] for i in order]).astype(np.float32)
    c = rng.integers(0, 256, (len(tris), 3))
    a = rng.integers(20, 236, len(tris))
    rgba8 = (c[:, 0] | (c[:, 1] << 8) | (c[:, 2] << 16) | (a << 24)).astype(np.uint32)
    return verts, rgba8, pixel_vp(W, H), np.asarray(areas)[order]


_ORACLE = {}


def oracle_layers(orc, seed):
    if seed not in _ORACLE:
        verts, rgba8, vp, areas = large_tri_scene(seed)
        fr = orc.raster(verts, vp, W, H, threads=4)
        o = orc.resolve(fr, rgba8, threads=4)
        # both depth paths occur among the nearest two layers
        big = np.flatnonzero(areas > 16384)
        small = np.flatnonzero(areas < 16384)
        for ids in (o["id1"], o["id2"]):
            assert np.isin(ids, big).sum() > W * H // 10
            assert np.isin(ids, small).sum() > 500
        _ORACLE[seed] = (verts, rgba8, vp, o)
    return _ORACLE[seed]


@pytest.mark.parametrize("tuning", [None, (4, 0, 2), (8, 10, 2), (16, 0, 2)])
@pytest.mark.parametrize("merge", [False, True])
@pytest.mark.parametrize("seed", [0, 1])
def test_large_triangles_persistent_passes(orc, sn, tuning, merge, seed):
    verts, rgba8, vp, o = oracle_layers(orc, seed)
    p = Passes(sn, verts, rgba8, vp, W, H)
    p.raster(merge=merge)
    sn.geometry_passes(p.scene, p.bins[0], p.bins[1], p.bins[2], p.l1, p.l2, p.l3, tuning, p.status)
    check_planes(p.planes(), o)


@pytest.mark.parametrize("seed", [0, 1])
def test_large_triangles_pass_launch_resolve(orc, sn, seed):
    """Every pass at full size: the pass launch that runs the network and the
    composite writes the oracle's nearest layer bit for bit and a frame within
    the BF16 tolerance of the oracle's."""
    from paper_2606_16747_b300.pipeline import Renderer
    verts, rgba8, vp, o = oracle_layers(orc, seed)
    mlp = scenes.mlp_xavier(4)
    r = Renderer(verts, rgba8, W, H, mlp=mlp, x_dtype=sn.BF16, fused=True, persistent=True,
                 tuning=(8, 0, 2), fuse_passes=True)
    r.set_camera(vp)
    r.star_frame(update_tiles=False)
    torch.cuda.synchronize()
    r.check_status()
    assert int(r.bins[1].mem[44:48].view(torch.int32).item()) == 1
    assert np.array_equal(r.l1["id1"].cpu().numpy(), o["id1"])
    assert np.array_equal(r.l1["z1"].cpu().numpy().view(np.uint32), o["z1"].view(np.uint32))
    f = orc.frame_star(verts, rgba8, vp, W, H, (W, H), (W, H), scenes.mlp_flat(mlp), threads=4)
    rgb = r.rgba32f.cpu().numpy().reshape(-1, 4)[:, :3]
    assert np.max(np.abs(rgb - f["rgb"])) <= TOL_BF16
