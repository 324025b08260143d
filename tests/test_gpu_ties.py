"""GPU parity on scenes full of exact depth ties (Sec. 3.3: layers ordered by
(depth, primitive id)).  Rectangles at a few shared depths, triangles
submitted in shuffled order, give ties at the nearest layer, at the second
layer and inside the tail, and triangles whose depth lower bound equals a
lane's current layer depth exactly.  Every geometry-pass path must give the
oracle's ids, counts and tail sums bit for bit: the separate pass kernels,
pass 1 with merged passes, the persistent launch under every tile shape, the
plain fused pipeline and the pass launch that also produces the frame."""
import numpy as np
import pytest
import torch

from paper_2606_16747_b300 import scenes
from tests.helpers import pixel_vp, tied_rect_scene
from tests.test_gpu_parity import TOL_BF16, TOL_FEAT, assert_frags_equal, dev, u32

pytestmark = pytest.mark.gpu

SIZES = [(256, 256), (333, 197)]
TUNINGS = [None, (4, 0, 1), (16, 0, 1), (4, 3, 1), (8, 0, 1), (8, 0, 2), (4, 10, 2), (16, 5, 2),
           (8, 7, 2)]


@pytest.fixture(scope="module")
def sn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_16747_b300 import build, star_nt
    build.build()
    return star_nt


def tie_scene(W, H, seed):
    rng = np.random.default_rng(500 + seed)
    verts, rgba8, _ = tied_rect_scene(rng, W, H, 40)
    return verts, rgba8, pixel_vp(W, H)


class Passes:
    """The three pass workspaces and planes of one frame at W x H, driven
    through the C ABI directly (merge per pass chosen by the test)."""

    def __init__(self, sn, verts, rgba8, vp, W, H):
        self.sn, self.W, self.H = sn, W, H
        P = W * H
        self.v, self.c = dev(verts), dev(rgba8.view(np.int32))
        self.scene = sn.scene_struct(self.v, self.c)
        self.vp = dev(np.asarray(vp, np.float32).reshape(16))
        self.size = dev(np.array([W, H], np.int32))
        self.bins = [sn.BinsBuffer(W, H, len(rgba8), 1 << 20) for _ in range(3)]
        i32 = dict(dtype=torch.int32, device="cuda")
        self.l1 = dict(id1=torch.full((P,), -7, **i32), z1=torch.full((P,), -7.0, device="cuda"))
        self.l2 = dict(id2=torch.full((P,), -7, **i32))
        self.l3 = dict(n=torch.full((P,), -7, **i32), tail=torch.full((4 * P,), -7, **i32),
                       t_tail=torch.full((P,), -7.0, device="cuda"))
        self.status = torch.zeros(1, **i32)

    def raster(self, merge):
        m = self.size if merge else None
        self.sn.raster_passes(self.scene, [(self.vp, self.size, self.W, self.H, self.bins[0], None),
                                           (self.vp, self.size, self.W, self.H, self.bins[1], m),
                                           (self.vp, self.size, self.W, self.H, self.bins[2], m)],
                              self.status)

    def planes(self):
        torch.cuda.synchronize()
        assert int(self.status.item()) == 0
        return dict(id1=self.l1["id1"].cpu().numpy(), z1=self.l1["z1"].cpu().numpy().view(np.uint32),
                    id2=self.l2["id2"].cpu().numpy(), n=u32(self.l3["n"]),
                    tail=u32(self.l3["tail"]).reshape(-1, 4), t_tail=self.l3["t_tail"].cpu().numpy())


def check_planes(got, o, layers=(1, 2, 3)):
    if 1 in layers:
        assert np.array_equal(got["id1"], o["id1"])
        assert np.array_equal(got["z1"], o["z1"].view(np.uint32))
    if 2 in layers:
        assert np.array_equal(got["id2"], o["id2"])
    if 3 in layers:
        assert np.array_equal(got["n"], o["n"])
        assert np.array_equal(got["tail"][:, 0], o["a_tail"])
        assert np.array_equal(got["tail"][:, 1:], o["s_tail"])
        rel = np.abs(got["t_tail"] - o["t_tail"]) / np.maximum(o["t_tail"], 1e-30)
        assert rel.max() <= 2e-6


_ORACLE = {}


def oracle_layers(orc, verts, rgba8, vp, W, H):
    key = (W, H, verts.tobytes(), rgba8.tobytes())
    if key in _ORACLE:
        return _ORACLE[key]
    fr = orc.raster(verts, vp, W, H, threads=4)
    o = orc.resolve(fr, rgba8, threads=4)
    # pixels whose two nearest fragments lie at the same depth
    ties = 0
    for p in range(W * H):
        z = np.sort(fr.z[fr.offsets[p]:fr.offsets[p + 1]])
        ties += z.size >= 2 and z[0] == z[1]
    assert ties > W * H // 4, ties
    _ORACLE[key] = o
    return o


@pytest.mark.parametrize("W,H", SIZES)
@pytest.mark.parametrize("seed", [0, 1])
def test_tie_fragments_bit_exact(orc, sn, W, H, seed):
    verts, rgba8, vp = tie_scene(W, H, seed)
    assert_frags_equal(orc, sn, verts, rgba8, vp, W, H)


@pytest.mark.parametrize("W,H", SIZES)
@pytest.mark.parametrize("seed", [0, 1])
def test_tie_separate_pass_kernels(orc, sn, W, H, seed):
    """Passes 1, 2 and 3 as three launches of the single-tile pass kernel at
    full size (no merge), and pass 1 with passes 2 and 3 merged into it."""
    verts, rgba8, vp = tie_scene(W, H, seed)
    o = oracle_layers(orc, verts, rgba8, vp, W, H)
    p = Passes(sn, verts, rgba8, vp, W, H)
    p.raster(merge=False)
    sn.geometry_pass(p.scene, p.bins[0], 1, p.l1, p.status)
    sn.geometry_pass(p.scene, p.bins[1], 2, p.l2, p.status)
    sn.geometry_pass(p.scene, p.bins[2], 3, p.l3, p.status)
    check_planes(p.planes(), o)
    q = Passes(sn, verts, rgba8, vp, W, H)
    q.raster(merge=True)
    sn.geometry_pass_merged(q.scene, q.bins[0], q.bins[1], q.bins[2], q.l1, q.l2, q.l3, q.status)
    check_planes(q.planes(), o)


@pytest.mark.parametrize("tuning", TUNINGS)
@pytest.mark.parametrize("merge", [False, True])
@pytest.mark.parametrize("W,H", SIZES)
def test_tie_persistent_passes(orc, sn, tuning, merge, W, H):
    """The persistent launch of the three passes, every tile shape and
    register budget, with passes 2 and 3 as passes of their own at full size
    or merged into pass 1."""
    verts, rgba8, vp = tie_scene(W, H, 0)
    o = oracle_layers(orc, verts, rgba8, vp, W, H)
    p = Passes(sn, verts, rgba8, vp, W, H)
    p.raster(merge=merge)
    sn.geometry_passes(p.scene, p.bins[0], p.bins[1], p.bins[2], p.l1, p.l2, p.l3, tuning, p.status)
    check_planes(p.planes(), o)


@pytest.mark.parametrize("W,H", SIZES)
def test_tie_plain_pipeline(orc, sn, W, H):
    """The plain full-resolution pipeline (one fused pass): nearest layer bit
    for bit, and the features and front terms, which hold the second layer's
    colour and the tail sums, within the float32 tolerance."""
    from tests.test_gpu_parity import run_plain
    verts, rgba8, vp = tie_scene(W, H, 1)
    mlp = scenes.mlp_xavier(2)
    r = run_plain(sn, verts, rgba8, vp, W, H, mlp)
    o = orc.frame_full(verts, rgba8, vp, W, H, scenes.mlp_flat(mlp), threads=4)
    assert np.array_equal(r.l1["id1"].cpu().numpy(), o["res"]["id1"])
    X = r.x.cpu().numpy().reshape(-1, 8)
    assert np.array_equal(X[:, 0], o["res"]["n"].astype(np.float32) / np.float32(64))
    assert np.max(np.abs(X[:, :5] - o["x"])) <= TOL_FEAT
    front = r.front.cpu().numpy().reshape(-1, 4)
    assert np.max(np.abs(front - o["front"])) <= TOL_FEAT


@pytest.mark.parametrize("tuning", [None, (4, 0, 1), (16, 6, 1), (4, 0, 2), (16, 4, 2)])
@pytest.mark.parametrize("W,H", SIZES)
def test_tie_pass_launch_resolve(orc, sn, tuning, W, H):
    """Every pass at full size: the pass launch that runs the network and the
    composite itself writes the oracle's nearest layer bit for bit and the
    frame of the separate resolve bit for bit, within the BF16 tolerance of
    the oracle's float64 frame."""
    from paper_2606_16747_b300.pipeline import Renderer
    verts, rgba8, vp = tie_scene(W, H, 0)
    mlp = scenes.mlp_xavier(4)
    outs = []
    for fuse in (False, True):
        r = Renderer(verts, rgba8, W, H, mlp=mlp, x_dtype=sn.BF16, fused=True, persistent=True,
                     tuning=tuning, fuse_passes=fuse)
        r.set_camera(vp)
        r.star_frame(update_tiles=False)
        torch.cuda.synchronize()
        r.check_status()
        resolved = int(r.bins[1].mem[44:48].view(torch.int32).item())
        assert resolved == (1 if fuse else 0)
        outs.append((r.rgba32f.clone(), r.rgba8_out.clone(), r.l1["id1"].clone(), r.l1["z1"].clone()))
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    o = orc.frame_star(verts, rgba8, vp, W, H, (W, H), (W, H), scenes.mlp_flat(mlp), threads=4)
    assert np.array_equal(outs[1][2].cpu().numpy(), o["r1"]["id1"])
    assert np.array_equal(outs[1][3].cpu().numpy().view(np.uint32), o["r1"]["z1"].view(np.uint32))
    rgb = outs[1][0].cpu().numpy().reshape(-1, 4)[:, :3]
    assert np.max(np.abs(rgb - o["rgb"])) <= TOL_BF16
