"""GPU parity of every C-ABI call against the CPU oracle on seeded inputs.

Integer and index results (fragment lists, layer ids, counts, tail sums,
quadtree masks, histograms) must be bit-exact.  Float results use the
tolerances stated per test: the kernels compute in float32, the oracle in
float64."""
import math
import os

import numpy as np
import pytest
import torch

from paper_2606_16747_b300 import scenes
from tests.helpers import pixel_vp, random_dyadic_scene, watertight_mesh

pytestmark = pytest.mark.gpu

# float32 tolerances (absolute, per channel)
TOL_FEAT = 2e-6      # features and front terms: a few float32 roundings of O(1) values
TOL_FRAME = 1e-5     # composite / reprojection
TOL_MLP32 = 1e-5     # float32 MLP vs float64


@pytest.fixture(scope="module")
def sn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_16747_b300 import build, star_nt
    build.build()
    return star_nt


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def u32(t):
    return t.cpu().numpy().view(np.uint32)


def gpu_raster(sn, verts, rgba8, vp32, W, H, cap_frags=None, pair_capacity=1 << 20):
    T = verts.shape[0]
    v = dev(verts.astype(np.float32))
    c = dev(rgba8.astype(np.uint32).view(np.int32))
    scene = sn.scene_struct(v, c)
    bins = sn.BinsBuffer(W, H, max(T, 1), pair_capacity)
    size = dev(np.array([W, H], np.int32))
    vp = dev(np.asarray(vp32, np.float32).reshape(16))
    cap = cap_frags if cap_frags is not None else max(1, 64 * W * H)
    frags = dict(count=torch.zeros(W * H, dtype=torch.int32, device="cuda"),
                 offset=torch.zeros(W * H + 1, dtype=torch.int32, device="cuda"),
                 z=torch.zeros(cap, dtype=torch.float32, device="cuda"),
                 prim=torch.zeros(cap, dtype=torch.int32, device="cuda"),
                 total=torch.zeros(1, dtype=torch.int32, device="cuda"))
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    sn.raster(scene, vp, size, W, H, bins, frags, status)
    torch.cuda.synchronize()
    return frags, int(status.item()), bins, (v, c, scene, size, vp)


def sorted_lists(counts, offsets, z, prim):
    """Per-pixel (z bits, prim) lists in key order (the kernel's order is free)."""
    out = []
    zb = z.view(np.uint32)
    for p in range(counts.size):
        a, b = int(offsets[p]), int(offsets[p + 1])
        out.append(sorted(zip(z[a:b].tolist(), prim[a:b].tolist(), zb[a:b].tolist())))
    return out


def assert_frags_equal(orc, sn, verts, rgba8, vp32, W, H):
    fr_o = orc.raster(verts, vp32, W, H)
    frags, st, _, _ = gpu_raster(sn, verts, rgba8, vp32, W, H)
    assert st == 0
    cnt = u32(frags["count"])
    assert np.array_equal(cnt, fr_o.counts)
    total = int(u32(frags["total"])[0])
    assert total == fr_o.total
    off = u32(frags["offset"])
    assert np.array_equal(off.astype(np.int64), fr_o.offsets)
    zg = frags["z"].cpu().numpy()[:total]
    pg = frags["prim"].cpu().numpy()[:total]
    assert sorted_lists(cnt, off, zg, pg) == sorted_lists(fr_o.counts, fr_o.offsets, fr_o.z, fr_o.prim)


# ---------------------------------------------------------------------------
# star_nt_raster

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_raster_dyadic_bit_exact(orc, sn, seed):
    W, H = 64, 32
    rng = np.random.default_rng(seed)
    v, c = random_dyadic_scene(rng, 40, W, H, grid=4)
    assert_frags_equal(orc, sn, v, c, pixel_vp(W, H), W, H)


def test_raster_watertight_mesh(orc, sn):
    W, H = 64, 64
    mesh = watertight_mesh(np.random.default_rng(3), W, H, 13, 11)
    c = np.full(mesh.shape[0], 0x80FFFFFF, np.uint32)
    frags, st, _, _ = gpu_raster(sn, mesh, c, pixel_vp(W, H), W, H)
    assert st == 0
    assert np.all(u32(frags["count"]) == 1)
    assert_frags_equal(orc, sn, mesh, c, pixel_vp(W, H), W, H)


@pytest.mark.parametrize("W,H", [(256, 256), (200, 120), (37, 29)])
def test_raster_perspective_scene_ragged(orc, sn, W, H):
    """Frustum scene at sizes with partial tiles on the right and bottom."""
    sc = scenes.frustum_scene(1, 32, W, H)
    assert_frags_equal(orc, sn, sc.verts, sc.rgba8, sc.cam.vp32, W, H)


def test_raster_screen_scene(orc, sn):
    sc = scenes.screen_scene(5, 3000, 320, 200, size_scale=0.5)
    assert_frags_equal(orc, sn, sc.verts, sc.rgba8, sc.cam.vp32, 320, 200)


@pytest.mark.parametrize("n_tris", [1500, 77])
def test_raster_culled_triangles(orc, sn, n_tris):
    """Set-up lanes of culled triangles, of visible ones and of the padding
    past the last triangle share warps (n_tris not a multiple of the 32
    triangles of a binning block): a camera that culls every triangle, one
    that sees none of them (all behind it), and a camera that culls part of
    the scene all match the oracle."""
    W, H = 96, 64
    sc = scenes.screen_scene(7, n_tris, W, H, size_scale=0.7)
    frags, st, _, _ = gpu_raster(sn, sc.verts, sc.rgba8, np.zeros(16, np.float32), W, H)
    assert st == 0 and int(u32(frags["total"])[0]) == 0
    behind = np.asarray(sc.cam.vp32, np.float32).reshape(4, 4) * np.array([1, 1, 1, -1], np.float32)[:, None]
    frags, st, _, _ = gpu_raster(sn, sc.verts, sc.rgba8, behind, W, H)
    assert st == 0 and int(u32(frags["total"])[0]) == 0
    # move every third triangle behind the camera: visible and culled triangles mix in a warp
    v = sc.verts.copy()
    v[::3, :, 2] = -v[::3, :, 2]
    assert_frags_equal(orc, sn, v, sc.rgba8, sc.cam.vp32, W, H)


def test_raster_empty_scene(orc, sn):
    W, H = 48, 40
    v = np.zeros((0, 3, 4), np.float32)
    frags, st, _, _ = gpu_raster(sn, v, np.zeros(0, np.uint32), pixel_vp(W, H), W, H)
    assert st == 0 and np.all(u32(frags["count"]) == 0) and int(u32(frags["total"])[0]) == 0


def test_raster_capacity_errors(orc, sn):
    """Too few (triangle, tile) pairs or fragments: ERR_CAPACITY, nothing
    written out of bounds, the fragment total still reported."""
    sc = scenes.frustum_scene(1, 32, 128, 128)
    frags, st, bins, _ = gpu_raster(sn, sc.verts, sc.rgba8, sc.cam.vp32, 128, 128, pair_capacity=8)
    assert st == sn.ERR_CAPACITY
    fr_o = orc.raster(sc.verts, sc.cam.vp32, 128, 128)
    frags, st, _, _ = gpu_raster(sn, sc.verts, sc.rgba8, sc.cam.vp32, 128, 128, cap_frags=fr_o.total - 1)
    assert st == sn.ERR_CAPACITY
    assert int(u32(frags["total"])[0]) == fr_o.total
    assert np.all(frags["z"].cpu().numpy() == 0)


# ---------------------------------------------------------------------------
# star_nt_build_inputs (fused full resolution and three-pass reduced)

def run_plain(sn, sc_verts, sc_rgba, vp32, W, H, mlp, x_dtype=None, bg=(1.0, 1.0, 1.0)):
    from paper_2606_16747_b300.pipeline import Renderer
    r = Renderer(sc_verts, sc_rgba, W, H, params=sn.default_params(bg=bg),
                 x_dtype=sn.F32 if x_dtype is None else x_dtype, mlp=mlp)
    r.set_camera(vp32)
    r.plain_frame()
    torch.cuda.synchronize()
    r.check_status()
    return r


def check_layers_full(orc_res, r, W, H):
    P = W * H
    assert np.array_equal(r.l1["id1"].cpu().numpy(), orc_res["id1"])
    assert np.array_equal(r.l1["z1"].cpu().numpy().view(np.uint32), orc_res["z1"].view(np.uint32))


@pytest.mark.parametrize("case", ["small", "ragged", "screen"])
def test_plain_frame_parity(orc, sn, case):
    if case == "small":
        sc = scenes.small_scene()
    elif case == "ragged":
        sc = scenes.frustum_scene(9, 48, 203, 117)
    else:
        sc = scenes.screen_scene(11, 4000, 400, 240, size_scale=0.6)
    W, H = sc.width, sc.height
    mlp = scenes.mlp_xavier(2)
    bg = (0.2, 0.4, 0.9)
    r = run_plain(sn, sc.verts, sc.rgba8, sc.cam.vp32, W, H, mlp, bg=bg)
    o = orc.frame_full(sc.verts, sc.rgba8, sc.cam.vp32, W, H, scenes.mlp_flat(mlp), bg, threads=4)
    res = o["res"]
    check_layers_full(res, r, W, H)
    X = r.x.cpu().numpy().reshape(-1, 8)
    flag = (res["n"] > 2)
    assert np.array_equal(X[:, 5] == 1.0, flag)
    assert np.array_equal(X[:, 0], (res["n"].astype(np.float32) / np.float32(64)))
    assert np.max(np.abs(X[:, :5] - o["x"])) <= TOL_FEAT
    front = r.front.cpu().numpy().reshape(-1, 4)
    assert np.max(np.abs(front - o["front"])) <= TOL_FEAT
    F = r.f.cpu().numpy().reshape(-1, 4)
    assert np.max(np.abs(F[:, :3] - o["f"])) <= TOL_MLP32
    rgb = r.rgba32f.cpu().numpy().reshape(-1, 4)
    assert np.max(np.abs(rgb[:, :3] - o["rgb"])) <= TOL_FRAME
    assert np.all(rgb[:, 3] == 1.0)


def test_three_pass_layers_and_features(orc, sn):
    """Passes 2 and 3 at reduced, different resolutions; per-pass planes are
    bit-exact at their own resolution, upscaled features within tolerance."""
    from paper_2606_16747_b300.pipeline import Renderer
    sc = scenes.screen_scene(13, 3000, 240, 176, size_scale=0.7)
    W, H = sc.width, sc.height
    W2, H2, W3, H3 = 145, 107, 61, 45
    mlp = scenes.mlp_xavier(4)
    r = Renderer(sc.verts, sc.rgba8, W, H, mlp=mlp)
    r.set_camera(sc.cam.vp32)
    r.state.view(torch.int32)[:6] = torch.tensor([W, H, W2, H2, W3, H3], dtype=torch.int32)
    r.star_frame(update_tiles=False)
    torch.cuda.synchronize()
    r.check_status()
    o = orc.frame_star(sc.verts, sc.rgba8, sc.cam.vp32, W, H, (W2, H2), (W3, H3),
                       scenes.mlp_flat(mlp), threads=4)
    assert np.array_equal(r.l1["id1"].cpu().numpy(), o["r1"]["id1"])
    assert np.array_equal(r.l2["id2"].cpu().numpy()[:W2 * H2], o["r2"]["id2"])
    assert np.array_equal(r.l3["n"].cpu().numpy()[:W3 * H3].view(np.uint32), o["r3"]["n"])
    tail = r.l3["tail"].cpu().numpy().view(np.uint32).reshape(-1, 4)[:W3 * H3]
    assert np.array_equal(tail[:, 0], o["r3"]["a_tail"])
    assert np.array_equal(tail[:, 1:], o["r3"]["s_tail"])
    t = r.l3["t_tail"].cpu().numpy()[:W3 * H3]
    assert np.max(np.abs(t - o["r3"]["t_tail"]) / np.maximum(o["r3"]["t_tail"], 1e-30)) <= 2e-6
    X = r.x.cpu().numpy().reshape(-1, 8)
    assert np.array_equal(X[:, 5] == 1.0, o["flag"] == 1)
    assert np.max(np.abs(X[:, :5] - o["x"])) <= 2e-5 * max(1.0, o["x"].max())
    front = r.front.cpu().numpy().reshape(-1, 4)
    assert np.max(np.abs(front - o["front"])) <= TOL_FEAT
    rgb = r.rgba32f.cpu().numpy().reshape(-1, 4)[:, :3]
    assert np.max(np.abs(rgb - o["rgb"])) <= TOL_FRAME


@pytest.mark.parametrize("sizes", [("full", "reduced"), ("reduced", "full"), ("full", "full")])
def test_merged_passes(orc, sn, sizes):
    """A pass whose device-side size equals the full size is taken over by
    pass 1 (merged); results equal the oracle's three passes at those sizes."""
    from paper_2606_16747_b300.pipeline import Renderer
    sc = scenes.screen_scene(23, 2500, 208, 144, size_scale=0.7)
    W, H = sc.width, sc.height
    s2 = (W, H) if sizes[0] == "full" else (131, 91)
    s3 = (W, H) if sizes[1] == "full" else (57, 40)
    mlp = scenes.mlp_xavier(4)
    r = Renderer(sc.verts, sc.rgba8, W, H, mlp=mlp)
    r.set_camera(sc.cam.vp32)
    r.state.view(torch.int32)[:6] = torch.tensor([W, H, *s2, *s3], dtype=torch.int32)
    r.star_frame(update_tiles=False)
    torch.cuda.synchronize()
    r.check_status()
    hdr2 = r.bins[1].mem[:64].view(torch.int32).cpu().numpy()
    hdr3 = r.bins[2].mem[:64].view(torch.int32).cpu().numpy()
    assert hdr2[8] == (sizes[0] == "full") and hdr3[8] == (sizes[1] == "full")
    o = orc.frame_star(sc.verts, sc.rgba8, sc.cam.vp32, W, H, s2, s3, scenes.mlp_flat(mlp), threads=4)
    assert np.array_equal(r.l1["id1"].cpu().numpy(), o["r1"]["id1"])
    assert np.array_equal(r.l2["id2"].cpu().numpy()[:s2[0] * s2[1]], o["r2"]["id2"])
    n3 = s3[0] * s3[1]
    assert np.array_equal(r.l3["n"].cpu().numpy()[:n3].view(np.uint32), o["r3"]["n"])
    tail = r.l3["tail"].cpu().numpy().view(np.uint32).reshape(-1, 4)[:n3]
    assert np.array_equal(tail[:, 0], o["r3"]["a_tail"]) and np.array_equal(tail[:, 1:], o["r3"]["s_tail"])
    front = r.front.cpu().numpy().reshape(-1, 4)
    assert np.max(np.abs(front - o["front"])) <= TOL_FEAT
    rgb = r.rgba32f.cpu().numpy().reshape(-1, 4)[:, :3]
    assert np.max(np.abs(rgb - o["rgb"])) <= TOL_FRAME


def test_t_tail_opaque_tail_and_determinism(orc, sn):
    """Opaque fragments in the tail give t_tail = 0 exactly; two runs of the
    same frame agree bit for bit."""
    sc = scenes.screen_scene(21, 2000, 160, 128, size_scale=0.8, alpha=(0.5, 1.0))
    mlp = scenes.mlp_xavier(2)
    r1 = run_plain(sn, sc.verts, sc.rgba8, sc.cam.vp32, 160, 128, mlp)
    r2 = run_plain(sn, sc.verts, sc.rgba8, sc.cam.vp32, 160, 128, mlp)
    for a, b in [(r1.x, r2.x), (r1.front, r2.front), (r1.rgba32f, r2.rgba32f)]:
        assert torch.equal(a, b)
    o = orc.frame_full(sc.verts, sc.rgba8, sc.cam.vp32, 160, 128, scenes.mlp_flat(mlp))
    X = r1.x.cpu().numpy().reshape(-1, 8)
    zero = o["res"]["t_tail"] == 0.0
    assert zero.sum() > 10 and np.all(X[zero, 1] == 0.0)


# ---------------------------------------------------------------------------
# star_nt_infer / star_nt_composite on seeded synthetic inputs

def synthetic_x(rng, P, empty_frac=0.2):
    x = np.zeros((P, 8), np.float32)
    x[:, 0] = rng.integers(3, 129, P) / 64.0
    x[:, 1] = rng.random(P)
    x[:, 2:5] = rng.random((P, 3))
    x[:, 5] = (rng.random(P) >= empty_frac).astype(np.float32)
    return x


@pytest.mark.parametrize("P", [1, 255, 4099])
def test_infer_f32(orc, sn, P):
    rng = np.random.default_rng(P)
    x = synthetic_x(rng, P)
    w = scenes.mlp_xavier(7)
    flat = scenes.mlp_flat(w)
    X = dev(x.reshape(-1))
    F = torch.full((P * 4,), -1.0, device="cuda")
    tw = {k: dev(v) for k, v in w.items()}
    sn.infer(sn.mlp_struct(tw), sn.F32, X, F, P)
    torch.cuda.synchronize()
    ref = orc.mlp_forward(flat.astype(np.float64), x[:, :5].astype(np.float64), x[:, 5].astype(np.uint8))
    got = F.cpu().numpy().reshape(P, 4)
    assert np.max(np.abs(got[:, :3] - ref)) <= TOL_MLP32
    assert np.all(got[:, 3] == 0)


def test_composite(orc, sn):
    rng = np.random.default_rng(0)
    P = 10007
    front = rng.random((P, 4)).astype(np.float32)
    front[:, :3] *= 0.8
    f = np.zeros((P, 4), np.float32)
    f[:, :3] = rng.random((P, 3)) * 0.6
    out = torch.zeros(P * 4, device="cuda")
    q = torch.zeros(P, dtype=torch.int32, device="cuda")
    sn.composite(dev(front.reshape(-1)), dev(f.reshape(-1)), P, out, q)
    torch.cuda.synchronize()
    ref = orc.composite(front.astype(np.float64), f[:, :3].astype(np.float64))
    got = out.cpu().numpy().reshape(P, 4)
    assert np.max(np.abs(got[:, :3] - ref)) <= 1e-6
    qo = orc.quantize(ref)
    qg = u32(q)
    # the 8-bit value may differ only where the exact value is within float32
    # rounding of a half-integer boundary
    frac = np.abs((np.clip(ref, 0, 1) * 255.0) % 1.0 - 0.5)
    safe = np.all(frac > 1e-4, axis=1)
    assert np.array_equal(qg[safe], qo[safe]) and safe.mean() > 0.99


# ---------------------------------------------------------------------------
# star_nt_quadtree on seeded images

def random_masks(rng, n):
    out = []
    for _ in range(n):
        m = 0
        if rng.random() < 0.7:
            m |= 1
            for c1 in range(4):
                if rng.random() < 0.5:
                    m |= 1 << (1 + c1)
                    for c2 in range(4):
                        if rng.random() < 0.4:
                            m |= 1 << (5 + 4 * c1 + c2)
        out.append(m)
    return np.array(out, np.uint32)


def blocky_image(rng, W, H, cell):
    """Piecewise-constant colours on random rectangles: hard edges at random
    positions, flat regions elsewhere."""
    img = np.full((H, W), 0xFF000000, np.uint32)
    for _ in range(40):
        x0, y0 = rng.integers(0, W), rng.integers(0, H)
        w, h = rng.integers(cell, 8 * cell), rng.integers(cell, 8 * cell)
        col = int(rng.integers(0, 1 << 24)) | 0xFF000000
        img[y0:y0 + h, x0:x0 + w] = col
    return img.reshape(-1)


@pytest.mark.parametrize("W,H,B,seed", [(200, 136, 16, 0), (1920, 1080, 16, 1), (1920, 1080, 64, 2),
                                        (333, 190, 64, 3)])
@pytest.mark.parametrize("iters", [2, 0])
def test_quadtree_bit_exact(orc, sn, W, H, B, seed, iters):
    rng = np.random.default_rng(seed)
    TX, TY = math.ceil(W / B), math.ceil(H / B)
    img = blocky_image(rng, W, H, B // 4)
    id1 = np.where(rng.random(W * H) < 0.9, 0, -1).astype(np.int32)
    id1[: W * (H // 3)] = -1
    mprev = random_masks(rng, TX * TY)
    params = sn.default_params(base_tile=B, tau_split=20.0, tau_merge=9.0, relax_iters=iters)
    ws = torch.zeros(sn.quadtree_ws_bytes(W, H, B), dtype=torch.uint8, device="cuda")
    mout = torch.zeros(TX * TY, dtype=torch.int32, device="cuda")
    state = torch.zeros(64, dtype=torch.uint8, device="cuda")
    sn.quadtree(dev(img.view(np.int32)), dev(id1), W, H, params, dev(mprev.view(np.int32)), mout,
                state, ws)
    torch.cuda.synchronize()
    mo, ho = orc.quadtree(img, id1, W, H, B, 20.0, 9.0, mprev, relax_iters=iters)
    assert np.array_equal(u32(mout), mo)
    st = sn.read_pass_state(state)
    assert st["hist"] == ho.tolist()
    wb, s2, s3, (W2, H2), (W3, H3) = orc.next_pass_sizes(ho, W, H)
    assert st["wbar"] == pytest.approx(wb, abs=1e-15)
    assert st["s2"] == pytest.approx(s2, rel=1e-6) and st["s3"] == pytest.approx(s3, rel=1e-6)
    assert (st["W2"], st["H2"], st["W3"], st["H3"]) == (W2, H2, W3, H3)


def test_quadtree_sequence_matches_oracle(orc, sn):
    """Several frames in a row over the same images keep identical masks."""
    rng = np.random.default_rng(5)
    W, H, B = 256, 160, 16
    TX, TY = 16, 10
    params = sn.default_params()
    ws = torch.zeros(sn.quadtree_ws_bytes(W, H, B), dtype=torch.uint8, device="cuda")
    state = torch.zeros(64, dtype=torch.uint8, device="cuda")
    mg = [torch.zeros(TX * TY, dtype=torch.int32, device="cuda") for _ in range(2)]
    mo = np.zeros(TX * TY, np.uint32)
    id1 = np.zeros(W * H, np.int32)
    for k in range(5):
        img = blocky_image(rng, W, H, 4)
        sn.quadtree(dev(img.view(np.int32)), dev(id1), W, H, params, mg[k % 2], mg[1 - k % 2], state, ws)
        mo, _ = orc.quadtree(img, id1, W, H, B, params.tau_split, params.tau_merge, mo)
        torch.cuda.synchronize()
        assert np.array_equal(u32(mg[1 - k % 2]), mo)


def test_quadtree_in_place(orc, sn):
    """mask_out may be mask_prev: a sequence updated in place matches the
    oracle frame by frame (the histogram is cleared inside the call)."""
    rng = np.random.default_rng(9)
    W, H, B = 200, 120, 16
    params = sn.default_params()
    ws = torch.zeros(sn.quadtree_ws_bytes(W, H, B), dtype=torch.uint8, device="cuda")
    state = torch.zeros(64, dtype=torch.uint8, device="cuda")
    m = torch.zeros(math.ceil(W / B) * math.ceil(H / B), dtype=torch.int32, device="cuda")
    mo = np.zeros(m.numel(), np.uint32)
    id1 = np.where(rng.random(W * H) < 0.8, 0, -1).astype(np.int32)
    for k in range(4):
        img = blocky_image(rng, W, H, 4)
        sn.quadtree(dev(img.view(np.int32)), dev(id1), W, H, params, m, m, state, ws)
        mo, ho = orc.quadtree(img, id1, W, H, B, params.tau_split, params.tau_merge, mo)
        torch.cuda.synchronize()
        assert np.array_equal(u32(m), mo)
        assert sn.read_pass_state(state)["hist"] == ho.tolist()


def test_workspaces_reused_across_calls(orc, sn):
    """The binning counters and the persistent launch's work counters clear
    themselves: one set of workspaces serves different scenes, cameras and
    pass sizes in a row with the results of fresh workspaces."""
    from paper_2606_16747_b300.pipeline import Renderer
    sc = scenes.screen_scene(17, 2000, 176, 112, size_scale=0.7)
    W, H = sc.width, sc.height
    cams = scenes.orbit_cameras(W, H, 40)
    sizes = [((W, H), (W, H)), ((131, 83), (61, 40)), ((99, 64), (W, H)), ((W, H), (88, 56))]
    reused = Renderer(sc.verts, sc.rgba8, W, H, mlp=scenes.mlp_xavier(4), x_dtype=sn.BF16, fused=True,
                      persistent=True)
    for k, (s2, s3) in enumerate(sizes):
        outs = []
        for r in (reused, Renderer(sc.verts, sc.rgba8, W, H, mlp=scenes.mlp_xavier(4), x_dtype=sn.BF16,
                                   fused=True, persistent=True)):
            r.set_camera(cams[10 * k].vp32)
            r.state.view(torch.int32)[:6] = torch.tensor([W, H, *s2, *s3], dtype=torch.int32)
            r.star_frame(update_tiles=False)
            torch.cuda.synchronize()
            r.check_status()
            outs.append((r.rgba32f.clone(), r.l1["id1"].clone()))
        assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


# ---------------------------------------------------------------------------
# star_nt_reproject

@pytest.mark.parametrize("W,H,dtheta", [(160, 96, 1 / 12), (1920, 1080, 1 / 6), (211, 97, 2.0),
                                        (3840, 2160, 0.5), (3840, 2160, 2.0)])
def test_reproject(orc, sn, W, H, dtheta):
    rng = np.random.default_rng(W)
    yy, xx = np.mgrid[0:H, 0:W]
    prev = np.stack([np.sin(xx / 7.0) * 0.5 + 0.5, np.cos(yy / 5.0) * 0.5 + 0.5,
                     rng.random((H, W)), np.ones((H, W))], -1).astype(np.float32).reshape(-1, 4)
    z1 = rng.uniform(0.9, 1.0, W * H).astype(np.float32)
    z1[rng.random(W * H) < 0.1] = 1.0
    vp_prev = scenes.camera(W, H, 10.0).vp64
    vp_cur = scenes.camera(W, H, 10.0 + dtheta).vp64
    out = torch.zeros(W * H * 4, device="cuda")
    q = torch.zeros(W * H, dtype=torch.int32, device="cuda")
    sn.reproject(dev(prev.reshape(-1)), dev(z1), dev(vp_prev.reshape(-1)), dev(vp_cur.reshape(-1)), W, H, out,
                 out_rgba8=q)
    torch.cuda.synchronize()
    ref = orc.reproject(prev, z1, vp_prev, vp_cur, W, H)
    got = out.cpu().numpy().reshape(-1, 4)
    assert np.max(np.abs(got - ref)) <= TOL_FRAME
    # the 8-bit copy quantises the float result: round half to even of
    # clamp(c, 0, 1) * 255, the product taken in float32 as the kernel does
    c = np.clip(got[:, :3], 0.0, 1.0).astype(np.float32) * np.float32(255.0)
    qc = np.rint(c).astype(np.uint32)
    qo = qc[:, 0] | (qc[:, 1] << 8) | (qc[:, 2] << 16) | np.uint32(0xFF000000)
    assert np.array_equal(u32(q), qo)


def test_reproject_identity(orc, sn):
    W, H = 128, 72
    rng = np.random.default_rng(1)
    prev = rng.random((W * H, 4)).astype(np.float32)
    z1 = rng.uniform(0.5, 1.0, W * H).astype(np.float32)
    vp = scenes.camera(W, H, 3.0).vp64.reshape(-1)
    out = torch.zeros(W * H * 4, device="cuda")
    sn.reproject(dev(prev.reshape(-1)), dev(z1), dev(vp), dev(vp), W, H, out)
    torch.cuda.synchronize()
    assert np.max(np.abs(out.cpu().numpy().reshape(-1, 4) - prev)) <= 1e-6


# ---------------------------------------------------------------------------
# full size: 1920x1080, 20k triangles, the launch configuration of the benchmark

def test_plain_frame_hd_full_size(orc, sn):
    sc = scenes.hd_scene()
    W, H = sc.width, sc.height
    mlp = scenes.mlp_xavier(2)
    r = run_plain(sn, sc.verts, sc.rgba8, sc.cam.vp32, W, H, mlp)
    o = orc.frame_full(sc.verts, sc.rgba8, sc.cam.vp32, W, H, scenes.mlp_flat(mlp), threads=16)
    check_layers_full(o["res"], r, W, H)
    X = r.x.cpu().numpy().reshape(-1, 8)
    assert np.max(np.abs(X[:, :5] - o["x"])) <= TOL_FEAT
    rgb = r.rgba32f.cpu().numpy().reshape(-1, 4)[:, :3]
    assert np.max(np.abs(rgb - o["rgb"])) <= TOL_FRAME


@pytest.mark.parametrize("workload", ["hd", "uhd"])
def test_star_frame_full_size(orc, sn, workload):
    """A real STAR-NT frame at full size in the benchmark's launch
    configuration (persistent passes, fused BF16 resolve, pass 2 merged
    above half size): pass-1 ids and depths and the merged pass-2 ids are
    bit-exact at full resolution, the pass-3 planes at their own size, and the
    frame is within the BF16 tolerance of the oracle's float64 frame."""
    from paper_2606_16747_b300.pipeline import Renderer
    sc = scenes.hd_scene() if workload == "hd" else scenes.uhd_scene()
    W, H = sc.width, sc.height
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "paper_2606_16747_b300", "weights", "tail_mlp.npz")
    mlp = dict(np.load(path))
    s2 = (math.ceil(0.71 * W), math.ceil(0.71 * H))      # merged into pass 1 (>= 0.5)
    s3 = (math.ceil(0.41 * W), math.ceil(0.41 * H))
    r = Renderer(sc.verts, sc.rgba8, W, H, mlp=mlp, x_dtype=sn.BF16, fused=True, persistent=True,
                 merge_scale2=0.5)
    r.set_camera(sc.cam.vp32)
    r.state.view(torch.int32)[:6] = torch.tensor([W, H, *s2, *s3], dtype=torch.int32)
    r.star_frame(update_tiles=False)
    torch.cuda.synchronize()
    r.check_status()
    o = orc.frame_star(sc.verts, sc.rgba8, sc.cam.vp32, W, H, (W, H), s3, scenes.mlp_flat(mlp),
                       threads=os.cpu_count() or 4)
    check_layers_full(o["r1"], r, W, H)
    assert np.array_equal(r.l2["id2"].cpu().numpy(), o["r2"]["id2"])
    P3 = s3[0] * s3[1]
    assert np.array_equal(u32(r.l3["n"])[:P3], o["r3"]["n"])
    tail = u32(r.l3["tail"])[:4 * P3].reshape(-1, 4)
    assert np.array_equal(tail[:, 0], o["r3"]["a_tail"]) and np.array_equal(tail[:, 1:], o["r3"]["s_tail"])
    rgb = r.rgba32f.cpu().numpy().reshape(-1, 4)[:, :3]
    err = np.abs(rgb - o["rgb"])
    assert err.max() <= TOL_BF16, (err.max() * 255, np.quantile(err, 0.999) * 255)


# ---------------------------------------------------------------------------
# star_nt_infer on the tcgen05 tensor cores (bf16 operands, fp32 accumulate)

TOL_BF16 = 2.0 / 255.0


def bf16_inputs(rng, P):
    x = synthetic_x(rng, P)
    xb = torch.from_numpy(x).to(torch.bfloat16)          # the input as the GPU receives it
    return xb, xb.to(torch.float64).numpy()


@pytest.mark.parametrize("P", [1, 127, 128, 129, 4099, 1 << 20])
def test_infer_bf16_tcgen05(orc, sn, P):
    rng = np.random.default_rng(1000 + P)
    xb, x64 = bf16_inputs(rng, P)
    w = scenes.mlp_xavier(7)
    flat = scenes.mlp_flat(w).astype(np.float64)
    X = xb.reshape(-1).cuda()
    F = torch.full((P * 4,), -1.0, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    tw = {k: dev(v) for k, v in w.items()}
    sn.infer(sn.mlp_struct(tw), sn.BF16, X, F, P, st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = orc.mlp_forward(flat, x64[:, :5], x64[:, 5].astype(np.uint8))
    got = F.cpu().numpy().reshape(P, 4)
    err = np.abs(got[:, :3] - ref)
    assert err.max() <= TOL_BF16, (err.max(), np.quantile(err, 0.999))
    assert np.all(got[x64[:, 5] == 0, :3] == 0) and np.all(got[:, 3] == 0)
    # repeated calls give identical bits
    F2 = torch.zeros_like(F)
    sn.infer(sn.mlp_struct(tw), sn.BF16, X, F2, P, st)
    torch.cuda.synchronize()
    assert torch.equal(F, F2)


def test_plain_frame_bf16(orc, sn):
    sc = scenes.screen_scene(17, 3000, 320, 208, size_scale=0.6)
    W, H = sc.width, sc.height
    mlp = scenes.mlp_xavier(2)
    r = run_plain(sn, sc.verts, sc.rgba8, sc.cam.vp32, W, H, mlp, x_dtype=sn.BF16)
    o = orc.frame_full(sc.verts, sc.rgba8, sc.cam.vp32, W, H, scenes.mlp_flat(mlp), threads=4)
    X = r.x.view(torch.bfloat16).to(torch.float64).cpu().numpy().reshape(-1, 8)
    ref_b = torch.from_numpy(o["x"]).to(torch.bfloat16).to(torch.float64).numpy()
    # float32 features rounded to bf16 may land one bf16 step away from the
    # float64 features rounded to bf16
    assert np.max(np.abs(X[:, :5] - ref_b) / np.maximum(np.abs(ref_b), 1e-3)) <= 2.0 ** -7
    assert np.array_equal(X[:, 5] == 1.0, o["res"]["n"] > 2)
    rgb = r.rgba32f.cpu().numpy().reshape(-1, 4)[:, :3]
    # frame error is the MLP error scaled by T_2 <= 1
    assert np.max(np.abs(rgb - o["rgb"])) <= TOL_BF16


def test_fused_resolve_equals_separate_kernels(orc, sn):
    """star_nt_resolve (upscale + features + tcgen05 MLP + composite in one
    kernel) gives the same frame as the three separate calls, and stays within
    the BF16 tolerance of the oracle's float64 frame."""
    from paper_2606_16747_b300.pipeline import Renderer
    sc = scenes.screen_scene(29, 3000, 333, 197, size_scale=0.7)   # ragged: 65601 px, partial tiles
    W, H = sc.width, sc.height
    mlp = scenes.mlp_xavier(4)
    outs = []
    for fused in (False, True):
        r = Renderer(sc.verts, sc.rgba8, W, H, mlp=mlp, x_dtype=sn.BF16, fused=fused)
        r.set_camera(sc.cam.vp32)
        r.state.view(torch.int32)[:6] = torch.tensor([W, H, 201, 119, 97, 57], dtype=torch.int32)
        r.star_frame(update_tiles=False)
        torch.cuda.synchronize()
        r.check_status()
        outs.append((r.rgba32f.clone(), r.rgba8_out.clone()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    o = orc.frame_star(sc.verts, sc.rgba8, sc.cam.vp32, W, H, (201, 119), (97, 57), scenes.mlp_flat(mlp),
                       threads=4)
    rgb = outs[1][0].cpu().numpy().reshape(-1, 4)[:, :3]
    assert np.max(np.abs(rgb - o["rgb"])) <= TOL_BF16


@pytest.mark.parametrize("tuning", [None, (16, 0, 1), (4, 3, 1), (8, 0, 2), (4, 10, 2), (16, 5, 2)])
@pytest.mark.parametrize("sizes", [((131, 91), (57, 40)), ("full", (57, 40)), ("full", "full")])
def test_persistent_passes_equal_separate(sn, tuning, sizes):
    """The three passes in one persistent launch give the same planes bit for
    bit as the separate pass kernels, for every tile shape."""
    from paper_2606_16747_b300.pipeline import Renderer
    sc = scenes.screen_scene(37, 2500, 208, 144, size_scale=0.7)
    W, H = sc.width, sc.height
    s2 = (W, H) if sizes[0] == "full" else sizes[0]
    s3 = (W, H) if sizes[1] == "full" else sizes[1]
    res = []
    for persistent in (False, True):
        r = Renderer(sc.verts, sc.rgba8, W, H, mlp=scenes.mlp_xavier(4), x_dtype=sn.BF16,
                     persistent=persistent, tuning=tuning if persistent else None)
        r.set_camera(sc.cam.vp32)
        r.state.view(torch.int32)[:6] = torch.tensor([W, H, *s2, *s3], dtype=torch.int32)
        r.star_frame(update_tiles=False)
        torch.cuda.synchronize()
        r.check_status()
        res.append([r.l1["id1"].clone(), r.l1["z1"].clone(), r.l2["id2"][:s2[0] * s2[1]].clone(),
                    r.l3["n"][:s3[0] * s3[1]].clone(), r.l3["tail"][:4 * s3[0] * s3[1]].clone(),
                    r.l3["t_tail"][:s3[0] * s3[1]].clone(), r.rgba32f.clone()])
    for a, b in zip(*res):
        assert torch.equal(a, b)


def test_pass_launch_resolve_empty_and_overflow(sn):
    """The pass launch that produces the frame: a scene whose triangles are
    all behind the camera gives the background everywhere; too small a pair
    capacity raises STAR_NT_ERR_CAPACITY in the status word (nothing hangs,
    nothing is written out of bounds)."""
    from paper_2606_16747_b300.pipeline import Renderer
    sc = scenes.screen_scene(29, 600, 200, 136, size_scale=0.7)
    W, H = sc.width, sc.height
    behind = sc.verts.copy()
    behind[..., 3] = -1.0      # w < 0: every triangle culled
    r = Renderer(behind, sc.rgba8, W, H, mlp=scenes.mlp_xavier(4), x_dtype=sn.BF16, fused=True,
                 persistent=True, params=sn.default_params(bg=(0.25, 0.5, 0.75)))
    r.set_camera(sc.cam.vp32)
    r.star_frame(update_tiles=False)
    torch.cuda.synchronize()
    r.check_status()
    assert int(r.bins[1].mem[44:48].view(torch.int32).item()) == 1   # the pass launch resolved it
    rgb = r.rgba32f.cpu().numpy().reshape(-1, 4)
    assert np.array_equal(rgb[:, :3], np.tile(np.float32([0.25, 0.5, 0.75]), (W * H, 1)))
    assert (r.l1["id1"].cpu().numpy() == -1).all()
    small = Renderer(sc.verts, sc.rgba8, W, H, mlp=scenes.mlp_xavier(4), x_dtype=sn.BF16, fused=True,
                     persistent=True, pair_capacity=64)
    small.set_camera(sc.cam.vp32)
    small.star_frame(update_tiles=False)
    torch.cuda.synchronize()
    assert int(small.status.item()) == sn.ERR_CAPACITY


def test_fixed_scales(orc, sn):
    """Fixed pass scales (the paper's ablation settings): every frame runs
    passes 2 and 3 at ceil(s W) x ceil(s H) whatever the quadtree's Eq. 2 says,
    and the frame is the oracle's at those sizes."""
    from paper_2606_16747_b300.pipeline import Renderer
    sc = scenes.screen_scene(43, 2500, 208, 144, size_scale=0.7, colours="coherent")
    W, H = sc.width, sc.height
    mlp = scenes.mlp_xavier(4)
    r = Renderer(sc.verts, sc.rgba8, W, H, mlp=mlp, x_dtype=sn.BF16, fused=True, persistent=True,
                 fixed_scales=(0.5, 0.25))
    r.set_camera(sc.cam.vp32)
    for _ in range(3):
        r.star_frame()   # the quadtree updates its state; the sizes stay fixed
    torch.cuda.synchronize()
    r.check_status()
    s2, s3 = (104, 72), (52, 36)
    for k, sz in ((1, s2), (2, s3)):
        hd = r.bins[k].header().cpu().numpy()
        assert (int(hd[0]), int(hd[1])) == sz
    o = orc.frame_star(sc.verts, sc.rgba8, sc.cam.vp32, W, H, s2, s3, scenes.mlp_flat(mlp), threads=4)
    rgb = r.rgba32f.cpu().numpy().reshape(-1, 4)[:, :3]
    assert np.max(np.abs(rgb - o["rgb"])) <= TOL_BF16


@pytest.mark.parametrize("tuning", [None, (16, 6, 1), (4, 3, 1), (8, 0, 1), (16, 4, 2)])
@pytest.mark.parametrize("sizes", ["full", "reduced3", "reduced2"])
def test_pass_launch_resolve_equals_resolve(orc, sn, tuning, sizes):
    """star_nt_geometry_passes_resolve: with every pass at full size the pass
    launch produces the frame itself, bit for bit the frame of the separate
    resolve, and writes id1 and z1; with a reduced pass it leaves the frame to
    the resolve (same frame again)."""
    from paper_2606_16747_b300.pipeline import Renderer
    sc = scenes.screen_scene(29, 3000, 333, 197, size_scale=0.7)   # ragged: partial tiles
    W, H = sc.width, sc.height
    s2 = (W, H) if sizes != "reduced2" else (201, 119)
    s3 = (W, H) if sizes != "reduced3" else (97, 57)
    mlp = scenes.mlp_xavier(4)
    outs = []
    for fuse in (False, True):
        r = Renderer(sc.verts, sc.rgba8, W, H, mlp=mlp, x_dtype=sn.BF16, fused=True, persistent=True,
                     tuning=tuning, fuse_passes=fuse)
        r.set_camera(sc.cam.vp32)
        r.state.view(torch.int32)[:6] = torch.tensor([W, H, *s2, *s3], dtype=torch.int32)
        r.rgba32f.fill_(-1.0)
        for _ in range(2):   # the second frame starts from the first's flags
            r.star_frame(update_tiles=False)
        torch.cuda.synchronize()
        r.check_status()
        resolved = int(r.bins[1].mem[44:48].view(torch.int32).item())   # BinsHeader.resolved
        outs.append((r.rgba32f.clone(), r.rgba8_out.clone(), r.l1["id1"].clone(), r.l1["z1"].clone(),
                     resolved))
    assert outs[0][4] == 0 and outs[1][4] == (1 if sizes == "full" else 0)
    for a, b in zip(outs[0][:4], outs[1][:4]):
        assert torch.equal(a, b)
    if sizes == "full" and tuning is None:
        o = orc.frame_star(sc.verts, sc.rgba8, sc.cam.vp32, W, H, (W, H), (W, H), scenes.mlp_flat(mlp),
                           threads=4)
        rgb = outs[1][0].cpu().numpy().reshape(-1, 4)[:, :3]
        assert np.max(np.abs(rgb - o["rgb"])) <= TOL_BF16


@pytest.mark.gpu
@pytest.mark.parametrize("persistent", [False, True])
def test_pass2_merge_scale(sn, persistent):
    """A pass 2 at least merge_scale of the full size is produced by pass 1 at
    the full size: the frame equals the one rendered with pass 2 requested at
    the full size, bit for bit, and the bins record the full size; below the
    scale nothing changes."""
    from paper_2606_16747_b300.pipeline import Renderer
    sc = scenes.screen_scene(41, 2500, 208, 144, size_scale=0.7)
    W, H = sc.width, sc.height

    def frame(s2, scale):
        r = Renderer(sc.verts, sc.rgba8, W, H, mlp=scenes.mlp_xavier(4), x_dtype=sn.BF16, fused=True,
                     persistent=persistent, merge_scale2=scale)
        r.set_camera(sc.cam.vp32)
        r.state.view(torch.int32)[:6] = torch.tensor([W, H, *s2, 57, 40], dtype=torch.int32)
        r.star_frame(update_tiles=False)
        torch.cuda.synchronize()
        r.check_status()
        hd = r.bins[1].header().cpu().numpy()
        return r.rgba32f.clone(), r.l2["id2"].clone(), (int(hd[0]), int(hd[1]))

    promoted = frame((131, 91), 0.6)       # 0.63 x 0.63 of full size: merged
    full = frame((W, H), 1.0)
    assert promoted[2] == (W, H)
    assert torch.equal(promoted[0], full[0]) and torch.equal(promoted[1], full[1])
    kept = frame((111, 77), 0.6)           # 0.53 of full size: a pass of its own
    plain = frame((111, 77), 1.0)
    assert kept[2] == (111, 77)
    assert torch.equal(kept[0], plain[0])


# FP8 (e4m3) tail MLP inside the fused resolve.  e4m3 keeps 3 mantissa bits,
# so every quantised input and hidden activation carries up to 2^-4 relative
# rounding and f(x) does not meet the 2/255 bar of the reduced-precision path
# (the compensated pairs below do).  Its error against the oracle is a
# measured figure that the benchmark reports, not a parity bound; what is
# asserted here holds at the float32 tolerance: pixels without a tail (f = 0)
# are the oracle's, and every pixel is finite and in range.


@pytest.mark.parametrize("kind", ["fp8", "fp8t"])
@pytest.mark.parametrize("weights", ["xavier", "trained"])
def test_fused_resolve_fp8_tailless_pixels(orc, sn, weights, kind):
    from paper_2606_16747_b300.pipeline import Renderer
    sc = scenes.screen_scene(29, 600, 333, 197, size_scale=0.7)    # ragged; pixels with and without a tail
    W, H = sc.width, sc.height
    if weights == "xavier":
        mlp = scenes.mlp_xavier(4)
    else:
        path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "paper_2606_16747_b300", "weights", "tail_mlp.npz")
        mlp = dict(np.load(path))
    r = Renderer(sc.verts, sc.rgba8, W, H, mlp=mlp, x_dtype=sn.BF16, fused=kind)
    r.set_camera(sc.cam.vp32)
    r.state.view(torch.int32)[:6] = torch.tensor([W, H, 201, 119, 97, 57], dtype=torch.int32)
    r.star_frame(update_tiles=False)
    torch.cuda.synchronize()
    r.check_status()
    o = orc.frame_star(sc.verts, sc.rgba8, sc.cam.vp32, W, H, (201, 119), (97, 57), scenes.mlp_flat(mlp),
                       threads=4)
    rgb = r.rgba32f.cpu().numpy().reshape(-1, 4)[:, :3]
    assert np.all(np.isfinite(rgb)) and rgb.min() >= 0.0
    no_tail = np.asarray(o["flag"]).ravel() == 0
    assert no_tail.sum() > 100
    assert np.abs(rgb - o["rgb"])[no_tail].max() <= TOL_FRAME


# Compensated FP8: e4m3 hi + lo pairs for every operand, the four products
# accumulated in fp32 on the tensor cores.  Each operand keeps about 2^-8
# relative rounding (hi to 2^-4, lo to 2^-4 of the remainder), the size of a
# bf16 operand's 2^-9 rounding of both operands, so the frame meets the same
# 2/255 bar as the bf16 path.
TOL_MLP = 2.0 / 255.0


@pytest.mark.parametrize("scaling", ["row", "tensor"])
@pytest.mark.parametrize("weights", ["xavier", "trained"])
def test_fused_resolve_fp8x2(orc, sn, weights, scaling):
    from paper_2606_16747_b300.pipeline import Renderer
    sc = scenes.screen_scene(29, 3000, 333, 197, size_scale=0.7)   # ragged: partial tiles
    W, H = sc.width, sc.height
    if weights == "xavier":
        mlp = scenes.mlp_xavier(4)
    else:
        path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "paper_2606_16747_b300", "weights", "tail_mlp.npz")
        mlp = dict(np.load(path))
    o = orc.frame_star(sc.verts, sc.rgba8, sc.cam.vp32, W, H, (201, 119), (97, 57), scenes.mlp_flat(mlp),
                       threads=4)
    errs = {}
    kinds = ("fp8x2", "fp8") if scaling == "row" else ("fp8x2t", "fp8t")
    for kind in kinds:
        r = Renderer(sc.verts, sc.rgba8, W, H, mlp=mlp, x_dtype=sn.BF16, fused=kind)
        r.set_camera(sc.cam.vp32)
        r.state.view(torch.int32)[:6] = torch.tensor([W, H, 201, 119, 97, 57], dtype=torch.int32)
        r.star_frame(update_tiles=False)
        torch.cuda.synchronize()
        r.check_status()
        errs[kind] = np.abs(r.rgba32f.cpu().numpy().reshape(-1, 4)[:, :3] - o["rgb"])
    err = errs[kinds[0]]
    assert err.max() <= TOL_MLP, err.max() * 255
    no_tail = np.asarray(o["flag"]).ravel() == 0
    if no_tail.any():
        assert err[no_tail].max() <= 1e-5
    # the compensation removes most of the plain e4m3 error
    assert err.max() < 0.5 * errs[kinds[1]].max()


# ---------------------------------------------------------------------------
# Comparison renderers of the evaluation (Sec. 4)

def test_unsorted_over_matches_oracle(orc, sn):
    sc = scenes.screen_scene(12, 800, 160, 96, size_scale=0.7)
    W, H = sc.width, sc.height
    frags, st, _, _ = gpu_raster(sn, sc.verts, sc.rgba8, sc.cam.vp32, W, H)
    assert st == 0
    out = torch.empty(W * H * 4, device="cuda")
    c = dev(sc.rgba8.astype(np.uint32).view(np.int32))
    bg = (0.2, 0.5, 1.0)
    sn.unsorted_over(frags, c, W, H, bg, out)
    torch.cuda.synchronize()
    fr = orc.raster(sc.verts, sc.cam.vp32, W, H, threads=4)
    ref = orc.unsorted_over(fr, sc.rgba8, bg)
    got = out.cpu().numpy().reshape(-1, 4)[:, :3]
    assert np.max(np.abs(got - ref)) <= TOL_FRAME


def test_wboit_matches_oracle(orc, sn):
    sc = scenes.screen_scene(13, 800, 160, 96, size_scale=0.7)
    W, H = sc.width, sc.height
    _, st, bins, keep = gpu_raster(sn, sc.verts, sc.rgba8, sc.cam.vp32, W, H)
    assert st == 0
    out = torch.empty(W * H * 4, device="cuda")
    out8 = torch.empty(W * H, dtype=torch.int32, device="cuda")
    bg = (0.2, 0.5, 1.0)
    sn.wboit(bins, scenes.NEAR, scenes.FAR, bg, out, out8)
    torch.cuda.synchronize()
    fr = orc.raster(sc.verts, sc.cam.vp32, W, H, threads=4)
    ref = orc.wboit(fr, sc.rgba8, scenes.NEAR, scenes.FAR, bg)
    got = out.cpu().numpy().reshape(-1, 4)[:, :3]
    # float32 sums of weights up to 3e3 in any order against float64
    assert np.max(np.abs(got - ref)) <= 1e-4
