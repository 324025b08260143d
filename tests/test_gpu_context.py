"""The context of the C ABI (star_nt_create, star_nt_workspace_size,
star_nt_bind_workspace, star_nt_frame, star_nt_tune, star_nt_destroy): a whole
STAR-NT step (real frame, interpolated frame, quadtree update) through one
call on one workspace.  Its frames, interpolated frames, masks and pass sizes
must equal, bit for bit, those of the same step composed from the separate
calls (pipeline.Renderer), frame after frame of an orbit; the step must
replay from a captured CUDA graph; the tuner must keep a candidate it timed."""
import numpy as np
import pytest
import torch

from paper_2606_16747_b300 import scenes

pytestmark = pytest.mark.gpu

MLP = {"bf16": 1, "fp8": 2, "fp8x2": 3}


@pytest.fixture(scope="module")
def sn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_16747_b300 import build, star_nt
    build.build()
    return star_nt


def _outs(W, H):
    P = W * H
    return (torch.full((P * 4,), -1.0, device="cuda"), torch.zeros(P, dtype=torch.int32, device="cuda"),
            torch.full((P * 4,), -1.0, device="cuda"), torch.zeros(P, dtype=torch.int32, device="cuda"))


def _setup(sn, kind, base_tile=16, merge=(0.5, 0.7), tuning=(8, 0, 2), W=333, H=197, n=3000):
    from paper_2606_16747_b300.pipeline import Renderer
    sc = scenes.screen_scene(31, n, W, H, size_scale=0.7, colours="coherent")
    mlp = scenes.mlp_xavier(4)
    fused = {"bf16": True, "fp8": "fp8", "fp8x2": "fp8x2"}[kind]
    r = Renderer(sc.verts, sc.rgba8, W, H, params=sn.default_params(base_tile=base_tile), mlp=mlp,
                 x_dtype=sn.BF16, fused=fused, persistent=True, tuning=tuning, merge_scale2=merge[0],
                 merge_scale3=merge[1])
    ctx = sn.Context(params=sn.default_params(base_tile=base_tile), mlp_type=MLP[kind], merge_scale2=merge[0],
                     merge_scale3=merge[1])
    ctx.set_tuning(tuning, True)
    ctx.bind(W, H, len(sc.rgba8))
    return sc, r, ctx


@pytest.mark.parametrize("kind,base_tile", [("bf16", 16), ("bf16", 64), ("fp8", 16), ("fp8x2", 64)])
def test_context_steps_equal_separate_calls(sn, kind, base_tile):
    sc, r, ctx = _setup(sn, kind, base_tile)
    W, H = sc.width, sc.height
    cams = scenes.orbit_cameras(W, H, 16, deg_per_s=30.0)
    out = _outs(W, H)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    for k in range(7):
        r.set_cameras(cams[2 * k].vp32, cams[2 * k].vp64.reshape(16), cams[2 * k + 1].vp64.reshape(16))
        r.step()
        ctx.frame(r.scene, r.mlp, r.vp, r.vp64_prev, r.vp64_cur, *out, status=st)
        torch.cuda.synchronize()
        r.check_status()
        assert int(st.item()) == sn.OK
        assert torch.equal(out[0], r.rgba32f) and torch.equal(out[1], r.rgba8_out), k
        assert torch.equal(out[2], r.interp_out) and torch.equal(out[3], r.interp_rgba8), k
        v = ctx.views()
        assert torch.equal(v["masks"], r.mask[0]), k
        assert torch.equal(v["id1"], r.l1["id1"]) and torch.equal(v["z1"], r.l1["z1"])
        a, b = sn.read_pass_state(v["state"]), r.pass_state()
        for key in ("W2", "H2", "W3", "H3", "hist", "wbar"):
            assert a[key] == b[key], (k, key)
    # the sequence really changed the pass sizes away from the first frame's
    assert (a["W2"], a["W3"]) != (W, W) or a["hist"][0] != sum(a["hist"])
    ctx.close()


def test_context_step_replays_from_a_graph(sn):
    """star_nt_frame captured once (the side stream forks and joins through
    the context's events) replays every frame of the sequence as the eager
    calls render it."""
    sc, r, ctx = _setup(sn, "bf16")
    _, _, ctx2 = _setup(sn, "bf16")
    W, H = sc.width, sc.height
    cams = scenes.orbit_cameras(W, H, 12, deg_per_s=30.0)
    vp = torch.zeros(16, device="cuda")
    v64 = torch.zeros(16, dtype=torch.float64, device="cuda")
    v64i = torch.zeros(16, dtype=torch.float64, device="cuda")
    eager, graphed = _outs(W, H), _outs(W, H)
    mlp = r.mlp

    def step():
        ctx2.frame(r.scene, mlp, vp, v64, v64i, *graphed)

    def set_cams(k):
        vp.copy_(torch.from_numpy(cams[2 * k].vp32.reshape(16)))
        v64.copy_(torch.from_numpy(cams[2 * k].vp64.reshape(16)))
        v64i.copy_(torch.from_numpy(cams[2 * k + 1].vp64.reshape(16)))

    set_cams(0)
    ctx.frame(r.scene, mlp, vp, v64, v64i, *eager)
    step()                                # the first frame eagerly on both, then capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g):
            step()
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    for k in range(1, 6):
        set_cams(k)
        ctx.frame(r.scene, mlp, vp, v64, v64i, *eager)
        g.replay()
        torch.cuda.synchronize()
        for a, b in zip(eager, graphed):
            assert torch.equal(a, b), k
    ctx.close()
    ctx2.close()


def test_context_tune(sn):
    """star_nt_tune times every candidate on the bound workspace and keeps
    the fastest; frames afterwards still equal the separate calls."""
    sc, r, ctx = _setup(sn, "bf16", merge=(1.0, 1.0))
    W, H = sc.width, sc.height
    cams = scenes.orbit_cameras(W, H, 12, deg_per_s=30.0)
    out = _outs(W, H)
    for k in range(3):
        r.set_cameras(cams[2 * k].vp32, cams[2 * k].vp64.reshape(16), cams[2 * k + 1].vp64.reshape(16))
        r.step()
        ctx.frame(r.scene, r.mlp, r.vp, r.vp64_prev, r.vp64_cur, *out)
    torch.cuda.synchronize()
    rep = ctx.tune(r.scene, r.mlp, r.vp, r.vp64_prev, out[0], out[1])
    assert len(rep["ms"]) == sn.TUNE_CANDIDATES and all(0.0 < v < 1e3 for v in rep["ms"].values())
    chosen = (rep["block_w"], rep["ctas_per_sm"], rep["pixels_per_thread"])
    assert rep["ms"][f"{chosen[0]}x{32 // chosen[0]}/{chosen[1]}/{chosen[2]}px"] == min(rep["ms"].values())
    assert ctx.tuning() == (chosen, rep["fuse_passes"])
    r.tuning, r.fuse_passes = chosen, rep["fuse_passes"]
    k = 3
    r.set_cameras(cams[2 * k].vp32, cams[2 * k].vp64.reshape(16), cams[2 * k + 1].vp64.reshape(16))
    r.step()
    ctx.frame(r.scene, r.mlp, r.vp, r.vp64_prev, r.vp64_cur, *out)
    torch.cuda.synchronize()
    assert torch.equal(out[0], r.rgba32f) and torch.equal(out[3], r.interp_rgba8)
    ctx.close()


def test_context_argument_errors(sn):
    sc, r, _ = _setup(sn, "bf16", n=600)
    W, H = sc.width, sc.height
    ctx = sn.Context()
    out = _outs(W, H)
    with pytest.raises(sn.StarNTError) as e:   # no workspace bound yet
        ctx.frame(r.scene, r.mlp, r.vp, r.vp64_prev, None, out[0], out[1])
    assert e.value.status == sn.ERR_ARG
    ctx.bind(W, H, 100)                        # fewer triangles than the scene holds
    with pytest.raises(sn.StarNTError) as e:
        ctx.frame(r.scene, r.mlp, r.vp, r.vp64_prev, None, out[0], out[1])
    assert e.value.status == sn.ERR_ARG
    with pytest.raises(sn.StarNTError):        # the real frame's two outputs are required
        ctx.frame(r.scene, r.mlp, r.vp, r.vp64_prev, None, out[0], None)
    with pytest.raises(sn.StarNTError):        # an unknown device
        sn.Context(device=torch.cuda.device_count())
    ctx.close()
