"""GPU parity of the DFAOIT comparison network (Sec. 3.3, the original
method's eleven-input network with a sigmoid output) against the oracle: its
network input and composite terms from the full-resolution pass, the float32
and the bf16 tensor-core forward, the whole frame C = C_t + C_b prod(1 - a),
and the backward kernel's gradient."""
import numpy as np
import pytest
import torch

from paper_2606_16747_b300 import scenes

pytestmark = pytest.mark.gpu

TOL_FEAT = 2e-6
TOL_F32 = 1e-5
TOL_BF16 = 2.0 / 255.0
SHAPES = (("w1", (32, 11)), ("b1", (32,)), ("w2", (16, 32)), ("b2", (16,)), ("w3", (3, 16)), ("b3", (3,)))


@pytest.fixture(scope="module")
def sn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_16747_b300 import build, star_nt
    build.build()
    return star_nt


def weights(seed):
    rng = np.random.default_rng(seed)
    w = {}
    for name, shape in SHAPES:
        if name.startswith("w"):
            lim = np.sqrt(6.0 / (shape[0] + shape[1]))
            w[name] = rng.uniform(-lim, lim, shape).astype(np.float32)
        else:
            w[name] = rng.uniform(-0.2, 0.2, shape).astype(np.float32)
    return w


def flat(w):
    return np.concatenate([w[k].ravel() for k, _ in SHAPES]).astype(np.float64)


def gpu_inputs(sn, sc, x_dtype, bg=(1.0, 1.0, 1.0)):
    W, H = sc.width, sc.height
    P = W * H
    v = torch.from_numpy(np.ascontiguousarray(sc.verts)).cuda()
    c = torch.from_numpy(np.ascontiguousarray(sc.rgba8).view(np.int32)).cuda()
    scene = sn.scene_struct(v, c)
    bins = sn.BinsBuffer(W, H, len(sc.rgba8), 1 << 20)
    size = torch.tensor([W, H], dtype=torch.int32, device="cuda")
    vp = torch.from_numpy(np.ascontiguousarray(sc.cam.vp32)).cuda()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    sn.raster(scene, vp, size, W, H, bins, None, st)
    x = torch.full((P * 16,), -1.0, dtype=torch.float32 if x_dtype == sn.F32 else torch.bfloat16, device="cuda")
    front = torch.empty(P * 4, device="cuda")
    l1 = dict(id1=torch.empty(P, dtype=torch.int32, device="cuda"), z1=torch.empty(P, device="cuda"))
    sn.build_inputs_dfaoit(scene, bins, l1, W, H, sn.default_params(bg=bg), x, x_dtype, front, st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    return x, front, l1, (v, c, scene, bins)


@pytest.mark.parametrize("case", ["ragged", "screen"])
def test_features_and_front(orc, sn, case):
    sc = (scenes.frustum_scene(9, 48, 203, 117) if case == "ragged"
          else scenes.screen_scene(11, 3000, 333, 197, size_scale=0.6))
    W, H = sc.width, sc.height
    bg = (0.2, 0.4, 0.9)
    x, front, l1, _ = gpu_inputs(sn, sc, sn.F32, bg)
    fr = orc.raster(sc.verts, sc.cam.vp32, W, H, threads=4)
    xo, t_all = orc.dfaoit_features(fr, sc.rgba8, threads=4)
    X = x.cpu().numpy().reshape(-1, 16)
    assert np.max(np.abs(X[:, :11] - xo)) <= TOL_FEAT * max(1.0, np.abs(xo).max())
    assert np.array_equal(X[:, 11] == 1.0, fr.counts > 0)
    assert np.all(X[:, 12:] == 0.0)
    F = front.cpu().numpy().reshape(-1, 4)
    assert np.max(np.abs(F[:, :3] - t_all[:, None] * np.array(bg)[None, :])) <= TOL_FEAT
    assert np.all(F[:, 3] == 1.0)
    r = orc.resolve(fr, sc.rgba8)
    assert np.array_equal(l1["id1"].cpu().numpy(), r["id1"])
    assert (fr.counts > 2).mean() > 0.2


def _x(rng, P):
    x = np.zeros((P, 16), np.float32)
    x[:, 0:10] = rng.random((P, 10))
    x[:, 10] = rng.integers(1, 100, P) / 64.0
    x[:, 11] = (rng.random(P) < 0.85).astype(np.float32)
    return x


@pytest.mark.parametrize("P", [1, 300, 4099])
def test_forward_f32(orc, sn, P):
    rng = np.random.default_rng(P)
    x = _x(rng, P)
    w = weights(3)
    tw = {k: torch.from_numpy(v).cuda() for k, v in w.items()}
    F = torch.full((P * 4,), -1.0, device="cuda")
    sn.infer_dfaoit(sn.mlp_struct(tw), sn.F32, torch.from_numpy(x.reshape(-1)).cuda(), F, P)
    torch.cuda.synchronize()
    ref = orc.mlp_dfaoit_forward(flat(w), x[:, :11].astype(np.float64), x[:, 11].astype(np.uint8))
    got = F.cpu().numpy().reshape(P, 4)
    assert np.max(np.abs(got[:, :3] - ref)) <= TOL_F32
    assert np.all(got[x[:, 11] == 0, :3] == 0.0) and np.all(got[:, 3] == 0.0)


@pytest.mark.parametrize("P", [1, 127, 128, 129, 4099, 1 << 20])
def test_forward_bf16_tcgen05(orc, sn, P):
    rng = np.random.default_rng(100 + P)
    x = _x(rng, P)
    xb = torch.from_numpy(x).to(torch.bfloat16)            # the input as the GPU receives it
    x64 = xb.to(torch.float64).numpy()
    w = weights(4)
    tw = {k: torch.from_numpy(v).cuda() for k, v in w.items()}
    X = xb.reshape(-1).cuda()
    F = torch.full((P * 4,), -1.0, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    sn.infer_dfaoit(sn.mlp_struct(tw), sn.BF16, X, F, P, st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref = orc.mlp_dfaoit_forward(flat(w), x64[:, :11], x64[:, 11].astype(np.uint8))
    got = F.cpu().numpy().reshape(P, 4)
    err = np.abs(got[:, :3] - ref)
    assert err.max() <= TOL_BF16, (err.max() * 255, np.quantile(err, 0.999) * 255)
    assert np.all(got[x64[:, 11] == 0, :3] == 0.0) and np.all(got[:, 3] == 0.0)
    F2 = torch.zeros_like(F)
    sn.infer_dfaoit(sn.mlp_struct(tw), sn.BF16, X, F2, P, st)
    torch.cuda.synchronize()
    assert torch.equal(F, F2)


@pytest.mark.parametrize("x_dtype,tol", [("f32", TOL_F32), ("bf16", TOL_BF16)])
def test_frame(orc, sn, x_dtype, tol):
    """Features, network and composite on a ragged scene: the frame against
    the oracle's DFAOIT frame."""
    sc = scenes.screen_scene(29, 3000, 333, 197, size_scale=0.7)
    W, H = sc.width, sc.height
    P = W * H
    dt = sn.F32 if x_dtype == "f32" else sn.BF16
    x, front, _, keep = gpu_inputs(sn, sc, dt)
    w = weights(5)
    tw = {k: torch.from_numpy(v).cuda() for k, v in w.items()}
    f = torch.empty(P * 4, device="cuda")
    out = torch.empty(P * 4, device="cuda")
    sn.infer_dfaoit(sn.mlp_struct(tw), dt, x, f, P)
    sn.composite(front, f, P, out, None)
    torch.cuda.synchronize()
    o = orc.frame_dfaoit(sc.verts, sc.rgba8, sc.cam.vp32, W, H, flat(w), threads=4)
    rgb = out.cpu().numpy().reshape(-1, 4)[:, :3]
    assert np.max(np.abs(rgb - o["rgb"])) <= tol


def test_backward_matches_oracle_gradient(orc, sn):
    from paper_2606_16747_b300 import train
    rng = np.random.default_rng(0)
    B = 5000
    x = _x(rng, B)
    x[:, 11] = 1.0
    y = np.zeros((B, 4), np.float32)
    y[:, :3] = rng.random((B, 3))
    w = weights(6)
    fl = flat(w)
    params = torch.tensor(fl.astype(np.float32), device="cuda")
    mlp = train.mlp_from_flat(params, shapes=SHAPES)
    X = torch.from_numpy(x.reshape(-1)).cuda()
    Y = torch.from_numpy(y.reshape(-1)).cuda()
    f = torch.empty(B * 4, device="cuda")
    sn.infer_dfaoit(mlp, sn.F32, X, f, B)
    dy = torch.empty(B * 4, device="cuda")
    loss = torch.empty(1, device="cuda")
    ws = torch.empty(sn.train_ws_bytes(B), dtype=torch.uint8, device="cuda")
    sn.mse_grad(f, Y, B, dy, loss, ws)
    g = torch.empty(963, device="cuda")
    sn.dfaoit_backward(mlp, X, dy, B, g, ws)
    torch.cuda.synchronize()
    lo, go = orc.mlp_dfaoit_mse_grad(fl, x[:, :11].astype(np.float64), y[:, :3].astype(np.float64))
    assert float(loss.item()) == pytest.approx(lo, rel=1e-5)
    gg = g.cpu().numpy()
    assert np.max(np.abs(gg - go)) <= 1e-5 * np.abs(go).max() + 1e-9
