"""GPU checks of the learned part: exact A-buffer and tail colour, the MLP
backward kernel against the oracle's float64 gradient and finite
differences, Adam, the autograd wrappers, and a short training run that must
beat the method without the network on held-out scenes."""
import numpy as np
import pytest
import torch

from paper_2606_16747_b300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_16747_b300 import build, star_nt
    build.build()
    return star_nt


def test_abuffer_and_exact_tail(orc, sn):
    from paper_2606_16747_b300 import train
    sc = scenes.screen_scene(31, 3000, 240, 160, size_scale=0.8)
    d = train.render_samples(sc)
    fr = orc.raster(sc.verts, sc.cam.vp32, sc.width, sc.height)
    r = orc.resolve(fr, sc.rgba8, (1.0, 1.0, 1.0))
    abuf = d["abuf"].cpu().numpy()
    tail = d["tail"].cpu().numpy()
    assert np.max(np.abs(abuf[:, :3] - r["abuf"])) <= 1e-5
    assert np.max(np.abs(abuf[:, 3] - r["t_all"])) <= 1e-5
    assert np.max(np.abs(tail[:, :3] - r["tail_rgb"])) <= 1e-5
    assert np.max(np.abs(tail[:, 3] - r["t_tail"])) <= 1e-5
    # Eq. 4 with the exact tail colour reproduces the A-buffer on the GPU too
    front = d["front"].cpu().numpy()
    rec = front[:, :3] + front[:, 3:4] * tail[:, :3]
    assert np.max(np.abs(rec - abuf[:, :3])) <= 2e-5


def _synthetic(rng, B):
    x = np.zeros((B, 8), np.float32)
    x[:, 0] = rng.integers(3, 100, B) / 64.0
    x[:, 1] = rng.random(B)
    x[:, 2:5] = rng.random((B, 3))
    x[:, 5] = 1.0
    y = np.zeros((B, 4), np.float32)
    y[:, :3] = rng.random((B, 3)) * 0.5
    return x, y


def test_backward_matches_oracle_gradient(orc, sn):
    from paper_2606_16747_b300 import train
    rng = np.random.default_rng(0)
    B = 5000
    x, y = _synthetic(rng, B)
    flat = scenes.mlp_flat(scenes.mlp_xavier(5))
    flat[160:192] += 0.1          # positive hidden biases: more active units
    params = torch.tensor(flat, device="cuda")
    X, Y = torch.tensor(x.reshape(-1), device="cuda"), torch.tensor(y.reshape(-1), device="cuda")
    p = params.clone().requires_grad_(True)
    f = train.TailMLPFunction.apply(X, p)
    loss = train.MSEFunction.apply(f, Y)
    loss.backward()
    lo, go = orc.mlp_mse_grad(flat.astype(np.float64), x[:, :5].astype(np.float64), y[:, :3].astype(np.float64))
    assert float(loss.item()) == pytest.approx(lo, rel=1e-5)
    g = p.grad.cpu().numpy()
    scale = np.abs(go).max()
    assert np.max(np.abs(g - go)) <= 1e-5 * scale + 1e-9
    # deterministic: a second backward gives identical bits
    p2 = params.clone().requires_grad_(True)
    train.MSEFunction.apply(train.TailMLPFunction.apply(X, p2), Y).backward()
    assert torch.equal(p.grad, p2.grad)


def test_backward_finite_differences(sn):
    from paper_2606_16747_b300 import train
    rng = np.random.default_rng(1)
    B = 2048
    x, y = _synthetic(rng, B)
    flat = scenes.mlp_flat(scenes.mlp_xavier(6)).astype(np.float64)
    flat[160:192] += 0.1
    X, Y = torch.tensor(x.reshape(-1), device="cuda"), torch.tensor(y.reshape(-1), device="cuda")

    def loss_at(v):
        p = torch.tensor(v.astype(np.float32), device="cuda")
        return float(train.MSEFunction.apply(train.TailMLPFunction.apply(X, p), Y).item())

    p = torch.tensor(flat.astype(np.float32), device="cuda", requires_grad=True)
    train.MSEFunction.apply(train.TailMLPFunction.apply(X, p), Y).backward()
    g = p.grad.cpu().numpy()
    h = 1e-2
    for i in [0, 7, 161, 200, 500, 705, 721, 768, 770]:
        a, b = flat.copy(), flat.copy()
        a[i] += h
        b[i] -= h
        fd = (loss_at(a) - loss_at(b)) / (2 * h)
        assert fd == pytest.approx(g[i], rel=3e-2, abs=2e-5), i


def test_adam_matches_oracle(orc, sn):
    rng = np.random.default_rng(2)
    n = 771
    p0 = rng.normal(size=n).astype(np.float32)
    pg, mg, vg = (torch.tensor(p0, device="cuda"), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda"))
    rounded = torch.zeros(n, device="cuda")
    po, mo, vo = p0.astype(np.float64), np.zeros(n), np.zeros(n)
    for step in range(1, 6):
        g = rng.normal(size=n).astype(np.float32)
        sn.adam(pg, torch.tensor(g, device="cuda"), mg, vg, step, bf16_rounded=rounded)
        orc.adam(po, g.astype(np.float64), mo, vo, step)
    assert np.max(np.abs(pg.cpu().numpy() - po)) <= 1e-6
    assert torch.equal(rounded, pg.to(torch.bfloat16).to(torch.float32))


def test_short_training_beats_no_network(sn):
    """A short run on a few scenes lowers the loss and the trained network
    beats f = 0 on held-out scenes (PSNR against the exact A-buffer)."""
    from paper_2606_16747_b300 import train
    x, y, _ = train.build_dataset(range(3000, 3008), 256, 256, log=None)
    assert x.shape[0] > 100000 and torch.all(x[:, 5] == 1.0)
    st = train.train(x, y, steps=400, batch=16384, log=None, every=100)
    hist = st["history"]
    assert hist[-1][1] < 0.5 * hist[0][1]
    ev = train.evaluate(train.flat_to_dict(st["master"]), range(3100, 3104), 256, 256)
    assert ev["mlp_f32"] > ev["zero"] + 10.0          # what the network adds to Eq. 4
    assert ev["mlp_f32"] > ev["heuristic"] - 3.0       # close to the plain tail estimate after a short run
    assert abs(ev["mlp_bf16"] - ev["mlp_f32"]) < 0.5


def test_weighted_mse_kernel(sn):
    """star_nt_wmse_grad: w = 1 reproduces star_nt_mse_grad bit for bit, and
    general weights give the definition's loss and gradient."""
    from paper_2606_16747_b300.train import _WS
    rng = np.random.default_rng(11)
    B = 5000
    f = torch.tensor(rng.uniform(-1, 2, size=(B, 4)).astype(np.float32), device="cuda")
    y = torch.tensor(rng.uniform(0, 1, size=(B, 4)).astype(np.float32), device="cuda")
    w = torch.tensor(rng.uniform(0, 1, size=B).astype(np.float32), device="cuda")
    ws = _WS.get(B, "cuda")
    dy0, l0 = torch.empty_like(f), torch.empty(1, device="cuda")
    dy1, l1 = torch.empty_like(f), torch.empty(1, device="cuda")
    sn.mse_grad(f, y, B, dy0, l0, ws)
    sn.mse_grad(f, y, B, dy1, l1, ws, w=torch.ones(B, device="cuda"))
    torch.cuda.synchronize()
    assert torch.equal(dy0, dy1) and torch.equal(l0, l1)
    sn.mse_grad(f, y, B, dy1, l1, ws, w=w)
    torch.cuda.synchronize()
    fd, yd, wd = (t.cpu().numpy().astype(np.float64) for t in (f, y, w))
    e = fd[:, :3] - yd[:, :3]
    assert abs(float(l1.item()) - (wd[:, None] * e * e).sum() / (3 * B)) <= 1e-5 * (1 + abs(float(l1.item())))
    assert np.allclose(dy1.cpu().numpy()[:, :3], 2 * wd[:, None] * e / (3 * B), rtol=1e-5, atol=1e-9)
    assert np.all(dy1.cpu().numpy()[:, 3] == 0)


def _grad(sn, flat, x, y):
    from paper_2606_16747_b300 import train
    X, Y = torch.tensor(x.reshape(-1), device="cuda"), torch.tensor(y.reshape(-1), device="cuda")
    p = torch.tensor(flat, device="cuda", requires_grad=True)
    loss = train.MSEFunction.apply(train.TailMLPFunction.apply(X, p), Y)
    loss.backward()
    return float(loss.item()), p.grad.cpu().numpy()


@pytest.mark.parametrize("B", [1, 127, 129, 100003])
def test_backward_batch_sizes(orc, sn, B):
    """The tensor-core contraction over the batch: a single partial tile, a
    ragged last tile, and (100,003 samples: 782 tiles) several tiles per CTA
    accumulated in tensor memory; the gradient within float32 rounding of
    the oracle's float64 one."""
    rng = np.random.default_rng(B)
    x, y = _synthetic(rng, B)
    flat = scenes.mlp_flat(scenes.mlp_xavier(7))
    flat[160:192] += 0.1
    lo, go = orc.mlp_mse_grad(flat.astype(np.float64), x[:, :5].astype(np.float64), y[:, :3].astype(np.float64))
    loss, g = _grad(sn, flat, x, y)
    assert loss == pytest.approx(lo, rel=1e-5)
    scale = np.abs(go).max()
    assert np.max(np.abs(g - go)) <= 1e-5 * scale + 1e-9


def test_backward_expired_wait(sn):
    """A tensor-core wait that runs out (bound 0) reports STAR_NT_ERR_TIMEOUT
    and poisons the gradient with NaN instead of returning a partial sum; the
    next call with the default bound gives the same bits as before."""
    rng = np.random.default_rng(3)
    B = 3000
    x, y = _synthetic(rng, B)
    flat = scenes.mlp_flat(scenes.mlp_xavier(8))
    params = torch.tensor(flat, device="cuda")
    from paper_2606_16747_b300 import train
    X = torch.tensor(x.reshape(-1), device="cuda")
    dy = torch.tensor(rng.standard_normal((B, 4)).astype(np.float32).reshape(-1), device="cuda")
    ws = torch.empty(sn.train_ws_bytes(B), dtype=torch.uint8, device="cuda")
    mlp = train.mlp_from_flat(params)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    g0 = torch.empty(771, device="cuda")
    sn.mlp_backward(mlp, X, dy, B, g0, ws, status)
    torch.cuda.synchronize()
    assert int(status.item()) == sn.OK and torch.isfinite(g0).all()
    g1 = torch.empty(771, device="cuda")
    sn.set_wait_limit(0)
    try:
        sn.mlp_backward(mlp, X, dy, B, g1, ws, status)
        torch.cuda.synchronize()
    finally:
        sn.set_wait_limit(10 ** 9)
    assert int(status.item()) == sn.ERR_TIMEOUT
    assert torch.isnan(g1).all()
    status.zero_()
    g2 = torch.empty(771, device="cuda")
    sn.mlp_backward(mlp, X, dy, B, g2, ws, status)
    torch.cuda.synchronize()
    assert int(status.item()) == sn.OK
    assert torch.equal(g0, g2)


@pytest.mark.parametrize("cols,dtype", [(1, torch.float32), (4, torch.float32), (8, torch.float32),
                                        (16, torch.float32), (3, torch.int32), (8, torch.bfloat16)])
def test_gather_rows(sn, cols, dtype):
    """The minibatch gather against torch indexing: 16-byte chunks where rows
    allow them, 4-byte words otherwise; repeated indices; an index out of
    range gives a zero row and STAR_NT_ERR_ARG."""
    rng = np.random.default_rng(cols)
    n_src, n = 10007, 4099
    src = torch.tensor(rng.standard_normal((n_src, cols)), device="cuda").to(dtype).contiguous()
    if src.numel() * src.element_size() // n_src % 4:
        pytest.skip("rows must be a multiple of 4 bytes")
    idx = torch.tensor(rng.integers(0, n_src, n), dtype=torch.int64, device="cuda")
    dst = torch.empty((n, cols), dtype=dtype, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    sn.gather_rows(src, idx, dst, status)
    torch.cuda.synchronize()
    assert int(status.item()) == sn.OK
    assert torch.equal(dst, src[idx])
    idx[7] = n_src
    idx[9] = -1
    sn.gather_rows(src, idx, dst, status)
    torch.cuda.synchronize()
    assert int(status.item()) == sn.ERR_ARG
    assert (dst[7] == 0).all() and (dst[9] == 0).all()
    keep = torch.ones(n, dtype=torch.bool, device="cuda")
    keep[7] = keep[9] = False
    assert torch.equal(dst[keep], src[idx[keep]])
