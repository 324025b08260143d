"""Pins of the oracle's tail-colour MLP (Sec. 3.3: 5-32-16-3, ReLU output,
MSE loss, Adam) against a hand-built network, torch float64 autograd,
finite differences and torch.optim.Adam."""
import numpy as np
import pytest
import torch

from paper_2606_16747_b300 import scenes


def _unflat(p):
    out, o = {}, 0
    for name, shape in scenes.MLP_SHAPES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def _torch_forward(p, x):
    t = {k: torch.tensor(v, dtype=torch.float64) for k, v in _unflat(p).items()}
    h = torch.relu(x @ t["w1"].T + t["b1"])
    h = torch.relu(h @ t["w2"].T + t["b2"])
    return torch.relu(h @ t["w3"].T + t["b3"])


def test_param_count():
    assert scenes.MLP_PARAM_COUNT == 771
    assert scenes.mlp_flat(scenes.mlp_xavier()).size == 771


def test_hand_built_network(orc):
    """Identity-like weights pass x2..x4 through; a negative output bias then
    shows the output ReLU: f = max(x_{2+k} - 0.1, 0)."""
    p = {n: np.zeros(s) for n, s in scenes.MLP_SHAPES}
    for k in range(5):
        p["w1"][k, k] = 1.0
    for k in range(16):
        p["w2"][k, k] = 1.0
    for k in range(3):
        p["w3"][k, 2 + k] = 1.0
    p["b3"][:] = -0.1
    flat = np.concatenate([p[n].reshape(-1) for n, _ in scenes.MLP_SHAPES])
    x = np.array([[0.3, 0.9, 0.05, 0.6, 0.1]])
    f = orc.mlp_forward(flat, x)
    assert f[0].tolist() == pytest.approx([0.0, 0.5, 0.0], abs=1e-15)


def test_forward_matches_torch_float64(orc):
    rng = np.random.default_rng(0)
    p = rng.normal(size=771) * 0.5
    x = rng.random((500, 5))
    f = orc.mlp_forward(p, x)
    ref = _torch_forward(p, torch.tensor(x)).numpy()
    assert np.max(np.abs(f - ref)) < 1e-13
    assert (f > 0).mean() > 0.2


def test_forward_zero_where_tail_empty(orc):
    rng = np.random.default_rng(1)
    p = rng.normal(size=771)
    x = rng.random((50, 5))
    flag = (rng.random(50) < 0.5).astype(np.uint8)
    f = orc.mlp_forward(p, x, flag)
    assert np.all(f[flag == 0] == 0)
    assert np.array_equal(f[flag == 1], orc.mlp_forward(p, x[flag == 1]))


def test_gradient_matches_torch_autograd(orc):
    rng = np.random.default_rng(2)
    p = rng.normal(size=771) * 0.5
    x = rng.random((300, 5))
    y = rng.random((300, 3))
    loss, g = orc.mlp_mse_grad(p, x, y)
    pt = torch.tensor(p, requires_grad=True)
    parts, o = {}, 0
    for name, shape in scenes.MLP_SHAPES:
        n = int(np.prod(shape))
        parts[name] = pt[o:o + n].reshape(shape)
        o += n
    xt = torch.tensor(x)
    h = torch.relu(xt @ parts["w1"].T + parts["b1"])
    h = torch.relu(h @ parts["w2"].T + parts["b2"])
    f = torch.relu(h @ parts["w3"].T + parts["b3"])
    lt = ((f - torch.tensor(y)) ** 2).mean()
    lt.backward()
    assert loss == pytest.approx(lt.item(), rel=1e-13)
    assert np.max(np.abs(g - pt.grad.numpy())) < 1e-13


def test_gradient_finite_differences(orc):
    rng = np.random.default_rng(3)
    p = rng.normal(size=771) * 0.5
    x = rng.random((64, 5))
    y = rng.random((64, 3))
    _, g = orc.mlp_mse_grad(p, x, y)
    h = 1e-6
    idx = np.concatenate([rng.choice(160, 6, replace=False), 160 + rng.choice(32, 3, replace=False),
                          192 + rng.choice(512, 6, replace=False), 704 + rng.choice(16, 3, replace=False),
                          720 + rng.choice(48, 4, replace=False), [768, 769, 770]])
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (orc.mlp_mse_grad(pp, x, y)[0] - orc.mlp_mse_grad(pm, x, y)[0]) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-6, abs=1e-9), i


def test_adam_matches_torch(orc):
    rng = np.random.default_rng(4)
    p0 = rng.normal(size=771)
    p, m, v = p0.copy(), np.zeros(771), np.zeros(771)
    pt = torch.tensor(p0, requires_grad=True)
    opt = torch.optim.Adam([pt], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for step in range(1, 6):
        g = rng.normal(size=771)
        orc.adam(p, g, m, v, step)
        opt.zero_grad()
        pt.grad = torch.tensor(g)
        opt.step()
    assert np.max(np.abs(p - pt.detach().numpy())) < 1e-14
