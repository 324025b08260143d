"""Failure detection on the GPU without a fault: every wait of the
tensor-core kernels (for an MMA commit or a TMA copy) is bounded.  With the
bound set to zero every such wait runs out at once; each call must then
report STAR_NT_ERR_TIMEOUT in its status word and return (the kernel lets the
work it has in flight finish and frees its tensor memory), and the device must
stay usable: the same frame rendered afterwards with the default bound equals
the frame rendered before, bit for bit."""
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


def _renderer(sn, sc, fused, fuse_passes=True):
    from paper_2606_16747_b300.pipeline import Renderer
    r = Renderer(sc.verts, sc.rgba8, sc.width, sc.height, mlp=scenes.mlp_xavier(4), x_dtype=sn.BF16,
                 fused=fused, persistent=True, fuse_passes=fuse_passes)
    r.set_camera(sc.cam.vp32)
    return r


def _frame(sn, r, state=None):
    if state is not None:
        r.state.view(torch.int32)[:6] = torch.tensor(state, dtype=torch.int32)
    r.status.zero_()
    r.star_frame(update_tiles=False)
    torch.cuda.synchronize()
    return int(r.status.item()), r.rgba32f.clone(), r.rgba8_out.clone()


@pytest.mark.parametrize("path", ["pass_launch", "resolve_bf16", "resolve_fp8", "resolve_fp8x2"])
def test_expired_waits_report_timeout(sn, path):
    sc = scenes.screen_scene(29, 2000, 333, 197, size_scale=0.7)
    W, H = sc.width, sc.height
    fused = {"pass_launch": True, "resolve_bf16": True, "resolve_fp8": "fp8", "resolve_fp8x2": "fp8x2"}[path]
    # every pass at full size: the pass launch produces the frame; a reduced
    # pass 3: the separate resolve does
    state = [W, H, W, H, W, H] if path == "pass_launch" else [W, H, 201, 119, 97, 57]
    r = _renderer(sn, sc, fused)
    st0, ref32, ref8 = _frame(sn, r, state)
    assert st0 == sn.OK
    assert sn.wait_limit() == 10 ** 9
    sn.set_wait_limit(0)
    try:
        st1, _, _ = _frame(sn, r, state)
    finally:
        sn.set_wait_limit(10 ** 9)
    assert st1 == sn.ERR_TIMEOUT
    st2, got32, got8 = _frame(sn, r, state)
    assert st2 == sn.OK
    assert torch.equal(got32, ref32) and torch.equal(got8, ref8)


def test_expired_waits_in_the_mlp(sn):
    """star_nt_infer on the tensor cores (TMA-fed): a zero bound stops it with
    STAR_NT_ERR_TIMEOUT; the next call with the default bound is exact again."""
    P = 100003
    rng = np.random.default_rng(3)
    x = np.zeros((P, 8), np.float32)
    x[:, 0] = rng.integers(3, 129, P) / 64.0
    x[:, 1:5] = rng.random((P, 4))
    x[:, 5] = 1.0
    X = torch.from_numpy(x).to(torch.bfloat16).reshape(-1).cuda()
    w = {k: torch.from_numpy(v).cuda() for k, v in scenes.mlp_xavier(7).items()}
    mlp = sn.mlp_struct(w)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    F_ref = torch.zeros(P * 4, device="cuda")
    sn.infer(mlp, sn.BF16, X, F_ref, P, st)
    torch.cuda.synchronize()
    assert int(st.item()) == sn.OK
    sn.set_wait_limit(0)
    try:
        F = torch.zeros(P * 4, device="cuda")
        sn.infer(mlp, sn.BF16, X, F, P, st)
        torch.cuda.synchronize()
    finally:
        sn.set_wait_limit(10 ** 9)
    assert int(st.item()) == sn.ERR_TIMEOUT
    st.zero_()
    sn.infer(mlp, sn.BF16, X, F, P, st)
    torch.cuda.synchronize()
    assert int(st.item()) == sn.OK and torch.equal(F, F_ref)
