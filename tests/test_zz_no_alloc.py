"""star_nt_quadtree_static: the quadtree entry point for callers that cannot
allocate device memory (it keeps its workspace in a fixed array inside the
library).  Called through the C ABI, its results must equal those of
star_nt_quadtree with a caller workspace, on two calls in a row."""
import ctypes
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sn():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_16747_b300 import build, star_nt
    build.build()
    L = star_nt.lib()
    L.star_nt_quadtree_static.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.POINTER(star_nt.Params),
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p]
    L.star_nt_quadtree_static.restype = ctypes.c_int32
    return star_nt


def _frame(rng, W, H):
    img = np.full((H, W), 0xFF000000, np.uint32)
    for _ in range(60):
        x0, y0 = rng.integers(0, W), rng.integers(0, H)
        w, h = rng.integers(4, 120), rng.integers(4, 120)
        img[y0:y0 + h, x0:x0 + w] = int(rng.integers(0, 1 << 24)) | 0xFF000000
    id1 = np.where(rng.random(W * H) < 0.85, 0, -1).astype(np.int32)
    return (torch.from_numpy(img.reshape(-1).view(np.int32)).cuda(), torch.from_numpy(id1).cuda())


def test_static_workspace_matches_caller_workspace(sn):
    L = sn.lib()
    W, H, B = 1000, 600, 16
    nt = math.ceil(W / B) * math.ceil(H / B)
    params = sn.default_params(base_tile=B)
    rng = np.random.default_rng(7)
    ws = torch.zeros(sn.quadtree_ws_bytes(W, H, B), dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    mask_ref = torch.zeros(nt, dtype=torch.int32, device="cuda")
    mask_new = torch.zeros(nt, dtype=torch.int32, device="cuda")
    for call in range(2):              # two calls in a row, the second on the first's masks
        img, id1 = _frame(rng, W, H)
        out_ref = torch.zeros(nt, dtype=torch.int32, device="cuda")
        out_new = torch.full((nt,), -1, dtype=torch.int32, device="cuda")
        st_ref = torch.zeros(64, dtype=torch.uint8, device="cuda")
        st_new = torch.full((64,), 255, dtype=torch.uint8, device="cuda")
        sn.quadtree(img, id1, W, H, params, mask_ref, out_ref, st_ref, ws)
        s = L.star_nt_quadtree_static(img.data_ptr(), id1.data_ptr(), W, H, ctypes.byref(params),
                                      mask_new.data_ptr(), out_new.data_ptr(), st_new.data_ptr(),
                                      stream)
        assert s == sn.OK
        torch.cuda.synchronize()
        assert torch.equal(out_ref, out_new), f"masks differ on call {call}"
        ref, new = sn.read_pass_state(st_ref), sn.read_pass_state(st_new)
        assert ref == new, f"pass state differs on call {call}"
        assert sum(ref["hist"]) > 0
        mask_ref, mask_new = out_ref, out_new


def test_static_workspace_rejects_oversized_frames(sn):
    L = sn.lib()
    params = sn.default_params(base_tile=16)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # 8192 x 8192 at 16-pixel tiles is 262144 tiles, beyond the 65536 the array holds
    s = L.star_nt_quadtree_static(16, 16, 8192, 8192, ctypes.byref(params), 16, 32, 48, stream)
    assert s == sn.ERR_CAPACITY
