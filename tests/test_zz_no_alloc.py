"""star_nt_quadtree_static: the quadtree entry point for callers that cannot
allocate device memory (a plug-in that only receives buffers from its host
application, or an engine that fixes its GPU memory at start-up and allows no
allocation on the frame path).  It keeps its workspace in a fixed array
inside the library.  Called through the C ABI, its results must equal those
of star_nt_quadtree with a caller workspace, on two calls in a row, for both
base tiles, with and without relaxation, at exactly the array's capacity, and
in a context the caller created itself."""
import ctypes
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

MAX_TILES = 65536   # STAR_NT_QT_STATIC_MAX_TILES


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


def _frame_np(rng, W, H, n_rects=60):
    img = np.full((H, W), 0xFF000000, np.uint32)
    for _ in range(n_rects):
        x0, y0 = rng.integers(0, W), rng.integers(0, H)
        w, h = rng.integers(4, 120), rng.integers(4, 120)
        img[y0:y0 + h, x0:x0 + w] = int(rng.integers(0, 1 << 24)) | 0xFF000000
    id1 = np.where(rng.random(W * H) < 0.85, 0, -1).astype(np.int32)
    return img.reshape(-1).view(np.int32), id1


def _frame(rng, W, H, n_rects=60):
    img, id1 = _frame_np(rng, W, H, n_rects)
    return torch.from_numpy(img).cuda(), torch.from_numpy(id1).cuda()


@pytest.mark.parametrize("W,H,B,iters,n_rects", [
    (1000, 600, 16, 2, 60), (1000, 600, 16, 0, 60), (1000, 600, 64, 2, 60), (1000, 600, 64, 0, 60),
    (4096, 4096, 16, 2, 4000),        # exactly the array's capacity: 256 x 256 base tiles
])
def test_static_workspace_matches_caller_workspace(sn, W, H, B, iters, n_rects):
    L = sn.lib()
    nt = math.ceil(W / B) * math.ceil(H / B)
    assert nt <= MAX_TILES
    params = sn.default_params(base_tile=B, relax_iters=iters)
    rng = np.random.default_rng(7 + B + iters)
    ws = torch.zeros(sn.quadtree_ws_bytes(W, H, B), dtype=torch.uint8, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    mask_ref = torch.zeros(nt, dtype=torch.int32, device="cuda")
    mask_new = torch.zeros(nt, dtype=torch.int32, device="cuda")
    for call in range(2):              # two calls in a row, the second on the first's masks
        img, id1 = _frame(rng, W, H, n_rects)
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
    """Frames with more base tiles than the array holds are refused before
    anything is enqueued (the pointers here are never touched)."""
    L = sn.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for W, H, B in ((8192, 8192, 16),        # 262,144 tiles
                    (16 * (MAX_TILES + 1), 16, 16),  # one tile past the limit
                    (64 * 257, 64 * 256, 64)):       # 65,792 tiles of 64 pixels
        params = sn.default_params(base_tile=B)
        s = L.star_nt_quadtree_static(16, 16, W, H, ctypes.byref(params), 16, 32, 48, stream)
        assert s == sn.ERR_CAPACITY, (W, H, B)


def test_static_workspace_in_a_context_of_the_caller(sn):
    """A host application may run its own CUDA context on the device.  The
    array's address is looked up in the context current at the call: after
    calls in the primary context, a call in a context created by the caller
    gives the same masks and state as the caller-workspace call there."""
    from cuda.bindings import driver as cu

    def ok(r):
        err = r[0] if isinstance(r, tuple) else r
        assert err == cu.CUresult.CUDA_SUCCESS, err
        return r[1] if isinstance(r, tuple) and len(r) > 1 else None

    L = sn.lib()
    W, H, B = 640, 384, 16
    nt = math.ceil(W / B) * math.ceil(H / B)
    params = sn.default_params(base_tile=B)
    rng = np.random.default_rng(11)
    img, id1 = _frame_np(rng, W, H)
    # primary context first, so that its address is cached
    mask = torch.zeros(nt, dtype=torch.int32, device="cuda")
    out_p = torch.zeros(nt, dtype=torch.int32, device="cuda")
    st_p = torch.zeros(64, dtype=torch.uint8, device="cuda")
    assert L.star_nt_quadtree_static(torch.from_numpy(img).cuda().data_ptr(),
                                     torch.from_numpy(id1).cuda().data_ptr(), W, H, ctypes.byref(params),
                                     mask.data_ptr(), out_p.data_ptr(), st_p.data_ptr(),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == sn.OK
    torch.cuda.synchronize()

    dev = ok(cu.cuDeviceGet(torch.cuda.current_device()))
    ctx = ok(cu.cuCtxCreate(None, 0, dev))          # current on this thread from here
    bufs = []
    try:
        def alloc(nbytes, host=None):
            p = ok(cu.cuMemAlloc(nbytes))
            bufs.append(p)
            if host is not None:
                ok(cu.cuMemcpyHtoD(p, host.ctypes.data, nbytes))
            else:
                ok(cu.cuMemsetD8(p, 0, nbytes))
            return int(p)

        d_img = alloc(img.nbytes, img)
        d_id1 = alloc(id1.nbytes, id1)
        d_mask = alloc(4 * nt)
        d_out_ref, d_out_new = alloc(4 * nt), alloc(4 * nt)
        d_st_ref, d_st_new = alloc(64), alloc(64)
        ws_bytes = sn.quadtree_ws_bytes(W, H, B)
        d_ws = alloc(ws_bytes)
        s1 = L.star_nt_quadtree(d_img, d_id1, W, H, ctypes.byref(params), d_mask, d_out_ref, d_st_ref,
                                d_ws, ctypes.c_size_t(ws_bytes), None)
        s2 = L.star_nt_quadtree_static(d_img, d_id1, W, H, ctypes.byref(params), d_mask, d_out_new,
                                       d_st_new, None)
        ok(cu.cuCtxSynchronize())
        assert s1 == sn.OK and s2 == sn.OK

        def fetch(p, n, dtype):
            h = np.zeros(n, dtype)
            ok(cu.cuMemcpyDtoH(h.ctypes.data, p, h.nbytes))
            return h

        m_ref, m_new = fetch(d_out_ref, nt, np.int32), fetch(d_out_new, nt, np.int32)
        st_ref, st_new = fetch(d_st_ref, 64, np.uint8), fetch(d_st_new, 64, np.uint8)
    finally:
        for p in bufs:
            cu.cuMemFree(p)
        cu.cuCtxDestroy(ctx)
    assert np.array_equal(m_ref, m_new)
    assert np.array_equal(st_ref, st_new)
    # and both equal the primary context's result on the same inputs
    assert np.array_equal(m_new, out_p.cpu().numpy())
    assert np.array_equal(st_new, st_p.cpu().numpy())
