"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point declared in include/star_nt.h, and rejects bad arguments
before enqueuing any work."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "star_nt.h")


@pytest.fixture(scope="module")
def sn():
    from paper_2606_16747_b300 import build, star_nt
    build.build()
    return star_nt


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(star_nt_\w+)\s*\(", text)))


def test_header_declares_the_six_calls():
    names = declared_functions()
    for call in ("star_nt_raster", "star_nt_build_inputs", "star_nt_infer", "star_nt_quadtree",
                 "star_nt_reproject", "star_nt_composite"):
        assert call in names


def test_library_exports_every_declared_symbol(sn):
    L = sn.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert set(sn.EXPORTS) <= set(declared_functions())


def test_version_status_and_defaults(sn):
    assert sn.lib().star_nt_version() == 1
    assert sn.status_string(sn.ERR_CAPACITY) == "capacity exceeded"
    p = sn.default_params()
    assert list(p.bg) == [1.0, 1.0, 1.0] and p.kappa_n == pytest.approx(1 / 64)
    assert (p.delta2, p.delta3, p.base_tile, p.relax_iters) == (2.2, 3.0, 16, 2)
    assert p.tau_merge < p.tau_split


def test_wait_limit(sn):
    """The bound of the tensor-core waits: default one second, settable,
    bounded above; rejected values leave it unchanged."""
    assert sn.wait_limit() == 10 ** 9
    L = sn.lib()
    try:
        sn.set_wait_limit(0)
        assert sn.wait_limit() == 0
        assert L.star_nt_set_wait_limit(60 * 10 ** 9 + 1) == sn.ERR_ARG
        assert sn.wait_limit() == 0
        sn.set_wait_limit(5 * 10 ** 8)
        assert sn.wait_limit() == 5 * 10 ** 8
    finally:
        sn.set_wait_limit(10 ** 9)


def test_workspace_sizes(sn):
    L = sn.lib()
    n = ctypes.c_size_t()
    assert L.star_nt_bins_bytes(1920, 1080, 20000, 1 << 20, ctypes.byref(n)) == sn.OK
    a = n.value
    assert L.star_nt_bins_bytes(1920, 1080, 20000, 2 << 20, ctypes.byref(n)) == sn.OK
    # per pair: the pair list (4 B) and the count launch's record of it (8 B + 4 B rank)
    assert n.value - a == 16 << 20
    assert L.star_nt_bins_bytes(0, 1080, 10, 10, ctypes.byref(n)) == sn.ERR_ARG
    assert L.star_nt_bins_bytes(100, 100, 10, 10, None) == sn.ERR_ARG
    assert sn.quadtree_ws_bytes(1920, 1080, 16) >= 2 * 120 * 68 * 4
    assert L.star_nt_quadtree_ws_bytes(1920, 1080, 32, ctypes.byref(n)) == sn.ERR_ARG


def test_bad_arguments_rejected_before_launch(sn):
    L = sn.lib()
    # null / inconsistent structures: rejected on the host
    assert L.star_nt_raster(None, None, None, None, None, None) == sn.ERR_ARG
    sc = sn.Scene(16, 16, 5)
    tgt = sn.Target(64, 64, 64, 64)
    bins = sn.Bins(256, 10, 64, 64, 4, 100)        # too small a workspace, too few triangles
    assert L.star_nt_raster(ctypes.byref(sc), ctypes.byref(tgt), ctypes.byref(bins), None, None, None) == sn.ERR_ARG
    w = sn.Mlp(16, 16, 16, 16, 16, 16)
    assert L.star_nt_infer(ctypes.byref(w), 7, 16, 16, 10, None, None) == sn.ERR_ARG     # bad dtype
    assert L.star_nt_infer(ctypes.byref(w), sn.F32, 8, 16, 10, None, None) == sn.ERR_ARG  # misaligned
    assert L.star_nt_infer(ctypes.byref(w), sn.BF16, 16, 16, 10, None, None) == sn.ERR_ARG  # not 256-aligned
    assert L.star_nt_composite(16, 16, -1, 16, 16, None) == sn.ERR_ARG
    assert L.star_nt_reproject(16, 16, 16, 16, 0, 10, 32, None, 48, None) == sn.ERR_ARG
    assert L.star_nt_reproject(16, 16, 16, 16, 10, 10, 16, None, 48, None) == sn.ERR_ARG  # in place
    assert L.star_nt_reproject(16, 16, 16, 16, 10, 10, 32, None, None, None) == sn.ERR_ARG  # no scratch
    p = sn.default_params()
    assert L.star_nt_quadtree(16, 16, 64, 64, ctypes.byref(p), 16, 16, 16, 256, 16, None) == sn.ERR_ARG  # small ws
    assert L.star_nt_quadtree(16, 16, 64, 64, ctypes.byref(p), 16, 16, 16, 272, 1 << 20, None) == sn.ERR_ARG  # ws alignment
    p.tau_merge = p.tau_split + 1.0
    assert L.star_nt_quadtree(16, 16, 64, 64, ctypes.byref(p), 16, 32, 16, 256, 1 << 20, None) == sn.ERR_ARG


@pytest.mark.parametrize("W,H,d2,d3,B", [(1920, 1080, 2.2, 3.0, 16), (3840, 2160, 2.2, 3.0, 64),
                                         (333, 197, 1.7, 2.6, 16), (96, 64, 0.0, 5.0, 64)])
def test_leaf_plan_matches_oracle_sizes(sn, orc, W, H, d2, d3, B):
    """The per-leaf plan (host code of the library) lists every (pass, level)
    size the oracle's Eq. 2 gives, each distinct size once, full size first."""
    p = sn.default_params(delta2=d2, delta3=d3, base_tile=B)
    plan = sn.leaf_plan(W, H, p)
    sizes = plan.sizes()
    assert sizes[0] == (W, H) and len(set(sizes)) == len(sizes) == plan.n_targets
    ref = orc.leaf_sizes(W, H, d2, d3)
    for q in (2, 3):
        for l, k in enumerate(plan.targets(q)):
            assert sizes[k] == ref[(q, l)]
    assert set(sizes) == {(W, H)} | set(ref.values())
    assert sn.leaf_ws_bytes(plan) % 256 == 0


def test_leaf_arguments_rejected(sn):
    L = sn.lib()
    p = sn.default_params(base_tile=32)
    plan = sn.LeafPlan()
    assert L.star_nt_leaf_plan_make(64, 64, ctypes.byref(p), ctypes.byref(plan)) == sn.ERR_ARG
    plan = sn.leaf_plan(64, 64, sn.default_params())
    n = ctypes.c_size_t()
    bad = sn.LeafPlan.from_buffer_copy(plan)
    bad.size[1][0] = 15                      # below a quarter of the width
    assert L.star_nt_leaf_ws_bytes(ctypes.byref(bad), ctypes.byref(n)) == sn.ERR_ARG
    bad = sn.LeafPlan.from_buffer_copy(plan)
    bad.target_of[1][2] = bad.n_targets      # unlisted target
    assert L.star_nt_leaf_ws_bytes(ctypes.byref(bad), ctypes.byref(n)) == sn.ERR_ARG
    sc = sn.Scene(16, 16, 5)
    assert L.star_nt_geometry_passes_leaf(ctypes.byref(sc), ctypes.byref(plan), None, None, 16, 256, 1 << 20,
                                          None, None, None) == sn.ERR_ARG
    assert L.star_nt_resolve_leaf(ctypes.byref(sc), ctypes.byref(plan), None, 16, None, None, 1, None, None,
                                  None, None) == sn.ERR_ARG


def test_pass_launch_resolve_arguments_rejected(sn):
    L = sn.lib()
    sc = sn.Scene(16, 16, 5)
    bins = sn.Bins(256, 1 << 20, 64, 64, 16, 1 << 10)
    lay = sn.Layers(16, 16, 16, 16, 16, 16)
    p = sn.default_params()
    w = sn.Mlp(16, 16, 16, 16, 16, 16)
    # no frame output, a misaligned frame, missing weights, the same workspace twice
    assert L.star_nt_geometry_passes_resolve(ctypes.byref(sc), ctypes.byref(bins), ctypes.byref(bins),
                                             ctypes.byref(bins), ctypes.byref(lay), ctypes.byref(lay),
                                             ctypes.byref(lay), ctypes.byref(p), ctypes.byref(w), None,
                                             None, None, None, None) == sn.ERR_ARG
    b2 = sn.Bins(512, 1 << 20, 64, 64, 16, 1 << 10)
    b3 = sn.Bins(768, 1 << 20, 64, 64, 16, 1 << 10)
    assert L.star_nt_geometry_passes_resolve(ctypes.byref(sc), ctypes.byref(bins), ctypes.byref(b2),
                                             ctypes.byref(b3), ctypes.byref(lay), ctypes.byref(lay),
                                             ctypes.byref(lay), ctypes.byref(p), ctypes.byref(w), 24,
                                             None, None, None, None) == sn.ERR_ARG
    w0 = sn.Mlp(16, None, 16, 16, 16, 16)
    assert L.star_nt_geometry_passes_resolve(ctypes.byref(sc), ctypes.byref(bins), ctypes.byref(b2),
                                             ctypes.byref(b3), ctypes.byref(lay), ctypes.byref(lay),
                                             ctypes.byref(lay), ctypes.byref(p), ctypes.byref(w0), 32,
                                             None, None, None, None) == sn.ERR_ARG
    assert L.star_nt_geometry_passes_resolve(ctypes.byref(sc), ctypes.byref(bins), ctypes.byref(bins),
                                             ctypes.byref(b3), ctypes.byref(lay), ctypes.byref(lay),
                                             ctypes.byref(lay), ctypes.byref(p), ctypes.byref(w), 32,
                                             None, None, None, None) == sn.ERR_ARG
    # block width 4, 8 or 16; one or two pixels per thread; at most 8 (one
    # pixel) or 10 (two) CTAs per SM
    for bad in (sn.Tuning(5, 0, 0), sn.Tuning(8, 0, 3), sn.Tuning(8, 9, 1), sn.Tuning(8, 11, 2),
                sn.Tuning(8, -1, 2)):
        assert L.star_nt_geometry_passes_resolve(ctypes.byref(sc), ctypes.byref(bins), ctypes.byref(b2),
                                                 ctypes.byref(b3), ctypes.byref(lay), ctypes.byref(lay),
                                                 ctypes.byref(lay), ctypes.byref(p), ctypes.byref(w), 32,
                                                 None, ctypes.byref(bad), None, None) == sn.ERR_ARG
        assert L.star_nt_geometry_passes(ctypes.byref(sc), ctypes.byref(bins), ctypes.byref(b2),
                                         ctypes.byref(b3), ctypes.byref(lay), ctypes.byref(lay),
                                         ctypes.byref(lay), ctypes.byref(bad), None, None) == sn.ERR_ARG


def test_leaf_passes_workspace_checked(sn):
    L = sn.lib()
    plan = sn.leaf_plan(64, 64, sn.default_params())
    need = sn.leaf_ws_bytes(plan)
    sc = sn.Scene(16, 16, 5)
    bins = (sn.Bins * plan.n_targets)()
    lays = (sn.Layers * plan.n_targets)()
    # a workspace one byte short, then a misaligned one
    assert L.star_nt_geometry_passes_leaf(ctypes.byref(sc), ctypes.byref(plan), bins, lays, 16, 256,
                                          need - 1, None, None, None) == sn.ERR_ARG
    assert L.star_nt_geometry_passes_leaf(ctypes.byref(sc), ctypes.byref(plan), bins, lays, 16, 272,
                                          need, None, None, None) == sn.ERR_ARG


def test_resolve_entry_points_reject_bad_arguments(sn):
    """The three resolve variants (bf16, e4m3, compensated e4m3) share their
    argument checks; the per-leaf resolve takes only the listed MLP types."""
    L = sn.lib()
    sc = sn.Scene(16, 16, 5)
    bins = sn.Bins(256, 1 << 20, 64, 64, 16, 1 << 10)
    lay = sn.Layers(16, 16, 16, 16, 16, 16)
    p = sn.default_params()
    w = sn.Mlp(16, 16, 16, 16, 16, 16)
    w0 = sn.Mlp(16, 16, 16, None, 16, 16)
    for fn in (L.star_nt_resolve, L.star_nt_resolve_fp8, L.star_nt_resolve_fp8x2):
        args = [ctypes.byref(sc), ctypes.byref(bins), ctypes.byref(bins), ctypes.byref(lay),
                ctypes.byref(lay), ctypes.byref(lay), 64, 64, ctypes.byref(p)]
        assert fn(*args, ctypes.byref(w), None, None, None, None) == sn.ERR_ARG       # no output
        assert fn(*args, ctypes.byref(w0), 32, None, None, None) == sn.ERR_ARG        # missing b2
        assert fn(*args, ctypes.byref(w), 24, None, None, None) == sn.ERR_ARG         # misaligned
        args[6] = 0
        assert fn(*args, ctypes.byref(w), 32, None, None, None) == sn.ERR_ARG         # empty frame
    plan = sn.leaf_plan(64, 64, sn.default_params())
    for t in (sn.F32, sn.E4M3X2 + 1):
        assert L.star_nt_resolve_leaf(ctypes.byref(sc), ctypes.byref(plan), ctypes.byref(lay), 16,
                                      ctypes.byref(p), ctypes.byref(w), t, 32, None, None,
                                      None) == sn.ERR_ARG


def test_context_calls_reject_bad_arguments(sn):
    """The context calls check their arguments on the host; without a CUDA
    device star_nt_create reports STAR_NT_ERR_CUDA and allocates nothing."""
    import torch
    L = sn.lib()
    h = ctypes.c_void_p()
    assert L.star_nt_create(0, None, None, None) == sn.ERR_ARG
    bad = sn.FrameOptions(7, 1.0, 1.0, 1)
    assert L.star_nt_create(0, None, ctypes.byref(bad), ctypes.byref(h)) == sn.ERR_ARG
    bad = sn.FrameOptions(sn.BF16, 0.0, 1.0, 1)
    assert L.star_nt_create(0, None, ctypes.byref(bad), ctypes.byref(h)) == sn.ERR_ARG
    p = sn.default_params(base_tile=32)
    assert L.star_nt_create(0, ctypes.byref(p), None, ctypes.byref(h)) == sn.ERR_ARG
    if not torch.cuda.is_available():
        assert L.star_nt_create(0, None, None, ctypes.byref(h)) == sn.ERR_CUDA and not h.value
    n = ctypes.c_size_t()
    assert L.star_nt_destroy(None) == sn.ERR_ARG
    assert L.star_nt_workspace_size(None, 64, 64, 10, ctypes.byref(n)) == sn.ERR_ARG
    assert L.star_nt_bind_workspace(None, 64, 64, 10, 256, 1 << 20, None) == sn.ERR_ARG
    assert L.star_nt_frame(None, None, None, None, None, None, None) == sn.ERR_ARG
    assert L.star_nt_tune(None, None, None, None, None, None, None, None) == sn.ERR_ARG
    assert L.star_nt_ctx_tuning(None, None, None) == sn.ERR_ARG
    o = sn.FrameOptions()
    L.star_nt_default_frame_options(ctypes.byref(o))
    assert (o.mlp_type, o.merge_scale2, o.merge_scale3, o.fuse_passes) == (sn.BF16, 1.0, 1.0, 1)


def test_training_arguments_rejected(sn):
    """The minibatch gather and the backward pass reject bad arguments on the
    host (fake device addresses: nothing is dereferenced or launched); an
    empty gather returns at once."""
    L = sn.lib()
    g = L.star_nt_gather_rows
    assert g(None, 10, 16, 4096, 10, 8192, None, None) == sn.ERR_ARG          # no source
    assert g(4096, 10, 6, 4096, 10, 8192, None, None) == sn.ERR_ARG           # row not whole words
    assert g(4098, 10, 16, 4096, 10, 8192, None, None) == sn.ERR_ARG          # source misaligned
    assert g(4096, 10, 16, 4100, 10, 8192, None, None) == sn.ERR_ARG          # indices misaligned
    assert g(4096, 0, 16, 4096, 10, 8192, None, None) == sn.ERR_ARG           # empty source
    assert g(4096, 10, 16, 4096, -1, 8192, None, None) == sn.ERR_ARG          # negative count
    assert g(4096, 10, 16, 4096, 0, 8192, None, None) == sn.OK                # nothing to do
    B = 100
    need = sn.train_ws_bytes(B)
    assert need > 0
    w = sn.Mlp(*([4096] * 6))
    bwd = L.star_nt_mlp_backward
    assert bwd(None, 4096, 8192, B, 12288, 16384, need, None, None) == sn.ERR_ARG        # no weights
    assert bwd(ctypes.byref(w), 4096, 8192, B, 12288, 16384, need - 4, None, None) == sn.ERR_ARG  # small ws
    assert bwd(ctypes.byref(w), 4100, 8192, B, 12288, 16384, need, None, None) == sn.ERR_ARG  # x misaligned
    assert bwd(ctypes.byref(w), 4096, 8192, B, 12288, 16400, need, None, None) == sn.ERR_ARG  # ws misaligned
    assert L.star_nt_dfaoit_backward(ctypes.byref(w), 4096, 8192, 0, 12288, 16384, need, None,
                                     None) == sn.ERR_ARG                                      # empty batch
