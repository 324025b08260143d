"""ctypes binding of libstar_nt.so (the C ABI in include/star_nt.h).

Argument marshalling only: every step of the frame runs in the library's
CUDA kernels.  Tensors are torch CUDA tensors; their device pointers are
passed as plain addresses together with the current CUDA stream.  There is
no fallback: if the library is missing or a call fails, an exception is
raised.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libstar_nt.so")

OK, ERR_ARG, ERR_CAPACITY, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED = range(6)
F32, BF16, E4M3, E4M3X2, E4M3_TENSOR, E4M3X2_TENSOR = 0, 1, 2, 3, 4, 5
LEAF_MAX_TARGETS = 9

# every entry point declared in include/star_nt.h
EXPORTS = ("star_nt_version", "star_nt_status_string", "star_nt_default_params",
           "star_nt_bins_bytes", "star_nt_raster", "star_nt_build_inputs", "star_nt_infer",
           "star_nt_composite", "star_nt_quadtree_ws_bytes", "star_nt_quadtree",
           "star_nt_reproject", "star_nt_geometry_pass", "star_nt_upscale_features",
           "star_nt_geometry_pass_merged", "star_nt_abuffer", "star_nt_train_ws_bytes",
           "star_nt_mse_grad", "star_nt_mlp_backward", "star_nt_adam", "star_nt_raster_passes",
           "star_nt_resolve", "star_nt_geometry_passes", "star_nt_resolve_fp8", "star_nt_preload",
           "star_nt_unsorted_over", "star_nt_wboit", "star_nt_wmse_grad", "star_nt_leaf_plan_make",
           "star_nt_leaf_ws_bytes", "star_nt_geometry_passes_leaf", "star_nt_resolve_leaf",
           "star_nt_geometry_passes_resolve", "star_nt_resolve_fp8x2", "star_nt_set_wait_limit",
           "star_nt_wait_limit", "star_nt_default_frame_options", "star_nt_create", "star_nt_destroy",
           "star_nt_workspace_size", "star_nt_bind_workspace", "star_nt_frame", "star_nt_tune",
           "star_nt_ctx_tuning", "star_nt_ctx_set_tuning", "star_nt_ctx_pass_state", "star_nt_resolve_mlp",
           "star_nt_build_inputs_dfaoit", "star_nt_infer_dfaoit", "star_nt_dfaoit_backward",
           "star_nt_gather_rows")

_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64


class Scene(ctypes.Structure):
    _fields_ = [("verts", _P), ("rgba8", _P), ("n_tris", _I32)]


class Target(ctypes.Structure):
    _fields_ = [("view_proj", _P), ("size", _P), ("max_w", _I32), ("max_h", _I32), ("merge_at", _P),
                ("merge_scale", ctypes.c_float)]


class Params(ctypes.Structure):
    _fields_ = [("bg", ctypes.c_float * 3), ("kappa_n", ctypes.c_float),
                ("tau_split", ctypes.c_double), ("tau_merge", ctypes.c_double),
                ("delta2", ctypes.c_double), ("delta3", ctypes.c_double),
                ("base_tile", _I32), ("relax_iters", _I32)]


class Bins(ctypes.Structure):
    _fields_ = [("mem", _P), ("bytes", ctypes.c_size_t), ("max_w", _I32), ("max_h", _I32),
                ("max_tris", _I32), ("pair_capacity", _I64)]


class Frags(ctypes.Structure):
    _fields_ = [("count", _P), ("offset", _P), ("z", _P), ("prim", _P), ("capacity", _I64),
                ("total", _P)]


class Layers(ctypes.Structure):
    _fields_ = [("id1", _P), ("z1", _P), ("id2", _P), ("n", _P), ("tail", _P), ("t_tail", _P)]


class Features(ctypes.Structure):
    _fields_ = [("x", _P), ("x_dtype", _I32), ("front", _P)]


class Mlp(ctypes.Structure):
    _fields_ = [("w1", _P), ("b1", _P), ("w2", _P), ("b2", _P), ("w3", _P), ("b3", _P)]


class Tuning(ctypes.Structure):
    _fields_ = [("block_w", _I32), ("ctas_per_sm", _I32), ("pixels_per_thread", _I32)]


class LeafPlan(ctypes.Structure):
    _fields_ = [("W", _I32), ("H", _I32), ("base_tile", _I32), ("n_targets", _I32),
                ("size", (_I32 * 2) * LEAF_MAX_TARGETS), ("target_of", (_I32 * 4) * 2)]

    def sizes(self):
        return [(self.size[k][0], self.size[k][1]) for k in range(self.n_targets)]

    def targets(self, p):
        """Target index of pass p (2 or 3) at levels 0..3."""
        return [self.target_of[p - 2][l] for l in range(4)]


class PassState(ctypes.Structure):
    _fields_ = [("W", _I32), ("H", _I32), ("W2", _I32), ("H2", _I32), ("W3", _I32), ("H3", _I32),
                ("s2", ctypes.c_float), ("s3", ctypes.c_float), ("wbar", ctypes.c_double),
                ("hist", ctypes.c_uint32 * 4)]


PASS_STATE_BYTES = ctypes.sizeof(PassState)


class FrameOptions(ctypes.Structure):
    _fields_ = [("mlp_type", _I32), ("merge_scale2", ctypes.c_float), ("merge_scale3", ctypes.c_float),
                ("fuse_passes", _I32)]


class Cameras(ctypes.Structure):
    _fields_ = [("vp", _P), ("vp64", _P), ("vp64_interp", _P)]


class FrameOut(ctypes.Structure):
    _fields_ = [("rgba32f", _P), ("rgba8", _P), ("interp_rgba32f", _P), ("interp_rgba8", _P)]


TUNE_CANDIDATES = 9


class TuneReport(ctypes.Structure):
    _fields_ = [("candidates", Tuning * TUNE_CANDIDATES), ("passes_ms", ctypes.c_float * TUNE_CANDIDATES),
                ("frame_ms", ctypes.c_float * 2), ("chosen", Tuning), ("fuse_passes", _I32),
                ("frame_merged", _I32)]

_lib = None


class StarNTError(RuntimeError):
    def __init__(self, call, status):
        self.status = status
        super().__init__(f"{call} failed: {status_string(status)} ({status})")


def lib():
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() "
                               "(or python paper_2606_16747_b300/build.py)")
        L = ctypes.CDLL(LIB_PATH)
        L.star_nt_version.restype = _I32
        L.star_nt_status_string.restype = ctypes.c_char_p
        L.star_nt_status_string.argtypes = [_I32]
        L.star_nt_default_params.argtypes = [ctypes.POINTER(Params)]
        L.star_nt_bins_bytes.argtypes = [_I32, _I32, _I32, _I64, ctypes.POINTER(ctypes.c_size_t)]
        L.star_nt_raster.argtypes = [ctypes.POINTER(Scene), ctypes.POINTER(Target),
                                     ctypes.POINTER(Bins), ctypes.POINTER(Frags), _P, _P]
        L.star_nt_raster_passes.argtypes = [ctypes.POINTER(Scene), _I32, ctypes.POINTER(Target),
                                            ctypes.POINTER(Bins), _P, _P]
        L.star_nt_build_inputs.argtypes = [ctypes.POINTER(Scene)] + [ctypes.POINTER(Bins)] * 3 + \
            [ctypes.POINTER(Layers)] * 3 + [_I32, _I32, ctypes.POINTER(Params),
                                            ctypes.POINTER(Features), _P, _P]
        L.star_nt_geometry_pass.argtypes = [ctypes.POINTER(Scene), ctypes.POINTER(Bins), _I32,
                                            ctypes.POINTER(Layers), _P, _P]
        L.star_nt_geometry_pass_merged.argtypes = [ctypes.POINTER(Scene)] + [ctypes.POINTER(Bins)] * 3 + \
            [ctypes.POINTER(Layers)] * 3 + [_P, _P]
        L.star_nt_geometry_passes.argtypes = [ctypes.POINTER(Scene)] + [ctypes.POINTER(Bins)] * 3 + \
            [ctypes.POINTER(Layers)] * 3 + [ctypes.POINTER(Tuning), _P, _P]
        L.star_nt_geometry_passes_resolve.argtypes = [ctypes.POINTER(Scene)] + [ctypes.POINTER(Bins)] * 3 + \
            [ctypes.POINTER(Layers)] * 3 + [ctypes.POINTER(Params), ctypes.POINTER(Mlp), _P, _P,
                                            ctypes.POINTER(Tuning), _P, _P]
        L.star_nt_upscale_features.argtypes = [ctypes.POINTER(Scene)] + [ctypes.POINTER(Bins)] * 2 + \
            [ctypes.POINTER(Layers)] * 3 + [_I32, _I32, ctypes.POINTER(Params),
                                            ctypes.POINTER(Features), _P]
        L.star_nt_resolve.argtypes = [ctypes.POINTER(Scene)] + [ctypes.POINTER(Bins)] * 2 + \
            [ctypes.POINTER(Layers)] * 3 + [_I32, _I32, ctypes.POINTER(Params), ctypes.POINTER(Mlp),
                                            _P, _P, _P, _P]
        L.star_nt_resolve_fp8.argtypes = L.star_nt_resolve.argtypes
        L.star_nt_resolve_fp8x2.argtypes = L.star_nt_resolve.argtypes
        L.star_nt_resolve_mlp.argtypes = [ctypes.POINTER(Scene)] + [ctypes.POINTER(Bins)] * 2 + \
            [ctypes.POINTER(Layers)] * 3 + [_I32, _I32, ctypes.POINTER(Params), ctypes.POINTER(Mlp), _I32,
                                            _P, _P, _P, _P]
        L.star_nt_infer.argtypes = [ctypes.POINTER(Mlp), _I32, _P, _P, _I64, _P, _P]
        L.star_nt_composite.argtypes = [_P, _P, _I64, _P, _P, _P]
        L.star_nt_quadtree_ws_bytes.argtypes = [_I32, _I32, _I32, ctypes.POINTER(ctypes.c_size_t)]
        L.star_nt_quadtree.argtypes = [_P, _P, _I32, _I32, ctypes.POINTER(Params), _P, _P, _P, _P,
                                       ctypes.c_size_t, _P]
        L.star_nt_reproject.argtypes = [_P, _P, _P, _P, _I32, _I32, _P, _P, _P, _P]
        L.star_nt_abuffer.argtypes = [ctypes.POINTER(Frags), _P, _I32, _I32, _P, _P, _P, _P]
        L.star_nt_unsorted_over.argtypes = [ctypes.POINTER(Frags), _P, _I32, _I32, _P, _P, _P]
        L.star_nt_wboit.argtypes = [ctypes.POINTER(Bins), ctypes.c_float, ctypes.c_float, _P, _P, _P, _P]
        L.star_nt_leaf_plan_make.argtypes = [_I32, _I32, ctypes.POINTER(Params), ctypes.POINTER(LeafPlan)]
        L.star_nt_leaf_ws_bytes.argtypes = [ctypes.POINTER(LeafPlan), ctypes.POINTER(ctypes.c_size_t)]
        L.star_nt_geometry_passes_leaf.argtypes = [ctypes.POINTER(Scene), ctypes.POINTER(LeafPlan),
                                                   ctypes.POINTER(Bins), ctypes.POINTER(Layers), _P, _P,
                                                   ctypes.c_size_t, ctypes.POINTER(Tuning), _P, _P]
        L.star_nt_resolve_leaf.argtypes = [ctypes.POINTER(Scene), ctypes.POINTER(LeafPlan),
                                           ctypes.POINTER(Layers), _P, ctypes.POINTER(Params),
                                           ctypes.POINTER(Mlp), _I32, _P, _P, _P, _P]
        L.star_nt_train_ws_bytes.argtypes = [_I64]
        L.star_nt_train_ws_bytes.restype = ctypes.c_size_t
        L.star_nt_mse_grad.argtypes = [_P, _P, _I64, _P, _P, _P, ctypes.c_size_t, _P]
        L.star_nt_wmse_grad.argtypes = [_P, _P, _P, _I64, _P, _P, _P, ctypes.c_size_t, _P]
        L.star_nt_mlp_backward.argtypes = [ctypes.POINTER(Mlp), _P, _P, _I64, _P, _P, ctypes.c_size_t, _P, _P]
        L.star_nt_adam.argtypes = [_P, _P, _P, _P, _I64, _I64, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_float, ctypes.c_float, _P, _P]
        L.star_nt_gather_rows.argtypes = [_P, _I64, _I32, _P, _I64, _P, _P, _P]
        L.star_nt_default_frame_options.argtypes = [ctypes.POINTER(FrameOptions)]
        L.star_nt_default_frame_options.restype = None
        L.star_nt_create.argtypes = [_I32, ctypes.POINTER(Params), ctypes.POINTER(FrameOptions),
                                     ctypes.POINTER(_P)]
        L.star_nt_destroy.argtypes = [_P]
        L.star_nt_workspace_size.argtypes = [_P, _I32, _I32, _I32, ctypes.POINTER(ctypes.c_size_t)]
        L.star_nt_bind_workspace.argtypes = [_P, _I32, _I32, _I32, _P, ctypes.c_size_t, _P]
        L.star_nt_frame.argtypes = [_P, ctypes.POINTER(Scene), ctypes.POINTER(Mlp), ctypes.POINTER(Cameras),
                                    ctypes.POINTER(FrameOut), _P, _P]
        L.star_nt_tune.argtypes = L.star_nt_frame.argtypes + [ctypes.POINTER(TuneReport)]
        L.star_nt_ctx_tuning.argtypes = [_P, ctypes.POINTER(Tuning), ctypes.POINTER(_I32)]
        L.star_nt_ctx_set_tuning.argtypes = [_P, ctypes.POINTER(Tuning), _I32]
        L.star_nt_ctx_pass_state.argtypes = [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                             ctypes.POINTER(_P)]
        L.star_nt_build_inputs_dfaoit.argtypes = [ctypes.POINTER(Scene), ctypes.POINTER(Bins),
                                                  ctypes.POINTER(Layers), _I32, _I32, ctypes.POINTER(Params),
                                                  ctypes.POINTER(Features), _P, _P]
        L.star_nt_infer_dfaoit.argtypes = [ctypes.POINTER(Mlp), _I32, _P, _P, _I64, _P, _P]
        L.star_nt_dfaoit_backward.argtypes = [ctypes.POINTER(Mlp), _P, _P, _I64, _P, _P, ctypes.c_size_t, _P, _P]
        L.star_nt_set_wait_limit.argtypes = [ctypes.c_uint64]
        L.star_nt_wait_limit.restype = ctypes.c_uint64
        for name in EXPORTS:
            if name not in ("star_nt_default_params", "star_nt_status_string", "star_nt_version",
                            "star_nt_train_ws_bytes", "star_nt_wait_limit",
                            "star_nt_default_frame_options"):
                getattr(L, name).restype = _I32
        _lib = L
    return _lib


def status_string(s: int) -> str:
    return lib().star_nt_status_string(int(s)).decode()


def _check(call, s):
    if s != OK:
        raise StarNTError(call, s)


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def set_wait_limit(ns: int):
    """Bound, in nanoseconds, of the tensor-core kernels' waits (process-wide;
    0 makes them run out at once)."""
    _check("star_nt_set_wait_limit", lib().star_nt_set_wait_limit(int(ns)))


def wait_limit() -> int:
    return int(lib().star_nt_wait_limit())


def default_params(**kw) -> Params:
    p = Params()
    lib().star_nt_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "bg":
            p.bg = (ctypes.c_float * 3)(*v)
        else:
            setattr(p, k, v)
    return p


class BinsBuffer:
    """Device workspace of one pass's binned triangles."""

    def __init__(self, max_w, max_h, max_tris, pair_capacity, device="cuda"):
        n = ctypes.c_size_t()
        _check("star_nt_bins_bytes", lib().star_nt_bins_bytes(max_w, max_h, max_tris, pair_capacity,
                                                              ctypes.byref(n)))
        self.mem = torch.zeros(n.value, dtype=torch.uint8, device=device)  # zero before first use
        self.c = Bins(self.mem.data_ptr(), n.value, max_w, max_h, max_tris, pair_capacity)

    def header(self):
        """size[2], tiles_x, tiles_y, n_tiles, n_pixels, n_pairs, n_tris (device int32 view)."""
        return self.mem[:32].view(torch.int32)


_preloaded = set()


def preload(device=None):
    """Load every kernel onto the device (once per device), before any frame
    is captured."""
    d = torch.cuda.current_device() if device is None else int(device)
    if d in _preloaded:
        return
    with torch.cuda.device(d):
        _check("star_nt_preload", lib().star_nt_preload())
    _preloaded.add(d)


def scene_struct(verts, rgba8) -> Scene:
    return Scene(verts.data_ptr(), rgba8.data_ptr(), int(rgba8.shape[0]))


def raster(scene: Scene, vp, size, max_w, max_h, bins: BinsBuffer, frags=None, status=None, stream=None,
           merge_at=None, merge_scale=1.0):
    tgt = Target(vp.data_ptr(), size.data_ptr(), max_w, max_h,
                 merge_at.data_ptr() if merge_at is not None else None, float(merge_scale))
    fr = None
    if frags is not None:
        fr = Frags(frags["count"].data_ptr(), frags["offset"].data_ptr(), frags["z"].data_ptr(),
                   frags["prim"].data_ptr(), int(frags["z"].numel()), frags["total"].data_ptr())
    _check("star_nt_raster", lib().star_nt_raster(ctypes.byref(scene), ctypes.byref(tgt),
                                                  ctypes.byref(bins.c),
                                                  ctypes.byref(fr) if fr is not None else None,
                                                  _ptr(status), _stream(stream)))


def raster_passes(scene: Scene, passes, status=None, stream=None):
    """passes: list of (vp, size, max_w, max_h, bins, merge_at or None[, merge_scale])."""
    n = len(passes)
    tgts = (Target * n)(*[Target(p[0].data_ptr(), p[1].data_ptr(), p[2], p[3],
                                 p[5].data_ptr() if p[5] is not None else None,
                                 float(p[6]) if len(p) > 6 else 1.0)
                          for p in passes])
    bins = (Bins * n)(*[p[4].c for p in passes])
    _check("star_nt_raster_passes", lib().star_nt_raster_passes(ctypes.byref(scene), n, tgts, bins,
                                                                _ptr(status), _stream(stream)))


def layers_struct(d) -> Layers:
    if d is None:
        return None
    g = lambda k: d[k].data_ptr() if d.get(k) is not None else None
    return Layers(g("id1"), g("z1"), g("id2"), g("n"), g("tail"), g("t_tail"))


def build_inputs(scene: Scene, bins1, bins2, bins3, layers1, layers2, layers3, W, H, params: Params,
                 x, x_dtype, front, status=None, stream=None):
    ls = [layers_struct(l) for l in (layers1, layers2, layers3)]
    feat = Features(x.data_ptr(), x_dtype, front.data_ptr())
    _check("star_nt_build_inputs", lib().star_nt_build_inputs(
        ctypes.byref(scene), ctypes.byref(bins1.c), ctypes.byref(bins2.c), ctypes.byref(bins3.c),
        *[ctypes.byref(l) if l is not None else None for l in ls], W, H, ctypes.byref(params),
        ctypes.byref(feat), _ptr(status), _stream(stream)))


def geometry_pass(scene: Scene, bins, mode, layers, status=None, stream=None):
    l = layers_struct(layers)
    _check("star_nt_geometry_pass", lib().star_nt_geometry_pass(ctypes.byref(scene), ctypes.byref(bins.c),
                                                                mode, ctypes.byref(l), _ptr(status),
                                                                _stream(stream)))


def geometry_pass_merged(scene: Scene, bins1, bins2, bins3, layers1, layers2, layers3, status=None,
                         stream=None):
    ls = [layers_struct(l) for l in (layers1, layers2, layers3)]
    _check("star_nt_geometry_pass_merged", lib().star_nt_geometry_pass_merged(
        ctypes.byref(scene), ctypes.byref(bins1.c), ctypes.byref(bins2.c), ctypes.byref(bins3.c),
        *[ctypes.byref(l) for l in ls], _ptr(status), _stream(stream)))


def geometry_passes(scene: Scene, bins1, bins2, bins3, layers1, layers2, layers3, tuning=None,
                    status=None, stream=None):
    ls = [layers_struct(l) for l in (layers1, layers2, layers3)]
    t = Tuning(*tuning) if tuning is not None else None
    _check("star_nt_geometry_passes", lib().star_nt_geometry_passes(
        ctypes.byref(scene), ctypes.byref(bins1.c), ctypes.byref(bins2.c), ctypes.byref(bins3.c),
        *[ctypes.byref(l) for l in ls], ctypes.byref(t) if t is not None else None, _ptr(status),
        _stream(stream)))


def geometry_passes_resolve(scene: Scene, bins1, bins2, bins3, layers1, layers2, layers3, params: Params,
                            w: Mlp, rgba32f=None, rgba8=None, tuning=None, status=None, stream=None):
    ls = [layers_struct(l) for l in (layers1, layers2, layers3)]
    t = Tuning(*tuning) if tuning is not None else None
    _check("star_nt_geometry_passes_resolve", lib().star_nt_geometry_passes_resolve(
        ctypes.byref(scene), ctypes.byref(bins1.c), ctypes.byref(bins2.c), ctypes.byref(bins3.c),
        *[ctypes.byref(l) for l in ls], ctypes.byref(params), ctypes.byref(w), _ptr(rgba32f), _ptr(rgba8),
        ctypes.byref(t) if t is not None else None, _ptr(status), _stream(stream)))


def upscale_features(scene: Scene, bins2, bins3, layers1, layers2, layers3, W, H, params: Params,
                     x, x_dtype, front, stream=None):
    ls = [layers_struct(l) for l in (layers1, layers2, layers3)]
    feat = Features(x.data_ptr(), x_dtype, front.data_ptr())
    _check("star_nt_upscale_features", lib().star_nt_upscale_features(
        ctypes.byref(scene), ctypes.byref(bins2.c), ctypes.byref(bins3.c),
        *[ctypes.byref(l) for l in ls], W, H, ctypes.byref(params), ctypes.byref(feat),
        _stream(stream)))


def resolve(scene: Scene, bins2, bins3, layers1, layers2, layers3, W, H, params: Params, w: Mlp,
            rgba32f=None, rgba8=None, status=None, stream=None):
    ls = [layers_struct(l) for l in (layers1, layers2, layers3)]
    _check("star_nt_resolve", lib().star_nt_resolve(
        ctypes.byref(scene), ctypes.byref(bins2.c), ctypes.byref(bins3.c), *[ctypes.byref(l) for l in ls],
        W, H, ctypes.byref(params), ctypes.byref(w), _ptr(rgba32f), _ptr(rgba8), _ptr(status),
        _stream(stream)))


def resolve_fp8(scene: Scene, bins2, bins3, layers1, layers2, layers3, W, H, params: Params, w: Mlp,
                rgba32f=None, rgba8=None, status=None, stream=None):
    ls = [layers_struct(l) for l in (layers1, layers2, layers3)]
    _check("star_nt_resolve_fp8", lib().star_nt_resolve_fp8(
        ctypes.byref(scene), ctypes.byref(bins2.c), ctypes.byref(bins3.c), *[ctypes.byref(l) for l in ls],
        W, H, ctypes.byref(params), ctypes.byref(w), _ptr(rgba32f), _ptr(rgba8), _ptr(status),
        _stream(stream)))


def resolve_fp8x2(scene: Scene, bins2, bins3, layers1, layers2, layers3, W, H, params: Params, w: Mlp,
                  rgba32f=None, rgba8=None, status=None, stream=None):
    ls = [layers_struct(l) for l in (layers1, layers2, layers3)]
    _check("star_nt_resolve_fp8x2", lib().star_nt_resolve_fp8x2(
        ctypes.byref(scene), ctypes.byref(bins2.c), ctypes.byref(bins3.c), *[ctypes.byref(l) for l in ls],
        W, H, ctypes.byref(params), ctypes.byref(w), _ptr(rgba32f), _ptr(rgba8), _ptr(status),
        _stream(stream)))


def resolve_mlp(scene: Scene, bins2, bins3, layers1, layers2, layers3, W, H, params: Params, w: Mlp, mlp_type,
                rgba32f=None, rgba8=None, status=None, stream=None):
    ls = [layers_struct(l) for l in (layers1, layers2, layers3)]
    _check("star_nt_resolve_mlp", lib().star_nt_resolve_mlp(
        ctypes.byref(scene), ctypes.byref(bins2.c), ctypes.byref(bins3.c), *[ctypes.byref(l) for l in ls],
        W, H, ctypes.byref(params), ctypes.byref(w), int(mlp_type), _ptr(rgba32f), _ptr(rgba8), _ptr(status),
        _stream(stream)))


def build_inputs_dfaoit(scene: Scene, bins, layers1, W, H, params: Params, x, x_dtype, front, status=None,
                        stream=None):
    """The DFAOIT comparison network's input x [W*H][16] and front terms."""
    feat = Features(x.data_ptr(), x_dtype, front.data_ptr())
    l = layers_struct(layers1)
    _check("star_nt_build_inputs_dfaoit", lib().star_nt_build_inputs_dfaoit(
        ctypes.byref(scene), ctypes.byref(bins.c), ctypes.byref(l) if l is not None else None, W, H,
        ctypes.byref(params), ctypes.byref(feat), _ptr(status), _stream(stream)))


def infer_dfaoit(w: Mlp, x_dtype, x, f, P, status=None, stream=None):
    _check("star_nt_infer_dfaoit", lib().star_nt_infer_dfaoit(ctypes.byref(w), x_dtype, _ptr(x), _ptr(f), int(P),
                                                              _ptr(status), _stream(stream)))


def dfaoit_backward(w: Mlp, x, dy, B, grad, ws, status=None, stream=None):
    _check("star_nt_dfaoit_backward", lib().star_nt_dfaoit_backward(ctypes.byref(w), _ptr(x), _ptr(dy), int(B),
                                                                    _ptr(grad), _ptr(ws), ws.numel(),
                                                                    _ptr(status), _stream(stream)))


def mlp_struct(w) -> Mlp:
    return Mlp(*[w[k].data_ptr() for k in ("w1", "b1", "w2", "b2", "w3", "b3")])


def infer(w: Mlp, x_dtype, x, f, P, status=None, stream=None):
    _check("star_nt_infer", lib().star_nt_infer(ctypes.byref(w), x_dtype, _ptr(x), _ptr(f), int(P),
                                                _ptr(status), _stream(stream)))


def composite(front, f, P, rgba32f=None, rgba8=None, stream=None):
    _check("star_nt_composite", lib().star_nt_composite(_ptr(front), _ptr(f), int(P), _ptr(rgba32f),
                                                        _ptr(rgba8), _stream(stream)))


def quadtree_ws_bytes(W, H, base):
    n = ctypes.c_size_t()
    _check("star_nt_quadtree_ws_bytes", lib().star_nt_quadtree_ws_bytes(W, H, base, ctypes.byref(n)))
    return n.value


def quadtree(rgba8, id1, W, H, params: Params, mask_prev, mask_out, state, ws, stream=None):
    _check("star_nt_quadtree", lib().star_nt_quadtree(_ptr(rgba8), _ptr(id1), W, H, ctypes.byref(params),
                                                      _ptr(mask_prev), _ptr(mask_out), _ptr(state),
                                                      _ptr(ws), ws.numel(), _stream(stream)))


# ---------------------------------------------------------------------------
# per-leaf pass resolution

def leaf_plan(W, H, params: Params) -> LeafPlan:
    p = LeafPlan()
    _check("star_nt_leaf_plan_make", lib().star_nt_leaf_plan_make(W, H, ctypes.byref(params), ctypes.byref(p)))
    return p


def leaf_ws_bytes(plan: LeafPlan) -> int:
    n = ctypes.c_size_t()
    _check("star_nt_leaf_ws_bytes", lib().star_nt_leaf_ws_bytes(ctypes.byref(plan), ctypes.byref(n)))
    return n.value


def _layers_array(layers):
    return (Layers * len(layers))(*[layers_struct(l) for l in layers])


def geometry_passes_leaf(scene: Scene, plan: LeafPlan, bins, layers, masks, ws, tuning=None,
                         status=None, stream=None):
    """bins, layers: one per plan target (BinsBuffer, dict of planes)."""
    b = (Bins * len(bins))(*[x.c for x in bins])
    t = Tuning(*tuning) if tuning is not None else None
    _check("star_nt_geometry_passes_leaf", lib().star_nt_geometry_passes_leaf(
        ctypes.byref(scene), ctypes.byref(plan), b, _layers_array(layers), _ptr(masks), _ptr(ws),
        ws.numel(), ctypes.byref(t) if t is not None else None, _ptr(status), _stream(stream)))


def resolve_leaf(scene: Scene, plan: LeafPlan, layers, masks, params: Params, w: Mlp, mlp_type=BF16,
                 rgba32f=None, rgba8=None, status=None, stream=None):
    _check("star_nt_resolve_leaf", lib().star_nt_resolve_leaf(
        ctypes.byref(scene), ctypes.byref(plan), _layers_array(layers), _ptr(masks),
        ctypes.byref(params), ctypes.byref(w), int(mlp_type), _ptr(rgba32f), _ptr(rgba8), _ptr(status),
        _stream(stream)))


REPROJECT_WS_BYTES = 128


def reproject(prev_rgba, prev_z1, vp_prev, vp_cur, W, H, out_rgba, ws=None, stream=None,
              out_rgba8=None):
    if ws is None:
        ws = torch.empty(REPROJECT_WS_BYTES, dtype=torch.uint8, device=prev_rgba.device)
    _check("star_nt_reproject", lib().star_nt_reproject(_ptr(prev_rgba), _ptr(prev_z1), _ptr(vp_prev),
                                                        _ptr(vp_cur), W, H, _ptr(out_rgba),
                                                        _ptr(out_rgba8), _ptr(ws), _stream(stream)))


def read_pass_state(state_tensor) -> dict:
    """Decode a device star_nt_pass_state (uint8 tensor) on the host."""
    raw = bytes(state_tensor.cpu().numpy().tobytes())
    st = PassState.from_buffer_copy(raw[:PASS_STATE_BYTES])
    return dict(W=st.W, H=st.H, W2=st.W2, H2=st.H2, W3=st.W3, H3=st.H3, s2=st.s2, s3=st.s3,
                wbar=st.wbar, hist=list(st.hist))


# ---------------------------------------------------------------------------
# exact resolve and training

def frags_struct(frags) -> Frags:
    return Frags(frags["count"].data_ptr(), frags["offset"].data_ptr(), frags["z"].data_ptr(),
                 frags["prim"].data_ptr(), int(frags["z"].numel()), frags["total"].data_ptr())


def abuffer(frags, rgba8, W, H, bg, rgb=None, tail=None, stream=None):
    f = frags_struct(frags)
    bgt = (ctypes.c_float * 3)(*bg)
    _check("star_nt_abuffer", lib().star_nt_abuffer(ctypes.byref(f), _ptr(rgba8), W, H, bgt, _ptr(rgb),
                                                    _ptr(tail), _stream(stream)))


def unsorted_over(frags, rgba8, W, H, bg, rgb, stream=None):
    f = frags_struct(frags)
    bgt = (ctypes.c_float * 3)(*bg)
    _check("star_nt_unsorted_over", lib().star_nt_unsorted_over(ctypes.byref(f), _ptr(rgba8), W, H, bgt,
                                                                _ptr(rgb), _stream(stream)))


def wboit(bins, znear, zfar, bg, rgba32f=None, rgba8=None, stream=None):
    bgt = (ctypes.c_float * 3)(*bg)
    _check("star_nt_wboit", lib().star_nt_wboit(ctypes.byref(bins.c), float(znear), float(zfar), bgt,
                                                _ptr(rgba32f), _ptr(rgba8), _stream(stream)))


def train_ws_bytes(B):
    return int(lib().star_nt_train_ws_bytes(int(B)))


def mse_grad(f, y, B, dy, loss, ws, stream=None, w=None):
    if w is None:
        _check("star_nt_mse_grad", lib().star_nt_mse_grad(_ptr(f), _ptr(y), int(B), _ptr(dy), _ptr(loss),
                                                          _ptr(ws), ws.numel(), _stream(stream)))
    else:
        _check("star_nt_wmse_grad", lib().star_nt_wmse_grad(_ptr(f), _ptr(y), _ptr(w), int(B), _ptr(dy),
                                                            _ptr(loss), _ptr(ws), ws.numel(),
                                                            _stream(stream)))


def mlp_backward(w: Mlp, x, dy, B, grad, ws, status=None, stream=None):
    _check("star_nt_mlp_backward", lib().star_nt_mlp_backward(ctypes.byref(w), _ptr(x), _ptr(dy), int(B),
                                                              _ptr(grad), _ptr(ws), ws.numel(),
                                                              _ptr(status), _stream(stream)))


def gather_rows(src, idx, dst, status=None, stream=None):
    """dst[i] = src[idx[i]] (row-major tensors with equal row sizes; idx int64)."""
    n_src = src.shape[0]
    row_bytes = src.numel() * src.element_size() // max(1, n_src)
    if dst.shape[0] != idx.numel() or dst.numel() * dst.element_size() != idx.numel() * row_bytes:
        raise ValueError("gather_rows: dst must hold idx.numel() rows of the source's size")
    _check("star_nt_gather_rows", lib().star_nt_gather_rows(_ptr(src), int(n_src), int(row_bytes), _ptr(idx),
                                                            int(idx.numel()), _ptr(dst), _ptr(status),
                                                            _stream(stream)))


def adam(params, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, bf16_rounded=None,
         stream=None):
    _check("star_nt_adam", lib().star_nt_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), params.numel(),
                                              int(step), lr, beta1, beta2, eps, _ptr(bf16_rounded),
                                              _stream(stream)))


# ---------------------------------------------------------------------------
# context: the whole step through star_nt_frame

class Context:
    """A star_nt_ctx on one device: create, bind one workspace (a torch
    allocation of star_nt_workspace_size bytes), then one call per step
    (real frame, interpolated frame, quadtree update); star_nt_tune chooses
    the launch tuning on the workload."""

    def __init__(self, device=None, params: Params = None, mlp_type=BF16, merge_scale2=1.0, merge_scale3=1.0,
                 fuse_passes=True):
        self.device = torch.cuda.current_device() if device is None else int(device)
        opt = FrameOptions()
        lib().star_nt_default_frame_options(ctypes.byref(opt))
        opt.mlp_type, opt.merge_scale2, opt.merge_scale3 = int(mlp_type), float(merge_scale2), float(merge_scale3)
        opt.fuse_passes = 1 if fuse_passes else 0
        self.params = params if params is not None else default_params()
        h = _P()
        _check("star_nt_create", lib().star_nt_create(self.device, ctypes.byref(self.params), ctypes.byref(opt),
                                                      ctypes.byref(h)))
        self.h = h
        self.ws = None

    def workspace_size(self, W, H, T) -> int:
        n = ctypes.c_size_t()
        _check("star_nt_workspace_size", lib().star_nt_workspace_size(self.h, W, H, T, ctypes.byref(n)))
        return n.value

    def bind(self, W, H, T, stream=None):
        n = self.workspace_size(W, H, T)
        self.ws = torch.empty(n, dtype=torch.uint8, device=f"cuda:{self.device}")
        _check("star_nt_bind_workspace", lib().star_nt_bind_workspace(self.h, W, H, T, self.ws.data_ptr(), n,
                                                                      _stream(stream)))
        self.W, self.H, self.T = W, H, T

    @staticmethod
    def _args(cams, out):
        c = Cameras(*[t.data_ptr() if t is not None else None for t in cams])
        o = FrameOut(*[t.data_ptr() if t is not None else None for t in out])
        return c, o

    def frame(self, scene: Scene, w: Mlp, vp, vp64, vp64_interp, rgba32f, rgba8, interp_rgba32f=None,
              interp_rgba8=None, status=None, stream=None):
        c, o = self._args((vp, vp64, vp64_interp), (rgba32f, rgba8, interp_rgba32f, interp_rgba8))
        _check("star_nt_frame", lib().star_nt_frame(self.h, ctypes.byref(scene), ctypes.byref(w), ctypes.byref(c),
                                                    ctypes.byref(o), _ptr(status), _stream(stream)))

    def tune(self, scene: Scene, w: Mlp, vp, vp64, rgba32f, rgba8, status=None, stream=None) -> dict:
        c, o = self._args((vp, vp64, None), (rgba32f, rgba8, None, None))
        r = TuneReport()
        _check("star_nt_tune", lib().star_nt_tune(self.h, ctypes.byref(scene), ctypes.byref(w), ctypes.byref(c),
                                                  ctypes.byref(o), _ptr(status), _stream(stream), ctypes.byref(r)))
        key = lambda t: f"{t.block_w}x{32 // t.block_w}/{t.ctas_per_sm}/{t.pixels_per_thread}px"
        return {"block_w": r.chosen.block_w, "ctas_per_sm": r.chosen.ctas_per_sm,
                "pixels_per_thread": r.chosen.pixels_per_thread, "fuse_passes": bool(r.fuse_passes),
                "ms": {key(r.candidates[k]): r.passes_ms[k] for k in range(TUNE_CANDIDATES)},
                "raster_passes_resolve_ms": {"pass launch resolves": r.frame_ms[1], "separate resolve": r.frame_ms[0],
                                             "frame merged": bool(r.frame_merged)}}

    def tuning(self):
        t, f = Tuning(), _I32()
        _check("star_nt_ctx_tuning", lib().star_nt_ctx_tuning(self.h, ctypes.byref(t), ctypes.byref(f)))
        return (t.block_w, t.ctas_per_sm, t.pixels_per_thread), bool(f.value)

    def set_tuning(self, tuning, fuse_passes=True):
        t = Tuning(*tuning)
        _check("star_nt_ctx_set_tuning", lib().star_nt_ctx_set_tuning(self.h, ctypes.byref(t), 1 if fuse_passes else 0))

    def views(self) -> dict:
        """The pass state, masks and nearest-layer planes inside the bound
        workspace, as tensors viewing it."""
        st, m, i1, z = _P(), _P(), _P(), _P()
        _check("star_nt_ctx_pass_state", lib().star_nt_ctx_pass_state(self.h, ctypes.byref(st), ctypes.byref(m),
                                                                      ctypes.byref(i1), ctypes.byref(z)))
        base = self.ws.data_ptr()
        P = self.W * self.H
        B = self.params.base_tile
        nt = ((self.W + B - 1) // B) * ((self.H + B - 1) // B)
        at = lambda p, n: self.ws[p.value - base:p.value - base + n]
        return {"state": at(st, PASS_STATE_BYTES), "masks": at(m, 4 * nt).view(torch.int32),
                "id1": at(i1, 4 * P).view(torch.int32), "z1": at(z, 4 * P).view(torch.float32)}

    def close(self):
        if getattr(self, "h", None):
            lib().star_nt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
