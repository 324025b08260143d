"""CPU oracle of the STAR-NT per-frame hot path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It is a thin numpy/ctypes layer over
``star_nt_oracle.c`` (float64 unless a convention fixes float32) and shares no
code with the CUDA path.  Functions mirror the paper's steps:

  raster         geometry passes: per-pixel fragment lists (Sec. 3)
  resolve        A-buffer (Eq. 1), two nearest layers, tail statistics,
                 exact tail colour and the terms of Eq. 4 (Sec. 3.3)
  upscale        bilinear upscale of reduced-resolution passes (Sec. 3.2)
  features       the five-float network input and the front terms (Sec. 3.3)
  mlp_*          the 5-32-16-3 tail-colour MLP, its MSE gradient and Adam
  composite      Eq. 4
  quadtree       adaptive screen-space tiles (Sec. 3.1) and Eq. 2
  reproject      depth-based temporal reprojection (Sec. 3.3, last paragraph)
  unsorted_over, wboit
                 the evaluation's comparison renderers (Sec. 4)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "star_nt_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

KAPPA_N = 1.0 / 64.0      # scale of the fragment-count feature
DELTA2, DELTA3 = 2.2, 3.0  # Eq. 2 offsets


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, IEEE float32/64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_D = ctypes.c_double


def _declare(L):
    L.orc_raster_count.argtypes = [_P, _I32, _P, _I32, _I32, _I32, _I32, _P]
    L.orc_raster_count.restype = _I64
    L.orc_raster_fill.argtypes = [_P, _I32, _P, _I32, _I32, _I32, _I32, _P, _P, _P, _P]
    L.orc_raster_fill.restype = _I64
    L.orc_resolve.argtypes = [_P, _P, _P, _P, _I32, _I32, _I32, _P] + [_P] * 12
    L.orc_resolve.restype = None
    L.orc_unsorted_over.argtypes = [_P, _P, _P, _I64, _P, _P]
    L.orc_wboit.argtypes = [_P, _P, _P, _P, _I64, ctypes.c_double, ctypes.c_double, _P, _P]
    L.orc_upscale.argtypes = [_P, _I32, _I32, _I32, _I32, _I32, _P]
    L.orc_tail_flag.argtypes = [_P, _I32, _I32, _I32, _I32, _P]
    L.orc_features.argtypes = [_I64, _P, _P, _P, _P, _P, _P, _P, _P, _D, _P, _P]
    L.orc_mlp_forward.argtypes = [_P, _P, _P, _I64, _P]
    L.orc_mlp_mse_grad.argtypes = [_P, _P, _P, _I64, _P]
    L.orc_mlp_mse_grad.restype = _D
    L.orc_adam.argtypes = [_P, _P, _P, _P, _I64, _I64, _D, _D, _D, _D]
    L.orc_composite.argtypes = [_P, _P, _I64, _P]
    L.orc_quantize.argtypes = [_P, _I64, _P]
    L.orc_pass_scale.argtypes = [_D, _D]
    L.orc_pass_scale.restype = _D
    L.orc_pass_size.argtypes = [_D, _I32]
    L.orc_pass_size.restype = _I32
    L.orc_quadtree.argtypes = [_P, _P, _I32, _I32, _I32, _D, _D, _I32, _P, _P, _P]
    L.orc_inverse4.argtypes = [_P, _P]
    L.orc_inverse4.restype = ctypes.c_int
    L.orc_reproject.argtypes = [_P, _P, _P, _P, _I32, _I32, _P]
    L.orc_dfaoit_features.argtypes = [_P, _P, _P, _P, _I64, _I64, _D, _P, _P]
    L.orc_dfaoit_features.restype = None
    L.orc_mlp_dfaoit_forward.argtypes = [_P, _P, _P, _I64, _P]
    L.orc_mlp_dfaoit_mse_grad.argtypes = [_P, _P, _P, _I64, _P]
    L.orc_mlp_dfaoit_mse_grad.restype = _D


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data


def _bands(H, threads):
    threads = max(1, min(int(threads), H))
    edges = np.linspace(0, H, threads + 1).astype(int)
    return [(int(edges[i]), int(edges[i + 1])) for i in range(threads) if edges[i + 1] > edges[i]]


class Frags:
    """Per-pixel fragment lists (CSR) of one geometry pass, in submission order."""

    def __init__(self, W, H, counts, offsets, z, prim):
        self.W, self.H = W, H
        self.counts, self.offsets, self.z, self.prim = counts, offsets, z, prim

    @property
    def total(self) -> int:
        return int(self.offsets[-1])


def raster(verts, vp32, W, H, threads=1) -> Frags:
    """Fragments of every triangle at every covered pixel centre of a W x H target."""
    L = lib()
    verts = _c(verts, np.float32)
    vp = _c(np.asarray(vp32).reshape(16), np.float32)
    T = verts.shape[0]
    counts = np.zeros(W * H, dtype=np.uint32)
    bands = _bands(H, threads)
    with ThreadPoolExecutor(len(bands)) as ex:
        list(ex.map(lambda b: L.orc_raster_count(_ptr(verts), T, _ptr(vp), W, H, b[0], b[1],
                                                 _ptr(counts)), bands))
    offsets = np.zeros(W * H + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    F = int(offsets[-1])
    z = np.empty(F, dtype=np.float32)
    prim = np.empty(F, dtype=np.int32)
    cursor = np.zeros(W * H, dtype=np.uint32)
    with ThreadPoolExecutor(len(bands)) as ex:
        list(ex.map(lambda b: L.orc_raster_fill(_ptr(verts), T, _ptr(vp), W, H, b[0], b[1],
                                                _ptr(offsets), _ptr(cursor), _ptr(z), _ptr(prim)),
                    bands))
    return Frags(W, H, counts, offsets, z, prim)


def resolve(fr: Frags, rgba8, bg=(1.0, 1.0, 1.0), threads=1) -> dict:
    """Sort each pixel's fragments by (z, prim) and evaluate the per-pixel terms."""
    L = lib()
    W, H, P = fr.W, fr.H, fr.W * fr.H
    rgba8 = _c(rgba8, np.uint32)
    bg = _c(bg, np.float64)
    out = dict(
        id1=np.empty(P, np.int32), z1=np.empty(P, np.float32), id2=np.empty(P, np.int32),
        n=np.empty(P, np.uint32), a_tail=np.empty(P, np.uint32), s_tail=np.empty((P, 3), np.uint32),
        t_tail=np.empty(P, np.float64), abuf=np.empty((P, 3), np.float64),
        tail_rgb=np.empty((P, 3), np.float64), front2=np.empty((P, 4), np.float64),
        layer2=np.empty((P, 4), np.float64), t_all=np.empty(P, np.float64))
    order = ["id1", "z1", "id2", "n", "a_tail", "s_tail", "t_tail", "abuf", "tail_rgb", "front2",
             "layer2", "t_all"]
    bands = _bands(H, threads)
    with ThreadPoolExecutor(len(bands)) as ex:
        list(ex.map(lambda b: L.orc_resolve(_ptr(fr.offsets), _ptr(fr.z), _ptr(fr.prim), _ptr(rgba8),
                                            W, b[0], b[1], _ptr(bg), *[_ptr(out[k]) for k in order]),
                    bands))
    return out


# ---------------------------------------------------------------------------
# The DFAOIT comparison network (Sec. 3.3): its eleven listed features, the
# 11 -> 32 -> 16 -> 3 network with a sigmoid output, and its composite
# C = C_t + C_b prod(1 - a_i).

DFAOIT_PARAMS = 963
DFAOIT_SHAPES = (("w1", (32, 11)), ("b1", (32,)), ("w2", (16, 32)), ("b2", (16,)), ("w3", (3, 16)),
                 ("b3", (3,)))


def dfaoit_features(fr: Frags, rgba8, kappa=KAPPA_N, threads=1):
    """(x [P, 11], t_all [P]) of every pixel (orc_dfaoit_features)."""
    L = lib()
    P = fr.W * fr.H
    rgba8 = _c(rgba8, np.uint32)
    x = np.empty((P, 11), np.float64)
    t_all = np.empty(P, np.float64)
    bands = _bands(fr.H, threads)
    with ThreadPoolExecutor(len(bands)) as ex:
        list(ex.map(lambda b: L.orc_dfaoit_features(_ptr(fr.offsets), _ptr(fr.z), _ptr(fr.prim), _ptr(rgba8),
                                                    b[0] * fr.W, b[1] * fr.W, float(kappa), _ptr(x),
                                                    _ptr(t_all)), bands))
    return x, t_all


def mlp_dfaoit_forward(params, x, flag=None):
    L = lib()
    params = _c(params, np.float64)
    assert params.size == DFAOIT_PARAMS
    x = _c(x, np.float64)
    n = x.shape[0]
    f = np.empty((n, 3), np.float64)
    fl = None if flag is None else _c(flag, np.uint8)
    L.orc_mlp_dfaoit_forward(_ptr(params), _ptr(x), _ptr(fl), n, _ptr(f))
    return f


def mlp_dfaoit_mse_grad(params, x, y):
    L = lib()
    params = _c(params, np.float64)
    x = _c(x, np.float64)
    y = _c(y, np.float64)
    g = np.empty(DFAOIT_PARAMS, np.float64)
    loss = L.orc_mlp_dfaoit_mse_grad(_ptr(params), _ptr(x), _ptr(y), x.shape[0], _ptr(g))
    return loss, g


def frame_dfaoit(verts, rgba8, vp32, W, H, params, bg=(1.0, 1.0, 1.0), threads=1):
    """The DFAOIT comparison frame at full resolution: features, network
    (f = 0 where a pixel has no fragment), C = f + t_all C_b."""
    fr = raster(verts, vp32, W, H, threads)
    x, t_all = dfaoit_features(fr, rgba8, threads=threads)
    flag = (fr.counts > 0).astype(np.uint8)
    f = mlp_dfaoit_forward(params, x, flag)
    rgb = f + t_all[:, None] * np.asarray(bg, np.float64)[None, :]
    return dict(x=x, t_all=t_all, flag=flag, f=f, rgb=rgb, frags=fr)


def unsorted_over(fr: Frags, rgba8, bg=(1.0, 1.0, 1.0)):
    L = lib()
    P = fr.W * fr.H
    out = np.empty((P, 3), np.float64)
    L.orc_unsorted_over(_ptr(fr.offsets), _ptr(fr.prim), _ptr(_c(rgba8, np.uint32)), P,
                        _ptr(_c(bg, np.float64)), _ptr(out))
    return out


def wboit(fr: Frags, rgba8, znear, zfar, bg=(1.0, 1.0, 1.0)):
    """Weighted blended OIT of each pixel's fragments (the evaluation's
    baseline OIT method), float64; the fragment depths are the raster's."""
    L = lib()
    P = fr.W * fr.H
    out = np.empty((P, 3), np.float64)
    L.orc_wboit(_ptr(fr.offsets), _ptr(_c(fr.z, np.float32)), _ptr(fr.prim), _ptr(_c(rgba8, np.uint32)),
                P, float(znear), float(zfar), _ptr(_c(bg, np.float64)), _ptr(out))
    return out


def upscale(src, Wp, Hp, W, H):
    """src [Hp*Wp, C] or [Hp*Wp] -> [H*W, C] / [H*W] bilinear, float64."""
    L = lib()
    s = _c(src, np.float64)
    C = 1 if s.ndim == 1 else s.shape[1]
    out = np.empty((H * W, C), np.float64)
    L.orc_upscale(_ptr(s), Wp, Hp, C, W, H, _ptr(out))
    return out[:, 0] if s.ndim == 1 else out


def tail_flag(n, Wp, Hp, W, H):
    L = lib()
    out = np.empty(H * W, np.uint8)
    L.orc_tail_flag(_ptr(_c(n, np.uint32)), Wp, Hp, W, H, _ptr(out))
    return out


def features(id1, rgba8, layer2, n_up, a_up, s_up, t_up, bg=(1.0, 1.0, 1.0), kappa=KAPPA_N):
    L = lib()
    P = int(np.asarray(id1).shape[0])
    x = np.empty((P, 5), np.float64)
    front = np.empty((P, 4), np.float64)
    L.orc_features(P, _ptr(_c(id1, np.int32)), _ptr(_c(rgba8, np.uint32)), _ptr(_c(layer2, np.float64)),
                   _ptr(_c(n_up, np.float64)), _ptr(_c(a_up, np.float64)), _ptr(_c(s_up, np.float64)),
                   _ptr(_c(t_up, np.float64)), _ptr(_c(bg, np.float64)), kappa, _ptr(x), _ptr(front))
    return x, front


def mlp_forward(params, x, flag=None):
    L = lib()
    x = _c(x, np.float64)
    n = x.shape[0]
    f = np.empty((n, 3), np.float64)
    fl = None if flag is None else _c(flag, np.uint8)
    L.orc_mlp_forward(_ptr(_c(params, np.float64)), _ptr(x), _ptr(fl), n, _ptr(f))
    return f


def mlp_mse_grad(params, x, y):
    L = lib()
    x = _c(x, np.float64)
    g = np.empty(771, np.float64)
    loss = L.orc_mlp_mse_grad(_ptr(_c(params, np.float64)), _ptr(x), _ptr(_c(y, np.float64)),
                              x.shape[0], _ptr(g))
    return float(loss), g


def adam(p, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam update of float64 arrays p, m, v."""
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().orc_adam(_ptr(p), _ptr(_c(g, np.float64)), _ptr(m), _ptr(v), p.size, step, lr, b1, b2, eps)


def composite(front, f):
    L = lib()
    front = _c(front, np.float64)
    P = front.shape[0]
    out = np.empty((P, 3), np.float64)
    L.orc_composite(_ptr(front), _ptr(_c(f, np.float64)), P, _ptr(out))
    return out


def quantize(rgb):
    L = lib()
    rgb = _c(rgb, np.float64)
    out = np.empty(rgb.shape[0], np.uint32)
    L.orc_quantize(_ptr(rgb), rgb.shape[0], _ptr(out))
    return out


def pass_scale(wbar, delta):
    return lib().orc_pass_scale(float(wbar), float(delta))


def pass_size(s, n):
    return lib().orc_pass_size(float(s), int(n))


def wbar(hist):
    """Scene complexity index: level-weighted mean of occupied leaves (Sec. 3.2)."""
    h = [int(v) for v in hist]
    tot = sum(h)
    return 0.0 if tot == 0 else sum(l * h[l] for l in range(4)) / tot


def quadtree(img, id1, W, H, base, tau_split, tau_merge, mask_prev, relax_iters=2):
    """One frame of tile evaluation; returns (mask, hist[4])."""
    L = lib()
    TX, TY = (W + base - 1) // base, (H + base - 1) // base
    mp = _c(mask_prev, np.uint32)
    assert mp.size == TX * TY
    mask = np.empty(TX * TY, np.uint32)
    hist = np.zeros(4, np.uint32)
    L.orc_quadtree(_ptr(_c(img, np.uint32)), _ptr(_c(id1, np.int32)), W, H, base, float(tau_split),
                   float(tau_merge), relax_iters, _ptr(mp), _ptr(mask), _ptr(hist))
    return mask, hist


# ---------------------------------------------------------------------------
# Per-leaf pass resolution: Eq. 2 with the scene index wbar replaced by the
# level l of the quadtree leaf holding the pixel, s_p(l) = clamp(2^(l -
# delta_p), 1/4, 1); each pixel takes passes 2 and 3 from the render target of
# its own leaf's scale (size ceil(s W) x ceil(s H), as for the global scale),
# upscaled bilinearly.

def leaf_levels(mask, W, H, base):
    """Level (0..3) of the leaf holding each pixel, [H*W] uint8, read from the
    per-tile split masks (bit 0 root; bits 1..4 the level-1 children; bits
    5..20 the level-2 nodes, 4 per level-1 child; child index 2 y_half + x_half)."""
    m = np.asarray(mask, np.uint32)
    TX = (W + base - 1) // base
    yy, xx = np.divmod(np.arange(W * H, dtype=np.int64), W)
    mt = m[(yy // base) * TX + xx // base].astype(np.int64)
    ly, lx = yy % base, xx % base
    h1, h2 = base // 2, base // 4
    c1 = 2 * (ly >= h1) + (lx >= h1)
    c2 = 2 * ((ly % h1) >= h2) + ((lx % h1) >= h2)
    root = (mt & 1) != 0
    split1 = root & (((mt >> (1 + c1)) & 1) != 0)
    split2 = split1 & (((mt >> (5 + 4 * c1 + c2)) & 1) != 0)
    return (root.astype(np.uint8) + split1 + split2).astype(np.uint8)


def leaf_sizes(W, H, delta2=None, delta3=None):
    """{(p, l): (W_p, H_p)} of passes p = 2, 3 at leaf levels l = 0..3."""
    d = {2: DELTA2 if delta2 is None else delta2, 3: DELTA3 if delta3 is None else delta3}
    out = {}
    for p in (2, 3):
        for l in range(4):
            s = pass_scale(float(l), d[p])
            out[(p, l)] = (pass_size(s, W), pass_size(s, H))
    return out


def frame_star_leaf(verts, rgba8, vp32, W, H, levels, params, bg=(1.0, 1.0, 1.0), threads=1,
                    delta2=None, delta3=None):
    """STAR-NT real frame with per-leaf resolution: pass 1 at W x H; a pixel
    whose leaf is at level l takes pass 2 from the target of size
    leaf_sizes[(2, l)] and pass 3 from that of leaf_sizes[(3, l)], each
    target resolved over the whole frame and upscaled bilinearly to W x H,
    before the features and the composite.  levels: [H*W] from leaf_levels."""
    lv = np.asarray(levels, np.uint8).reshape(-1)
    assert lv.size == W * H
    sizes = leaf_sizes(W, H, delta2, delta3)
    res = {(W, H): resolve(raster(verts, vp32, W, H, threads), rgba8, bg, threads)}
    for l in range(4):
        if np.any(lv == l):
            for p in (2, 3):
                sz = sizes[(p, l)]
                if sz not in res:
                    res[sz] = resolve(raster(verts, vp32, sz[0], sz[1], threads), rgba8, bg, threads)
    r1 = res[(W, H)]
    layer2 = np.empty((W * H, 4))
    n_up = np.empty(W * H)
    a_up = np.empty(W * H)
    s_up = np.empty((W * H, 3))
    t_up = np.empty(W * H)
    flag = np.empty(W * H, np.uint8)
    for l in range(4):
        sel = lv == l
        if not sel.any():
            continue
        (W2, H2), (W3, H3) = sizes[(2, l)], sizes[(3, l)]
        r2, r3 = res[(W2, H2)], res[(W3, H3)]
        layer2[sel] = upscale(r2["layer2"], W2, H2, W, H)[sel]
        n_up[sel] = upscale(r3["n"].astype(np.float64), W3, H3, W, H)[sel]
        a_up[sel] = upscale(r3["a_tail"].astype(np.float64), W3, H3, W, H)[sel]
        s_up[sel] = upscale(r3["s_tail"].astype(np.float64), W3, H3, W, H)[sel]
        t_up[sel] = upscale(r3["t_tail"], W3, H3, W, H)[sel]
        flag[sel] = tail_flag(r3["n"], W3, H3, W, H)[sel]
    x, front = features(r1["id1"], rgba8, layer2, n_up, a_up, s_up, t_up, bg)
    f = mlp_forward(params64(params), x, flag)
    rgb = composite(front, f)
    return dict(res=res, layer2=layer2, n_up=n_up, flag=flag, x=x, front=front, f=f, rgb=rgb)


def next_pass_sizes(hist, W, H, delta2=DELTA2, delta3=DELTA3):
    """Eq. 2 applied to the histogram: (wbar, s2, s3, (W2, H2), (W3, H3))."""
    wb = wbar(hist)
    s2, s3 = pass_scale(wb, delta2), pass_scale(wb, delta3)
    return wb, s2, s3, (pass_size(s2, W), pass_size(s2, H)), (pass_size(s3, W), pass_size(s3, H))


def inverse4(a):
    out = np.empty(16, np.float64)
    ok = lib().orc_inverse4(_ptr(_c(np.asarray(a).reshape(16), np.float64)), _ptr(out))
    if not ok:
        raise ValueError("singular matrix")
    return out.reshape(4, 4)


def reproject(prev, z1, vp_prev, vp_cur, W, H):
    L = lib()
    out = np.empty((W * H, 4), np.float64)
    L.orc_reproject(_ptr(_c(prev, np.float32)), _ptr(_c(z1, np.float32)),
                    _ptr(_c(np.asarray(vp_prev).reshape(16), np.float64)),
                    _ptr(_c(np.asarray(vp_cur).reshape(16), np.float64)), W, H, _ptr(out))
    return out


# ---------------------------------------------------------------------------
# Whole frames, composed from the steps above.

def params64(params_flat32):
    return np.asarray(params_flat32, dtype=np.float32).astype(np.float64)


def frame_full(verts, rgba8, vp32, W, H, params, bg=(1.0, 1.0, 1.0), threads=1):
    """Plain full-resolution neural OIT frame: every pass at W x H."""
    fr = raster(verts, vp32, W, H, threads)
    r = resolve(fr, rgba8, bg, threads)
    flag = (r["n"] > 2).astype(np.uint8)
    x, front = features(r["id1"], rgba8, r["layer2"], r["n"].astype(np.float64),
                        r["a_tail"].astype(np.float64), r["s_tail"].astype(np.float64),
                        r["t_tail"], bg)
    f = mlp_forward(params64(params), x, flag)
    rgb = composite(front, f)
    return dict(frags=fr, res=r, flag=flag, x=x, front=front, f=f, rgb=rgb)


def frame_star(verts, rgba8, vp32, W, H, size2, size3, params, bg=(1.0, 1.0, 1.0), threads=1):
    """STAR-NT real frame: pass 1 at W x H, pass 2 at size2, pass 3 at size3,
    both upscaled bilinearly before the features and the composite."""
    W2, H2 = size2
    W3, H3 = size3
    r1 = resolve(raster(verts, vp32, W, H, threads), rgba8, bg, threads)
    r2 = resolve(raster(verts, vp32, W2, H2, threads), rgba8, bg, threads)
    r3 = resolve(raster(verts, vp32, W3, H3, threads), rgba8, bg, threads)
    layer2 = upscale(r2["layer2"], W2, H2, W, H)
    n_up = upscale(r3["n"].astype(np.float64), W3, H3, W, H)
    a_up = upscale(r3["a_tail"].astype(np.float64), W3, H3, W, H)
    s_up = upscale(r3["s_tail"].astype(np.float64), W3, H3, W, H)
    t_up = upscale(r3["t_tail"], W3, H3, W, H)
    flag = tail_flag(r3["n"], W3, H3, W, H)
    x, front = features(r1["id1"], rgba8, layer2, n_up, a_up, s_up, t_up, bg)
    f = mlp_forward(params64(params), x, flag)
    rgb = composite(front, f)
    return dict(r1=r1, r2=r2, r3=r3, layer2=layer2, n_up=n_up, a_up=a_up, s_up=s_up, t_up=t_up,
                flag=flag, x=x, front=front, f=f, rgb=rgb)
