// context.cu -- the context of the C ABI: one object per device and frame
// size holding the method's parameters, the frame options (MLP operand type,
// merge scales of the reduced passes), the launch tuning of the persistent
// pass launches (chosen on the caller's own workload by star_nt_tune), a
// second stream with two events (the interpolated frame and the quadtree
// update run side by side), and the layout of one caller-allocated workspace
// that holds every buffer of the frame path between frames: the three pass
// workspaces, the pass planes, the quadtree masks and state, and the
// reprojection scratch.  star_nt_frame enqueues a whole STAR-NT step (Fig. 1):
// the real frame (pass 1 at full size, passes 2 and 3 at the sizes the
// quadtree chose on the previous frame, network, composite), the interpolated
// frame that reprojects it, and the quadtree update for the next frame.
#include <stddef.h>
#include <string.h>

#include <new>

#include "common.cuh"

struct star_nt_ctx {
  int device;
  star_nt_params params;
  star_nt_frame_options opt;
  star_nt_tuning tuning;
  int32_t fuse_passes;   // the pass launch also produces the frame (every pass at full size)
  cudaStream_t side;     // the interpolated frame, beside the quadtree update
  cudaEvent_t fork, join;
  // the bound workspace
  bool bound;
  int32_t W, H, T;
  char *ws;
  size_t ws_bytes;
};

namespace star {

// Offsets of the parts of a context workspace (256-byte aligned each).
struct CtxLayout {
  size_t bins[3];
  size_t bins_bytes;
  int64_t pair_cap;
  size_t size_full;  // int32 {W, H}
  size_t state;      // star_nt_pass_state
  size_t id1, z1, id2, n, tail, t_tail;
  size_t masks;
  int32_t n_tiles;
  size_t qt, qt_bytes;
  size_t reproj;
  size_t total;
};

// (triangle, tile) pairs each pass workspace holds: 96 per triangle (a
// triangle of the synthetic scenes touches a few tiles on average), at least
// 2^20.
inline int64_t ctx_pair_capacity(int32_t T) {
  const int64_t c = 96 * (int64_t)T;
  return c > (1 << 20) ? c : (1 << 20);
}

inline star_nt_status ctx_layout(const star_nt_params &p, int32_t W, int32_t H, int32_t T, CtxLayout &L) {
  if (W <= 0 || H <= 0 || T < 0 || W > 16384 || H > 16384) return STAR_NT_ERR_ARG;
  L.pair_cap = ctx_pair_capacity(T);
  if (star_nt_bins_bytes(W, H, T > 0 ? T : 1, L.pair_cap, &L.bins_bytes) != STAR_NT_OK) return STAR_NT_ERR_ARG;
  if (star_nt_quadtree_ws_bytes(W, H, p.base_tile, &L.qt_bytes) != STAR_NT_OK) return STAR_NT_ERR_ARG;
  const size_t P = (size_t)W * H;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, 256);
    return at;
  };
  for (int k = 0; k < 3; ++k) L.bins[k] = take(L.bins_bytes);
  L.size_full = take(8);
  L.state = take(sizeof(star_nt_pass_state));
  L.id1 = take(4 * P);
  L.z1 = take(4 * P);
  L.id2 = take(4 * P);
  L.n = take(4 * P);
  L.tail = take(16 * P);
  L.t_tail = take(4 * P);
  L.n_tiles = ((W + p.base_tile - 1) / p.base_tile) * ((H + p.base_tile - 1) / p.base_tile);
  L.masks = take(4 * (size_t)L.n_tiles);
  L.qt = take(L.qt_bytes);
  L.reproj = take(STAR_NT_REPROJECT_WS_BYTES);
  L.total = o;
  return STAR_NT_OK;
}

// First frame: every pass at full size, every quadtree leaf at level 0.
__global__ void k_ctx_init(int32_t *size_full, star_nt_pass_state *st, int W, int H) {
  size_full[0] = W;
  size_full[1] = H;
  st->W = st->W2 = st->W3 = W;
  st->H = st->H2 = st->H3 = H;
  st->s2 = st->s3 = 1.0f;
  st->wbar = 0.0;
  for (int k = 0; k < 4; ++k) st->hist[k] = 0u;
}

// The frame's views of the bound workspace.
struct CtxViews {
  star_nt_bins bins[3];
  star_nt_target tgt[3];
  star_nt_layers l1, l2, l3;
  uint32_t *masks;
  star_nt_pass_state *state;
  void *qt;
  size_t qt_bytes;
  void *reproj;
};

inline CtxViews ctx_views(const star_nt_ctx *c, const float *vp) {
  CtxLayout L;
  ctx_layout(c->params, c->W, c->H, c->T, L);
  char *m = c->ws;
  CtxViews v;
  for (int k = 0; k < 3; ++k)
    v.bins[k] = star_nt_bins{m + L.bins[k], L.bins_bytes, c->W, c->H, c->T > 0 ? c->T : 1, L.pair_cap};
  const int32_t *full = reinterpret_cast<const int32_t *>(m + L.size_full);
  const int32_t *st = reinterpret_cast<const int32_t *>(m + L.state);
  v.tgt[0] = star_nt_target{vp, full, c->W, c->H, nullptr, 1.0f};
  v.tgt[1] = star_nt_target{vp, st + 2, c->W, c->H, full, c->opt.merge_scale2};  // {W2, H2}
  v.tgt[2] = star_nt_target{vp, st + 4, c->W, c->H, full, c->opt.merge_scale3};  // {W3, H3}
  v.l1 = star_nt_layers{reinterpret_cast<int32_t *>(m + L.id1), reinterpret_cast<float *>(m + L.z1), nullptr,
                        nullptr, nullptr, nullptr};
  v.l2 = star_nt_layers{nullptr, nullptr, reinterpret_cast<int32_t *>(m + L.id2), nullptr, nullptr, nullptr};
  v.l3 = star_nt_layers{nullptr, nullptr, nullptr, reinterpret_cast<uint32_t *>(m + L.n),
                        reinterpret_cast<uint32_t *>(m + L.tail), reinterpret_cast<float *>(m + L.t_tail)};
  v.masks = reinterpret_cast<uint32_t *>(m + L.masks);
  v.state = reinterpret_cast<star_nt_pass_state *>(m + L.state);
  v.qt = m + L.qt;
  v.qt_bytes = L.qt_bytes;
  v.reproj = m + L.reproj;
  return v;
}

// Runs f with the context's device current, restoring the caller's.
template <class F>
inline cudaError_t on_device(int dev, F &&f) {
  int old = 0;
  cudaError_t e = cudaGetDevice(&old);
  if (e != cudaSuccess) return e;
  if (old != dev && (e = cudaSetDevice(dev)) != cudaSuccess) return e;
  const cudaError_t r = f();
  if (old != dev) cudaSetDevice(old);
  return r;
}

}  // namespace star

using namespace star;

extern "C" void star_nt_default_frame_options(star_nt_frame_options *o) {
  if (!o) return;
  o->mlp_type = STAR_NT_BF16;
  o->merge_scale2 = 1.0f;
  o->merge_scale3 = 1.0f;
  o->fuse_passes = 1;
}

static bool options_valid(const star_nt_frame_options &o) {
  if (o.mlp_type != STAR_NT_BF16 && o.mlp_type != STAR_NT_E4M3 && o.mlp_type != STAR_NT_E4M3X2 &&
      o.mlp_type != STAR_NT_E4M3_TENSOR && o.mlp_type != STAR_NT_E4M3X2_TENSOR)
    return false;
  return o.merge_scale2 > 0.0f && o.merge_scale2 <= 1.0f && o.merge_scale3 > 0.0f && o.merge_scale3 <= 1.0f;
}

static bool params_valid(const star_nt_params &p) {
  return (p.base_tile == 16 || p.base_tile == 64) && p.relax_iters >= 0 && p.relax_iters <= 8 &&
         p.tau_merge < p.tau_split;
}

extern "C" star_nt_status star_nt_create(int32_t device, const star_nt_params *params,
                                         const star_nt_frame_options *options, star_nt_ctx **out) {
  if (!out) return STAR_NT_ERR_ARG;
  *out = nullptr;
  star_nt_params p;
  star_nt_default_params(&p);
  if (params) p = *params;
  star_nt_frame_options o;
  star_nt_default_frame_options(&o);
  if (options) o = *options;
  if (!params_valid(p) || !options_valid(o)) return STAR_NT_ERR_ARG;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) {
    cudaGetLastError();
    return STAR_NT_ERR_CUDA;
  }
  if (device < 0 || device >= n) return STAR_NT_ERR_ARG;
  star_nt_ctx *c = new (std::nothrow) star_nt_ctx();
  if (!c) return STAR_NT_ERR_CAPACITY;
  c->device = device;
  c->params = p;
  c->opt = o;
  c->tuning = star_nt_tuning{8, 0, 2};
  c->fuse_passes = o.fuse_passes ? 1 : 0;
  c->bound = false;
  const cudaError_t e = on_device(device, [&] {
    cudaError_t r = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
    if (r != cudaSuccess) return r;
    if ((r = cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming)) != cudaSuccess) return r;
    return cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming);
  });
  if (e != cudaSuccess) {
    delete c;
    return STAR_NT_ERR_CUDA;
  }
  *out = c;
  return STAR_NT_OK;
}

extern "C" star_nt_status star_nt_destroy(star_nt_ctx *c) {
  if (!c) return STAR_NT_ERR_ARG;
  on_device(c->device, [&] {
    cudaStreamSynchronize(c->side);
    cudaEventDestroy(c->fork);
    cudaEventDestroy(c->join);
    cudaStreamDestroy(c->side);
    return cudaSuccess;
  });
  delete c;
  return STAR_NT_OK;
}

extern "C" star_nt_status star_nt_workspace_size(const star_nt_ctx *c, int32_t W, int32_t H, int32_t T,
                                                 size_t *bytes) {
  if (!c || !bytes) return STAR_NT_ERR_ARG;
  CtxLayout L;
  const star_nt_status s = ctx_layout(c->params, W, H, T, L);
  if (s != STAR_NT_OK) return s;
  *bytes = L.total;
  return STAR_NT_OK;
}

extern "C" star_nt_status star_nt_bind_workspace(star_nt_ctx *c, int32_t W, int32_t H, int32_t T, void *ws,
                                                 size_t ws_bytes, void *stream) {
  if (!c || !ws || ((uintptr_t)ws & 255u)) return STAR_NT_ERR_ARG;
  CtxLayout L;
  if (ctx_layout(c->params, W, H, T, L) != STAR_NT_OK || ws_bytes < L.total) return STAR_NT_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(ws, 0, L.total, st) != cudaSuccess) return STAR_NT_ERR_CUDA;
  char *m = (char *)ws;
  k_ctx_init<<<1, 1, 0, st>>>(reinterpret_cast<int32_t *>(m + L.size_full),
                              reinterpret_cast<star_nt_pass_state *>(m + L.state), W, H);
  if (cudaGetLastError() != cudaSuccess) return STAR_NT_ERR_CUDA;
  c->W = W;
  c->H = H;
  c->T = T;
  c->ws = m;
  c->ws_bytes = ws_bytes;
  c->bound = true;
  return STAR_NT_OK;
}

extern "C" star_nt_status star_nt_ctx_tuning(const star_nt_ctx *c, star_nt_tuning *tuning,
                                             int32_t *fuse_passes) {
  if (!c) return STAR_NT_ERR_ARG;
  if (tuning) *tuning = c->tuning;
  if (fuse_passes) *fuse_passes = c->fuse_passes;
  return STAR_NT_OK;
}

extern "C" star_nt_status star_nt_ctx_set_tuning(star_nt_ctx *c, const star_nt_tuning *tuning,
                                                 int32_t fuse_passes) {
  if (!c || !tuning) return STAR_NT_ERR_ARG;
  PassTuning tu;
  if (!pass_tuning(tuning, tu)) return STAR_NT_ERR_ARG;
  c->tuning = *tuning;
  c->fuse_passes = fuse_passes ? 1 : 0;
  return STAR_NT_OK;
}

extern "C" star_nt_status star_nt_ctx_pass_state(const star_nt_ctx *c, star_nt_pass_state **state,
                                                 uint32_t **masks, int32_t **id1, float **z1) {
  if (!c || !c->bound) return STAR_NT_ERR_ARG;
  CtxViews v = ctx_views(c, nullptr);
  if (state) *state = v.state;
  if (masks) *masks = v.masks;
  if (id1) *id1 = v.l1.id1;
  if (z1) *z1 = v.l1.z1;
  return STAR_NT_OK;
}

// The real frame's stages: the raster of the three passes, the pass launch,
// the resolve.
static star_nt_status real_frame(const star_nt_ctx *c, const CtxViews &v, const star_nt_scene *scene,
                                 const star_nt_mlp *w, float *rgba32f, uint32_t *rgba8, int32_t *d_status,
                                 cudaStream_t st, bool raster = true, bool passes = true,
                                 bool resolve = true) {
  star_nt_status s = STAR_NT_OK;
  if (raster && (s = star_nt_raster_passes(scene, 3, v.tgt, v.bins, d_status, st)) != STAR_NT_OK) return s;
  if (passes) {
    if (c->opt.mlp_type == STAR_NT_BF16 && c->fuse_passes)
      s = star_nt_geometry_passes_resolve(scene, &v.bins[0], &v.bins[1], &v.bins[2], &v.l1, &v.l2, &v.l3,
                                          &c->params, w, rgba32f, rgba8, &c->tuning, d_status, st);
    else
      s = star_nt_geometry_passes(scene, &v.bins[0], &v.bins[1], &v.bins[2], &v.l1, &v.l2, &v.l3,
                                  &c->tuning, d_status, st);
    if (s != STAR_NT_OK) return s;
  }
  if (resolve)
    s = star_nt_resolve_mlp(scene, &v.bins[1], &v.bins[2], &v.l1, &v.l2, &v.l3, c->W, c->H, &c->params, w,
                            c->opt.mlp_type, rgba32f, rgba8, d_status, st);
  return s;
}

static bool frame_args_ok(const star_nt_ctx *c, const star_nt_scene *scene, const star_nt_mlp *w,
                          const star_nt_cameras *cams, const star_nt_frame_out *out) {
  if (!c || !c->bound || !scene || !w || !cams || !out || !cams->vp) return false;
  if (scene->n_tris < 0 || scene->n_tris > (c->T > 0 ? c->T : 1)) return false;
  if (!out->rgba32f || !out->rgba8) return false;  // the reprojection and the quadtree read them
  if (cams->vp64_interp && (!cams->vp64 || (!out->interp_rgba32f && !out->interp_rgba8))) return false;
  return true;
}

extern "C" star_nt_status star_nt_frame(star_nt_ctx *c, const star_nt_scene *scene, const star_nt_mlp *w,
                                        const star_nt_cameras *cams, const star_nt_frame_out *out,
                                        int32_t *d_status, void *stream) {
  if (!frame_args_ok(c, scene, w, cams, out)) return STAR_NT_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const CtxViews v = ctx_views(c, cams->vp);
  star_nt_status s = real_frame(c, v, scene, w, out->rgba32f, out->rgba8, d_status, st);
  if (s != STAR_NT_OK) return s;
  const bool interp = cams->vp64_interp != nullptr;
  if (interp) {
    // the interpolated frame needs only the real frame's colour and depth:
    // it runs on the side stream while the quadtree updates the tiles
    if (cudaEventRecord(c->fork, st) != cudaSuccess || cudaStreamWaitEvent(c->side, c->fork, 0) != cudaSuccess)
      return STAR_NT_ERR_CUDA;
    s = star_nt_reproject(out->rgba32f, v.l1.z1, cams->vp64, cams->vp64_interp, c->W, c->H,
                          out->interp_rgba32f, out->interp_rgba8, v.reproj, c->side);
    if (s != STAR_NT_OK) return s;
    if (cudaEventRecord(c->join, c->side) != cudaSuccess) return STAR_NT_ERR_CUDA;
  }
  s = star_nt_quadtree(out->rgba8, v.l1.id1, c->W, c->H, &c->params, v.masks, v.masks, v.state, v.qt,
                       v.qt_bytes, st);
  if (s != STAR_NT_OK) return s;
  if (interp && cudaStreamWaitEvent(st, c->join, 0) != cudaSuccess) return STAR_NT_ERR_CUDA;
  return STAR_NT_OK;
}

// Average ms of reps runs of f on stream st, timed with CUDA events (one
// untimed run first).
template <class F>
static float time_ms(cudaStream_t st, int reps, F &&f) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  f();
  cudaEventRecord(e0, st);
  for (int i = 0; i < reps; ++i) f();
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms / reps;
}

extern "C" star_nt_status star_nt_tune(star_nt_ctx *c, const star_nt_scene *scene, const star_nt_mlp *w,
                                       const star_nt_cameras *cams, const star_nt_frame_out *out,
                                       int32_t *d_status, void *stream, star_nt_tune_report *report) {
  if (!frame_args_ok(c, scene, w, cams, out)) return STAR_NT_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
    return STAR_NT_ERR_ARG;  // the tuner synchronises: not inside a capture
  static const star_nt_tuning kCand[STAR_NT_TUNE_CANDIDATES] = {
      {8, 0, 2}, {4, 0, 2}, {16, 0, 2}, {8, 10, 2}, {4, 10, 2}, {8, 0, 1}, {4, 0, 1}, {8, 6, 1}, {4, 6, 1}};
  const CtxViews v = ctx_views(c, cams->vp);
  const star_nt_tuning keep = c->tuning;
  const int32_t keep_fuse = c->fuse_passes;
  star_nt_tune_report r;
  memset(&r, 0, sizeof(r));
  star_nt_status s = STAR_NT_OK;
  const int reps = 10;
  // the pass sizes in force: the raster of the current state, once
  if ((s = star_nt_raster_passes(scene, 3, v.tgt, v.bins, d_status, st)) != STAR_NT_OK) return s;
  int best = 0;
  for (int k = 0; k < STAR_NT_TUNE_CANDIDATES; ++k) {
    c->tuning = kCand[k];
    r.candidates[k] = kCand[k];
    r.passes_ms[k] = time_ms(st, reps, [&] {
      if (s == STAR_NT_OK) s = real_frame(c, v, scene, w, out->rgba32f, out->rgba8, d_status, st, false, true, false);
    });
    if (r.passes_ms[k] < r.passes_ms[best]) best = k;
  }
  c->tuning = kCand[best];
  r.chosen = kCand[best];
  r.fuse_passes = keep_fuse;
  if (s == STAR_NT_OK && c->opt.mlp_type == STAR_NT_BF16 && c->opt.fuse_passes) {
    // with that shape: does the pass launch produce the frame (when every pass
    // runs at full size), or the separate resolve?  The raster resets the
    // frame's resolved mark, so both settings start every run alike.
    for (int fuse = 1; fuse >= 0; --fuse) {
      c->fuse_passes = fuse;
      r.frame_ms[fuse] = time_ms(st, reps, [&] {
        if (s == STAR_NT_OK) s = real_frame(c, v, scene, w, out->rgba32f, out->rgba8, d_status, st);
      });
    }
    // the merged words of the pass-2 and pass-3 bins headers after the raster
    int32_t mg[2] = {0, 0};
    for (int q = 0; q < 2 && s == STAR_NT_OK; ++q)
      if (cudaMemcpyAsync(&mg[q], static_cast<char *>(v.bins[q + 1].mem) + offsetof(BinsHeader, merged),
                          sizeof(int32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        s = STAR_NT_ERR_CUDA;
    if (s == STAR_NT_OK && cudaStreamSynchronize(st) != cudaSuccess) s = STAR_NT_ERR_CUDA;
    r.frame_merged = mg[0] != 0 && mg[1] != 0 ? 1 : 0;
    r.fuse_passes = r.frame_ms[1] <= r.frame_ms[0] || !r.frame_merged ? 1 : 0;
  }
  if (s != STAR_NT_OK || cudaGetLastError() != cudaSuccess) {
    c->tuning = keep;
    c->fuse_passes = keep_fuse;
    return s != STAR_NT_OK ? s : STAR_NT_ERR_CUDA;
  }
  c->fuse_passes = r.fuse_passes;
  if (report) *report = r;
  return STAR_NT_OK;
}
