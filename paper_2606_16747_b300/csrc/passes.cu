// passes.cu -- star_nt_build_inputs: the three geometry passes (nearest,
// second-nearest, tail statistics; Sec. 3, Sec. 3.3), the bilinear upscale of
// the reduced passes (Sec. 3.2) and the network input / front terms of
// Eq. 4.
#include <math.h>

#include <cuda_bf16.h>

#include "pass_body.cuh"

namespace star {

// One tile per CTA of 128 threads, two pixels per thread (pass_body2).
template <int MODE>
__global__ void __launch_bounds__(128, 8) k_pass(BinsView bv, const uint32_t *__restrict__ rgba8,
                                              PassOut po, FeatOut fo) {
  __shared__ WalkStage stage;
  pass_body2<MODE>(bv, rgba8, po, stage, blockIdx.x, fo);
}

// Pass 1 at full resolution; when pass 2 and/or pass 3 are marked merged
// (their size equals the full size) it keeps the two nearest fragments and
// the tail sums as well and writes their planes at full resolution.
__global__ void __launch_bounds__(128, 10) k_pass_merged(BinsView bv, const BinsHeader *hd2,
                                                      const BinsHeader *hd3,
                                                      const uint32_t *__restrict__ rgba8, PassOut o1,
                                                      PassOut o2, PassOut o3) {
  __shared__ WalkStage stage;
  const bool m2 = hd2->merged != 0, m3 = hd3->merged != 0;
  if (!m2 && !m3) {
    pass_body2<kTop1>(bv, rgba8, o1, stage, blockIdx.x);
    return;
  }
  PassOut o = o1;
  o.id2 = m2 ? o2.id2 : nullptr;
  if (!m3) {  // two layers, no tail sums: the top-2 traversal with its depth skip
    pass_body2<kTop2>(bv, rgba8, o, stage, blockIdx.x);
    return;
  }
  o.n = o3.n;
  o.tail = o3.tail;
  o.t_tail = o3.t_tail;
  pass_body2<kTail>(bv, rgba8, o, stage, blockIdx.x);
}

// All geometry passes of a real frame in one persistent launch: CTAs take
// (pass, tile) items from a queue counter in order - every tile of pass 1,
// then of pass 2, then of pass 3 - until the items run out, so tiles of uneven
// cost and passes of different resolutions share one launch without a tail
// between passes.  Pass 1 takes over merged passes as k_pass_merged does.
// MINB: CTAs per SM the register budget is cut for (6: 40 registers per
// thread; 8: 32 registers, a few spilled, more warps to cover the barrier
// waits of uneven pixel blocks).
template <int BW, int MINB>
__global__ void __launch_bounds__(256, MINB) k_passes(BinsView v1, BinsView v2, BinsView v3,
                                                   const uint32_t *__restrict__ rgba8, PassOut o1,
                                                   PassOut o2, PassOut o3, uint32_t *queue) {
  __shared__ TileStage stage;
  __shared__ int s_item;
  if (v2.hd->resolved) return;  // star_nt_geometry_passes_resolve's launch did the passes
  const bool m2 = v2.hd->merged != 0, m3 = v3.hd->merged != 0;
  const int n1 = v1.hd->n_tiles, n2 = v2.hd->n_tiles, n3 = v3.hd->n_tiles;
  const int total = n1 + n2 + n3;
  PassOut om = o1;  // pass 1 with the merged passes' outputs
  om.id2 = m2 ? o2.id2 : nullptr;
  om.n = m3 ? o3.n : nullptr;
  om.tail = m3 ? o3.tail : nullptr;
  om.t_tail = m3 ? o3.t_tail : nullptr;
  o2.id1 = nullptr;
  o2.z1 = nullptr;
  o3.id1 = nullptr;
  o3.z1 = nullptr;
  o3.id2 = nullptr;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(queue, 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();  // every thread has the item before s_item is reused
    if (item >= total) {
      // the last CTA out resets the queue and the exit count for the next launch
      if (threadIdx.x == 0 && atomicAdd(queue + 1, 1u) == gridDim.x - 1) {
        queue[0] = 0u;
        queue[1] = 0u;
      }
      break;
    }
    if (item < n1) {
      if (m3) pass_body<kTail, BW>(v1, rgba8, om, FeatOut{}, stage, item);
      else if (m2) pass_body<kTop2, BW>(v1, rgba8, om, FeatOut{}, stage, item);
      else pass_body<kTop1, BW>(v1, rgba8, o1, FeatOut{}, stage, item);
    } else if (item < n1 + n2) {
      pass_body<kTop2, BW>(v2, rgba8, o2, FeatOut{}, stage, item - n1);
    } else {
      pass_body<kTail, BW>(v3, rgba8, o3, FeatOut{}, stage, item - n1 - n2);
    }
  }
}

// k_passes with two pixels per thread (pass_body2): CTAs of 128 threads, one
// tile each; MINB 8 gives a 64-register budget (the default), 10 a 48-register
// one (the walk then spills a little).
template <int BW, int MINB>
__global__ void __launch_bounds__(128, MINB) k_passes2(BinsView v1, BinsView v2, BinsView v3,
                                                    const uint32_t *__restrict__ rgba8, PassOut o1,
                                                    PassOut o2, PassOut o3, uint32_t *queue) {
  __shared__ WalkStage stage;
  __shared__ int s_item;
  if (v2.hd->resolved) return;  // star_nt_geometry_passes_resolve's launch did the passes
  const bool m2 = v2.hd->merged != 0, m3 = v3.hd->merged != 0;
  const int n1 = v1.hd->n_tiles, n2 = v2.hd->n_tiles, n3 = v3.hd->n_tiles;
  const int total = n1 + n2 + n3;
  PassOut om = o1;
  om.id2 = m2 ? o2.id2 : nullptr;
  om.n = m3 ? o3.n : nullptr;
  om.tail = m3 ? o3.tail : nullptr;
  om.t_tail = m3 ? o3.t_tail : nullptr;
  o2.id1 = nullptr;
  o2.z1 = nullptr;
  o3.id1 = nullptr;
  o3.z1 = nullptr;
  o3.id2 = nullptr;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(queue, 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= total) {
      if (threadIdx.x == 0 && atomicAdd(queue + 1, 1u) == gridDim.x - 1) {
        queue[0] = 0u;
        queue[1] = 0u;
      }
      break;
    }
    if (item < n1) {
      if (m3) pass_body2<kTail, BW>(v1, rgba8, om, stage, item);
      else if (m2) pass_body2<kTop2, BW>(v1, rgba8, om, stage, item);
      else pass_body2<kTop1, BW>(v1, rgba8, o1, stage, item);
    } else if (item < n1 + n2) {
      pass_body2<kTop2, BW>(v2, rgba8, o2, stage, item - n1);
    } else {
      pass_body2<kTail, BW>(v3, rgba8, o3, stage, item - n1 - n2);
    }
  }
}

// Full-resolution features from pass 1 (full res) and the bilinear upscale
// of passes 2 and 3 (their own resolutions, read from their bins headers).
__global__ void __launch_bounds__(256) k_features(FeatIn in, FeatOut fo) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31);
  const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (x >= in.W || y >= in.H) return;
  if (in.hd2->n_pixels <= 0 || in.hd3->n_pixels <= 0) return;  // a pass was rejected
  float xv[6];
  float4 fr;
  pixel_features(in, fo.bg0, fo.bg1, fo.bg2, fo.kappa, x, y, xv, fr);
  store_features(fo, (size_t)y * in.W + x, xv, fr);
}

}  // namespace star

using namespace star;

static PassOut pass_out(const star_nt_layers *l) {
  PassOut o = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  if (l) {
    o.id1 = l->id1;
    o.z1 = l->z1;
    o.id2 = l->id2;
    o.n = l->n;
    o.tail = reinterpret_cast<uint4 *>(l->tail);
    o.t_tail = l->t_tail;
  }
  return o;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static bool layers_ok(const star_nt_layers *l) {
  if (!l) return true;
  return aligned16(l->tail) && aligned16(l->id1) && aligned16(l->z1) && aligned16(l->id2) &&
         aligned16(l->n) && aligned16(l->t_tail);
}

static bool make_feat(const star_nt_params *params, const star_nt_features *out, FeatOut &fo) {
  if (!params || !out || !out->x || !out->front) return false;
  if (out->x_dtype != STAR_NT_F32 && out->x_dtype != STAR_NT_BF16) return false;
  if (!aligned16(out->x) || !aligned16(out->front)) return false;
  fo.x = out->x;
  fo.x_dtype = out->x_dtype;
  fo.front = reinterpret_cast<float4 *>(out->front);
  fo.bg0 = params->bg[0];
  fo.bg1 = params->bg[1];
  fo.bg2 = params->bg[2];
  fo.kappa = params->kappa_n;
  return true;
}

static int tiles_of(const star_nt_bins *b) {
  return ((b->max_w + kTile - 1) / kTile) * ((b->max_h + kTile - 1) / kTile);
}

extern "C" star_nt_status star_nt_geometry_pass(const star_nt_scene *scene, const star_nt_bins *bins,
                                                int32_t mode, const star_nt_layers *layers,
                                                int32_t *d_status, void *stream) {
  (void)d_status;
  if (!scene || !bins || !bins->mem || !layers || !layers_ok(layers)) return STAR_NT_ERR_ARG;
  if (scene->n_tris > 0 && !scene->rgba8) return STAR_NT_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  BinsView v = bins_view(*bins);
  PassOut o = pass_out(layers);
  FeatOut fo = {};
  const int tiles = tiles_of(bins);
  switch (mode) {
    case 1:
      if (!layers->id1 && !layers->z1) return STAR_NT_ERR_ARG;
      k_pass<kTop1><<<tiles, 128, 0, st>>>(v, scene->rgba8, o, fo);
      break;
    case 2:
      if (!layers->id2) return STAR_NT_ERR_ARG;
      k_pass<kTop2><<<tiles, 128, 0, st>>>(v, scene->rgba8, o, fo);
      break;
    case 3:
      if (!layers->n || !layers->tail || !layers->t_tail) return STAR_NT_ERR_ARG;
      k_pass<kTail><<<tiles, 128, 0, st>>>(v, scene->rgba8, o, fo);
      break;
    default:
      return STAR_NT_ERR_ARG;
  }
  return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
}

extern "C" star_nt_status star_nt_geometry_pass_merged(const star_nt_scene *scene,
                                                       const star_nt_bins *b1,
                                                       const star_nt_bins *b2,
                                                       const star_nt_bins *b3,
                                                       const star_nt_layers *l1,
                                                       const star_nt_layers *l2,
                                                       const star_nt_layers *l3, int32_t *d_status,
                                                       void *stream) {
  (void)d_status;
  if (!scene || !b1 || !b2 || !b3 || !b1->mem || !b2->mem || !b3->mem || !l1 || !l2 || !l3)
    return STAR_NT_ERR_ARG;
  if (!l1->id1 && !l1->z1) return STAR_NT_ERR_ARG;
  if (!l2->id2 || !l3->n || !l3->tail || !l3->t_tail) return STAR_NT_ERR_ARG;
  if (!layers_ok(l1) || !layers_ok(l2) || !layers_ok(l3)) return STAR_NT_ERR_ARG;
  if (scene->n_tris > 0 && !scene->rgba8) return STAR_NT_ERR_ARG;
  BinsView v1 = bins_view(*b1), v2 = bins_view(*b2), v3 = bins_view(*b3);
  PassOut o1 = pass_out(l1);
  o1.id2 = nullptr; o1.n = nullptr; o1.tail = nullptr; o1.t_tail = nullptr;
  k_pass_merged<<<tiles_of(b1), 128, 0, (cudaStream_t)stream>>>(v1, v2.hd, v3.hd, scene->rgba8, o1,
                                                                pass_out(l2), pass_out(l3));
  return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
}

extern "C" star_nt_status star_nt_geometry_passes(const star_nt_scene *scene,
                                                  const star_nt_bins *b1, const star_nt_bins *b2,
                                                  const star_nt_bins *b3, const star_nt_layers *l1,
                                                  const star_nt_layers *l2,
                                                  const star_nt_layers *l3,
                                                  const star_nt_tuning *tuning, int32_t *d_status,
                                                  void *stream) {
  (void)d_status;
  if (!scene || !b1 || !b2 || !b3 || !b1->mem || !b2->mem || !b3->mem || !l1 || !l2 || !l3)
    return STAR_NT_ERR_ARG;
  if ((!l1->id1 && !l1->z1) || !l2->id2 || !l3->n || !l3->tail || !l3->t_tail) return STAR_NT_ERR_ARG;
  if (!layers_ok(l1) || !layers_ok(l2) || !layers_ok(l3)) return STAR_NT_ERR_ARG;
  if (scene->n_tris > 0 && !scene->rgba8) return STAR_NT_ERR_ARG;
  if (b1->mem == b2->mem || b1->mem == b3->mem || b2->mem == b3->mem) return STAR_NT_ERR_ARG;
  PassTuning tu;
  if (!pass_tuning(tuning, tu)) return STAR_NT_ERR_ARG;
  const int bw = tu.bw, per_sm = tu.per_sm;
  cudaStream_t st = (cudaStream_t)stream;
  BinsView v1 = bins_view(*b1), v2 = bins_view(*b2), v3 = bins_view(*b3);
  PassOut o1 = pass_out(l1), o2 = pass_out(l2), o3 = pass_out(l3);
  o1.id2 = nullptr; o1.n = nullptr; o1.tail = nullptr; o1.t_tail = nullptr;
  uint32_t *queue = &v1.hd->queue;  // queue[0] work counter, queue[1] exit count (pad[0])
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  auto launch = [&](auto kern, int threads = 256) {
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, 0);
    const int k = per_sm > 0 ? (per_sm < occ ? per_sm : occ) : occ;
    kern<<<sms * (k > 0 ? k : 1), threads, 0, st>>>(v1, v2, v3, scene->rgba8, o1, o2, o3, queue);
  };
  if (tu.pix == 2) {  // two pixels per thread: 10 the 10-CTA budget, 0..9 the 8-CTA one
    const bool wide2 = per_sm == 10;
    if (bw == 8) wide2 ? launch(k_passes2<8, 10>, 128) : launch(k_passes2<8, 8>, 128);
    else if (bw == 16) wide2 ? launch(k_passes2<16, 10>, 128) : launch(k_passes2<16, 8>, 128);
    else wide2 ? launch(k_passes2<4, 10>, 128) : launch(k_passes2<4, 8>, 128);
    return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
  }
  // ctas_per_sm 0 or 8: the 8-CTA register budget at full occupancy; 1..7: the
  // 6-CTA budget, grid capped at that many CTAs per SM
  const bool wide = per_sm == 0 || per_sm == 8;
  if (bw == 8) wide ? launch(k_passes<8, 8>) : launch(k_passes<8, 6>);
  else if (bw == 16) wide ? launch(k_passes<16, 8>) : launch(k_passes<16, 6>);
  else wide ? launch(k_passes<4, 8>) : launch(k_passes<4, 6>);
  return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
}

extern "C" star_nt_status star_nt_upscale_features(const star_nt_scene *scene, const star_nt_bins *b2,
                                           const star_nt_bins *b3, const star_nt_layers *l1,
                                           const star_nt_layers *l2, const star_nt_layers *l3,
                                           int32_t W, int32_t H, const star_nt_params *params,
                                           const star_nt_features *out, void *stream) {
  FeatOut fo;
  if (!scene || !b2 || !b3 || !b2->mem || !b3->mem || !make_feat(params, out, fo)) return STAR_NT_ERR_ARG;
  if (W <= 0 || H <= 0 || !l1 || !l1->id1 || !l2 || !l2->id2 || !l3 || !l3->n || !l3->tail ||
      !l3->t_tail || !layers_ok(l1) || !layers_ok(l2) || !layers_ok(l3))
    return STAR_NT_ERR_ARG;
  if (scene->n_tris > 0 && !scene->rgba8) return STAR_NT_ERR_ARG;
  BinsView v2 = bins_view(*b2), v3 = bins_view(*b3);
  dim3 grid((W + 31) / 32, (H + 7) / 8);
  FeatIn in{W, H, v2.hd, v3.hd, scene->rgba8, l1->id1, l2->id2, l3->n,
            reinterpret_cast<const uint4 *>(l3->tail), l3->t_tail};
  k_features<<<grid, 256, 0, (cudaStream_t)stream>>>(in, fo);
  return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
}

extern "C" star_nt_status star_nt_build_inputs(const star_nt_scene *scene, const star_nt_bins *b1,
                                               const star_nt_bins *b2, const star_nt_bins *b3,
                                               const star_nt_layers *l1,
                                               const star_nt_layers *l2,
                                               const star_nt_layers *l3, int32_t W, int32_t H,
                                               const star_nt_params *params,
                                               const star_nt_features *out, int32_t *d_status,
                                               void *stream) {
  FeatOut fo;
  if (!scene || !b1 || !b2 || !b3 || !make_feat(params, out, fo)) return STAR_NT_ERR_ARG;
  if (W <= 0 || H <= 0 || b1->max_w < W || b1->max_h < H) return STAR_NT_ERR_ARG;
  if (!layers_ok(l1) || !layers_ok(l2) || !layers_ok(l3)) return STAR_NT_ERR_ARG;
  if (scene->n_tris > 0 && !scene->rgba8) return STAR_NT_ERR_ARG;
  const bool fused = (b1->mem == b2->mem) && (b2->mem == b3->mem);
  if (fused) {
    BinsView v1 = bins_view(*b1);
    k_pass<kFused><<<tiles_of(b1), 128, 0, (cudaStream_t)stream>>>(v1, scene->rgba8, pass_out(l1), fo);
    return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
  }
  if (!l1 || !l1->id1 || !l2 || !l2->id2 || !l3 || !l3->n || !l3->tail || !l3->t_tail)
    return STAR_NT_ERR_ARG;
  star_nt_layers b = {}, c = {};
  b.id2 = l2->id2;
  c.n = l3->n;
  c.tail = l3->tail;
  c.t_tail = l3->t_tail;
  star_nt_status s;
  if ((s = star_nt_geometry_pass_merged(scene, b1, b2, b3, l1, l2, l3, d_status, stream)) !=
      STAR_NT_OK)
    return s;
  if ((s = star_nt_geometry_pass(scene, b2, 2, &b, d_status, stream)) != STAR_NT_OK) return s;
  if ((s = star_nt_geometry_pass(scene, b3, 3, &c, d_status, stream)) != STAR_NT_OK) return s;
  return star_nt_upscale_features(scene, b2, b3, l1, l2, l3, W, H, params, out, stream);
}

extern "C" star_nt_status star_nt_build_inputs_dfaoit(const star_nt_scene *scene, const star_nt_bins *bins,
                                                      const star_nt_layers *layers1, int32_t W, int32_t H,
                                                      const star_nt_params *params,
                                                      const star_nt_features *out, int32_t *d_status,
                                                      void *stream) {
  (void)d_status;
  FeatOut fo;
  if (!scene || !bins || !bins->mem || !make_feat(params, out, fo)) return STAR_NT_ERR_ARG;
  if (W <= 0 || H <= 0 || bins->max_w < W || bins->max_h < H) return STAR_NT_ERR_ARG;
  if (!layers_ok(layers1)) return STAR_NT_ERR_ARG;
  if (scene->n_tris > 0 && !scene->rgba8) return STAR_NT_ERR_ARG;
  if (fo.x_dtype == STAR_NT_BF16 && ((uintptr_t)out->x & 255u)) return STAR_NT_ERR_ARG;  // TMA source
  BinsView v = bins_view(*bins);
  PassOut o = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  if (layers1) o = pass_out(layers1);
  k_pass<kFusedDfaoit><<<tiles_of(bins), 128, 0, (cudaStream_t)stream>>>(v, scene->rgba8, o, fo);
  return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
}

namespace star {
// Loads this file's kernels onto the current device (see star_nt_preload).
cudaError_t preload_passes() {
  cudaFuncAttributes a;
  cudaError_t e = cudaSuccess, r;
  if ((r = cudaFuncGetAttributes(&a, k_pass<kTop1>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_pass<kTop2>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_pass<kTail>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_pass<kFused>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_pass<kFusedDfaoit>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_pass_merged)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes<4, 6>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes<8, 6>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes<16, 6>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes<4, 8>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes<8, 8>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes<16, 8>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes2<4, 10>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes2<8, 10>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes2<16, 10>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes2<4, 8>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes2<8, 8>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes2<16, 8>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_features)) != cudaSuccess) e = r;
  return e;
}
}  // namespace star
