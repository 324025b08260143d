// baselines.cu -- the comparison renderers of the evaluation (Sec. 4): a naive
// renderer that blends with "over" in submission order, whose error E_random
// anchors the Q measure, and weighted blended OIT (WBOIT, McGuire and Bavoil
// 2013), the paper's baseline OIT method.  Neither is on the STAR-NT path.
#include <math.h>

#include "common.cuh"
#include "features.cuh"
#include "raster_tile.cuh"

namespace star {

__device__ __forceinline__ void over_rgba8(uint32_t c, float &T, float &r, float &g, float &b) {
  const float a = (float)(c >> 24) / 255.0f;
  const float w = T * a;
  r += w * ((float)(c & 255u) / 255.0f);
  g += w * ((float)((c >> 8) & 255u) / 255.0f);
  b += w * ((float)((c >> 16) & 255u) / 255.0f);
  T *= 1.0f - a;
}

// Naive blending: each pixel's fragments composited with "over" in the order
// a renderer without OIT would submit them, increasing primitive id (the ids
// of the synthetic scenes are unrelated to depth, so this is a random order).
__global__ void __launch_bounds__(128) k_unsorted_over(const uint32_t *__restrict__ count,
                                                       const uint32_t *__restrict__ offset,
                                                       const int32_t *__restrict__ prims,
                                                       const uint32_t *__restrict__ rgba8, long long P,
                                                       float bg0, float bg1, float bg2,
                                                       float4 *__restrict__ rgb) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const int n = (int)count[p];
  const uint32_t base = offset[p];
  float T = 1.0f, r = 0.f, g = 0.f, b = 0.f;
  int last = -1;
  for (int i = 0; i < n; ++i) {  // next id in increasing order (ids are distinct per pixel)
    int best = 0x7fffffff;
    for (int k = 0; k < n; ++k) {
      const int id = prims[base + k];
      if (id > last && id < best) best = id;
    }
    over_rgba8(__ldg(rgba8 + best), T, r, g, b);
    last = best;
  }
  rgb[p] = make_float4(r + T * bg0, g + T * bg1, b + T * bg2, T);
}

// WBOIT weight of a fragment at view depth d with opacity a, the authors'
// recommended depth weight (their Eq. 7):
// w(d, a) = a * clamp(10 / (1e-5 + (d/5)^2 + (d/200)^6), 1e-2, 3e3).
__device__ __forceinline__ float wboit_weight(float d, float a) {
  const float u = d * 0.2f, v = d * 0.005f;
  const float v2 = v * v;
  const float w = 10.0f / (1e-5f + u * u + v2 * v2 * v2);
  return a * fminf(fmaxf(w, 1e-2f), 3e3f);
}

// WBOIT in one pass over the binned tiles of a full-resolution target: per
// pixel the sums of (a c) w and a w with w = w(d, a), and the product of
// (1 - a) (kept, order-free, as a fixed-point -log2 sum and an opaque count;
// the sum alone also gives 0 for an opaque fragment, as in the tail
// statistics); then
// C = (sum (a c) w / max(sum a w, 1e-5)) (1 - T) + T C_b.
// View depth from NDC z in [0, 1]: d = n f / (f - z (f - n)).
__global__ void __launch_bounds__(256) k_wboit(BinsView bv, float znear, float zfar, float bg0,
                                               float bg1, float bg2, float4 *__restrict__ out,
                                               uint32_t *__restrict__ out8) {
  __shared__ TileStage stage;
  const BinsHeader *hd = bv.hd;
  if ((int64_t)hd->n_pairs > bv.pair_capacity) return;
  const int tile = blockIdx.x;
  if (tile >= hd->n_tiles) return;
  const int W = hd->size[0], H = hd->size[1];
  const TilePixel tp = tile_pixel<8>(tile, hd->tiles_x);
  const float nf = znear * zfar, fmn = zfar - znear;
  float sr = 0.f, sg = 0.f, sb = 0.f, sa = 0.f;
  unsigned long long lg = 0;
  uint32_t opq = 0;
  for_each_fragment(bv, tile, tp, stage, [] { return INFINITY; },
                    [&](const TriSetup &T, uint32_t, long long e0, long long e2) {
    const float z = frag_depth(T, e0, e2);
    const float d = nf / (zfar - z * fmn);
    const float a = (float)(uint32_t)(T.ba >> 32) * (1.0f / 255.0f);
    const float w = wboit_weight(d, a);
    const float k = w * (1.0f / 65025.0f);  // (a8 c8) / 255^2 = a c
    sr += (float)(uint32_t)(T.rg & 0xffffffffull) * k;
    sg += (float)(uint32_t)(T.rg >> 32) * k;
    sb += (float)(uint32_t)(T.ba & 0xffffffffull) * k;
    sa += a * w;
    lg += T.lg;
    opq += T.opq;
  });
  if (tp.px >= W || tp.py >= H) return;
  const float t = tail_transmittance(lg, opq);
  const float inv = 1.0f / fmaxf(sa, 1e-5f);
  const float r = sr * inv * (1.0f - t) + t * bg0;
  const float g = sg * inv * (1.0f - t) + t * bg1;
  const float b = sb * inv * (1.0f - t) + t * bg2;
  const size_t p = (size_t)tp.py * W + tp.px;
  if (out) out[p] = make_float4(r, g, b, t);
  if (out8) out8[p] = quantize_rgba8(r, g, b);
}

}  // namespace star

using namespace star;

extern "C" star_nt_status star_nt_unsorted_over(const star_nt_frags *frags, const uint32_t *rgba8,
                                                int32_t W, int32_t H, const float *bg, float *rgb,
                                                void *stream) {
  if (!frags || !frags->count || !frags->offset || !frags->prim || !rgba8 || !bg || !rgb || W <= 0 ||
      H <= 0 || ((uintptr_t)rgb & 15u))
    return STAR_NT_ERR_ARG;
  const long long P = (long long)W * H;
  k_unsorted_over<<<(unsigned)((P + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
      frags->count, frags->offset, frags->prim, rgba8, P, bg[0], bg[1], bg[2],
      reinterpret_cast<float4 *>(rgb));
  return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
}

extern "C" star_nt_status star_nt_wboit(const star_nt_bins *bins, float znear, float zfar,
                                        const float *bg, float *rgba32f, uint32_t *rgba8,
                                        void *stream) {
  if (!bins || !bins->mem || !bg || (!rgba32f && !rgba8) || ((uintptr_t)rgba32f & 15u))
    return STAR_NT_ERR_ARG;
  if (!(znear > 0.0f) || !(zfar > znear)) return STAR_NT_ERR_ARG;
  const int tiles = ((bins->max_w + kTile - 1) / kTile) * ((bins->max_h + kTile - 1) / kTile);
  k_wboit<<<tiles, 256, 0, (cudaStream_t)stream>>>(bins_view(*bins), znear, zfar, bg[0], bg[1], bg[2],
                                                   reinterpret_cast<float4 *>(rgba32f), rgba8);
  return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
}

namespace star {
// Loads this file's kernels onto the current device (see star_nt_preload).
cudaError_t preload_baselines() {
  cudaFuncAttributes a;
  cudaError_t e = cudaSuccess, r;
  if ((r = cudaFuncGetAttributes(&a, k_unsorted_over)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_wboit)) != cudaSuccess) e = r;
  return e;
}
}  // namespace star
