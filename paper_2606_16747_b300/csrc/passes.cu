// passes.cu -- star_nt_build_inputs: the three geometry passes (nearest,
// second-nearest, tail statistics; Sec. 3, Sec. 3.3), the bilinear upscale of
// the reduced passes (Sec. 3.2) and the network input / front terms of
// Eq. 4.
//
// Tail statistics are accumulated over every fragment and the two nearest
// are subtracted at the end: all sums are exact integers, and the tail
// transmittance is carried as an integer sum of fixed-point -log2(1 - alpha)
// (2^-32 units) plus a count of opaque fragments, so the result does not
// depend on the order in which fragments arrive.
#include <math.h>

#include <cuda_bf16.h>

#include "common.cuh"
#include "raster_tile.cuh"

namespace star {

enum PassMode { kTop1 = 1, kTop2 = 2, kTail = 3, kFused = 4 };

struct PassOut {
  int32_t *id1;
  float *z1;
  int32_t *id2;
  uint32_t *n;
  uint4 *tail;
  float *t_tail;
};

struct FeatOut {
  void *x;
  int x_dtype;
  float4 *front;
  float bg0, bg1, bg2;
  float kappa;
};

__device__ __forceinline__ float tail_transmittance(unsigned long long lg, uint32_t opq) {
  if (opq) return 0.0f;
  const uint32_t k = (uint32_t)(lg >> 32);
  if (k >= 160u) return 0.0f;
  const float frac = __uint2float_rn((uint32_t)lg) * 2.3283064365386963e-10f;  // 2^-32
  return ldexpf(exp2f(-frac), -(int)k);
}

// straight RGBA8 to float (c8 / 255, by a multiply: within one rounding of
// the quotient)
__device__ __forceinline__ void unpack_rgba(uint32_t c, float &r, float &g, float &b, float &a) {
  constexpr float k = 1.0f / 255.0f;
  r = (float)(c & 255u) * k;
  g = (float)((c >> 8) & 255u) * k;
  b = (float)((c >> 16) & 255u) * k;
  a = (float)(c >> 24) * k;
}

// Network input row and front terms of one full-resolution pixel.
__device__ __forceinline__ void write_features(const FeatOut &fo, size_t p, float a1, float r1,
                                               float g1, float b1, float pr2, float pg2, float pb2,
                                               float a2, float n, float A, float Sr, float Sg,
                                               float Sb, float t, bool flag) {
  const float T2 = (1.0f - a1) * (1.0f - a2);
  const float Tall = T2 * t;
  float4 fr;
  fr.x = a1 * r1 + (1.0f - a1) * pr2 + Tall * fo.bg0;
  fr.y = a1 * g1 + (1.0f - a1) * pg2 + Tall * fo.bg1;
  fr.z = a1 * b1 + (1.0f - a1) * pb2 + Tall * fo.bg2;
  fr.w = T2;
  fo.front[p] = fr;
  float x[6];
  x[0] = n * fo.kappa;
  x[1] = t;
  const float inv = A > 0.0f ? __frcp_rn(255.0f * A) : 0.0f;
  x[2] = Sr * inv;
  x[3] = Sg * inv;
  x[4] = Sb * inv;
  x[5] = flag ? 1.0f : 0.0f;
  if (fo.x_dtype == STAR_NT_F32) {
    float4 *X = reinterpret_cast<float4 *>(fo.x) + 2 * p;
    X[0] = make_float4(x[0], x[1], x[2], x[3]);
    X[1] = make_float4(x[4], x[5], 0.0f, 0.0f);
  } else {
    __nv_bfloat162 h0 = __floats2bfloat162_rn(x[0], x[1]);
    __nv_bfloat162 h1 = __floats2bfloat162_rn(x[2], x[3]);
    __nv_bfloat162 h2 = __floats2bfloat162_rn(x[4], x[5]);
    uint4 v;
    v.x = *reinterpret_cast<uint32_t *>(&h0);
    v.y = *reinterpret_cast<uint32_t *>(&h1);
    v.z = *reinterpret_cast<uint32_t *>(&h2);
    v.w = 0u;
    reinterpret_cast<uint4 *>(fo.x)[p] = v;
  }
}

// One geometry pass over one tile.  MODE selects what is kept: the nearest
// fragment, the two nearest, the two nearest plus tail sums, or all of it
// plus the full-resolution network input (fused plain pipeline).
template <int MODE>
__device__ __forceinline__ void pass_body(const BinsView &bv, const uint32_t *__restrict__ rgba8,
                                          const PassOut &po, const FeatOut &fo, TileStage &stage) {
  const BinsHeader *hd = bv.hd;
  if ((int64_t)hd->n_pairs > bv.pair_capacity) return;
  const int tile = blockIdx.x;
  if (tile >= hd->n_tiles) return;
  const int W = hd->size[0], H = hd->size[1];
  const TilePixel tp = tile_pixel(tile, hd->tiles_x);

  float z1 = INFINITY, z2 = INFINITY;
  int i1 = 0x7fffffff, i2 = 0x7fffffff;
  uint32_t N = 0, opq = 0;
  unsigned long long rg = 0, ba = 0, lg = 0;
  for_each_fragment(bv, tile, tp, stage, [&](const TriSetup &T, uint32_t id_u, float z) {
    const int id = (int)id_u;
    if (MODE == kTop1) {
      if (z < z1 || (z == z1 && id < i1)) { z1 = z; i1 = id; }
    } else {
      if (z < z2 || (z == z2 && id < i2)) {
        if (z < z1 || (z == z1 && id < i1)) {
          z2 = z1; i2 = i1; z1 = z; i1 = id;
        } else {
          z2 = z; i2 = id;
        }
      }
    }
    if (MODE >= kTail) {
      ++N;
      rg += T.rg;
      ba += T.ba;
      lg += T.lg;
      opq += T.opq;
    }
  });
  if (tp.px >= W || tp.py >= H) return;
  const size_t p = (size_t)tp.py * W + tp.px;
  const bool has1 = i1 != 0x7fffffff, has2 = i2 != 0x7fffffff;
  if (po.id1) po.id1[p] = has1 ? i1 : -1;
  if (po.z1) po.z1[p] = has1 ? z1 : 1.0f;
  if (MODE >= kTop2 && po.id2) po.id2[p] = has2 ? i2 : -1;
  if (MODE >= kTail) {
    // remove the two nearest fragments from the all-fragment sums
    if (has1) {
      const TriSetup &S = bv.setups[i1];
      rg -= S.rg; ba -= S.ba; lg -= S.lg; opq -= S.opq;
    }
    if (has2) {
      const TriSetup &S = bv.setups[i2];
      rg -= S.rg; ba -= S.ba; lg -= S.lg; opq -= S.opq;
    }
    const uint32_t A = (uint32_t)(ba >> 32), Sr = (uint32_t)rg, Sg = (uint32_t)(rg >> 32),
                   Sb = (uint32_t)ba;
    const float t = tail_transmittance(lg, opq);
    if (po.n) po.n[p] = N;
    if (po.tail) po.tail[p] = make_uint4(A, Sr, Sg, Sb);
    if (po.t_tail) po.t_tail[p] = t;
    if (MODE == kFused) {
      float r1 = 0, g1 = 0, b1 = 0, a1 = 0, r2 = 0, g2 = 0, b2 = 0, a2 = 0;
      if (has1) unpack_rgba(__ldg(rgba8 + i1), r1, g1, b1, a1);
      if (has2) unpack_rgba(__ldg(rgba8 + i2), r2, g2, b2, a2);
      write_features(fo, p, a1, r1, g1, b1, a2 * r2, a2 * g2, a2 * b2, a2, (float)N, (float)A,
                     (float)Sr, (float)Sg, (float)Sb, t, N > 2);
    }
  }
}

template <int MODE>
__global__ void __launch_bounds__(256) k_pass(BinsView bv, const uint32_t *__restrict__ rgba8,
                                              PassOut po, FeatOut fo) {
  __shared__ TileStage stage;
  pass_body<MODE>(bv, rgba8, po, fo, stage);
}

// Pass 1 at full resolution; when pass 2 and/or pass 3 are marked merged
// (their size equals the full size) it keeps the two nearest fragments and
// the tail sums as well and writes their planes at full resolution.
__global__ void __launch_bounds__(256, 6) k_pass_merged(BinsView bv, const BinsHeader *hd2,
                                                     const BinsHeader *hd3,
                                                     const uint32_t *__restrict__ rgba8, PassOut o1,
                                                     PassOut o2, PassOut o3) {
  __shared__ TileStage stage;
  const bool m2 = hd2->merged != 0, m3 = hd3->merged != 0;
  if (!m2 && !m3) {
    pass_body<kTop1>(bv, rgba8, o1, FeatOut{}, stage);
    return;
  }
  PassOut o = o1;
  o.id2 = m2 ? o2.id2 : nullptr;
  o.n = m3 ? o3.n : nullptr;
  o.tail = m3 ? o3.tail : nullptr;
  o.t_tail = m3 ? o3.t_tail : nullptr;
  pass_body<kTail>(bv, rgba8, o, FeatOut{}, stage);
}

// Full-resolution features from pass 1 (full res) and the bilinear upscale
// of passes 2 and 3 (their own resolutions, read from their bins headers).
// All plane loads are issued before any of them is used (the sample indices
// are clamped, so every load is valid) to keep many requests in flight; zero
// bilinear weights then drop their samples exactly.
__global__ void __launch_bounds__(256) k_features(int W, int H, const BinsHeader *hd2,
                                                  const BinsHeader *hd3,
                                                  const uint32_t *__restrict__ rgba8,
                                                  const int32_t *__restrict__ id1,
                                                  const int32_t *__restrict__ id2,
                                                  const uint32_t *__restrict__ n3,
                                                  const uint4 *__restrict__ tail3,
                                                  const float *__restrict__ t3, FeatOut fo) {
  const int x = blockIdx.x * 32 + (threadIdx.x & 31);
  const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
  if (x >= W || y >= H) return;
  if (hd2->n_pixels <= 0 || hd3->n_pixels <= 0) return;  // a pass was rejected
  const size_t p = (size_t)y * W + x;
  const int W2 = hd2->size[0], H2 = hd2->size[1];
  const int W3 = hd3->size[0], H3 = hd3->size[1];
  const Axis ax2 = upscale_axis(x, W2, W), ay2 = upscale_axis(y, H2, H);
  const Axis ax3 = upscale_axis(x, W3, W), ay3 = upscale_axis(y, H3, H);
  size_t q2[4], q3[4];
  q2[0] = (size_t)ay2.i0 * W2 + ax2.i0; q2[1] = (size_t)ay2.i0 * W2 + ax2.i1;
  q2[2] = (size_t)ay2.i1 * W2 + ax2.i0; q2[3] = (size_t)ay2.i1 * W2 + ax2.i1;
  q3[0] = (size_t)ay3.i0 * W3 + ax3.i0; q3[1] = (size_t)ay3.i0 * W3 + ax3.i1;
  q3[2] = (size_t)ay3.i1 * W3 + ax3.i0; q3[3] = (size_t)ay3.i1 * W3 + ax3.i1;
  // issue every plane load
  const int i1 = __ldg(id1 + p);
  int i2[4];
  uint32_t nn[4];
  uint4 tl[4];
  float tt[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    i2[k] = __ldg(id2 + q2[k]);
    nn[k] = __ldg(n3 + q3[k]);
    tl[k] = __ldg(tail3 + q3[k]);
    tt[k] = __ldg(t3 + q3[k]);
  }
  // colour gathers (independent of each other)
  const uint32_t c1 = i1 >= 0 ? __ldg(rgba8 + i1) : 0u;
  uint32_t c2[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) c2[k] = i2[k] >= 0 ? __ldg(rgba8 + i2[k]) : 0u;

  float r1, g1, b1, a1;
  unpack_rgba(c1, r1, g1, b1, a1);
  const float rx = __frcp_rn((float)ax2.den), ry = __frcp_rn((float)ay2.den);
  const float wx2 = (float)ax2.rem * rx, wy2 = (float)ay2.rem * ry;
  const float w2[4] = {(1.0f - wy2) * (1.0f - wx2), (1.0f - wy2) * wx2, wy2 * (1.0f - wx2), wy2 * wx2};
  float L2[4] = {0, 0, 0, 0};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (w2[k] == 0.0f || i2[k] < 0) continue;
    float r, g, b, a;
    unpack_rgba(c2[k], r, g, b, a);
    L2[0] += w2[k] * (a * r);
    L2[1] += w2[k] * (a * g);
    L2[2] += w2[k] * (a * b);
    L2[3] += w2[k] * a;
  }
  const float wx3 = (float)ax3.rem * rx, wy3 = (float)ay3.rem * ry;  // same denominators 2W, 2H
  const float w3[4] = {(1.0f - wy3) * (1.0f - wx3), (1.0f - wy3) * wx3, wy3 * (1.0f - wx3), wy3 * wx3};
  const long long wi3[4] = {(long long)(ay3.den - ay3.rem) * (ax3.den - ax3.rem),
                            (long long)(ay3.den - ay3.rem) * ax3.rem,
                            (long long)ay3.rem * (ax3.den - ax3.rem), (long long)ay3.rem * ax3.rem};
  float nf = 0, A = 0, Sr = 0, Sg = 0, Sb = 0, t = 0;
  long long nexact = 0;  // upscaled N times (2W)(2H), exact
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (wi3[k] == 0) continue;  // exact zero weight
    nf += w3[k] * (float)nn[k];
    A += w3[k] * (float)tl[k].x;
    Sr += w3[k] * (float)tl[k].y;
    Sg += w3[k] * (float)tl[k].z;
    Sb += w3[k] * (float)tl[k].w;
    t += w3[k] * tt[k];
    nexact += wi3[k] * (long long)nn[k];
  }
  const bool flag = nexact > 2LL * ax3.den * ay3.den;
  write_features(fo, p, a1, r1, g1, b1, L2[0], L2[1], L2[2], L2[3], nf, A, Sr, Sg, Sb, t, flag);
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
      k_pass<kTop1><<<tiles, 256, 0, st>>>(v, scene->rgba8, o, fo);
      break;
    case 2:
      if (!layers->id2) return STAR_NT_ERR_ARG;
      k_pass<kTop2><<<tiles, 256, 0, st>>>(v, scene->rgba8, o, fo);
      break;
    case 3:
      if (!layers->n || !layers->tail || !layers->t_tail) return STAR_NT_ERR_ARG;
      k_pass<kTail><<<tiles, 256, 0, st>>>(v, scene->rgba8, o, fo);
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
  k_pass_merged<<<tiles_of(b1), 256, 0, (cudaStream_t)stream>>>(v1, v2.hd, v3.hd, scene->rgba8, o1,
                                                                pass_out(l2), pass_out(l3));
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
  k_features<<<grid, 256, 0, (cudaStream_t)stream>>>(W, H, v2.hd, v3.hd, scene->rgba8, l1->id1, l2->id2,
                                                     l3->n, reinterpret_cast<const uint4 *>(l3->tail),
                                                     l3->t_tail, fo);
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
    k_pass<kFused><<<tiles_of(b1), 256, 0, (cudaStream_t)stream>>>(v1, scene->rgba8, pass_out(l1), fo);
    return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
  }
  if (!l1 || !l1->id1 || !l2 || !l2->id2 || !l3 || !l3->n || !l3->tail || !l3->t_tail)
    return STAR_NT_ERR_ARG;
  star_nt_layers a = *l1, b = {}, c = {};
  b.id2 = l2->id2;
  c.n = l3->n;
  c.tail = l3->tail;
  c.t_tail = l3->t_tail;
  a.id2 = nullptr; a.n = nullptr; a.tail = nullptr; a.t_tail = nullptr;
  star_nt_status s;
  if ((s = star_nt_geometry_pass_merged(scene, b1, b2, b3, l1, l2, l3, d_status, stream)) !=
      STAR_NT_OK)
    return s;
  if ((s = star_nt_geometry_pass(scene, b2, 2, &b, d_status, stream)) != STAR_NT_OK) return s;
  if ((s = star_nt_geometry_pass(scene, b3, 3, &c, d_status, stream)) != STAR_NT_OK) return s;
  return star_nt_upscale_features(scene, b2, b3, l1, l2, l3, W, H, params, out, stream);
}
