// features.cuh -- network input and front terms of a full-resolution pixel
// (Sec. 3.2 last paragraph, Sec. 3.3, Eq. 4): colour unpacking, the bilinear
// upscale of passes 2 and 3, and the stored layouts.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"
#include "qt_cells.cuh"

namespace star {

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
  const float e = exp2f(-frac);
  // e in [0.5, 1]: e 2^-k is normal for k <= 125, where one multiply by 2^-k is exact
  return k <= 125u ? e * __int_as_float((int)(127u - k) << 23) : ldexpf(e, -(int)k);
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

// Network input x = [kappa N, t_tail, S / (255 A)] plus the tail flag, and
// the front terms (C_exact,2 + T_all C_b, T_2) of one full-resolution pixel.
__device__ __forceinline__ void feature_terms(float a1, float r1, float g1, float b1, float pr2,
                                              float pg2, float pb2, float a2, float n, float A,
                                              float Sr, float Sg, float Sb, float t, bool flag,
                                              float bg0, float bg1, float bg2, float kappa,
                                              float (&x)[6], float4 &fr) {
  const float T2 = (1.0f - a1) * (1.0f - a2);
  const float Tall = T2 * t;
  fr.x = a1 * r1 + (1.0f - a1) * pr2 + Tall * bg0;
  fr.y = a1 * g1 + (1.0f - a1) * pg2 + Tall * bg1;
  fr.z = a1 * b1 + (1.0f - a1) * pb2 + Tall * bg2;
  fr.w = T2;
  x[0] = n * kappa;
  x[1] = t;
  const float inv = A > 0.0f ? __frcp_rn(255.0f * A) : 0.0f;
  x[2] = Sr * inv;
  x[3] = Sg * inv;
  x[4] = Sb * inv;
  x[5] = flag ? 1.0f : 0.0f;
}

// Store a pixel's network input (x_dtype layout) and front terms.
__device__ __forceinline__ void store_features(const FeatOut &fo, size_t p, const float (&x)[6],
                                               const float4 &fr) {
  fo.front[p] = fr;
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

// Network input row and front terms of one full-resolution pixel, stored.
__device__ __forceinline__ void write_features(const FeatOut &fo, size_t p, float a1, float r1,
                                               float g1, float b1, float pr2, float pg2, float pb2,
                                               float a2, float n, float A, float Sr, float Sg,
                                               float Sb, float t, bool flag) {
  float x[6];
  float4 fr;
  feature_terms(a1, r1, g1, b1, pr2, pg2, pb2, a2, n, A, Sr, Sg, Sb, t, flag, fo.bg0, fo.bg1, fo.bg2,
                fo.kappa, x, fr);
  store_features(fo, p, x, fr);
}

// Network input of the DFAOIT comparison network and its composite terms
// (Sec. 3.3: the features the paper lists for the original method), at full
// resolution: x = [a1 c1 + (1 - a1) a2 c2 (3), the tail's straight colour mean
// C / (255 m) (3) and opacity mean A / (255 m), the tail's premultiplied sum
// S / 255^2 (3), kappa N] with m = N - 2 tail fragments (means 0 without a
// tail), the flag N >= 1 at element 11; front = (T_all C_b, 1) with T_all =
// (1 - a1)(1 - a2) t_tail, so that star_nt_composite gives C_t + T_all C_b.
// x: [P][16] float32 or bfloat16.
__device__ __forceinline__ void write_dfaoit_features(const FeatOut &fo, size_t p, float a1, float r1,
                                                      float g1, float b1, float pr2, float pg2, float pb2,
                                                      float a2, uint32_t N, float A, float Sr, float Sg,
                                                      float Sb, float Cr, float Cg, float Cb, float t) {
  float x[16];
  x[0] = a1 * r1 + (1.0f - a1) * pr2;
  x[1] = a1 * g1 + (1.0f - a1) * pg2;
  x[2] = a1 * b1 + (1.0f - a1) * pb2;
  const float inv_m = N > 2 ? __frcp_rn(255.0f * (float)(N - 2)) : 0.0f;
  constexpr float k255sq = 1.0f / 65025.0f;
  x[3] = Cr * inv_m;
  x[4] = Cg * inv_m;
  x[5] = Cb * inv_m;
  x[6] = A * inv_m;
  x[7] = Sr * k255sq;
  x[8] = Sg * k255sq;
  x[9] = Sb * k255sq;
  x[10] = (float)N * fo.kappa;
  x[11] = N >= 1 ? 1.0f : 0.0f;
#pragma unroll
  for (int k = 12; k < 16; ++k) x[k] = 0.0f;
  const float Tall = (1.0f - a1) * (1.0f - a2) * t;
  fo.front[p] = make_float4(Tall * fo.bg0, Tall * fo.bg1, Tall * fo.bg2, 1.0f);
  if (fo.x_dtype == STAR_NT_F32) {
    float4 *X = reinterpret_cast<float4 *>(fo.x) + 4 * p;
#pragma unroll
    for (int q = 0; q < 4; ++q) X[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
  } else {
    uint32_t h[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      __nv_bfloat162 v = __floats2bfloat162_rn(x[2 * q], x[2 * q + 1]);
      h[q] = *reinterpret_cast<uint32_t *>(&v);
    }
    uint4 *X = reinterpret_cast<uint4 *>(fo.x) + 2 * p;
    X[0] = make_uint4(h[0], h[1], h[2], h[3]);
    X[1] = make_uint4(h[4], h[5], h[6], h[7]);
  }
}

// Inputs of the full-resolution features: pass 1 at full resolution, passes
// 2 and 3 at their own resolutions (read from their bins headers).
struct FeatIn {
  int W, H;
  const BinsHeader *hd2, *hd3;
  const uint32_t *rgba8;
  const int32_t *id1, *id2;
  const uint32_t *n3;
  const uint4 *tail3;
  const float *t3;

  // nothing to do: a pass was rejected by its raster, or the pass launch
  // already produced the frame (the three words are loaded together: a CTA
  // that returns at once waits for one round trip, not three)
  __device__ __forceinline__ bool rejected() const {
    const int r = hd2->resolved, n2 = hd2->n_pixels, n3 = hd3->n_pixels;
    return (r != 0) | (n2 <= 0) | (n3 <= 0);
  }
};

// Per-leaf variant: pass 2 and pass 3 of pixel (x, y) come from the targets
// that the level of its quadtree leaf maps them to (per-pixel lookups in the
// kernel's parameter memory).
constexpr int kLeafMaxTargets = STAR_NT_LEAF_MAX_TARGETS;
struct FeatInLeaf {
  int W, H;
  int B, tiles_x;                       // quadtree base tile side, tiles per row
  uint32_t n_tris;                      // ids read from the planes are checked against it
  const uint32_t *masks;
  const uint32_t *rgba8;
  const int32_t *id1;
  int32_t target_of[2][4];              // [pass 2, pass 3][level]
  int32_t size[kLeafMaxTargets][2];
  const int32_t *id2[kLeafMaxTargets];
  const uint32_t *n3[kLeafMaxTargets];
  const uint4 *tail3[kLeafMaxTargets];
  const float *t3[kLeafMaxTargets];

  __device__ __forceinline__ bool rejected() const { return false; }
};

// Plane samples of one pixel: its pass-1 id, the ids at its four pass-2
// bilinear taps and the pass-3 planes at its four pass-3 taps (taps ordered
// (i0, j0), (i1, j0), (i0, j1), (i1, j1)).
struct PixelTaps {
  int i1;
  int i2[4];
  uint32_t nn[4];
  uint4 tl[4];
  float tt[4];
};

// Network input x[0..5] (x5 = tail flag) and front terms from a pixel's taps
// and bilinear axes (pass 2: ax2, ay2; pass 3: ax3, ay3).  Zero bilinear
// weights drop their samples exactly (so a tap of weight zero may hold any
// value); a second-layer id is used only below id_limit (0x80000000: any
// id >= 0).
__device__ __forceinline__ void features_from_taps(const PixelTaps &tp, const Axis &ax2,
                                                   const Axis &ay2, const Axis &ax3, const Axis &ay3,
                                                   const uint32_t *__restrict__ rgba8,
                                                   uint32_t id_limit, float bg0, float bg1,
                                                   float bg2, float kappa, float (&xo)[6],
                                                   float4 &front) {
  // colour gathers (independent of each other)
  const uint32_t c1 = tp.i1 >= 0 ? __ldg(rgba8 + tp.i1) : 0u;
  uint32_t c2[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) c2[k] = (uint32_t)tp.i2[k] < id_limit ? __ldg(rgba8 + tp.i2[k]) : 0u;

  float r1, g1, b1, a1;
  unpack_rgba(c1, r1, g1, b1, a1);
  const float rx = __frcp_rn((float)ax2.den), ry = __frcp_rn((float)ay2.den);
  const float wx2 = (float)ax2.rem * rx, wy2 = (float)ay2.rem * ry;
  const float w2[4] = {(1.0f - wy2) * (1.0f - wx2), (1.0f - wy2) * wx2, wy2 * (1.0f - wx2), wy2 * wx2};
  float L2[4] = {0, 0, 0, 0};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (w2[k] == 0.0f || (uint32_t)tp.i2[k] >= id_limit) continue;
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
    nf += w3[k] * (float)tp.nn[k];
    A += w3[k] * (float)tp.tl[k].x;
    Sr += w3[k] * (float)tp.tl[k].y;
    Sg += w3[k] * (float)tp.tl[k].z;
    Sb += w3[k] * (float)tp.tl[k].w;
    t += w3[k] * tp.tt[k];
    nexact += wi3[k] * (long long)tp.nn[k];
  }
  const bool flag = nexact > 2LL * ax3.den * ay3.den;
  feature_terms(a1, r1, g1, b1, L2[0], L2[1], L2[2], L2[3], nf, A, Sr, Sg, Sb, t, flag, bg0, bg1, bg2,
                kappa, xo, front);
}

// Network input and front terms of pixel (x, y), with pass 2 (W2 x H2) and
// pass 3 (W3 x H3) upscaled bilinearly from the planes in global memory.
// All plane loads are issued before any of them is used (the sample indices
// are clamped, so every load is valid) to keep many requests in flight.  A
// pass at the full size upscales by the identity (tap 0 with weight 1, the
// others with weight 0), so only tap 0 is read; the test is uniform over the
// launch.
__device__ __forceinline__ void pixel_features_at(
    int W, int H, const uint32_t *__restrict__ rgba8, const int32_t *__restrict__ id1,
    int W2, int H2, const int32_t *__restrict__ id2, int W3, int H3,
    const uint32_t *__restrict__ n3, const uint4 *__restrict__ tail3,
    const float *__restrict__ t3, uint32_t id_limit, float bg0, float bg1, float bg2,
    float kappa, int x, int y, float (&xo)[6], float4 &front) {
  const size_t p = (size_t)y * W + x;
  const Axis ax2 = upscale_axis(x, W2, W), ay2 = upscale_axis(y, H2, H);
  const Axis ax3 = upscale_axis(x, W3, W), ay3 = upscale_axis(y, H3, H);
  size_t q2[4], q3[4];
  q2[0] = (size_t)ay2.i0 * W2 + ax2.i0; q2[1] = (size_t)ay2.i0 * W2 + ax2.i1;
  q2[2] = (size_t)ay2.i1 * W2 + ax2.i0; q2[3] = (size_t)ay2.i1 * W2 + ax2.i1;
  q3[0] = (size_t)ay3.i0 * W3 + ax3.i0; q3[1] = (size_t)ay3.i0 * W3 + ax3.i1;
  q3[2] = (size_t)ay3.i1 * W3 + ax3.i0; q3[3] = (size_t)ay3.i1 * W3 + ax3.i1;
  const bool full2 = W2 == W && H2 == H, full3 = W3 == W && H3 == H;
  PixelTaps tp;
  tp.i1 = __ldg(id1 + p);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (k == 0 || !full2) {
      tp.i2[k] = __ldg(id2 + q2[k]);
    } else {
      tp.i2[k] = -1;
    }
    if (k == 0 || !full3) {
      tp.nn[k] = __ldg(n3 + q3[k]);
      tp.tl[k] = __ldg(tail3 + q3[k]);
      tp.tt[k] = __ldg(t3 + q3[k]);
    } else {
      tp.nn[k] = 0u;
      tp.tl[k] = make_uint4(0u, 0u, 0u, 0u);
      tp.tt[k] = 0.0f;
    }
  }
  features_from_taps(tp, ax2, ay2, ax3, ay3, rgba8, id_limit, bg0, bg1, bg2, kappa, xo, front);
}

// Global pass sizes (Eq. 2 over the frame), read from the bins headers.
__device__ __forceinline__ void pixel_features(const FeatIn &in, float bg0, float bg1, float bg2,
                                               float kappa, int x, int y, float (&xo)[6],
                                               float4 &front) {
  pixel_features_at(in.W, in.H, in.rgba8, in.id1, in.hd2->size[0], in.hd2->size[1], in.id2,
                    in.hd3->size[0], in.hd3->size[1], in.n3, in.tail3, in.t3, 0x80000000u, bg0, bg1,
                    bg2, kappa, x, y, xo, front);
}

// Per-leaf pass sizes: the targets of the level of the pixel's leaf.
__device__ __forceinline__ void pixel_features(const FeatInLeaf &in, float bg0, float bg1, float bg2,
                                               float kappa, int x, int y, float (&xo)[6],
                                               float4 &front) {
  const int B = in.B;
  const uint32_t m = __ldg(in.masks + (y / B) * in.tiles_x + x / B);
  const int l = leaf_level(m, x % B, y % B, B);
  const int k2 = in.target_of[0][l], k3 = in.target_of[1][l];
  pixel_features_at(in.W, in.H, in.rgba8, in.id1, in.size[k2][0], in.size[k2][1], in.id2[k2],
                    in.size[k3][0], in.size[k3][1], in.n3[k3], in.tail3[k3], in.t3[k3], in.n_tris,
                    bg0, bg1, bg2, kappa, x, y, xo, front);
}


}  // namespace star
