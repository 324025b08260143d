// pass_body.cuh -- one geometry pass over one 16 x 16 tile (Sec. 3, Sec. 3.3):
// the per-pixel state of the nearest, second-nearest and tail-statistics
// passes and the tile traversal that feeds it.
//
// Tail statistics are accumulated over every fragment and the two nearest
// are subtracted at the end: all sums are exact integers, and the tail
// transmittance is carried as an integer sum of fixed-point -log2(1 - alpha)
// (2^-32 units) plus a count of opaque fragments, so the result does not
// depend on the order in which fragments arrive.
#pragma once

#include <math.h>

#include "common.cuh"
#include "features.cuh"
#include "raster_tile.cuh"
#include "tile_walk.cuh"

namespace star {

// kFusedDfaoit: the plain pipeline's single pass with the network input of
// the DFAOIT comparison network (its tail sums add the straight colours).
enum PassMode { kTop1 = 1, kTop2 = 2, kTail = 3, kFused = 4, kFusedDfaoit = 5 };

// r8 | g8 << 21 | b8 << 42: per-channel sums of straight colours fit 21 bits
// for up to 8224 fragments per pixel
__device__ __forceinline__ unsigned long long spread_rgb(uint32_t c8) {
  return (unsigned long long)(c8 & 255u) | ((unsigned long long)((c8 >> 8) & 255u) << 21) |
         ((unsigned long long)((c8 >> 16) & 255u) << 42);
}

struct PassOut {
  int32_t *id1;
  float *z1;
  int32_t *id2;
  uint32_t *n;
  uint4 *tail;
  float *t_tail;
};

// Per-thread state of one geometry pass over one tile.  MODE selects what is
// kept: the nearest fragment, the two nearest, the two nearest plus tail sums,
// or all of it plus the full-resolution network input (fused plain pipeline).
struct PassAcc {
  float z1, z2;
  int i1, i2;
  uint32_t N;
  unsigned long long rg, ba, lg;
  unsigned long long cs;  // straight colour sums (kFusedDfaoit only)

  __device__ __forceinline__ void reset() {
    z1 = z2 = INFINITY;
    i1 = i2 = 0x7fffffff;
    N = 0u;
    rg = ba = lg = 0ull;
    cs = 0ull;
  }

  // A fragment deeper than the current k-th nearest cannot enter the top k:
  // the passes without tail sums let the warp skip a triangle whose depth
  // lower bound exceeds every lane's k-th depth (lanes outside the target
  // never store, so they never hold a skip back); the tail passes must see
  // every fragment and only skip the depth of such fragments.
  template <int MODE>
  __device__ __forceinline__ float bound(bool inside) const {
    if (MODE >= kTail) return INFINITY;
    return inside ? (MODE == kTop1 ? z1 : z2) : -INFINITY;
  }

  // A fragment of T: the tail sums (MODE >= kTail).
  template <int MODE>
  __device__ __forceinline__ void accumulate(const TriSetup &T) {
    ++N;
    rg += T.rg;
    ba += T.ba;
    lg += T.lg;
    if (MODE == kFusedDfaoit) cs += spread_rgb(T.c8);
  }

  // A fragment with the tail constants rg, ba, lg (and colour c8) of its
  // triangle, loaded once by the caller.
  template <int MODE>
  __device__ __forceinline__ void accumulate_terms(unsigned long long trg, unsigned long long tba,
                                                   unsigned long long tlg, uint32_t c8) {
    ++N;
    rg += trg;
    ba += tba;
    lg += tlg;
    if (MODE == kFusedDfaoit) cs += spread_rgb(c8);
  }

  // A fragment at depth z offered to the KM nearest, ordered by (depth, id).
  template <int KM>
  __device__ __forceinline__ void insert(float z, int id) {
    const bool lt1 = z < z1 || (z == z1 && id < i1);
    if (KM == kTop1) {
      z1 = lt1 ? z : z1;
      i1 = lt1 ? id : i1;
    } else {
      // (z1, i1) precedes (z2, i2), so lt1 implies lt2
      const bool lt2 = z < z2 || (z == z2 && id < i2);
      const float nz2 = lt1 ? z1 : z;
      const int ni2 = lt1 ? i1 : id;
      z2 = lt2 ? nz2 : z2;
      i2 = lt2 ? ni2 : i2;
      z1 = lt1 ? z : z1;
      i1 = lt1 ? id : i1;
    }
  }

  template <int MODE>
  __device__ __forceinline__ void visit(const TriSetup &T, int id, long long e0, long long e2) {
    if (MODE >= kTail) accumulate<MODE>(T);
    if (MODE == kTop1) insert<kTop1>(frag_depth(T, e0, e2), id);
    else if (!(T.zlo > z2)) insert<kTop2>(frag_depth(T, e0, e2), id);
  }

  // Network input and front terms of pixel p once every pass ran at the full
  // resolution (MODE kTail): the tail sums less the two nearest fragments, as
  // finish<kFused> computes them; id1 and z1 are stored when po asks for them.
  __device__ __forceinline__ void resolve_terms(const TriSetup *__restrict__ setups,
                                                const uint32_t *__restrict__ rgba8, const PassOut &po,
                                                float bg0, float bg1, float bg2, float kappa, size_t p,
                                                float (&xv)[6], float4 &fr) {
    const bool has1 = i1 != 0x7fffffff, has2 = i2 != 0x7fffffff;
    if (po.id1) po.id1[p] = has1 ? i1 : -1;
    if (po.z1) po.z1[p] = has1 ? z1 : 1.0f;
    if (has1) {
      const TriSetup &S = setups[i1];
      rg -= S.rg; ba -= S.ba; lg -= S.lg;
    }
    if (has2) {
      const TriSetup &S = setups[i2];
      rg -= S.rg; ba -= S.ba; lg -= S.lg;
    }
    const uint32_t A = (uint32_t)(ba >> 32), Sr = (uint32_t)rg, Sg = (uint32_t)(rg >> 32),
                   Sb = (uint32_t)ba;
    const float t = tail_transmittance(lg, 0u);
    float r1 = 0, g1 = 0, b1 = 0, a1 = 0, r2 = 0, g2 = 0, b2 = 0, a2 = 0;
    if (has1) unpack_rgba(__ldg(rgba8 + i1), r1, g1, b1, a1);
    if (has2) unpack_rgba(__ldg(rgba8 + i2), r2, g2, b2, a2);
    feature_terms(a1, r1, g1, b1, a2 * r2, a2 * g2, a2 * b2, a2, (float)N, (float)A, (float)Sr,
                  (float)Sg, (float)Sb, t, N > 2, bg0, bg1, bg2, kappa, xv, fr);
  }

  // Planes of pixel p (tail sums less the two nearest fragments).
  template <int MODE>
  __device__ __forceinline__ void finish(const TriSetup *__restrict__ setups,
                                         const uint32_t *__restrict__ rgba8, const PassOut &po,
                                         const FeatOut &fo, size_t p) {
    const bool has1 = i1 != 0x7fffffff, has2 = i2 != 0x7fffffff;
    if (po.id1) po.id1[p] = has1 ? i1 : -1;
    if (po.z1) po.z1[p] = has1 ? z1 : 1.0f;
    if (MODE >= kTop2 && po.id2) po.id2[p] = has2 ? i2 : -1;
    if (MODE >= kTail) {
      if (has1) {
        const TriSetup &S = setups[i1];
        rg -= S.rg; ba -= S.ba; lg -= S.lg;
        if (MODE == kFusedDfaoit) cs -= spread_rgb(S.c8);
      }
      if (has2) {
        const TriSetup &S = setups[i2];
        rg -= S.rg; ba -= S.ba; lg -= S.lg;
        if (MODE == kFusedDfaoit) cs -= spread_rgb(S.c8);
      }
      const uint32_t A = (uint32_t)(ba >> 32), Sr = (uint32_t)rg, Sg = (uint32_t)(rg >> 32),
                     Sb = (uint32_t)ba;
      const float t = tail_transmittance(lg, 0u);
      if (po.n) po.n[p] = N;
      if (po.tail) po.tail[p] = make_uint4(A, Sr, Sg, Sb);
      if (po.t_tail) po.t_tail[p] = t;
      if (MODE == kFused || MODE == kFusedDfaoit) {
        float r1 = 0, g1 = 0, b1 = 0, a1 = 0, r2 = 0, g2 = 0, b2 = 0, a2 = 0;
        if (has1) unpack_rgba(__ldg(rgba8 + i1), r1, g1, b1, a1);
        if (has2) unpack_rgba(__ldg(rgba8 + i2), r2, g2, b2, a2);
        if (MODE == kFused)
          write_features(fo, p, a1, r1, g1, b1, a2 * r2, a2 * g2, a2 * b2, a2, (float)N, (float)A,
                         (float)Sr, (float)Sg, (float)Sb, t, N > 2);
        else
          write_dfaoit_features(fo, p, a1, r1, g1, b1, a2 * r2, a2 * g2, a2 * b2, a2, N, (float)A,
                                (float)Sr, (float)Sg, (float)Sb, (float)(uint32_t)(cs & 0x1FFFFFu),
                                (float)(uint32_t)((cs >> 21) & 0x1FFFFFu), (float)(uint32_t)(cs >> 42), t);
      }
    }
  }
};

// One geometry pass over one tile (one CTA; the tile's triangles staged in
// chunks by for_each_fragment).
template <int MODE, int BW = 8>
__device__ __forceinline__ void pass_body(const BinsView &bv, const uint32_t *__restrict__ rgba8,
                                          const PassOut &po, const FeatOut &fo, TileStage &stage,
                                          int tile) {
  const BinsHeader *hd = bv.hd;
  if ((int64_t)hd->n_pairs > bv.pair_capacity) return;
  if (tile >= hd->n_tiles) return;
  const int W = hd->size[0], H = hd->size[1];
  const TilePixel tp = tile_pixel<BW>(tile, hd->tiles_x);
  const bool inside = tp.px < W && tp.py < H;
  PassAcc acc;
  acc.reset();
  for_each_fragment<BW, true>(
      bv, tile, tp, stage, [&] { return acc.template bound<MODE>(inside); },
      [&](const TriSetup &T, uint32_t id, long long e0, long long e2) {
        acc.template visit<MODE>(T, (int)id, e0, e2);
      });
  if (!inside) return;
  acc.template finish<MODE>(bv.setups, rgba8, po, fo, (size_t)tp.py * W + tp.px);
}

// pass_body with two pixels per thread (a CTA of 128 threads per tile, see
// tile_pixel and walk_tile2): the triangle loads and the loop are shared by
// both pixels.
template <int MODE, int BW = 8>
__device__ __forceinline__ void pass_body2(const BinsView &bv, const uint32_t *__restrict__ rgba8,
                                           const PassOut &po, WalkStage &stage, int tile,
                                           const FeatOut &fo = FeatOut{}) {
  constexpr int BH = 32 / BW;
  const BinsHeader *hd = bv.hd;
  if ((int64_t)hd->n_pairs > bv.pair_capacity) return;
  if (tile >= hd->n_tiles) return;
  const int W = hd->size[0], H = hd->size[1];
  const TilePixel tp = tile_pixel<BW, 2>(tile, hd->tiles_x);
  const bool in0 = tp.px < W && tp.py < H, in1 = tp.px < W && tp.py + BH < H;
  PassAcc a0, a1;
  a0.reset();
  a1.reset();
  walk_tile2<MODE, BW>(bv, tile, tp, stage, in0, in1, a0, a1);
  if (in0) a0.template finish<MODE>(bv.setups, rgba8, po, fo, (size_t)tp.py * W + tp.px);
  if (in1) a1.template finish<MODE>(bv.setups, rgba8, po, fo, (size_t)(tp.py + BH) * W + tp.px);
}

}  // namespace star
