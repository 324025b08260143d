// raster_tile.cuh -- per-tile fragment traversal shared by the geometry-pass
// kernels.  One CTA of 256 threads owns one 16 x 16-pixel tile; each warp owns
// a BW x (32 / BW) block of it (BW = 8 by default, the tile shape the tuner
// chooses from) and lane l the pixel (l % BW, l / BW) of that block.  The tile's binned triangles are staged in shared
// memory kChunk at a time.  Each warp then classifies the staged triangles
// for its own block, one triangle per lane (bounding box, then the three edge
// functions at the block's most favourable pixel centre, exact in int64),
// compacts the hits into a warp-private list with a ballot, and walks only
// that list, evaluating the three exact edge functions at its pixels.
#pragma once

#include "common.cuh"

namespace star {

struct TilePixel {
  int px, py;    // pixel of this thread
  int bx0, by0;  // origin of this warp's 8 x 4 block
  int tx0, ty0;  // origin of the tile
};

// PIX = 2: a CTA of 128 threads owns the tile; warp w owns a BW x (64 / BW)
// block and lane l the pixels (l % BW, l / BW) and (l % BW, l / BW + 32 / BW)
// of it (px, py is the first).
template <int BW = 8, int PIX = 1>
__device__ __forceinline__ TilePixel tile_pixel(int tile, int tiles_x) {
  constexpr int BH = 32 / BW, PER_ROW = kTile / BW;
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  TilePixel t;
  t.tx0 = tx * kTile;
  t.ty0 = ty * kTile;
  t.bx0 = t.tx0 + (w % PER_ROW) * BW;
  t.by0 = t.ty0 + (w / PER_ROW) * (PIX * BH);
  t.px = t.bx0 + (l % BW);
  t.py = t.by0 + (l / BW);
  return t;
}

// Canonical float32 depth of a covered pixel: b1 = E_20 / A, b2 = E_01 / A,
// z = (z0 + b1 dz1) + b2 dz2, one rounding per operation, -0 folded to +0.
// The edge values of a covered pixel lie in [0, A]; when A fits int32 they
// are converted as int32 (the same correctly rounded float; the int64
// conversion runs on the float64 pipe, which is narrow on this part).
__device__ __forceinline__ float frag_depth(const TriSetup &T, long long e0b, long long e2b) {
  const long long e01 = e0b - (long long)(T.own & 1u) + 1;
  const long long e20 = e2b - (long long)((T.own >> 2) & 1u) + 1;
  float f20, f01;
  if (T.own & kOwnSmall) {
    f20 = __int2float_rn((int)e20);
    f01 = __int2float_rn((int)e01);
  } else {
    f20 = __ll2float_rn(e20);
    f01 = __ll2float_rn(e01);
  }
  const float b1 = __fmul_rn(f20, T.r);
  const float b2 = __fmul_rn(f01, T.r);
  float z = __fadd_rn(__fadd_rn(T.z0, __fmul_rn(b1, T.dz1)), __fmul_rn(b2, T.dz2));
  return __fadd_rn(z, 0.0f);
}

// May the triangle cover a pixel centre of the BW x (32 / BW) block at
// (bx0, by0)?  False only when it certainly does not (bounding box, or one
// edge function negative at every centre of the block).
template <int BW = 8, int BH = 32 / BW>
__device__ __forceinline__ bool block_maybe(const TriSetup &T, int bx0, int by0) {
  if (T.xb < bx0 || T.xa > bx0 + BW - 1 || T.yb < by0 || T.ya > by0 + BH - 1) return false;
  const int Pxlo = bx0 * kSub + kSub / 2, Pxhi = Pxlo + (BW - 1) * kSub;
  const int Pylo = by0 * kSub + kSub / 2, Pyhi = Pylo + (BH - 1) * kSub;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const long long mx = T.c[e] + (long long)T.dx[e] * (T.dx[e] > 0 ? Pyhi : Pylo) -
                         (long long)T.dy[e] * (T.dy[e] > 0 ? Pxlo : Pxhi);
    if (mx < 0) return false;
  }
  return true;
}

// Shared-memory staging area of one tile CTA.
struct TileStage {
  TriSetup tri[kChunk];
  uint32_t id[kChunk];
  uint32_t src[kChunk];     // binned ids before the depth sort
  float key[kChunk];        // their depth lower bounds
  uint8_t rank[kChunk];     // staged position of each binned entry
  uint8_t list[8][kChunk];  // per-warp lists of staged triangle indices
};

// Calls visit(T, prim_id, e0, e2) for every triangle of the tile covering
// this thread's pixel centre, with the biased edge functions 0 and 2 there
// (frag_depth gives the fragment's depth from them).  Must be called by all
// 256 threads.
//
// bound() is this thread's depth bound: a staged triangle is skipped by the
// whole warp when its depth lower bound exceeds bound() on every lane (no
// fragment of it can then matter to the caller); return INFINITY to visit
// every fragment.  With SORTED, each staged chunk is ordered by depth lower
// bound (ties by binned position) first, so that near triangles come first
// and raise the bounds early; the set of fragments visited is the same.
//
// PIX = 2 (two pixels per thread, see tile_pixel): visit(j, T, prim_id, e0, e2)
// for pixel j of the thread; bound() is then the larger of its two bounds.
template <int BW = 8, bool SORTED = false, int PIX = 1, class Bound, class Visit>
__device__ __forceinline__ void for_each_fragment(const BinsView &bv, int tile, const TilePixel &tp,
                                                  TileStage &st, Bound &&bound, Visit &&visit) {
  constexpr int BH = 32 / BW;
  const int Px = tp.px * kSub + kSub / 2, Py = tp.py * kSub + kSub / 2;
  const int warp = threadIdx.x >> 5;
  const uint32_t beg = bv.tile_offset[tile], end = bv.tile_offset[tile + 1];
  for (uint32_t base = beg; base < end; base += kChunk) {
    const int n = (int)min((uint32_t)kChunk, end - base);
    __syncthreads();
    if (SORTED) {
      const int t = threadIdx.x;
      if (t < n) {
        const uint32_t id = __ldg(bv.pairs + base + t);
        st.src[t] = id;
        st.key[t] = __ldg(&bv.setups[id].zlo);
      }
      __syncthreads();
      if (t < n) {  // rank by (key, position): a permutation of 0 .. n-1
        const float kt = st.key[t];
        int r = 0;
        for (int j = 0; j < n; ++j) {
          const float kj = st.key[j];
          r += (kj < kt || (kj == kt && j < t)) ? 1 : 0;
        }
        st.rank[t] = (uint8_t)r;
      }
      __syncthreads();
      for (int i = threadIdx.x; i < n * 7; i += blockDim.x) {
        const int k = i / 7, part = i - 7 * k;
        const uint32_t id = st.src[k];
        const int d = st.rank[k];
        reinterpret_cast<uint4 *>(st.tri + d)[part] =
            __ldg(reinterpret_cast<const uint4 *>(bv.setups + id) + part);
        if (part == 0) st.id[d] = id;
      }
    } else {
      for (int i = threadIdx.x; i < n * 7; i += blockDim.x) {
        const int k = i / 7, part = i - 7 * k;
        const uint32_t id = __ldg(bv.pairs + base + k);
        reinterpret_cast<uint4 *>(st.tri + k)[part] =
            __ldg(reinterpret_cast<const uint4 *>(bv.setups + id) + part);
        if (part == 0) st.id[k] = id;
      }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    int m = 0;
    for (int k0 = 0; k0 < n; k0 += 32) {
      const int k = k0 + lane;
      const bool hit = k < n && block_maybe<BW, PIX * BH>(st.tri[k], tp.bx0, tp.by0);
      const uint32_t b = __ballot_sync(0xffffffffu, hit);
      if (hit) st.list[warp][m + __popc(b & ((1u << lane) - 1u))] = (uint8_t)k;
      m += __popc(b);
    }
    __syncwarp();
    for (int i = 0; i < m; ++i) {  // m is warp-uniform
      const int k = st.list[warp][i];
      const TriSetup &T = st.tri[k];
      if (__all_sync(0xffffffffu, T.zlo > bound())) continue;
      const long long e0 = (long long)T.dx[0] * Py + T.c[0] - (long long)T.dy[0] * Px;
      const long long e1 = (long long)T.dx[1] * Py + T.c[1] - (long long)T.dy[1] * Px;
      const long long e2 = (long long)T.dx[2] * Py + T.c[2] - (long long)T.dy[2] * Px;
      if constexpr (PIX == 1) {
        if ((e0 | e1 | e2) < 0) continue;
        visit(T, st.id[k], e0, e2);
      } else {
        // the second pixel, BH rows below: each edge function grows by dx BH kSub
        const long long f0 = e0 + (long long)T.dx[0] * (BH * kSub);
        const long long f1 = e1 + (long long)T.dx[1] * (BH * kSub);
        const long long f2 = e2 + (long long)T.dx[2] * (BH * kSub);
        const bool a = (e0 | e1 | e2) >= 0, b = (f0 | f1 | f2) >= 0;
        if (!(a || b)) continue;
        const uint32_t id = st.id[k];
        if (a) visit(0, T, id, e0, e2);
        if (b) visit(1, T, id, f0, f2);
      }
    }
  }
}

}  // namespace star
