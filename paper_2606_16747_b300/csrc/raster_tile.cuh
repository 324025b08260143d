// raster_tile.cuh -- per-tile fragment traversal shared by the geometry-pass
// kernels.  One CTA of 256 threads owns one 16 x 16-pixel tile; warp w owns
// the 8 x 4 block at ((w & 1) * 8, (w >> 1) * 4) and lane l the pixel
// (l & 7, l >> 3) of it.  The tile's binned triangles are staged in shared
// memory kChunk at a time; a warp skips a triangle whose bounding box misses
// its block (a warp-uniform branch), otherwise every lane evaluates the three
// exact int64 edge functions at its pixel centre.
#pragma once

#include "common.cuh"

namespace star {

struct TilePixel {
  int px, py;    // pixel of this thread
  int bx0, by0;  // origin of this warp's 8 x 4 block
};

__device__ __forceinline__ TilePixel tile_pixel(int tile, int tiles_x) {
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  TilePixel t;
  t.bx0 = tx * kTile + (w & 1) * 8;
  t.by0 = ty * kTile + (w >> 1) * 4;
  t.px = t.bx0 + (l & 7);
  t.py = t.by0 + (l >> 3);
  return t;
}

// Canonical float32 depth of a covered pixel: b1 = E_20 / A, b2 = E_01 / A,
// z = (z0 + b1 dz1) + b2 dz2, one rounding per operation, -0 folded to +0.
__device__ __forceinline__ float frag_depth(const TriSetup &T, long long e0b, long long e2b) {
  const long long e01 = e0b - (long long)(T.own & 1u) + 1;
  const long long e20 = e2b - (long long)((T.own >> 2) & 1u) + 1;
  const float b1 = __fmul_rn(__ll2float_rn(e20), T.r);
  const float b2 = __fmul_rn(__ll2float_rn(e01), T.r);
  float z = __fadd_rn(__fadd_rn(T.z0, __fmul_rn(b1, T.dz1)), __fmul_rn(b2, T.dz2));
  return __fadd_rn(z, 0.0f);
}

// Calls visit(T, prim_id, depth) for every triangle of the tile covering
// this thread's pixel centre.  Must be called by all 256 threads.
template <class Visit>
__device__ __forceinline__ void for_each_fragment(const BinsView &bv, int tile, const TilePixel &tp,
                                                  TriSetup *s_tri, uint32_t *s_id, Visit &&visit) {
  const int Px = tp.px * kSub + kSub / 2, Py = tp.py * kSub + kSub / 2;
  const uint32_t beg = bv.tile_offset[tile], end = bv.tile_offset[tile + 1];
  for (uint32_t base = beg; base < end; base += kChunk) {
    const int n = (int)min((uint32_t)kChunk, end - base);
    __syncthreads();
    for (int i = threadIdx.x; i < n * 7; i += blockDim.x) {
      const int k = i / 7, part = i - 7 * k;
      const uint32_t id = __ldg(bv.pairs + base + k);
      reinterpret_cast<uint4 *>(s_tri + k)[part] =
          __ldg(reinterpret_cast<const uint4 *>(bv.setups + id) + part);
      if (part == 0) s_id[k] = id;
    }
    __syncthreads();
#pragma unroll 2
    for (int k = 0; k < n; ++k) {
      const TriSetup &T = s_tri[k];
      if (T.xb < tp.bx0 || T.xa > tp.bx0 + 7 || T.yb < tp.by0 || T.ya > tp.by0 + 3) continue;
      const long long e0 = (long long)T.dx[0] * Py + T.c[0] - (long long)T.dy[0] * Px;
      const long long e1 = (long long)T.dx[1] * Py + T.c[1] - (long long)T.dy[1] * Px;
      const long long e2 = (long long)T.dx[2] * Py + T.c[2] - (long long)T.dy[2] * Px;
      if ((e0 | e1 | e2) < 0) continue;
      visit(T, s_id[k], frag_depth(T, e0, e2));
    }
  }
}

}  // namespace star
