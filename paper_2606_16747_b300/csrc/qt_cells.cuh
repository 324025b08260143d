// qt_cells.cuh -- the 8 x 8 level-3 cells of a quadtree base tile (Sec. 3.1)
// as bits of a 64-bit word (bit 8 cy + cx), and the cells of each leaf level
// under a tile's 21-bit split mask (bit 0 root; bits 1..4 level-1 children;
// bits 5..20 level-2 nodes, 4 per level-1 child; child index 2 y_half + x_half).
#pragma once

#include <stdint.h>

namespace star {

constexpr unsigned long long kCol0 = 0x0101010101010101ull, kCol7 = kCol0 << 7;
constexpr unsigned long long kRow0 = 0xFFull, kRow7 = kRow0 << 56;

// cells of level-1 quadrant q (child index 2 y_half + x_half)
__device__ __forceinline__ unsigned long long quad_cells(int q) {
  return 0x0F0F0F0Full << ((q & 1) * 4 + (q >> 1) * 32);
}
// cells of level-2 node q2 = 4 c1 + c2 (mask bit 5 + q2)
__device__ __forceinline__ unsigned long long node2_cells(int q2) {
  const int c1 = q2 >> 2, c2 = q2 & 3;
  const int i = (c1 & 1) * 2 + (c2 & 1), j = (c1 >> 1) * 2 + (c2 >> 1);
  return 0x0303ull << (2 * i + 16 * j);
}

// Cells whose leaf is at level >= 2 (d2) and at level 3 (d3) under mask m.
__device__ __forceinline__ void deep_cells(uint32_t m, unsigned long long &d2, unsigned long long &d3) {
  d2 = 0ull;
  d3 = 0ull;
  if (!(m & 1u)) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (!((m >> (1 + q)) & 1u)) continue;
    d2 |= quad_cells(q);
#pragma unroll
    for (int c2 = 0; c2 < 4; ++c2)
      if ((m >> (5 + 4 * q + c2)) & 1u) d3 |= node2_cells(4 * q + c2);
  }
}

// Level of the leaf holding pixel (lx, ly) of a base tile of side B.
__device__ __forceinline__ int leaf_level(uint32_t m, int lx, int ly, int B) {
  if (!(m & 1u)) return 0;
  const int h1 = B >> 1, h2 = B >> 2;
  const int c1 = ((ly >= h1) << 1) | (lx >= h1);
  if (!((m >> (1 + c1)) & 1u)) return 1;
  const int c2 = (((ly % h1) >= h2) << 1) | ((lx % h1) >= h2);
  return ((m >> (5 + 4 * c1 + c2)) & 1u) ? 3 : 2;
}

}  // namespace star
