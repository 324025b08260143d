// common.cuh -- shared device-side definitions of the STAR-NT CUDA path.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "star_nt.h"

namespace star {

constexpr int kSub = 256;         // sub-pixel steps per pixel (1/256 px fixed point)
constexpr float kGuard = 32768.f; // |screen coordinate| limit, pixels
constexpr int kTile = 16;         // raster tile side (pixels)
constexpr int kChunk = 128;       // triangles staged in shared memory per round

// Triangle set up for one render target.  Edge e runs from vertex e to vertex
// e+1 (mod 3) after the vertices are ordered for a positive area; its
// function E_e(P) = dx * Py - dy * Px + c is exact in int64, and c already
// holds the tie bias (own_e - 1) so that a pixel centre is covered iff all
// three biased values are >= 0.
struct __align__(16) TriSetup {
  int32_t dx[3], dy[3];
  long long c[3];
  float z0, dz1, dz2, r;      // depth plane: z = (z0 + b1 dz1) + b2 dz2, r = 1/area
  int16_t xa, xb, ya, yb;     // covered-pixel bounding box (clamped), empty if xa > xb
  uint32_t own;               // bit e set: edge e owns ties; kOwnSmall: area < 2^31
  uint32_t opq;               // 1 when a8 == 255 (the comparison renderers' opaque count)
  unsigned long long rg;      // a8*r8 | (a8*g8) << 32
  unsigned long long ba;      // a8*b8 | a8 << 32
  unsigned long long lg;      // round(-log2(1 - a8/255) * 2^32); 160 * 2^32 when opaque (a sum
                              // holding it has tail transmittance exactly 0)
  float zlo;                  // lower bound of every fragment depth of the triangle
  uint32_t c8;                // straight colour: r8 | g8 << 8 | b8 << 16
};
static_assert(sizeof(TriSetup) == 112, "TriSetup layout");

// TriSetup::own flag: the doubled area (and so every edge value of a covered
// pixel) fits int32, so fragment depths may convert edge values as int32.
constexpr uint32_t kOwnSmall = 8u;

// Header at the start of a bins workspace.
struct __align__(16) BinsHeader {
  int32_t size[2];     // render-target size of the pass (copied from the target)
  int32_t tiles_x, tiles_y;
  int32_t n_tiles;     // tiles_x * tiles_y
  int32_t n_pixels;    // size[0] * size[1]
  uint32_t n_pairs;    // (triangle, tile) pairs needed
  int32_t n_tris;
  int32_t merged;      // 1: the pass runs at full size and is taken over by pass 1
  uint32_t queue;      // work counter of the persistent pass launch (zero between launches)
  uint32_t queue_exit; // CTAs done with the launch (zero between launches)
  int32_t resolved;    // 1: the pass launch also produced the frame (pass 1 ran the network)
  uint32_t ents;       // (triangle, tile) pairs recorded by the count launch (zero between calls)
  uint32_t pad[3];
};
static_assert(sizeof(BinsHeader) == 64, "BinsHeader layout");

// Offsets of the parts of a bins workspace.  ent / ent_rank: the count
// launch's record of every (triangle, tile) pair with its rank inside its
// tile, scattered into pairs once the tile offsets are known.
struct BinsLayout {
  size_t header, setups, tile_count, tile_offset, ent, ent_rank, pairs, scan_tmp, total;
  int32_t max_tiles;
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

inline BinsLayout bins_layout(int32_t max_w, int32_t max_h, int32_t max_tris, int64_t pairs) {
  BinsLayout L;
  int32_t tx = (max_w + kTile - 1) / kTile, ty = (max_h + kTile - 1) / kTile;
  L.max_tiles = tx * ty;
  size_t o = 0;
  L.header = o;      o = align_up(o + sizeof(BinsHeader), 256);
  L.setups = o;      o = align_up(o + sizeof(TriSetup) * (size_t)max_tris, 256);
  L.tile_count = o;  o = align_up(o + 4 * (size_t)(L.max_tiles + 4), 256);  // + ticket, + vector tail
  L.tile_offset = o; o = align_up(o + 4 * (size_t)(L.max_tiles + 1), 256);
  L.ent = o;         o = align_up(o + 8 * (size_t)pairs, 256);
  L.ent_rank = o;    o = align_up(o + 4 * (size_t)pairs, 256);
  L.pairs = o;       o = align_up(o + 4 * (size_t)pairs, 256);
  L.scan_tmp = o;    o = align_up(o + 4 * 8192, 256);
  L.total = o;
  return L;
}

// Device view of a bins workspace.
struct BinsView {
  BinsHeader *hd;
  TriSetup *setups;
  uint32_t *tile_count, *tile_offset, *pairs, *scan_tmp;
  uint2 *ent;         // (triangle, tile) of recorded pair e
  uint32_t *ent_rank;  // its rank inside the tile
  int32_t max_tiles;
  int32_t max_w, max_h;
  int64_t pair_capacity;
};

inline BinsView bins_view(const star_nt_bins &b) {
  BinsLayout L = bins_layout(b.max_w, b.max_h, b.max_tris, b.pair_capacity);
  char *m = (char *)b.mem;
  BinsView v;
  v.hd = (BinsHeader *)(m + L.header);
  v.setups = (TriSetup *)(m + L.setups);
  v.tile_count = (uint32_t *)(m + L.tile_count);
  v.tile_offset = (uint32_t *)(m + L.tile_offset);
  v.ent = (uint2 *)(m + L.ent);
  v.ent_rank = (uint32_t *)(m + L.ent_rank);
  v.pairs = (uint32_t *)(m + L.pairs);
  v.scan_tmp = (uint32_t *)(m + L.scan_tmp);
  v.max_tiles = L.max_tiles;
  v.max_w = b.max_w;
  v.max_h = b.max_h;
  v.pair_capacity = b.pair_capacity;
  return v;
}

// Host check of a per-leaf plan: target 0 is the full resolution, every
// target lies between a quarter of it and all of it on both axes (so a
// 16-sample target tile maps to at most 64 + 5 full-resolution pixels per
// axis), and every (pass, level) maps to a listed target.
// Host: a persistent pass launch's tuning (NULL: the defaults), decoded.
struct PassTuning {
  int bw, per_sm, pix;
};
inline bool pass_tuning(const star_nt_tuning *t, PassTuning &o) {
  o.bw = t ? t->block_w : 8;
  o.per_sm = t ? t->ctas_per_sm : 0;
  o.pix = t && t->pixels_per_thread ? t->pixels_per_thread : 2;
  if (o.bw != 4 && o.bw != 8 && o.bw != 16) return false;
  if (o.pix != 1 && o.pix != 2) return false;
  return o.per_sm >= 0 && o.per_sm <= (o.pix == 2 ? 10 : 8);
}

inline bool leaf_plan_valid(const star_nt_leaf_plan *p) {
  if (!p || p->W <= 0 || p->H <= 0 || (p->base_tile != 16 && p->base_tile != 64)) return false;
  if (p->n_targets < 1 || p->n_targets > STAR_NT_LEAF_MAX_TARGETS) return false;
  if (p->size[0][0] != p->W || p->size[0][1] != p->H) return false;
  for (int k = 0; k < p->n_targets; ++k) {
    const long long w = p->size[k][0], h = p->size[k][1];
    if (w < 1 || h < 1 || w > p->W || h > p->H || 4 * w < p->W || 4 * h < p->H) return false;
  }
  for (int q = 0; q < 2; ++q)
    for (int l = 0; l < 4; ++l)
      if (p->target_of[q][l] < 0 || p->target_of[q][l] >= p->n_targets) return false;
  return true;
}

// 8-bit RGBA of a float colour: round half to even of clamp(c, 0, 1) * 255,
// alpha 255.
__device__ __forceinline__ uint32_t quantize_rgba8(float r, float g, float b) {
  const uint32_t R = __float2uint_rn(__saturatef(r) * 255.0f);
  const uint32_t G = __float2uint_rn(__saturatef(g) * 255.0f);
  const uint32_t B = __float2uint_rn(__saturatef(b) * 255.0f);
  return R | (G << 8) | (B << 16) | (255u << 24);
}
__device__ __forceinline__ uint32_t quantize_rgba8(float4 c) { return quantize_rgba8(c.x, c.y, c.z); }

// Bound, in nanoseconds, of the tensor-core kernels' waits for an MMA commit
// or a TMA copy (star_nt_set_wait_limit); passed to each launch.
unsigned long long wait_limit_ns();

// First error wins.
__device__ inline void raise_status(int32_t *status, int32_t code) {
  if (status) atomicCAS(status, STAR_NT_OK, code);
}

__device__ inline long long floor_div_ll(long long a, long long b) {  // b > 0
  long long q = a / b;
  if ((a % b) != 0 && a < 0) --q;
  return q;
}

// Bilinear source axis of the upscale: u * 2W = (2x + 1) Wp - W (exact).
// All quantities fit in int32 for frames up to 16384 pixels wide; the floor
// division uses a float estimate corrected by one exact integer step.
struct Axis {
  int i0, i1;
  int rem, den;
};
__device__ inline Axis upscale_axis(int x, int Wp, int W) {
  const int num = (2 * x + 1) * Wp - W;
  const int den = 2 * W;
  int q = __float2int_rd(__fdividef((float)num, (float)den));
  int rem = num - q * den;
  if (rem < 0) { --q; rem += den; }
  if (rem >= den) { ++q; rem -= den; }
  Axis a;
  a.rem = rem;
  a.den = den;
  a.i0 = q < 0 ? 0 : (q > Wp - 1 ? Wp - 1 : q);
  a.i1 = q + 1 < 0 ? 0 : (q + 1 > Wp - 1 ? Wp - 1 : q + 1);
  return a;
}

// Exclusive scan of up to 8192 * 8192 uint32 values (n read on the device),
// total written to *total.  Three launches; tmp holds 8192 block sums.
cudaError_t scan_exclusive_u32(const uint32_t *in, uint32_t *out, const int32_t *n_dev,
                               int32_t n_max, uint32_t *tmp, uint32_t *total,
                               cudaStream_t st);

}  // namespace star
