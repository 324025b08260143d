// leaf.cu -- per-leaf pass resolution, the per-tile variant of Sec. 3.2 /
// Eq. 2: every pixel takes passes 2 and 3 at the scale that Eq. 2 gives for
// the level of its own quadtree leaf, s_p(l) = clamp(2^(l - delta_p), 1/4, 1),
// instead of the frame-wide scene index wbar.
//
// The scales depend on the level only, so a frame has a fixed set of render
// targets (at most one per (pass, level), plus the full resolution).  Each
// frame:
//  1. k_leaf_modes: for every 16 x 16 tile of every target, whether some pixel
//     needs pass 2 and/or pass 3 from it.  A pixel needs the samples of
//     nonzero weight of its bilinear footprint (the same upscale_axis as the
//     resolve), so the full-resolution pixels that need a target tile form
//     a rectangle; the tile needs pass p when a pixel of that rectangle lies
//     in a leaf whose level maps pass p to the target, tested on the masks'
//     8 x 8 level-3 cells (leaf levels are constant over a cell).
//  2. k_passes_leaf: one persistent launch over the tiles of all targets, as
//     k_passes: each tile runs the cheapest traversal its mode allows (pass 1
//     alone, the two nearest, or the two nearest plus tail sums); tiles no
//     pixel needs are skipped.
#include <math.h>

#include "pass_body.cuh"
#include "qt_cells.cuh"

namespace star {

constexpr int kLeafT = STAR_NT_LEAF_MAX_TARGETS;

struct LeafModeArgs {
  int W, H, B, base_tiles_x;
  int n_targets;
  int32_t size[kLeafT][2];
  int32_t tiles_x[kLeafT];
  int32_t tile_start[kLeafT + 1];  // prefix of the targets' tile counts
  uint32_t levels2[kLeafT];        // bit l: level l takes pass 2 from the target
  uint32_t levels3[kLeafT];        // bit l: level l takes pass 3 from the target
};

// Full-resolution pixels of one axis whose bilinear footprint on a target
// axis of Wk samples (nonzero weights only) meets samples [a, b]: an interval
// [lo, hi] (lo > hi when empty).  The footprint ends are monotone in the
// pixel, so the candidates c0..c1 (which bracket every such pixel for
// Wk >= W / 4) are tested by the warp and the first and last kept.
__device__ __forceinline__ void needed_pixels(int a, int b, int Wk, int W, int lane, int &lo, int &hi) {
  int c0 = (int)((long long)a * W / Wk) - 2;
  int c1 = (int)(((long long)(b + 1) * W + Wk - 1) / Wk) + 1;
  c0 = c0 < 0 ? 0 : c0;
  c1 = c1 > W - 1 ? W - 1 : c1;
  lo = 0x7fffffff;
  hi = -1;
  for (int x0 = c0; x0 <= c1; x0 += 32) {  // uniform over the warp
    const int x = x0 + lane;
    bool need = false;
    if (x <= c1) {
      const Axis ax = upscale_axis(x, Wk, W);
      const int f1 = ax.rem ? ax.i1 : ax.i0;  // i1 carries weight only when rem > 0
      need = ax.i0 <= b && f1 >= a;
    }
    const uint32_t bal = __ballot_sync(0xffffffffu, need);
    if (bal) {
      lo = min(lo, x0 + __ffs(bal) - 1);
      hi = max(hi, x0 + 31 - __clz(bal));
    }
  }
}

// Level-3 cells of a base tile (origin ox, oy; side B) inside the pixel
// rectangle [x0, x1] x [y0, y1] (which meets the tile).
__device__ __forceinline__ unsigned long long rect_cells(int x0, int x1, int y0, int y1, int ox, int oy,
                                                         int B) {
  const int cs = B >> 3;
  const int cx0 = (max(x0, ox) - ox) / cs, cx1 = (min(x1, ox + B - 1) - ox) / cs;
  const int cy0 = (max(y0, oy) - oy) / cs, cy1 = (min(y1, oy + B - 1) - oy) / cs;
  const unsigned long long row = (unsigned long long)(((2u << cx1) - (1u << cx0)) & 0xFFu);
  const unsigned long long rows = kCol0 & (~0ull << (8 * cy0)) & (~0ull >> (8 * (7 - cy1)));
  return row * rows;  // one copy of the row bits per selected row, no carries
}

// One warp per target tile: mode bit 0 = pass 2 needed, bit 1 = pass 3.
__global__ void __launch_bounds__(256) k_leaf_modes(LeafModeArgs a,
                                                    const uint32_t *__restrict__ masks,
                                                    uint8_t *__restrict__ modes) {
  const int item = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (item >= a.tile_start[a.n_targets]) return;  // uniform over the warp
  int k = 0;
  while (item >= a.tile_start[k + 1]) ++k;
  const uint32_t lv2 = a.levels2[k], lv3 = a.levels3[k];
  uint32_t mode = 0u;
  if (lv2 | lv3) {
    const int tile = item - a.tile_start[k];
    const int tx = tile % a.tiles_x[k], ty = tile / a.tiles_x[k];
    const int Wk = a.size[k][0], Hk = a.size[k][1];
    int x0, x1, y0, y1;
    needed_pixels(tx * kTile, min(tx * kTile + kTile - 1, Wk - 1), Wk, a.W, lane, x0, x1);
    needed_pixels(ty * kTile, min(ty * kTile + kTile - 1, Hk - 1), Hk, a.H, lane, y0, y1);
    bool n2 = false, n3 = false;
    if (x0 <= x1 && y0 <= y1) {
      const int B = a.B;
      const int bx0 = x0 / B, by0 = y0 / B;
      const int nbx = x1 / B - bx0 + 1, nb = nbx * (y1 / B - by0 + 1);
      for (int i = lane; i < nb; i += 32) {
        const int btx = bx0 + i % nbx, bty = by0 + i / nbx;
        const uint32_t m = __ldg(masks + (size_t)bty * a.base_tiles_x + btx);
        const unsigned long long r = rect_cells(x0, x1, y0, y1, btx * B, bty * B, B);
        // levels present in the rectangle's cells (one pass over the mask)
        unsigned long long d2, d3;
        deep_cells(m, d2, d3);
        const bool root = (m & 1u) != 0u;
        const uint32_t present = ((!root && r) ? 1u : 0u) | ((root && (r & ~d2)) ? 2u : 0u) |
                                 ((r & d2 & ~d3) ? 4u : 0u) | ((r & d3) ? 8u : 0u);
        n2 |= (present & lv2) != 0u;
        n3 |= (present & lv3) != 0u;
      }
    }
    n2 = __any_sync(0xffffffffu, n2);
    n3 = __any_sync(0xffffffffu, n3);
    mode = (n2 ? 1u : 0u) | (n3 ? 2u : 0u);
  }
  if (lane == 0) modes[item] = (uint8_t)mode;
}

struct LeafPassArgs {
  BinsView bv[kLeafT];
  PassOut out[kLeafT];
  int32_t size[kLeafT][2];
  int32_t tile_start[kLeafT + 1];
  int n_targets;
};

// All tiles of all targets in one persistent launch (items in target order:
// the full resolution first).  Target 0 always runs pass 1 and adds the two
// nearest / the tail sums where its mode asks; the other targets run only
// where some pixel needs them.
template <int BW, int MINB, int PIX = 1>
__global__ void __launch_bounds__(PIX == 2 ? 128 : 256, MINB) k_passes_leaf(LeafPassArgs a,
                                                        const uint8_t *__restrict__ modes,
                                                        const uint32_t *__restrict__ rgba8,
                                                        uint32_t *queue, int32_t *status) {
  __shared__ union {
    TileStage t;  // one pixel per thread: for_each_fragment
    WalkStage w;  // two pixels per thread: walk_tile2
  } stage;
  __shared__ int s_item;
  const int total = a.tile_start[a.n_targets];
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
    int k = 0;
    while (item >= a.tile_start[k + 1]) ++k;
    const int tile = item - a.tile_start[k];
    const BinsView &bv = a.bv[k];
    const BinsHeader *hd = bv.hd;
    if (hd->size[0] != a.size[k][0] || hd->size[1] != a.size[k][1] || hd->merged != 0) {
      if (threadIdx.x == 0 && tile == 0) raise_status(status, STAR_NT_ERR_ARG);
      continue;  // binned at another size than the plan's: skipped
    }
    const uint32_t m = __ldg(modes + item);
    if (PIX == 2) {
      if (m & 2u) pass_body2<kTail, BW>(bv, rgba8, a.out[k], stage.w, tile);
      else if (m & 1u) pass_body2<kTop2, BW>(bv, rgba8, a.out[k], stage.w, tile);
      else if (k == 0) pass_body2<kTop1, BW>(bv, rgba8, a.out[0], stage.w, tile);
    } else {
      if (m & 2u) pass_body<kTail, BW>(bv, rgba8, a.out[k], FeatOut{}, stage.t, tile);
      else if (m & 1u) pass_body<kTop2, BW>(bv, rgba8, a.out[k], FeatOut{}, stage.t, tile);
      else if (k == 0) pass_body<kTop1, BW>(bv, rgba8, a.out[0], FeatOut{}, stage.t, tile);
    }
  }
}

}  // namespace star

using namespace star;

static void plan_add(star_nt_leaf_plan *p, int q, int l, int32_t w, int32_t h) {
  for (int k = 0; k < p->n_targets; ++k)
    if (p->size[k][0] == w && p->size[k][1] == h) {
      p->target_of[q][l] = k;
      return;
    }
  p->size[p->n_targets][0] = w;
  p->size[p->n_targets][1] = h;
  p->target_of[q][l] = p->n_targets++;
}

extern "C" star_nt_status star_nt_leaf_plan_make(int32_t W, int32_t H, const star_nt_params *params,
                                                 star_nt_leaf_plan *plan) {
  if (!params || !plan || W <= 0 || H <= 0) return STAR_NT_ERR_ARG;
  if (params->base_tile != 16 && params->base_tile != 64) return STAR_NT_ERR_ARG;
  if (!(params->delta2 == params->delta2) || !(params->delta3 == params->delta3)) return STAR_NT_ERR_ARG;
  star_nt_leaf_plan p = {};
  p.W = W;
  p.H = H;
  p.base_tile = params->base_tile;
  p.n_targets = 1;
  p.size[0][0] = W;
  p.size[0][1] = H;
  const double delta[2] = {params->delta2, params->delta3};
  for (int q = 0; q < 2; ++q)
    for (int l = 0; l < 4; ++l) {
      double s = exp2((double)l - delta[q]);  // Eq. 2 with wbar = l
      s = s < 0.25 ? 0.25 : (s > 1.0 ? 1.0 : s);
      plan_add(&p, q, l, (int32_t)ceil(s * (double)W), (int32_t)ceil(s * (double)H));
    }
  *plan = p;
  return STAR_NT_OK;
}

static int target_tiles(const star_nt_leaf_plan *p, int k) {
  return ((p->size[k][0] + kTile - 1) / kTile) * ((p->size[k][1] + kTile - 1) / kTile);
}

extern "C" star_nt_status star_nt_leaf_ws_bytes(const star_nt_leaf_plan *plan, size_t *bytes) {
  if (!bytes || !leaf_plan_valid(plan)) return STAR_NT_ERR_ARG;
  size_t n = 0;
  for (int k = 0; k < plan->n_targets; ++k) n += (size_t)target_tiles(plan, k);
  *bytes = align_up(n, 256);
  return STAR_NT_OK;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

extern "C" star_nt_status star_nt_geometry_passes_leaf(const star_nt_scene *scene,
                                                       const star_nt_leaf_plan *plan,
                                                       const star_nt_bins *bins,
                                                       const star_nt_layers *layers,
                                                       const uint32_t *masks, void *ws,
                                                       size_t ws_bytes,
                                                       const star_nt_tuning *tuning,
                                                       int32_t *d_status, void *stream) {
  if (!scene || !bins || !layers || !masks || !ws || ((uintptr_t)ws & 255u)) return STAR_NT_ERR_ARG;
  if (!leaf_plan_valid(plan)) return STAR_NT_ERR_ARG;
  if (scene->n_tris < 0 || (scene->n_tris > 0 && !scene->rgba8)) return STAR_NT_ERR_ARG;
  size_t need = 0;
  if (star_nt_leaf_ws_bytes(plan, &need) != STAR_NT_OK || ws_bytes < need) return STAR_NT_ERR_ARG;
  PassTuning tu;
  if (!pass_tuning(tuning, tu)) return STAR_NT_ERR_ARG;
  const int bw = tu.bw, per_sm = tu.per_sm;
  const int n = plan->n_targets;
  LeafModeArgs ma = {};
  LeafPassArgs pa = {};
  ma.W = plan->W;
  ma.H = plan->H;
  ma.B = plan->base_tile;
  ma.base_tiles_x = (plan->W + plan->base_tile - 1) / plan->base_tile;
  ma.n_targets = pa.n_targets = n;
  for (int k = 0; k < n; ++k) {
    const star_nt_bins &b = bins[k];
    if (!b.mem || b.max_w < plan->size[k][0] || b.max_h < plan->size[k][1]) return STAR_NT_ERR_ARG;
    for (int j = 0; j < k; ++j)
      if (bins[j].mem == b.mem) return STAR_NT_ERR_ARG;  // distinct workspaces
    const star_nt_layers &L = layers[k];
    if (!aligned16(L.id1) || !aligned16(L.z1) || !aligned16(L.id2) || !aligned16(L.n) ||
        !aligned16(L.tail) || !aligned16(L.t_tail))
      return STAR_NT_ERR_ARG;
    ma.size[k][0] = pa.size[k][0] = plan->size[k][0];
    ma.size[k][1] = pa.size[k][1] = plan->size[k][1];
    ma.tiles_x[k] = (plan->size[k][0] + kTile - 1) / kTile;
    ma.tile_start[k + 1] = pa.tile_start[k + 1] = ma.tile_start[k] + target_tiles(plan, k);
    pa.bv[k] = bins_view(b);
    PassOut &o = pa.out[k];
    o.id1 = k == 0 ? L.id1 : nullptr;
    o.z1 = k == 0 ? L.z1 : nullptr;
    o.id2 = L.id2;
    o.n = L.n;
    o.tail = reinterpret_cast<uint4 *>(L.tail);
    o.t_tail = L.t_tail;
  }
  if (!layers[0].id1 || !layers[0].z1) return STAR_NT_ERR_ARG;
  for (int l = 0; l < 4; ++l) {
    const int k2 = plan->target_of[0][l], k3 = plan->target_of[1][l];
    ma.levels2[k2] |= 1u << l;
    ma.levels3[k3] |= 1u << l;
    if (!layers[k2].id2 || !layers[k3].n || !layers[k3].tail || !layers[k3].t_tail) return STAR_NT_ERR_ARG;
  }
  const int total = ma.tile_start[n];
  cudaStream_t st = (cudaStream_t)stream;
  uint8_t *modes = (uint8_t *)ws;
  k_leaf_modes<<<(total + 7) / 8, 256, 0, st>>>(ma, masks, modes);
  uint32_t *queue = &pa.bv[0].hd->queue;  // queue[0] work counter, queue[1] exit count
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  auto launch = [&](auto kern, int threads = 256) {
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, 0);
    const int c = per_sm > 0 ? (per_sm < occ ? per_sm : occ) : occ;
    kern<<<sms * (c > 0 ? c : 1), threads, 0, st>>>(pa, modes, scene->rgba8, queue, d_status);
  };
  if (tu.pix == 2) {  // two pixels per thread, budgets as star_nt_geometry_passes
    const bool wide2 = per_sm == 10;
    if (bw == 8) wide2 ? launch(k_passes_leaf<8, 10, 2>, 128) : launch(k_passes_leaf<8, 8, 2>, 128);
    else if (bw == 16) wide2 ? launch(k_passes_leaf<16, 10, 2>, 128) : launch(k_passes_leaf<16, 8, 2>, 128);
    else wide2 ? launch(k_passes_leaf<4, 10, 2>, 128) : launch(k_passes_leaf<4, 8, 2>, 128);
    return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
  }
  const bool wide = per_sm == 0 || per_sm == 8;  // register budget as star_nt_geometry_passes
  if (bw == 8) wide ? launch(k_passes_leaf<8, 8>) : launch(k_passes_leaf<8, 6>);
  else if (bw == 16) wide ? launch(k_passes_leaf<16, 8>) : launch(k_passes_leaf<16, 6>);
  else wide ? launch(k_passes_leaf<4, 8>) : launch(k_passes_leaf<4, 6>);
  return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
}

namespace star {
// Loads this file's kernels onto the current device (see star_nt_preload).
cudaError_t preload_leaf() {
  cudaFuncAttributes a;
  cudaError_t e = cudaSuccess, r;
  if ((r = cudaFuncGetAttributes(&a, k_leaf_modes)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes_leaf<4, 6>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes_leaf<8, 6>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes_leaf<16, 6>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes_leaf<4, 8>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes_leaf<8, 8>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes_leaf<16, 8>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes_leaf<4, 10, 2>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes_leaf<8, 10, 2>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes_leaf<16, 10, 2>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes_leaf<4, 8, 2>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes_leaf<8, 8, 2>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes_leaf<16, 8, 2>)) != cudaSuccess) e = r;
  return e;
}
}  // namespace star
