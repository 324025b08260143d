// raster.cu -- star_nt_raster: triangle set-up, tile binning and the optional
// materialised fragment lists of one geometry pass (Sec. 3, Fig. 1).
#include <math.h>

#include "common.cuh"
#include "raster_tile.cuh"

namespace star {

// ---------------------------------------------------------------------------
// Fixed-point tail weights: lg[a] = round(-log2(1 - a/255) * 2^32) for
// a = 0 .. 254, tabulated at compile time so that set-up does no float64
// arithmetic (slow on this part).  log2 x = k + ln(m) / ln 2 with x = 2^k m,
// m in [1, 2), and ln m = 2 atanh z = 2 (z + z^3/3 + z^5/5 + ...) with
// z = (m - 1) / (m + 1) <= 1/3: 40 terms are far below double rounding.
struct LgTable {
  unsigned long long v[256];
};

constexpr double series_log2(double x) {  // x >= 1
  int k = 0;
  while (x >= 2.0) {
    x *= 0.5;
    ++k;
  }
  const double z = (x - 1.0) / (x + 1.0), z2 = z * z;
  double term = z, sum = 0.0;
  for (int n = 0; n < 40; ++n) {
    sum += term / (2 * n + 1);
    term *= z2;
  }
  return k + 2.0 * sum / 0.69314718055994530942;  // ln 2
}

constexpr LgTable make_lg_table() {
  LgTable t{};
  for (int a = 0; a < 255; ++a) {
    const double v = series_log2(255.0 / (255.0 - a)) * 4294967296.0;
    t.v[a] = (unsigned long long)(v + 0.5);
  }
  // opaque: past the exponent at which the tail transmittance is exactly 0,
  // so a sum holding an opaque fragment gives 0
  t.v[255] = 160ull << 32;
  return t;
}

__device__ const LgTable g_lg = make_lg_table();

// ---------------------------------------------------------------------------
// Triangle set-up by four lanes of a warp (q = lane % 4): lanes 0..2 each
// transform one vertex, lane 3 fetches the colour; the snapped vertices are
// exchanged by shuffles; lanes 0..2 each set up one edge and lane 3 the depth
// plane, bounding box and colour sums.  The arithmetic is that of one thread
// doing it all: float32 with one rounding per operation (order fixed), drop
// triangles with a vertex behind the camera, outside NDC z in [0, 1] or
// outside the guard band, snap to 1/256 pixel, order the vertices for a
// positive area, then store the biased edge functions, depth plane, pixel
// bounding box and colour sums.  All 32 lanes of the warp must call it;
// `store` false (a triangle index past the end) skips the writes.
__device__ __forceinline__ void triangle_setup_x4(int t, bool store, const float *__restrict__ verts,
                                                  const uint32_t *__restrict__ rgba8,
                                                  const float *__restrict__ vp, int W, int H,
                                                  bool size_ok, TriSetup *out) {
  const unsigned full = 0xffffffffu;
  const int q = threadIdx.x & 3;
  float m[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) m[i] = __ldg(vp + i);
  const float4 *V = reinterpret_cast<const float4 *>(verts) + 3 * (size_t)t;
  const uint32_t col = (store && q == 3) ? __ldg(rgba8 + t) : 0u;
  // ---- lanes 0..2: vertex q
  bool okq = true;
  float sxq = 0.0f, syq = 0.0f, znq = 0.0f;
  if (store && q < 3) {
    const float4 p = __ldg(V + q);
    float c[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float acc = __fmul_rn(m[4 * i + 0], p.x);
      acc = __fadd_rn(acc, __fmul_rn(m[4 * i + 1], p.y));
      acc = __fadd_rn(acc, __fmul_rn(m[4 * i + 2], p.z));
      acc = __fadd_rn(acc, __fmul_rn(m[4 * i + 3], p.w));
      c[i] = acc;
    }
    if (!(c[3] > 0.0f)) okq = false;
    const float nx = __fdiv_rn(c[0], c[3]), ny = __fdiv_rn(c[1], c[3]), nz = __fdiv_rn(c[2], c[3]);
    if (!(nz >= 0.0f && nz <= 1.0f)) okq = false;
    sxq = __fmul_rn(__fadd_rn(__fmul_rn(nx, 0.5f), 0.5f), (float)W);
    syq = __fmul_rn(__fsub_rn(0.5f, __fmul_rn(ny, 0.5f)), (float)H);
    if (!(fabsf(sxq) <= kGuard && fabsf(syq) <= kGuard)) okq = false;
    znq = __fadd_rn(nz, 0.0f);
  }
  const long long Xq = okq ? __float2ll_rn(__fmul_rn(sxq, (float)kSub)) : 0ll;
  const long long Yq = okq ? __float2ll_rn(__fmul_rn(syq, (float)kSub)) : 0ll;
  // ---- exchange within the group of four lanes
  bool ok = size_ok;
  long long X[3], Y[3];
  float zn[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    // every lane takes part in every shuffle (no short-circuit around them)
    const int okk = __shfl_sync(full, (int)okq, k, 4);
    ok = ok && okk != 0;
    X[k] = __shfl_sync(full, Xq, k, 4);
    Y[k] = __shfl_sync(full, Yq, k, 4);
    zn[k] = __shfl_sync(full, znq, k, 4);
  }
  long long area = 0;
  if (ok) {
    area = (X[1] - X[0]) * (Y[2] - Y[0]) - (Y[1] - Y[0]) * (X[2] - X[0]);
    if (area == 0) ok = false;
  }
  if (ok && area < 0) {  // no culling: swap v1 and v2 for a positive area
    long long tx = X[1], ty = Y[1];
    X[1] = X[2]; Y[1] = Y[2]; X[2] = tx; Y[2] = ty;
    float tz = zn[1]; zn[1] = zn[2]; zn[2] = tz;
    area = -area;
  }
  // ---- lanes 0..2: edge q
  // edge from vertex q to vertex q + 1 (mod 3); selects keep X, Y in registers
  const long long Xa = q == 1 ? X[1] : (q == 2 ? X[2] : X[0]);
  const long long Ya = q == 1 ? Y[1] : (q == 2 ? Y[2] : Y[0]);
  const long long Xb = q == 0 ? X[1] : (q == 1 ? X[2] : X[0]);
  const long long Yb = q == 0 ? Y[1] : (q == 1 ? Y[2] : Y[0]);
  const long long dx = Xb - Xa, dy = Yb - Ya;
  const uint32_t o = (dy > 0 || (dy == 0 && dx < 0)) ? 1u : 0u;
  const uint32_t own = __shfl_sync(full, o, 0, 4) | (__shfl_sync(full, o, 1, 4) << 1) |
                       (__shfl_sync(full, o, 2, 4) << 2);
  if (!store) return;
  if (q < 3) {
    out->dx[q] = ok ? (int32_t)dx : 0;
    out->dy[q] = ok ? (int32_t)dy : 0;
    out->c[q] = ok ? dy * Xa - dx * Ya + (long long)o - 1 : -1ll;
    return;
  }
  // ---- lane 3: depth plane, bounding box, colour sums
  TriSetup &S = *out;
  S.xa = 1;
  S.xb = 0;
  S.ya = 1;
  S.yb = 0;
  if (ok) {
    S.own = own | (area <= 0x7fffffffLL ? kOwnSmall : 0u);
    S.z0 = zn[0];
    S.dz1 = __fsub_rn(zn[1], zn[0]);
    S.dz2 = __fsub_rn(zn[2], zn[0]);
    S.r = __frcp_rn(__ll2float_rn(area));
    // Every fragment depth is an interpolation of the vertex depths in [0, 1]
    // with barycentric weights >= 0 summing to 1 up to a few roundings of
    // 2^-24, so it is at least min(z) - 2^-21; 2^-16 leaves ample room.
    S.zlo = __fsub_rn(fminf(zn[0], fminf(zn[1], zn[2])), 1.52587890625e-05f);
    long long minx = min(X[0], min(X[1], X[2])), maxx = max(X[0], max(X[1], X[2]));
    long long miny = min(Y[0], min(Y[1], Y[2])), maxy = max(Y[0], max(Y[1], Y[2]));
    long long xa = -floor_div_ll(-(minx - kSub / 2), kSub), xb = floor_div_ll(maxx - kSub / 2, kSub);
    long long ya = -floor_div_ll(-(miny - kSub / 2), kSub), yb = floor_div_ll(maxy - kSub / 2, kSub);
    xa = max(xa, 0LL); ya = max(ya, 0LL);
    xb = min(xb, (long long)W - 1); yb = min(yb, (long long)H - 1);
    if (xa <= xb && ya <= yb) {
      S.xa = (int16_t)xa; S.xb = (int16_t)xb; S.ya = (int16_t)ya; S.yb = (int16_t)yb;
    }
  } else {
    S.own = 0; S.z0 = S.dz1 = S.dz2 = S.r = 0.0f;
    S.zlo = INFINITY;
  }
  const unsigned long long a8 = col >> 24, r8 = col & 255u, g8 = (col >> 8) & 255u,
                           b8 = (col >> 16) & 255u;
  S.opq = a8 == 255 ? 1u : 0u;
  S.rg = (a8 * r8) | ((a8 * g8) << 32);
  S.ba = (a8 * b8) | (a8 << 32);
  S.c8 = (uint32_t)col & 0xFFFFFFu;
  S.lg = g_lg.v[a8];
}

// Render-target size of a pass, validated against the workspace: a size
// beyond it empties the pass instead of writing out of bounds.
__device__ __forceinline__ bool pass_size(const int32_t *size, const BinsView &bv, int &W, int &H) {
  const bool ok = size[0] > 0 && size[1] > 0 && size[0] <= bv.max_w && size[1] <= bv.max_h;
  W = ok ? size[0] : 0;
  H = ok ? size[1] : 0;
  return ok;
}

// Tile range and conservative tile test shared by the two binning kernels.
// A tile is kept unless one edge function is negative at every pixel centre
// of the tile clipped to the triangle's bounding box (its maximum over the
// corner centres is negative), which never drops a covered pixel.
__device__ __forceinline__ bool tile_hit(const TriSetup &T, int tx, int ty) {
  const int xlo = max(tx * kTile, (int)T.xa), xhi = min(tx * kTile + kTile - 1, (int)T.xb);
  const int ylo = max(ty * kTile, (int)T.ya), yhi = min(ty * kTile + kTile - 1, (int)T.yb);
  const int Pxlo = xlo * kSub + kSub / 2, Pxhi = xhi * kSub + kSub / 2;
  const int Pylo = ylo * kSub + kSub / 2, Pyhi = yhi * kSub + kSub / 2;
  bool hit = true;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const long long mx = T.c[e] + (long long)T.dx[e] * (T.dx[e] > 0 ? Pyhi : Pylo) -
                         (long long)T.dy[e] * (T.dy[e] > 0 ? Pxlo : Pxhi);
    if (mx < 0) hit = false;
  }
  return hit;
}

// Candidate tiles of a set-up triangle: its bounding box in tiles.
__device__ __forceinline__ int tile_span(const TriSetup &T, int &tx0, int &ty0, int &ntx) {
  if (T.xa > T.xb || T.ya > T.yb) return 0;
  tx0 = T.xa / kTile;
  ty0 = T.ya / kTile;
  ntx = T.xb / kTile - tx0 + 1;
  return ntx * (T.yb / kTile - ty0 + 1);
}

constexpr int kBinThreads = 128;
constexpr int kBinTris = 16;  // triangles per binning block: four threads per triangle set it up

// (triangle, tile) candidates of one block's kBinTris triangles, whose
// set-ups are staged in shared memory (tri[i] = triangle t0 + i), flattened
// so that all kBinThreads threads walk an equal share: a warp scan of the
// per-triangle candidate counts, then a binary search per candidate; a
// candidate that passes tile_hit is a pair.  The walk runs in rounds of
// kCountBatch candidates per thread: the
// candidates' tile tests first, then their tile-count increments (independent
// atomics, all in flight together; each returns the pair's rank inside its
// tile), then one reservation per warp and round in the pair record for the
// warp's hits and their writes.  The fill then only scatters the record.  The order
// of a tile's pairs is not fixed.
constexpr int kCountBatch = 4;
__device__ __forceinline__ void count_pairs(const TriSetup *tri, int t0, int n_tris, int tiles_x,
                                            int *s_off, const BinsView &bv) {
  static_assert(kBinTris <= 32 && kBinThreads >= 4 * kBinTris, "one warp scans the candidate counts");
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid < 32) {
    int tx0 = 0, ty0 = 0, ntx = 1;
    const int nt = tid < kBinTris && t0 + tid < n_tris ? tile_span(tri[tid], tx0, ty0, ntx) : 0;
    int v = nt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, v, o);
      if (tid >= o) v += y;
    }
    if (tid < kBinTris) s_off[tid + 1] = v;
    if (tid == 0) s_off[0] = 0;
  }
  __syncthreads();
  const int total = s_off[kBinTris];
  const int64_t cap = bv.pair_capacity;
  for (int r0 = 0; r0 < total; r0 += kBinThreads * kCountBatch) {  // uniform over the block
    int tile[kCountBatch], tr[kCountBatch];
#pragma unroll
    for (int b = 0; b < kCountBatch; ++b) {
      tile[b] = -1;
      tr[b] = 0;
      const int q = r0 + b * kBinThreads + tid;
      if (q < total) {
        int lo = 0, hi = kBinTris - 1;  // largest j with s_off[j] <= q
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_off[mid] <= q) lo = mid; else hi = mid - 1;
        }
        const TriSetup &T = tri[lo];
        int ax0, ay0, anx;
        tile_span(T, ax0, ay0, anx);
        const int k = q - s_off[lo];
        const int tx = ax0 + k % anx, ty = ay0 + k / anx;
        if (tile_hit(T, tx, ty)) {
          tile[b] = ty * tiles_x + tx;
          tr[b] = t0 + lo;
        }
      }
    }
    uint32_t rank[kCountBatch];
    int cnt = 0;
#pragma unroll
    for (int b = 0; b < kCountBatch; ++b) {
      rank[b] = tile[b] >= 0 ? atomicAdd(bv.tile_count + tile[b], 1u) : 0u;
      cnt += tile[b] >= 0 ? 1 : 0;
    }
    int incl = cnt;  // this thread's hits after the warp's earlier lanes'
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int wsum = __shfl_sync(0xffffffffu, incl, 31);
    uint32_t base = 0u;
    if (lane == 0 && wsum) base = atomicAdd(&bv.hd->ents, (uint32_t)wsum);
    uint32_t e = __shfl_sync(0xffffffffu, base, 0) + (uint32_t)(incl - cnt);
#pragma unroll
    for (int b = 0; b < kCountBatch; ++b) {
      if (tile[b] < 0) continue;
      if ((int64_t)e < cap) {  // beyond capacity the fill raises STAR_NT_ERR_CAPACITY
        bv.ent[e] = make_uint2((uint32_t)tr[b], (uint32_t)tile[b]);
        bv.ent_rank[e] = rank[b];
      }
      ++e;
    }
  }
}

// Up to STAR_NT_MAX_RASTER_PASSES passes are binned by the same launches
// (blockIdx.y = pass).
constexpr int kMaxPasses = STAR_NT_MAX_RASTER_PASSES;
struct PassSet {
  BinsView bv[kMaxPasses];
  const float *vp[kMaxPasses];
  const int32_t *size[kMaxPasses];
  const int32_t *merge_at[kMaxPasses];
  float merge_scale[kMaxPasses];
};

// Set-up (four threads per triangle, kept in shared memory for the
// candidate walk and copied out for the pass kernels) and per-tile candidate
// counts.
__global__ void __launch_bounds__(kBinThreads) k_bin_count(const float *__restrict__ verts,
                                                           const uint32_t *__restrict__ rgba8,
                                                           int n_tris, PassSet ps, int32_t *status) {
  __shared__ int s_off[kBinTris + 1];
  __shared__ TriSetup s_tri[kBinTris];
  const BinsView &bv = ps.bv[blockIdx.y];
  const int32_t *size = ps.size[blockIdx.y];
  const int32_t *merge_at = ps.merge_at[blockIdx.y];
  int W, H;
  const bool size_ok = pass_size(size, bv, W, H);
  // merged: taken over by pass 1 at the full size merge_at (whose planes it
  // then writes), when the pass is at least merge_scale of it on both axes
  const float ms = ps.merge_scale[blockIdx.y];
  const bool merged = size_ok && merge_at && merge_at[0] <= bv.max_w && merge_at[1] <= bv.max_h &&
                      (float)W >= ms * (float)merge_at[0] && (float)H >= ms * (float)merge_at[1];
  const int tiles_x = merged ? 0 : (W + kTile - 1) / kTile;
  const int n_tiles = tiles_x * (merged ? 0 : (H + kTile - 1) / kTile);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    BinsHeader *hd = bv.hd;
    if (merged) {
      W = merge_at[0];
      H = merge_at[1];
    }
    hd->size[0] = W;
    hd->size[1] = H;
    hd->tiles_x = tiles_x;
    hd->tiles_y = merged ? 0 : (H + kTile - 1) / kTile;
    hd->n_tiles = n_tiles;
    hd->n_pixels = W * H;
    hd->n_tris = n_tris;
    hd->merged = merged ? 1 : 0;
    hd->resolved = 0;
    if (!size_ok) raise_status(status, STAR_NT_ERR_ARG);
  }
  if (!merged) {  // a merged pass is taken over by pass 1: no triangles binned
    const int t0 = blockIdx.x * kBinTris;
    const int j = threadIdx.x >> 2;  // four lanes per triangle (all warps take part)
    triangle_setup_x4(t0 + j, j < kBinTris && t0 + j < n_tris, verts, rgba8, ps.vp[blockIdx.y], W, H,
                      size_ok, s_tri + (j < kBinTris ? j : 0));
    __syncthreads();
    const int nb = min(kBinTris, n_tris - t0);
    for (int i = threadIdx.x; i < nb * 7; i += kBinThreads)
      reinterpret_cast<uint4 *>(bv.setups + t0)[i] = reinterpret_cast<const uint4 *>(s_tri)[i];
    count_pairs(s_tri, t0, n_tris, tiles_x, s_off, bv);
  }
}

// Pair lists: every recorded pair goes to its tile's offset plus its rank
// (a scatter over the record; positions are distinct by construction).
constexpr int kFillThreads = 256;
__global__ void __launch_bounds__(kFillThreads) k_bin_fill(PassSet ps, int32_t *status) {
  const BinsView &bv = ps.bv[blockIdx.y];
  const BinsHeader *hd = bv.hd;
  if (hd->n_tiles == 0) return;  // empty or merged pass
  const uint32_t n = hd->n_pairs;
  if ((int64_t)n > bv.pair_capacity) {
    if (blockIdx.x == 0 && threadIdx.x == 0) raise_status(status, STAR_NT_ERR_CAPACITY);
    return;
  }
  for (uint32_t i = blockIdx.x * kFillThreads + threadIdx.x; i < n; i += gridDim.x * kFillThreads) {
    const uint2 en = __ldg(bv.ent + i);
    bv.pairs[__ldg(bv.tile_offset + en.y) + __ldg(bv.ent_rank + i)] = en.x;
  }
}

// Exclusive scan of the tile counts, one block of 1024 threads per pass, in
// rounds of 4096 counts: thread t holds counts [4 (r 1024 + t), +4) of round
// r, so that every load and store of a warp is one coalesced 512-byte run.
// The loads of up to four rounds are in flight together.  Writes the
// offsets and the total pair count, and zeroes the counts it consumed and the
// pair record's counter: the workspace leaves every call with zero counters,
// ready for the next (no clearing launch).
constexpr int kScanRounds = 4;

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *s_warp, uint32_t *total);

__global__ void __launch_bounds__(1024) k_scan_tiles(PassSet ps) {
  __shared__ uint32_t s_warp[32];
  const BinsView &bv = ps.bv[blockIdx.x];
  const int n = bv.hd->n_tiles;
  const int tid = threadIdx.x;
  uint32_t carry = 0;
  for (int base = 0; base < n; base += kScanRounds * 4096) {
    uint4 v[kScanRounds];
#pragma unroll
    for (int r = 0; r < kScanRounds; ++r) {
      const int i = base + 4 * (r * 1024 + tid);
      v[r] = i < n ? *reinterpret_cast<const uint4 *>(bv.tile_count + i) : make_uint4(0u, 0u, 0u, 0u);
      if (i + 1 >= n) v[r].y = 0u;
      if (i + 2 >= n) v[r].z = 0u;
      if (i + 3 >= n) v[r].w = 0u;
    }
#pragma unroll
    for (int r = 0; r < kScanRounds; ++r) {
      const int i = base + 4 * (r * 1024 + tid);
      if (base + r * 4096 >= n) break;  // uniform over the block
      const uint32_t sum = v[r].x + v[r].y + v[r].z + v[r].w;
      uint32_t tot;
      const uint32_t ex = block_excl_scan(sum, s_warp, &tot) + carry;
      const uint4 o = make_uint4(ex, ex + v[r].x, ex + v[r].x + v[r].y, ex + v[r].x + v[r].y + v[r].z);
      if (i + 3 < n) {
        *reinterpret_cast<uint4 *>(bv.tile_offset + i) = o;
        *reinterpret_cast<uint4 *>(bv.tile_count + i) = make_uint4(0u, 0u, 0u, 0u);
      } else if (i < n) {
        const uint32_t oo[4] = {o.x, o.y, o.z, o.w};
        for (int e = 0; e < n - i; ++e) {
          bv.tile_offset[i + e] = oo[e];
          bv.tile_count[i + e] = 0u;  // consumed: zero again for the next call
        }
      }
      carry += tot;
      __syncthreads();  // s_warp is reused by the next round
    }
  }
  if (tid == 0) {
    bv.tile_offset[n] = carry;
    bv.hd->n_pairs = carry;  // = the pairs the count recorded
    bv.hd->ents = 0u;        // zero again for the next call
  }
}

// ---------------------------------------------------------------------------
// Exclusive scan (three launches).  Block b of the first and last launches
// covers items [8192 b, 8192 (b + 1)); 1024 threads x 8 items.
constexpr int kScanThreads = 1024, kScanItems = 8, kScanBlock = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *s_warp, uint32_t *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = s_warp[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  const uint32_t before = warp ? s_warp[warp - 1] : 0u;
  if (total) *total = s_warp[31];
  return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ in,
                                                              const int32_t *n_dev, uint32_t *tmp) {
  __shared__ uint32_t s_warp[32];
  const int n = *n_dev;
  const size_t b0 = (size_t)blockIdx.x * kScanBlock;
  if (b0 >= (size_t)n) return;
  uint32_t s = 0;
  const size_t i0 = b0 + (size_t)threadIdx.x * kScanItems;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k)
    if (i0 + k < (size_t)n) s += in[i0 + k];
  uint32_t tot;
  block_excl_scan(s, s_warp, &tot);
  if (threadIdx.x == 0) tmp[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(uint32_t *tmp, const int32_t *n_dev,
                                                              uint32_t *out, uint32_t *total) {
  __shared__ uint32_t s_warp[32];
  const int n = *n_dev;
  const int nb = (n + kScanBlock - 1) / kScanBlock;
  uint32_t v[kScanItems], s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int i = threadIdx.x * kScanItems + k;
    v[k] = i < nb ? tmp[i] : 0u;
    s += v[k];
  }
  uint32_t tot;
  uint32_t run = block_excl_scan(s, s_warp, &tot);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int i = threadIdx.x * kScanItems + k;
    if (i < nb) tmp[i] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) {
    out[n] = tot;
    if (total) *total = tot;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_final(const uint32_t *__restrict__ in,
                                                             uint32_t *__restrict__ out,
                                                             const int32_t *n_dev,
                                                             const uint32_t *tmp) {
  __shared__ uint32_t s_warp[32];
  const int n = *n_dev;
  const size_t b0 = (size_t)blockIdx.x * kScanBlock;
  if (b0 >= (size_t)n) return;
  const size_t i0 = b0 + (size_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems], s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = i0 + k < (size_t)n ? in[i0 + k] : 0u;
    s += v[k];
  }
  uint32_t run = block_excl_scan(s, s_warp, nullptr) + tmp[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (i0 + k < (size_t)n) out[i0 + k] = run;
    run += v[k];
  }
}

cudaError_t scan_exclusive_u32(const uint32_t *in, uint32_t *out, const int32_t *n_dev, int32_t n_max,
                               uint32_t *tmp, uint32_t *total, cudaStream_t st) {
  const int nb = (n_max + kScanBlock - 1) / kScanBlock;
  if (nb > kScanBlock) return cudaErrorInvalidValue;
  const int g = nb > 0 ? nb : 1;
  k_scan_reduce<<<g, kScanThreads, 0, st>>>(in, n_dev, tmp);
  k_scan_blocks<<<1, kScanThreads, 0, st>>>(tmp, n_dev, out, total);
  k_scan_final<<<g, kScanThreads, 0, st>>>(in, out, n_dev, tmp);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Materialised fragments: per-pixel counts, then the lists themselves.
__global__ void __launch_bounds__(256) k_frag_count(BinsView bv, uint32_t *count) {
  __shared__ TileStage stage;
  const BinsHeader *hd = bv.hd;
  if ((int64_t)hd->n_pairs > bv.pair_capacity) return;
  const int tile = blockIdx.x;
  const int W = hd->size[0], H = hd->size[1];
  if (hd->merged) {  // fragments of a merged pass are not listed: zero counts
    const int tx = (W + kTile - 1) / kTile, ty = (H + kTile - 1) / kTile;
    if (tile < tx * ty) {
      const TilePixel tp = tile_pixel<8>(tile, tx);
      if (tp.px < W && tp.py < H) count[tp.py * W + tp.px] = 0;
    }
    return;
  }
  if (tile >= hd->n_tiles) return;
  const TilePixel tp = tile_pixel<8>(tile, hd->tiles_x);
  uint32_t n = 0;
  for_each_fragment(bv, tile, tp, stage, [] { return INFINITY; },
                    [&](const TriSetup &, uint32_t, long long, long long) { ++n; });
  if (tp.px < W && tp.py < H) count[tp.py * W + tp.px] = n;
}

__global__ void __launch_bounds__(256) k_frag_fill(BinsView bv, const uint32_t *offset,
                                                   const uint32_t *total, int64_t capacity,
                                                   float *zs, int32_t *prims, int32_t *status) {
  __shared__ TileStage stage;
  const BinsHeader *hd = bv.hd;
  if ((int64_t)hd->n_pairs > bv.pair_capacity) return;
  if ((int64_t)*total > capacity) {
    if (blockIdx.x == 0 && threadIdx.x == 0) raise_status(status, STAR_NT_ERR_CAPACITY);
    return;
  }
  const int tile = blockIdx.x;
  if (tile >= hd->n_tiles) return;
  const int W = hd->size[0], H = hd->size[1];
  const TilePixel tp = tile_pixel<8>(tile, hd->tiles_x);
  const bool inside = tp.px < W && tp.py < H;
  uint32_t pos = inside ? offset[tp.py * W + tp.px] : 0u;
  for_each_fragment(bv, tile, tp, stage, [] { return INFINITY; },
                    [&](const TriSetup &T, uint32_t id, long long e0, long long e2) {
    if (inside) {
      zs[pos] = frag_depth(T, e0, e2);
      prims[pos] = (int32_t)id;
      ++pos;
    }
  });
}

}  // namespace star

using namespace star;

extern "C" star_nt_status star_nt_bins_bytes(int32_t max_w, int32_t max_h, int32_t max_tris,
                                             int64_t pair_capacity, size_t *bytes) {
  if (!bytes || max_w <= 0 || max_h <= 0 || max_tris < 0 || pair_capacity < 0 ||
      max_w > 16384 || max_h > 16384 || pair_capacity > 0xffffffffLL)
    return STAR_NT_ERR_ARG;
  *bytes = bins_layout(max_w, max_h, max_tris, pair_capacity).total;
  return STAR_NT_OK;
}

static star_nt_status check_pass(const star_nt_scene *scene, const star_nt_target *target,
                                 const star_nt_bins *bins) {
  if (!target || !bins || !bins->mem || !target->view_proj || !target->size) return STAR_NT_ERR_ARG;
  if (scene->n_tris > bins->max_tris) return STAR_NT_ERR_ARG;
  if (target->max_w <= 0 || target->max_h <= 0 || target->max_w > bins->max_w ||
      target->max_h > bins->max_h)
    return STAR_NT_ERR_ARG;
  size_t need = 0;
  if (star_nt_bins_bytes(bins->max_w, bins->max_h, bins->max_tris, bins->pair_capacity, &need) !=
          STAR_NT_OK ||
      bins->bytes < need || ((uintptr_t)bins->mem & 255u))
    return STAR_NT_ERR_ARG;
  return STAR_NT_OK;
}

extern "C" star_nt_status star_nt_raster_passes(const star_nt_scene *scene, int32_t n_passes,
                                                const star_nt_target *targets,
                                                const star_nt_bins *bins, int32_t *d_status,
                                                void *stream) {
  if (!scene || !targets || !bins || n_passes < 1 || n_passes > kMaxPasses) return STAR_NT_ERR_ARG;
  if (scene->n_tris < 0 || (scene->n_tris > 0 && (!scene->verts || !scene->rgba8)) ||
      ((uintptr_t)scene->verts & 15u))
    return STAR_NT_ERR_ARG;
  PassSet ps = {};
  for (int i = 0; i < n_passes; ++i) {
    const star_nt_status s = check_pass(scene, targets + i, bins + i);
    if (s != STAR_NT_OK) return s;
    for (int j = 0; j < i; ++j)
      if (bins[j].mem == bins[i].mem) return STAR_NT_ERR_ARG;  // distinct workspaces
    ps.bv[i] = bins_view(bins[i]);
    ps.vp[i] = targets[i].view_proj;
    ps.size[i] = targets[i].size;
    ps.merge_at[i] = targets[i].merge_at;
    const float ms = targets[i].merge_scale;
    if (!(ms <= 1.0f)) return STAR_NT_ERR_ARG;  // NaN or above 1
    ps.merge_scale[i] = ms > 0.0f ? ms : 1.0f;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int T = scene->n_tris;
  const dim3 grid(T > 0 ? (T + kBinTris - 1) / kBinTris : 1, n_passes);
  k_bin_count<<<grid, kBinThreads, 0, st>>>(scene->verts, scene->rgba8, T, ps, d_status);
  k_scan_tiles<<<n_passes, 1024, 0, st>>>(ps);
  {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_bin_fill<<<dim3(4 * sms, n_passes), kFillThreads, 0, st>>>(ps, d_status);
  }
  return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
}

extern "C" star_nt_status star_nt_raster(const star_nt_scene *scene, const star_nt_target *target,
                                         const star_nt_bins *bins, const star_nt_frags *frags,
                                         int32_t *d_status, void *stream) {
  if (!scene || !target || !bins) return STAR_NT_ERR_ARG;
  if (frags && (!frags->count || !frags->offset || !frags->total ||
                (frags->capacity > 0 && (!frags->z || !frags->prim)) || frags->capacity < 0))
    return STAR_NT_ERR_ARG;
  star_nt_status s = star_nt_raster_passes(scene, 1, target, bins, d_status, stream);
  if (s != STAR_NT_OK || !frags) return s;
  cudaStream_t st = (cudaStream_t)stream;
  BinsView bv = bins_view(*bins);
  const int P = target->max_w * target->max_h;
  const int tiles = ((target->max_w + kTile - 1) / kTile) * ((target->max_h + kTile - 1) / kTile);
  k_frag_count<<<tiles, 256, 0, st>>>(bv, frags->count);
  if (scan_exclusive_u32(frags->count, frags->offset, &bv.hd->n_pixels, P, bv.scan_tmp, frags->total,
                         st) != cudaSuccess)
    return STAR_NT_ERR_CUDA;
  k_frag_fill<<<tiles, 256, 0, st>>>(bv, frags->offset, frags->total, frags->capacity, frags->z,
                                     frags->prim, d_status);
  return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
}

namespace star {
// Loads this file's kernels onto the current device (see star_nt_preload).
cudaError_t preload_raster() {
  cudaFuncAttributes a;
  cudaError_t e = cudaSuccess, r;
  if ((r = cudaFuncGetAttributes(&a, k_bin_count)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_bin_fill)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_scan_tiles)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_scan_reduce)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_scan_blocks)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_scan_final)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_frag_count)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_frag_fill)) != cudaSuccess) e = r;
  return e;
}
}  // namespace star
