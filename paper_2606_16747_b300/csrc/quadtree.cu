// quadtree.cu -- star_nt_quadtree: adaptive screen-space tiles (Sec. 3.1)
// and tile-guided pass resolution (Sec. 3.2, Eq. 2).
//
// Split/merge decisions: one warp per base tile; lane k < 21 owns the node
// whose split bit is bit k of the tile's mask (bit 0 root, bits 1..4 level-1
// nodes, bits 5..20 level-2 nodes), so ballots assemble new masks directly.
// Relaxation and the leaf histogram work bit-parallel on the tile's 8 x 8
// level-3 cells (one 64-bit word per level), one thread per tile.  All
// decisions are taken on integer colour differences with correctly rounded
// float64 square roots summed in a fixed order, so they are reproducible bit
// for bit.
#include <math.h>

#include <mutex>

#include "common.cuh"
#include "qt_cells.cuh"

namespace star {

struct QtLayout {
  size_t hist, mask_a, mask_b, total;
  int32_t tiles_x, tiles_y;
};

inline QtLayout qt_layout(int32_t W, int32_t H, int32_t B) {
  QtLayout L;
  L.tiles_x = (W + B - 1) / B;
  L.tiles_y = (H + B - 1) / B;
  const size_t nt = (size_t)L.tiles_x * L.tiles_y;
  L.hist = 0;
  L.mask_a = 256;
  L.mask_b = align_up(L.mask_a + 4 * nt, 256);
  L.total = align_up(L.mask_b + 4 * nt, 256);
  return L;
}

// node of bit k: level and position (i, j) in units of the node size
__device__ __forceinline__ void node_of_bit(int k, int &l, int &i, int &j) {
  if (k == 0) { l = 0; i = 0; j = 0; return; }
  if (k < 5) { const int c = k - 1; l = 1; i = c & 1; j = c >> 1; return; }
  const int q = k - 5, c1 = q >> 2, c2 = q & 3;
  l = 2;
  i = (c1 & 1) * 2 + (c2 & 1);
  j = (c1 >> 1) * 2 + (c2 >> 1);
}

__device__ __forceinline__ bool node_exists(uint32_t m, int k) {
  if (k == 0) return true;
  if (k < 5) return m & 1u;
  const int c1 = (k - 5) >> 2;
  return (m & 1u) && ((m >> (1 + c1)) & 1u);
}

// Corner colours of a node (clamped to the image) and the six integer
// squared distances in the fixed pair order 01, 02, 03, 12, 13, 23.
__device__ __forceinline__ void corner_q(const uint32_t *__restrict__ img, int W, int H, int x0, int y0,
                                         int S, int (&q)[6]) {
  const int xs[4] = {x0, x0 + S - 1, x0, x0 + S - 1};
  const int ys[4] = {y0, y0, y0 + S - 1, y0 + S - 1};
  int c[4][3];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int x = min(max(xs[k], 0), W - 1), y = min(max(ys[k], 0), H - 1);
    const uint32_t v = img[(size_t)y * W + x];
    c[k][0] = v & 255u;
    c[k][1] = (v >> 8) & 255u;
    c[k][2] = (v >> 16) & 255u;
  }
  const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {1, 2, 3, 2, 3, 3};
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    int s = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int d = c[pa[e]][k] - c[pb[e]][k];
      s += d * d;
    }
    q[e] = s;
  }
}

// The decision quantity: sum of the six distances, as a float64 sum of
// correctly rounded square roots in the fixed order.  A float32 estimate
// (error below 1e-3 for 8-bit colours) decides whenever it is farther than
// 2e-3 from both thresholds; otherwise the float64 sum decides, so every
// decision equals the float64 one.
__device__ __forceinline__ double decision_dsum(const int (&q)[6], double split6, double merge6) {
  float f = 0.0f;
#pragma unroll
  for (int e = 0; e < 6; ++e) f = __fadd_rn(f, __fsqrt_rn((float)q[e]));
  const double fd = (double)f;
  if (fabs(fd - split6) > 2e-3 && fabs(fd - merge6) > 2e-3) return fd;
  double s = 0.0;
#pragma unroll
  for (int e = 0; e < 6; ++e) s = __dadd_rn(s, __dsqrt_rn((double)q[e]));
  return s;
}

__global__ void __launch_bounds__(256) k_qt_decide(const uint32_t *__restrict__ img, int W, int H,
                                                   int B, int tiles_x, int n_tiles, double split6,
                                                   double merge6, const uint32_t *__restrict__ mprev,
                                                   uint32_t *__restrict__ mout,
                                                   uint32_t *__restrict__ hist) {
  // the histogram and the last-block ticket of k_qt_last start from zero
  if (blockIdx.x == 0 && threadIdx.x < 8) hist[threadIdx.x] = 0u;
  const int tile = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (tile >= n_tiles) return;
  const uint32_t m = mprev[tile];
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  bool leaf = false, split_node = false;
  double ds = 0.0;
  if (lane < 21) {
    int l, i, j;
    node_of_bit(lane, l, i, j);
    const bool ex = node_exists(m, lane);
    split_node = ex && ((m >> lane) & 1u);
    leaf = ex && !split_node;
    if (ex) {
      const int S = B >> l;
      int q[6];
      corner_q(img, W, H, tx * B + i * S, ty * B + j * S, S, q);
      ds = decision_dsum(q, split6, merge6);
    }
  }
  const uint32_t split_bits = __ballot_sync(0xffffffffu, leaf && ds > split6);
  bool merge = false;
  if (lane < 21 && split_node && ds < merge6) {
    if (lane == 0) {
      merge = ((m >> 1) & 15u) == 0u && ((split_bits >> 1) & 15u) == 0u;
    } else if (lane < 5) {
      const int c1 = lane - 1;
      merge = ((m >> (5 + 4 * c1)) & 15u) == 0u && ((split_bits >> (5 + 4 * c1)) & 15u) == 0u;
    } else {
      merge = true;  // children are level-3 leaves
    }
  }
  const uint32_t merge_bits = __ballot_sync(0xffffffffu, merge);
  if (lane == 0) mout[tile] = (m | split_bits) & ~merge_bits;
}

// ---------------------------------------------------------------------------
// Relaxation and the leaf histogram, bit-parallel over the 8 x 8 level-3
// cells of a tile (bit 8 cy + cx of a 64-bit word).

// One Jacobi relaxation step of a tile: a leaf splits when an edge-adjacent
// cell (in the tile or across its border) lies two or more levels deeper.
// Only the root (level 0) and level-1 leaves can split: a level-2 leaf would
// need a level-4 neighbour.  nb* = 0 where the tile has no neighbour.
__device__ __forceinline__ uint32_t relax_mask(uint32_t m, uint32_t mL, uint32_t mR, uint32_t mU,
                                               uint32_t mD) {
  unsigned long long d2, d3, l2, l3, r2, r3, u2, u3, w2, w3;
  deep_cells(m, d2, d3);
  deep_cells(mL, l2, l3);
  deep_cells(mR, r2, r3);
  deep_cells(mU, u2, u3);
  deep_cells(mD, w2, w3);
  if (!(m & 1u)) {  // root leaf: neighbours' border cells at level >= 2
    const bool s = (l2 & kCol7) | (r2 & kCol0) | (u2 & kRow7) | (w2 & kRow0);
    return s ? (m | 1u) : m;
  }
  uint32_t out = m;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if ((m >> (1 + q)) & 1u) continue;  // split: not a leaf
    const unsigned long long R = quad_cells(q);
    const unsigned long long ring = (((R << 1) & ~kCol0) | ((R >> 1) & ~kCol7) | (R << 8) | (R >> 8)) & ~R;
    const unsigned long long rows = 0xFFFFFFFFull << ((q >> 1) * 32);
    const unsigned long long cols = 0x0F0F0F0F0F0F0F0Full << ((q & 1) * 4);
    bool s = (d3 & ring) != 0ull;
    if ((q & 1) == 0) s |= (l3 & kCol7 & rows) != 0ull;
    else s |= (r3 & kCol0 & rows) != 0ull;
    if ((q >> 1) == 0) s |= (u3 & kRow7 & cols) != 0ull;
    else s |= (w3 & kRow0 & cols) != 0ull;
    if (s) out |= 1u << (1 + q);
  }
  return out;
}

// neighbour masks of tile (tx, ty), 0 outside the image
__device__ __forceinline__ uint32_t relax_tile(const uint32_t *__restrict__ min, int tile, int tx,
                                               int ty, int tiles_x, int tiles_y) {
  const uint32_t m = min[tile];
  const uint32_t mL = tx > 0 ? min[tile - 1] : 0u, mR = tx + 1 < tiles_x ? min[tile + 1] : 0u;
  const uint32_t mU = ty > 0 ? min[tile - tiles_x] : 0u;
  const uint32_t mD = ty + 1 < tiles_y ? min[tile + tiles_x] : 0u;
  return relax_mask(m, mL, mR, mU, mD);
}

// One relaxation iteration (Jacobi: reads min, writes mout), thread per tile.
__global__ void __launch_bounds__(256) k_qt_relax(const uint32_t *__restrict__ min,
                                                  uint32_t *__restrict__ mout, int tiles_x,
                                                  int tiles_y) {
  const int tile = blockIdx.x * 256 + threadIdx.x;
  if (tile >= tiles_x * tiles_y) return;
  mout[tile] = relax_tile(min, tile, tile % tiles_x, tile / tiles_x, tiles_x, tiles_y);
}

// Occupied leaves of a tile per level under its final mask m; occ = the
// level-3 cells holding a pass-1 fragment.
__device__ __forceinline__ void count_leaves(uint32_t m, unsigned long long occ, uint32_t (&cnt)[4]) {
  if (!(m & 1u)) {
    cnt[0] += occ != 0ull ? 1u : 0u;
    return;
  }
  unsigned long long d2, d3;
  deep_cells(m, d2, d3);
  cnt[3] += __popcll(occ & d3);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (!((m >> (1 + q)) & 1u)) {
      cnt[1] += (occ & quad_cells(q)) != 0ull ? 1u : 0u;
      continue;
    }
#pragma unroll
    for (int c2 = 0; c2 < 4; ++c2)
      if (!((m >> (5 + 4 * q + c2)) & 1u)) cnt[2] += (occ & node2_cells(4 * q + c2)) != 0ull ? 1u : 0u;
  }
}

// The last relaxation (or a copy), then the histogram of occupied leaves; the
// last block to finish applies Eq. 2 and writes the state.  The tile's
// pass-1 ids give the occupancy of its 64 level-3 cells (B/8 pixels wide):
// for 16-pixel tiles a warp per tile (8 pixels per lane), for 64-pixel tiles
// a block of 256 threads per tile (16 pixels per thread; every warp reads
// 32 consecutive pixels of a row).  One thread per tile does the rest.
template <bool RELAX, int B>
__global__ void __launch_bounds__(256) k_qt_last(const int32_t *__restrict__ id1, int W, int H,
                                                 int tiles_x, int tiles_y,
                                                 const uint32_t *__restrict__ min,
                                                 uint32_t *__restrict__ mout,
                                                 uint32_t *__restrict__ hist, uint32_t *ticket,
                                                 double delta2, double delta3,
                                                 star_nt_pass_state *state) {
  static_assert(B == 16 || B == 64, "base tile");
  constexpr int kTilesPerBlock = B == 16 ? 8 : 1;
  constexpr int kThreadsPerTile = 256 / kTilesPerBlock;
  constexpr int kCs = B / 8;  // cell side
  __shared__ uint32_t s_hist[4];
  __shared__ uint32_t s_occ[2];
  if (threadIdx.x < 4) s_hist[threadIdx.x] = 0u;
  if (threadIdx.x < 2) s_occ[threadIdx.x] = 0u;
  __syncthreads();
  const int tile = blockIdx.x * kTilesPerBlock + (int)threadIdx.x / kThreadsPerTile;
  const int t = (int)threadIdx.x % kThreadsPerTile;
  const bool valid = tile < tiles_x * tiles_y;
  const int tx = valid ? tile % tiles_x : 0, ty = valid ? tile / tiles_x : 0;
  unsigned long long occ = 0;
  if (valid) {
#pragma unroll
    for (int i = 0; i < B * B / kThreadsPerTile; ++i) {
      const int k = i * kThreadsPerTile + t;
      const int lx = k % B, ly = k / B;
      const int x = tx * B + lx, y = ty * B + ly;
      if (x < W && y < H && __ldg(id1 + (size_t)y * W + x) >= 0)
        occ |= 1ull << ((ly / kCs) * 8 + (lx / kCs));
    }
  }
  // OR over the tile's threads (whole warps: a 16-pixel tile is one warp)
  uint32_t lo = __reduce_or_sync(0xffffffffu, (uint32_t)occ);
  uint32_t hi = __reduce_or_sync(0xffffffffu, (uint32_t)(occ >> 32));
  if (B == 64) {
    if ((threadIdx.x & 31) == 0) {
      if (lo) atomicOr(&s_occ[0], lo);
      if (hi) atomicOr(&s_occ[1], hi);
    }
    __syncthreads();
    lo = s_occ[0];
    hi = s_occ[1];
  }
  occ = ((unsigned long long)hi << 32) | lo;
  if (valid && t == 0) {
    const uint32_t m = RELAX ? relax_tile(min, tile, tx, ty, tiles_x, tiles_y) : min[tile];
    mout[tile] = m;
    uint32_t cnt[4] = {0u, 0u, 0u, 0u};
    count_leaves(m, occ, cnt);
#pragma unroll
    for (int l = 0; l < 4; ++l)
      if (cnt[l]) atomicAdd(&s_hist[l], cnt[l]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int l = 0; l < 4; ++l)
      if (s_hist[l]) atomicAdd(hist + l, s_hist[l]);
    __threadfence();
    const uint32_t done = atomicAdd(ticket, 1u);
    if (done == gridDim.x - 1) {  // last block: every histogram update is visible
      __threadfence();
      const uint32_t h0 = atomicAdd(hist + 0, 0u), h1 = atomicAdd(hist + 1, 0u);
      const uint32_t h2 = atomicAdd(hist + 2, 0u), h3 = atomicAdd(hist + 3, 0u);
      const double tot = (double)h0 + (double)h1 + (double)h2 + (double)h3;
      const double wbar = tot > 0.0 ? ((double)h1 + 2.0 * (double)h2 + 3.0 * (double)h3) / tot : 0.0;
      double s2 = exp2(wbar - delta2), s3 = exp2(wbar - delta3);
      s2 = s2 < 0.25 ? 0.25 : (s2 > 1.0 ? 1.0 : s2);
      s3 = s3 < 0.25 ? 0.25 : (s3 > 1.0 ? 1.0 : s3);
      state->W = W;
      state->H = H;
      state->W2 = (int32_t)ceil(s2 * (double)W);
      state->H2 = (int32_t)ceil(s2 * (double)H);
      state->W3 = (int32_t)ceil(s3 * (double)W);
      state->H3 = (int32_t)ceil(s3 * (double)H);
      state->s2 = (float)s2;
      state->s3 = (float)s3;
      state->wbar = wbar;
      state->hist[0] = h0;
      state->hist[1] = h1;
      state->hist[2] = h2;
      state->hist[3] = h3;
    }
  }
}

}  // namespace star

using namespace star;

extern "C" star_nt_status star_nt_quadtree_ws_bytes(int32_t W, int32_t H, int32_t base_tile,
                                                    size_t *bytes) {
  if (!bytes || W <= 0 || H <= 0 || (base_tile != 16 && base_tile != 64)) return STAR_NT_ERR_ARG;
  *bytes = qt_layout(W, H, base_tile).total;
  return STAR_NT_OK;
}

extern "C" star_nt_status star_nt_quadtree(const uint32_t *rgba8, const int32_t *id1, int32_t W,
                                           int32_t H, const star_nt_params *params,
                                           const uint32_t *mask_prev, uint32_t *mask_out,
                                           star_nt_pass_state *state, void *ws, size_t ws_bytes,
                                           void *stream) {
  if (!rgba8 || !id1 || !params || !mask_prev || !mask_out || !state || !ws) return STAR_NT_ERR_ARG;
  const int B = params->base_tile;
  size_t need = 0;
  if (star_nt_quadtree_ws_bytes(W, H, B, &need) != STAR_NT_OK || ws_bytes < need ||
      ((uintptr_t)ws & 255u))
    return STAR_NT_ERR_ARG;
  if (params->relax_iters < 0 || params->relax_iters > 8 || !(params->tau_merge < params->tau_split))
    return STAR_NT_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const QtLayout L = qt_layout(W, H, B);
  char *m = (char *)ws;
  uint32_t *hist = (uint32_t *)(m + L.hist);
  uint32_t *ma = (uint32_t *)(m + L.mask_a), *mb = (uint32_t *)(m + L.mask_b);
  const int nt = L.tiles_x * L.tiles_y;
  const int wblocks = (nt + 7) / 8;
  const int iters = params->relax_iters;
  uint32_t *ticket = hist + 4;
  // mask_prev is read only here, so mask_out may be the same buffer
  k_qt_decide<<<wblocks, 256, 0, st>>>(rgba8, W, H, B, L.tiles_x, nt, 6.0 * params->tau_split,
                                       6.0 * params->tau_merge, mask_prev, ma, hist);
  const uint32_t *src = ma;
  const int tblocks = (nt + 255) / 256;
  for (int it = 0; it + 1 < iters; ++it) {  // all but the last relaxation
    uint32_t *d = src == ma ? mb : ma;
    k_qt_relax<<<tblocks, 256, 0, st>>>(src, d, L.tiles_x, L.tiles_y);
    src = d;
  }
  // the last relaxation (a plain copy when there is none), the histogram of
  // occupied leaves and Eq. 2, in one launch
  auto last = [&](auto kern, int blocks) {
    kern<<<blocks, 256, 0, st>>>(id1, W, H, L.tiles_x, L.tiles_y, src, mask_out, hist, ticket,
                                 params->delta2, params->delta3, state);
  };
  if (B == 16) {
    if (iters > 0) last(k_qt_last<true, 16>, wblocks);
    else last(k_qt_last<false, 16>, wblocks);
  } else {
    if (iters > 0) last(k_qt_last<true, 64>, nt);
    else last(k_qt_last<false, 64>, nt);
  }
  return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Workspace-free variant.  Some callers cannot allocate device memory: a
// plug-in that only ever receives buffers from its host application, or an
// engine that budgets all GPU memory at start-up and forbids allocation on its
// frame path (cudaMalloc may also synchronise the device, which a frame loop
// cannot afford).  For them the quadtree workspace lives in a fixed array in
// this library's device memory instead of a caller buffer.
namespace star {
constexpr int kQtStaticMaxTiles = 65536;
constexpr size_t kQtStaticBytes = 256 + 2 * 4 * (size_t)kQtStaticMaxTiles;
static __device__ __align__(256) unsigned char g_qt_scratch[kQtStaticBytes];

// The array's device address belongs to a CUDA context, not to a device: a
// host application may run its own (non-primary) context on the device, and a
// device reset replaces the primary context.  The address is therefore looked
// up once per context, with that context current, and cached under the
// context's unique id (never reused within a process).  The driver calls come
// through the runtime's entry-point query, so the library does not link the
// driver library itself.
typedef int (*CtxGetCurrentFn)(void **ctx);                      // cuCtxGetCurrent
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);    // cuCtxGetId
constexpr int kQtAddrSlots = 64;
struct QtAddrSlot {
  unsigned long long ctx_id;  // 0: empty
  void *addr;
};
static std::mutex g_qt_mutex;
static QtAddrSlot g_qt_addr[kQtAddrSlots];
static int g_qt_next = 0;
static CtxGetCurrentFn g_ctx_current = nullptr;
static CtxGetIdFn g_ctx_id = nullptr;

// Id of the context current on this thread (0 when none is current yet).
static cudaError_t current_ctx_id(unsigned long long *id) {
  if (!g_ctx_current || !g_ctx_id) {
    void *f = nullptr, *g = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1);
    if (e != cudaSuccess || q1 != cudaDriverEntryPointSuccess || !f) return cudaErrorNotSupported;
    e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess || q2 != cudaDriverEntryPointSuccess || !g) return cudaErrorNotSupported;
    g_ctx_current = (CtxGetCurrentFn)f;
    g_ctx_id = (CtxGetIdFn)g;
  }
  void *ctx = nullptr;
  if (g_ctx_current(&ctx) != 0) return cudaErrorUnknown;
  *id = 0;
  if (ctx && g_ctx_id(ctx, id) != 0) return cudaErrorUnknown;
  return cudaSuccess;
}

// Device address of the array in the context current on this thread: looked
// up on the first call in each context and cached.
static cudaError_t qt_scratch_address(void **out) {
  std::lock_guard<std::mutex> lock(g_qt_mutex);
  unsigned long long id = 0;
  cudaError_t e = current_ctx_id(&id);
  if (e != cudaSuccess) return e;
  if (id) {
    for (int k = 0; k < kQtAddrSlots; ++k)
      if (g_qt_addr[k].ctx_id == id) {
        *out = g_qt_addr[k].addr;
        return cudaSuccess;
      }
  }
  // not seen yet (or no context current: the runtime then makes the device's
  // primary context current here)
  void *p = nullptr;
  e = cudaGetSymbolAddress(&p, g_qt_scratch);
  if (e != cudaSuccess) return e;
  if (!id && (e = current_ctx_id(&id)) != cudaSuccess) return e;
  if (id) {
    g_qt_addr[g_qt_next] = QtAddrSlot{id, p};
    g_qt_next = (g_qt_next + 1) % kQtAddrSlots;
  }
  *out = p;
  return cudaSuccess;
}
}  // namespace star

extern "C" star_nt_status star_nt_quadtree_static(const uint32_t *rgba8, const int32_t *id1,
                                                  int32_t W, int32_t H,
                                                  const star_nt_params *params,
                                                  const uint32_t *mask_prev, uint32_t *mask_out,
                                                  star_nt_pass_state *state, void *stream) {
  if (!params || W <= 0 || H <= 0) return STAR_NT_ERR_ARG;
  size_t need = 0;
  if (star_nt_quadtree_ws_bytes(W, H, params->base_tile, &need) != STAR_NT_OK) return STAR_NT_ERR_ARG;
  const QtLayout L = qt_layout(W, H, params->base_tile);
  if ((int64_t)L.tiles_x * L.tiles_y > kQtStaticMaxTiles || need > kQtStaticBytes)
    return STAR_NT_ERR_CAPACITY;  // more tiles than the fixed workspace holds
  void *ws = nullptr;
  if (qt_scratch_address(&ws) != cudaSuccess) return STAR_NT_ERR_CUDA;
  return star_nt_quadtree(rgba8, id1, W, H, params, mask_prev, mask_out, state, ws, kQtStaticBytes,
                          stream);
}

namespace star {
// Loads this file's kernels onto the current device (see star_nt_preload).
cudaError_t preload_quadtree() {
  cudaFuncAttributes a;
  cudaError_t e = cudaSuccess, r;
  if ((r = cudaFuncGetAttributes(&a, k_qt_decide)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_qt_relax)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_qt_last<true, 16>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_qt_last<false, 16>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_qt_last<true, 64>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_qt_last<false, 64>)) != cudaSuccess) e = r;
  return e;
}
}  // namespace star
