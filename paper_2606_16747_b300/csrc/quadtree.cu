// quadtree.cu -- star_nt_quadtree: adaptive screen-space tiles (Sec. 3.1)
// and tile-guided pass resolution (Sec. 3.2, Eq. 2).
//
// One warp per base tile; lane k < 21 owns the node whose split bit is bit k
// of the tile's mask (bit 0 root, bits 1..4 level-1 nodes, bits 5..20
// level-2 nodes), so ballots assemble new masks directly.  All decisions are
// taken on integer colour differences with correctly rounded float64 square
// roots summed in a fixed order, so they are reproducible bit for bit.
#include <math.h>

#include <mutex>

#include "common.cuh"

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

// Cells (level-3 cells, row-major bit index 8 cy + cx) covered by node k:
// k < 21 is the node of mask bit k, k >= 21 the level-3 cell k - 21.
struct RegionTable {
  unsigned long long m[85];
};
constexpr RegionTable make_regions() {
  RegionTable t{};
  for (int k = 0; k < 85; ++k) {
    int l = 3, i = 0, j = 0;
    if (k == 0) {
      l = 0;
    } else if (k < 5) {
      l = 1; i = (k - 1) & 1; j = (k - 1) >> 1;
    } else if (k < 21) {
      const int q = k - 5, c1 = q >> 2, c2 = q & 3;
      l = 2; i = (c1 & 1) * 2 + (c2 & 1); j = (c1 >> 1) * 2 + (c2 >> 1);
    } else {
      i = (k - 21) & 7; j = (k - 21) >> 3;
    }
    const int span = 8 >> l;
    unsigned long long r = 0;
    for (int b = 0; b < span; ++b)
      for (int a = 0; a < span; ++a) r |= 1ull << ((j * span + b) * 8 + (i * span + a));
    t.m[k] = r;
  }
  return t;
}
__constant__ RegionTable kRegions = make_regions();

// level of the leaf covering level-3 cell (cx, cy) of a tile, 0 <= cx, cy < 8
__device__ __forceinline__ int cell_level(uint32_t m, int cx, int cy) {
  if (!(m & 1u)) return 0;
  const int c1 = ((cy >> 2) << 1) | (cx >> 2);
  if (!((m >> (1 + c1)) & 1u)) return 1;
  const int c2 = (((cy >> 1) & 1) << 1) | ((cx >> 1) & 1);
  if (!((m >> (5 + 4 * c1 + c2)) & 1u)) return 2;
  return 3;
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
                                                   uint32_t *__restrict__ mout) {
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

// One relaxation iteration (Jacobi: reads min, writes mout), warp per tile.
// With LAST, the warp then counts the occupied leaves of its tile's final
// mask, and the last block to finish applies Eq. 2 and writes the state.
__device__ __forceinline__ bool relax_split(uint32_t m, uint32_t mL, uint32_t mR, uint32_t mU,
                                            uint32_t mD, int tx, int ty, int tiles_x, int tiles_y,
                                            int lane) {
  if (lane >= 21) return false;
  int l, i, j;
  node_of_bit(lane, l, i, j);
  if (!(node_exists(m, lane) && !((m >> lane) & 1u))) return false;
  const int span = 8 >> l, cx0 = i * span, cy0 = j * span;
  int deepest = 0;
  for (int k = 0; k < span; ++k) {
    // left / right columns and top / bottom rows just outside the leaf
    if (cx0 > 0) deepest = max(deepest, cell_level(m, cx0 - 1, cy0 + k));
    else if (tx > 0) deepest = max(deepest, cell_level(mL, 7, cy0 + k));
    if (cx0 + span < 8) deepest = max(deepest, cell_level(m, cx0 + span, cy0 + k));
    else if (tx + 1 < tiles_x) deepest = max(deepest, cell_level(mR, 0, cy0 + k));
    if (cy0 > 0) deepest = max(deepest, cell_level(m, cx0 + k, cy0 - 1));
    else if (ty > 0) deepest = max(deepest, cell_level(mU, cx0 + k, 7));
    if (cy0 + span < 8) deepest = max(deepest, cell_level(m, cx0 + k, cy0 + span));
    else if (ty + 1 < tiles_y) deepest = max(deepest, cell_level(mD, cx0 + k, 0));
  }
  return deepest >= l + 2;
}

template <bool RELAX, bool LAST>
__global__ void __launch_bounds__(256) k_qt_relax(const int32_t *__restrict__ id1, int W, int H, int B,
                                                  int tiles_x, int tiles_y,
                                                  const uint32_t *__restrict__ min,
                                                  uint32_t *__restrict__ mout,
                                                  uint32_t *__restrict__ hist, uint32_t *ticket,
                                                  double delta2, double delta3,
                                                  star_nt_pass_state *state) {
  __shared__ uint32_t s_hist[4];
  if (LAST) {
    if (threadIdx.x < 4) s_hist[threadIdx.x] = 0u;
    __syncthreads();
  }
  const int tile = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (tile < tiles_x * tiles_y) {
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    uint32_t m = min[tile];
    if (RELAX) {
      const uint32_t mL = tx > 0 ? min[tile - 1] : 0u, mR = tx + 1 < tiles_x ? min[tile + 1] : 0u;
      const uint32_t mU = ty > 0 ? min[tile - tiles_x] : 0u;
      const uint32_t mD = ty + 1 < tiles_y ? min[tile + tiles_x] : 0u;
      m |= __ballot_sync(0xffffffffu, relax_split(m, mL, mR, mU, mD, tx, ty, tiles_x, tiles_y, lane));
    }
    if (lane == 0) mout[tile] = m;
    if (LAST) {
      // occupancy of the tile's 64 level-3 cells (B/8 pixels wide)
      const int cs = B / 8;
      unsigned long long occ = 0;
      for (int k = lane; k < B * B; k += 32) {
        const int lx = k % B, ly = k / B;
        const int x = tx * B + lx, y = ty * B + ly;
        if (x < W && y < H && id1[(size_t)y * W + x] >= 0) occ |= 1ull << ((ly / cs) * 8 + (lx / cs));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) occ |= __shfl_xor_sync(0xffffffffu, occ, o);
      // leaves: lanes own the 21 nodes of levels 0..2, then the 64 level-3 cells
      uint32_t cnt[4] = {0, 0, 0, 0};
      for (int k = lane; k < 21 + 64; k += 32) {
        int l, i, j;
        bool isleaf;
        if (k < 21) {
          node_of_bit(k, l, i, j);
          isleaf = node_exists(m, k) && !((m >> k) & 1u);
        } else {
          l = 3;
          i = (k - 21) & 7;
          j = (k - 21) >> 3;
          isleaf = cell_level(m, i, j) == 3;
        }
        if (isleaf && (occ & kRegions.m[k])) ++cnt[l];
      }
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        uint32_t c = cnt[l];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0 && c) atomicAdd(&s_hist[l], c);
      }
    }
  }
  if (!LAST) return;
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
  if (!rgba8 || !id1 || !params || !mask_prev || !mask_out || !state || !ws || mask_prev == mask_out)
    return STAR_NT_ERR_ARG;
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
  cudaMemsetAsync(hist, 0, 32, st);  // histogram and the last-block ticket
  uint32_t *ticket = hist + 4;
  k_qt_decide<<<wblocks, 256, 0, st>>>(rgba8, W, H, B, L.tiles_x, nt, 6.0 * params->tau_split,
                                       6.0 * params->tau_merge, mask_prev, ma);
  const uint32_t *src = ma;
  for (int it = 0; it + 1 < iters; ++it) {  // all but the last relaxation
    uint32_t *d = src == ma ? mb : ma;
    k_qt_relax<true, false><<<wblocks, 256, 0, st>>>(id1, W, H, B, L.tiles_x, L.tiles_y, src, d, hist,
                                                     ticket, params->delta2, params->delta3, state);
    src = d;
  }
  // the last relaxation (a plain copy when there is none), the histogram of
  // occupied leaves and Eq. 2, in one launch
  if (iters > 0)
    k_qt_relax<true, true><<<wblocks, 256, 0, st>>>(id1, W, H, B, L.tiles_x, L.tiles_y, src, mask_out,
                                                    hist, ticket, params->delta2, params->delta3, state);
  else
    k_qt_relax<false, true><<<wblocks, 256, 0, st>>>(id1, W, H, B, L.tiles_x, L.tiles_y, src, mask_out,
                                                     hist, ticket, params->delta2, params->delta3, state);
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

constexpr int kMaxDevices = 64;
static std::mutex g_qt_mutex;
static void *g_qt_addr[kMaxDevices];  // device address of g_qt_scratch, per device

// Device address of the array on the current device, looked up once per
// device (with that device current) and cached.
static cudaError_t qt_scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_qt_mutex);
  if (!g_qt_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_qt_scratch);
    if (e != cudaSuccess) return e;
    g_qt_addr[dev] = p;
  }
  *out = g_qt_addr[dev];
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
