// passes_resolve.cu -- star_nt_geometry_passes_resolve: the persistent
// geometry-pass launch of star_nt_geometry_passes that, when both reduced
// passes are merged into pass 1 (every pass at the full resolution), also
// produces the frame: each pass-1 tile CTA turns its 256 pixels' two nearest
// fragments and tail sums into the network input (Sec. 3.3), runs the tail MLP
// on the tcgen05 tensor cores as two M = 128 tiles (bf16 operands, fp32
// accumulation in tensor memory, biases inside the MMAs as in star_nt_resolve)
// and writes the composite of Eq. 4.  The reduced planes then never reach
// memory and the frame needs no separate resolve; the launch marks pass 2's
// bins header resolved, and star_nt_resolve returns at once.  With the passes
// at reduced sizes it is star_nt_geometry_passes.
//
// The upscale of a full-resolution plane is the identity (tap weight 1), so
// the frame equals the one star_nt_resolve computes from the planes, bit for
// bit.  Thread t of the CTA owns row t % 128 of MLP tile t / 128; warps 0-3
// read tensor-memory lanes of tile 0, warps 4-7 those of tile 1.
#include <math.h>

#include "pass_body.cuh"
#include "tc_primitives.cuh"

namespace star {

struct ResolveArgs {
  const float *w1, *b1, *w2, *b2, *w3, *b3;
  float bg0, bg1, bg2, kappa;
  float4 *out;
  uint32_t *out8;
  unsigned long long wait_ns;  // bound of the MMA waits
};

// Static shared memory of the launch: the tile's staging area, reused for the
// two 128-row MLP operand tiles once the tile's traversal is over (per tile
// 8 KB: X in the first core column, then H1 in four, then H2 in two), then
// the constant operands (the ones and zero blocks of the bias columns, the
// weights in the K-major core-matrix layout of star_nt_resolve) and the MMA
// barrier.  The ones block follows the operand tiles, so the layer-1 A
// operand [X | ones] has a positive core-column stride.
constexpr uint32_t kTmemCols = 64;  // 32 columns per MLP tile
struct __align__(128) FusedSmem {
  union {
    TileStage stage;   // one pixel per thread: for_each_fragment
    WalkStage wstage;  // two pixels per thread: walk_tile2
    uint8_t h[2][8192];
  } u;
  __align__(128) uint8_t ones[2048];
  uint8_t zeros[2048];
  uint8_t w1[1024];  // N = 32, K = 16 (bias in K 8, 9): 2 core columns of 512 bytes
  uint8_t w2[1536];  // N = 16, K = 48 (bias in K 32, 33): 6 of 256
  uint8_t w3[1024];  // N = 16, K = 32 (bias in K 16, 17): 4 of 256
  unsigned long long bar;
  uint32_t tmem;
  volatile int abort;
};

// One pass-1 tile with every pass merged: traversal, network input, the three
// MLP layers on tcgen05, composite.  Called by all 256 threads.  ph is the
// phase of the MMA barrier (three completions per tile).
template <int BW>
__device__ __forceinline__ void pass_resolve_body(const BinsView &bv, const uint32_t *__restrict__ rgba8,
                                                  const PassOut &po, const ResolveArgs &ra,
                                                  FusedSmem &fs, uint32_t tmem, uint32_t &ph,
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
      bv, tile, tp, fs.u.stage, [&] { return acc.template bound<kTail>(inside); },
      [&](const TriSetup &T, uint32_t id, long long e0, long long e2) {
        acc.template visit<kTail>(T, (int)id, e0, e2);
      });
  float xv[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float4 front = make_float4(0.f, 0.f, 0.f, 0.f);
  const size_t p = (size_t)tp.py * W + tp.px;
  if (inside) acc.resolve_terms(bv.setups, rgba8, po, ra.bg0, ra.bg1, ra.bg2, ra.kappa, p, xv, front);
  const bool flag = xv[5] != 0.0f;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int t = tid >> 7, row = tid & 127;
  __syncthreads();  // every warp is done with the staging area
  uint8_t *h = fs.u.h[t];
  *reinterpret_cast<uint4 *>(h + row * 16) =
      make_uint4(pack_bf16(xv[0], xv[1]), pack_bf16(xv[2], xv[3]), pack_bf16(xv[4], xv[5]), 0u);
  const uint32_t bar = smem_u32(&fs.bar);
  const uint32_t lane_tmem = tmem + ((uint32_t)((warp & 3) * 32) << 16) + 32u * t;
  fence_async_smem();
  fence_before();
  __syncthreads();
  // ---- layer 1: [X | ones] (K = 16) against [W1 | b1], N = 32
  if (tid == 0) {
    fence_after();
    const uint64_t dW1 = smem_desc(smem_u32(fs.w1), 512, 128);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const uint32_t a = smem_u32(fs.u.h[k]);
      mma_bf16(tmem + 32 * k, smem_desc(a, smem_u32(fs.ones) - a, 128), dW1, idesc_bf16(32), 0u);
    }
    mma_commit(bar);
  }
  mma_wait_cta(bar, ph, &fs.abort, ra.wait_ns);
  ph ^= 1u;
  // eight columns (one K core column of H1) per tensor-memory load: the
  // register budget of the pass traversal leaves no room for wider loads
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    float d[8];
    tmem_ld8(lane_tmem + 8 * kc, d);
    *reinterpret_cast<uint4 *>(h + kc * 2048 + row * 16) =
        make_uint4(pack_relu_bf16(d[0], d[1]), pack_relu_bf16(d[2], d[3]), pack_relu_bf16(d[4], d[5]),
                   pack_relu_bf16(d[6], d[7]));
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  // ---- layer 2: [H1 | ones | 0] (K = 48) against [W2 | b2], N = 16, over D1
  if (tid == 0 && !fs.abort) {
    fence_after();
    const uint32_t w2 = smem_u32(fs.w2);
    const uint64_t dOnes = smem_desc(smem_u32(fs.ones), 2048, 128);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const uint32_t a = smem_u32(fs.u.h[k]);
      mma_bf16(tmem + 32 * k, smem_desc(a, 2048, 128), smem_desc(w2, 256, 128), idesc_bf16(16), 0u);
      mma_bf16(tmem + 32 * k, smem_desc(a + 4096, 2048, 128), smem_desc(w2 + 512, 256, 128),
               idesc_bf16(16), 1u);
      mma_bf16(tmem + 32 * k, dOnes, smem_desc(w2 + 1024, 256, 128), idesc_bf16(16), 1u);
    }
    mma_commit(bar);
  }
  if (!fs.abort) mma_wait_cta(bar, ph, &fs.abort, ra.wait_ns);  // fs.abort is uniform after a barrier
  ph ^= 1u;
#pragma unroll
  for (int kc = 0; kc < 2; ++kc) {
    float d[8];
    tmem_ld8(lane_tmem + 8 * kc, d);
    *reinterpret_cast<uint4 *>(h + kc * 2048 + row * 16) =
        make_uint4(pack_relu_bf16(d[0], d[1]), pack_relu_bf16(d[2], d[3]), pack_relu_bf16(d[4], d[5]),
                   pack_relu_bf16(d[6], d[7]));
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  // ---- layer 3: [H2 | ones | 0] (K = 32) against [W3 | b3], D3 in columns 16..31
  if (tid == 0 && !fs.abort) {
    fence_after();
    const uint32_t w3 = smem_u32(fs.w3);
    const uint64_t dOnes = smem_desc(smem_u32(fs.ones), 2048, 128);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      mma_bf16(tmem + 32 * k + 16, smem_desc(smem_u32(fs.u.h[k]), 2048, 128), smem_desc(w3, 256, 128),
               idesc_bf16(16), 0u);
      mma_bf16(tmem + 32 * k + 16, dOnes, smem_desc(w3 + 512, 256, 128), idesc_bf16(16), 1u);
    }
    mma_commit(bar);
  }
  if (!fs.abort) mma_wait_cta(bar, ph, &fs.abort, ra.wait_ns);  // fs.abort is uniform after a barrier
  ph ^= 1u;
  // ---- composite, Eq. 4
  {
    uint32_t r[4];
    asm volatile("{\n tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n tcgen05.wait::ld.sync.aligned;\n}"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(lane_tmem + 16)
                 : "memory");
    if (inside) {
      float f0 = 0.f, f1 = 0.f, f2 = 0.f;
      if (flag) {
        f0 = fmaxf(__uint_as_float(r[0]), 0.0f);
        f1 = fmaxf(__uint_as_float(r[1]), 0.0f);
        f2 = fmaxf(__uint_as_float(r[2]), 0.0f);
      }
      const float cr = fmaf(front.w, f0, front.x), cg = fmaf(front.w, f1, front.y),
                  cb = fmaf(front.w, f2, front.z);
      if (ra.out) ra.out[p] = make_float4(cr, cg, cb, 1.0f);
      if (ra.out8) ra.out8[p] = quantize_rgba8(cr, cg, cb);
    }
  }
  fence_before();
  __syncthreads();  // tensor memory and the operand tiles are free for the next tile
}

// pass_resolve_body with two pixels per thread (a CTA of 128 threads per
// tile, see tile_pixel): thread t owns row t of both MLP tiles, its first
// pixel in tile 0 and its second in tile 1; warp w reads tensor-memory lanes
// 32 w .. 32 w + 31 of both.
template <int BW>
__device__ __forceinline__ void pass_resolve_body2(const BinsView &bv, const uint32_t *__restrict__ rgba8,
                                                   const PassOut &po, const ResolveArgs &ra,
                                                   FusedSmem &fs, uint32_t tmem, uint32_t &ph,
                                                   int tile) {
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
  walk_tile2<kTail, BW>(bv, tile, tp, fs.u.wstage, in0, in1, a0, a1);
  float xv0[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, xv1[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float4 front0 = make_float4(0.f, 0.f, 0.f, 0.f), front1 = front0;
  const size_t p0 = (size_t)tp.py * W + tp.px, p1 = p0 + (size_t)BH * W;
  if (in0) a0.resolve_terms(bv.setups, rgba8, po, ra.bg0, ra.bg1, ra.bg2, ra.kappa, p0, xv0, front0);
  if (in1) a1.resolve_terms(bv.setups, rgba8, po, ra.bg0, ra.bg1, ra.bg2, ra.kappa, p1, xv1, front1);
  const bool flag0 = xv0[5] != 0.0f, flag1 = xv1[5] != 0.0f;
  const int tid = threadIdx.x, warp = tid >> 5, row = tid;
  __syncthreads();  // every warp is done with the staging area
  *reinterpret_cast<uint4 *>(fs.u.h[0] + row * 16) =
      make_uint4(pack_bf16(xv0[0], xv0[1]), pack_bf16(xv0[2], xv0[3]), pack_bf16(xv0[4], xv0[5]), 0u);
  *reinterpret_cast<uint4 *>(fs.u.h[1] + row * 16) =
      make_uint4(pack_bf16(xv1[0], xv1[1]), pack_bf16(xv1[2], xv1[3]), pack_bf16(xv1[4], xv1[5]), 0u);
  const uint32_t bar = smem_u32(&fs.bar);
  const uint32_t lane_tmem = tmem + ((uint32_t)(warp * 32) << 16);
  fence_async_smem();
  fence_before();
  __syncthreads();
  // ---- layer 1: [X | ones] (K = 16) against [W1 | b1], N = 32
  if (tid == 0) {
    fence_after();
    const uint64_t dW1 = smem_desc(smem_u32(fs.w1), 512, 128);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const uint32_t a = smem_u32(fs.u.h[k]);
      mma_bf16(tmem + 32 * k, smem_desc(a, smem_u32(fs.ones) - a, 128), dW1, idesc_bf16(32), 0u);
    }
    mma_commit(bar);
  }
  mma_wait_cta(bar, ph, &fs.abort, ra.wait_ns);
  ph ^= 1u;
#pragma unroll
  for (int t = 0; t < 2; ++t)
#pragma unroll
    for (int kc = 0; kc < 4; kc += 2) {  // two K core columns of H1 per tensor-memory load
      float d[16];
      tmem_ld16(lane_tmem + 32 * t + 8 * kc, d);
#pragma unroll
      for (int h = 0; h < 2; ++h)
        *reinterpret_cast<uint4 *>(fs.u.h[t] + (kc + h) * 2048 + row * 16) =
            make_uint4(pack_relu_bf16(d[8 * h], d[8 * h + 1]), pack_relu_bf16(d[8 * h + 2], d[8 * h + 3]),
                       pack_relu_bf16(d[8 * h + 4], d[8 * h + 5]), pack_relu_bf16(d[8 * h + 6], d[8 * h + 7]));
    }
  fence_async_smem();
  fence_before();
  __syncthreads();
  // ---- layer 2: [H1 | ones | 0] (K = 48) against [W2 | b2], N = 16, over D1
  if (tid == 0 && !fs.abort) {
    fence_after();
    const uint32_t w2 = smem_u32(fs.w2);
    const uint64_t dOnes = smem_desc(smem_u32(fs.ones), 2048, 128);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const uint32_t a = smem_u32(fs.u.h[k]);
      mma_bf16(tmem + 32 * k, smem_desc(a, 2048, 128), smem_desc(w2, 256, 128), idesc_bf16(16), 0u);
      mma_bf16(tmem + 32 * k, smem_desc(a + 4096, 2048, 128), smem_desc(w2 + 512, 256, 128),
               idesc_bf16(16), 1u);
      mma_bf16(tmem + 32 * k, dOnes, smem_desc(w2 + 1024, 256, 128), idesc_bf16(16), 1u);
    }
    mma_commit(bar);
  }
  if (!fs.abort) mma_wait_cta(bar, ph, &fs.abort, ra.wait_ns);  // fs.abort is uniform after a barrier
  ph ^= 1u;
#pragma unroll
  for (int t = 0; t < 2; ++t) {  // both K core columns of H2 in one tensor-memory load
    float d[16];
    tmem_ld16(lane_tmem + 32 * t, d);
#pragma unroll
    for (int h = 0; h < 2; ++h)
      *reinterpret_cast<uint4 *>(fs.u.h[t] + h * 2048 + row * 16) =
          make_uint4(pack_relu_bf16(d[8 * h], d[8 * h + 1]), pack_relu_bf16(d[8 * h + 2], d[8 * h + 3]),
                     pack_relu_bf16(d[8 * h + 4], d[8 * h + 5]), pack_relu_bf16(d[8 * h + 6], d[8 * h + 7]));
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  // ---- layer 3: [H2 | ones | 0] (K = 32) against [W3 | b3], D3 in columns 16..31
  if (tid == 0 && !fs.abort) {
    fence_after();
    const uint32_t w3 = smem_u32(fs.w3);
    const uint64_t dOnes = smem_desc(smem_u32(fs.ones), 2048, 128);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      mma_bf16(tmem + 32 * k + 16, smem_desc(smem_u32(fs.u.h[k]), 2048, 128), smem_desc(w3, 256, 128),
               idesc_bf16(16), 0u);
      mma_bf16(tmem + 32 * k + 16, dOnes, smem_desc(w3 + 512, 256, 128), idesc_bf16(16), 1u);
    }
    mma_commit(bar);
  }
  if (!fs.abort) mma_wait_cta(bar, ph, &fs.abort, ra.wait_ns);  // fs.abort is uniform after a barrier
  ph ^= 1u;
  // ---- composite, Eq. 4
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    uint32_t r[4];
    asm volatile("{\n tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n tcgen05.wait::ld.sync.aligned;\n}"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(lane_tmem + 32 * t + 16)
                 : "memory");
    const bool in = t ? in1 : in0, flag = t ? flag1 : flag0;
    const float4 front = t ? front1 : front0;
    const size_t p = t ? p1 : p0;
    if (in) {
      float f0 = 0.f, f1 = 0.f, f2 = 0.f;
      if (flag) {
        f0 = fmaxf(__uint_as_float(r[0]), 0.0f);
        f1 = fmaxf(__uint_as_float(r[1]), 0.0f);
        f2 = fmaxf(__uint_as_float(r[2]), 0.0f);
      }
      const float cr = fmaf(front.w, f0, front.x), cg = fmaf(front.w, f1, front.y),
                  cb = fmaf(front.w, f2, front.z);
      if (ra.out) ra.out[p] = make_float4(cr, cg, cb, 1.0f);
      if (ra.out8) ra.out8[p] = quantize_rgba8(cr, cg, cb);
    }
  }
  fence_before();
  __syncthreads();  // tensor memory and the operand tiles are free for the next tile
}

// The fused launch: with both reduced passes merged, every pass-1 tile runs
// pass_resolve_body (items from a work counter, as k_passes); otherwise every
// CTA returns at once and star_nt_geometry_passes' launch that follows does
// the passes.  Tensor memory is allocated by every CTA at the start (and
// released on either exit); the constant operands are staged once per CTA.
// PIX = 1: 256 threads, 6 CTAs per SM (the 40-register budget); PIX = 2:
// 128 threads with two pixels each, 8 CTAs per SM (8 x 64 columns: all of
// tensor memory).
template <int BW, int PIX = 1>
__global__ void __launch_bounds__(PIX == 2 ? 128 : 256, PIX == 2 ? 8 : 6)
    k_passes_resolve(BinsView v1, BinsView v2, BinsView v3, const uint32_t *__restrict__ rgba8,
                     PassOut o1, ResolveArgs ra, uint32_t *queue, int32_t *status) {
  extern __shared__ uint8_t smem_raw[];  // FusedSmem, 128-byte aligned
  // rounded up to 128 bytes by pointer arithmetic on the shared array, so
  // that the compiler keeps every access in the shared address space
  FusedSmem &fs = *reinterpret_cast<FusedSmem *>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
  __shared__ int s_item;
  const int tid = threadIdx.x;
  if (tid < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&fs.tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  const bool fuse = v2.hd->merged != 0 && v3.hd->merged != 0;  // uniform over the launch
  if (fuse) {
    if (blockIdx.x == 0 && tid == 0) v2.hd->resolved = 1;
    for (int i = tid; i < (int)(sizeof(fs.zeros) + sizeof(fs.w1) + sizeof(fs.w2) + sizeof(fs.w3)) / 4;
         i += blockDim.x)
      reinterpret_cast<uint32_t *>(fs.zeros)[i] = 0u;
    __syncthreads();
    put_ones_block(fs.ones, tid, blockDim.x);
    for (int i = tid; i < 32 * 5; i += blockDim.x) put_w(fs.w1, i / 5, i % 5, 512, ra.w1[i]);
    for (int i = tid; i < 16 * 32; i += blockDim.x) put_w(fs.w2, i / 32, i % 32, 256, ra.w2[i]);
    for (int i = tid; i < 3 * 16; i += blockDim.x) put_w(fs.w3, i / 16, i % 16, 256, ra.w3[i]);
    if (tid < 32) put_bias(fs.w1, tid, 8, 512, ra.b1[tid]);
    if (tid < 16) put_bias(fs.w2, tid, 32, 256, ra.b2[tid]);
    if (tid < 3) put_bias(fs.w3, tid, 16, 256, ra.b3[tid]);
    if (tid == 0) {
      mbar_init(smem_u32(&fs.bar), 1);
      fs.abort = 0;
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_async_smem();
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = fs.tmem;
  if (fuse) {
    PassOut om = o1;  // pass 1 writes id1 and z1; the merged planes are not needed
    om.id2 = nullptr;
    om.n = nullptr;
    om.tail = nullptr;
    om.t_tail = nullptr;
    const int total = v1.hd->n_tiles;
    uint32_t ph = 0u;
    for (;;) {
      if (tid == 0) s_item = (int)atomicAdd(queue, 1u);
      __syncthreads();
      const int item = s_item;
      const bool aborted = fs.abort != 0;
      __syncthreads();  // every thread has the item before s_item is reused
      if (item >= total || aborted) {
        // the last CTA out resets the queue and the exit count for the next launch
        if (tid == 0 && atomicAdd(queue + 1, 1u) == gridDim.x - 1) {
          queue[0] = 0u;
          queue[1] = 0u;
        }
        break;
      }
      if (PIX == 2) pass_resolve_body2<BW>(v1, rgba8, om, ra, fs, tmem, ph, item);
      else pass_resolve_body<BW>(v1, rgba8, om, ra, fs, tmem, ph, item);
    }
    if (fs.abort && tid == 0) raise_status(status, STAR_NT_ERR_TIMEOUT);
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (tid < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                 : "memory");
}

}  // namespace star

using namespace star;

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static PassOut pass_out_of(const star_nt_layers *l) {
  PassOut o = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  o.id1 = l->id1;
  o.z1 = l->z1;
  return o;
}

// dynamic shared memory of one CTA (FusedSmem and its alignment slack)
constexpr size_t kFusedSmemBytes = sizeof(FusedSmem) + 128;
static_assert(kFusedSmemBytes <= 48 * 1024, "dynamic shared memory within the default limit");

extern "C" star_nt_status star_nt_geometry_passes_resolve(
    const star_nt_scene *scene, const star_nt_bins *b1, const star_nt_bins *b2, const star_nt_bins *b3,
    const star_nt_layers *l1, const star_nt_layers *l2, const star_nt_layers *l3,
    const star_nt_params *params, const star_nt_mlp *w, float *rgba32f, uint32_t *rgba8,
    const star_nt_tuning *tuning, int32_t *d_status, void *stream) {
  if (!scene || !b1 || !b2 || !b3 || !b1->mem || !b2->mem || !b3->mem || !l1 || !l2 || !l3 || !params)
    return STAR_NT_ERR_ARG;
  if ((!l1->id1 && !l1->z1) || !l2->id2 || !l3->n || !l3->tail || !l3->t_tail) return STAR_NT_ERR_ARG;
  for (const star_nt_layers *l : {l1, l2, l3})
    if (!aligned16(l->id1) || !aligned16(l->z1) || !aligned16(l->id2) || !aligned16(l->n) ||
        !aligned16(l->tail) || !aligned16(l->t_tail))
      return STAR_NT_ERR_ARG;
  if (!w || !w->w1 || !w->b1 || !w->w2 || !w->b2 || !w->w3 || !w->b3 || (!rgba32f && !rgba8))
    return STAR_NT_ERR_ARG;
  if (!aligned16(rgba32f)) return STAR_NT_ERR_ARG;
  if (scene->n_tris > 0 && !scene->rgba8) return STAR_NT_ERR_ARG;
  if (b1->mem == b2->mem || b1->mem == b3->mem || b2->mem == b3->mem) return STAR_NT_ERR_ARG;
  PassTuning tu;
  if (!pass_tuning(tuning, tu)) return STAR_NT_ERR_ARG;
  const int bw = tu.bw, per_sm = tu.per_sm;
  cudaStream_t st = (cudaStream_t)stream;
  BinsView v1 = bins_view(*b1), v2 = bins_view(*b2), v3 = bins_view(*b3);
  PassOut o1 = pass_out_of(l1);
  ResolveArgs ra = {w->w1, w->b1, w->w2, w->b2, w->w3, w->b3, params->bg[0], params->bg[1],
                    params->bg[2], params->kappa_n, reinterpret_cast<float4 *>(rgba32f), rgba8,
                    wait_limit_ns()};
  uint32_t *queue = &v1.hd->queue;  // queue[0] work counter, queue[1] exit count
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // one pixel per thread: 6 CTAs of 256 threads per SM (the 40-register
  // budget; 6 x 64 tensor-memory columns of the SM's 512); two pixels per
  // thread: 8 CTAs of 128 threads (8 x 64 columns); fewer when tuned
  const int cmax = tu.pix == 2 ? 8 : 6;
  const int c = per_sm > 0 && per_sm < cmax ? per_sm : cmax;
  const int threads = tu.pix == 2 ? 128 : 256;
  auto launch = [&](auto kern) {
    kern<<<sms * c, threads, kFusedSmemBytes, st>>>(v1, v2, v3, scene->rgba8, o1, ra, queue, d_status);
  };
  if (tu.pix == 2) {
    if (bw == 8) launch(k_passes_resolve<8, 2>);
    else if (bw == 16) launch(k_passes_resolve<16, 2>);
    else launch(k_passes_resolve<4, 2>);
  } else {
    if (bw == 8) launch(k_passes_resolve<8>);
    else if (bw == 16) launch(k_passes_resolve<16>);
    else launch(k_passes_resolve<4>);
  }
  if (cudaGetLastError() != cudaSuccess) return STAR_NT_ERR_CUDA;
  // the passes themselves when a reduced pass is not merged (returns at once
  // when the launch above resolved the frame)
  return star_nt_geometry_passes(scene, b1, b2, b3, l1, l2, l3, tuning, d_status, stream);
}

namespace star {
// Loads this file's kernels onto the current device (see star_nt_preload).
cudaError_t preload_passes_resolve() {
  cudaFuncAttributes a;
  cudaError_t e = cudaSuccess, r;
  if ((r = cudaFuncGetAttributes(&a, k_passes_resolve<4>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes_resolve<8>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes_resolve<16>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes_resolve<4, 2>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes_resolve<8, 2>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_passes_resolve<16, 2>)) != cudaSuccess) e = r;
  return e;
}
}  // namespace star
