// tile_walk.cuh -- the tile traversal of the two-pixel pass kernels: CTAs of
// 128 threads, one 16 x 16 tile each; warp w owns a BW x (64 / BW) block of it
// and lane l the pixels (l % BW, l / BW) and (l % BW, l / BW + 32 / BW) of that
// block (see tile_pixel).
//
// Edge functions in 32 bits.  E_e(P) = dx_e Py - dy_e Px + c_e is exact in
// int64 (sub-pixel coordinates within the guard band, so |dx_e|, |dy_e| <=
// 2^24).  Inside one tile P = P00 + 256 (x, y) for its pixel (x, y), so
// E_e = E00 + 256 (dx_e y - dy_e x), and with g = floor(E00 / 256) and
// r = E00 - 256 g in [0, 255]:
//     E_e >= 0  <=>  g + dx_e y - dy_e x >= 0,
// because dx_e y - dy_e x is an integer.  |dx_e y - dy_e x| < 2^29 for
// x, y < 16, so clamping g to [-2^30, 2^30] keeps the sign of every pixel's
// test and every sum within int32.  A pixel's biased edge value is then
// 256 (g + dx_e y - dy_e x) + r.  When the doubled area fits int32
// (TriSetup::own & kOwnSmall), the edge values of covered pixels lie in
// [-1, area] and fit too, and g was never clamped (|E00| < 2^31 + 15 * 256 *
// (|dx_e| + |dy_e|) < 2^38), so the fragment depth takes its edge values from
// 32-bit arithmetic as well; other triangles take them in int64.  Coverage,
// fragment sets, depths and sums are those of the int64 evaluation, bit for bit.
//
// Each staging round sorts the tile's binned triangles by depth lower bound
// (ties by binned position), so that near triangles come first: a pixel then
// evaluates the depth of a fragment only while the fragment may still enter
// its k nearest.  From the first triangle that lies behind every lane's k-th
// depth on, no later one of the round can enter any pixel's k nearest: the
// passes without tail sums stop the warp's walk there, and the tail passes
// finish the round in a loop that only tests coverage and adds tail sums.
#pragma once

#include "raster_tile.cuh"

namespace star {

constexpr int kWalkChunk = 128;  // triangles staged per round (one per thread)

// Shared-memory staging area of one tile CTA.
struct WalkStage {
  TriSetup tri[kWalkChunk];
  int4 te[kWalkChunk];  // g of edges 0..2 (clamped) and the depth biases u_0 | u_2 << 16 (below)
  uint32_t id[kWalkChunk];
  float key[kWalkChunk];
  uint8_t list[4][kWalkChunk];  // per-warp lists of staged triangles touching the block
  uint8_t perm[kWalkChunk];     // perm[r] = slot of the triangle of rank r
};

// g of the three edges at the centre of the tile's pixel (0, 0), and for
// edges 0 and 2 the term u_e = r_e - (own_e - 1) in [0, 256] that turns
// 256 (g_e + dx_e y - dy_e x) into the edge function's value without its tie
// bias (the value the fragment depth takes).
__device__ __forceinline__ int4 tile_edge_bases(const int4 &p0, const int4 &p1, const int4 &p2, uint32_t own,
                                                int tx0, int ty0) {
  // the set-up's first 48 bytes: dx[3], dy[3], c[3] (int64, low word first)
  const int dx[3] = {p0.x, p0.y, p0.z}, dy[3] = {p0.w, p1.x, p1.y};
  const long long c[3] = {(long long)(((unsigned long long)(uint32_t)p1.w << 32) | (uint32_t)p1.z),
                          (long long)(((unsigned long long)(uint32_t)p2.y << 32) | (uint32_t)p2.x),
                          (long long)(((unsigned long long)(uint32_t)p2.w << 32) | (uint32_t)p2.z)};
  const int Px0 = tx0 * kSub + kSub / 2, Py0 = ty0 * kSub + kSub / 2;
  int g[3];
  uint32_t r[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const long long E = (long long)dx[e] * Py0 + c[e] - (long long)dy[e] * Px0;
    const long long q = E >> 8;  // floor(E / 256): arithmetic shift
    r[e] = (uint32_t)(E & 255);
    g[e] = (int)(q < -(1ll << 30) ? -(1ll << 30) : (q > (1ll << 30) ? (1ll << 30) : q));
  }
  const uint32_t u0 = r[0] - (own & 1u) + 1u, u2 = r[2] - ((own >> 2) & 1u) + 1u;
  return make_int4(g[0], g[1], g[2], (int)(u0 | u2 << 16));
}

// Stages binned entries [base, base + n), n <= kWalkChunk <= blockDim.x:
// thread t < n copies entry t's set-up to slot t with 16-byte asynchronous
// copies as soon as its id is known, stores its key and the tile's edge
// bases beside it, then ranks the key among the round's keys (ties by binned
// position): perm[r] is the slot of rank r, so the round is walked sorted by
// (depth lower bound, binned position).
__device__ __forceinline__ void walk_stage(const BinsView &bv, uint32_t base, int n, WalkStage &st,
                                           int tx0, int ty0) {
  const int t = threadIdx.x;
  float kt = 0.0f;
  if (t < n) {
    const uint32_t id = __ldg(bv.pairs + base + t);
    const int4 *g = reinterpret_cast<const int4 *>(bv.setups + id);
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(st.tri + t);
#pragma unroll
    for (int p = 0; p < 7; ++p)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d + 16u * p), "l"(g + p) : "memory");
    kt = __ldg(&bv.setups[id].zlo);
    st.key[t] = kt;
    st.id[t] = id;
    st.te[t] = tile_edge_bases(__ldg(g), __ldg(g + 1), __ldg(g + 2), (uint32_t)__ldg(g + 4).z, tx0, ty0);
  }
  __syncthreads();  // the keys
  if (t < n) {
    int r = 0;
    for (int j = 0; j < n; ++j) {
      const float kj = st.key[j];
      r += (kj < kt || (kj == kt && j < t)) ? 1 : 0;
    }
    st.perm[r] = (uint8_t)t;
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();  // the permutation and the set-ups
}

// May the triangle cover a pixel centre of the BW x BH2 block at tile-local
// (bxl, byl) (absolute origin bx0, by0)?  False only when it certainly does
// not: the bounding box, or one edge negative at every centre of the block
// (its largest value over the block is at one corner).
template <int BW, int BH2>
__device__ __forceinline__ bool block_maybe32(const TriSetup &T, const int4 &te, int bx0, int by0,
                                              int bxl, int byl) {
  if (T.xb < bx0 || T.xa > bx0 + BW - 1 || T.yb < by0 || T.ya > by0 + BH2 - 1) return false;
  const int gb[3] = {te.x, te.y, te.z};
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int dx = T.dx[e], dy = T.dy[e];
    const int mx = gb[e] + dx * (dx > 0 ? byl + BH2 - 1 : byl) - dy * (dy > 0 ? bxl : bxl + BW - 1);
    if (mx < 0) return false;
  }
  return true;
}

// Canonical float32 depth of a covered pixel (the arithmetic of frag_depth)
// from the pixel's tile-relative values of edges 0 and 2 (ga, gc) and their
// depth terms (u = u_0 | u_2 << 16), or, for a triangle whose area does not
// fit int32, from the int64 edge functions at the pixel centre (Px, Py).
// 256 g + u, taken modulo 2^32, is the edge function's value without its tie
// bias: it fits int32 when the area does.  The depth plane pl = (z0, dz1,
// dz2, r) and the ownership bits own are the triangle's, loaded once by the
// caller for both of its pixels.
__device__ __forceinline__ float frag_depth_tile(const TriSetup &T, float4 pl, uint32_t own, int ga, int gc,
                                                 uint32_t u, int Px, int Py) {
  float f20, f01;
  if (own & kOwnSmall) {
    const int e01 = (int)(((uint32_t)ga << 8) + (u & 0xFFFFu));
    const int e20 = (int)(((uint32_t)gc << 8) + (u >> 16));
    f20 = __int2float_rn(e20);
    f01 = __int2float_rn(e01);
  } else {
    const long long e0b = (long long)T.dx[0] * Py + T.c[0] - (long long)T.dy[0] * Px;
    const long long e2b = (long long)T.dx[2] * Py + T.c[2] - (long long)T.dy[2] * Px;
    f20 = __ll2float_rn(e2b - (long long)((own >> 2) & 1u) + 1);
    f01 = __ll2float_rn(e0b - (long long)(own & 1u) + 1);
  }
  const float b1 = __fmul_rn(f20, pl.w);
  const float b2 = __fmul_rn(f01, pl.w);
  const float z = __fadd_rn(__fadd_rn(pl.x, __fmul_rn(b1, pl.y)), __fmul_rn(b2, pl.z));
  return __fadd_rn(z, 0.0f);
}

// The traversal of one tile for both pixels of every thread.  Acc is the
// per-pixel state (PassAcc): accumulate_terms<MODE>(rg, ba, lg, c8) adds a
// fragment with its triangle's tail constants to the tail sums (MODE >=
// kTail), insert<KM>(z, id) offers it to the k nearest, z1 and z2 are the
// nearest depths so far.  A walked triangle's tail constants, depth plane and
// ownership bits are read from the staging area once for both pixels.  Called
// by all 128 threads, after a CTA barrier that follows every earlier use of st.
template <int MODE, int BW, class Acc>
__device__ __forceinline__ void walk_tile2(const BinsView &bv, int tile, const TilePixel &tp, WalkStage &st,
                                           bool in0, bool in1, Acc &a0, Acc &a1) {
  constexpr int BH = 32 / BW;
  constexpr bool TAIL = MODE >= 3;  // kTail, kFused, kFusedDfaoit
  constexpr int KM = MODE == 1 ? 1 : 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lx = tp.px - tp.tx0, ly = tp.py - tp.ty0;  // the second pixel is BH rows below
  const int bxl = tp.bx0 - tp.tx0, byl = tp.by0 - tp.ty0;
  const int Px = tp.px * kSub + kSub / 2, Py0 = tp.py * kSub + kSub / 2, Py1 = Py0 + BH * kSub;
  // a pixel outside the target never stores: its bounds start below every
  // depth, so it never evaluates one
  if (!in0) a0.z1 = a0.z2 = -INFINITY;
  if (!in1) a1.z1 = a1.z2 = -INFINITY;
  const uint32_t beg = bv.tile_offset[tile], end = bv.tile_offset[tile + 1];
  for (uint32_t base = beg; base < end; base += kWalkChunk) {
    const int n = (int)min((uint32_t)kWalkChunk, end - base);
    if (base != beg) __syncthreads();  // the walks of the previous round are over
    walk_stage(bv, base, n, st, tp.tx0, tp.ty0);
    int m = 0;
    for (int r0 = 0; r0 < n; r0 += 32) {  // in rank order; the lists hold slots
      const int r = r0 + lane;
      const int k = r < n ? st.perm[r] : 0;
      const bool hit = r < n && block_maybe32<BW, 2 * BH>(st.tri[k], st.te[k], tp.bx0, tp.by0, bxl, byl);
      const uint32_t b = __ballot_sync(0xffffffffu, hit);
      if (hit) st.list[warp][m + __popc(b & ((1u << lane) - 1u))] = (uint8_t)k;
      m += __popc(b);
    }
    __syncwarp();
    int i = 0;
    for (; i < m; ++i) {  // m is warp-uniform
      const int k = st.list[warp][i];
      const TriSetup &T = st.tri[k];
      // the k-th depth of each pixel
      const float b0 = KM == 1 ? a0.z1 : a0.z2;
      const float b1 = KM == 1 ? a1.z1 : a1.z2;
      // once this triangle lies behind every lane's bound, so does every
      // later one of the round (sorted keys, falling bounds): no depth is
      // needed any more, only the tail sums below
      if (__all_sync(0xffffffffu, T.zlo > fmaxf(b0, b1))) break;
      const int4 te = st.te[k];
      const int dx0 = T.dx[0], dx1 = T.dx[1], dx2 = T.dx[2];
      const int ga = te.x + dx0 * ly - T.dy[0] * lx;
      const int gb = te.y + dx1 * ly - T.dy[1] * lx;
      const int gc = te.z + dx2 * ly - T.dy[2] * lx;
      const int ha = ga + dx0 * BH, hb = gb + dx1 * BH, hc = gc + dx2 * BH;
      const bool c0 = (ga | gb | gc) >= 0, c1 = (ha | hb | hc) >= 0;
      if (!(c0 || c1)) continue;
      const int id = (int)st.id[k];
      const unsigned long long trg = T.rg, tba = T.ba, tlg = T.lg;
      const uint32_t tc8 = MODE == 5 ? T.c8 : 0u;  // kFusedDfaoit
      const float4 pl = make_float4(T.z0, T.dz1, T.dz2, T.r);
      const uint32_t own = T.own;
      if (c0) {
        if (TAIL) a0.template accumulate_terms<MODE>(trg, tba, tlg, tc8);
        if (!(T.zlo > b0)) a0.template insert<KM>(frag_depth_tile(T, pl, own, ga, gc, (uint32_t)te.w, Px, Py0), id);
      }
      if (c1) {
        if (TAIL) a1.template accumulate_terms<MODE>(trg, tba, tlg, tc8);
        if (!(T.zlo > b1)) a1.template insert<KM>(frag_depth_tile(T, pl, own, ha, hc, (uint32_t)te.w, Px, Py1), id);
      }
    }
    if (TAIL) {
      for (; i < m; ++i) {  // the rest of the round: coverage and tail sums
        const TriSetup &T = st.tri[st.list[warp][i]];
        const int4 te = st.te[st.list[warp][i]];
        const int dx0 = T.dx[0], dx1 = T.dx[1], dx2 = T.dx[2];
        const int ga = te.x + dx0 * ly - T.dy[0] * lx;
        const int gb = te.y + dx1 * ly - T.dy[1] * lx;
        const int gc = te.z + dx2 * ly - T.dy[2] * lx;
        const unsigned long long trg = T.rg, tba = T.ba, tlg = T.lg;
        const uint32_t tc8 = MODE == 5 ? T.c8 : 0u;  // kFusedDfaoit
        if ((ga | gb | gc) >= 0) a0.template accumulate_terms<MODE>(trg, tba, tlg, tc8);
        if (((ga + dx0 * BH) | (gb + dx1 * BH) | (gc + dx2 * BH)) >= 0)
          a1.template accumulate_terms<MODE>(trg, tba, tlg, tc8);
      }
    }
  }
}

}  // namespace star
