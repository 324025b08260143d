// train.cu -- the learned part: exact A-buffer resolve (the ground truth of
// Sec. 4 and the tail-colour target of Sec. 3.3), and training of the tail
// MLP with MSE and Adam (Sec. 3.3): loss gradient, backpropagation to the 771
// parameters, Adam update with a bf16 copy of the updated weights.
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"
#include "tc_primitives.cuh"

namespace star {

// ---------------------------------------------------------------------------
// A-buffer: per pixel, its fragments sorted by (z, primitive id), composited
// front to back; the tail colour composites fragments 3..N only.
constexpr int kLocalFrags = 96;

__device__ __forceinline__ bool key_less(float za, int ia, float zb, int ib) {
  return za < zb || (za == zb && ia < ib);
}

__device__ __forceinline__ void over_step(uint32_t c, float &T, float &r, float &g, float &b) {
  const float a = (float)(c >> 24) / 255.0f;
  const float w = T * a;
  r += w * ((float)(c & 255u) / 255.0f);
  g += w * ((float)((c >> 8) & 255u) / 255.0f);
  b += w * ((float)((c >> 16) & 255u) / 255.0f);
  T *= 1.0f - a;
}

__global__ void __launch_bounds__(128) k_abuffer(const uint32_t *__restrict__ count,
                                                 const uint32_t *__restrict__ offset,
                                                 const float *__restrict__ zs,
                                                 const int32_t *__restrict__ prims,
                                                 const uint32_t *__restrict__ rgba8, long long P,
                                                 float bg0, float bg1, float bg2,
                                                 float4 *__restrict__ rgb, float4 *__restrict__ tail) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const int n = (int)count[p];
  const uint32_t base = offset[p];
  float T = 1.0f, r = 0.f, g = 0.f, b = 0.f;       // whole pixel
  float Tt = 1.0f, rt = 0.f, gt = 0.f, bt = 0.f;   // tail (fragments 3..N)
  if (n <= kLocalFrags) {
    float z[kLocalFrags];
    int id[kLocalFrags];
    for (int i = 0; i < n; ++i) {  // insertion sort by (z, id)
      const float zi = zs[base + i];
      const int ii = prims[base + i];
      int j = i - 1;
      while (j >= 0 && key_less(zi, ii, z[j], id[j])) {
        z[j + 1] = z[j];
        id[j + 1] = id[j];
        --j;
      }
      z[j + 1] = zi;
      id[j + 1] = ii;
    }
    for (int i = 0; i < n; ++i) {
      const uint32_t c = __ldg(rgba8 + id[i]);
      over_step(c, T, r, g, b);
      if (i >= 2) over_step(c, Tt, rt, gt, bt);
    }
  } else {  // long lists: selection of the next key in order
    float zl = -INFINITY;
    int il = -1;
    for (int i = 0; i < n; ++i) {
      float zb = INFINITY;
      int ib = 0x7fffffff;
      for (int k = 0; k < n; ++k) {
        const float zk = zs[base + k];
        const int ik = prims[base + k];
        if (key_less(zl, il, zk, ik) && key_less(zk, ik, zb, ib)) { zb = zk; ib = ik; }
      }
      const uint32_t c = __ldg(rgba8 + ib);
      over_step(c, T, r, g, b);
      if (i >= 2) over_step(c, Tt, rt, gt, bt);
      zl = zb;
      il = ib;
    }
  }
  if (rgb) rgb[p] = make_float4(r + T * bg0, g + T * bg1, b + T * bg2, T);
  if (tail) tail[p] = make_float4(rt, gt, bt, Tt);
}

// ---------------------------------------------------------------------------
// MSE over B samples x 3 channels, optionally weighted per sample (w NULL:
// all 1): L = sum_i w_i |f_i - y_i|^2 / (3B), dL/df_i = 2 w_i (f_i - y_i) / (3B).
__global__ void __launch_bounds__(256) k_mse(const float4 *__restrict__ f, const float4 *__restrict__ y,
                                             const float *__restrict__ w, long long B,
                                             float4 *__restrict__ dy, float *__restrict__ partial) {
  __shared__ float s[8];
  const float scale = 1.0f / (3.0f * (float)B);
  float acc = 0.0f;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < B; i += (long long)gridDim.x * 256) {
    const float4 a = f[i], t = y[i];
    const float wi = w ? w[i] : 1.0f;
    const float dx = a.x - t.x, dyv = a.y - t.y, dz = a.z - t.z;
    acc += wi * (dx * dx + dyv * dyv + dz * dz);
    const float k = 2.0f * wi * scale;
    dy[i] = make_float4(k * dx, k * dyv, k * dz, 0.0f);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < 8; ++w) t += s[w];
    partial[blockIdx.x] = t * scale;
  }
}

__global__ void k_sum_partials(const float *__restrict__ partial, int n, float *__restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float t = 0.0f;
    for (int i = 0; i < n; ++i) t += partial[i];
    *out = t;
  }
}

// ---------------------------------------------------------------------------
// Backpropagation of the networks NIN -> 32 -> 16 -> 3 with ReLU hidden
// layers: the tail MLP (NIN = 5, ReLU output, 771 parameters) and the DFAOIT
// comparison network (NIN = 11, sigmoid output, 963 parameters).
//
// Per sample i the forward pass is recomputed and the gradients at the three
// layers' pre-activations, g3 = dL/dz3, g2 = dL/dz2, g1 = dL/dz1, follow by
// the chain rule (CUDA cores: a few hundred multiply-adds per sample with
// K = NIN, 32 and 16).  With a_i = (x_i, h1_i, h2_i, 1), the inputs of the
// three layers and the bias input (NIN + 49 values), and g_i = (g1_i, g2_i,
// g3_i) (51 values), every parameter's gradient is one entry of the
// contraction over the batch
//     D = sum_i a_i g_i^T:  dW1[o][k] = D[x_k][g1_o], db1[o] = D[1][g1_o],
//     dW2[o][k] = D[h1_k][g2_o], db2[o] = D[1][g2_o], dW3, db3 alike,
// which runs on the tcgen05 tensor cores.  A CTA of 128 threads (one sample
// each) writes a_i into rows 0..63 and g_i into rows 64..127 of sample
// column i of an operand P (128 rows x 128 samples) in shared memory, and
// accumulates P P_g^T (M = 128, N = 64: P's g rows as the B operand, K = the
// samples) in tensor memory over the tiles it takes; rows 0..63 of the
// accumulator are D (rows 64..127 hold g g^T, unused).  The operands are bf16:
// each float32 value v is carried as three planes, hi = bf16(v), mid =
// bf16(v - hi), lo = bf16(v - hi - mid) (round to nearest, 24 significant bits
// together), and the six products hi.hi, hi.mid, mid.hi, hi.lo, lo.hi,
// mid.mid leave out terms below 2^-26 of each product, so D agrees with a
// float32 evaluation up to rounding order.  Each CTA writes its D entries as
// one row of partial sums; the rows are added in CTA order (deterministic).
template <int NIN>
struct Net {
  static constexpr int kW1 = 0, kB1 = 32 * NIN, kW2 = kB1 + 32, kB2 = kW2 + 512, kW3 = kB2 + 16,
                       kB3 = kW3 + 48, kParams = kB3 + 3;
  static constexpr int kXStride = NIN == 5 ? 2 : 4;     // float4 per input row ([P][8] or [P][16])
  static constexpr int kA = NIN + 49;                   // a_i: x, h1, h2, 1
  static_assert(kA <= 64, "a_i fits rows 0..63");
};
constexpr int kParamsMax = Net<11>::kParams;

// operand P in shared memory, K-major without swizzle: 8 x 8 bf16 core
// matrices (8 rows of 16 bytes); the 16 row groups of one 8-sample chunk
// lie 128 bytes apart, chunks kGradChunk apart (16 bytes more than the
// chunk, so that the 32 lanes of a warp, 32 consecutive samples, store one
// row into 16 different banks)
constexpr int kGradTile = 128;                       // samples per tile (one per thread)
constexpr uint32_t kGradChunk = 16 * 128 + 16;       // bytes between 8-sample chunks
constexpr uint32_t kGradPlane = 16 * kGradChunk;     // one bf16 plane of P (33,024 bytes)
constexpr uint32_t kGradSmem = 3 * kGradPlane + 4 * 1024;  // hi, mid, lo planes; the weights
constexpr int kGradCtasPerSm = 2;

// v = hi + mid + lo to 24 significant bits; row r of sample column col
__device__ __forceinline__ void put_split3(uint8_t *col, int r, float v) {
  const __nv_bfloat16 hi = __float2bfloat16_rn(v);
  const float r1 = v - __bfloat162float(hi);
  const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
  const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
  uint8_t *p = col + (r >> 3) * 128 + (r & 7) * 16;
  *reinterpret_cast<__nv_bfloat16 *>(p) = hi;
  *reinterpret_cast<__nv_bfloat16 *>(p + kGradPlane) = mid;
  *reinterpret_cast<__nv_bfloat16 *>(p + 2 * kGradPlane) = lo;
}

// forward pass of sample i (weights in s, Net<NIN> layout); zeros for i >= B
template <int NIN>
__device__ __forceinline__ void sample_forward(const float *s, const float4 *__restrict__ X, long long i,
                                               long long B, float (&x)[NIN], float (&h1)[32], float (&h2)[16],
                                               float (&z3)[3]) {
  using N = Net<NIN>;
  if (i >= B) {
#pragma unroll
    for (int k = 0; k < NIN; ++k) x[k] = 0.0f;
#pragma unroll
    for (int k = 0; k < 32; ++k) h1[k] = 0.0f;
#pragma unroll
    for (int k = 0; k < 16; ++k) h2[k] = 0.0f;
    z3[0] = z3[1] = z3[2] = 0.0f;
    return;
  }
  {
    float v[4 * N::kXStride];
#pragma unroll
    for (int q = 0; q < N::kXStride; ++q) {
      const float4 t = X[N::kXStride * i + q];
      v[4 * q] = t.x;
      v[4 * q + 1] = t.y;
      v[4 * q + 2] = t.z;
      v[4 * q + 3] = t.w;
    }
#pragma unroll
    for (int k = 0; k < NIN; ++k) x[k] = v[k];
  }
#pragma unroll
  for (int o = 0; o < 32; ++o) {
    float t = s[N::kB1 + o];
#pragma unroll
    for (int k = 0; k < NIN; ++k) t = fmaf(s[N::kW1 + NIN * o + k], x[k], t);
    h1[o] = fmaxf(t, 0.0f);
  }
#pragma unroll
  for (int o = 0; o < 16; ++o) {
    float t = s[N::kB2 + o];
#pragma unroll
    for (int k = 0; k < 32; ++k) t = fmaf(s[N::kW2 + 32 * o + k], h1[k], t);
    h2[o] = fmaxf(t, 0.0f);
  }
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    float t = s[N::kB3 + o];
#pragma unroll
    for (int k = 0; k < 16; ++k) t = fmaf(s[N::kW3 + 16 * o + k], h2[k], t);
    z3[o] = t;
  }
}

// sample column col of P: rows 0..NIN+48 a = (x, h1, h2, 1), rows 64..114
// g = (g1, g2, g3), the backward pass written row by row as it goes (the
// hidden activations survive only as their ReLU masks); zeros for i >= B
template <int NIN, bool SIGMOID>
__device__ __forceinline__ void sample_write(const float *s, uint8_t *col, const float (&x)[NIN],
                                             const float (&h1)[32], const float (&h2)[16], const float (&z3)[3],
                                             const float4 *__restrict__ dY, long long i, long long B) {
  using N = Net<NIN>;
  const bool valid = i < B;
  uint32_t m1 = 0u, m2 = 0u;
#pragma unroll
  for (int k = 0; k < NIN; ++k) put_split3(col, k, x[k]);
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    put_split3(col, NIN + k, h1[k]);
    m1 |= (h1[k] > 0.0f ? 1u : 0u) << k;
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    put_split3(col, NIN + 32 + k, h2[k]);
    m2 |= (h2[k] > 0.0f ? 1u : 0u) << k;
  }
  put_split3(col, NIN + 48, valid ? 1.0f : 0.0f);
  float g3[3] = {0.0f, 0.0f, 0.0f};
  if (valid) {
    const float4 d = dY[i];
    const float dd[3] = {d.x, d.y, d.z};
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      if (SIGMOID) {
        const float f = 1.0f / (1.0f + expf(-z3[o]));
        g3[o] = dd[o] * f * (1.0f - f);
      } else {
        g3[o] = z3[o] > 0.0f ? dd[o] : 0.0f;
      }
    }
  }
#pragma unroll
  for (int o = 0; o < 3; ++o) put_split3(col, 64 + 48 + o, g3[o]);
  float g2[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    float t = 0.0f;
#pragma unroll
    for (int o = 0; o < 3; ++o) t = fmaf(s[N::kW3 + 16 * o + k], g3[o], t);
    g2[k] = (m2 >> k) & 1u ? t : 0.0f;
    put_split3(col, 64 + 32 + k, g2[k]);
  }
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    float t = 0.0f;
#pragma unroll
    for (int o = 0; o < 16; ++o) t = fmaf(s[N::kW2 + 32 * o + k], g2[o], t);
    put_split3(col, 64 + k, (m1 >> k) & 1u ? t : 0.0f);
  }
}

template <int NIN, bool SIGMOID>
__global__ void __launch_bounds__(128, kGradCtasPerSm)
    k_mlp_grad_tc(const float *__restrict__ w1, const float *__restrict__ b1, const float *__restrict__ w2,
                  const float *__restrict__ b2, const float *__restrict__ w3, const float *__restrict__ b3,
                  const float4 *__restrict__ X, const float4 *__restrict__ dY, long long B, int n_tiles,
                  float *__restrict__ partial, unsigned long long wait_ns, int32_t *status) {
  using N = Net<NIN>;
  extern __shared__ __align__(128) uint8_t smem[];  // P: hi, mid, lo planes; then the weights
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  float *s = reinterpret_cast<float *>(smem + 3 * kGradPlane);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(64)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  for (int i = tid; i < 32 * NIN; i += 128) s[N::kW1 + i] = w1[i];
  for (int i = tid; i < 512; i += 128) s[N::kW2 + i] = w2[i];
  if (tid < 32) s[N::kB1 + tid] = b1[tid];
  if (tid < 16) s[N::kB2 + tid] = b2[tid];
  if (tid < 48) s[N::kW3 + tid] = w3[tid];
  if (tid < 3) s[N::kB3 + tid] = b3[tid];
  // the rows of P past a_i and g_i stay zero
  for (uint32_t i = tid; i < 3 * kGradPlane / 16; i += 128)
    reinterpret_cast<uint4 *>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    mbar_init(smem_u32(&bar), 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot, p0 = smem_u32(smem);
  uint8_t *col = smem + (tid >> 3) * kGradChunk + (tid & 7) * 2;  // this thread's sample column
  uint32_t ph = 0u;
  int done = 0;  // tiles accumulated (CTA-uniform)
  bool pending = false;
  for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const long long i = (long long)tile * kGradTile + tid;
    float x[NIN], h1[32], h2[16], z3[3];
    sample_forward<NIN>(s, X, i, B, x, h1, h2, z3);  // overlaps the previous tile's MMAs
    if (pending) {  // the previous tile's MMAs have read P
      mma_wait_cta(smem_u32(&bar), ph, &abort_flag, wait_ns);
      ph ^= 1u;
      pending = false;
    }
    if (abort_flag) break;  // uniform: read after the CTA barrier of the wait
    sample_write<NIN, SIGMOID>(s, col, x, h1, h2, z3, dY, i, B);
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (tid == 0) {
      fence_after();
      // (A plane, B plane): hi.hi, hi.mid, mid.hi, hi.lo, lo.hi, mid.mid
      constexpr uint32_t pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};
#pragma unroll 1
      for (int j = 0; j < kGradTile / 16; ++j) {  // K steps of 16 samples: two 8-sample chunks
        const uint32_t off = 2u * (uint32_t)j * kGradChunk;
#pragma unroll
        for (int q = 0; q < 6; ++q)
          mma_bf16(tmem, smem_desc(p0 + pa[q] * kGradPlane + off, kGradChunk, 128),
                   smem_desc(p0 + pb[q] * kGradPlane + off + 8 * 128, kGradChunk, 128), idesc_bf16(64),
                   (done > 0 || j > 0 || q > 0) ? 1u : 0u);
      }
      mma_commit(smem_u32(&bar));
    }
    pending = true;
    ++done;
  }
  if (pending) {
    mma_wait_cta(smem_u32(&bar), ph, &abort_flag, wait_ns);
    ph ^= 1u;
  }
  // rows 0..63 of the accumulator (tensor-memory lanes of warps 0 and 1):
  // thread m holds D[m][0..63], m the index of a_i, the column that of g_i
  if (warp < 2) {
    float d[64];
    if (done > 0) {
      float t[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), t);
#pragma unroll
      for (int n = 0; n < 32; ++n) d[n] = t[n];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + 32u, t);
#pragma unroll
      for (int n = 0; n < 32; ++n) d[32 + n] = t[n];
    } else {
#pragma unroll
      for (int n = 0; n < 64; ++n) d[n] = 0.0f;
    }
    if (abort_flag) {  // an incomplete sum: the gradient reads as NaN
#pragma unroll
      for (int n = 0; n < 64; ++n) d[n] = __int_as_float(0x7fc00000);
    }
    float *out = partial + (size_t)blockIdx.x * N::kParams;
    const int m = tid;
    if (m < NIN) {
#pragma unroll
      for (int o = 0; o < 32; ++o) out[N::kW1 + NIN * o + m] = d[o];
    } else if (m < NIN + 32) {
#pragma unroll
      for (int o = 0; o < 16; ++o) out[N::kW2 + 32 * o + (m - NIN)] = d[32 + o];
    } else if (m < NIN + 48) {
#pragma unroll
      for (int o = 0; o < 3; ++o) out[N::kW3 + 16 * o + (m - NIN - 32)] = d[48 + o];
    } else if (m == NIN + 48) {
#pragma unroll
      for (int o = 0; o < 32; ++o) out[N::kB1 + o] = d[o];
#pragma unroll
      for (int o = 0; o < 16; ++o) out[N::kB2 + o] = d[32 + o];
#pragma unroll
      for (int o = 0; o < 3; ++o) out[N::kB3 + o] = d[48 + o];
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64) : "memory");
  if (tid == 0 && abort_flag) raise_status(status, STAR_NT_ERR_TIMEOUT);
}

// grad[p] = the sum over rows c of partial[c][p] in a fixed order: warp w of
// a block adds rows w, w + 16, w + 32, ... for its block's 32 parameters
// (lane = parameter), then warp 0 adds the 16 warp sums in warp order
constexpr int kReduceWarps = 16;
__global__ void __launch_bounds__(32 * kReduceWarps) k_mlp_bwd_reduce(const float *__restrict__ partial, int rows,
                                                                     int n_params, float *__restrict__ grad) {
  __shared__ float s[kReduceWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int p = blockIdx.x * 32 + lane;
  float t = 0.0f;
  if (p < n_params) {
#pragma unroll 4
    for (int c = warp; c < rows; c += kReduceWarps) t += partial[(size_t)c * n_params + p];
  }
  s[warp][lane] = t;
  __syncthreads();
  if (warp == 0 && p < n_params) {
    float u = 0.0f;
#pragma unroll
    for (int w = 0; w < kReduceWarps; ++w) u += s[w][lane];
    grad[p] = u;
  }
}

// ---------------------------------------------------------------------------
// Adam (bias-corrected) on the float32 master weights, plus the weights
// rounded to bfloat16 (stored as float32) for the next forward pass.
__global__ void k_adam(float *__restrict__ prm, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, long long n, float lr, float b1, float b2, float eps,
                       float c1, float c2, float *__restrict__ rounded) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float p = prm[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  prm[i] = p;
  if (rounded) rounded[i] = __bfloat162float(__float2bfloat16_rn(p));
}

}  // namespace star

using namespace star;

extern "C" star_nt_status star_nt_abuffer(const star_nt_frags *frags, const uint32_t *rgba8, int32_t W,
                                          int32_t H, const float *bg, float *rgb, float *tail,
                                          void *stream) {
  if (!frags || !frags->count || !frags->offset || !rgba8 || !bg || W <= 0 || H <= 0 || (!rgb && !tail))
    return STAR_NT_ERR_ARG;
  if (((uintptr_t)rgb & 15u) || ((uintptr_t)tail & 15u)) return STAR_NT_ERR_ARG;
  const long long P = (long long)W * H;
  k_abuffer<<<(unsigned)((P + 127) / 128), 128, 0, (cudaStream_t)stream>>>(
      frags->count, frags->offset, frags->z, frags->prim, rgba8, P, bg[0], bg[1], bg[2],
      reinterpret_cast<float4 *>(rgb), reinterpret_cast<float4 *>(tail));
  return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
}

static int mse_blocks(int64_t B) {
  long long g = (B + 255) / 256;
  return (int)(g > 1024 ? 1024 : (g < 1 ? 1 : g));
}

// the backward's per-CTA partial sums (at most one row per tile), then the
// loss partials of star_nt_mse_grad in the last 4 KB
extern "C" size_t star_nt_train_ws_bytes(int64_t B) {
  if (B <= 0) return 0;
  const size_t tiles = (size_t)((B + kGradTile - 1) / kGradTile);
  return align_up(tiles * kParamsMax * 4, 256) + align_up(4 * 1024, 256);
}

static star_nt_status mse_grad(const float *f, const float *y, const float *w, int64_t B, float *dy,
                               float *loss, void *ws, size_t ws_bytes, void *stream) {
  if (B <= 0 || !f || !y || !dy || !loss || !ws || ws_bytes < star_nt_train_ws_bytes(B))
    return STAR_NT_ERR_ARG;
  if (((uintptr_t)f & 15u) || ((uintptr_t)y & 15u) || ((uintptr_t)dy & 15u) || ((uintptr_t)ws & 255u))
    return STAR_NT_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  float *partial = reinterpret_cast<float *>((char *)ws + star_nt_train_ws_bytes(B) - 4 * 1024);
  const int g = mse_blocks(B);
  k_mse<<<g, 256, 0, st>>>(reinterpret_cast<const float4 *>(f), reinterpret_cast<const float4 *>(y), w,
                           B, reinterpret_cast<float4 *>(dy), partial);
  k_sum_partials<<<1, 32, 0, st>>>(partial, g, loss);
  return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
}

extern "C" star_nt_status star_nt_mse_grad(const float *f, const float *y, int64_t B, float *dy,
                                           float *loss, void *ws, size_t ws_bytes, void *stream) {
  return mse_grad(f, y, nullptr, B, dy, loss, ws, ws_bytes, stream);
}

extern "C" star_nt_status star_nt_wmse_grad(const float *f, const float *y, const float *w, int64_t B,
                                            float *dy, float *loss, void *ws, size_t ws_bytes,
                                            void *stream) {
  if (!w) return STAR_NT_ERR_ARG;
  return mse_grad(f, y, w, B, dy, loss, ws, ws_bytes, stream);
}

template <int NIN, bool SIGMOID>
static star_nt_status mlp_backward(const star_nt_mlp *w, const float *x, const float *dy, int64_t B,
                                   float *grad, void *ws, size_t ws_bytes, int32_t *d_status, void *stream) {
  using N = Net<NIN>;
  if (!w || !w->w1 || !w->b1 || !w->w2 || !w->b2 || !w->w3 || !w->b3 || !x || !dy || !grad || B <= 0 ||
      !ws || ws_bytes < star_nt_train_ws_bytes(B))
    return STAR_NT_ERR_ARG;
  if (((uintptr_t)x & 15u) || ((uintptr_t)dy & 15u) || ((uintptr_t)ws & 255u)) return STAR_NT_ERR_ARG;
  const long long n_tiles = (B + kGradTile - 1) / kGradTile;
  if (n_tiles > (1ll << 30)) return STAR_NT_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_mlp_grad_tc<NIN, SIGMOID>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kGradSmem) != cudaSuccess)
      return STAR_NT_ERR_CUDA;
    attr = true;
  }
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)(n_tiles < (long long)sms * kGradCtasPerSm ? n_tiles : (long long)sms * kGradCtasPerSm);
  float *partial = reinterpret_cast<float *>(ws);
  k_mlp_grad_tc<NIN, SIGMOID><<<grid, 128, kGradSmem, st>>>(
      w->w1, w->b1, w->w2, w->b2, w->w3, w->b3, reinterpret_cast<const float4 *>(x),
      reinterpret_cast<const float4 *>(dy), B, (int)n_tiles, partial, wait_limit_ns(), d_status);
  k_mlp_bwd_reduce<<<(N::kParams + 31) / 32, 32 * kReduceWarps, 0, st>>>(partial, grid, N::kParams, grad);
  return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
}

extern "C" star_nt_status star_nt_mlp_backward(const star_nt_mlp *w, const float *x, const float *dy,
                                               int64_t B, float *grad, void *ws, size_t ws_bytes,
                                               int32_t *d_status, void *stream) {
  return mlp_backward<5, false>(w, x, dy, B, grad, ws, ws_bytes, d_status, stream);
}

extern "C" star_nt_status star_nt_dfaoit_backward(const star_nt_mlp *w, const float *x, const float *dy,
                                                  int64_t B, float *grad, void *ws, size_t ws_bytes,
                                                  int32_t *d_status, void *stream) {
  return mlp_backward<11, true>(w, x, dy, B, grad, ws, ws_bytes, d_status, stream);
}

// ---------------------------------------------------------------------------
// Minibatch rows: dst[i] = src[idx[i]] for rows of row_bytes bytes, in 16-byte
// chunks when rows and both bases allow it, else 4-byte words; one thread per
// chunk (grid-stride).  An index outside [0, n_src) is reported in the status
// word and its row is written as zeros.
template <class T>
__global__ void __launch_bounds__(256) k_gather_rows(const T *__restrict__ src, long long n_src,
                                                     const int64_t *__restrict__ idx, long long n, int per_row,
                                                     T *__restrict__ dst, int32_t *status) {
  const long long total = n * per_row;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const long long i = k / per_row;
    const int c = (int)(k - i * per_row);
    const long long r = __ldg(idx + i);
    T v;
    if (r >= 0 && r < n_src) {
      v = __ldg(src + r * per_row + c);
    } else {
      v = T();
      if (c == 0) raise_status(status, STAR_NT_ERR_ARG);
    }
    dst[k] = v;
  }
}

extern "C" star_nt_status star_nt_gather_rows(const void *src, int64_t n_src, int32_t row_bytes,
                                              const int64_t *idx, int64_t n, void *dst, int32_t *d_status,
                                              void *stream) {
  if (!src || !idx || !dst || n_src <= 0 || n < 0 || row_bytes <= 0 || (row_bytes & 3) ||
      row_bytes > (1 << 20) || ((uintptr_t)src & 3u) || ((uintptr_t)dst & 3u) || ((uintptr_t)idx & 7u))
    return STAR_NT_ERR_ARG;
  if (n == 0) return STAR_NT_OK;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaStream_t st = (cudaStream_t)stream;
  const bool wide = (row_bytes & 15) == 0 && !((uintptr_t)src & 15u) && !((uintptr_t)dst & 15u);
  const int per_row = wide ? row_bytes / 16 : row_bytes / 4;
  const long long total = (long long)n * per_row;
  long long grid = (total + 255) / 256;
  if (grid > (long long)sms * 16) grid = (long long)sms * 16;
  if (wide)
    k_gather_rows<uint4><<<(unsigned)grid, 256, 0, st>>>(static_cast<const uint4 *>(src), n_src, idx, n, per_row,
                                                          static_cast<uint4 *>(dst), d_status);
  else
    k_gather_rows<uint32_t><<<(unsigned)grid, 256, 0, st>>>(static_cast<const uint32_t *>(src), n_src, idx, n,
                                                             per_row, static_cast<uint32_t *>(dst), d_status);
  return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
}

extern "C" star_nt_status star_nt_adam(float *params, const float *grad, float *m, float *v, int64_t n,
                                       int64_t step, float lr, float beta1, float beta2, float eps,
                                       float *bf16_rounded, void *stream) {
  if (!params || !grad || !m || !v || n <= 0 || step < 1) return STAR_NT_ERR_ARG;
  const float c1 = (float)(1.0 - pow((double)beta1, (double)step));
  const float c2 = (float)(1.0 - pow((double)beta2, (double)step));
  k_adam<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      params, grad, m, v, n, lr, beta1, beta2, eps, c1, c2, bf16_rounded);
  return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
}

namespace star {
// Loads this file's kernels onto the current device (see star_nt_preload).
cudaError_t preload_train() {
  cudaFuncAttributes a;
  cudaError_t e = cudaSuccess, r;
  if ((r = cudaFuncGetAttributes(&a, k_abuffer)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_mse)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_sum_partials)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_mlp_grad_tc<5, false>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_mlp_grad_tc<11, true>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_mlp_bwd_reduce)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_adam)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_gather_rows<uint4>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_gather_rows<uint32_t>)) != cudaSuccess) e = r;
  return e;
}
}  // namespace star
