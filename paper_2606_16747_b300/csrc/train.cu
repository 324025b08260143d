// train.cu -- the learned part: exact A-buffer resolve (the ground truth of
// Sec. 4 and the tail-colour target of Sec. 3.3), and training of the tail
// MLP with MSE and Adam (Sec. 3.3): loss gradient, backpropagation to the 771
// parameters, Adam update with a bf16 copy of the updated weights.
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"

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
// comparison network (NIN = 11, sigmoid output, 963 parameters).  Stage 1:
// per sample, recompute the forward pass and the per-layer gradients
// g3 = dL/dz3, g2 = dL/dz2, g1 = dL/dz1 (z: pre-activation), stored with the
// activations: row = [h1(32) h2(16) g1(32) g2(16) g3(3) x(NIN)].  Stage 2: per
// chunk of samples, every parameter's partial sum.  Stage 3: the partial sums
// added in chunk order (deterministic).
template <int NIN>
struct Net {
  static constexpr int kRow = (99 + NIN + 3) / 4 * 4;  // row length, padded to 4 floats
  static constexpr int kW1 = 0, kB1 = 32 * NIN, kW2 = kB1 + 32, kB2 = kW2 + 512, kW3 = kB2 + 16,
                       kB3 = kW3 + 48, kParams = kB3 + 3;
  static constexpr int kXStride = NIN == 5 ? 2 : 4;     // float4 per input row ([P][8] or [P][16])
};
constexpr int kChunkS = 1024;
constexpr int kRowMax = Net<11>::kRow;
constexpr int kParamsMax = Net<11>::kParams;

template <int NIN, bool SIGMOID>
__global__ void __launch_bounds__(256) k_mlp_bwd_rows(const float *__restrict__ w1, const float *__restrict__ b1,
                                                      const float *__restrict__ w2, const float *__restrict__ b2,
                                                      const float *__restrict__ w3, const float *__restrict__ b3,
                                                      const float4 *__restrict__ X, const float4 *__restrict__ dY,
                                                      long long B, float *__restrict__ rows) {
  using N = Net<NIN>;
  __shared__ float s[N::kParams + 1];
  for (int i = threadIdx.x; i < 32 * NIN; i += 256) s[N::kW1 + i] = w1[i];
  for (int i = threadIdx.x; i < 512; i += 256) s[N::kW2 + i] = w2[i];
  if (threadIdx.x < 32) s[N::kB1 + threadIdx.x] = b1[threadIdx.x];
  if (threadIdx.x < 16) s[N::kB2 + threadIdx.x] = b2[threadIdx.x];
  if (threadIdx.x < 48) s[N::kW3 + threadIdx.x] = w3[threadIdx.x];
  if (threadIdx.x < 3) s[N::kB3 + threadIdx.x] = b3[threadIdx.x];
  __syncthreads();
  const long long i = (long long)blockIdx.x * 256 + threadIdx.x;
  if (i >= B) return;
  float x[NIN];
  {
    float v[4 * N::kXStride];
#pragma unroll
    for (int q = 0; q < N::kXStride; ++q) {
      const float4 a = X[N::kXStride * i + q];
      v[4 * q] = a.x;
      v[4 * q + 1] = a.y;
      v[4 * q + 2] = a.z;
      v[4 * q + 3] = a.w;
    }
#pragma unroll
    for (int k = 0; k < NIN; ++k) x[k] = v[k];
  }
  float h1[32], h2[16], z3[3];
#pragma unroll
  for (int o = 0; o < 32; ++o) {
    float a = s[N::kB1 + o];
#pragma unroll
    for (int k = 0; k < NIN; ++k) a = fmaf(s[N::kW1 + NIN * o + k], x[k], a);
    h1[o] = fmaxf(a, 0.0f);
  }
#pragma unroll
  for (int o = 0; o < 16; ++o) {
    float a = s[N::kB2 + o];
#pragma unroll
    for (int k = 0; k < 32; ++k) a = fmaf(s[N::kW2 + 32 * o + k], h1[k], a);
    h2[o] = fmaxf(a, 0.0f);
  }
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    float a = s[N::kB3 + o];
#pragma unroll
    for (int k = 0; k < 16; ++k) a = fmaf(s[N::kW3 + 16 * o + k], h2[k], a);
    z3[o] = a;
  }
  const float4 d = dY[i];
  const float dd[3] = {d.x, d.y, d.z};
  float g3[3], g2[16], g1[32];
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    if (SIGMOID) {
      const float f = 1.0f / (1.0f + expf(-z3[o]));
      g3[o] = dd[o] * f * (1.0f - f);
    } else {
      g3[o] = z3[o] > 0.0f ? dd[o] : 0.0f;
    }
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    float a = 0.0f;
#pragma unroll
    for (int o = 0; o < 3; ++o) a = fmaf(s[N::kW3 + 16 * o + k], g3[o], a);
    g2[k] = h2[k] > 0.0f ? a : 0.0f;
  }
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    float a = 0.0f;
#pragma unroll
    for (int o = 0; o < 16; ++o) a = fmaf(s[N::kW2 + 32 * o + k], g2[o], a);
    g1[k] = h1[k] > 0.0f ? a : 0.0f;
  }
  float *row = rows + (size_t)i * N::kRow;
#pragma unroll
  for (int k = 0; k < 32; ++k) row[k] = h1[k];
#pragma unroll
  for (int k = 0; k < 16; ++k) row[32 + k] = h2[k];
#pragma unroll
  for (int k = 0; k < 32; ++k) row[48 + k] = g1[k];
#pragma unroll
  for (int k = 0; k < 16; ++k) row[80 + k] = g2[k];
#pragma unroll
  for (int k = 0; k < 3; ++k) row[96 + k] = g3[k];
#pragma unroll
  for (int k = 0; k < NIN; ++k) row[99 + k] = x[k];
}

// parameter p (in w1, b1, w2, b2, w3, b3 order) as a product of two row
// entries (second index < 0: bias, factor 1)
template <int NIN>
__device__ __forceinline__ void param_factors(int p, int &a, int &b) {
  using N = Net<NIN>;
  if (p < N::kB1) { a = 48 + p / NIN; b = 99 + p % NIN; return; }            // dW1[o][k] = g1[o] x[k]
  if (p < N::kW2) { a = 48 + (p - N::kB1); b = -1; return; }                 // db1
  if (p < N::kB2) { const int q = p - N::kW2; a = 80 + q / 32; b = q % 32; return; }  // dW2 = g2 h1
  if (p < N::kW3) { a = 80 + (p - N::kB2); b = -1; return; }                 // db2
  if (p < N::kB3) { const int q = p - N::kW3; a = 96 + q / 16; b = 32 + q % 16; return; }  // dW3 = g3 h2
  a = 96 + (p - N::kB3); b = -1;                                             // db3
}

template <int NIN>
__global__ void __launch_bounds__(256) k_mlp_bwd_partial(const float *__restrict__ rows, long long B,
                                                         float *__restrict__ partial) {
  using N = Net<NIN>;
  __shared__ float s_rows[32 * N::kRow];
  const long long s0 = (long long)blockIdx.x * kChunkS;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  int fa[4], fb[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int p = threadIdx.x + 256 * j;
    if (p < N::kParams) param_factors<NIN>(p, fa[j], fb[j]);
    else { fa[j] = 0; fb[j] = -2; }
  }
  for (long long c = s0; c < s0 + kChunkS && c < B; c += 32) {
    const int m = (int)min((long long)32, B - c);
    __syncthreads();
    for (int k = threadIdx.x; k < m * N::kRow; k += 256) s_rows[k] = rows[(size_t)c * N::kRow + k];
    __syncthreads();
    for (int r = 0; r < m; ++r) {
      const float *row = s_rows + r * N::kRow;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (fb[j] == -2) continue;
        acc[j] = fmaf(row[fa[j]], fb[j] >= 0 ? row[fb[j]] : 1.0f, acc[j]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int p = threadIdx.x + 256 * j;
    if (p < N::kParams) partial[(size_t)blockIdx.x * N::kParams + p] = acc[j];
  }
}

__global__ void k_mlp_bwd_reduce(const float *__restrict__ partial, int chunks, int n_params,
                                 float *__restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_params) return;
  float t = 0.0f;
  for (int c = 0; c < chunks; ++c) t += partial[(size_t)c * n_params + p];
  grad[p] = t;
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

extern "C" size_t star_nt_train_ws_bytes(int64_t B) {
  if (B <= 0) return 0;
  const size_t rows = (size_t)B * kRowMax * 4;
  const size_t chunks = (size_t)((B + kChunkS - 1) / kChunkS);
  return align_up(rows, 256) + align_up(chunks * kParamsMax * 4, 256) + align_up(4 * 1024, 256);
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
                                   float *grad, void *ws, size_t ws_bytes, void *stream) {
  using N = Net<NIN>;
  if (!w || !w->w1 || !w->b1 || !w->w2 || !w->b2 || !w->w3 || !w->b3 || !x || !dy || !grad || B <= 0 ||
      !ws || ws_bytes < star_nt_train_ws_bytes(B))
    return STAR_NT_ERR_ARG;
  if (((uintptr_t)x & 15u) || ((uintptr_t)dy & 15u) || ((uintptr_t)ws & 255u)) return STAR_NT_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  float *rows = reinterpret_cast<float *>(ws);
  float *partial = reinterpret_cast<float *>((char *)ws + align_up((size_t)B * kRowMax * 4, 256));
  const int chunks = (int)((B + kChunkS - 1) / kChunkS);
  k_mlp_bwd_rows<NIN, SIGMOID><<<(unsigned)((B + 255) / 256), 256, 0, st>>>(
      w->w1, w->b1, w->w2, w->b2, w->w3, w->b3, reinterpret_cast<const float4 *>(x),
      reinterpret_cast<const float4 *>(dy), B, rows);
  k_mlp_bwd_partial<NIN><<<chunks, 256, 0, st>>>(rows, B, partial);
  k_mlp_bwd_reduce<<<(N::kParams + 255) / 256, 256, 0, st>>>(partial, chunks, N::kParams, grad);
  return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
}

extern "C" star_nt_status star_nt_mlp_backward(const star_nt_mlp *w, const float *x, const float *dy,
                                               int64_t B, float *grad, void *ws, size_t ws_bytes,
                                               void *stream) {
  return mlp_backward<5, false>(w, x, dy, B, grad, ws, ws_bytes, stream);
}

extern "C" star_nt_status star_nt_dfaoit_backward(const star_nt_mlp *w, const float *x, const float *dy,
                                                  int64_t B, float *grad, void *ws, size_t ws_bytes,
                                                  void *stream) {
  return mlp_backward<11, true>(w, x, dy, B, grad, ws, ws_bytes, stream);
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
  if ((r = cudaFuncGetAttributes(&a, k_mlp_bwd_rows<5, false>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_mlp_bwd_partial<5>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_mlp_bwd_rows<11, true>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_mlp_bwd_partial<11>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_mlp_bwd_reduce)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_adam)) != cudaSuccess) e = r;
  return e;
}
}  // namespace star
