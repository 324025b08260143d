// dfaoit.cu -- the DFAOIT comparison network of Sec. 3.3: the original
// method's network predicts the whole transparency colour C_t from the
// features the paper lists for it (the exact blend of the two front
// fragments, the tail's mean colour and opacity, its accumulated
// premultiplied colour, the fragment count: eleven inputs), with ReLU hidden
// layers of 32 and 16 units and a sigmoid output; the frame is
// C = C_t + C_b prod(1 - a_i).  STAR-NT's five-input tail network replaces it
// (the "10 -> 5 features" comparison of Table 2's inference columns).  The
// float32 forward runs on the CUDA cores; the bf16 forward is the tensor-core
// kernel of mlp_tc.cu instantiated for eleven inputs.
#include <math.h>

#include "common.cuh"

namespace star {

// weights in shared memory: w1[32][11], b1[32], w2[16][32], b2[16], w3[3][16], b3[3]
constexpr int kDW1 = 0, kDB1 = 352, kDW2 = 384, kDB2 = 896, kDW3 = 912, kDB3 = 960, kDParams = 963;

// One pixel per thread; X rows of 16 floats (x0..x10, flag, 0..), F rows of 4.
__global__ void __launch_bounds__(256) k_dfaoit_f32(const float *__restrict__ w1, const float *__restrict__ b1,
                                                    const float *__restrict__ w2, const float *__restrict__ b2,
                                                    const float *__restrict__ w3, const float *__restrict__ b3,
                                                    const float4 *__restrict__ X, float4 *__restrict__ F,
                                                    long long P) {
  __shared__ float s[kDParams + 1];
  for (int i = threadIdx.x; i < 352; i += 256) s[kDW1 + i] = w1[i];
  for (int i = threadIdx.x; i < 512; i += 256) s[kDW2 + i] = w2[i];
  if (threadIdx.x < 32) s[kDB1 + threadIdx.x] = b1[threadIdx.x];
  if (threadIdx.x < 16) s[kDB2 + threadIdx.x] = b2[threadIdx.x];
  if (threadIdx.x < 48) s[kDW3 + threadIdx.x] = w3[threadIdx.x];
  if (threadIdx.x < 3) s[kDB3 + threadIdx.x] = b3[threadIdx.x];
  __syncthreads();
  for (long long p = (long long)blockIdx.x * 256 + threadIdx.x; p < P; p += (long long)gridDim.x * 256) {
    float x[16];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 v = X[4 * p + q];
      x[4 * q] = v.x;
      x[4 * q + 1] = v.y;
      x[4 * q + 2] = v.z;
      x[4 * q + 3] = v.w;
    }
    if (x[11] == 0.0f) {
      F[p] = make_float4(0.f, 0.f, 0.f, 0.f);
      continue;
    }
    float h1[32], h2[16];
#pragma unroll
    for (int o = 0; o < 32; ++o) {
      float a = s[kDB1 + o];
#pragma unroll
      for (int k = 0; k < 11; ++k) a = fmaf(s[kDW1 + 11 * o + k], x[k], a);
      h1[o] = fmaxf(a, 0.0f);
    }
#pragma unroll
    for (int o = 0; o < 16; ++o) {
      float a = s[kDB2 + o];
#pragma unroll
      for (int k = 0; k < 32; ++k) a = fmaf(s[kDW2 + 32 * o + k], h1[k], a);
      h2[o] = fmaxf(a, 0.0f);
    }
    float f[3];
#pragma unroll
    for (int o = 0; o < 3; ++o) {
      float a = s[kDB3 + o];
#pragma unroll
      for (int k = 0; k < 16; ++k) a = fmaf(s[kDW3 + 16 * o + k], h2[k], a);
      f[o] = 1.0f / (1.0f + expf(-a));
    }
    F[p] = make_float4(f[0], f[1], f[2], 0.0f);
  }
}

}  // namespace star

using namespace star;

cudaError_t star_launch_dfaoit_bf16(const star_nt_mlp *w, const void *x, float *f, int64_t P,
                                    int32_t *d_status, cudaStream_t st);

extern "C" star_nt_status star_nt_infer_dfaoit(const star_nt_mlp *w, int32_t x_dtype, const void *x, float *f,
                                               int64_t P, int32_t *d_status, void *stream) {
  if (!w || !w->w1 || !w->b1 || !w->w2 || !w->b2 || !w->w3 || !w->b3 || P < 0) return STAR_NT_ERR_ARG;
  if (P > 0 && (!x || !f)) return STAR_NT_ERR_ARG;
  if (((uintptr_t)x & 15u) || ((uintptr_t)f & 15u)) return STAR_NT_ERR_ARG;
  if (P == 0) return STAR_NT_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (x_dtype == STAR_NT_F32) {
    long long g = (P + 255) / 256;
    if (g > 148 * 16) g = 148 * 16;
    k_dfaoit_f32<<<(unsigned)g, 256, 0, st>>>(w->w1, w->b1, w->w2, w->b2, w->w3, w->b3,
                                              reinterpret_cast<const float4 *>(x), reinterpret_cast<float4 *>(f),
                                              P);
    return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
  }
  if (x_dtype == STAR_NT_BF16) {
    if ((uintptr_t)x & 255u) return STAR_NT_ERR_ARG;
    return star_launch_dfaoit_bf16(w, x, f, P, d_status, st) == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
  }
  return STAR_NT_ERR_ARG;
}

namespace star {
// Loads this file's kernels onto the current device (see star_nt_preload).
cudaError_t preload_dfaoit() {
  cudaFuncAttributes a;
  return cudaFuncGetAttributes(&a, k_dfaoit_f32);
}
}  // namespace star
