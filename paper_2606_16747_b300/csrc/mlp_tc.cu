// mlp_tc.cu -- the tail-colour MLP 5 -> 32 -> 16 -> 3 (Sec. 3.3) on the
// tcgen05 tensor cores: bf16 operands, fp32 accumulation in tensor memory.
//
// One CTA of 128 threads runs a persistent loop over 128-pixel tiles.  Per
// tile, three chained MMAs (M = 128 pixels); each bias rides in its MMA as two
// weight columns against a constant operand block whose rows are (1, 1, 0, ...):
//   D1[128x32] = [X | 1]    [W1 | b1]^T   (K = 16: 5 inputs, then the ones block)
//   D2[128x16] = [H1 | 1 0] [W2 | b2]^T   (K = 48: three K = 16 steps)
//   D3[128x16] = [H2 | 1 0] [W3 | b3]^T   (K = 32; N padded 3 -> 16)
// X tiles arrive by TMA (double buffered, one tile ahead); after each MMA
// the four warps read their 32 accumulator rows from tensor memory, apply
// ReLU while packing to bf16, and write the next layer's operand to shared
// memory.  Operands use the no-swizzle K-major layout: 8-row x 16-byte core
// matrices, LBO = distance between K-adjacent core matrices, SBO = between
// 8-row groups.  Every mbarrier wait is bounded (star_nt_set_wait_limit); on
// expiry the kernel sets STAR_NT_ERR_TIMEOUT, stops, lets the MMA or copy in
// flight land (a second, fixed bound), frees its tensor memory and returns.
// The same kernel, templated on the input count and the output activation,
// runs the DFAOIT comparison network (11 inputs, sigmoid output): its X rows
// are 16 bf16 wide, loaded as two TMA boxes of one core column each, and
// layer 1 takes two K = 16 MMAs (the inputs, then the bias block).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cuda_bf16.h>

#include "common.cuh"
#include "tc_primitives.cuh"

namespace star {

constexpr int kMlpThreads = 128;
constexpr int kRows = 128;
constexpr uint32_t kTmemCols = 64;          // D1: 0..31, D2: 32..47, D3: 48..63
constexpr int kMlpCtasPerSm = 8;            // 8 x 64 columns = all of tensor memory

// Shared memory map (bytes from a 1024-aligned base) of the network with NIN
// inputs: NIN = 5 (the tail MLP, X rows of 8 bf16: the inputs and the tail
// flag) or NIN = 11 (the DFAOIT comparison network, X rows of 16 bf16, the
// flag at element 11).  An X tile is XB bytes: one core column (K 0..7) for
// NIN = 5, two (K 0..7, K 8..15) for NIN = 11.
template <int NIN>
struct MlpMap {
  static constexpr uint32_t XB = NIN == 5 ? 2048 : 4096;
  static constexpr uint32_t SX = 0;                 // 2 X tiles (TMA targets)
  static constexpr uint32_t SC = 2 * XB;            // ones block: rows (1, 1, 0, ...)
  static constexpr uint32_t SZ = SC + 2048;         // zero block
  static constexpr uint32_t SH1 = SZ + 2048;        // 4 core columns x 2048
  static constexpr uint32_t SH2 = SH1 + 8192;       // 2 core columns x 2048
  // W1: N = 32; K = 16 (inputs 0..7, bias in K 8, 9) for NIN = 5, K = 32
  // (inputs 0..15, bias in K 16, 17) for NIN = 11: core columns of 512
  static constexpr uint32_t KB1 = NIN == 5 ? 8 : 16;  // K of b1's hi part
  static constexpr uint32_t SW1 = SH2 + 4096;
  static constexpr uint32_t SW2 = SW1 + (NIN == 5 ? 1024 : 2048);  // N=16, K=48 (bias in K 32, 33): 6 x 256
  static constexpr uint32_t SW3 = SW2 + 1536;       // N=16, K=32 (bias in K 16, 17): 4 x 256
  static constexpr uint32_t SBar = SW3 + 1024;      // tma[2], mma, tmem slot, abort flag
  static constexpr uint32_t Used = SBar + 32;
  // requested dynamic shared memory: caps residency at 8 CTAs per SM (NIN = 5)
  // or 7 (NIN = 11), so that 64 tensor-memory columns per CTA always suffice
  static constexpr uint32_t Bytes = NIN == 5 ? 26 * 1024 : 30 * 1024;
  // byte offset of the flag within an X tile row's core column
  static constexpr uint32_t FlagCol = NIN == 5 ? 0 : 2048;
  static constexpr uint32_t FlagByte = NIN == 5 ? 10 : 6;
};
static_assert(MlpMap<5>::SW1 == 20480 && MlpMap<5>::SBar == 24064, "shared memory map of the tail MLP");

// NIN inputs; SIGMOID: sigmoid output (the DFAOIT network), else ReLU.
template <int NIN, bool SIGMOID>
__global__ void __launch_bounds__(kMlpThreads, kMlpCtasPerSm)
    k_mlp_bf16(const __grid_constant__ CUtensorMap xmap, const float *__restrict__ w1,
               const float *__restrict__ b1, const float *__restrict__ w2,
               const float *__restrict__ b2, const float *__restrict__ w3,
               const float *__restrict__ b3, float4 *__restrict__ F, long long P,
               int32_t *status, unsigned long long wait_ns) {
  using M = MlpMap<NIN>;
  constexpr uint32_t kSX = M::SX, kSC = M::SC, kSZ = M::SZ, kSH1 = M::SH1, kSH2 = M::SH2, kSW1 = M::SW1,
                     kSW2 = M::SW2, kSW3 = M::SW3, kSBar = M::SBar, kXB = M::XB;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                            ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t sbase = smem_u32(sm);
  const uint32_t bar_tma0 = sbase + kSBar, bar_tma1 = sbase + kSBar + 8, bar_mma = sbase + kSBar + 16;
  uint32_t *s_tmem = reinterpret_cast<uint32_t *>(sm + kSBar + 24);
  volatile int *s_abort = reinterpret_cast<volatile int *>(sm + kSBar + 28);

  // weights and bias columns (bf16, zero padded), the ones and zero blocks
  for (int i = tid; i < (int)(kSBar - kSC) / 4; i += kMlpThreads)
    reinterpret_cast<uint32_t *>(sm + kSC)[i] = 0u;
  __syncthreads();
  put_ones_block(sm + kSC, tid, kMlpThreads);
  for (int i = tid; i < 32 * NIN; i += kMlpThreads) put_w(sm + kSW1, i / NIN, i % NIN, 512, w1[i]);
  for (int i = tid; i < 16 * 32; i += kMlpThreads) put_w(sm + kSW2, i / 32, i % 32, 256, w2[i]);
  for (int i = tid; i < 3 * 16; i += kMlpThreads) put_w(sm + kSW3, i / 16, i % 16, 256, w3[i]);
  if (tid < 32) put_bias(sm + kSW1, tid, M::KB1, 512, b1[tid]);
  if (tid < 16) put_bias(sm + kSW2, tid, 32, 256, b2[tid]);
  if (tid < 3) put_bias(sm + kSW3, tid, 16, 256, b3[tid]);
  if (tid == 0) {
    mbar_init(bar_tma0, 1);
    mbar_init(bar_tma1, 1);
    mbar_init(bar_mma, 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(s_tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *s_tmem;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const int row = warp * 32 + (tid & 31);

  const long long ntiles = (P + kRows - 1) / kRows;
  long long tile = blockIdx.x;
  uint32_t ph_tma[2] = {0u, 0u}, ph_mma = 0u;
  int buf = 0;
  bool tma_pending = false;          // a TMA load in flight (thread 0)
  uint32_t pend_bar = 0, pend_ph = 0;
  const uint64_t dW1 = smem_desc(sbase + kSW1, 512, 128);
  const uint64_t dW1b = smem_desc(sbase + kSW1 + 1024, 512, 128);  // NIN = 11: K 16..31 (bias)
  const uint64_t dW2[3] = {smem_desc(sbase + kSW2, 256, 128), smem_desc(sbase + kSW2 + 512, 256, 128),
                           smem_desc(sbase + kSW2 + 1024, 256, 128)};
  const uint64_t dW3[2] = {smem_desc(sbase + kSW3, 256, 128), smem_desc(sbase + kSW3 + 512, 256, 128)};
  const uint64_t dH1a = smem_desc(sbase + kSH1, 2048, 128), dH1b = smem_desc(sbase + kSH1 + 4096, 2048, 128);
  const uint64_t dH2 = smem_desc(sbase + kSH2, 2048, 128);
  const uint64_t dOnes = smem_desc(sbase + kSC, kSZ - kSC, 128);  // K block: ones, then zeros

  if (tid == 0 && tile < ntiles) {
    mbar_expect_tx(bar_tma0, kXB);
    tma_load_2d(sbase + kSX, &xmap, 0, (int)(tile * kRows), bar_tma0);
    if (NIN == 11) tma_load_2d(sbase + kSX + 2048, &xmap, 8, (int)(tile * kRows), bar_tma0);
    tma_pending = true;
    pend_bar = bar_tma0;
    pend_ph = 0u;
  }
  while (tile < ntiles) {
    const long long next = tile + gridDim.x;
    const uint32_t xs = sbase + kSX + buf * kXB;
    // ---- layer 1
    if (tid == 0) {
      if (!mbar_wait(buf ? bar_tma1 : bar_tma0, ph_tma[buf], wait_ns)) {
        *s_abort = 1;
      } else {
        tma_pending = false;
        ph_tma[buf] ^= 1u;
        fence_after();
        if (NIN == 5) {
          // [X | ones] (K = 16) against [W1 | b1]
          mma_bf16(tmem + 0, smem_desc(xs, sbase + kSC - xs, 128), dW1, idesc_bf16(32), 0u);
        } else {
          // X (K = 16, two core columns) against W1, then [ones | 0] against b1
          mma_bf16(tmem + 0, smem_desc(xs, 2048, 128), dW1, idesc_bf16(32), 0u);
          mma_bf16(tmem + 0, smem_desc(sbase + kSC, kSZ - kSC, 128), dW1b, idesc_bf16(32), 1u);
        }
        mma_commit(bar_mma);
        if (next < ntiles) {
          const uint32_t nb = buf ? bar_tma0 : bar_tma1;
          const uint32_t nx = sbase + kSX + (buf ^ 1) * kXB;
          mbar_expect_tx(nb, kXB);
          tma_load_2d(nx, &xmap, 0, (int)(next * kRows), nb);
          if (NIN == 11) tma_load_2d(nx + 2048, &xmap, 8, (int)(next * kRows), nb);
          tma_pending = true;
          pend_bar = nb;
          pend_ph = ph_tma[buf ^ 1];
        }
      }
    }
    __syncthreads();
    if (*s_abort) break;
    if (!mbar_wait(bar_mma, ph_mma, wait_ns)) {  // stop, but let the MMA finish first
      *s_abort = 1;
      mbar_wait(bar_mma, ph_mma, kDrainNs);
    }
    ph_mma ^= 1u;
    fence_after();
    const float flag = __bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(
        sm + kSX + buf * kXB + M::FlagCol + row * 16 + M::FlagByte));
    {
      float d[32];
      tmem_ld32(tmem + lane_base + 0, d);
      uint32_t pk[16];
#pragma unroll
      for (int j = 0; j < 16; ++j)
        pk[j] = pack_relu_bf16(d[2 * j], d[2 * j + 1]);
#pragma unroll
      for (int kc = 0; kc < 4; ++kc)
        *reinterpret_cast<uint4 *>(sm + kSH1 + kc * 2048 + row * 16) =
            make_uint4(pk[4 * kc], pk[4 * kc + 1], pk[4 * kc + 2], pk[4 * kc + 3]);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (*s_abort) break;
    // ---- layer 2
    if (tid == 0) {
      fence_after();
      mma_bf16(tmem + 32, dH1a, dW2[0], idesc_bf16(16), 0u);
      mma_bf16(tmem + 32, dH1b, dW2[1], idesc_bf16(16), 1u);
      mma_bf16(tmem + 32, dOnes, dW2[2], idesc_bf16(16), 1u);
      mma_commit(bar_mma);
    }
    if (!mbar_wait(bar_mma, ph_mma, wait_ns)) {  // stop, but let the MMA finish first
      *s_abort = 1;
      mbar_wait(bar_mma, ph_mma, kDrainNs);
    }
    ph_mma ^= 1u;
    fence_after();
    {
      float d[16];
      tmem_ld16(tmem + lane_base + 32, d);
      uint32_t pk[8];
#pragma unroll
      for (int j = 0; j < 8; ++j)
        pk[j] = pack_relu_bf16(d[2 * j], d[2 * j + 1]);
#pragma unroll
      for (int kc = 0; kc < 2; ++kc)
        *reinterpret_cast<uint4 *>(sm + kSH2 + kc * 2048 + row * 16) =
            make_uint4(pk[4 * kc], pk[4 * kc + 1], pk[4 * kc + 2], pk[4 * kc + 3]);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (*s_abort) break;
    // ---- layer 3
    if (tid == 0) {
      fence_after();
      mma_bf16(tmem + 48, dH2, dW3[0], idesc_bf16(16), 0u);
      mma_bf16(tmem + 48, dOnes, dW3[1], idesc_bf16(16), 1u);
      mma_commit(bar_mma);
    }
    if (!mbar_wait(bar_mma, ph_mma, wait_ns)) {  // stop, but let the MMA finish first
      *s_abort = 1;
      mbar_wait(bar_mma, ph_mma, kDrainNs);
    }
    ph_mma ^= 1u;
    fence_after();
    {
      float d[16];
      tmem_ld16(tmem + lane_base + 48, d);
      const long long p = tile * kRows + row;
      if (p < P) {
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (flag != 0.0f) {
          if (SIGMOID) {
            o.x = 1.0f / (1.0f + __expf(-d[0]));
            o.y = 1.0f / (1.0f + __expf(-d[1]));
            o.z = 1.0f / (1.0f + __expf(-d[2]));
          } else {
            o.x = fmaxf(d[0], 0.0f);
            o.y = fmaxf(d[1], 0.0f);
            o.z = fmaxf(d[2], 0.0f);
          }
        }
        F[p] = o;
      }
    }
    fence_before();
    __syncthreads();
    if (*s_abort) break;
    buf ^= 1;
    tile = next;
  }
  if (*s_abort && tid == 0) {
    raise_status(status, STAR_NT_ERR_TIMEOUT);
    if (tma_pending) mbar_wait(pend_bar, pend_ph, kDrainNs);  // let the copy land before exiting
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                 : "memory");
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace star

using namespace star;

// Launch of k_mlp_bf16<NIN, SIGMOID> over P rows of X (bf16, rows of 8
// elements for NIN = 5, 16 for NIN = 11; 256-byte aligned).
template <int NIN, bool SIGMOID>
static cudaError_t launch_mlp_bf16(const star_nt_mlp *w, const void *x, float *f, int64_t P,
                                   int32_t *d_status, cudaStream_t st) {
  using M = MlpMap<NIN>;
  static_assert(M::Used + 1024 <= M::Bytes, "shared memory map");
  if (P <= 0) return cudaSuccess;
  if (P > 0x7fffffffLL) return cudaErrorInvalidValue;
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap map;
  constexpr cuuint64_t kCols = NIN == 5 ? 8 : 16;
  const cuuint64_t dims[2] = {kCols, (cuuint64_t)P};
  const cuuint64_t strides[1] = {2 * kCols};
  const cuuint32_t box[2] = {8, (cuuint32_t)kRows};   // one core column of a 128-row tile
  const cuuint32_t estr[2] = {1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(x), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_mlp_bf16<NIN, SIGMOID>, cudaFuncAttributeMaxDynamicSharedMemorySize, M::Bytes) !=
        cudaSuccess)
      return cudaErrorInvalidValue;
    attr = true;
  }
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long ntiles = (P + kRows - 1) / kRows;
  long long grid = (long long)sms * kMlpCtasPerSm;
  if (grid > ntiles) grid = ntiles;
  k_mlp_bf16<NIN, SIGMOID><<<(unsigned)grid, kMlpThreads, M::Bytes, st>>>(
      map, w->w1, w->b1, w->w2, w->b2, w->w3, w->b3, reinterpret_cast<float4 *>(f), P, d_status,
      wait_limit_ns());
  return cudaGetLastError();
}

cudaError_t star_launch_mlp_bf16(const star_nt_mlp *w, const void *x, float *f, int64_t P,
                                 int32_t *d_status, cudaStream_t st) {
  return launch_mlp_bf16<5, false>(w, x, f, P, d_status, st);
}

cudaError_t star_launch_dfaoit_bf16(const star_nt_mlp *w, const void *x, float *f, int64_t P,
                                    int32_t *d_status, cudaStream_t st) {
  return launch_mlp_bf16<11, true>(w, x, f, P, d_status, st);
}

namespace star {
// Loads this file's kernels onto the current device (see star_nt_preload).
cudaError_t preload_mlp_tc() {
  cudaFuncAttributes a;
  cudaError_t e = cudaSuccess, r;
  if ((r = cudaFuncGetAttributes(&a, k_mlp_bf16<5, false>)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_mlp_bf16<11, true>)) != cudaSuccess) e = r;
  return e;
}
}  // namespace star
