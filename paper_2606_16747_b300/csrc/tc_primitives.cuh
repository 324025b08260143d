// tc_primitives.cuh -- inline-PTX wrappers for the tcgen05 tensor cores,
// tensor memory, mbarriers and TMA, shared by the tensor-core kernels.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace star {

// Waits for an MMA commit or a TMA copy are bounded by a limit given at
// launch (star_nt_set_wait_limit, one second by default).  When one runs out
// the kernel stops its work; before it frees tensor memory or exits it still
// waits for the work it has in flight, under this second, fixed bound.
constexpr unsigned long long kDrainNs = 1000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok != 0;
}

// bounded wait: false when the phase did not complete within limit_ns
// (limit 0: false at once, without polling)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, unsigned long long limit_ns) {
  if (limit_ns == 0) return false;
  if (mbar_try(bar, phase)) return true;
  const unsigned long long t0 = globaltimer();
  while (!mbar_try(bar, phase))
    if (globaltimer() - t0 > limit_ns) return false;
  return true;
}

// The CTA waits for an MMA commit: one thread polls the mbarrier (bounded by
// limit_ns; on expiry it sets *abort and then drains the commit under
// kDrainNs, so that no MMA still writes tensor memory or reads the operands
// when the CTA goes on) while the others wait at the CTA barrier, which takes
// no issue slots; the tcgen05 fences order the MMA's tensor-memory writes
// before every thread's following tensor-memory loads.
__device__ __forceinline__ void mma_wait_cta(uint32_t bar, uint32_t phase, volatile int *abort,
                                             unsigned long long limit_ns) {
  if (threadIdx.x == 0 && !mbar_wait(bar, phase, limit_ns)) {
    *abort = 1;
    mbar_wait(bar, phase, kDrainNs);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture; no swizzle
  return d;
}

// kind::f16 instruction descriptor: bf16 A and B, fp32 D, K-major, M = 128
__host__ __device__ constexpr uint32_t idesc_bf16(uint32_t n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// kind::f8f6f4 instruction descriptor: e4m3 A and B (format code 0), fp32 D,
// K-major, M = 128 (K = 32 per instruction)
__host__ __device__ constexpr uint32_t idesc_e4m3(uint32_t n) {
  return (1u << 4) | ((n >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void mma_e4m3(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// four fp32 values to e4m3 (round to nearest even, saturating), byte i = v_i
__device__ __forceinline__ uint32_t pack4_e4m3(float v0, float v1, float v2, float v3) {
  uint32_t r;
  asm("{\n .reg .b16 lo, hi;\n"
      " cvt.rn.satfinite.e4m3x2.f32 lo, %2, %1;\n"
      " cvt.rn.satfinite.e4m3x2.f32 hi, %4, %3;\n"
      " mov.b32 %0, {lo, hi};\n}\n"
      : "=r"(r)
      : "f"(v0), "f"(v1), "f"(v2), "f"(v3));
  return r;
}

// four e4m3 bytes back to fp32, byte i -> v[i] (exact: every e4m3 value is
// an f16 value)
__device__ __forceinline__ void unpack4_e4m3(uint32_t q, float (&v)[4]) {
  asm("{\n .reg .b16 a, b, h0, h1, h2, h3;\n .reg .b32 p, q;\n"
      " mov.b32 {a, b}, %4;\n"
      " cvt.rn.f16x2.e4m3x2 p, a;\n"
      " cvt.rn.f16x2.e4m3x2 q, b;\n"
      " mov.b32 {h0, h1}, p;\n"
      " mov.b32 {h2, h3}, q;\n"
      " cvt.f32.f16 %0, h0;\n cvt.f32.f16 %1, h1;\n cvt.f32.f16 %2, h2;\n cvt.f32.f16 %3, h3;\n}\n"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
      : "r"(q));
}

// v = hi + lo + r with hi = e4m3(v), lo = e4m3(v - hi): |r| <= 2^-8 |v| for
// normal lo (e4m3 rounds to 2^-4 of the value), 2^-10 below the normal range
__device__ __forceinline__ void split4_e4m3(float v0, float v1, float v2, float v3, uint32_t &hi,
                                            uint32_t &lo) {
  hi = pack4_e4m3(v0, v1, v2, v3);
  float d[4];
  unpack4_e4m3(hi, d);
  lo = pack4_e4m3(v0 - d[0], v1 - d[1], v2 - d[2], v3 - d[3]);
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Tensor-memory loads: the load and its wait form one asm statement, so the
// destination registers are defined (and may be moved or spilled by the
// compiler) only once the asynchronous load has completed.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "{\n tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      " tcgen05.wait::ld.sync.aligned;\n}"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "{\n tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      " tcgen05.wait::ld.sync.aligned;\n}"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("{\n tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               " tcgen05.wait::ld.sync.aligned;\n}"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                 "=r"(r[7])
               : "r"(taddr)
               : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t *>(&h);
}

// ReLU of two fp32 values packed as bf16x2 (lo in the low half), round to
// nearest even: one cvt
__device__ __forceinline__ uint32_t pack_relu_bf16(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// one bf16 weight into the K-major core-matrix layout of a B operand
__device__ __forceinline__ void put_w(uint8_t *base, int n, int k, int lbo, float v) {
  __nv_bfloat16 h = __float2bfloat16_rn(v);
  *reinterpret_cast<__nv_bfloat16 *>(base + (k >> 3) * lbo + n * 16 + (k & 7) * 2) = h;
}

// one e4m3 weight into the K-major core-matrix layout of a B operand
// (16 elements per 16-byte core-matrix row)
__device__ __forceinline__ void put_w8(uint8_t *base, int n, int k, int lbo, float v) {
  base[(k >> 4) * lbo + n * 16 + (k & 15)] = (uint8_t)(pack4_e4m3(v, 0.f, 0.f, 0.f) & 255u);
}

// the e4m3 pair (hi, lo) of split4_e4m3 for one weight, as bytes
__device__ __forceinline__ void split_w8(float v, uint8_t &hi, uint8_t &lo) {
  uint32_t h, l;
  split4_e4m3(v, 0.f, 0.f, 0.f, h, l);
  hi = (uint8_t)(h & 255u);
  lo = (uint8_t)(l & 255u);
}

// A bias enters an MMA as two weight columns (k, k + 1) against an A operand
// block whose rows hold (1, 1, 0, ...): b = hi + lo with hi = bf16(b) and
// lo = bf16(b - hi), so the bias reaches the fp32 accumulator to about 2^-16
// of its size and no epilogue add is needed.
__device__ __forceinline__ void put_bias(uint8_t *base, int n, int k, int lbo, float b) {
  const float hi = __bfloat162float(__float2bfloat16_rn(b));
  put_w(base, n, k, lbo, hi);
  put_w(base, n, k + 1, lbo, b - hi);
}

// rows (1, 1, 0, 0, 0, 0, 0, 0) in bf16: the constant core-matrix column of
// the bias columns, 128 rows x 16 bytes
__device__ __forceinline__ void put_ones_block(uint8_t *base, int tid, int nthreads) {
  for (int r = tid; r < 128; r += nthreads)
    *reinterpret_cast<uint4 *>(base + r * 16) = make_uint4(0x3F803F80u, 0u, 0u, 0u);
}

}  // namespace star
