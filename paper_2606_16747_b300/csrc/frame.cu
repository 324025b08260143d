// frame.cu -- float32 tail-colour MLP on the CUDA cores (Sec. 3.3), the
// composite of Eq. 4, depth-based reprojection (Sec. 3.3, last paragraph)
// and the small C-ABI utilities.
#include <math.h>

#include <atomic>

#include "common.cuh"

namespace star {

// ---------------------------------------------------------------------------
// MLP 5 -> 32 -> 16 -> 3, ReLU everywhere, float32 with the weights in
// shared memory (every lane reads the same weight: broadcast).
constexpr int kW1 = 0, kB1 = 160, kW2 = 192, kB2 = 704, kW3 = 720, kB3 = 768;

// Two pixels per thread: every shared-memory weight read feeds two FMAs.
__device__ __forceinline__ void mlp_f32_pair(const float *s, const float (&xa)[5], const float (&xb)[5],
                                             float (&fa)[3], float (&fb)[3]) {
  float ha[32], hb[32];
#pragma unroll
  for (int o = 0; o < 32; ++o) {
    float a = s[kB1 + o], b = a;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const float w = s[kW1 + 5 * o + i];
      a = fmaf(w, xa[i], a);
      b = fmaf(w, xb[i], b);
    }
    ha[o] = fmaxf(a, 0.0f);
    hb[o] = fmaxf(b, 0.0f);
  }
  float ga[16], gb[16];
#pragma unroll
  for (int o = 0; o < 16; ++o) {
    float a = s[kB2 + o], b = a;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const float w = s[kW2 + 32 * o + i];
      a = fmaf(w, ha[i], a);
      b = fmaf(w, hb[i], b);
    }
    ga[o] = fmaxf(a, 0.0f);
    gb[o] = fmaxf(b, 0.0f);
  }
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    float a = s[kB3 + o], b = a;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const float w = s[kW3 + 16 * o + i];
      a = fmaf(w, ga[i], a);
      b = fmaf(w, gb[i], b);
    }
    fa[o] = fmaxf(a, 0.0f);
    fb[o] = fmaxf(b, 0.0f);
  }
}

__global__ void __launch_bounds__(256, 2) k_mlp_f32(const float *__restrict__ w1, const float *__restrict__ b1,
                                                 const float *__restrict__ w2, const float *__restrict__ b2,
                                                 const float *__restrict__ w3, const float *__restrict__ b3,
                                                 const float4 *__restrict__ X, float4 *__restrict__ F,
                                                 long long P) {
  __shared__ __align__(16) float s[776];
  for (int i = threadIdx.x; i < 160; i += 256) s[kW1 + i] = w1[i];
  for (int i = threadIdx.x; i < 512; i += 256) s[kW2 + i] = w2[i];
  if (threadIdx.x < 32) s[kB1 + threadIdx.x] = b1[threadIdx.x];
  if (threadIdx.x < 16) s[kB2 + threadIdx.x] = b2[threadIdx.x];
  if (threadIdx.x < 48) s[kW3 + threadIdx.x] = w3[threadIdx.x];
  if (threadIdx.x < 3) s[kB3 + threadIdx.x] = b3[threadIdx.x];
  __syncthreads();
  const long long half = (P + 1) / 2;  // thread i takes pixels i and i + half
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < half; i += (long long)gridDim.x * 256) {
    const long long pa = i, pb = i + half;
    const bool hb = pb < P;
    const float4 xa0 = X[2 * pa], xa1 = X[2 * pa + 1];
    float4 xb0 = make_float4(0.f, 0.f, 0.f, 0.f), xb1 = xb0;
    if (hb) {
      xb0 = X[2 * pb];
      xb1 = X[2 * pb + 1];
    }
    const float xa[5] = {xa0.x, xa0.y, xa0.z, xa0.w, xa1.x};
    const float xb[5] = {xb0.x, xb0.y, xb0.z, xb0.w, xb1.x};
    float fa[3], fb[3];
    mlp_f32_pair(s, xa, xb, fa, fb);
    F[pa] = xa1.y == 0.0f ? make_float4(0.f, 0.f, 0.f, 0.f) : make_float4(fa[0], fa[1], fa[2], 0.0f);
    if (hb) F[pb] = xb1.y == 0.0f ? make_float4(0.f, 0.f, 0.f, 0.f) : make_float4(fb[0], fb[1], fb[2], 0.0f);
  }
}

// ---------------------------------------------------------------------------
// Eq. 4 with the first and last terms already in front.rgb.
__global__ void __launch_bounds__(256) k_composite(const float4 *__restrict__ front,
                                                   const float4 *__restrict__ f, long long P,
                                                   float4 *__restrict__ out, uint32_t *__restrict__ q) {
  for (long long p = (long long)blockIdx.x * 256 + threadIdx.x; p < P; p += (long long)gridDim.x * 256) {
    const float4 a = front[p], b = f[p];
    const float r = fmaf(a.w, b.x, a.x), g = fmaf(a.w, b.y, a.y), bl = fmaf(a.w, b.z, a.z);
    if (out) out[p] = make_float4(r, g, bl, 1.0f);
    if (q) q[p] = quantize_rgba8(make_float4(r, g, bl, 1.0f));
  }
}

// ---------------------------------------------------------------------------
// Reprojection.  With M = VP_prev inv(VP_cur) and E = M - I, the previous
// clip position of v = (ndc_x, ndc_y, d, 1) is v + E v.  With the pixel
// centre written as px = x + 1/2 - W/2, py = y + 1/2 - H/2 (ndc_x = 2 px / W,
// ndc_y = -2 py / H), the screen offset of the sample is
//   dx = (b0 - px a3) / (1 + a3),  dy = (b1 - py a3) / (1 + a3),
//   b0 = (W/2) E_0 v,  b1 = -(H/2) E_1 v,  a3 = E_3 v,
// each b_k and a3 linear in (px, py, d, 1) with coefficients taken once per
// call in float64.  Under camera motion the depth and constant terms of b0
// and b1 cancel (at a 2 degree orbit step at 3840 wide, about 700 px each
// against an offset of 120 px), so float32 would lose about 1e-4 px there:
// the per-pixel arithmetic is float-float (hi + lo pairs, error-free products
// by FMA, error-free sums), which keeps the sample position to about 1e-9 px;
// only the bilinear weights and the blend are plain float32.
//
// inv(a) by cofactors: twelve 2x2 minors of rows 0-1 (s) and rows 2-3 (c),
// the determinant, then one entry of the adjugate per thread.  Sixteen
// threads; every value is the same expression as a one-thread evaluation.
__device__ __forceinline__ double minor2(const double *a, int k) {
  switch (k) {
    case 0: return a[0] * a[5] - a[4] * a[1];
    case 1: return a[0] * a[6] - a[4] * a[2];
    case 2: return a[0] * a[7] - a[4] * a[3];
    case 3: return a[1] * a[6] - a[5] * a[2];
    case 4: return a[1] * a[7] - a[5] * a[3];
    case 5: return a[2] * a[7] - a[6] * a[3];
    case 6: return a[8] * a[13] - a[12] * a[9];     // c0
    case 7: return a[8] * a[14] - a[12] * a[10];    // c1
    case 8: return a[8] * a[15] - a[12] * a[11];    // c2
    case 9: return a[9] * a[14] - a[13] * a[10];    // c3
    case 10: return a[9] * a[15] - a[13] * a[11];   // c4
    default: return a[10] * a[15] - a[14] * a[11];  // c5
  }
}

__device__ __forceinline__ double adjugate(const double *a, const double *s, const double *c, int k) {
  switch (k) {
    case 0: return a[5] * c[5] - a[6] * c[4] + a[7] * c[3];
    case 1: return -a[1] * c[5] + a[2] * c[4] - a[3] * c[3];
    case 2: return a[13] * s[5] - a[14] * s[4] + a[15] * s[3];
    case 3: return -a[9] * s[5] + a[10] * s[4] - a[11] * s[3];
    case 4: return -a[4] * c[5] + a[6] * c[2] - a[7] * c[1];
    case 5: return a[0] * c[5] - a[2] * c[2] + a[3] * c[1];
    case 6: return -a[12] * s[5] + a[14] * s[2] - a[15] * s[1];
    case 7: return a[8] * s[5] - a[10] * s[2] + a[11] * s[1];
    case 8: return a[4] * c[4] - a[5] * c[2] + a[7] * c[0];
    case 9: return -a[0] * c[4] + a[1] * c[2] - a[3] * c[0];
    case 10: return a[12] * s[4] - a[13] * s[2] + a[15] * s[0];
    case 11: return -a[8] * s[4] + a[9] * s[2] - a[11] * s[0];
    case 12: return -a[4] * c[3] + a[5] * c[1] - a[6] * c[0];
    case 13: return a[0] * c[3] - a[1] * c[1] + a[2] * c[0];
    case 14: return -a[12] * s[3] + a[13] * s[1] - a[14] * s[0];
    default: return a[8] * s[3] - a[9] * s[1] + a[10] * s[0];
  }
}

// Coefficients of b0, b1, a3 in (px, py, d, 1), once per call in float64,
// each stored as a float pair (hi, lo), hi + lo = the float64 value to about
// 2^-48 of it: C[row][term][2], rows b0, b1, a3.  One warp: threads 0..15
// own one entry of E each; threads 0..11 then one coefficient each.
__global__ void __launch_bounds__(32) k_reproject_matrix(const double *__restrict__ vp_prev,
                                                         const double *__restrict__ vp_cur, int W,
                                                         int H, float *__restrict__ C) {
  __shared__ double a[16], sc[12], inv[16], E[16], s_id;
  const int t = threadIdx.x;
  if (t < 16) a[t] = vp_cur[t];
  __syncwarp();
  if (t < 12) sc[t] = minor2(a, t);
  __syncwarp();
  if (t == 0) {
    const double *s = sc, *c = sc + 6;
    s_id = 1.0 / (s[0] * c[5] - s[1] * c[4] + s[2] * c[3] + s[3] * c[2] - s[4] * c[1] + s[5] * c[0]);
  }
  __syncwarp();
  if (t < 16) inv[t] = adjugate(a, sc, sc + 6, t) * s_id;
  __syncwarp();
  if (t < 16) {
    const int r = t >> 2, c = t & 3;
    double m = 0.0;
    for (int k = 0; k < 4; ++k) m += vp_prev[4 * r + k] * inv[4 * k + c];
    E[t] = m - (r == c ? 1.0 : 0.0);
  }
  __syncwarp();
  if (t < 12) {
    const int row = t >> 2, term = t & 3;
    const double w = (double)W, h = (double)H;
    double v;
    if (row == 0) {        // b0 = (W/2) E_0 v
      const double f[4] = {1.0, -w / h, 0.5 * w, 0.5 * w};
      v = f[term] * E[term];
    } else if (row == 1) { // b1 = -(H/2) E_1 v
      const double f[4] = {-h / w, 1.0, -0.5 * h, -0.5 * h};
      v = f[term] * E[4 + term];
    } else {               // a3 = E_3 v
      const double f[4] = {2.0 / w, -2.0 / h, 1.0, 1.0};
      v = f[term] * E[12 + term];
    }
    const float hi = (float)v;
    C[2 * t] = hi;
    C[2 * t + 1] = (float)(v - (double)hi);
  }
}

// float-float helpers: a value is hi + lo with |lo| <= ulp(hi) / 2.  The
// intrinsics keep every rounding explicit (no contraction into FMAs).
struct FF {
  float hi, lo;
};
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
}
__device__ __forceinline__ FF ff_norm(float s, float e) {  // |s| >= |e|
  const float h = __fadd_rn(s, e);
  return FF{h, __fsub_rn(e, __fsub_rn(h, s))};
}
// hi + lo of c t for a float-float coefficient c and a float t (the product
// of the hi parts error-free by FMA)
__device__ __forceinline__ FF ff_mul_f(float ch, float cl, float t) {
  const float p = __fmul_rn(ch, t);
  return FF{p, __fmaf_rn(cl, t, __fmaf_rn(ch, t, -p))};
}
// a row's value L + c2 d, where L = (c0 px) + (c1 py + c3) comes as the
// block's column and row terms (unnormalised float-float pairs) and c2 d is
// taken here
__device__ __forceinline__ FF ff_row_split(FF col, FF row, float c2h, float c2l, float d) {
  float s, e;
  two_sum(row.hi, col.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(row.lo, col.lo));
  const FF pd = ff_mul_f(c2h, c2l, d);
  float s2, e2;
  two_sum(s, pd.hi, s2, e2);
  return ff_norm(s2, __fadd_rn(e, __fadd_rn(pd.lo, e2)));
}
// (b - t a) inv, inv a float-float reciprocal of the denominator
__device__ __forceinline__ FF ff_offset_inv(FF b, float t, FF a, FF inv) {
  const FF ta = ff_mul_f(a.hi, a.lo, t);
  float s, e;
  two_sum(b.hi, -ta.hi, s, e);
  const FF num = ff_norm(s, __fadd_rn(e, __fsub_rn(b.lo, ta.lo)));
  const float q = __fmul_rn(num.hi, inv.hi);
  const float r = __fmaf_rn(num.hi, inv.hi, -q);
  return ff_norm(q, __fadd_rn(r, __fmaf_rn(num.hi, inv.lo, __fmul_rn(num.lo, inv.hi))));
}
// integer part and fractional weight of x + o (o float-float, |o| < 2^22)
__device__ __forceinline__ void ff_split(int x, FF o, int &i, float &f) {
  float fl = floorf(o.hi);
  float fr = __fadd_rn(__fsub_rn(o.hi, fl), o.lo);
  if (fr < 0.0f) { fr = __fadd_rn(fr, 1.0f); fl -= 1.0f; }
  if (fr >= 1.0f) { fr = __fsub_rn(fr, 1.0f); fl += 1.0f; }
  i = x + (int)fl;
  f = fr;
}

__global__ void __launch_bounds__(256) k_reproject(const float4 *__restrict__ prev,
                                                   const float *__restrict__ z1,
                                                   const float *__restrict__ Cg, int W, int H,
                                                   float4 *__restrict__ out,
                                                   uint32_t *__restrict__ q) {
  // per block of 32 x 8 pixels, each coefficient row's (px) and (py, 1)
  // parts once: s_col[row][column] = c0 px, s_row[row][y] = c1 py + c3
  __shared__ FF s_col[3][32], s_row[3][8];
  const int t = threadIdx.x;
  if (t < 96) {
    const int k = t >> 5, c = t & 31;
    const int xc = (int)blockIdx.x * 32 + c;
    const float px = 0.5f * (float)(2 * xc + 1 - W);
    s_col[k][c] = ff_mul_f(__ldg(Cg + 8 * k), __ldg(Cg + 8 * k + 1), px);
  } else if (t < 120) {
    const int k = (t - 96) >> 3, r = (t - 96) & 7;
    const int yr = (int)blockIdx.y * 8 + r;
    const float py = 0.5f * (float)(2 * yr + 1 - H);
    const FF p = ff_mul_f(__ldg(Cg + 8 * k + 2), __ldg(Cg + 8 * k + 3), py);
    float s, e;
    two_sum(p.hi, __ldg(Cg + 8 * k + 6), s, e);
    s_row[k][r] = FF{s, __fadd_rn(e, __fadd_rn(p.lo, __ldg(Cg + 8 * k + 7)))};
  }
  __syncthreads();
  const int lx = t & 31, ly = t >> 5;
  const int x = blockIdx.x * 32 + lx;
  const int y = blockIdx.y * 8 + ly;
  if (x >= W || y >= H) return;
  const size_t p = (size_t)y * W + x;
  // pixel centre relative to the image centre: exact half-integers
  const float px = 0.5f * (float)(2 * x + 1 - W), py = 0.5f * (float)(2 * y + 1 - H);
  const float d = z1[p];
  const FF a3 = ff_row_split(s_col[2][lx], s_row[2][ly], __ldg(Cg + 20), __ldg(Cg + 21), d);
  float s, e;
  two_sum(1.0f, a3.hi, s, e);
  const FF den = ff_norm(s, __fadd_rn(e, a3.lo));
  if (!(den.hi > 0.0f)) {
    const float4 v = prev[p];
    if (out) out[p] = v;
    if (q) q[p] = quantize_rgba8(v);
    return;
  }
  // 1 / den to float-float: one Newton step from the approximate float
  // reciprocal (relative error 2^-22 squared by the step)
  float r0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(den.hi));
  const float res = __fmaf_rn(-den.lo, r0, __fmaf_rn(-den.hi, r0, 1.0f));
  const FF inv = ff_norm(r0, __fmul_rn(r0, res));
  FF dx = ff_offset_inv(ff_row_split(s_col[0][lx], s_row[0][ly], __ldg(Cg + 4), __ldg(Cg + 5), d), px, a3, inv);
  FF dy = ff_offset_inv(ff_row_split(s_col[1][lx], s_row[1][ly], __ldg(Cg + 12), __ldg(Cg + 13), d), py, a3, inv);
  const float lxb = 2.0f * W + 2.0f, lyb = 2.0f * H + 2.0f;  // far outside: clamped to the edge anyway
  if (!(fabsf(dx.hi) <= lxb)) dx = FF{copysignf(lxb, dx.hi), 0.0f};
  if (!(fabsf(dy.hi) <= lyb)) dy = FF{copysignf(lyb, dy.hi), 0.0f};
  int ix, iy;
  float fx, fy;
  ff_split(x, dx, ix, fx);
  ff_split(y, dy, iy, fy);
  const int x0 = min(max(ix, 0), W - 1), x1 = min(max(ix + 1, 0), W - 1);
  const int y0 = min(max(iy, 0), H - 1), y1 = min(max(iy + 1, 0), H - 1);
  // W, H <= 32768: pixel indices fit 32 bits
  const float4 *r0p = prev + y0 * W, *r1p = prev + y1 * W;
  const float4 v00 = r0p[x0], v10 = r0p[x1], v01 = r1p[x0], v11 = r1p[x1];
  float4 o;
  o.x = (1.f - fy) * ((1.f - fx) * v00.x + fx * v10.x) + fy * ((1.f - fx) * v01.x + fx * v11.x);
  o.y = (1.f - fy) * ((1.f - fx) * v00.y + fx * v10.y) + fy * ((1.f - fx) * v01.y + fx * v11.y);
  o.z = (1.f - fy) * ((1.f - fx) * v00.z + fx * v10.z) + fy * ((1.f - fx) * v01.z + fx * v11.z);
  if (out) {  // the 8-bit copy takes no alpha
    o.w = (1.f - fy) * ((1.f - fx) * v00.w + fx * v10.w) + fy * ((1.f - fx) * v01.w + fx * v11.w);
    out[p] = o;
  }
  if (q) q[p] = quantize_rgba8(o);
}

static int grid_for(long long P) {
  long long g = (P + 255) / 256;
  if (g > 148 * 16) g = 148 * 16;
  return g < 1 ? 1 : (int)g;
}

}  // namespace star

using namespace star;

cudaError_t star_launch_mlp_bf16(const star_nt_mlp *w, const void *x, float *f, int64_t P,
                                 int32_t *d_status, cudaStream_t st);

extern "C" int32_t star_nt_version(void) { return STAR_NT_VERSION; }

// Bound of the tensor-core kernels' waits, read at every launch.
static std::atomic<unsigned long long> g_wait_limit_ns{1000000000ull};

namespace star {
unsigned long long wait_limit_ns() { return g_wait_limit_ns.load(std::memory_order_relaxed); }
}  // namespace star

extern "C" star_nt_status star_nt_set_wait_limit(uint64_t ns) {
  if (ns > STAR_NT_MAX_WAIT_LIMIT_NS) return STAR_NT_ERR_ARG;
  g_wait_limit_ns.store(ns, std::memory_order_relaxed);
  return STAR_NT_OK;
}

extern "C" uint64_t star_nt_wait_limit(void) { return g_wait_limit_ns.load(std::memory_order_relaxed); }

extern "C" const char *star_nt_status_string(int32_t s) {
  switch (s) {
    case STAR_NT_OK: return "ok";
    case STAR_NT_ERR_ARG: return "invalid argument";
    case STAR_NT_ERR_CAPACITY: return "capacity exceeded";
    case STAR_NT_ERR_CUDA: return "CUDA error";
    case STAR_NT_ERR_TIMEOUT: return "device wait timed out";
    case STAR_NT_ERR_UNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

extern "C" void star_nt_default_params(star_nt_params *p) {
  if (!p) return;
  p->bg[0] = p->bg[1] = p->bg[2] = 1.0f;
  p->kappa_n = 1.0f / 64.0f;
  p->tau_split = 24.0;
  p->tau_merge = 12.0;
  p->delta2 = 2.2;
  p->delta3 = 3.0;
  p->base_tile = 16;
  p->relax_iters = 2;
}

extern "C" star_nt_status star_nt_infer(const star_nt_mlp *w, int32_t x_dtype, const void *x,
                                        float *f, int64_t P, int32_t *d_status, void *stream) {
  if (!w || !w->w1 || !w->b1 || !w->w2 || !w->b2 || !w->w3 || !w->b3 || P < 0) return STAR_NT_ERR_ARG;
  if (P > 0 && (!x || !f)) return STAR_NT_ERR_ARG;
  if (((uintptr_t)x & 15u) || ((uintptr_t)f & 15u)) return STAR_NT_ERR_ARG;
  if (P == 0) return STAR_NT_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (x_dtype == STAR_NT_F32) {
    k_mlp_f32<<<grid_for(P), 256, 0, st>>>(w->w1, w->b1, w->w2, w->b2, w->w3, w->b3,
                                           reinterpret_cast<const float4 *>(x),
                                           reinterpret_cast<float4 *>(f), P);
    return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
  }
  if (x_dtype == STAR_NT_BF16) {
    if ((uintptr_t)x & 255u) return STAR_NT_ERR_ARG;
    return star_launch_mlp_bf16(w, x, f, P, d_status, st) == cudaSuccess ? STAR_NT_OK
                                                                          : STAR_NT_ERR_CUDA;
  }
  return STAR_NT_ERR_ARG;
}

extern "C" star_nt_status star_nt_composite(const float *front, const float *f, int64_t P,
                                            float *rgba32f, uint32_t *rgba8, void *stream) {
  if (P < 0 || (P > 0 && (!front || !f || (!rgba32f && !rgba8)))) return STAR_NT_ERR_ARG;
  if (((uintptr_t)front & 15u) || ((uintptr_t)f & 15u) || ((uintptr_t)rgba32f & 15u))
    return STAR_NT_ERR_ARG;
  if (P == 0) return STAR_NT_OK;
  k_composite<<<grid_for(P), 256, 0, (cudaStream_t)stream>>>(
      reinterpret_cast<const float4 *>(front), reinterpret_cast<const float4 *>(f), P,
      reinterpret_cast<float4 *>(rgba32f), rgba8);
  return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
}

extern "C" star_nt_status star_nt_reproject(const float *prev_rgba, const float *prev_z1,
                                            const double *vp_prev, const double *vp_cur, int32_t W,
                                            int32_t H, float *out_rgba, uint32_t *out_rgba8,
                                            void *ws, void *stream) {
  if (W <= 0 || H <= 0 || W > 32768 || H > 32768 || !prev_rgba || !prev_z1 || !vp_prev || !vp_cur ||
      (!out_rgba && !out_rgba8) ||
      !ws || prev_rgba == out_rgba)
    return STAR_NT_ERR_ARG;
  if (((uintptr_t)prev_rgba & 15u) || ((uintptr_t)out_rgba & 15u) || ((uintptr_t)vp_prev & 7u) ||
      ((uintptr_t)vp_cur & 7u) || ((uintptr_t)ws & 15u))
    return STAR_NT_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  float *C = reinterpret_cast<float *>(ws);
  k_reproject_matrix<<<1, 32, 0, st>>>(vp_prev, vp_cur, W, H, C);
  dim3 grid((W + 31) / 32, (H + 7) / 8);
  k_reproject<<<grid, 256, 0, st>>>(reinterpret_cast<const float4 *>(prev_rgba), prev_z1, C, W, H,
                                    reinterpret_cast<float4 *>(out_rgba), out_rgba8);
  return cudaGetLastError() == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
}

namespace star {
// Loads this file's kernels onto the current device (see star_nt_preload).
cudaError_t preload_frame() {
  cudaFuncAttributes a;
  cudaError_t e = cudaSuccess, r;
  if ((r = cudaFuncGetAttributes(&a, k_mlp_f32)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_composite)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_reproject_matrix)) != cudaSuccess) e = r;
  if ((r = cudaFuncGetAttributes(&a, k_reproject)) != cudaSuccess) e = r;
  return e;
}
}  // namespace star

namespace star {
cudaError_t preload_raster();
cudaError_t preload_passes();
cudaError_t preload_mlp_tc();
cudaError_t preload_resolve_tc();
cudaError_t preload_quadtree();
cudaError_t preload_train();
cudaError_t preload_baselines();
cudaError_t preload_leaf();
cudaError_t preload_passes_resolve();
cudaError_t preload_dfaoit();
}  // namespace star

extern "C" star_nt_status star_nt_preload(void) {
  cudaError_t e = cudaSuccess, r;
  if ((r = preload_raster()) != cudaSuccess) e = r;
  if ((r = preload_passes()) != cudaSuccess) e = r;
  if ((r = preload_frame()) != cudaSuccess) e = r;
  if ((r = preload_mlp_tc()) != cudaSuccess) e = r;
  if ((r = preload_resolve_tc()) != cudaSuccess) e = r;
  if ((r = preload_quadtree()) != cudaSuccess) e = r;
  if ((r = preload_train()) != cudaSuccess) e = r;
  if ((r = preload_baselines()) != cudaSuccess) e = r;
  if ((r = preload_leaf()) != cudaSuccess) e = r;
  if ((r = preload_passes_resolve()) != cudaSuccess) e = r;
  if ((r = preload_dfaoit()) != cudaSuccess) e = r;
  return e == cudaSuccess ? STAR_NT_OK : STAR_NT_ERR_CUDA;
}
