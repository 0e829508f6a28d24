// Device helpers shared by the libmbt kernels: the counter-based normal
// generator, bit-level float/double conversions, warp reductions and the
// Blackwell (sm_103a) asynchronous-copy / tensor-memory primitives.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "mbt_internal.h"

namespace mbt {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the 4x32
// S-box, each a pair of 32x32->64 multiplications, with the Weyl key bump
// between rounds.  counter = (pair, bunch, turn, tag), key = seed.
// ---------------------------------------------------------------------------
struct Words4 { uint32_t w0, w1, w2, w3; };

__device__ __forceinline__ Words4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;   // mul.wide.u32
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)p1;
    c3 = (uint32_t)p0;
    c0 = n0;
    c2 = n2;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return Words4{c0, c1, c2, c3};
}

// FP64 uniform on (0,1): top 53 bits of hi:lo times 2^-53, plus 2^-54.
__device__ __forceinline__ double u01_f64(uint32_t hi, uint32_t lo) {
  const uint64_t x = ((uint64_t)hi << 32) | lo;
  return __dadd_rn(__dmul_rn((double)(x >> 11), 0x1.0p-53), 0x1.0p-54);
}

// The same uniform to FP32 accuracy (relative error ~2^-24 everywhere, never 0).
__device__ __forceinline__ float u01_f32(uint32_t hi, uint32_t lo) {
  return fmaf(__uint2float_rn(lo), 0x1.0p-64f, __uint2float_rn(hi) * 0x1.0p-32f) + 0x1.0p-54f;
}

// Box-Muller pair: r_even = R cos(2 pi u2), r_odd = R sin(2 pi u2), R = sqrt(-2 ln u1).
__device__ __forceinline__ void normal_pair_f64(const Words4 &w, double &r_even, double &r_odd) {
  const double u1 = u01_f64(w.w0, w.w1);
  const double u2 = u01_f64(w.w2, w.w3);
  const double R = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  r_even = R * c;
  r_odd = R * s;
}

__device__ __forceinline__ void normal_pair_f32(const Words4 &w, float &r_even, float &r_odd) {
  const float u1 = u01_f32(w.w0, w.w1);
  const float u2 = u01_f32(w.w2, w.w3);
  const float R = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  r_even = R * c;
  r_odd = R * s;
}

// ---------------------------------------------------------------------------
// float <-> double on the integer pipe.  GB300's FP64 unit issues ~1.7
// operations per clock per SM; these keep the mixed-precision push to one
// FP64 instruction (the delta accumulation) per particle.
// ---------------------------------------------------------------------------
// Exact widening of a normal float; zero and subnormal inputs give a signed
// zero, infinities and NaN keep their class.
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t sign = u & 0x80000000u;
  const uint32_t mag = u & 0x7FFFFFFFu;
  uint32_t hi = sign | ((mag >> 3) + (896u << 20));
  uint32_t lo = mag << 29;
  if (mag < 0x00800000u) { hi = sign; lo = 0u; }
  if (mag >= 0x7F800000u) { hi = sign | 0x7FF00000u | ((mag & 0x007FFFFFu) >> 3); lo = mag << 29; }
  return __hiloint2double((int)hi, (int)lo);
}

// Narrowing by truncation toward zero of the significand (error < 1 float
// ulp); magnitudes below 2^-126 give a signed zero, NaN stays NaN.
__device__ __forceinline__ float f64_to_f32_trunc(double d) {
  const uint32_t hi = (uint32_t)__double2hiint(d);
  const uint32_t lo = (uint32_t)__double2loint(d);
  const uint32_t sign = hi & 0x80000000u;
  const uint32_t mag = hi & 0x7FFFFFFFu;
  uint32_t f = sign | (((mag - (896u << 20)) << 3) | (lo >> 29));
  if (mag < (897u << 20)) f = sign;
  if (mag >= (1151u << 20)) f = sign | 0x7F800000u | ((mag > 0x7FF00000u || (mag == 0x7FF00000u && lo)) ? 0x400000u : 0u);
  return __uint_as_float(f);
}

// ---------------------------------------------------------------------------
// complex helpers (double2 = re, im)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {  // a*b + c
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

__device__ __forceinline__ double2 shfl_up_d2(double2 v, int d) {
  return make_double2(__shfl_up_sync(0xFFFFFFFFu, v.x, d), __shfl_up_sync(0xFFFFFFFFu, v.y, d));
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

// Inclusive warp scan of affine maps x -> A x + B (lane i ends with the
// composition of lanes 0..i, lane 0 applied first).
__device__ __forceinline__ void warp_scan_affine(double2 &A, double2 &B) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const double2 Ap = shfl_up_d2(A, d);
    const double2 Bp = shfl_up_d2(B, d);
    if (lane >= d) {
      B = cfma(A, Bp, B);
      A = cmul(A, Ap);
    }
  }
}

__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------
// sm_103a asynchronous copies, mbarriers and tensor memory (inline PTX).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
// Bulk (non-tensor) global -> shared copy through the TMA engine; dst, src
// 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for a phase with a wall-clock limit; false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, unsigned long long limit_ns) {
  const unsigned long long t0 = global_timer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_timer_ns() - t0 > limit_ns) return false;
  }
  return true;
}

// Tensor memory allocation (one full warp executes these).
__device__ __forceinline__ void tmem_alloc(uint32_t *slot_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot_smem)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major operand without swizzle: 8x16-byte
// core matrices, lbo = byte step between core matrices along K, sbo = byte
// step between 8-row groups along M/N.
__device__ __forceinline__ uint64_t smem_desc_kmajor(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version for sm_100-family tensor cores
  return d;                 // base offset 0, absolute LBO mode off, no swizzle
}

// Instruction descriptor of tcgen05.mma kind::f16: BF16 A and B (K-major),
// FP32 accumulator, M x N tile.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4)                      // D format: F32
         | (1u << 7)                    // A format: BF16
         | (1u << 10)                   // B format: BF16
         | ((uint32_t)(N >> 3) << 17)   // N / 8
         | ((uint32_t)(M >> 4) << 24);  // M / 16
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

// 32 lanes x 32 columns of 32-bit values from tensor memory (warp-collective).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace mbt
