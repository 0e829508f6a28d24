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
// between rounds.  counter = (quad, bunch, turn, tag), key = seed.
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

// Box-Muller on two 32-bit words, u = (w + 1/2) 2^-32: r_cos = R cos(2 pi u2),
// r_sin = R sin(2 pi u2), R = sqrt(-2 ln u1).  The four words of one Philox
// block give the normals of the quad of consecutive particles 4q .. 4q+3.
__device__ __forceinline__ void box_muller_f64(uint32_t a, uint32_t b, double &r_cos, double &r_sin) {
  const double u1 = ((double)a + 0.5) * 0x1.0p-32;
  const double u2 = ((double)b + 0.5) * 0x1.0p-32;
  const double R = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  r_cos = R * c;
  r_sin = R * s;
}

__device__ __forceinline__ void normal_quad_f64(const Words4 &w, double (&r)[4]) {
  box_muller_f64(w.w0, w.w1, r[0], r[1]);
  box_muller_f64(w.w2, w.w3, r[2], r[3]);
}

// The same to FP32 accuracy with the special-function unit.  cos(2 pi u2) =
// -cos(2 pi u2 - pi), likewise sin, so the MUFU argument lies in [-pi, pi)
// where its absolute error is about 2^-21.
__device__ __forceinline__ void box_muller_f32(uint32_t a, uint32_t b, float &r_cos, float &r_sin) {
  const float u1 = fmaf(__uint2float_rn(a), 0x1.0p-32f, 0x1.0p-33f);
  const float u2 = fmaf(__uint2float_rn(b), 0x1.0p-32f, 0x1.0p-33f);
  const float R2 = -2.0f * __logf(u1);
  const float R = R2 * rsqrtf(fmaxf(R2, 1e-30f));
  float s, c;
  __sincosf(fmaf(6.28318530717958647f, u2, -3.14159265358979324f), &s, &c);
  r_cos = -R * c;
  r_sin = -R * s;
}

__device__ __forceinline__ void normal_quad_f32(const Words4 &w, float (&r)[4]) {
  box_muller_f32(w.w0, w.w1, r[0], r[1]);
  box_muller_f32(w.w2, w.w3, r[2], r[3]);
}

// ---------------------------------------------------------------------------
// float <-> double on the integer pipe.  GB300's FP64 unit issues ~1.6 lanes
// per clock per SM (20 clocks per warp instruction), conversions included;
// these keep the mixed-precision push to one FP64 instruction (the delta
// accumulation) per particle.
// ---------------------------------------------------------------------------
// Widening of a float by exponent rebias (exact for normal floats).  Zero and
// subnormals map to +-2^-127 and non-finite values to +-2^128: both far
// outside anything a particle increment can be, and harmless there.
// (sign kept by the arithmetic shift and the mask; equal to
// (u & 0x80000000) | (((u & 0x7FFFFFFF) >> 3) + (896 << 20)) for every u.)
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t hi = (uint32_t)(((int)u >> 3) & (int)0x8FFFFFFF) + (896u << 20);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// 2^x on the special-function unit (subnormal results flushed to zero).
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Narrowing by truncation of the significand (error below one float ulp),
// exact in exponent for 2^-126 <= |d| < 2^128.  The caller guarantees d is
// never exactly zero (the widened increments above are never zero, so no
// accumulated delta is); magnitudes below 2^-126 come out as tiny subnormal
// floats, non-finite values as arbitrary finite ones.
__device__ __forceinline__ float f64_to_f32_trunc(double d) {
  const uint32_t hi = (uint32_t)__double2hiint(d);
  const uint32_t lo = (uint32_t)__double2loint(d);
  return __uint_as_float((__funnelshift_l(lo, hi, 3) - (896u << 23)) | (hi & 0x80000000u));
}

// A float near d for every finite |d| < 2^128 (a reference value for moment
// sums, not a rounding): 0 for |d| < 2^-100, where the narrowing above does
// not apply, the truncated value otherwise.  Integer pipe only.
// A fixed-point dipole sum (int64 in units of u, a power of two) as FP32:
// its high and low 32-bit words converted separately, q = hi 2^32 + lo, so
// that no 64-bit conversion is needed (the result is within 2^-23 of q u).
__device__ __forceinline__ float dip_q_to_f(long long q, float u) {
  const float hi = (float)(int)(q >> 32), lo = (float)(unsigned)(q & 0xFFFFFFFFLL);
  return fmaf(hi, 4294967296.f, lo) * u;
}

__device__ __forceinline__ float f64_to_f32_ref(double d) {
  const uint32_t hi = (uint32_t)__double2hiint(d);
  return (hi & 0x7FF00000u) < ((1023u - 100u) << 20) ? 0.f : f64_to_f32_trunc(d);
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
// composition of lanes 0..i, lane 0 applied first), for lanes below `width`
// (warp-uniform): a level of stride d >= width changes no such lane.  Not
// unrolled: the post kernel runs it once per turn, after the push has
// displaced its code from the caches, so its code length counts more than the
// loop overhead.
__device__ __forceinline__ void warp_scan_affine(double2 &A, double2 &B, int width = 32) {
  const int lane = threadIdx.x & 31;
#pragma unroll 1
  for (int d = 1; d < width; d <<= 1) {
    const double2 Ap = shfl_up_d2(A, d);
    const double2 Bp = shfl_up_d2(B, d);
    if (lane >= d) {
      B = cfma(A, Bp, B);
      A = cmul(A, Ap);
    }
  }
}

// Programmatic dependent launch: let the next kernel of the stream begin its
// prologue, and wait until the previous kernel has completed (its memory
// visible).  Both are no-ops when the launch did not opt in.
__device__ __forceinline__ void grid_dependents_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

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
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
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
