// ozaki.cuh -- pieces shared by the tensor-core forms of W V_r (tsmm_oz.cu with mma.sync,
// tsmm_tc.cu with tcgen05): bulk copies on an mbarrier, exponents, and the splitting of a
// float-float value into six bf16-exact integer digits (Ozaki splitting; see tsmm_oz.cu).
#pragma once
#include "tsqr_kernels.cuh"

namespace tt {
namespace ozk {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void oz_bar_init(uint64_t* b) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void oz_expect(uint64_t* b, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                   smem_u32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void oz_bulk(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(b))
      : "memory");
}
__device__ __forceinline__ bool oz_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for the phase with this parity; false after about kWaitCycles
__device__ __forceinline__ bool oz_wait(uint64_t* b, uint32_t parity) {
  if (oz_try(b, parity)) return true;
  const long long t0 = clock64();
  while (!oz_try(b, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}

// biased exponent of |x| as if x were FP32 (x < 2^(be - 126)); 0 for zero
__device__ __forceinline__ int oz_bexp(df x) { return (__float_as_int(x.hi) >> 23) & 0xFF; }
__device__ __forceinline__ int oz_bexp(double x) {
  const int e = (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF);
  // FP64 exponent e - 1023 = FP32 biased exponent - 127; clamp into FP32's range
  const int f = e - 896;
  return e == 0 ? 0 : (f < 1 ? 1 : (f > 254 ? 254 : f));
}
// a word whose maximum over a row gives the row's largest exponent (oz_bexp_of)
__device__ __forceinline__ unsigned oz_key(df x) { return (unsigned)__float_as_int(x.hi) & 0x7F800000u; }
__device__ __forceinline__ unsigned oz_key(double x) {
  return (unsigned)((unsigned long long)__double_as_longlong(x) >> 32) & 0x7FF00000u;
}
__device__ __forceinline__ int oz_bexp_of(unsigned key, df*, int = 0) { return (int)(key >> 23); }
// FP64 values read as x 2^-sh (the input's exponent shift, engine.h XRange)
__device__ __forceinline__ int oz_bexp_of(unsigned key, double*, int sh = 0) {
  const int e = (int)(key >> 20);
  const int f = e - 896 - sh;
  return e == 0 ? 0 : (f < 1 ? 1 : (f > 254 ? 254 : f));
}
// 2^-E with E = be - 126, for scaling values into (-1, 1)
__device__ __forceinline__ float oz_inv_scale(int be) {
  const int s = 253 - be;  // biased exponent of 2^(126 - be)
  return __int_as_float((s < 1 ? 1 : (s > 254 ? 254 : s)) << 23);
}
// 2^e as FP32 (0 below the normal range)
__device__ __forceinline__ float oz_pow2(int e) {
  const int b = e + 127;
  return b < 1 ? 0.f : __int_as_float((b > 254 ? 254 : b) << 23);
}

// six digits of (hi + lo) 2^-E (see the header); d[a-1] = d_a.  Rounding to the nearest
// integer by adding and subtracting 1.5 * 2^23 (|t| <= 256 here): FMA-pipe operations only.
__device__ __forceinline__ void oz_digits(df x, float sc, float (&d)[6]) {
  constexpr float M = 12582912.f;  // 1.5 * 2^23
  float rem = x.hi * sc;
  const float sl = x.lo * sc;
  d[0] = __fsub_rn(__fmaf_rn(rem, 128.f, M), M);
  rem = __fmaf_rn(rem, 128.f, -d[0]);
  d[1] = __fsub_rn(__fmaf_rn(rem, 256.f, M), M);
  rem = __fmaf_rn(rem, 256.f, -d[1]);
  d[2] = __fsub_rn(__fmaf_rn(rem, 256.f, M), M);
  rem = __fmaf_rn(rem, 256.f, -d[2]);
  const float t = __fmaf_rn(sl, 2147483648.f, rem * 256.f);  // the low word enters at weight 2^31
  d[3] = __fsub_rn(__fadd_rn(t, M), M);
  rem = __fsub_rn(t, d[3]);
  d[4] = __fsub_rn(__fmaf_rn(rem, 256.f, M), M);
  rem = __fmaf_rn(rem, 256.f, -d[4]);
  d[5] = __fsub_rn(__fmaf_rn(rem, 256.f, M), M);
}

// two digits as a bf16 pair: a digit has at most 8 significant bits, so its bf16 is the
// upper half of its FP32 word; the smaller k goes to the low half
__device__ __forceinline__ uint32_t oz_pack(float lo_k, float hi_k) {
  return __byte_perm(__float_as_uint(lo_k), __float_as_uint(hi_k), 0x7632);
}

template <class S>
__device__ __forceinline__ S oz_zero() { return S{}; }

// FP64-accurate splitting (native FP64 form): seven signed digits of x relative to 2^(eM -
// 1022), the power of two above the largest magnitude of x's row (eM = that entry's biased
// exponent field), computed with integer operations only.  x is first made the integer
// v = x 2^(1084 - eM) (|v| < 2^62; bits below 2^-62 of the row maximum are dropped), then
// cut from the top into d_a at weight 2^(63 - 8a), a = 1..7, each rounded to nearest (so
// |d_a| <= 128, exact in bf16); the remainder, below 2^-56 of the row maximum, is dropped.
__device__ __forceinline__ float oz_small_int_to_float(int q) {
  // |q| < 2^22: 1.5 * 2^23 + q as a float, minus 1.5 * 2^23 (integer operations only)
  return __fsub_rn(__int_as_float(0x4B400000 + q), 12582912.0f);
}
__device__ __forceinline__ void oz64_digits(double x, int eM, float (&d)[7]) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  const long long M = (b & 0xFFFFFFFFFFFFFll) | (e ? (1ll << 52) : 0ll);
  const int sh = 9 - (eM - (e ? e : 1));
  long long v = sh >= 0 ? (M << sh) : (sh > -63 ? (M >> -sh) : 0ll);
  if (b < 0) v = -v;
#pragma unroll
  for (int a = 0; a < 7; ++a) {
    const int p = 55 - 8 * a;
    const long long q = (v + (1ll << (p - 1))) >> p;
    v -= q << p;
    d[a] = oz_small_int_to_float((int)q);
  }
}

}  // namespace ozk
}  // namespace tt
