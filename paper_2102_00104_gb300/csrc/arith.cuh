// arith.cuh -- the three arithmetics of the engine behind one set of overloads.
//
//   double : native FP64 (GB300 issues FP64 FMAs at ~1/70 of the FP32 rate)
//   df     : float-float, value = hi + lo with two FP32 words (~48 bits),
//            built from the error-free transformations TwoSum (Knuth, TAOCP
//            vol. 2, 4.2.2) and TwoProd via FMA (the FMA form of Dekker 1971).
//   float  : FP32 (the FP32-storage form's panels and W*V_r)
//
// Every building block of an error-free transformation uses the _rn
// intrinsics so that the compiler cannot contract or reassociate it.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <float.h>

struct __align__(8) df {
  float hi, lo;
};

// ----------------------------------------------------------------------------
// error-free transformations
__device__ __forceinline__ void eft_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void eft_fast_two_sum(float a, float b, float& s, float& e) {
  // requires |a| >= |b| (or a == 0)
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void eft_two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// ----------------------------------------------------------------------------
// df operations ("sloppy" variants: normwise error ~ 2^-47 of the operands)
__device__ __forceinline__ df mkdf(float h, float l) { df r; r.hi = h; r.lo = l; return r; }
__device__ __forceinline__ df df_norm(float s, float e) {
  df r; eft_fast_two_sum(s, e, r.hi, r.lo); return r;
}
__device__ __forceinline__ df add(df a, df b) {
  float s, e; eft_two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_norm(s, e);
}
__device__ __forceinline__ df neg(df a) { return mkdf(-a.hi, -a.lo); }
__device__ __forceinline__ df sub(df a, df b) { return add(a, neg(b)); }
__device__ __forceinline__ df mul(df a, df b) {
  float p, e; eft_two_prod(a.hi, b.hi, p, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_norm(p, e);
}
// fmac(a, b, c) = a*b + c ; fnmac(a, b, c) = c - a*b
__device__ __forceinline__ df fmac(df a, df b, df c) {
  float p, e; eft_two_prod(a.hi, b.hi, p, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s, e2; eft_two_sum(p, c.hi, s, e2);
  e2 = __fadd_rn(e2, __fadd_rn(e, c.lo));
  return df_norm(s, e2);
}
__device__ __forceinline__ df fnmac(df a, df b, df c) { return fmac(neg(a), b, c); }
__device__ __forceinline__ df dfdiv(df a, df b) {
  // long division: q1 = a/b in FP32, remainder in df, two correction terms
  float q1 = __fdiv_rn(a.hi, b.hi);
  df r = fnmac(mkdf(q1, 0.f), b, a);
  float q2 = __fdiv_rn(r.hi, b.hi);
  r = fnmac(mkdf(q2, 0.f), b, r);
  float q3 = __fdiv_rn(r.hi, b.hi);
  df q = df_norm(q1, q2);
  return add(q, mkdf(q3, 0.f));
}
__device__ __forceinline__ df div_(df a, df b) { return dfdiv(a, b); }
// hardware approximations (PTX rcp.approx / sqrt.approx, relative error about one ulp);
// every use below is followed by a Newton step in float-float
__device__ __forceinline__ float rcp_seed(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sqrt_seed(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// 1/b: FP32 reciprocal seed and one Newton step in df (relative error ~ (2^-23)^2)
__device__ __forceinline__ df rcp_(df b) {
  const float r0 = rcp_seed(b.hi);
  const df e = fnmac(b, mkdf(r0, 0.f), mkdf(1.f, 0.f));   // 1 - b r0
  return fmac(mkdf(r0, 0.f), e, mkdf(r0, 0.f));           // r0 + r0 e
}
__device__ __forceinline__ df sqrt_(df a) {
  // one Newton correction of the FP32 root: x + (a - x^2) / (2x), residual in df
  if (!(a.hi > 0.f)) return mkdf(0.f, 0.f);
  float x = sqrt_seed(a.hi);
  float p, e; eft_two_prod(x, x, p, e);
  df res = sub(a, mkdf(p, e));
  float corr = __fmul_rn(res.hi, rcp_seed(__fmul_rn(2.f, x)));
  return df_norm(x, corr);
}
__device__ __forceinline__ bool is_pos(df a) { return a.hi > 0.f; }
__device__ __forceinline__ bool is_gt(df a, df b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ df abs_(df a) { return a.hi < 0.f ? neg(a) : a; }
__device__ __forceinline__ double to_f64(df a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ df shfl_xor(df a, int m) {
  return mkdf(__shfl_xor_sync(0xffffffffu, a.hi, m), __shfl_xor_sync(0xffffffffu, a.lo, m));
}
__device__ __forceinline__ df shfl_idx(df a, int src) {
  return mkdf(__shfl_sync(0xffffffffu, a.hi, src), __shfl_sync(0xffffffffu, a.lo, src));
}

// ----------------------------------------------------------------------------
// double and float with the same names
__device__ __forceinline__ double add(double a, double b) { return a + b; }
__device__ __forceinline__ double sub(double a, double b) { return a - b; }
__device__ __forceinline__ double neg(double a) { return -a; }
__device__ __forceinline__ double mul(double a, double b) { return a * b; }
__device__ __forceinline__ double fmac(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ double fnmac(double a, double b, double c) { return __fma_rn(-a, b, c); }
__device__ __forceinline__ double div_(double a, double b) { return a / b; }
__device__ __forceinline__ double rcp_(double b) { return 1.0 / b; }
__device__ __forceinline__ double sqrt_(double a) { return a > 0.0 ? sqrt(a) : 0.0; }
__device__ __forceinline__ bool is_pos(double a) { return a > 0.0; }
__device__ __forceinline__ bool is_gt(double a, double b) { return a > b; }
__device__ __forceinline__ double abs_(double a) { return fabs(a); }
__device__ __forceinline__ double to_f64(double a) { return a; }
__device__ __forceinline__ double shfl_xor(double a, int m) { return __shfl_xor_sync(0xffffffffu, a, m); }
__device__ __forceinline__ double shfl_idx(double a, int s) { return __shfl_sync(0xffffffffu, a, s); }

__device__ __forceinline__ float add(float a, float b) { return a + b; }
__device__ __forceinline__ float sub(float a, float b) { return a - b; }
__device__ __forceinline__ float neg(float a) { return -a; }
__device__ __forceinline__ float mul(float a, float b) { return a * b; }
__device__ __forceinline__ float fmac(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float fnmac(float a, float b, float c) { return __fmaf_rn(-a, b, c); }
__device__ __forceinline__ float div_(float a, float b) { return a / b; }
__device__ __forceinline__ float rcp_(float b) { return 1.0f / b; }
__device__ __forceinline__ float sqrt_(float a) { return a > 0.f ? sqrtf(a) : 0.f; }
__device__ __forceinline__ bool is_pos(float a) { return a > 0.f; }
__device__ __forceinline__ bool is_gt(float a, float b) { return a > b; }
__device__ __forceinline__ float abs_(float a) { return fabsf(a); }
__device__ __forceinline__ double to_f64(float a) { return (double)a; }
__device__ __forceinline__ float shfl_xor(float a, int m) { return __shfl_xor_sync(0xffffffffu, a, m); }
__device__ __forceinline__ float shfl_idx(float a, int s) { return __shfl_sync(0xffffffffu, a, s); }

// ----------------------------------------------------------------------------
// lazy float-float sums for reductions: value = s + e with e unnormalised.
// Each addition is one TwoSum of the leading words plus plain adds of the
// trailing ones, so a chain of additions waits only on the FP32 add of the
// leading words; lz_fin normalises once (with a full TwoSum) at the end.
struct dfl {
  float s, e;
};
__device__ __forceinline__ dfl lz(df a) { dfl r; r.s = a.hi; r.e = a.lo; return r; }
__device__ __forceinline__ float lz(float a) { return a; }
__device__ __forceinline__ double lz(double a) { return a; }
__device__ __forceinline__ dfl lz_add(dfl a, dfl b) {
  dfl r; float t;
  eft_two_sum(a.s, b.s, r.s, t);
  r.e = __fadd_rn(__fadd_rn(a.e, b.e), t);
  return r;
}
__device__ __forceinline__ float lz_add(float a, float b) { return a + b; }
__device__ __forceinline__ double lz_add(double a, double b) { return a + b; }
__device__ __forceinline__ df lz_fin(dfl a) { df r; eft_two_sum(a.s, a.e, r.hi, r.lo); return r; }
__device__ __forceinline__ float lz_fin(float a) { return a; }
__device__ __forceinline__ double lz_fin(double a) { return a; }
// acc + a*b with a lazy accumulator: TwoProd of the leading words, the cross terms
// and both rounding errors go to the trailing word (12 FP32 instructions)
__device__ __forceinline__ dfl lz_fmac(df a, df b, dfl acc) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s, t;
  eft_two_sum(acc.s, p, s, t);
  dfl r;
  r.s = s;
  r.e = __fadd_rn(acc.e, __fadd_rn(e, t));
  return r;
}
__device__ __forceinline__ float lz_fmac(float a, float b, float acc) { return __fmaf_rn(a, b, acc); }
__device__ __forceinline__ double lz_fmac(double a, double b, double acc) { return __fma_rn(a, b, acc); }
// c - a*b without the final renormalisation (12 FP32 instructions): the pair
// (hi, lo) stays an exact-sum representation whose trailing word may reach a
// few ulps of the leading one; every operation here accepts such pairs.  Used for
// values that are updated many times (panel columns), renormalised when stored.
__device__ __forceinline__ df fnmac_nr(df a, df b, df c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s, t;
  eft_two_sum(c.hi, -p, s, t);
  return mkdf(s, __fadd_rn(__fsub_rn(c.lo, e), t));
}
// back to a normalised pair (hi = the FP32 rounding of the value).  A product
// of two pairs drops lo*lo, which is only negligible when one factor is
// normalised: pivot columns are renormalised before they are used.
__device__ __forceinline__ df renorm(df a) { df r; eft_two_sum(a.hi, a.lo, r.hi, r.lo); return r; }
__device__ __forceinline__ float renorm(float a) { return a; }
__device__ __forceinline__ double renorm(double a) { return a; }
__device__ __forceinline__ float fnmac_nr(float a, float b, float c) { return __fmaf_rn(-a, b, c); }
__device__ __forceinline__ double fnmac_nr(double a, double b, double c) { return __fma_rn(-a, b, c); }
__device__ __forceinline__ dfl shfl_xor_m(dfl a, int m, unsigned mask) {
  dfl r;
  r.s = __shfl_xor_sync(mask, a.s, m);
  r.e = __shfl_xor_sync(mask, a.e, m);
  return r;
}
__device__ __forceinline__ double shfl_xor_m(double a, int m, unsigned mask) { return __shfl_xor_sync(mask, a, m); }
__device__ __forceinline__ float shfl_xor_m(float a, int m, unsigned mask) { return __shfl_xor_sync(mask, a, m); }
// lazy sum over an aligned group of G lanes (G divides 32; mask = the group's lanes)
template <int G, class Z>
__device__ __forceinline__ Z lz_gsum(Z a, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) a = lz_add(a, shfl_xor_m(a, o, mask));
  return a;
}
__device__ __forceinline__ dfl shfl_xor(dfl a, int m) {
  dfl r;
  r.s = __shfl_xor_sync(0xffffffffu, a.s, m);
  r.e = __shfl_xor_sync(0xffffffffu, a.e, m);
  return r;
}

// ----------------------------------------------------------------------------
// traits: zero, smallest positive normalised number (eps_FP of Alg. 6), and
// conversions between storage and compute types.
template <class C> struct Tr;
template <> struct Tr<double> {
  __device__ static double zero() { return 0.0; }
  __device__ static double one() { return 1.0; }
  __device__ static double eps() { return DBL_MIN; }
  __device__ static double of(double x) { return x; }
};
template <> struct Tr<float> {
  __device__ static float zero() { return 0.f; }
  __device__ static float one() { return 1.f; }
  __device__ static float eps() { return FLT_MIN; }
  __device__ static float of(double x) { return (float)x; }
};
template <> struct Tr<df> {
  __device__ static df zero() { return mkdf(0.f, 0.f); }
  __device__ static df one() { return mkdf(1.f, 0.f); }
  __device__ static df eps() { return mkdf(FLT_MIN, 0.f); }
  __device__ static df of(double x) {
    float h = (float)x;
    return mkdf(h, (float)(x - (double)h));
  }
};

// df from an FP64 value without FP64 instructions: hi = the FP64 value cut to
// 24 significant bits, lo = the next 23 bits (47 bits kept).  Exponents outside
// the normal FP32 range flush to zero / overflow to infinity.
__device__ __forceinline__ df df_from_f64_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7FF);
  const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
  const int fe = e - 1023 + 127;
  if (fe <= 0) return mkdf(0.f, 0.f);
  if (fe >= 255) return mkdf(__int_as_float((int)(sign | 0x7F800000u)), 0.f);
  const float hi = __int_as_float((int)(sign | ((unsigned)fe << 23) | (unsigned)(mant >> 29)));
  // remaining 29 bits; keep the top 23 of them as an exact small integer
  const unsigned rem23 = (unsigned)((mant & 0x1FFFFFFFull) >> 6);
  const float f = __fsub_rn(__int_as_float((int)(0x4B000000u | rem23)), 8388608.0f);
  // value of one unit of rem23: 2^(e - 1023 - 52 + 6)
  const int se = e - 1069 + 127;
  const float scale = se > 0 ? __int_as_float(se << 23) : 0.f;
  float lo = __fmul_rn(f, scale);
  lo = sign ? -lo : lo;
  return mkdf(hi, lo);
}

// storage -> compute
template <class C, class S> struct Ld;
template <> struct Ld<df, double> { __device__ static df f(double x) { return df_from_f64_bits(x); } };
template <> struct Ld<df, df> { __device__ static df f(df x) { return x; } };
template <> struct Ld<df, float> { __device__ static df f(float x) { return mkdf(x, 0.f); } };
template <> struct Ld<double, double> { __device__ static double f(double x) { return x; } };
template <> struct Ld<float, float> { __device__ static float f(float x) { return x; } };
template <> struct Ld<float, double> { __device__ static float f(double x) { return (float)x; } };
template <> struct Ld<float, df> { __device__ static float f(df x) { return x.hi; } };
template <> struct Ld<double, float> { __device__ static double f(float x) { return (double)x; } };
template <> struct Ld<double, df> { __device__ static double f(df x) { return to_f64(x); } };
template <class C, class S> __device__ __forceinline__ C ld_as(S x) { return Ld<C, S>::f(x); }

// compute -> storage
template <class S, class C> struct St;
template <> struct St<df, df> { __device__ static df f(df x) { return x; } };
template <> struct St<double, df> { __device__ static double f(df x) { return to_f64(x); } };
template <> struct St<float, df> { __device__ static float f(df x) { return x.hi; } };
template <> struct St<double, double> { __device__ static double f(double x) { return x; } };
template <> struct St<float, float> { __device__ static float f(float x) { return x; } };
template <> struct St<double, float> { __device__ static double f(float x) { return (double)x; } };
template <> struct St<df, float> { __device__ static df f(float x) { return mkdf(x, 0.f); } };
template <> struct St<df, double> { __device__ static df f(double x) { return Tr<df>::of(x); } };
template <class S, class C> __device__ __forceinline__ S st_as(C x) { return St<S, C>::f(x); }
