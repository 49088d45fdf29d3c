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

#include "engine.h"

using tt::XRange;
using tt::kXrBias;
using tt::kXrNonfinite;

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
  if (!(a.hi > 0.f)) return a.hi != a.hi ? a : mkdf(0.f, 0.f);  // NaN stays NaN
  float x = sqrt_seed(a.hi);
  float p, e; eft_two_prod(x, x, p, e);
  df res = sub(a, mkdf(p, e));
  float corr = __fmul_rn(res.hi, rcp_seed(__fmul_rn(2.f, x)));
  return df_norm(x, corr);
}
__device__ __forceinline__ bool is_pos(df a) { return a.hi > 0.f; }
__device__ __forceinline__ float fp32_lead(df a) { return a.hi; }
__device__ __forceinline__ float fp32_lead(float a) { return a; }
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
__device__ __forceinline__ double sqrt_(double a) { return a > 0.0 ? sqrt(a) : (a != a ? a : 0.0); }
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
__device__ __forceinline__ float sqrt_(float a) { return a > 0.f ? sqrtf(a) : (a != a ? a : 0.f); }
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

// ----------------------------------------------------------------------------
// The Householder reflector of one column (Alg. 6): panel part y with D = ||y||^2 and
// pivot entry R_jj.  alpha = -sign(R_jj) sqrt(R_jj^2 + D) becomes the new R_jj; with
// v = [R_jj - alpha; y] and t = ||v||^2 / 2 the reflector is I - v v^T / t.  Returns
// alpha, piv = R_jj - alpha and rt = 1 / t.
template <class C>
struct Refl {
  C alpha, piv, rt;
};
// Native FP64: the guard eps_FP of Alg. 6 (DBL_MIN) keeps t > 0 for a zero column.
__device__ __forceinline__ Refl<double> householder(double rjj, double D, double eps) {
  double t = fmac(rjj, rjj, D) + eps;
  double alpha = sqrt_(t + eps);
  if (rjj > 0.0) alpha = -alpha;
  t = fnmac(alpha, rjj, t);
  return {alpha, rjj - alpha, 1.0 / t};
}
// FP32 and float-float read their input shifted so that max |x| lies in [0.5, 1)
// (engine.h, XRange).  There an additive FLT_MIN would be a relative error of t for any
// column of norm below ~2^-39, and the reflector would no longer be orthogonal.  Instead a
// column with R_jj^2 + D < 2^-100 (norm below 2^-50 of the largest input entry) is left
// as it is: the reflector is the identity (rt = 0, alpha = R_jj), which drops at most
// 2^-50 max|x| of that column's remainder.
constexpr float kReflTiny = 7.8886090522101181e-31f;  // 2^-100
template <class C>
__device__ __forceinline__ Refl<C> householder_shifted(C rjj, C D) {
  C t = fmac(rjj, rjj, D);
  if (fp32_lead(t) < kReflTiny) return {rjj, Tr<C>::zero(), Tr<C>::zero()};
  C alpha = sqrt_(t);
  if (is_pos(rjj)) alpha = neg(alpha);
  t = fnmac(alpha, rjj, t);
  return {alpha, sub(rjj, alpha), rcp_(t)};
}
__device__ __forceinline__ Refl<float> householder(float rjj, float D, float) {
  return householder_shifted<float>(rjj, D);
}
__device__ __forceinline__ Refl<df> householder(df rjj, df D, df) {
  return householder_shifted<df>(rjj, D);
}

// A value of a matrix already scaled to max |a| in [0.5, 1), with entries below 2^-62 set
// to zero in float-float: their squares would leave FP32's normal range (the Jacobi
// sweeps compare products of column norms); they change no singular value by more than
// 2^-62 m of the largest entry.  FP64 and FP32 values are returned unchanged.
__device__ __forceinline__ df flush_tiny(df a) {
  return fabsf(a.hi) < 2.168404344971009e-19f ? mkdf(0.f, 0.f) : a;  // 2^-62
}
__device__ __forceinline__ double flush_tiny(double a) { return a; }
__device__ __forceinline__ float flush_tiny(float a) { return a; }

// df from an FP64 value times 2^-sh without FP64 instructions: hi = the scaled value cut
// to 24 significant bits, lo = the next 23 bits (47 bits kept).  A subnormal input is
// first scaled up exactly by 2^64 (one FP64 multiply, only on that rare path).  Scaled
// exponents below the normal FP32 range flush to zero, above it overflow to infinity;
// the caller picks sh so that neither happens to entries that matter (engine.h, XRange).
__device__ __forceinline__ df df_from_f64_sh(double x, int sh) {
  // branch-free (selects only), so that an unrolled run of loads and conversions keeps
  // its loads together
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e0 = (int)((b >> 52) & 0x7FF);
  const unsigned long long m0 = b & 0xFFFFFFFFFFFFFull;
  // a subnormal moves its leading bit to the implicit position (s = 0 for normal values)
  const int s = e0 == 0 ? __clzll((long long)m0) - 11 : 0;
  const unsigned long long mant = (m0 << s) & 0xFFFFFFFFFFFFFull;
  const int e = e0 == 0 ? 1 - s : e0;
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int fe = e - 1023 + 127 - sh;
  const float hi = __int_as_float((int)(sign | ((unsigned)(fe & 0xFF) << 23) | (unsigned)(mant >> 29)));
  // remaining 29 bits; keep the top 23 of them as an exact small integer
  const unsigned rem23 = (unsigned)((mant & 0x1FFFFFFFull) >> 6);
  const float f = __fsub_rn(__int_as_float((int)(0x4B000000u | rem23)), 8388608.0f);
  // value of one unit of rem23: 2^(e - 1023 - 52 + 6 - sh)
  const int se = e - 1069 + 127 - sh;
  const float scale = __int_as_float((se > 0 ? (se < 255 ? se : 254) : 0) << 23);
  float lo = se > 0 ? __fmul_rn(f, scale) : 0.f;
  lo = sign ? -lo : lo;
  // infinity stays infinity, NaN stays NaN; out of range: zero or infinity
  const float special = __int_as_float((int)(sign | 0x7F800000u | (m0 ? 0x400000u : 0u)));
  const float inf = __int_as_float((int)(sign | 0x7F800000u));
  const bool zero = (e0 == 0 && m0 == 0ull) || fe <= 0;
  const bool over = fe >= 255;
  float rh = e0 == 2047 ? special : (over ? inf : (zero ? 0.f : hi));
  float rl = (e0 == 2047 || over || zero) ? 0.f : lo;
  return mkdf(rh, rl);
}
__device__ __forceinline__ df df_from_f64_bits(double x) { return df_from_f64_sh(x, 0); }

// encoded exponent (engine.h, XRange) of an FP32 value, subnormals included: 0 for zero
__device__ __forceinline__ int f32_expo_enc(float x) {
  const unsigned b = __float_as_uint(x);
  const int e = (int)((b >> 23) & 0xFF);
  if (e == 255) return kXrNonfinite;
  if (e != 0) return e - 127 + kXrBias;
  if ((b << 1) == 0u) return 0;
  return (int)((__float_as_uint(x * 16777216.0f) >> 23) & 0xFF) - 127 - 24 + kXrBias;
}
__device__ __forceinline__ int expo_enc(float x) { return f32_expo_enc(x); }

// encoded exponent (engine.h, XRange) of an FP64 value, subnormals included: 0 for zero
__device__ __forceinline__ int f64_expo_enc(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 2047) return kXrNonfinite;
  if (e != 0) return e - 1023 + kXrBias;
  if ((b << 1) == 0ull) return 0;
  return (int)((__double_as_longlong(x * 18446744073709551616.0) >> 52) & 0x7FF) - 1023 - 64 +
         kXrBias;
}
__device__ __forceinline__ int expo_enc(double x) { return f64_expo_enc(x); }

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

// Entries below 2^-62 of 2^sh (the largest magnitude is in [2^(sh-1), 2^sh)) are read as
// zero: their squares and products would leave FP32's normal range, where a Householder
// reflector built from underflowed sums is no longer orthogonal.  Over n entries this
// changes X by at most sqrt(n) 2^-62 max|x| in the Frobenius norm (2^-47 max|x| for 2^30
// entries), below the float-float rounding of the decomposition.
constexpr int kXrFlush = 62;

// Reader of the input X of a level: the plain storage-to-compute conversion, except FP64
// read in float-float and FP32 read in FP32 or float-float, which are shifted by 2^-sh
// and record the largest exponent they met (two integer instructions per entry).
template <class C, class S>
struct XRead {
  int sh = 0;
  bool flush = false;
  unsigned efield = 0;
  __device__ __forceinline__ void set(int shift, bool fl) { sh = shift; flush = fl; }
  __device__ __forceinline__ C operator()(S x) { return Ld<C, S>::f(x); }
  __device__ __forceinline__ static int seen_of(unsigned) { return 0; }
};
template <>
struct XRead<df, double> {
  int sh = 0;
  bool flush = false;    // true once sh comes from the input's exponent range
  unsigned efield = 0;   // largest (hi word & 0x7FF00000) seen, i.e. the exponent field << 20
  // exponent fields [lo, lo + span] convert on the fast path: normal, not below the flush
  // threshold, and inside FP32's range after the shift
  int lo = 897;
  unsigned span = 1150 - 897;
  __device__ __forceinline__ void set(int shift, bool fl) {
    sh = shift;
    flush = fl;
    const int l = max(1, (fl ? 1023 - kXrFlush : 897) + shift);
    const int h = min(2046, 1150 + shift);
    lo = l;
    span = h >= l ? (unsigned)(h - l) : 0u;
    if (h < l) lo = 4096;  // nothing is fast
  }
  __device__ __forceinline__ df operator()(double x) {
    const unsigned hw = (unsigned)__double2hiint(x);
    const unsigned lw = (unsigned)__double2loint(x);
    const unsigned h = hw & 0x7FF00000u;
    efield = max(efield, h);
    const int e0 = (int)(h >> 20);
    if ((unsigned)(e0 - lo) <= span) {
      // the top 24 significant bits in hi, the next 23 in lo (as df_from_f64_sh)
      const int fe = e0 - 896 - sh;
      const float hi = __uint_as_float((hw & 0x80000000u) | ((unsigned)fe << 23) |
                                       ((hw & 0xFFFFFu) << 3) | (lw >> 29));
      const unsigned rem23 = (lw >> 6) & 0x7FFFFFu;
      const float f = __fsub_rn(__uint_as_float(0x4B000000u | rem23), 8388608.0f);
      const int se = fe - 46;
      float lof = __fmul_rn(f, __uint_as_float(se > 0 ? (unsigned)se << 23 : 0u));
      return mkdf(hi, (hw & 0x80000000u) ? -lof : lof);
    }
    // zero, subnormal, below the flush threshold, too large, infinity, NaN
    // floor(log2 |x|) < sh - kXrFlush: for a normal x its exponent field is below
    // 1023 + sh - kXrFlush; a subnormal x (field 0, |x| < 2^-1022) is below whenever
    // sh - kXrFlush > -1023 (otherwise the whole tensor is of subnormal size: kept)
    const bool tiny = flush && (e0 != 0 ? e0 < 1023 + sh - kXrFlush : sh - kXrFlush > -1023);
    return tiny ? mkdf(0.f, 0.f) : df_from_f64_sh(x, sh);
  }
  // encoded exponent (engine.h, XRange) of the largest field (subnormals count as zero:
  // only large entries can leave the safe window)
  __device__ __forceinline__ static int seen_of(unsigned ef) {
    const int f = (int)(ef >> 20);
    return f == 0 ? 0 : (f == 2047 ? kXrNonfinite : f - 1023 + kXrBias);
  }
};
// FP32 value times 2^-sh, exactly (exponent arithmetic); with `flush`, values below
// 2^(sh - kXrFlush) are read as zero (the same rule as for FP64 input)
__device__ __forceinline__ float f32_shift(float x, int sh, bool flush) {
  // branch-free (selects only); a subnormal is first scaled by 2^24 (exact)
  const unsigned b0 = __float_as_uint(x);
  const int e0 = (int)((b0 >> 23) & 0xFF);
  const bool sub = e0 == 0;
  const unsigned b = sub ? __float_as_uint(x * 16777216.0f) : b0;
  const int e = (int)((b >> 23) & 0xFF);
  const int shx = sub ? sh + 24 : sh;
  const int fe = e - shx;
  const float v = __uint_as_float((b & 0x807FFFFFu) | ((unsigned)(fe & 0xFF) << 23));
  const float inf = __uint_as_float((b & 0x80000000u) | 0x7F800000u);
  const bool zero = (b0 << 1) == 0u || fe <= 0 || (flush && e - 127 < shx - kXrFlush);
  return e0 == 255 ? x : (fe >= 255 ? inf : (zero ? 0.f : v));
}
template <>
struct XRead<float, float> {
  int sh = 0;
  bool flush = false;
  unsigned efield = 0;   // largest (bits & 0x7F800000) seen, i.e. the exponent field << 23
  int lo = 1;            // exponent fields [lo, lo + span]: shifted by subtracting sh << 23
  unsigned span = 253;
  __device__ __forceinline__ void set(int shift, bool fl) {
    sh = shift;
    flush = fl;
    const int l = max(1, (fl ? 127 - kXrFlush : 1) + shift);
    const int h = min(254, 254 + shift);
    lo = l;
    span = h >= l ? (unsigned)(h - l) : 0u;
    if (h < l) lo = 4096;
  }
  __device__ __forceinline__ float operator()(float x) {
    const unsigned b = __float_as_uint(x);
    const unsigned ef = b & 0x7F800000u;
    efield = max(efield, ef);
    if ((unsigned)((int)(ef >> 23) - lo) <= span) return __uint_as_float(b - ((unsigned)sh << 23));
    return f32_shift(x, sh, flush);
  }
  // encoded exponent (engine.h, XRange) of the largest field (subnormals count as zero)
  __device__ __forceinline__ static int seen_of(unsigned ef) {
    const int f = (int)(ef >> 23);
    return f == 0 ? 0 : (f == 255 ? kXrNonfinite : f - 127 + kXrBias);
  }
};
template <>
struct XRead<df, float> {
  XRead<float, float> r;
  int sh = 0;
  bool flush = false;
  unsigned efield = 0;
  __device__ __forceinline__ void set(int shift, bool fl) {
    sh = shift;
    flush = fl;
    r.set(shift, fl);
  }
  __device__ __forceinline__ df operator()(float x) {
    const float v = r(x);
    efield = r.efield;
    return mkdf(v, 0.f);
  }
  __device__ __forceinline__ static int seen_of(unsigned ef) { return XRead<float, float>::seen_of(ef); }
};
// Start of a level kernel that reads X through `rd`: false when this launch is the
// re-run of the first level and the first pass was fine (the kernel then returns).
template <class C, class S>
__device__ __forceinline__ bool xr_begin(const XRange* xr, int xfix, XRead<C, S>& rd) {
  if (!xr) return true;
  if (xfix && !xr->redo) return false;
  rd.set(xfix ? xr->k : tt::xr_shift_for(xr->sample), true);
  return true;
}
// End of such a kernel: the largest exponent of the first pass, one atomic per warp.
template <class C, class S>
__device__ __forceinline__ void xr_end(XRange* xr, int xfix, const XRead<C, S>& rd) {
  if (!xr || xfix) return;
  unsigned e = rd.efield;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if ((threadIdx.x & 31) == 0 && e) atomicMax(&xr->seen, XRead<C, S>::seen_of(e));
}
