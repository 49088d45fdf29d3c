// tsqr_blk.cu -- blocked TSQR level kernel of the native FP64 form (Sec. 3.2 panels with
// the reflectors of Alg. 6, applied block by block).
//
// A CTA folds a contiguous range of 128-row panels into one triangle R, like the
// column-owned kernel, but the m columns of a panel are taken in blocks of KB = 8:
//
//   1. the reflector chain of the block (Alg. 6, column by column) runs on the block's
//      own columns only: warp w < 4 owns columns j0 + w and j0 + w + 4 (PB / 32 rows per
//      lane) and publishes each reflector (pivot entry, 1/t, the panel part x in shared
//      memory) on an mbarrier; the owner of the next pivot column applies the current
//      pivot to it and publishes before it updates its other column, so the critical
//      path (one reflector per step) meets no other chain warp's FP64 work;
//   2. the block's eight reflectors H_i = I - rt_i v_i v_i^T, v_i = [piv_i e_{j0+i}; x_i],
//      act on the columns right of the block as one transformation (compact WY,
//      Schreiber & Van Loan 1989): with W = V^T C (W_ic = piv_i R_{j0+i,c} + x_i . P_c)
//      and z_i = rt_i (W_i - sum_{i'<i} (x_i' . x_i) z_i') row by row,
//          R_{j0+i,c} -= piv_i z_ic,   P_c -= X Z;
//   3. the two products with the panel, X^T [X | P_trailing] (K = PB rows) and X Z
//      (K = 8), run on the tensor cores (mma.sync bf16, FP32 accumulation) with
//      FP64-accurate Ozaki splitting (Ozaki, Ogita, Oishi, Rump 2012): every value
//      becomes the 56-bit fixed-point magnitude of x relative to its group's largest
//      exponent (a column over the panel's rows, or a row over the block's columns),
//      cut into seven unsigned bytes d_0..d_6 (exact in bf16; the sign rides on every
//      digit); the products of one level l = a + b <= 6 summed over <= 32 terms stay
//      below 2^24 and are exact in FP32, the level sums are gathered in integers and
//      combined into one FP64 value (levels above 6 are dropped: < 2^-55 of the
//      group scale).
//
// The FP64 pipe of this part runs one warp instruction per ~70 clocks per SM sub-partition,
// so the reflector chain (norms, dot products, square root and reciprocal) stays in FP64
// while the bulk of the multiply-adds (the trailing update, 7/8 of them for m = 64) moves
// to the tensor cores and the integer/FP32 pipes.  Every wait is bounded (kWaitCycles).
#include "ozaki.cuh"
#include "tsqr_col.cuh"

namespace tt {
namespace blk {

// Layouts: (MX = largest m, PB = rows per panel) = (64, 128) and (80, 96), both two CTAs
// per SM.  The chain holds PB / 32 rows per lane; the panel product takes PB / 16 k-steps.
constexpr int NW = 8;          // warps per CTA (two CTAs per SM)
constexpr int NT = NW * 32;
constexpr int KB = 8;          // reflectors per block
constexpr int NLV = 7;         // digit levels kept

// panel value (r, c) at r * MX + (c ^ swz(r)): conflict-free for a warp reading a column
// (lane -> row) and for the mma fragments of the panel product (lane -> (column, row pair))
__device__ __forceinline__ int swz(int r) { return ((r & 7) << 1) | ((r >> 3) & 1); }
template <int MX>
__device__ __forceinline__ int pix(int r, int c) { return r * MX + (c ^ swz(r)); }
// packed upper triangle of R, row-major
template <int MX>
__device__ __forceinline__ int rix(int i, int c) { return i * MX - (i * (i - 1)) / 2 + (c - i); }

template <int MX, int PB>
struct Smem {
  static constexpr int kMX = MX, kPB = PB;
  static constexpr bool kWide = false;
  double P[PB * MX];
  double R[MX * (MX + 1) / 2];
  double Z[KB * MX];   // W_ic, then z_ic in place (c = panel column)
  double G[KB * KB];   // G[i'][i] = x_i' . x_i
  double piv[MX];
  double rt[MX];
  int L1[NLV * MX * KB];  // level sums of X^T [X | P] (A row rho, column i)
  int colE[MX];           // largest biased exponent field of each panel column
  int zE[MX];             // ... of each column of Z
  unsigned long long bar[MX];
  int abort_flag;
};

// The wide layouts (80 < m <= 512): R is a packed triangle per CTA in global memory (an
// L2-resident slice of the level's scratch); the 8 rows of the block being factored are
// staged in shared memory (Rb, row i at i * MX), read at the block's start and written
// back at its end.  The panel product's level sums stay in each warp (a warp takes whole
// 16-row tiles over the panel's rows), so no shared level-sum table is needed.
template <int MX, int PB>
struct SmemW {
  static constexpr int kMX = MX, kPB = PB;
  static constexpr bool kWide = true;
  double P[PB * MX];
  double Rb[KB * MX];
  double Z[KB * MX];
  double G[KB * KB];
  double piv[MX];
  double rt[MX];
  int colE[MX];
  int zE[MX];
  unsigned long long bar[MX];
  int abort_flag;
};

// R_{i,c} of the CTA's triangle for a row i of the current block (first row j0)
template <int MX, int PB>
__device__ __forceinline__ double& Rref(Smem<MX, PB>& S, int i, int c, int) { return S.R[rix<MX>(i, c)]; }
template <int MX, int PB>
__device__ __forceinline__ double& Rref(SmemW<MX, PB>& S, int i, int c, int j0) { return S.Rb[(i - j0) * MX + c]; }

template <int MX, int PB>
__host__ __device__ constexpr size_t smem_bytes() { return MX > 80 ? sizeof(SmemW<MX, PB>) : sizeof(Smem<MX, PB>); }

// ---- FP64-accurate digits ------------------------------------------------------------
// u = floor(|x| 2^(1078 - em)) < 2^56 for |x| < 2^(em - 1022), as (hi: 24 bits, lo: 32 bits)
__device__ __forceinline__ void fx56(double x, int em, uint32_t& hi, uint32_t& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (e ? (1ull << 52) : 0ull);
  const int s = (e ? e : 1) - em + 3;  // u = M 2^s, s <= 3
  const unsigned long long u = s >= 0 ? (M << s) : (s > -64 ? (M >> -s) : 0ull);
  hi = (uint32_t)(u >> 32);
  lo = (uint32_t)u;
}
// byte k (0..3) of w as an FP32 integer 0..255 (2^23 + n with its 2^23 taken away)
template <int K>
__device__ __forceinline__ uint32_t dig(uint32_t w) {
  return __float_as_uint(__fadd_rn(__uint_as_float(__byte_perm(w, 0x4B000000u, 0x7650u | K)), -8388608.f));
}
// bf16 pair (low half: value a, high half: value b) of the seven digits of two values
__device__ __forceinline__ void digits2(double a, int ema, double b, int emb, uint32_t (&d)[NLV]) {
  uint32_t ha, la, hb, lb;
  fx56(a, ema, ha, la);
  fx56(b, emb, hb, lb);
  const uint32_t sg = ((uint32_t)((unsigned long long)__double_as_longlong(a) >> 63) << 15) |
                      ((uint32_t)((unsigned long long)__double_as_longlong(b) >> 63) << 31);
  d[0] = __byte_perm(dig<2>(ha), dig<2>(hb), 0x7632) | sg;
  d[1] = __byte_perm(dig<1>(ha), dig<1>(hb), 0x7632) | sg;
  d[2] = __byte_perm(dig<0>(ha), dig<0>(hb), 0x7632) | sg;
  d[3] = __byte_perm(dig<3>(la), dig<3>(lb), 0x7632) | sg;
  d[4] = __byte_perm(dig<2>(la), dig<2>(lb), 0x7632) | sg;
  d[5] = __byte_perm(dig<1>(la), dig<1>(lb), 0x7632) | sg;
  d[6] = __byte_perm(dig<0>(la), dig<0>(lb), 0x7632) | sg;
}
__device__ __forceinline__ int efield(double x) {
  return (int)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF);
}

__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void mma1688(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(b0));
}

// 2^e as a product of two exact powers of two (0 far below the normal range)
__device__ __forceinline__ double pow2_split(double v, int e) {
  const int e1 = e / 2, e2 = e - e / 2;
  const double p1 = e1 < -1022 ? 0.0 : __longlong_as_double((long long)(e1 + 1023) << 52);
  const double p2 = e2 < -1022 ? 0.0 : __longlong_as_double((long long)(e2 + 1023) << 52);
  return v * p1 * p2;
}
// x 2^e for an FP64 x: the exponent field moved by e when the result stays normal, else
// two exact multiplies
__device__ __forceinline__ double scale2(double x, int e) {
  const long long b = __double_as_longlong(x);
  const int f = (int)((b >> 52) & 0x7FF);
  if (f != 0 && f + e >= 1 && f + e <= 2046) return __longlong_as_double(b + ((long long)e << 52));
  return pow2_split(x, e);
}


// ---- reflector scalars: FP32 seeds refined by FP64 Newton steps ----------------------------
// A dependent FP64 operation costs ~64 clocks on this part and the library's square root and
// reciprocal ~10 and ~6 of them; the chain needs one of each per column.  Here the seed is
// the FP32 approximation (rsqrt.approx / rcp.approx, |error| < 2^-21) of the value scaled
// into [1, 4) by an exact power of two, and Newton's iteration in FP64 refines it:
// sqrt: s <- s + (T - s^2) h with h ~ 1/(2 sqrt T) (twice: error ~2^-66 before rounding);
// reciprocal: r <- r (1 + q + q^2), q = 1 - t r (error ~q^3).  Measured against CUDA's
// sqrt and division on 2^20 values spread over 2^+-1000: at most 1.4 and 2.0 units in the
// last place.  Zero, subnormal, infinite and NaN arguments take the library functions.
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long e = (u >> 23) & 0xFF, mnt = u & 0x7FFFFF;
  return __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) | ((e - 127 + 1023) << 52) | (mnt << 29)));
}
__device__ __forceinline__ double sqrt_fast(double T) {
  const long long b = __double_as_longlong(T);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0 || e == 0x7FF) return sqrt(T);
  const int k = (e - 1023) >> 1;
  const long long mb = b - ((long long)(2 * k) << 52);  // T 2^-2k in [1, 4)
  const float f = __uint_as_float((unsigned)((((mb >> 52) & 0x7FF) - 1023 + 127) << 23) | (unsigned)((mb >> 29) & 0x7FFFFF));
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(f));
  const double s0 = f2d_exact(f * y), h0 = f2d_exact(0.5f * y);
  const double s = __longlong_as_double(__double_as_longlong(s0) + ((long long)k << 52));
  const double h = __longlong_as_double(__double_as_longlong(h0) - ((long long)k << 52));
  double r = fma(-s, s, T);
  const double s1 = fma(r, h, s);
  r = fma(-s1, s1, T);
  return fma(r, h, s1);
}
__device__ __forceinline__ double rcp_fast(double t) {
  const long long b = __double_as_longlong(t);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e <= 1 || e >= 0x7FE) return 1.0 / t;
  const int k = e - 1023;
  const long long mb = b - ((long long)k << 52);  // |t| 2^-k in [1, 2)
  const float f = __uint_as_float((unsigned)(127u << 23) | (unsigned)((mb >> 29) & 0x7FFFFF));
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(f));
  double r = __longlong_as_double(__double_as_longlong(f2d_exact(y)) - ((long long)k << 52));
  if (b < 0) r = -r;
  const double q = fma(-t, r, 1.0);
  return fma(r, fma(q, q, q), r);
}
__device__ __forceinline__ Refl<double> householder_fast(double rjj, double D, double eps) {
  double t = fma(rjj, rjj, D) + eps;
  double alpha = sqrt_fast(t + eps);
  if (rjj > 0.0) alpha = -alpha;
  t = fma(-alpha, rjj, t);
  return {alpha, rjj - alpha, rcp_fast(t)};
}

// ---- phase 1: the reflector chain of one block ---------------------------------------
// the chain on four warps: warp w owns columns j0 + w (A) and j0 + w + 4 (B).  The owner of
// the next pivot column applies the current pivot to that column and publishes its reflector
// before it updates its other column, so the critical path meets no other chain warp's
// FP64 work on its sub-partition.
template <class SM>
__device__ __forceinline__ void apply_piv(SM& S, double (&a)[SM::kPB / 32], const double (&x)[SM::kPB / 32],
                                          double piv, double rt, int jp, int j, int j0, int lane) {
  constexpr int RPL = SM::kPB / 32;
  double d0 = 0.0, d1 = 0.0;
#pragma unroll
  for (int q = 0; q + 1 < RPL; q += 2) {
    d0 = fma(x[q], a[q], d0);
    d1 = fma(x[q + 1], a[q + 1], d1);
  }
  if constexpr (RPL % 2) d0 = fma(x[RPL - 1], a[RPL - 1], d0);
  const double d = colk::warp_allsum<double>(d0 + d1);
  double& rr = Rref(S, jp, j, j0);
  const double r = rr;
  const double c = fma(piv, r, d) * rt;
  if (lane == 0) rr = fma(-c, piv, r);
#pragma unroll
  for (int q = 0; q < RPL; ++q) a[q] = fma(-c, x[q], a[q]);
}
template <class SM>
__device__ __forceinline__ void publish_col(SM& S, double (&a)[SM::kPB / 32], int j, int j0, int lane) {
  constexpr int RPL = SM::kPB / 32, MX = SM::kMX;
  double n0 = 0.0, n1 = 0.0;
#pragma unroll
  for (int q = 0; q + 1 < RPL; q += 2) {
    n0 = fma(a[q], a[q], n0);
    n1 = fma(a[q + 1], a[q + 1], n1);
  }
  if constexpr (RPL % 2) n0 = fma(a[RPL - 1], a[RPL - 1], n0);
  const double D = colk::warp_allsum<double>(n0 + n1);
  double& rjj = Rref(S, j, j, j0);
  const Refl<double> h = householder_fast(rjj, D, Tr<double>::eps());
#pragma unroll
  for (int q = 0; q < RPL; ++q) S.P[pix<MX>(lane + 32 * q, j)] = a[q];
  if (lane == 0) {
    S.piv[j] = h.piv;
    S.rt[j] = h.rt;
    rjj = h.alpha;
  }
  __syncwarp();
  if (lane == 0) colk::mbar_arrive(reinterpret_cast<uint64_t*>(&S.bar[j]));
  // the column's exponent (read by the tensor-core phases, after the block's barrier)
  int em = 0;
#pragma unroll
  for (int q = 0; q < RPL; ++q) em = max(em, efield(a[q]));
#pragma unroll
  for (int o = 16; o; o >>= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
  if (lane == 0) S.colE[j] = em;
}
template <class SM>
__device__ __forceinline__ bool chain(SM& S, int j0, int kb, int w, int lane, uint32_t par, int* status) {
  constexpr int RPL = SM::kPB / 32, MX = SM::kMX;
  const int ja = j0 + w, jb = j0 + w + 4;
  const bool hasb = w + 4 < kb;
  double a[RPL], b[RPL];
#pragma unroll
  for (int q = 0; q < RPL; ++q) {
    a[q] = S.P[pix<MX>(lane + 32 * q, ja)];
    b[q] = hasb ? S.P[pix<MX>(lane + 32 * q, jb)] : 0.0;
  }
  if (w == 0) publish_col(S, a, ja, j0, lane);
  const int last = hasb ? w + 4 : w;  // pivots needed: 0 .. last-1
  for (int jj = 0; jj < last; ++jj) {
    const int jp = j0 + jj;
    if (!colk::mbar_wait(reinterpret_cast<uint64_t*>(&S.bar[jp]), par)) {
      if (lane == 0) {
        if (status) atomicOr(status, DEV_ERR_TIMEOUT);
        *reinterpret_cast<volatile int*>(&S.abort_flag) = 1;
      }
      return false;
    }
    double x[RPL];
#pragma unroll
    for (int q = 0; q < RPL; ++q) x[q] = S.P[pix<MX>(lane + 32 * q, jp)];
    const double piv = S.piv[jp], rt = S.rt[jp];
    if (jj < w) {
      apply_piv(S, a, x, piv, rt, jp, ja, j0, lane);
      if (jj == w - 1) publish_col(S, a, ja, j0, lane);
    }
    if (hasb) {
      apply_piv(S, b, x, piv, rt, jp, jb, j0, lane);
      if (jj == w + 3) publish_col(S, b, jb, j0, lane);
    }
  }
  return true;
}

// ---- phase 2: level sums of X^T [X | P_t] on the tensor cores ----------------------------
// A = the panel's columns j0 .. m-1 as rows (rho), B = X (columns j0 .. j0+7), K = panel rows.
// Warp w takes m-tile w % mt and the k-steps w / mt, + nkc, ...  (at most four: the sums of
// one level over two k-steps stay below 2^24, so the FP32 accumulators are emptied into
// integers every two k-steps)
template <int MX, int PB>
__device__ __forceinline__ void prod1(Smem<MX, PB>& S, int j0, int m, int w, int lane) {
  const int g = lane >> 2, t = lane & 3;
  const int M1 = m - j0;
  const int mt = (M1 + 15) >> 4;
  const int nkc = (PB / 16) / mt;
  if (w >= mt * nkc) return;
  const int tile = w % mt, chunk = w / mt;
  const int rho0 = 16 * tile + g, rho1 = rho0 + 8;
  const bool in0 = rho0 < M1, in1 = rho1 < M1;
  const int ca0 = j0 + rho0, ca1 = j0 + rho1;
  const int ema0 = in0 ? max(S.colE[ca0], 1) : 1, ema1 = in1 ? max(S.colE[ca1], 1) : 1;
  const int cb = j0 + g;
  const int emb = max(S.colE[cb], 1);
  int ia[NLV][4];
  float acc[NLV][4];
#pragma unroll
  for (int l = 0; l < NLV; ++l)
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      ia[l][h] = 0;
      acc[l][h] = 0.f;
    }
  int n = 0;
  for (int kk = chunk; kk < PB / 16; kk += nkc) {
    const int r0 = 16 * kk + 2 * t;
    uint32_t A[NLV][4], B[NLV][2];
    {
      uint32_t d[NLV];
      const double v00 = in0 ? S.P[pix<MX>(r0, ca0)] : 0.0, v01 = in0 ? S.P[pix<MX>(r0 + 1, ca0)] : 0.0;
      const double v10 = in1 ? S.P[pix<MX>(r0, ca1)] : 0.0, v11 = in1 ? S.P[pix<MX>(r0 + 1, ca1)] : 0.0;
      const double v20 = in0 ? S.P[pix<MX>(r0 + 8, ca0)] : 0.0, v21 = in0 ? S.P[pix<MX>(r0 + 9, ca0)] : 0.0;
      const double v30 = in1 ? S.P[pix<MX>(r0 + 8, ca1)] : 0.0, v31 = in1 ? S.P[pix<MX>(r0 + 9, ca1)] : 0.0;
      digits2(v00, ema0, v01, ema0, d);
#pragma unroll
      for (int a = 0; a < NLV; ++a) A[a][0] = d[a];
      digits2(v10, ema1, v11, ema1, d);
#pragma unroll
      for (int a = 0; a < NLV; ++a) A[a][1] = d[a];
      digits2(v20, ema0, v21, ema0, d);
#pragma unroll
      for (int a = 0; a < NLV; ++a) A[a][2] = d[a];
      digits2(v30, ema1, v31, ema1, d);
#pragma unroll
      for (int a = 0; a < NLV; ++a) A[a][3] = d[a];
      digits2(S.P[pix<MX>(r0, cb)], emb, S.P[pix<MX>(r0 + 1, cb)], emb, d);
#pragma unroll
      for (int b = 0; b < NLV; ++b) B[b][0] = d[b];
      digits2(S.P[pix<MX>(r0 + 8, cb)], emb, S.P[pix<MX>(r0 + 9, cb)], emb, d);
#pragma unroll
      for (int b = 0; b < NLV; ++b) B[b][1] = d[b];
    }
#pragma unroll
    for (int a = 0; a < NLV; ++a)
#pragma unroll
      for (int b = 0; a + b < NLV; ++b) mma16816(acc[a + b], A[a], B[b][0], B[b][1]);
    if (++n == 2) {
      n = 0;
#pragma unroll
      for (int l = 0; l < NLV; ++l)
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          ia[l][h] += __float2int_rn(acc[l][h]);
          acc[l][h] = 0.f;
        }
    }
  }
#pragma unroll
  for (int l = 0; l < NLV; ++l)
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      ia[l][h] += __float2int_rn(acc[l][h]);
      const int rho = (h >> 1) ? rho1 : rho0;
      const int i = 2 * t + (h & 1);
      if (rho < M1) atomicAdd(&S.L1[(l * MX + rho) * KB + i], ia[l][h]);
    }
}

// ---- phase 3: G, W, Z and the R rows of the block ---------------------------------------
__device__ __forceinline__ double level_value(const int (&s)[NLV], int e) {
  long long shi = 0, slo = 0;
#pragma unroll
  for (int l = 0; l < 4; ++l) shi = shi * 256 + s[l];
#pragma unroll
  for (int l = 4; l < NLV; ++l) slo = slo * 256 + s[l];
  return pow2_split(fma((double)slo, 0x1p-24, (double)shi), e);
}

// an FP32 integer value |x| < 2^22 as an int: 1.5 2^23 + x has x in its low mantissa bits
__device__ __forceinline__ int f2i_small(float x) {
  return __float_as_int(__fadd_rn(x, 12582912.f)) - 0x4B400000;
}

// ---- phase 4: P_t -= X Z on the tensor cores ---------------------------------------------
// warp w takes panel rows 16w .. 16w+15; K = 8, one mma per digit pair.  The sum runs over
// the block's columns, whose scales may differ by any power of two, so the product is taken
// as (X D^-1)(D Z) with D = diag(2^(E_i - 1023)), E_i the exponent of column i of X (exact
// scalings, folded into the digit exponents): A = X D^-1 with one exponent per row, B = D Z
// with one exponent per column (zE, formed with the same scaling)
__device__ __forceinline__ int ef1(double x) { return x != 0.0 ? max(efield(x), 1) : 0; }
template <class SM>
__device__ __forceinline__ void prod2(SM& S, int j0, int m, int tile, int ntb, int nte, int lane) {
  constexpr int MX = SM::kMX;
  const int g = lane >> 2, t = lane & 3;
  const int ra = 16 * tile + g, rb = ra + 8;
  const int E0 = max(S.colE[j0 + 2 * t], 1), E1 = max(S.colE[j0 + 2 * t + 1], 1);
  const double xa0 = S.P[pix<MX>(ra, j0 + 2 * t)], xa1 = S.P[pix<MX>(ra, j0 + 2 * t + 1)];
  const double xb0 = S.P[pix<MX>(rb, j0 + 2 * t)], xb1 = S.P[pix<MX>(rb, j0 + 2 * t + 1)];
  // exponents of the rows of X D^-1
  auto fa = [](double x, int E) { return x != 0.0 ? ef1(x) - E + 1023 : 0; };
  int ea = max(fa(xa0, E0), fa(xa1, E1)), eb = max(fa(xb0, E0), fa(xb1, E1));
#pragma unroll
  for (int o = 1; o < 4; o <<= 1) {
    ea = max(ea, __shfl_xor_sync(0xffffffffu, ea, o));
    eb = max(eb, __shfl_xor_sync(0xffffffffu, eb, o));
  }
  ea = max(ea, 1);
  eb = max(eb, 1);
  uint32_t Aa[NLV], Ab[NLV];
  digits2(xa0, ea + E0 - 1023, xa1, ea + E1 - 1023, Aa);
  digits2(xb0, eb + E0 - 1023, xb1, eb + E1 - 1023, Ab);
  // n-tiles ntb .. nte-1 of the columns right of the block
  const int cend = min(m, j0 + KB + 8 * nte);
  for (int cn0 = j0 + KB + 8 * ntb; cn0 < cend; cn0 += 8) {
    const int cn = cn0 + g;  // B column of this lane
    uint32_t Bd[NLV];
    {
      const bool in = cn < m;
      const int ez = in ? max(S.zE[cn], 1) : 1;
      digits2(in ? S.Z[(2 * t) * MX + cn] : 0.0, ez - E0 + 1023, in ? S.Z[(2 * t + 1) * MX + cn] : 0.0,
              ez - E1 + 1023, Bd);
    }
    float acc[NLV][4];
#pragma unroll
    for (int l = 0; l < NLV; ++l) acc[l][0] = acc[l][1] = acc[l][2] = acc[l][3] = 0.f;
#pragma unroll
    for (int a = 0; a < NLV; ++a)
#pragma unroll
      for (int b = 0; a + b < NLV; ++b) mma1688(acc[a + b], Aa[a], Ab[a], Bd[b]);
    // outputs (ra | rb, cn0 + 2t + {0, 1}): P -= 2^(e_row + e_z - 2084) (shi + slo 2^-24),
    // formed as an integer T = shi 2^16 + (slo >> 8) < 2^62 (the bits dropped are below
    // 2^-56 of one digit product's scale) and converted once
    int emx[2] = {0, 0};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int c = cn0 + 2 * t + (h & 1);
      const int row = (h >> 1) ? rb : ra;
      if (c < m) {
        long long shi = 0, slo = 0;
#pragma unroll
        for (int l = 0; l < 4; ++l) shi = shi * 256 + f2i_small(acc[l][h]);
#pragma unroll
        for (int l = 4; l < NLV; ++l) slo = slo * 256 + f2i_small(acc[l][h]);
        const long long T = shi * 65536 + (slo >> 8);
        const int e = ((h >> 1) ? eb : ea) + max(S.zE[c], 1) - 2084 - 16;
        const double y = scale2(__ll2double_rn(T), e);
        const int ix = pix<MX>(row, c);
        const double v = S.P[ix] - y;
        S.P[ix] = v;
        emx[h & 1] = max(emx[h & 1], efield(v));
      }
    }
    // the column maxima of the updated values (lanes with the same t hold the same columns)
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
      emx[0] = max(emx[0], __shfl_xor_sync(0xffffffffu, emx[0], o));
      emx[1] = max(emx[1], __shfl_xor_sync(0xffffffffu, emx[1], o));
    }
    if (g == 0) {
      const int c = cn0 + 2 * t;
      if (c < m) atomicMax(&S.colE[c], emx[0]);
      if (c + 1 < m) atomicMax(&S.colE[c + 1], emx[1]);
    }
  }
}


// ---- the wide layouts' panel product: a warp takes whole 16-row tiles of A over all PB
// rows (PB / 16 k-steps; the level sums of two k-steps stay below 2^24 in FP32 and are
// emptied into integers), and forms G and W from its own sums
template <int MX, int PB>
__device__ __forceinline__ void prod1w(SmemW<MX, PB>& S, int j0, int m, int w, int lane) {
  const int g = lane >> 2, t = lane & 3;
  const int M1 = m - j0;
  const int mt = (M1 + 15) >> 4;
  const int cb = j0 + g;
  const int emb = max(S.colE[cb], 1);
  for (int tile = w; tile < mt; tile += NW) {
    const int rho0 = 16 * tile + g, rho1 = rho0 + 8;
    const bool in0 = rho0 < M1, in1 = rho1 < M1;
    const int ca0 = j0 + rho0, ca1 = j0 + rho1;
    const int ema0 = in0 ? max(S.colE[ca0], 1) : 1, ema1 = in1 ? max(S.colE[ca1], 1) : 1;
    int ia[NLV][4];
    float acc[NLV][4];
#pragma unroll
    for (int l = 0; l < NLV; ++l)
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        ia[l][h] = 0;
        acc[l][h] = 0.f;
      }
#pragma unroll 1
    for (int kk = 0; kk < PB / 16; ++kk) {
      const int r0 = 16 * kk + 2 * t;
      uint32_t A[NLV][4], B[NLV][2];
      {
        uint32_t d[NLV];
        const double v00 = in0 ? S.P[pix<MX>(r0, ca0)] : 0.0, v01 = in0 ? S.P[pix<MX>(r0 + 1, ca0)] : 0.0;
        const double v10 = in1 ? S.P[pix<MX>(r0, ca1)] : 0.0, v11 = in1 ? S.P[pix<MX>(r0 + 1, ca1)] : 0.0;
        const double v20 = in0 ? S.P[pix<MX>(r0 + 8, ca0)] : 0.0, v21 = in0 ? S.P[pix<MX>(r0 + 9, ca0)] : 0.0;
        const double v30 = in1 ? S.P[pix<MX>(r0 + 8, ca1)] : 0.0, v31 = in1 ? S.P[pix<MX>(r0 + 9, ca1)] : 0.0;
        digits2(v00, ema0, v01, ema0, d);
#pragma unroll
        for (int a = 0; a < NLV; ++a) A[a][0] = d[a];
        digits2(v10, ema1, v11, ema1, d);
#pragma unroll
        for (int a = 0; a < NLV; ++a) A[a][1] = d[a];
        digits2(v20, ema0, v21, ema0, d);
#pragma unroll
        for (int a = 0; a < NLV; ++a) A[a][2] = d[a];
        digits2(v30, ema1, v31, ema1, d);
#pragma unroll
        for (int a = 0; a < NLV; ++a) A[a][3] = d[a];
        digits2(S.P[pix<MX>(r0, cb)], emb, S.P[pix<MX>(r0 + 1, cb)], emb, d);
#pragma unroll
        for (int b = 0; b < NLV; ++b) B[b][0] = d[b];
        digits2(S.P[pix<MX>(r0 + 8, cb)], emb, S.P[pix<MX>(r0 + 9, cb)], emb, d);
#pragma unroll
        for (int b = 0; b < NLV; ++b) B[b][1] = d[b];
      }
#pragma unroll
      for (int a = 0; a < NLV; ++a)
#pragma unroll
        for (int b = 0; a + b < NLV; ++b) mma16816(acc[a + b], A[a], B[b][0], B[b][1]);
      if (kk & 1) {
#pragma unroll
        for (int l = 0; l < NLV; ++l)
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            ia[l][h] += __float2int_rn(acc[l][h]);
            acc[l][h] = 0.f;
          }
      }
    }
    // G (rho < 8) and W (rho >= 8): the level sums of this tile's outputs
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int rho = (h >> 1) ? rho1 : rho0;
      const int i = 2 * t + (h & 1);
      if (rho >= M1) continue;
      int sl[NLV];
#pragma unroll
      for (int l = 0; l < NLV; ++l) sl[l] = ia[l][h] + __float2int_rn(acc[l][h]);
      const double val = level_value(sl, max(S.colE[j0 + rho], 1) + max(S.colE[j0 + i], 1) - 2084);
      if (rho < KB) S.G[rho * KB + i] = val;
      else S.Z[i * MX + j0 + rho] = fma(S.piv[j0 + i], S.Rb[i * MX + j0 + rho], val);
    }
  }
}

}  // namespace blk

// R packed as in the column-owned kernel's output: block blockIdx.x of the stacked R's
template <int MX, int PB, class RO>
__global__ void __launch_bounds__(blk::NT, 2)
k_tsqr_blk(const double* __restrict__ W, int64_t rows, int64_t ld, const int* __restrict__ m_ptr,
           int m_val, int mmax, RO* __restrict__ Rout, int64_t ldR, int mb, int64_t npanels,
           int* status) {
  using namespace blk;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int RPL = PB / 32;
  Smem<MX, PB>& S = *reinterpret_cast<Smem<MX, PB>*>(smem_raw);
  const int m = m_ptr ? *m_ptr : m_val;
  if (m < 1 || m > MX || m > mmax || m > mb || blockDim.x != NT) {
    if (threadIdx.x == 0 && status) atomicOr(status, DEV_ERR_SHAPE);
    return;
  }
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  for (int i = tid; i < MX * (MX + 1) / 2; i += NT) S.R[i] = 0.0;
  for (int i = tid; i < NLV * MX * KB; i += NT) S.L1[i] = 0;
  for (int i = tid; i < MX; i += NT) colk::mbar_init(reinterpret_cast<uint64_t*>(&S.bar[i]), 1);
  if (tid == 0) S.abort_flag = 0;
  __syncthreads();
  const int64_t p0 = (int64_t)blockIdx.x * npanels / gridDim.x;
  const int64_t p1 = (int64_t)(blockIdx.x + 1) * npanels / gridDim.x;
  bool ok = true;
  for (int64_t p = p0; p < p1 && ok; ++p) {
    const uint32_t par = (uint32_t)((p - p0) & 1);
    // the panel: warp w loads columns w, w + 8, ... (all loads first, then the stores)
    {
      double v[MX / NW][RPL];
#pragma unroll
      for (int s = 0; s < MX / NW; ++s) {
        const int c = w + NW * s;
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
          const int64_t row = p * PB + lane + 32 * q;
          v[s][q] = (c < m && row < rows) ? W[row + (int64_t)c * ld] : 0.0;
        }
      }
#pragma unroll
      for (int s = 0; s < MX / NW; ++s) {
        const int c = w + NW * s;
        if (c < m) {
          int em = 0;
#pragma unroll
          for (int q = 0; q < RPL; ++q) {
            S.P[pix<MX>(lane + 32 * q, c)] = v[s][q];
            em = max(em, efield(v[s][q]));
          }
#pragma unroll
          for (int o = 16; o; o >>= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
          if (lane == 0) S.colE[c] = em;
        }
      }
      // warm L2 with this CTA's next panel (one request per 128-byte line)
      if (p + 1 < p1 && (lane & 15) == 0) {
#pragma unroll
        for (int s = 0; s < MX / NW; ++s) {
          const int c = w + NW * s;
#pragma unroll
          for (int q = 0; q < RPL; ++q) {
            const int64_t row = (p + 1) * PB + lane + 32 * q;
            if (c < m && row < rows) asm volatile("prefetch.global.L2 [%0];" ::"l"(W + row + (int64_t)c * ld));
          }
        }
      }
    }
    __syncthreads();
    if (w < 4 && w < min(KB, m)) chain(S, 0, min(KB, m), w, lane, par, status);
    __syncthreads();
    for (int j0 = 0;; j0 += KB) {
      if (*reinterpret_cast<volatile int*>(&S.abort_flag)) {
        ok = false;
        break;
      }
      if (j0 + KB >= m) break;  // no columns right of the last block
      prod1(S, j0, m, w, lane);
      __syncthreads();
      // G (rho < 8) and W (rho >= 8) from the level sums; the sums are cleared for the next block
      const int M1 = m - j0;
      for (int idx = tid; idx < M1 * KB; idx += NT) {
        const int rho = idx / KB, i = idx % KB;
        int s[NLV];
#pragma unroll
        for (int l = 0; l < NLV; ++l) {
          s[l] = S.L1[(l * MX + rho) * KB + i];
          S.L1[(l * MX + rho) * KB + i] = 0;
        }
        const double val = level_value(s, max(S.colE[j0 + rho], 1) + max(S.colE[j0 + i], 1) - 2084);
        if (rho < KB) S.G[rho * KB + i] = val;
        else S.Z[i * MX + j0 + rho] = fma(S.piv[j0 + i], S.R[rix<MX>(j0 + i, j0 + rho)], val);
      }
      __syncthreads();
      // Z row by row per column (z_i = rt_i (W_i - sum_{i'<i} G_i'i z_i')), the block's R rows;
      // zE = the exponent of column c of D Z (D as in prod2)
      for (int c = j0 + KB + tid; c < m; c += NT) {
        double z[KB];
        int ez = 0;
#pragma unroll
        for (int i = 0; i < KB; ++i) {
          double acc = S.Z[i * MX + c];
#pragma unroll
          for (int q = 0; q < i; ++q) acc = fma(-S.G[q * KB + i], z[q], acc);
          z[i] = acc * S.rt[j0 + i];
          S.Z[i * MX + c] = z[i];
          const int ri = rix<MX>(j0 + i, c);
          S.R[ri] = fma(-S.piv[j0 + i], z[i], S.R[ri]);
          if (z[i] != 0.0) ez = max(ez, ef1(z[i]) + max(S.colE[j0 + i], 1) - 1023);
        }
        S.zE[c] = ez;
        S.colE[c] = 0;  // recomputed from the updated panel values
      }
      __syncthreads();
      // P -= X Z: first the next block's columns (one n-tile, a 16-row m-tile per warp),
      // then the next block's reflector chain (warps 0-3) runs beside the rest of the
      // update (warps 4-7; disjoint columns of P, colE and R)
      if (w < PB / 16) prod2(S, j0, m, w, 0, 1, lane);
      __syncthreads();
      const int j1 = j0 + KB, kb1 = min(KB, m - j1);
      if (w < 4) {
        if (w < kb1) chain(S, j1, kb1, w, lane, par, status);
      } else {
        for (int tile = w - 4; tile < PB / 16; tile += 4) prod2(S, j0, m, tile, 1, MX / 8, lane);
      }
      __syncthreads();
    }
  }
  __syncthreads();
  if (*reinterpret_cast<volatile int*>(&S.abort_flag)) return;
  for (int idx = tid; idx < mb * m; idx += NT) {
    const int i = idx % mb, k = idx / mb;
    const double v = (i < m && i <= k) ? S.R[blk::rix<MX>(i, k)] : 0.0;
    Rout[(int64_t)blockIdx.x * mb + i + (int64_t)k * ldR] = st_as<RO>(v);
  }
}


// The wide layouts: R in the global slice Rg (packed upper triangle per CTA).
template <int MX, int PB>
__global__ void __launch_bounds__(blk::NT, (MX <= 256 ? 2 : 1))
k_tsqr_blkw(const double* __restrict__ W, int64_t rows, int64_t ld, const int* __restrict__ m_ptr,
            int m_val, int mmax, double* __restrict__ Rout, int64_t ldR, int mb, int64_t npanels,
            double* __restrict__ Rscr, int* status) {
  using namespace blk;
  constexpr int RPL = PB / 32, NMT = PB / 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SmemW<MX, PB>& S = *reinterpret_cast<SmemW<MX, PB>*>(smem_raw);
  const int m = m_ptr ? *m_ptr : m_val;
  if (m < 1 || m > MX || m > mmax || m > mb || blockDim.x != NT) {
    if (threadIdx.x == 0 && status) atomicOr(status, DEV_ERR_SHAPE);
    return;
  }
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  double* Rg = Rscr + (size_t)blockIdx.x * ((size_t)MX * (MX + 1) / 2);
  for (int i = tid; i < MX * (MX + 1) / 2; i += NT) Rg[i] = 0.0;
  for (int i = tid; i < MX; i += NT) colk::mbar_init(reinterpret_cast<uint64_t*>(&S.bar[i]), 1);
  if (tid == 0) S.abort_flag = 0;
  __syncthreads();
  // the block's rows of R between the global slice and shared memory
  auto stage_in = [&](int j0, int tl, int nthr) {
    const int kb = min(KB, m - j0);
    for (int idx = tl; idx < kb * MX; idx += nthr) {
      const int i = idx / MX, c = idx % MX;
      if (c >= j0 + i && c < m) S.Rb[i * MX + c] = Rg[rix<MX>(j0 + i, c)];
    }
  };
  auto stage_out = [&](int j0) {
    const int kb = min(KB, m - j0);
    for (int idx = tid; idx < kb * MX; idx += NT) {
      const int i = idx / MX, c = idx % MX;
      if (c >= j0 + i && c < m) Rg[rix<MX>(j0 + i, c)] = S.Rb[i * MX + c];
    }
  };
  const int64_t p0 = (int64_t)blockIdx.x * npanels / gridDim.x;
  const int64_t p1 = (int64_t)(blockIdx.x + 1) * npanels / gridDim.x;
  bool ok = true;
  for (int64_t p = p0; p < p1 && ok; ++p) {
    const uint32_t par = (uint32_t)((p - p0) & 1);
    // the panel, 8 columns per warp at a time (all loads of a group first)
    for (int c0 = 0; c0 < m; c0 += 8 * NW) {
      double v[8][RPL];
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int c = c0 + w + NW * s;
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
          const int64_t row = p * PB + lane + 32 * q;
          v[s][q] = (c < m && row < rows) ? W[row + (int64_t)c * ld] : 0.0;
        }
      }
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int c = c0 + w + NW * s;
        if (c < m) {
          int em = 0;
#pragma unroll
          for (int q = 0; q < RPL; ++q) {
            S.P[pix<MX>(lane + 32 * q, c)] = v[s][q];
            em = max(em, efield(v[s][q]));
          }
#pragma unroll
          for (int o = 16; o; o >>= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
          if (lane == 0) S.colE[c] = em;
        }
      }
    }
    if (p + 1 < p1 && (lane & 15) == 0) {
      for (int c = w; c < m; c += NW) {
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
          const int64_t row = (p + 1) * PB + lane + 32 * q;
          if (row < rows) asm volatile("prefetch.global.L2 [%0];" ::"l"(W + row + (int64_t)c * ld));
        }
      }
    }
    stage_in(0, tid, NT);
    __syncthreads();
    if (w < 4 && w < min(KB, m)) chain(S, 0, min(KB, m), w, lane, par, status);
    __syncthreads();
    for (int j0 = 0;; j0 += KB) {
      if (*reinterpret_cast<volatile int*>(&S.abort_flag)) {
        ok = false;
        break;
      }
      if (j0 + KB >= m) {  // the last block: its rows of R go back to the slice
        stage_out(j0);
        __syncthreads();
        break;
      }
      prod1w(S, j0, m, w, lane);
      __syncthreads();
      for (int c = j0 + KB + tid; c < m; c += NT) {
        double z[KB];
        int ez = 0;
#pragma unroll
        for (int i = 0; i < KB; ++i) {
          double acc = S.Z[i * MX + c];
#pragma unroll
          for (int q = 0; q < i; ++q) acc = fma(-S.G[q * KB + i], z[q], acc);
          z[i] = acc * S.rt[j0 + i];
          S.Z[i * MX + c] = z[i];
          S.Rb[i * MX + c] = fma(-S.piv[j0 + i], z[i], S.Rb[i * MX + c]);
          if (z[i] != 0.0) ez = max(ez, ef1(z[i]) + max(S.colE[j0 + i], 1) - 1023);
        }
        S.zE[c] = ez;
        S.colE[c] = 0;
      }
      __syncthreads();
      stage_out(j0);
      __syncthreads();
      // the next block's columns of P (warps 0..NMT-1) while warps 4-7 stage its rows of R
      const int j1 = j0 + KB, kb1 = min(KB, m - j1);
      if (w < 4) {
        if (w < NMT) prod2(S, j0, m, w, 0, 1, lane);
      } else {
        stage_in(j1, tid - 128, NT - 128);
      }
      __syncthreads();
      // the next block's chain (warps 0-3) beside the rest of P -= X Z (warps 4-7)
      if (w < 4) {
        if (w < kb1) chain(S, j1, kb1, w, lane, par, status);
      } else {
        constexpr int WPT = 4 / NMT;  // warps per 16-row tile
        const int u = w - 4;
        for (int nt = 1 + u / NMT; nt < MX / 8; nt += WPT) prod2(S, j0, m, u % NMT, nt, nt + 1, lane);
      }
      __syncthreads();
    }
  }
  __syncthreads();
  if (*reinterpret_cast<volatile int*>(&S.abort_flag)) return;
  for (int idx = tid; idx < mb * m; idx += NT) {
    const int i = idx % mb, k = idx / mb;
    const double v = (i < m && i <= k) ? Rg[blk::rix<MX>(i, k)] : 0.0;
    Rout[(int64_t)blockIdx.x * mb + i + (int64_t)k * ldR] = v;
  }
}

// layouts by m_max: (64, 128) and (80, 96) with R in shared memory, (160, 64), (256, 32)
// and (512, 32) with R in a global slice; two CTAs per SM up to m = 256
size_t tsqr_blk_smem(int m_max) {
  if (m_max <= 64) return blk::smem_bytes<64, 128>();
  if (m_max <= 80) return blk::smem_bytes<80, 96>();
  if (m_max <= 160) return blk::smem_bytes<160, 64>();
  if (m_max <= 256) return blk::smem_bytes<256, 32>();
  return blk::smem_bytes<512, 32>();
}
int tsqr_blk_rows(int m_max) {
  return m_max <= 64 ? 128 : m_max <= 80 ? 96 : m_max <= 160 ? 64 : 32;
}
int tsqr_blk_per_sm(int m_max) { return m_max <= 256 ? 2 : 1; }
size_t tsqr_blk_scratch(int m_max, int64_t ctas) {
  if (m_max <= 80) return 0;
  const size_t mx = m_max <= 160 ? 160 : m_max <= 256 ? 256 : 512;
  return (size_t)ctas * (mx * (mx + 1) / 2) * sizeof(double);
}

namespace {
template <class K>
cudaError_t blk_attrs(K kern, size_t sm) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  // two CTAs per SM where they fit: the largest shared-memory carveout
  return cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}
template <int MX, int PB>
cudaError_t run_blkw(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev, void* Rout, int64_t ldR,
                     void* Rscr, int* status, cudaStream_t s) {
  auto kern = k_tsqr_blkw<MX, PB>;
  const size_t sm = blk::smem_bytes<MX, PB>();
  cudaError_t e = blk_attrs(kern, sm);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)L.ctas, blk::NT, sm, s>>>(static_cast<const double*>(W), L.rows, ld, m_dev, L.mval, L.mmax,
                                             static_cast<double*>(Rout), ldR, L.mb, L.panels,
                                             static_cast<double*>(Rscr), status);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_tsqr_blk(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev, void* Rout,
                            int64_t ldR, void* Rscr, int* status, cudaStream_t s) {
  if (L.in != Fmt::F64 || L.comp != Fmt::F64 || L.out != Fmt::F64 || L.mmax > 512 ||
      L.pr != tsqr_blk_rows(L.mmax) || (L.mmax > 80 && !Rscr))
    return cudaErrorInvalidValue;
  if (L.mmax > 256) return run_blkw<512, 32>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
  if (L.mmax > 160) return run_blkw<256, 32>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
  if (L.mmax > 80) return run_blkw<160, 64>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
  auto kern = L.mmax <= 64 ? k_tsqr_blk<64, 128, double> : k_tsqr_blk<80, 96, double>;
  const size_t sm = tsqr_blk_smem(L.mmax);
  cudaError_t e = blk_attrs(kern, sm);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)L.ctas, blk::NT, sm, s>>>(static_cast<const double*>(W), L.rows, ld, m_dev, L.mval,
                                             L.mmax, static_cast<double*>(Rout), ldR, L.mb, L.panels,
                                             status);
  return cudaGetLastError();
}

}  // namespace tt
