// tsmm_ws.cu -- Y = W V(:, 0:r) of Alg. 2 (the W V_r step, TSMM of Sec. 4.1.2) for an FP64 W
// (the native FP64 form's products, and the float-float form's first product, whose W is
// the input X) on the fifth-generation tensor cores, as a warp-specialised pipeline:
//
//   TMA warp     cp.async.bulk.tensor.2d loads 128-row tiles of W (column-major FP64) into
//                three shared-memory stages;
//   digit warps  (eight: two per 32-row quarter, each taking half of a row's k range) turn
//                a tile into seven FP16 digit planes, one k-step (16 columns) at a time,
//                and store them with tcgen05.st into one of four digit slots in tensor
//                memory (lane = row, two k per 32-bit column), the A operand of the MMAs;
//   MMA thread   issues, per k-step, one tcgen05.mma.kind::f16 per digit a of W against
//                V's digits 0..6-a stacked along N, accumulating every digit product of
//                one level a + b into the same block of tensor memory (two accumulator
//                buffers of 7 x 16 columns, so a tile's products overlap the read-back of
//                the previous tile);
//   epilogue     (four warps, one per tensor-memory lane quarter) reads the seven levels
//                back with tcgen05.ld, combines them in integer arithmetic and writes Y
//                (FP64 rounded once, or float-float).
//
// Splitting (an Ozaki scheme: Ozaki, Ogita, Oishi, Rump, Numer. Algorithms 59, 2012, with
// integer digits): row i of W is scaled by a power of two above its largest entry,
// |v| = |W_ik| 2^(1085 - E_i) as a 64-bit integer, E_i the largest biased exponent field of
// the row, raised by one where that entry is within 2^-8 of the next power of two, so that
// |v| < 2^63 - 2^55.  |v| is cut into balanced base-256 digits by adding
// C = 0x8080808080808080: the bytes 7..1 of |v| + C, each less 128, are digits d_0..d_6 in
// [-128, 128) with |v| = sum_a d_a 2^(56 - 8a) up to the dropped byte (|error| <= 2^7 + 1,
// 2^-55 of the row's largest entry); the digits of a negative entry are these negated.  A
// digit is made as s ((1024 + byte) - 1152) by one FP16 fused multiply-add, s the sign.
// V's columns are cut the same way.  A product of two digits is at most 2^14 in magnitude;
// a level L = a + b sums at most 7 x 64 of them, below 2^23, so the FP32 accumulation of
// the tensor cores is exact.  The levels L = 0..6 are kept (28 digit products), the result
// is
//     Y_ij = 2^(E_i + F_j - 2106) sum_L acc_L 2^(48 - 8L),
// formed as a 64-bit integer and rounded once to FP64 (or cut into a float-float pair).
//
// Every wait is bounded; a role whose wait runs out raises the CTA's abort flag, every other
// role leaves its loop at its next wait, the bulk copies and MMAs in flight are waited for
// (bounded), the tensor memory is freed, and DEV_ERR_TIMEOUT is reported.
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "ozaki.cuh"

namespace tt {

namespace {

using namespace ozk;

constexpr int WS_TR = 128;        // rows per tile: M of one tcgen05.mma
constexpr int WS_MAXM = 64;       // k <= 64: a level's sum stays below 2^23
constexpr int WS_NN = 16;         // output columns per level block (r <= 16)
constexpr int WS_ND = 7;          // digits per value
constexpr int WS_KT = WS_MAXM / 16;
constexpr int WS_WARPS = 14;      // 0-3 epilogue, 4-11 digits, 12 TMA, 13 MMA
constexpr int WS_THREADS = 32 * WS_WARPS;
constexpr int WS_NWS = 3;         // W stages
constexpr int WS_NDS = 4;         // digit slots
constexpr int WS_NER = 8;         // row-exponent ring (tiles)
// tensor memory: accumulator buffers at columns 0 and 128 (7 x 16 used), digit slot s at
// 256 + 64 s (digit a of a k-step in columns 8a .. 8a+7: sixteen FP16 k per lane)
constexpr uint32_t WS_TMCOLS = 512;
constexpr uint32_t WS_TM_A = 256;

struct WsBars {
  uint64_t wfull[WS_NWS], wempty[WS_NWS];   // W stages: TMA landed / digit warps done reading
  uint64_t dfull[WS_NDS], dempty[WS_NDS];   // digit slots: written / MMAs done reading
  uint64_t afull[2], aempty[2];   // accumulators: products ready / read back
  uint64_t xch[4];                // row-maximum exchange of the two digit warps of a quarter
  uint64_t done;                  // the MMA thread's final drain
  uint32_t tmem;
  int abort_flag;
};

// dynamic shared memory: W stages, V's digit planes, then the small arrays
__host__ __device__ constexpr size_t ws_off_b(int m_max) { return WS_NWS * (size_t)WS_TR * m_max * 8; }
__host__ __device__ constexpr size_t ws_bplane(int kt) { return (size_t)WS_NN * 32 * kt; }
__host__ __device__ constexpr size_t ws_off_small(int m_max) {
  return ws_off_b(m_max) + WS_ND * ws_bplane((m_max + 15) / 16);
}
__host__ __device__ constexpr size_t ws_smem(int m_max) {
  // Erow[WS_NER][128], Xch[2][2][2][128], Fe[16] ints, then the barriers
  return ws_off_small(m_max) + (WS_NER * WS_TR + 8 * WS_TR + WS_NN) * sizeof(int) + sizeof(WsBars) + 64;
}

__device__ __forceinline__ void ws_bar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void ws_arrive(uint64_t* b) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(b))
               : "memory");
}
// wait for the phase with this parity; gives up (and raises the abort flag) after about
// kWaitCycles, or at once when another role has raised it
__device__ __forceinline__ bool ws_wait(uint64_t* b, uint32_t parity, int* abort_flag) {
  if (oz_try(b, parity)) return true;
  const long long t0 = clock64();
  while (!oz_try(b, parity)) {
    __nanosleep(256);  // a waiting role leaves its issue slots to the digit warps
    if (*reinterpret_cast<volatile int*>(abort_flag)) return false;
    if (clock64() - t0 > kWaitCycles) {
      *reinterpret_cast<volatile int*>(abort_flag) = 1;
      return false;
    }
  }
  return true;
}
// the same without the abort flag (the final drains)
__device__ __forceinline__ void ws_drain(uint64_t* b, uint32_t parity) {
  if (oz_try(b, parity)) return;
  const long long t0 = clock64();
  while (!oz_try(b, parity))
    if (clock64() - t0 > kWaitCycles) return;
}

__device__ __forceinline__ void ws_tma_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// shared-memory matrix descriptor: K-major, no swizzle, next core matrix along K at +128
// bytes, next 8-row group at +sbo bytes, descriptor version 1 (bits 46-47)
__device__ __forceinline__ uint64_t ws_desc(uint32_t addr, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(128u >> 4) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// instruction descriptor of kind::f16: D FP32, A and B FP16, both K-major, M = 128, N = nn
__host__ __device__ constexpr uint32_t ws_idesc(int nn) {
  return (1u << 4) | ((uint32_t)(nn >> 3) << 17) | ((128u >> 4) << 24);
}
// D (tensor memory) += A (tensor memory) B (shared memory descriptor)
__device__ __forceinline__ void ws_mma(uint32_t dtm, uint32_t atm, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(dtm),
      "r"(atm), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void ws_st4(uint32_t taddr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(a), "r"(b),
               "r"(c), "r"(d)
               : "memory");
}
__device__ __forceinline__ void ws_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(b))
               : "memory");
}
__device__ __forceinline__ void ws_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void ws_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void ws_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                 "=r"(v[7])
               : "r"(taddr));
}

// |v| + C of an FP64 value of a row (or column) with scale exponent Eb >= 1 (ws_scale_exp):
// |v| = |x| 2^(1085 - Eb) as a 64-bit integer (below 2^63 - 2^55), C = 0x8080808080808080,
// returned as two words.  The sign of x is applied to the digits afterwards: the balanced
// digits of -|v| are those of |v| negated.  FAST (Eb >= 56): every entry is read with the
// implicit bit, which for a zero or subnormal entry leaves a value below 2^7 that the
// dropped byte absorbs (without carry); otherwise zero and subnormal entries are decoded
// exactly.  NEAR (every entry of the row has Eb - max(e, 1) <= 31): one funnel shift.
template <bool FAST, bool NEAR>
__device__ __forceinline__ void ws_fix(double x, int Eb, uint32_t& wh, uint32_t& wl) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const int e = (int)((hi >> 20) & 0x7FFu);
  uint32_t mh;
  int d;
  if (FAST) {
    mh = (hi & 0xFFFFFu) | 0x100000u;
    d = Eb - e;
  } else {
    mh = (hi & 0xFFFFFu) | (e ? 0x100000u : 0u);
    d = Eb - max(e, 1);
  }
  // (M << 10) >> d with d >= 0
  const uint32_t h9 = __funnelshift_l(lo, mh, 10), l9 = lo << 10;
  uint32_t h1, l2;
  if (NEAR) {
    l2 = __funnelshift_r(l9, h9, (uint32_t)d);
    h1 = h9 >> d;
  } else {
    // a funnel shift by min(d, 32), then by max(d - 32, 0)
    const uint32_t l1 = __funnelshift_rc(l9, h9, (uint32_t)d);
    h1 = __funnelshift_rc(h9, 0u, (uint32_t)d);
    l2 = __funnelshift_rc(l1, h1, (uint32_t)max(d - 32, 0));
  }
  const uint64_t w = (((uint64_t)h1 << 32) | (uint64_t)l2) + 0x8080808080808080ull;
  wh = (uint32_t)(w >> 32);
  wl = (uint32_t)w;
}

// FP16 pair s (1024 + b) - 1152 s = s (b - 128) for the signs s = +-1 of x (low half) and y
// (high half), exactly; S holds (s_x, s_y), T = -1152 S
__device__ __forceinline__ uint32_t ws_h2(uint32_t pr, uint32_t S, uint32_t T) {
  uint32_t o;
  asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(o) : "r"(pr), "r"(S), "r"(T));
  return o;
}
// the seven digits of two values x (low half) and y (high half) from their words |v| + C
// and the high words of x and y (their signs): digit a is byte 7 - a, less 128, times the
// value's sign
__device__ __forceinline__ void ws_digits(uint32_t xh, uint32_t xl, uint32_t yh, uint32_t yl, uint32_t xs,
                                          uint32_t ys, uint32_t (&d)[WS_ND]) {
  constexpr uint32_t K = 0x64646464u;  // FP16 exponent byte of 1024
  const uint32_t sp = __byte_perm(xs, ys, 0x7030) & 0x80008000u;
  const uint32_t S = sp | 0x3C003C00u, T = sp ^ 0xE480E480u;
  const uint32_t H1 = __byte_perm(xh, yh, 0x5140), H2 = __byte_perm(xh, yh, 0x7362);
  const uint32_t L1 = __byte_perm(xl, yl, 0x5140), L2 = __byte_perm(xl, yl, 0x7362);
  d[0] = ws_h2(__byte_perm(H2, K, 0x4342), S, T);
  d[1] = ws_h2(__byte_perm(H2, K, 0x4140), S, T);
  d[2] = ws_h2(__byte_perm(H1, K, 0x4342), S, T);
  d[3] = ws_h2(__byte_perm(H1, K, 0x4140), S, T);
  d[4] = ws_h2(__byte_perm(L2, K, 0x4342), S, T);
  d[5] = ws_h2(__byte_perm(L2, K, 0x4140), S, T);
  d[6] = ws_h2(__byte_perm(L1, K, 0x4342), S, T);
}
// scale exponent of a row (or column) from the largest of its entries' high words
// (sign cleared): the largest exponent field, plus one where the mantissa's top 20 bits
// reach 0xFDFDF (so that |v| = |x| 2^(1085 - Eb) stays below 2^64 - C); at least 1;
// kWsNonfinite where the row holds an infinity or a NaN (its digits are then all zero)
constexpr int kWsNonfinite = 4096;
__device__ __forceinline__ int ws_scale_exp(uint32_t mx) {
  if ((mx >> 20) == 0x7FFu) return kWsNonfinite;
  return max((int)(mx >> 20) + ((mx & 0xFFFFFu) >= 0xFDFDFu ? 1 : 0), 1);
}
template <bool FAST, bool NEAR>
__device__ __forceinline__ void ws_digits8_(const double (&x)[8], int Eb, uint32_t (&dd)[4][WS_ND]) {
  uint32_t wh[8], wl[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) ws_fix<FAST, NEAR>(x[c], Eb, wh[c], wl[c]);
#pragma unroll
  for (int p = 0; p < 4; ++p)
    ws_digits(wh[2 * p], wl[2 * p], wh[2 * p + 1], wl[2 * p + 1], (uint32_t)__double2hiint(x[2 * p]),
              (uint32_t)__double2hiint(x[2 * p + 1]), dd[p]);
}
// digits of eight consecutive k of one row (or column), one 16-byte row of a core matrix
// per plane; near: every entry of the row is within 2^31 of the scale (ws_fix)
__device__ __forceinline__ void ws_digits8(const double (&x)[8], int Eb, bool near, uint32_t (&dd)[4][WS_ND]) {
  if (Eb >= 56) {
    if (near) ws_digits8_<true, true>(x, Eb, dd);
    else ws_digits8_<true, false>(x, Eb, dd);
  } else {
    if (near) ws_digits8_<false, true>(x, Eb, dd);
    else ws_digits8_<false, false>(x, Eb, dd);
  }
}

// Y_ij from the seven exact level sums (FP32 integers) of one output:
// U = sum_L acc_L 2^(38 - 8L) (the part below 2^-10 of level 6 rounded off) as a 64-bit
// integer, Y = U 2^(Eb + Fb - 2096) rounded to nearest (by integer operations where the
// result leaves the normal range); NaN where the row or the column held a non-finite value
__device__ __forceinline__ double ws_combine(const uint32_t (&v)[WS_ND][8], int c, int Eb, int Fb, int sh) {
  if (Eb == kWsNonfinite || Fb == kWsNonfinite) return __longlong_as_double(0x7FF8000000000000ll);
  int l[WS_ND];
#pragma unroll
  for (int L = 0; L < WS_ND; ++L) l[L] = __float2int_rn(__uint_as_float(v[L][c]));
  const long long shi = (long long)(l[0] * 256 + l[1]) * 65536 + (long long)(l[2] * 256 + l[3]);
  const long long slo = (long long)l[4] * 65536 + (long long)(l[5] * 256 + l[6]);
  const long long U = shi * 16384 + ((slo + 512) >> 10);
  const int X = Eb + Fb - 2096 - sh;
  // |U| < 2^58: for 2^-1022 <= 2^X <= 2^966 the result is normal, rounded once (U to FP64;
  // the power of two is exact)
  if (X >= -1022 && X <= 966) return __ll2double_rn(U) * __longlong_as_double((long long)(X + 1023) << 52);
  if (U == 0) return 0.0;
  const unsigned long long A = U < 0 ? (unsigned long long)(-U) : (unsigned long long)U;
  const int lz = __clzll((long long)A);
  const int be = Eb + Fb - lz - 1010 - sh;  // biased exponent of the result
  const unsigned long long sgn = U < 0 ? 0x8000000000000000ull : 0ull;
  unsigned long long bits;
  if (be >= 1) {
    const unsigned long long N = A << lz;
    // the implicit bit lands in the exponent field (hence be - 1); a rounding carry moves
    // the exponent up by one, to infinity at the top
    bits = be > 2046 ? 0x7FF0000000000000ull
                     : ((unsigned long long)(be - 1) << 52) + (N >> 11) + ((N >> 10) & 1ull);
  } else {
    // subnormal result: A on the grid of 2^-1074, rounded once (a carry into bit 52 gives
    // the smallest normal number)
    const int t = 1022 + sh - Eb - Fb;  // Y = (A 2^-t) 2^-1074
    bits = t <= 0 ? (A << -t) : (t >= 64 ? 0ull : (A >> t) + ((A >> (t - 1)) & 1ull));
  }
  return __longlong_as_double((long long)(bits | sgn));
}

// V read as FP64 (a float-float value as the FP64 sum of its words: 53 bits of its ~48)
__device__ __forceinline__ double ws_f64(double v) { return v; }
__device__ __forceinline__ double ws_f64(df v) { return (double)v.hi + (double)v.lo; }
// one output in the format of Y: FP64, or float-float (the top 48 bits of the integer U
// turned into an FP32 pair by two exact conversions and a two-sum, then scaled by 2^X;
// through FP64 where 2^X leaves FP32's range)
template <class VT>
__device__ __forceinline__ VT ws_out(const uint32_t (&v)[WS_ND][8], int c, int Eb, int Fb, int sh);
template <>
__device__ __forceinline__ double ws_out<double>(const uint32_t (&v)[WS_ND][8], int c, int Eb, int Fb, int sh) {
  return ws_combine(v, c, Eb, Fb, sh);
}
template <>
__device__ __forceinline__ df ws_out<df>(const uint32_t (&v)[WS_ND][8], int c, int Eb, int Fb, int sh) {
  const int X = Eb + Fb - 2096 - sh;
  if (Eb != kWsNonfinite && Fb != kWsNonfinite && X >= -126 && X <= 69) {
    int l[WS_ND];
#pragma unroll
    for (int L = 0; L < WS_ND; ++L) l[L] = __float2int_rn(__uint_as_float(v[L][c]));
    const long long shi = (long long)(l[0] * 256 + l[1]) * 65536 + (long long)(l[2] * 256 + l[3]);
    const long long slo = (long long)l[4] * 65536 + (long long)(l[5] * 256 + l[6]);
    const long long U = shi * 16384 + ((slo + 512) >> 10);
    // U = U_h 2^34 + U_m 2^10 + (0 .. 2^10): both parts exact in FP32 (|U| < 2^58)
    const float fh = __int2float_rn((int)(U >> 34));
    const float fm = __int2float_rn((int)((U >> 10) & 0xFFFFFFll));
    float hs, he;
    eft_two_sum(fh * 17179869184.f, fm * 1024.f, hs, he);
    const float p = __int_as_float((X + 127) << 23);
    return mkdf(hs * p, he * p);
  }
  const double y = ws_combine(v, c, Eb, Fb, sh);
  const float h = __double2float_rn(y);
  return mkdf(h, isfinite(h) ? __double2float_rn(y - (double)h) : 0.f);
}

// Y(:, 0:r) = W V(:, 0:r), W rows x m FP64 (through the tensor map tmW: 128-row boxes of
// m_max columns), V m x r (leading dimension ldV) and Y rows x r (ldy) both FP64 or both
// float-float (VT).  FP64 input
// read as W 2^-k with k = xr->k where xr is given (the shifted input pipeline).
template <class VT>
__global__ void __launch_bounds__(WS_THREADS, 1)
k_tsmm_ws(const __grid_constant__ CUtensorMap tmW, int64_t rows, const int* __restrict__ m_ptr,
          int m_val, const VT* __restrict__ V, int ldV, const int* __restrict__ r_ptr, int r_val,
          VT* __restrict__ Y, int64_t ldy, int m_max, int* status, const XRange* xr) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int m = m_ptr ? *m_ptr : m_val;
  const int sh = xr ? xr->k : 0;
  const int r = r_ptr ? *r_ptr : r_val;
  if (m < 1 || m > m_max || m_max > WS_MAXM || r < 1 || r > WS_NN || r > m ||
      blockDim.x != WS_THREADS) {
    if (threadIdx.x == 0 && status) atomicOr(status, DEV_ERR_SHAPE);
    return;
  }
  const int kt = (m_max + 15) / 16;
  const size_t wstage = (size_t)WS_TR * m_max * 8;
  unsigned char* Wst = smem_raw;                   // W stages, column-major 128 x m_max
  unsigned char* Bd = smem_raw + ws_off_b(m_max);  // V's seven digit planes
  int* Erow = reinterpret_cast<int*>(smem_raw + ws_off_small(m_max));  // [WS_NER][128]
  int* Xch = Erow + WS_NER * WS_TR;  // [tile parity][k-half][largest, smallest][128]
  int* Fe = Xch + 8 * WS_TR;                                           // [16]
  WsBars& B = *reinterpret_cast<WsBars*>(Fe + WS_NN);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  if (tid == 0) {
    for (int s = 0; s < WS_NWS; ++s) {
      ws_bar_init(&B.wfull[s], 1);
      ws_bar_init(&B.wempty[s], 8);
    }
    for (int s = 0; s < WS_NDS; ++s) {
      ws_bar_init(&B.dfull[s], 8);
      ws_bar_init(&B.dempty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      ws_bar_init(&B.afull[s], 2);
      ws_bar_init(&B.aempty[s], 4);
    }
    for (int q = 0; q < 4; ++q) ws_bar_init(&B.xch[q], 2);
    ws_bar_init(&B.done, 1);
    B.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 13) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&B.tmem)),
                 "r"(WS_TMCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (warp == 12 && lane == 0)
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmW)) : "memory");
  // V's column scale exponents and digit planes: row n of plane b holds column n's digits
  // b along k
  for (int j = warp; j < WS_NN; j += WS_WARPS) {
    uint32_t mx = 0;
    if (j < r)
      for (int k = lane; k < m; k += 32) mx = max(mx, (uint32_t)__double2hiint(ws_f64(V[k + (size_t)j * ldV])) & 0x7FFFFFFFu);
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) Fe[j] = ws_scale_exp(mx);
  }
  __syncthreads();
  for (int idx = tid; idx < WS_NN * 2 * kt; idx += WS_THREADS) {
    const int n = idx % WS_NN, kg = idx / WS_NN;
    double x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int k = 8 * kg + c;
      x[c] = (n < r && k < m) ? ws_f64(V[k + (size_t)n * ldV]) : 0.0;
    }
    uint32_t dd[4][WS_ND];
    ws_digits8(x, Fe[n], false, dd);
    const size_t off = (size_t)(n >> 3) * 256 * kt + (size_t)kg * 128 + (size_t)(n & 7) * 16;
#pragma unroll
    for (int b = 0; b < WS_ND; ++b)
      *reinterpret_cast<uint4*>(Bd + b * ws_bplane(kt) + off) = make_uint4(dd[0][b], dd[1][b], dd[2][b], dd[3][b]);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  ws_fence_before();
  __syncthreads();
  ws_fence_after();
  const uint32_t tmem = B.tmem;
  const int64_t ntiles = (rows + WS_TR - 1) / WS_TR;

  if (warp == 12) {
    // ---- TMA: tile n of this CTA into stage n mod WS_NWS ---------------------------------
    if (lane == 0) {
      int n = 0;
      for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++n) {
        const int st = n % WS_NWS;
        if (!ws_wait(&B.wempty[st], ((n / WS_NWS) & 1) ^ 1, &B.abort_flag)) break;
        oz_expect(&B.wfull[st], (uint32_t)wstage);
        ws_tma_2d(Wst + st * wstage, &tmW, (int)(t * WS_TR), 0, &B.wfull[st]);
      }
      // the copies in flight land before the CTA leaves: the last use u of stage s
      for (int s = 0; s < WS_NWS && s < n; ++s) {
        const int u = s + WS_NWS * ((n - 1 - s) / WS_NWS);
        ws_drain(&B.wfull[s], (uint32_t)((u / WS_NWS) & 1));
      }
    }
    __syncwarp();
  } else if (warp >= 4 && warp < 12) {
    // ---- digits: row i, k-half h of every k-step -----------------------------------------
    const int q = warp & 3, h = (warp - 4) >> 2, i = 32 * q + lane;
    int n = 0, kc = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++n) {
      const int st = n % WS_NWS;
      if (!ws_wait(&B.wfull[st], (n / WS_NWS) & 1, &B.abort_flag)) break;
      const double* Wt = reinterpret_cast<const double*>(Wst + st * wstage);
      double x[WS_KT][8];
      uint32_t em = 0, en = 0x7FFFFFFFu;
#pragma unroll
      for (int kk = 0; kk < WS_KT; ++kk)
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int k = 16 * kk + 8 * h + c;
          x[kk][c] = (kk < kt && k < m) ? Wt[(size_t)k * WS_TR + i] : 0.0;
          const uint32_t a = (uint32_t)__double2hiint(x[kk][c]) & 0x7FFFFFFFu;
          em = max(em, a);
          en = min(en, a);
        }
      // the stage is read: back to the TMA warp
      __syncwarp();
      if (lane == 0) ws_arrive(&B.wempty[st]);
      // the row's largest and smallest high words, with the other k-half's
      Xch[((n & 1) * 4 + 2 * h) * WS_TR + i] = (int)em;
      Xch[((n & 1) * 4 + 2 * h + 1) * WS_TR + i] = (int)en;
      __syncwarp();
      if (lane == 0) ws_arrive(&B.xch[q]);
      if (!ws_wait(&B.xch[q], n & 1, &B.abort_flag)) break;
      em = max(em, (uint32_t)Xch[((n & 1) * 4 + 2 * (h ^ 1)) * WS_TR + i]);
      en = min(en, (uint32_t)Xch[((n & 1) * 4 + 2 * (h ^ 1) + 1) * WS_TR + i]);
      const int Eb = ws_scale_exp(em);
      const bool near = Eb - max((int)(en >> 20), 1) <= 31;
#pragma unroll
      for (int kk = 0; kk < WS_KT; ++kk) {
        if (kk >= kt) break;
        const int slot = kc % WS_NDS;
        if (!ws_wait(&B.dempty[slot], ((kc / WS_NDS) & 1) ^ 1, &B.abort_flag)) {
          ok = false;
          break;
        }
        ws_fence_after();
        // (after the slot wait: the MMAs of a k-step WS_NDS back have completed, so the
        // epilogue is past the tile WS_NDS + 2 back, the entry's previous reader)
        if (kk == 0 && h == 0) Erow[(n % WS_NER) * WS_TR + i] = Eb;
        uint32_t dd[4][WS_ND];
        ws_digits8(x[kk], Eb, near, dd);
        const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + WS_TM_A + 64u * slot + 4u * h;
#pragma unroll
        for (int a = 0; a < WS_ND; ++a) ws_st4(ta + 8u * a, dd[0][a], dd[1][a], dd[2][a], dd[3][a]);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        ws_fence_before();
        __syncwarp();
        if (lane == 0) ws_arrive(&B.dfull[slot]);
        ++kc;
      }
    }
  } else if (warp == 13) {
    // ---- MMA issue: the 7 digit products of each k-step into accumulator n mod 2 ---------
    if (lane == 0) {
      const uint32_t b0 = smem_u32(Bd);
      int n = 0, kc = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++n) {
        const int acc = n & 1;
        if (!ws_wait(&B.aempty[acc], ((n >> 1) & 1) ^ 1, &B.abort_flag)) break;
        ws_fence_after();
        for (int kk = 0; kk < kt; ++kk) {
          const int slot = kc % WS_NDS;
          if (!ws_wait(&B.dfull[slot], (kc / WS_NDS) & 1, &B.abort_flag)) {
            ok = false;
            break;
          }
          ws_fence_after();
          const uint64_t bd = ws_desc(b0 + 256u * kk, 256u * kt);
#pragma unroll
          for (int a = 0; a < WS_ND; ++a)
            ws_mma(tmem + (uint32_t)(acc * 128 + 16 * a), tmem + WS_TM_A + 64u * slot + 8u * a, bd,
                   ws_idesc(16 * (WS_ND - a)), (kk | a) ? 1u : 0u);
          ws_commit(&B.dempty[slot]);
          ++kc;
        }
        if (!ok) break;
        ws_commit(&B.afull[acc]);
        ws_arrive(&B.afull[acc]);
      }
      // every MMA issued has completed before the tensor memory is freed
      ws_commit(&B.done);
      ws_drain(&B.done, 0);
    }
    __syncwarp();
  } else {
    // ---- epilogue: lane quarter q = warp, row i -------------------------------------------
    const int q = warp, i = 32 * q + lane;
    int n = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++n) {
      const int acc = n & 1;
      if (!ws_wait(&B.afull[acc], (n >> 1) & 1, &B.abort_flag)) break;
      ws_fence_after();
      const int Eb = Erow[(n % WS_NER) * WS_TR + i];
      const int64_t row = t * WS_TR + i;
      const uint32_t tb = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * 128);
      for (int half = 0; half < 2; ++half) {
        if (half == 1 && r <= 8) break;
        uint32_t v[WS_ND][8];
#pragma unroll
        for (int L = 0; L < WS_ND; ++L) ws_ld8(tb + (uint32_t)(16 * L + 8 * half), v[L]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (half == 1 || r <= 8) {
          // the accumulator is read: back to the MMA thread
          ws_fence_before();
          __syncwarp();
          if (lane == 0) ws_arrive(&B.aempty[acc]);
        }
        if (row < rows) {
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const int j = 8 * half + c;
            if (j < r) Y[row + (int64_t)j * ldy] = ws_out<VT>(v, c, Eb, Fe[j], sh);
          }
        }
      }
    }
  }
  ws_fence_before();
  __syncthreads();
  if (tid == 0 && status && *reinterpret_cast<volatile int*>(&B.abort_flag)) atomicOr(status, DEV_ERR_TIMEOUT);
  if (warp == 13) {
    ws_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(WS_TMCOLS) : "memory");
  }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda)
PFN_cuTensorMapEncodeTiled_v12000 ws_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

}  // namespace

// usable for these formats and sizes ("tsmm.ws": 0 never, 1 for an FP64 W with FP64 V and Y
// (native FP64 arithmetic, or the float-float form's stand-alone product) or float-float V
// and Y (the float-float form's first product, W = X))
bool tsmm_ws_ok(Fmt in, Fmt comp, Fmt vfmt, Fmt out, int m_max, int r_max) {
  if (tune_get("tsmm.ws", 1) == 0) return false;
  if (in != Fmt::F64 || (comp != Fmt::F64 && comp != Fmt::DF) || vfmt != out) return false;
  if (vfmt != Fmt::F64 && !(vfmt == Fmt::DF && comp == Fmt::DF)) return false;
  if (m_max < 16 || m_max > WS_MAXM || r_max < 1 || r_max > WS_NN) return false;
  return ws_smem(m_max) <= 227 * 1024;
}

size_t tsmm_ws_smem(int m_max) { return ws_smem(m_max); }

// One launch over all row tiles, or *used = false (nothing launched) where a tensor map of
// W cannot be made: W not 16-byte aligned, a leading dimension of an odd number of
// values, fewer than 128 or 2^31 and more rows.  The map covers c.m_max columns of W; with
// m_dev set, the caller's W holds that many columns (the driver's unfoldings do).
cudaError_t launch_tsmm_ws(const TsmmCfg& c, const void* W, int64_t rows, int64_t ld, const int* m_dev,
                           const void* V, int ldV, const int* r_dev, void* Y, int64_t ldy, int* status,
                           cudaStream_t s, bool* used) {
  *used = false;
  if (c.in != Fmt::F64 || c.out != c.vfmt || (c.vfmt != Fmt::F64 && c.vfmt != Fmt::DF)) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(W) & 15) != 0 || (ld & 1) != 0 || rows < WS_TR || rows >= (1ll << 31) ||
      ld < rows)
    return cudaSuccess;
  PFN_cuTensorMapEncodeTiled_v12000 enc = ws_encoder();
  if (!enc) return cudaSuccess;
  CUtensorMap tm;
  const cuuint64_t gdim[2] = {(cuuint64_t)rows, (cuuint64_t)c.m_max};
  const cuuint64_t gstr[1] = {(cuuint64_t)ld * 8};
  const cuuint32_t box[2] = {(cuuint32_t)WS_TR, (cuuint32_t)c.m_max};
  const cuuint32_t est[2] = {1, 1};
  if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void*>(W), gdim, gstr, box, est,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaSuccess;
  const size_t smem = ws_smem(c.m_max);
  const bool dfv = c.vfmt == Fmt::DF;
  cudaError_t e = dfv ? cudaFuncSetAttribute(k_tsmm_ws<df>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                      : cudaFuncSetAttribute(k_tsmm_ws<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (rows + WS_TR - 1) / WS_TR;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(ntiles, c.ctas));
  if (dfv)
    k_tsmm_ws<df><<<grid, WS_THREADS, smem, s>>>(tm, rows, m_dev, c.m_max, static_cast<const df*>(V), ldV, r_dev,
                                                 c.r_max, static_cast<df*>(Y), ldy, c.m_max, status, c.xr);
  else
    k_tsmm_ws<double><<<grid, WS_THREADS, smem, s>>>(tm, rows, m_dev, c.m_max, static_cast<const double*>(V), ldV,
                                                     r_dev, c.r_max, static_cast<double*>(Y), ldy, c.m_max, status,
                                                     c.xr);
  *used = true;
  return cudaGetLastError();
}

}  // namespace tt
