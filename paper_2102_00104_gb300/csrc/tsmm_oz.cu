// tsmm_oz.cu -- Y = W V(:, 0:r) of Alg. 2 line 11 (TSMM, Sec. 4.1.2) for the float-float
// form on the tensor cores, by Ozaki splitting (Ozaki, Ogita, Oishi, Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012).
//
// Every value of a row i of W is scaled by 2^-E_i (|W_ik| < 2^E_i) and cut into six
// signed integer digits d_1..d_6, s = W_ik 2^-E_i ~ sum_a d_a 2^(1-8a): d_1 = rint(s 2^7),
// then d_a = rint(rem 2^8) of the remainder (|d_a| <= 128; the digit that takes the low
// word of the float-float pair stays <= 192).  Column j of V is cut the same way with
// its own 2^F_j.  Digits are exact in bf16, their products are exact, and the products
// of one level L = a + b summed over k (m <= 96) stay below 2^24, so mma.sync bf16 with
// FP32 accumulation sums every level exactly:
//     Y_ij = 2^(E_i + F_j) sum_{L=2..7} acc_L 2^(2 - 8L),  acc_L = sum_k sum_{a+b=L} d_a e_b.
// Levels above 7 are dropped (21 digit pairs).  The error is about sqrt(m) 2^-46 of
// 2^(E_i + F_j) (normwise, not relative to each entry); the levels are added in
// float-float from the smallest.
//
// Data path: a CTA of 4 warps takes 64-row tiles of W.  A full tile comes into shared
// memory by bulk asynchronous copies (cp.async.bulk, one per column of the tile, 512 B,
// completing on an mbarrier) into one of two buffers, so the copy of the next tile runs
// while the current one is computed; a tile that ends early, or a W whose columns do not
// start on 16-byte boundaries, is loaded with plain loads.  Warp w takes rows 16w..16w+15
// of the tile: lane (g, t) holds rows g and g+8 and k = 16 kk + 2t, 2t+1, 2t+8, 2t+9 of
// every k-step, i.e. the A fragment of mma.m16n8k16.  V's digits are built once per CTA,
// already in B-fragment order, in shared memory.

#include <algorithm>

#include "ozaki.cuh"

namespace tt {

namespace {

using namespace ozk;

constexpr int OZ_TR = 64;               // rows per tile
constexpr int OZ_WARPS = 4;
constexpr int OZ_THREADS = 32 * OZ_WARPS;
constexpr int OZ_CS = OZ_TR * 8 + 32;   // bytes per staged column (padded: conflict-free reads)
constexpr int OZ_MAXM = 96;             // sum of one level over k stays below 2^24
constexpr int OZ_MAXR = 64;   // r_max > 32 runs as two launches of up to 32 columns (oz_col0)

__device__ __forceinline__ void oz_mma(float (&c)[4], const uint32_t (&a)[4], uint2 b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}


// NT n-tiles of 8 output columns (r <= 8 NT).  Shared memory: two tile buffers
// (m_max columns of OZ_CS bytes each), V's digits in B-fragment order
// (kt x 6 x NT x 32 uint2), the column exponents, two mbarriers.
// X64 (native FP64 form): seven digits per value from its FP64 bits (oz64_digits), levels
// 2..8 (28 digit products per k-step and n-tile), and an integer-then-FP64 combination of
// the exact level sums, so that Y is rounded once to FP64 from a sum accurate to ~2^-56
// of 2^(E_i + F_j).
template <int NT, bool X64, class S, class VS, class SO>
__global__ void __launch_bounds__(OZ_THREADS)
k_tsmm_oz(const S* __restrict__ W, int64_t rows, int64_t ld, const int* __restrict__ m_ptr,
          int m_val, const VS* __restrict__ V, int ldV, const int* __restrict__ r_ptr, int r_val,
          SO* __restrict__ Y, int64_t ldy, int m_max, int r_max, int nbuf, int* status,
          const XRange* xr, int col0) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  XRead<df, S> rd;  // W read as W 2^-sh (FP64 input of the float-float form)
  rd.set(xr ? xr->k : 0, xr != nullptr);
  const int m = m_ptr ? *m_ptr : m_val;
  const int r_all = r_ptr ? *r_ptr : r_val;
  // this launch's columns: col0 .. col0 + 8 NT - 1 of V and Y (the second launch of an
  // r_max > 32 product has nothing to do when the rank found is <= 32)
  if (col0 > 0 && r_all <= col0) return;
  const int r = min(r_all - col0, 8 * NT);
  V += (size_t)col0 * ldV;
  Y += (int64_t)col0 * ldy;
  if (m < 1 || m > m_max || m_max > OZ_MAXM || r < 1 || r_all > r_max || r_all > m || r > 8 * NT ||
      nbuf < 1 || nbuf > 2) {
    if (threadIdx.x == 0 && status) atomicOr(status, DEV_ERR_SHAPE);
    return;
  }
  constexpr int ND = X64 ? 7 : 6;  // digits per value
  const int kt = (m_max + 15) / 16;
  unsigned char* buf0 = smem_raw;
  unsigned char* buf1 = smem_raw + (size_t)m_max * OZ_CS;  // (nbuf = 2)
  uint2* Bf = reinterpret_cast<uint2*>(smem_raw + nbuf * (size_t)m_max * OZ_CS);  // [kk][b][nt][lane]
  int* Fe = reinterpret_cast<int*>(Bf + (size_t)kt * ND * NT * 32);            // [8 NT]
  uint64_t* bar = reinterpret_cast<uint64_t*>(Fe + 8 * NT);                    // [2], 8-aligned
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int g = lane >> 2, tq = lane & 3;

  const int64_t ntiles = (rows + OZ_TR - 1) / OZ_TR;
  const int64_t nfull = rows / OZ_TR;
  // bulk copies need 16-byte aligned column starts and whole tiles
  const bool tma = (ld % 2 == 0) && ((reinterpret_cast<uintptr_t>(W) & 15) == 0);
  if (tid == 0) {
    oz_bar_init(&bar[0]);
    oz_bar_init(&bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // column exponents of V(:, 0:r): F_j with |V_kj| < 2^(F_j) as a biased FP32 exponent
  // (X64: the largest biased FP64 exponent field of the column)
  for (int j = w; j < 8 * NT; j += OZ_WARPS) {
    int be = 0;
    if (j < r)
      for (int k = lane; k < m; k += 32) {
        if constexpr (X64)
          be = max(be, (int)((__double_as_longlong((double)V[k + (size_t)j * ldV]) >> 52) & 0x7FF));
        else
          be = max(be, oz_bexp(ld_as<df>(V[k + (size_t)j * ldV])));
      }
    for (int o = 16; o; o >>= 1) be = max(be, __shfl_xor_sync(0xffffffffu, be, o));
    if (lane == 0) Fe[j] = be;
  }
  __syncthreads();
  // V's digits in B-fragment order: lane (g, t) of n-tile nt holds column 8 nt + g at
  // k = 16 kk + 2t, 2t+1 (first register) and 2t+8, 2t+9 (second)
  for (int idx = tid; idx < kt * NT * 32; idx += OZ_THREADS) {
    const int ln = idx & 31, nt = (idx >> 5) % NT, kk = idx / (32 * NT);
    const int j = 8 * nt + (ln >> 2);
    const int k0 = 16 * kk + 2 * (ln & 3);
    float d[4][7];
    const int ks[4] = {k0, k0 + 1, k0 + 8, k0 + 9};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool in = j < r && ks[q] < m;
      if constexpr (X64) {
        oz64_digits(in ? (double)V[ks[q] + (size_t)j * ldV] : 0.0, Fe[j], d[q]);
      } else {
        const df v = in ? ld_as<df>(V[ks[q] + (size_t)j * ldV]) : Tr<df>::zero();
        float d6[6];
        oz_digits(v, oz_inv_scale(Fe[j]), d6);
#pragma unroll
        for (int b = 0; b < 6; ++b) d[q][b] = d6[b];
      }
    }
#pragma unroll
    for (int b = 0; b < ND; ++b)
      Bf[((size_t)(kk * ND + b) * NT + nt) * 32 + ln] =
          make_uint2(oz_pack(d[0][b], d[1][b]), oz_pack(d[2][b], d[3][b]));
  }
  __syncthreads();

  // tiles of this CTA: blockIdx.x, + gridDim.x, ...; bulk copies for full tiles
  // copies issued and waited for per buffer (thread 0's count, for a clean exit)
  int nissued[2] = {0, 0}, nwaited[2] = {0, 0};
  auto issue = [&](int64_t tile, int bi) {
    const int64_t r0 = tile * OZ_TR;
    unsigned char* buf = bi ? buf1 : buf0;
    oz_expect(&bar[bi], (uint32_t)(m * OZ_TR * 8));
    for (int k = 0; k < m; ++k)
      oz_bulk(buf + (size_t)k * OZ_CS, W + r0 + (int64_t)k * ld, OZ_TR * 8, &bar[bi]);
    ++nissued[bi];
  };
  int64_t tile = blockIdx.x;
  if (tid == 0 && tma && tile < nfull) issue(tile, 0);
  bool ok = true;
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    const int bi = nbuf == 2 ? (it & 1) : 0;
    unsigned char* buf = bi ? buf1 : buf0;
    const bool bulk = tma && tile < nfull;
    const int64_t r0 = tile * OZ_TR;
    const int64_t nxt = tile + gridDim.x;
    // two buffers: the next tile's copy starts now (its buffer was released at the end
    // of the last tile); one buffer: it starts once this tile is done
    if (nbuf == 2 && tid == 0 && tma && nxt < nfull) issue(nxt, bi ^ 1);
    if (bulk) {
      // this buffer's (it / nbuf)-th use
      if (!oz_wait(&bar[bi], (uint32_t)((it / nbuf) & 1))) ok = false;
      else if (tid == 0) ++nwaited[bi];
    } else {
      for (int idx = tid; idx < m * OZ_TR; idx += OZ_THREADS) {
        const int i = idx % OZ_TR, k = idx / OZ_TR;
        const int64_t row = r0 + i;
        reinterpret_cast<S*>(buf + (size_t)k * OZ_CS)[i] =
            row < rows ? W[row + (int64_t)k * ld] : oz_zero<S>();
      }
      __syncthreads();
    }
    if (__syncthreads_or(!ok)) {
      ok = false;
      break;
    }

    // rows g and g+8 of this warp's 16: exponent of the row maximum over k < m
    const int rg = 16 * w + g;
    unsigned key0 = 0, key1 = 0;
    for (int kk = 0; kk < kt; ++kk) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = 16 * kk + 2 * tq + (q & 1) + 8 * (q >> 1);
        if (k < m) {
          const S* c = reinterpret_cast<const S*>(buf + (size_t)k * OZ_CS);
          key0 = max(key0, oz_key(c[rg]));
          key1 = max(key1, oz_key(c[rg + 8]));
        }
      }
    }
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
      key0 = max(key0, __shfl_xor_sync(0xffffffffu, key0, o));
      key1 = max(key1, __shfl_xor_sync(0xffffffffu, key1, o));
    }
    const int be0 = oz_bexp_of(key0, (S*)nullptr, rd.sh), be1 = oz_bexp_of(key1, (S*)nullptr, rd.sh);
    const float sc0 = oz_inv_scale(be0), sc1 = oz_inv_scale(be1);
    // X64: the rows' largest biased FP64 exponent fields
    const int eM0 = (int)(key0 >> 20), eM1 = (int)(key1 >> 20);

    float acc[ND][NT][4];
#pragma unroll
    for (int L = 0; L < ND; ++L)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) acc[L][nt][0] = acc[L][nt][1] = acc[L][nt][2] = acc[L][nt][3] = 0.f;

    for (int kk = 0; kk < kt; ++kk) {
      // digits of this lane's 8 values: dq[q][row half][digit], q = k offset 0, 1, 8, 9
      float dd[4][2][7];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = 16 * kk + 2 * tq + (q & 1) + 8 * (q >> 1);
        const S* c = reinterpret_cast<const S*>(buf + (size_t)(k < m ? k : 0) * OZ_CS);
        if constexpr (X64) {
          oz64_digits(k < m ? (double)c[rg] : 0.0, eM0, dd[q][0]);
          oz64_digits(k < m ? (double)c[rg + 8] : 0.0, eM1, dd[q][1]);
        } else {
          const df x0 = k < m ? rd(c[rg]) : Tr<df>::zero();
          const df x1 = k < m ? rd(c[rg + 8]) : Tr<df>::zero();
          float d0[6], d1[6];
          oz_digits(x0, sc0, d0);
          oz_digits(x1, sc1, d1);
#pragma unroll
          for (int a = 0; a < 6; ++a) {
            dd[q][0][a] = d0[a];
            dd[q][1][a] = d1[a];
          }
        }
      }
#pragma unroll
      for (int a = 0; a < ND; ++a) {
        const uint32_t af[4] = {oz_pack(dd[0][0][a], dd[1][0][a]), oz_pack(dd[0][1][a], dd[1][1][a]),
                                oz_pack(dd[2][0][a], dd[3][0][a]), oz_pack(dd[2][1][a], dd[3][1][a])};
        // b = 0 .. ND-1-a (0-based: digit a pairs with b while a + b <= ND - 1), level a + b
#pragma unroll
        for (int b = 0; b + a <= ND - 1; ++b)
#pragma unroll
          for (int nt = 0; nt < NT; ++nt)
            oz_mma(acc[a + b][nt], af, Bf[((size_t)(kk * ND + b) * NT + nt) * 32 + lane]);
      }
    }

    if constexpr (X64) {
      // Y = 2^(eM + fM - 2082) (S_hi + 2^-24 S_lo) with the exact level sums (levels
      // l = 0..6 at weights 2^(24 - 8l) in S_hi, l = 4..6 at 2^(48 - 8l) in S_lo)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          const int j = 8 * nt + 2 * tq + (h & 1);
          const int64_t row = r0 + rg + 8 * (h >> 1);
          if (j >= r || row >= rows) continue;
          long long shi = 0, slo = 0;
#pragma unroll
          for (int l = 0; l < 4; ++l) shi = (shi << 8) + (long long)__float2int_rn(acc[l][nt][h]);
#pragma unroll
          for (int l = 4; l < 7; ++l) slo = (slo << 8) + (long long)__float2int_rn(acc[l][nt][h]);
          const double t = __fma_rn((double)slo, 0x1p-24, (double)shi);
          const int e = ((h >> 1) ? eM1 : eM0) + Fe[j] - 2082;
          // 2^e as two exact powers of two inside FP64's normal range (0 far below it)
          const int e1 = e / 2, e2 = e - e / 2;
          const double p1 = e1 < -1022 ? 0.0 : __longlong_as_double((long long)(e1 + 1023) << 52);
          const double p2 = e2 < -1022 ? 0.0 : __longlong_as_double((long long)(e2 + 1023) << 52);
          Y[row + (int64_t)j * ldy] = st_as<SO>((double)(t * p1 * p2));
        }
      }
    } else {
    // Y = 2^(E + F) sum_L acc_L 2^(2 - 8L), L = 2..7 (index L - 2), smallest level first
    const int E0 = be0 - 126, E1 = be1 - 126;
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int j = 8 * nt + 2 * tq + (h & 1);
        const int64_t row = r0 + rg + 8 * (h >> 1);
        if (j >= r || row >= rows) continue;
        // 2^(E + F + 2 - 16): the level-2 weight; level L adds 2^(-8 (L - 2)) (exact
        // unless the product leaves FP32's normal range, i.e. for values near 1e-38)
        const int e = ((h >> 1) ? E1 : E0) + (Fe[j] - 126) - 14;
        const float p2 = oz_pow2(e);
        float s = acc[5][nt][h] * (p2 * 0x1p-40f), err = 0.f;
#pragma unroll
        for (int L = 4; L >= 0; --L) {
          const float x = acc[L][nt][h] * (p2 * (L == 4 ? 0x1p-32f : L == 3 ? 0x1p-24f : L == 2 ? 0x1p-16f : L == 1 ? 0x1p-8f : 1.f));
          float sn, ee;
          eft_two_sum(s, x, sn, ee);
          s = sn;
          err += ee;
        }
        Y[row + (int64_t)j * ldy] = st_as<SO>(df_norm(s, err));
      }
    }
    }
    // everyone is done reading this buffer (generic proxy) before a bulk copy
    // (async proxy) refills it
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (nbuf == 1 && tid == 0 && tma && nxt < nfull) issue(nxt, 0);
  }
  if (!ok && tid == 0) {
    if (status) atomicOr(status, DEV_ERR_TIMEOUT);
    // let the copies already issued land before the CTA leaves (bounded waits)
    for (int b = 0; b < 2; ++b)
      for (; nwaited[b] < nissued[b]; ++nwaited[b])
        if (!oz_wait(&bar[b], (uint32_t)(nwaited[b] & 1))) break;
  }
}

}  // namespace

bool tsmm_oz_ok(Fmt in, Fmt comp, Fmt vfmt, Fmt out, int m_max, int r_max) {
  // "tsmm.oz": 0 never, 1 where the float-float kernel is clearly ALU-bound, 2 whenever
  // it applies.  Float-float costs ~12 FP32 instructions per m r product against
  // 8 (m + r) bytes of traffic per row; with GB300's FP32 rate over its HBM bandwidth that
  // is ALU-bound from m r / (m + r) ~ 3.4 on.  Measured on GB300: 2^27 x 8 -> 5 (ratio
  // 3.1) 5.7 ms float-float vs 11.4 ms here; 2^24 x 40 -> 5 (4.4) 2.9 vs 3.1 ms;
  // 2^24 x 64 -> 10 (8.6) 6.2 vs 4.7 ms; 2^21 x 80 -> 10 (8.9) 0.96 vs 0.87 ms.
  const int mode = tune_get("tsmm.oz", 1);
  if (mode == 0) return false;
  if (m_max < 1 || m_max > OZ_MAXM || r_max < 1 || r_max > OZ_MAXR) return false;
  if (comp == Fmt::F64) {
    // the FP64-accurate form (native FP64 arithmetic): FP64 W, V and Y; "tsmm.oz64" [1].
    // Worth it wherever the FP64 pipe would do m multiply-adds per output (m >= 16).
    return tune_get("tsmm.oz64", 1) != 0 && m_max >= 16 && in == Fmt::F64 && vfmt == Fmt::F64 &&
           out == Fmt::F64;
  }
  if (mode == 1 && (m_max < 16 || m_max * r_max < 6 * (m_max + r_max))) return false;
  if (comp != Fmt::DF) return false;
  const bool types = (in == Fmt::F64 && vfmt == Fmt::DF && out == Fmt::DF) ||
                     (in == Fmt::DF && vfmt == Fmt::DF && out == Fmt::DF) ||
                     (in == Fmt::F64 && vfmt == Fmt::F64 && out == Fmt::F64);
  return types;
}

size_t tsmm_oz_smem(int m_max, int r_max, int nbuf, bool x64) {
  const int nt = r_max <= 8 ? 1 : (r_max <= 16 ? 2 : 4);  // per launch (r_max > 32: 4)
  const int kt = (m_max + 15) / 16;
  const int nd = x64 ? 7 : 6;
  return nbuf * (size_t)m_max * OZ_CS + (size_t)kt * nd * nt * 32 * sizeof(uint2) + 8 * nt * sizeof(int) + 16;
}

namespace {
template <int NT, class S, class VS, class SO, bool X64 = false>
cudaError_t run_oz(const TsmmCfg& c, const void* W, int64_t rows, int64_t ld, const int* m_dev,
                   const void* V, int ldV, const int* r_dev, void* Y, int64_t ldy, int* status,
                   cudaStream_t s) {
  auto k = k_tsmm_oz<NT, X64, S, VS, SO>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem);
  if (e != cudaSuccess) return e;
  // up to 32 columns per launch: r_max > 32 takes a second launch for columns 32..r-1
  for (int col0 = 0; col0 < c.r_max; col0 += 8 * NT) {
    k<<<(unsigned)c.ctas, OZ_THREADS, c.smem, s>>>(static_cast<const S*>(W), rows, ld, m_dev, c.m_max,
                                                   static_cast<const VS*>(V), ldV, r_dev, c.r_max,
                                                   static_cast<SO*>(Y), ldy, c.m_max, c.r_max, c.rc,
                                                   status, c.xr, col0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <class S, class VS, class SO, bool X64 = false>
cudaError_t run_oz_nt(const TsmmCfg& c, const void* W, int64_t rows, int64_t ld, const int* m_dev,
                      const void* V, int ldV, const int* r_dev, void* Y, int64_t ldy, int* status,
                      cudaStream_t s) {
  if (c.r_max <= 8) return run_oz<1, S, VS, SO, X64>(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
  if (c.r_max <= 16) return run_oz<2, S, VS, SO, X64>(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
  return run_oz<4, S, VS, SO, X64>(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
}
}  // namespace

cudaError_t launch_tsmm_oz(const TsmmCfg& c, const void* W, int64_t rows, int64_t ld,
                           const int* m_dev, const void* V, int ldV, const int* r_dev, void* Y,
                           int64_t ldy, int* status, cudaStream_t s) {
  if (c.comp == Fmt::F64 && c.in == Fmt::F64 && c.vfmt == Fmt::F64 && c.out == Fmt::F64)
    return run_oz_nt<double, double, double, true>(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
  if (c.in == Fmt::F64 && c.vfmt == Fmt::DF && c.out == Fmt::DF)
    return run_oz_nt<double, df, df>(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
  if (c.in == Fmt::DF && c.vfmt == Fmt::DF && c.out == Fmt::DF)
    return run_oz_nt<df, df, df>(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
  if (c.in == Fmt::F64 && c.vfmt == Fmt::F64 && c.out == Fmt::F64)
    return run_oz_nt<double, double, double>(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
  return cudaErrorInvalidValue;
}

}  // namespace tt
