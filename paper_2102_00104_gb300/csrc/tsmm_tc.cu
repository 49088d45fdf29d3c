// tsmm_tc.cu -- Y = W V(:, 0:r) of Alg. 2 line 11 for the float-float form on the fifth-
// generation tensor cores (tcgen05): the same Ozaki splitting as tsmm_oz.cu (six bf16-exact
// digits per value, one exponent per row of W and per column of V, levels 2..7 summed
// exactly in FP32), with the digit products issued as tcgen05.mma by one thread into six
// FP32 level accumulators in tensor memory.
//
// A CTA of 512 threads takes 128-row tiles of W (M = 128 of one MMA).  The tile comes into
// shared memory by bulk copies (one per column, on an mbarrier); thread (i, q) = (row,
// quarter) finds row i's largest exponent with the other three quarters (through shared
// memory) and writes the row's digits for k-groups q, q+4, ... straight into six digit
// planes in the canonical
// K-major layout of the MMA (core matrices of 8 rows x 16 bytes: the core of row group g
// and k-group kg at g * 256 kt + kg * 128 bytes; the next core along K at +128 bytes, the
// next along M at +256 kt).  V's digits sit in six planes of the same layout (N = 16 or 32
// rows, contiguous, so that planes b = 0..5-a form one operand of N = 16 (6 - a) rows).
// Thread 0 then issues, per k-step of 16, one tcgen05.mma.kind::f16 per digit a of W
// (bf16 in, FP32 accumulate, M = 128, N = 16 (6 - a)) against V's digits 0..5-a, into
// its own block of tensor-memory columns (336 of 512: the block of (a, b) holds the
// product of digits a and b), commits them to an mbarrier, and starts the bulk copy of
// the next tile into the freed tile buffer.  The products are read back with tcgen05.ld
// (warp w reads lanes 32 (w mod 4) .. of tensor memory, output columns 4 (w / 4) ..),
// the ones of a level a + b are summed (exactly: the level's sum stays below 2^24), and
// the levels are added in float-float from the smallest, as in tsmm_oz.cu.
//
// Every wait is bounded (kWaitCycles); a CTA whose wait runs out sets DEV_ERR_TIMEOUT,
// lets the copies it issued land (bounded), frees its tensor memory and returns.
#include <algorithm>

#include "ozaki.cuh"

namespace tt {

namespace {

using namespace ozk;

constexpr int TC_TR = 128;              // rows per tile: M of one tcgen05.mma
constexpr int TC_THREADS = 512;         // four threads per row
constexpr int TC_CS = TC_TR * 8;        // bytes per staged column of W
constexpr int TC_MAXM = 80;             // k-steps <= 5; one level summed over k < 2^24

// shared-memory descriptor: K-major, no swizzle, next core along K at +128 bytes, next
// 8-row group at +sbo bytes; descriptor version 1 (bits 46-47) of this GPU family
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)(128u >> 4) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::f16: D FP32, A and B bf16, both K-major, M = 128, N = nn
__host__ __device__ constexpr uint32_t tc_idesc(int nn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(nn >> 3) << 17) | ((128u >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t idesc,
                                       uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtm),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

template <int CPW>
__device__ __forceinline__ void tc_ld(uint32_t taddr, float (&v)[CPW]);
template <>
__device__ __forceinline__ void tc_ld<4>(uint32_t taddr, float (&v)[4]) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// NN = 16 output columns (r <= 16).  Shared memory: the W tile (m_max columns of TC_CS
// bytes), six A digit planes (128 x 16 kt bf16 each), six B digit planes (NN x 16 kt bf16
// each, contiguous), the row and column exponents, two mbarriers, the TMEM address.
template <int NN, class S, class VS, class SO>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_tsmm_tc(const S* __restrict__ W, int64_t rows, int64_t ld, const int* __restrict__ m_ptr,
          int m_val, const VS* __restrict__ V, int ldV, const int* __restrict__ r_ptr, int r_val,
          SO* __restrict__ Y, int64_t ldy, int m_max, int r_max, int* status,
          const XRange* xr) {
  constexpr int NL = 6;                // levels 2..7
  constexpr int CPW = NN / 4;          // output columns per warp in the read-back
  constexpr uint32_t TMCOLS = 512;     // 21 blocks of NN columns (336)
  static_assert(NN == 16, "one MMA per digit of W needs 21 NN-column blocks within 512");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int m = m_ptr ? *m_ptr : m_val;
  const int r = r_ptr ? *r_ptr : r_val;
  if (m < 1 || m > m_max || m_max > TC_MAXM || r < 1 || r > r_max || r > m || r > NN ||
      blockDim.x != TC_THREADS) {
    if (threadIdx.x == 0 && status) atomicOr(status, DEV_ERR_SHAPE);
    return;
  }
  const int kt = (m_max + 15) / 16;
  const uint32_t sbo = 256u * (uint32_t)kt;       // next 8-row group of a digit plane
  const size_t aplane = (size_t)TC_TR * 32 * kt;  // 128 rows x 16 kt bf16
  const size_t bplane = (size_t)NN * 32 * kt;
  unsigned char* Wt = smem_raw;
  unsigned char* Ap = Wt + (size_t)m_max * TC_CS;   // 1024-byte aligned
  unsigned char* Bp = Ap + NL * aplane;
  int* Erow = reinterpret_cast<int*>(Bp + NL * bplane);
  int* Fe = Erow + TC_TR;
  uint64_t* bar = reinterpret_cast<uint64_t*>(Fe + NN);  // [0] tile copy, [1] MMAs
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  // row i of the tile, quarter q of its k-groups: a warp holds 32 consecutive rows of one
  // quarter, so its reads of the tile and its digit writes are contiguous
  const int i = tid & (TC_TR - 1), q = tid >> 7;
  __shared__ unsigned s_key[4][TC_TR];

  const int64_t ntiles = (rows + TC_TR - 1) / TC_TR;
  const int64_t nfull = rows / TC_TR;
  const bool tma = (ld % 2 == 0) && ((reinterpret_cast<uintptr_t>(W) & 15) == 0);
  if (tid == 0) {
    oz_bar_init(&bar[0]);
    oz_bar_init(&bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(TMCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // column exponents of V(:, 0:r)
  for (int j = w; j < NN; j += TC_THREADS / 32) {
    int be = 0;
    if (j < r)
      for (int k = lane; k < m; k += 32) be = max(be, oz_bexp(ld_as<df>(V[k + (size_t)j * ldV])));
    for (int o = 16; o; o >>= 1) be = max(be, __shfl_xor_sync(0xffffffffu, be, o));
    if (lane == 0) Fe[j] = be;
  }
  __syncthreads();
  // V's digit planes: row n of plane b holds column n of V's b-th digits along k
  for (int idx = tid; idx < NN * 2 * kt; idx += TC_THREADS) {
    const int n = idx % NN, kg = idx / NN;
    const float sc = oz_inv_scale(Fe[n]);
    float d[8][6];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int k = 8 * kg + c;
      const df v = (n < r && k < m) ? ld_as<df>(V[k + (size_t)n * ldV]) : Tr<df>::zero();
      oz_digits(v, sc, d[c]);
    }
    const size_t off = (size_t)(n >> 3) * sbo + (size_t)kg * 128 + (size_t)(n & 7) * 16;
#pragma unroll
    for (int b = 0; b < 6; ++b)
      *reinterpret_cast<uint4*>(Bp + b * bplane + off) =
          make_uint4(oz_pack(d[0][b], d[1][b]), oz_pack(d[2][b], d[3][b]),
                     oz_pack(d[4][b], d[5][b]), oz_pack(d[6][b], d[7][b]));
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  // first tensor-memory column of the products of W's digit a (blocks b = 0..5-a)
  auto colbase = [](int a) { return NN * (6 * a - a * (a - 1) / 2); };

  int nissued = 0, nwaited = 0;  // tile copies (thread 0's count, for a clean exit)
  auto issue = [&](int64_t tile) {
    const int64_t r0 = tile * TC_TR;
    oz_expect(&bar[0], (uint32_t)(m * TC_TR * 8));
    for (int k = 0; k < m; ++k)
      oz_bulk(Wt + (size_t)k * TC_CS, W + r0 + (int64_t)k * ld, TC_TR * 8, &bar[0]);
    ++nissued;
  };
  int64_t tile = blockIdx.x;
  if (tid == 0 && tma && tile < nfull) issue(tile);
  bool ok = true;
  for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
    const bool bulk = tma && tile < nfull;
    const int64_t r0 = tile * TC_TR;
    if (bulk) {
      // every earlier tile of this CTA was a full one: this is the copy barrier's it-th phase
      if (!oz_wait(&bar[0], (uint32_t)(it & 1))) ok = false;
      else if (tid == 0) ++nwaited;
    } else {
      for (int idx = tid; idx < m * TC_TR; idx += TC_THREADS) {
        const int ii = idx % TC_TR, k = idx / TC_TR;
        const int64_t row = r0 + ii;
        reinterpret_cast<S*>(Wt + (size_t)k * TC_CS)[ii] =
            row < rows ? W[row + (int64_t)k * ld] : oz_zero<S>();
      }
      __syncthreads();
    }
    if (__syncthreads_or(!ok)) {
      ok = false;
      break;
    }
    // row i's exponent: the largest over k < m, from the four quarters' k-groups
    unsigned key = 0;
    for (int kg = q; kg < 2 * kt; kg += 4)
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int k = 8 * kg + c;
        if (k < m) key = max(key, oz_key(reinterpret_cast<const S*>(Wt + (size_t)k * TC_CS)[i]));
      }
    s_key[q][i] = key;
    __syncthreads();
    key = max(max(s_key[0][i], s_key[1][i]), max(s_key[2][i], s_key[3][i]));
    XRead<df, S> rd;  // W read as W 2^-sh (FP64 input of the float-float form)
    rd.set(xr ? xr->k : 0, xr != nullptr);
    const int be = oz_bexp_of(key, (S*)nullptr, rd.sh);
    if (q == 0) Erow[i] = be;
    const float sc = oz_inv_scale(be);
    // digits of row i, k-groups q, q+4, ...: one 16-byte core-matrix row per plane
    const size_t rowoff = (size_t)(i >> 3) * sbo + (size_t)(i & 7) * 16;
    for (int kg = q; kg < 2 * kt; kg += 4) {
      float d[8][6];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int k = 8 * kg + c;
        const df x = k < m ? rd(reinterpret_cast<const S*>(Wt + (size_t)k * TC_CS)[i])
                           : Tr<df>::zero();
        oz_digits(x, sc, d[c]);
      }
#pragma unroll
      for (int a = 0; a < 6; ++a)
        *reinterpret_cast<uint4*>(Ap + a * aplane + rowoff + (size_t)kg * 128) =
            make_uint4(oz_pack(d[0][a], d[1][a]), oz_pack(d[2][a], d[3][a]),
                       oz_pack(d[4][a], d[5][a]), oz_pack(d[6][a], d[7][a]));
    }
    // digits visible to the tensor cores; the tile buffer is free for the next copy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      const uint32_t a0 = smem_u32(Ap), b0 = smem_u32(Bp);
      for (int kk = 0; kk < kt; ++kk)
        for (int a = 0; a < 6; ++a) {
          const uint64_t ad = tc_desc(a0 + (uint32_t)(a * aplane) + 256u * kk, sbo);
          const uint64_t bd = tc_desc(b0 + 256u * kk, sbo);  // V's digit planes 0 .. 5 - a
          tc_mma(tmem + (uint32_t)colbase(a), ad, bd, tc_idesc(NN * (6 - a)), kk > 0 ? 1u : 0u);
        }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_u32(&bar[1]))
          : "memory");
      const int64_t nxt = tile + gridDim.x;
      if (tma && nxt < nfull) issue(nxt);
    }
    // wait for this tile's products, read the six levels back, add them up
    if (!oz_wait(&bar[1], (uint32_t)(it & 1))) ok = false;
    tc_fence_after();
    if (ok) {
      const int wq = w & 3, cg = w >> 2;
      float acc[NL][CPW];
#pragma unroll
      for (int L = 0; L < NL; ++L)
#pragma unroll
        for (int cn = 0; cn < CPW; ++cn) acc[L][cn] = 0.f;
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        // the products of digit a with V's digits 0 .. 5-a: all loads, then one wait
        float v[6][CPW];
#pragma unroll
        for (int b = 0; a + b <= 5; ++b)
          tc_ld<CPW>(tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)(colbase(a) + b * NN + cg * CPW), v[b]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int b = 0; a + b <= 5; ++b)
#pragma unroll
          for (int cn = 0; cn < CPW; ++cn) acc[a + b][cn] += v[b][cn];  // exact: integers < 2^24
      }
      const int rr = 32 * wq + lane;
      const int64_t row = r0 + rr;
      const int E = Erow[rr] - 126;
#pragma unroll
      for (int cn = 0; cn < CPW; ++cn) {
        const int j = cg * CPW + cn;
        if (j >= r || row >= rows) continue;
        const float p2 = oz_pow2(E + (Fe[j] - 126) - 14);
        float s = acc[5][cn] * (p2 * 0x1p-40f), err = 0.f;
#pragma unroll
        for (int L = 4; L >= 0; --L) {
          const float x = acc[L][cn] *
                          (p2 * (L == 4 ? 0x1p-32f : L == 3 ? 0x1p-24f : L == 2 ? 0x1p-16f : L == 1 ? 0x1p-8f : 1.f));
          float sn, ee;
          eft_two_sum(s, x, sn, ee);
          s = sn;
          err += ee;
        }
        Y[row + (int64_t)j * ldy] = st_as<SO>(df_norm(s, err));
      }
    }
    tc_fence_before();
    if (__syncthreads_or(!ok)) {
      ok = false;
      break;
    }
  }
  if (!ok && tid == 0) {
    if (status) atomicOr(status, DEV_ERR_TIMEOUT);
    for (; nwaited < nissued; ++nwaited)
      if (!oz_wait(&bar[0], (uint32_t)(nwaited & 1))) break;
  }
  tc_fence_before();
  __syncthreads();
  if (w == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMCOLS)
                 : "memory");
}

size_t tc_smem(int m_max, int nn) {
  const int kt = (m_max + 15) / 16;
  return (size_t)m_max * TC_CS + 6 * (size_t)TC_TR * 32 * kt + 6 * (size_t)nn * 32 * kt +
         TC_TR * sizeof(int) + nn * sizeof(int) + 2 * sizeof(uint64_t) + 16;
}

template <int NN, class S, class VS, class SO>
cudaError_t run_tc(const TsmmCfg& c, const void* W, int64_t rows, int64_t ld, const int* m_dev,
                   const void* V, int ldV, const int* r_dev, void* Y, int64_t ldy, int* status,
                   cudaStream_t s) {
  auto k = k_tsmm_tc<NN, S, VS, SO>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)c.ctas, TC_THREADS, c.smem, s>>>(static_cast<const S*>(W), rows, ld, m_dev, c.m_max,
                                                 static_cast<const VS*>(V), ldV, r_dev, c.r_max,
                                                 static_cast<SO*>(Y), ldy, c.m_max, c.r_max, status,
                                                 c.xr);
  return cudaGetLastError();
}

template <class S, class VS, class SO>
cudaError_t run_tc_nn(const TsmmCfg& c, const void* W, int64_t rows, int64_t ld, const int* m_dev,
                      const void* V, int ldV, const int* r_dev, void* Y, int64_t ldy, int* status,
                      cudaStream_t s) {
  return run_tc<16, S, VS, SO>(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
}

}  // namespace

// usable for these formats and sizes ("tsmm.tc" 0 never, 1 where tsmm_oz would run)
bool tsmm_tc_ok(Fmt in, Fmt comp, Fmt vfmt, Fmt out, int m_max, int r_max) {
  if (tune_get("tsmm.tc", 0) == 0 || r_max > 32) return false;
  if (!tsmm_oz_ok(in, comp, vfmt, out, m_max, r_max)) return false;
  if (m_max > TC_MAXM || r_max > 16) return false;
  // dynamic shared memory plus the 2 KB of the static row-key array
  return tc_smem(m_max, 16) + 4 * TC_TR * sizeof(unsigned) <= 227 * 1024;
}

// at least half of an SM's shared memory: one CTA per SM, so the 512 tensor-memory
// columns a CTA allocates are always free when it starts
size_t tsmm_tc_smem(int m_max, int r_max) {
  (void)r_max;
  return std::max<size_t>(tc_smem(m_max, 16), 120 * 1024);
}

cudaError_t launch_tsmm_tc(const TsmmCfg& c, const void* W, int64_t rows, int64_t ld,
                           const int* m_dev, const void* V, int ldV, const int* r_dev, void* Y,
                           int64_t ldy, int* status, cudaStream_t s) {
  if (c.in == Fmt::F64 && c.vfmt == Fmt::DF && c.out == Fmt::DF)
    return run_tc_nn<double, df, df>(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
  if (c.in == Fmt::DF && c.vfmt == Fmt::DF && c.out == Fmt::DF)
    return run_tc_nn<df, df, df>(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
  if (c.in == Fmt::F64 && c.vfmt == Fmt::F64 && c.out == Fmt::F64)
    return run_tc_nn<double, double, double>(c, W, rows, ld, m_dev, V, ldV, r_dev, Y, ldy, status, s);
  return cudaErrorInvalidValue;
}

}  // namespace tt
