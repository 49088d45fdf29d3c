// tsqr_col.cuh -- column-owned TSQR level kernel (Alg. 6 panels, Sec. 3.2).
//
// One CTA folds a contiguous range of row panels into one triangle R (a flat
// tree) and writes R as one block of the stacked output, like the other level
// kernels.  The layout differs from the row-group CTA kernel:
//
//   column k of the panel belongs to warp  k mod NW  (slot c = k / NW);
//   lane l of that warp holds rows  l + 32 q  (q < PRL) of it, PR = 32 PRL rows.
//
// Panel values are updated without renormalising the float-float pairs
// (fnmac_nr) and dot products use lazy accumulators (lz_fmac); the pivot
// column is renormalised before it is published, so every product has one
// normalised factor (a product of two pairs drops lo*lo).
//
// So the dot products of Alg. 6 (pivot column with column k) never leave the
// warp that owns column k: a butterfly reduce-scatter over the 32 lanes sums
// all of the warp's active columns at once (about one add per column per lane).
// Every entry R_jk of the triangle is read and written by the owner of column
// k only.  The only data that crosses warps is the pivot column M_j with its
// reflector (pivot entry R_jj - alpha and 1/t), which the owner of column j
// publishes in one of two shared-memory slots.  The owner of column j+1 builds
// that slot one step early (look-ahead): inside step j it applies reflector j
// to column j+1 first, forms D_{j+1}, alpha, the pivot entry and 1/t, and
// publishes them while the other warps are still updating their columns.
//
// There is no CTA-wide barrier per column: each slot has a FULL mbarrier (one
// arrival: the publisher) and an EMPTY mbarrier (one arrival per warp, after
// the warp has copied the slot into registers).  A warp starts step j as soon
// as pivot j is published, and the publisher of pivot g waits only until every
// warp has read pivot g-2 (the previous content of its slot), so warps drift
// apart by up to two columns and the look-ahead chain hides behind the other
// warps' updates.  Every wait is bounded (kWaitCycles); a warp whose wait runs
// out sets DEV_ERR_TIMEOUT and stops, and the others then run out too.
//
// The column-step code is unrolled over the slot block JB = j / NW so that the
// set of active slots (JB .. CLW-1) is known at compile time and the
// dot-product chains of different columns interleave.
#pragma once
#include "tsqr_kernels.cuh"

namespace tt {
namespace colk {

__device__ __forceinline__ int prow(int j, int mstr) { return j * mstr - (j * (j - 1)) / 2; }

__host__ __device__ constexpr int pow2ceil(int a) { return a <= 1 ? 1 : 2 * pow2ceil((a + 1) / 2); }
__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }

// ---- mbarrier helpers (shared::cta) ------------------------------------------------
__device__ __forceinline__ uint32_t sptr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sptr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(sptr(b))
               : "memory");
}
// try_wait suspends the warp until the phase completes or the hint (ns) elapses, so a
// waiting warp does not take issue slots from the others
__device__ __forceinline__ bool mbar_test(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(sptr(b)), "r"(parity), "r"(1000000u)
      : "memory");
  return ok != 0;
}
// wait for the completion of the phase with the given parity; false once `limit` SM clock
// cycles passed (kWaitCycles, about 2 s, in the kernels)
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity, long long limit = kWaitCycles) {
  if (mbar_test(b, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_test(b, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

struct Sync {
  uint64_t* full;   // [2]
  uint64_t* empty;  // [2]
  int* status;
  int* abort;       // shared flag: some warp gave up
};

__device__ __forceinline__ bool give_up(const Sync& S, int lane) {
  if (lane == 0) {
    if (S.status) atomicOr(S.status, DEV_ERR_TIMEOUT);
    *reinterpret_cast<volatile int*>(S.abort) = 1;
  }
  return false;
}

// sum over the 32 lanes (every lane gets it), with lazy float-float additions
template <class C>
__device__ __forceinline__ C warp_allsum(C v) {
  auto z = lz(v);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) z = lz_add(z, shfl_xor(z, o));
  return lz_fin(z);
}

template <class C>
__device__ __forceinline__ C sel(bool p, C a, C b) { return p ? a : b; }

// Reduce-scatter of V per-lane partial sums over the 32 lanes: afterwards the
// result holds, in every lane, the full sum of slot  lane >> (5 - log2 V).
template <int V, class C>
__device__ __forceinline__ C butterfly(const C (&s)[V], int lane) {
  decltype(lz(s[0])) z[V];
#pragma unroll
  for (int i = 0; i < V; ++i) z[i] = lz(s[i]);
#pragma unroll
  for (int lev = 0; (V >> lev) > 1; ++lev) {
    const int half = (V >> lev) / 2;
    const int bit = 16 >> lev;
    const bool up = (lane & bit) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const auto send = sel(up, z[i], z[i + half]);
      const auto keep = sel(up, z[i + half], z[i]);
      z[i] = lz_add(keep, shfl_xor(send, bit));
    }
  }
#pragma unroll
  for (int bit = 16 >> ilog2(V); bit > 0; bit >>= 1) z[0] = lz_add(z[0], shfl_xor(z[0], bit));
  return lz_fin(z[0]);
}

// x . y over this lane's PRL rows: two interleaved lazy float-float chains
template <int PRL, class C>
__device__ __forceinline__ C dot_rows(const C (&x)[PRL], const C (&y)[PRL]) {
  auto a0 = lz(Tr<C>::zero());
  auto a1 = lz(Tr<C>::zero());
#pragma unroll
  for (int q = 0; q + 1 < PRL; q += 2) {
    a0 = lz_fmac(x[q], y[q], a0);
    a1 = lz_fmac(x[q + 1], y[q + 1], a1);
  }
  if constexpr (PRL % 2) a0 = lz_fmac(x[PRL - 1], y[PRL - 1], a0);
  return lz_fin(lz_add(a0, a1));
}

// Reflector of column jn (Alg. 6) from the column's panel values x (after all
// earlier reflectors of this panel) and R_{jn,jn}; publishes x, the pivot entry
// R_jj - alpha and 1/t as pivot number g (slot g & 1) and stores R_{jn,jn} = alpha.
template <int PRL, class C>
__device__ __forceinline__ bool publish_r(const C (&x)[PRL], C rjj, int jn, uint32_t g, C* R,
                                          int mstr, C* slots, const Sync& S, int lane, C eps) {
  constexpr int PR = 32 * PRL;
  const int rn = prow(jn, mstr);
  const C D = warp_allsum(dot_rows<PRL>(x, x));
  const Refl<C> h = householder(rjj, D, eps);
  const C alpha = h.alpha, pivn = h.piv, rtn = h.rt;
  const int sl = g & 1;
  const uint32_t use = g >> 1;
  // the slot's previous pivot (g - 2) must have been read by every warp
  if (use >= 1 && !mbar_wait(&S.empty[sl], (use - 1) & 1)) return give_up(S, lane);
  C* slot = slots + sl * (PR + 2);
#pragma unroll
  for (int q = 0; q < PRL; ++q) slot[lane + 32 * q] = x[q];
  if (lane == 0) {
    slot[PR] = pivn;
    slot[PR + 1] = rtn;
    R[rn] = alpha;
  }
  __syncwarp();
  if (lane == 0) mbar_arrive(&S.full[sl]);
  return true;
}
template <int PRL, class C>
__device__ __forceinline__ bool publish(const C (&x)[PRL], int jn, uint32_t g, C* R, int mstr,
                                        C* slots, const Sync& S, int lane, C eps) {
  return publish_r<PRL>(x, R[prow(jn, mstr)], jn, g, R, mstr, slots, S, lane, eps);
}

// One column step j = JB * NW + jj for warp w; pivot j is pivot number g.
template <int JB, int NW, int CLW, int PRL, class C>
__device__ __forceinline__ bool col_step(C (&a)[CLW][PRL], int j, int jj, uint32_t g, int m, int w,
                                         int lane, C* R, int mstr, C* slots, const Sync& S, C eps) {
  constexpr int PR = 32 * PRL;
  constexpr int A = CLW - JB;       // slots JB .. CLW-1 may still be active
  constexpr int V = pow2ceil(A);
  constexpr int L = ilog2(V);
  // take pivot j
  const int sl = g & 1;
  if (!mbar_wait(&S.full[sl], (g >> 1) & 1)) return give_up(S, lane);
  const C* slot = slots + sl * (PR + 2);
  C pv[PRL];
#pragma unroll
  for (int q = 0; q < PRL; ++q) pv[q] = slot[lane + 32 * q];
  const C piv = slot[PR];
  const C rt = slot[PR + 1];
  __syncwarp();
  if (lane == 0) mbar_arrive(&S.empty[sl]);
  const int rj = prow(j, mstr);

  // look-ahead: the owner of column j+1 applies reflector j to it and publishes reflector j+1
  if (j + 1 < m && w == (jj + 1) % NW) {
    const bool same = jj + 1 < NW;  // column j+1 sits in slot JB, else in slot JB+1
    C x[PRL];
#pragma unroll
    for (int q = 0; q < PRL; ++q) x[q] = a[JB][q];
    if constexpr (JB + 1 < CLW) {
      if (!same) {
#pragma unroll
        for (int q = 0; q < PRL; ++q) x[q] = a[JB + 1][q];
      }
    }
    const C r = R[rj + 1];
    const C d = warp_allsum(dot_rows<PRL>(pv, x));
    const C c = mul(fmac(piv, r, d), rt);
    if (lane == 0) R[rj + 1] = fnmac(c, piv, r);
#pragma unroll
    for (int q = 0; q < PRL; ++q) x[q] = renorm(fnmac_nr(c, pv[q], x[q]));
    if (same) {
#pragma unroll
      for (int q = 0; q < PRL; ++q) a[JB][q] = x[q];
    }
    if constexpr (JB + 1 < CLW) {
      if (!same) {
#pragma unroll
        for (int q = 0; q < PRL; ++q) a[JB + 1][q] = x[q];
      }
    }
    if (!publish<PRL>(x, j + 1, g + 1, R, mstr, slots, S, lane, eps)) return false;
  }

  // dot products of the pivot with every column k > j+1 this warp owns
  const bool first_live = w > jj + 1;  // slot JB holds a column k > j+1
  C s[V];
#pragma unroll
  for (int i = 0; i < V; ++i) s[i] = Tr<C>::zero();
  if (first_live) s[0] = dot_rows<PRL>(pv, a[JB]);
#pragma unroll
  for (int c = JB + 1; c < CLW; ++c) s[c - JB] = dot_rows<PRL>(pv, a[c]);
  const C tot = butterfly<V>(s, lane);
  // coefficient c_k = (piv R_jk + M_j . M_k) / t for this lane's slot; row j of R
  const int idx = lane >> (5 - L);
  const int k = w + NW * (JB + idx);
  const bool act = idx < A && k > j + 1 && k < m;
  C ck = Tr<C>::zero();
  if (act) {
    const C rjk = R[rj + (k - j)];
    ck = mul(fmac(piv, rjk, tot), rt);
    if ((lane & ((1 << (5 - L)) - 1)) == 0) R[rj + (k - j)] = fnmac(ck, piv, rjk);
  }
  // rank-1 update of the owned columns (an inactive slot has c_k = 0, an exact no-op)
  if (first_live) {
    const C cb = shfl_idx(ck, 0);
#pragma unroll
    for (int q = 0; q < PRL; ++q) a[JB][q] = fnmac_nr(cb, pv[q], a[JB][q]);
  }
#pragma unroll
  for (int c = JB + 1; c < CLW; ++c) {
    const C cb = shfl_idx(ck, (c - JB) << (5 - L));
#pragma unroll
    for (int q = 0; q < PRL; ++q) a[c][q] = fnmac_nr(cb, pv[q], a[c][q]);
  }
  return true;
}

template <int JB, int NW, int CLW, int PRL, class C>
__device__ __forceinline__ bool col_blocks(C (&a)[CLW][PRL], uint32_t g0, int m, int w, int lane,
                                           C* R, int mstr, C* slots, const Sync& S, C eps) {
  if constexpr (JB < CLW) {
    if (JB * NW < m) {
#pragma unroll 1
      for (int jj = 0; jj < NW; ++jj) {
        const int j = JB * NW + jj;
        if (j >= m) break;
        if (!col_step<JB, NW, CLW, PRL, C>(a, j, jj, g0 + j, m, w, lane, R, mstr, slots, S, eps))
          return false;
      }
      return col_blocks<JB + 1, NW, CLW, PRL, C>(a, g0, m, w, lane, R, mstr, slots, S, eps);
    }
  }
  return true;
}

}  // namespace colk

// R is packed (upper triangle, row-major) with row stride mmax: row j holds
// columns j..mmax-1 from offset j*mmax - j(j-1)/2.  Shared memory: four
// mbarriers and an abort flag (64 bytes), R (unless RG_MEM, where R is a
// per-CTA slice of Rglob that stays in L2), then two pivot slots of PR + 2 values.
template <int NW, int CLW, int PRL, int MINB, bool RG_MEM, class C, class S, class RO>
__global__ void __launch_bounds__(NW * 32, MINB)
k_tsqr_col(const S* __restrict__ W, int64_t rows, int64_t ld, const int* __restrict__ m_ptr,
           int m_val, int mmax, RO* __restrict__ Rout, int64_t ldR, int mb, int64_t npanels,
           C* __restrict__ Rglob, int* status, XRange* xr, int xfix) {
  constexpr int PR = 32 * PRL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  XRead<C, S> rd;
  if (!xr_begin(xr, xfix, rd)) return;
  const int m = m_ptr ? *m_ptr : m_val;
  if (m < 1 || m > NW * CLW || m > mmax || m > mb || blockDim.x != NW * 32) {
    if (threadIdx.x == 0 && status) atomicOr(status, DEV_ERR_SHAPE);
    return;
  }
  const int mstr = mmax;
  const size_t tri = (size_t)mmax * (mmax + 1) / 2;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  int* abort_flag = reinterpret_cast<int*>(smem_raw + 32);
  C* base = reinterpret_cast<C*>(smem_raw + 64);
  C* R = RG_MEM ? Rglob + (size_t)blockIdx.x * tri : base;
  C* slots = RG_MEM ? base : base + tri;
  const int tid = threadIdx.x, nt = NW * 32;
  const int w = tid >> 5, lane = tid & 31;
  colk::Sync sy{bars, bars + 2, status, abort_flag};
  if (tid == 0) {
    colk::mbar_init(&bars[0], 1);
    colk::mbar_init(&bars[1], 1);
    colk::mbar_init(&bars[2], NW);
    colk::mbar_init(&bars[3], NW);
    *abort_flag = 0;
  }
  for (size_t i = tid; i < tri; i += nt) R[i] = Tr<C>::zero();
  __syncthreads();
  const C eps = Tr<C>::eps();
  const int64_t p0 = (int64_t)blockIdx.x * npanels / gridDim.x;
  const int64_t p1 = (int64_t)(blockIdx.x + 1) * npanels / gridDim.x;
  uint32_t g = 0;  // running pivot number of this CTA (m per panel)
  for (int64_t p = p0; p < p1; ++p, g += (uint32_t)m) {
    C a[CLW][PRL];
    {
      // every load of the panel first, then the conversions (which may branch)
      S raw[CLW][PRL];
#pragma unroll
      for (int c = 0; c < CLW; ++c) {
        const int k = w + NW * c;
#pragma unroll
        for (int q = 0; q < PRL; ++q) {
          const int64_t row = p * PR + lane + 32 * q;
          raw[c][q] = (row < rows && k < m) ? W[row + (int64_t)k * ld] : S{};
        }
      }
#pragma unroll
      for (int c = 0; c < CLW; ++c) {
        const int k = w + NW * c;
#pragma unroll
        for (int q = 0; q < PRL; ++q) {
          const int64_t row = p * PR + lane + 32 * q;
          a[c][q] = (row < rows && k < m) ? rd(raw[c][q]) : Tr<C>::zero();
        }
      }
    }
    // warm L2 with the next panel of this CTA (two requests per 256-byte column segment)
    if (p + 1 < p1 && (lane & 15) == 0) {
#pragma unroll
      for (int c = 0; c < CLW; ++c) {
        const int k = w + NW * c;
#pragma unroll
        for (int q = 0; q < PRL; ++q) {
          const int64_t row = (p + 1) * PR + lane + 32 * q;
          if (row < rows && k < m) {
            const S* ptr = W + row + (int64_t)k * ld;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
          }
        }
      }
    }
    // reflector of column 0 from its owner (warp 0), then the column steps
    if (w == 0 && !colk::publish<PRL>(a[0], 0, g, R, mstr, slots, sy, lane, eps)) break;
    if (!colk::col_blocks<0, NW, CLW, PRL, C>(a, g, m, w, lane, R, mstr, slots, sy, eps)) break;
  }
  __syncthreads();
  if (*reinterpret_cast<volatile int*>(abort_flag)) return;
  xr_end(xr, xfix, rd);
  for (int idx = tid; idx < mb * m; idx += nt) {
    const int i = idx % mb, k = idx / mb;
    C v = Tr<C>::zero();
    if (i < m && i <= k) v = R[colk::prow(i, mstr) + (k - i)];
    Rout[(int64_t)blockIdx.x * mb + i + (int64_t)k * ldR] = st_as<RO>(v);
  }
}

namespace colk {

template <int NW, int CLW, int PRL, int MINB, class C, class S, class RO>
cudaError_t run_col(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev, void* Rout,
                    int64_t ldR, int* status, cudaStream_t s) {
  auto kern = k_tsqr_col<NW, CLW, PRL, MINB, false, C, S, RO>;
  if (L.smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<(unsigned)L.ctas, NW * 32, L.smem, s>>>(static_cast<const S*>(W), L.rows, ld, m_dev, L.mval,
                                                L.mmax, static_cast<RO*>(Rout), ldR, L.mb, L.panels,
                                                nullptr, status, L.xr, L.xfix);
  return cudaGetLastError();
}

// default layouts (ids 0-4) of the 8-byte arithmetics
template <class C, class S, class RO>
cudaError_t run_default(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev, void* Rout,
                        int64_t ldR, int* status, cudaStream_t s) {
  switch (L.cfg) {
    case 0: return run_col<16, 2, 8, 1, C, S, RO>(L, W, ld, m_dev, Rout, ldR, status, s);
    case 1: return run_col<16, 4, 8, 1, C, S, RO>(L, W, ld, m_dev, Rout, ldR, status, s);
    case 2: return run_col<16, 5, 4, 1, C, S, RO>(L, W, ld, m_dev, Rout, ldR, status, s);
    case 3: return run_col<16, 8, 4, 1, C, S, RO>(L, W, ld, m_dev, Rout, ldR, status, s);
    case 4: return run_col<20, 8, 3, 1, C, S, RO>(L, W, ld, m_dev, Rout, ldR, status, s);
    default: return cudaErrorInvalidValue;
  }
}

// defaults and the autotuner's alternatives (ids 5-9) of the float-float arithmetic
template <class S>
cudaError_t run_df_tuned(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev, void* Rout,
                         int64_t ldR, int* status, cudaStream_t s) {
  switch (L.cfg) {
    case 5: return run_col<12, 6, 8, 1, df, S, df>(L, W, ld, m_dev, Rout, ldR, status, s);
    case 6: return run_col<16, 4, 4, 1, df, S, df>(L, W, ld, m_dev, Rout, ldR, status, s);
    case 7: return run_col<16, 5, 6, 1, df, S, df>(L, W, ld, m_dev, Rout, ldR, status, s);
    case 8: return run_col<8, 8, 4, 2, df, S, df>(L, W, ld, m_dev, Rout, ldR, status, s);
    case 9: return run_col<8, 4, 8, 2, df, S, df>(L, W, ld, m_dev, Rout, ldR, status, s);
    default: return run_default<df, S, df>(L, W, ld, m_dev, Rout, ldR, status, s);
  }
}

}  // namespace colk

// upper levels (float-float) and the native FP64 form, in their own translation unit
cudaError_t tsqr_col_upper(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev,
                           void* Rout, int64_t ldR, int* status, cudaStream_t s);

}  // namespace tt
