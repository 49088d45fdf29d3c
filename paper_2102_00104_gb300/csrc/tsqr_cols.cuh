// tsqr_cols.cuh -- column-owned TSQR level kernel for wide panels (m up to 512).
//
// The same scheme as k_tsqr_col (tsqr_col.cuh): warp k mod NW owns column k, the
// Alg. 6 dot products reduce inside the owning warp, the owner of column j+1 builds
// reflector j+1 one step ahead and publishes it in a double-buffered slot guarded by
// FULL/EMPTY mbarriers.  For m beyond what registers hold, the panel (PR = 32 PRL
// rows) lives in shared memory, column k at offset k * PR, and each step streams a
// warp's live columns through registers in chunks of CH columns (one butterfly
// reduce-scatter per chunk).  R, too large for shared memory, is a packed triangle per
// CTA in global memory that stays in L2; the R entries a step needs are loaded at the
// start of the step, before the dot products, so their latency overlaps the arithmetic.
#pragma once
#include "tsqr_col.cuh"

namespace tt {

template <int NW, int CH, int PRL, class C, class S, class RO>
__global__ void __launch_bounds__(NW * 32, 1)
k_tsqr_cols(const S* __restrict__ W, int64_t rows, int64_t ld, const int* __restrict__ m_ptr,
            int m_val, int mmax, RO* __restrict__ Rout, int64_t ldR, int mb, int64_t npanels,
            C* __restrict__ Rglob, int* status, XRange* xr, int xfix) {
  using namespace colk;
  constexpr int PR = 32 * PRL;
  constexpr int L = ilog2(CH);
  constexpr int MAXCH = 8;   // chunks per warp: m <= NW * CH * MAXCH
  extern __shared__ __align__(16) unsigned char smem_raw[];
  XRead<C, S> rd;
  if (!xr_begin(xr, xfix, rd)) return;
  const int m = m_ptr ? *m_ptr : m_val;
  if (m < 1 || m > mmax || m > mb || m > NW * CH * MAXCH || blockDim.x != NW * 32) {
    if (threadIdx.x == 0 && status) atomicOr(status, DEV_ERR_SHAPE);
    return;
  }
  const int mstr = mmax;
  const size_t tri = (size_t)mmax * (mmax + 1) / 2;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw);
  int* abort_flag = reinterpret_cast<int*>(smem_raw + 32);
  C* slots = reinterpret_cast<C*>(smem_raw + 64);
  C* panel = slots + 2 * (PR + 2);  // column k at panel + k * PR
  C* R = Rglob + (size_t)blockIdx.x * tri;
  const int tid = threadIdx.x, nt = NW * 32;
  const int w = tid >> 5, lane = tid & 31;
  Sync sy{bars, bars + 2, status, abort_flag};
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], NW);
    mbar_init(&bars[3], NW);
    *abort_flag = 0;
  }
  for (size_t i = tid; i < tri; i += nt) R[i] = Tr<C>::zero();
  __syncthreads();
  const C eps = Tr<C>::eps();
  const int nslot = (m - w + NW - 1) / NW;  // columns of this warp: w, w + NW, ...
  const int64_t p0 = (int64_t)blockIdx.x * npanels / gridDim.x;
  const int64_t p1 = (int64_t)(blockIdx.x + 1) * npanels / gridDim.x;
  uint32_t g = 0;
  bool ok = true;
  for (int64_t p = p0; p < p1 && ok; ++p, g += (uint32_t)m) {
    // this warp's columns of the panel into shared memory (only the owner touches them)
    for (int c = 0; c < nslot; ++c) {
      const int k = w + NW * c;
      C* col = panel + (size_t)k * PR;
#pragma unroll
      for (int q = 0; q < PRL; ++q) {
        const int64_t row = p * PR + lane + 32 * q;
        col[lane + 32 * q] = row < rows ? rd(W[row + (int64_t)k * ld]) : Tr<C>::zero();
      }
    }
    __syncwarp();
    if (w == 0) {
      C x[PRL];
#pragma unroll
      for (int q = 0; q < PRL; ++q) x[q] = panel[lane + 32 * q];
      if (!publish<PRL>(x, 0, g, R, mstr, slots, sy, lane, eps)) { ok = false; break; }
    }
    for (int j = 0; j < m && ok; ++j) {
      const uint32_t gj = g + j;
      const int sl = gj & 1;
      // R entries of this step, loaded before anything waits: row j of the live columns
      const int rj = prow(j, mstr);
      const int cfirst = (j + 2 - w + NW - 1) / NW > 0 ? (j + 2 - w + NW - 1) / NW : 0;  // k > j+1
      const int nch = (nslot - cfirst + CH - 1) / CH;
      const int idx = lane >> (5 - L);
      C rjk[MAXCH];
#pragma unroll
      for (int h = 0; h < MAXCH; ++h) {
        rjk[h] = Tr<C>::zero();
        const int k = w + NW * (cfirst + h * CH + idx);
        if (h < nch && k < m) rjk[h] = R[rj + (k - j)];
      }
      const bool la = j + 1 < m && w == (j + 1) % NW;
      C r1 = Tr<C>::zero(), rdd = Tr<C>::zero();
      if (la) {
        r1 = R[rj + 1];
        rdd = R[prow(j + 1, mstr)];
      }
      if (!mbar_wait(&sy.full[sl], (gj >> 1) & 1)) { ok = give_up(sy, lane); break; }
      const C* slot = slots + sl * (PR + 2);
      C pv[PRL];
#pragma unroll
      for (int q = 0; q < PRL; ++q) pv[q] = slot[lane + 32 * q];
      const C piv = slot[PR];
      const C rt = slot[PR + 1];
      __syncwarp();
      if (lane == 0) mbar_arrive(&sy.empty[sl]);

      if (la) {
        C* col = panel + (size_t)(j + 1) * PR;
        C x[PRL];
#pragma unroll
        for (int q = 0; q < PRL; ++q) x[q] = col[lane + 32 * q];
        const C d = warp_allsum(dot_rows<PRL>(pv, x));
        const C c = mul(fmac(piv, r1, d), rt);
        if (lane == 0) R[rj + 1] = fnmac(c, piv, r1);
#pragma unroll
        for (int q = 0; q < PRL; ++q) {
          x[q] = renorm(fnmac_nr(c, pv[q], x[q]));
          col[lane + 32 * q] = x[q];
        }
        if (!publish_r<PRL>(x, rdd, j + 1, gj + 1, R, mstr, slots, sy, lane, eps)) { ok = false; break; }
      }
      // live columns k > j+1 in chunks of CH: dots, reduce-scatter, c_k and row j of R, update
      for (int h = 0; h < nch; ++h) {
        const int c0 = cfirst + h * CH;
        C xs[CH][PRL];
        C sdot[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          const int k = w + NW * (c0 + u);
          if (c0 + u < nslot && k < m) {
            const C* col = panel + (size_t)k * PR;
#pragma unroll
            for (int q = 0; q < PRL; ++q) xs[u][q] = col[lane + 32 * q];
          } else {
#pragma unroll
            for (int q = 0; q < PRL; ++q) xs[u][q] = Tr<C>::zero();
          }
          sdot[u] = dot_rows<PRL>(pv, xs[u]);
        }
        const C tot = butterfly<CH>(sdot, lane);
        const int k = w + NW * (c0 + idx);
        const bool act = c0 + idx < nslot && k > j + 1 && k < m;
        C ck = Tr<C>::zero();
        C rk = Tr<C>::zero();
#pragma unroll
        for (int hh = 0; hh < MAXCH; ++hh)
          if (hh == h) rk = rjk[hh];
        if (act) {
          ck = mul(fmac(piv, rk, tot), rt);
          if ((lane & ((1 << (5 - L)) - 1)) == 0) R[rj + (k - j)] = fnmac(ck, piv, rk);
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
          const C cb = shfl_idx(ck, u << (5 - L));
          const int ku = w + NW * (c0 + u);
          if (c0 + u < nslot && ku < m) {
            C* col = panel + (size_t)ku * PR;
#pragma unroll
            for (int q = 0; q < PRL; ++q) col[lane + 32 * q] = fnmac_nr(cb, pv[q], xs[u][q]);
          }
        }
      }
    }
  }
  __syncthreads();
  if (*reinterpret_cast<volatile int*>(abort_flag)) return;
  xr_end(xr, xfix, rd);
  for (int i2 = tid; i2 < mb * m; i2 += nt) {
    const int i = i2 % mb, k = i2 / mb;
    C v = Tr<C>::zero();
    if (i < m && i <= k) v = R[prow(i, mstr) + (k - i)];
    Rout[(int64_t)blockIdx.x * mb + i + (int64_t)k * ldR] = st_as<RO>(v);
  }
}

}  // namespace tt
