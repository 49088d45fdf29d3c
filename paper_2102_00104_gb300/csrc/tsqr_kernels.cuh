// tsqr_kernels.cuh -- Q-less TSQR level kernels (Alg. 6 panels in a flat tree,
// Sec. 3.2 of the paper).
//
// A level splits the rows of W into panels; every warp walks a contiguous
// range of panels and folds each one into its own triangle R by the
// Householder QR of [M; R] (Alg. 6, read as: the reflector of column j acts on
// all rows of the panel M and on row j of R, pivot R[j][j]).  The scaled,
// reflector of Alg. 6 is used (householder() in arith.cuh):
//   t = ||u||^2 (+ eps_FP in native FP64) ; alpha = -+sqrt(t) (sign opposite to the pivot)
//   t = t - alpha * R_jj ; piv = R_jj - alpha
// (in FP32 and float-float, whose input is shifted to max |x| ~ 1, a column with
// t < 2^-100 leaves the reflector as the identity instead of adding eps_FP)
// and every later column k is updated with c_k = (piv * R_jk + M_j . M_k) / t:
//   R_jk <- R_jk - c_k * piv ,   M_ik <- M_ik - c_k * M_ij
// (this is w <- w - (v^T w) v with v = u / sqrt(t), written without the root).
// The warp finally writes R as one block of the stacked output, so the next
// level is the same kernel applied to the tall matrix of stacked R's.
//
// narrow kernel (m <= MAXM <= 16): tsqr_narrow.cuh.
// wide kernel (m <= 32*NCH): the panel sits in shared memory (row-major, odd
//   row stride), lane l owns columns l, l+32, ...; each lane computes whole
//   dot products, so a column step needs only two broadcasts; R lives in a
//   per-warp global scratch (row-major).
#pragma once
#include "arith.cuh"
#include "engine.h"

namespace tt {

template <Fmt F> struct FT;
template <> struct FT<Fmt::F64> { using T = double; };
template <> struct FT<Fmt::DF> { using T = df; };
template <> struct FT<Fmt::F32> { using T = float; };

template <int NCH, class C, class S, class RO>
__global__ void __launch_bounds__(128)
k_tsqr_wide(const S* __restrict__ W, int64_t rows, int64_t ld, const int* __restrict__ m_ptr,
            int m_val, int pr, int mstr, C* __restrict__ Rscr, int mbs, RO* __restrict__ Rout,
            int64_t ldR, int mb, int64_t npanels, int* status, XRange* xr, int xfix) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  XRead<C, S> rd;
  if (!xr_begin(xr, xfix, rd)) return;
  const int m = m_ptr ? *m_ptr : m_val;
  if (m < 1 || m > 32 * NCH || m > mbs || m > mstr || m > mb || (pr & 31) != 0) {
    if (threadIdx.x == 0 && status) atomicOr(status, DEV_ERR_SHAPE);
    return;
  }
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * nw + w;
  const int64_t nwt = (int64_t)gridDim.x * nw;
  C* P = reinterpret_cast<C*>(smem_raw) + (size_t)w * pr * mstr;
  C* R = Rscr + (size_t)gw * mbs * mbs;
  for (int i = 0; i < m; ++i)
    for (int k = lane; k < m; k += 32) R[(size_t)i * mbs + k] = Tr<C>::zero();
  __syncwarp();
  const C eps = Tr<C>::eps();
  const int64_t p0 = gw * npanels / nwt, p1 = (gw + 1) * npanels / nwt;
  for (int64_t p = p0; p < p1; ++p) {
    const int64_t r0 = p * pr;
    for (int i = lane; i < pr; i += 32) {
      const int64_t row = r0 + i;
      const bool ok = row < rows;
      for (int k = 0; k < m; ++k)
        P[(size_t)i * mstr + k] = ok ? rd(W[row + (int64_t)k * ld]) : Tr<C>::zero();
    }
    __syncwarp();
    for (int j = 0; j < m; ++j) {
      C s[NCH], rr[NCH];
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        const int k = lane + 32 * c;
        s[c] = Tr<C>::zero();
        rr[c] = Tr<C>::zero();
        if (k >= j && k < m) {
          C a0 = Tr<C>::zero(), a1 = Tr<C>::zero(), a2 = Tr<C>::zero(), a3 = Tr<C>::zero();
          const C* pj = P + j;
          const C* pk = P + k;
          for (int i = 0; i < pr; i += 4) {
            a0 = fmac(pj[(size_t)(i + 0) * mstr], pk[(size_t)(i + 0) * mstr], a0);
            a1 = fmac(pj[(size_t)(i + 1) * mstr], pk[(size_t)(i + 1) * mstr], a1);
            a2 = fmac(pj[(size_t)(i + 2) * mstr], pk[(size_t)(i + 2) * mstr], a2);
            a3 = fmac(pj[(size_t)(i + 3) * mstr], pk[(size_t)(i + 3) * mstr], a3);
          }
          s[c] = add(add(a0, a1), add(a2, a3));
          rr[c] = R[(size_t)j * mbs + k];
        }
      }
      C dj = Tr<C>::zero(), rjj = Tr<C>::zero();
#pragma unroll
      for (int c = 0; c < NCH; ++c)
        if (c == (j >> 5)) { dj = s[c]; rjj = rr[c]; }
      dj = shfl_idx(dj, j & 31);
      rjj = shfl_idx(rjj, j & 31);
      const Refl<C> h = householder(rjj, dj, eps);
      const C alpha = h.alpha, piv = h.piv, tinv = h.rt;
#pragma unroll
      for (int c = 0; c < NCH; ++c) {
        const int k = lane + 32 * c;
        if (k > j && k < m) {
          const C cc = mul(fmac(piv, rr[c], s[c]), tinv);
          R[(size_t)j * mbs + k] = fnmac(cc, piv, rr[c]);
          const C* pj = P + j;
          C* pk = P + k;
          for (int i = 0; i < pr; ++i) pk[(size_t)i * mstr] = fnmac(cc, pj[(size_t)i * mstr], pk[(size_t)i * mstr]);
        }
      }
      if (lane == (j & 31)) R[(size_t)j * mbs + j] = alpha;
      __syncwarp();
    }
  }
  xr_end(xr, xfix, rd);
  for (int i = 0; i < mb; ++i)
    for (int k = lane; k < m; k += 32) {
      C v = Tr<C>::zero();
      if (i <= k && i < m) v = R[(size_t)i * mbs + k];
      Rout[gw * mb + i + (int64_t)k * ldR] = st_as<RO>(v);
    }
}

}  // namespace tt
