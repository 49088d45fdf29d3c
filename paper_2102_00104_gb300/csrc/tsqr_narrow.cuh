// tsqr_narrow.cuh -- the narrow Q-less TSQR level kernel (m <= MAXM <= 16), Alg. 6 panels
// folded into one R per warp (flat tree, Sec. 3.2), with the scaled reflector written out in
// tsqr_kernels.cuh.
//
// Lane l holds rows l, l+32, ... of the panel in registers (32 * K rows per panel, K = 32 /
// MAXM by default).  A column step j forms, per lane, the lazy float-float partial sums of
// the dot products of pivot column j with every column k >= j; one reduce-scatter butterfly
// over all MAXM columns (log2 MAXM halving levels, then an allreduce over the 32 / MAXM lanes
// of a group) leaves lane l with the total of column l / (32 / MAXM), and the lane group of
// each column forms its coefficient c_k and its R[j][k].
#pragma once
#include "tsqr_kernels.cuh"

namespace tt {

// Rows of the panel from a column-major matrix W (rows x m, leading dimension ld), read
// through the input reader (exponent shift of X, see arith.cuh).
template <class C, class S>
struct MatRows {
  const S* W;
  int64_t ld;
  XRead<C, S> rd;
  template <int MAXM>
  __device__ __forceinline__ void row(int64_t r, bool ok, int m, C (&out)[MAXM]) {
    // every load of the row first, then the conversions (which may branch)
    S raw[MAXM];
#pragma unroll
    for (int k = 0; k < MAXM; ++k) raw[k] = (ok && k < m) ? W[r + (int64_t)k * ld] : S{};
#pragma unroll
    for (int k = 0; k < MAXM; ++k) out[k] = (ok && k < m) ? rd(raw[k]) : Tr<C>::zero();
  }
};

// The narrow TSQR of one warp's panels (flat tree): rows come from `src.row`.
template <int MAXM, int K, class C, class RO, class Src>
__device__ __forceinline__ void narrow_body(Src& src, C (*R)[MAXM], int64_t rows, int m,
                                            RO* __restrict__ Rout, int64_t ldR, int mb,
                                            int64_t p0, int64_t p1, int64_t gw, int normalize) {
  constexpr int PR = 32 * K;
  constexpr int LG = MAXM == 4 ? 2 : (MAXM == 8 ? 3 : 4);  // log2(MAXM)
  constexpr int G = 32 / MAXM;                               // lanes per column after the butterfly
  static_assert((1 << LG) == MAXM, "MAXM is 4, 8 or 16");
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < MAXM * MAXM; i += 32) R[i / MAXM][i % MAXM] = Tr<C>::zero();
  __syncwarp();
  const C eps = Tr<C>::eps();
  for (int64_t p = p0; p < p1; ++p) {
    C a[K][MAXM];
    const int64_t r0 = p * PR;
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const int64_t row = r0 + lane + 32 * q;
      src.template row<MAXM>(row, row < rows, m, a[q]);
    }
    for (int j = 0; j < m; ++j) {
      // pivot column j, renormalised (a product of two float-float pairs drops lo*lo)
      C pv[K];
#pragma unroll
      for (int q = 0; q < K; ++q) pv[q] = Tr<C>::zero();
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k == j) {
#pragma unroll
          for (int q = 0; q < K; ++q) pv[q] = renorm(a[q][k]);
        }
      // Gram row of the pivot over this warp's panel rows: lazy partial sums per lane, then
      // one reduce-scatter butterfly, after which the G lanes of group k = lane / G hold
      // the whole sum for column k
      decltype(lz(Tr<C>::zero())) z[MAXM];
#pragma unroll
      for (int k = 0; k < MAXM; ++k) {
        z[k] = lz(Tr<C>::zero());
        if (k >= j) {
#pragma unroll
          for (int q = 0; q < K; ++q) z[k] = lz_fmac(pv[q], a[q][k], z[k]);
        }
      }
#pragma unroll
      for (int lev = 0; lev < LG; ++lev) {
        const int half = MAXM >> (lev + 1);
        const int bit = 16 >> lev;
        const bool up = (lane & bit) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
          const auto send = up ? z[i] : z[i + half];
          const auto keep = up ? z[i + half] : z[i];
          z[i] = lz_add(keep, shfl_xor(send, bit));
        }
      }
#pragma unroll
      for (int bit = 16 >> LG; bit > 0; bit >>= 1) z[0] = lz_add(z[0], shfl_xor(z[0], bit));
      const C tot = lz_fin(z[0]);     // column idx's sum
      const int idx = lane / G;
      // reflector scalars (identical in every lane); D = ||M_j||^2 from group j
      const C D = shfl_idx(tot, j * G);
      const C rjj = R[j][j];
      const Refl<C> h = householder(rjj, D, eps);
      const C alpha = h.alpha, piv = h.piv, rt = h.rt;
      // coefficient of this group's column: c_k = (piv R_jk + M_j . M_k) / t
      C ck = Tr<C>::zero(), rnew = Tr<C>::zero();
      const bool own = idx > j && idx < m;
      if (own) {
        const C rjk = R[j][idx];
        ck = mul(fmac(piv, rjk, tot), rt);
        rnew = fnmac(ck, piv, rjk);
      }
      __syncwarp();  // every lane has read row j of R before it changes
      if (own && (lane & (G - 1)) == 0) R[j][idx] = rnew;
      if (lane == 0) R[j][j] = alpha;
      // rank-1 update of the later columns (c_k = 0 is an exact no-op); the pairs are
      // renormalised (normalize != 0): left unnormalised, an exactly rank-deficient panel
      // lost accuracy in the next dot products (rank-1 tensor: sigma_2 = 1e-8 for 1e-16)
#pragma unroll
      for (int k = 0; k < MAXM; ++k)
        if (k > j) {
          const C cb = shfl_idx(ck, k * G);
#pragma unroll
          for (int q = 0; q < K; ++q) {
            a[q][k] = fnmac_nr(cb, pv[q], a[q][k]);
            if (normalize) a[q][k] = renorm(a[q][k]);
          }
        }
      __syncwarp();
    }
  }
  // stacked output block: rows gw*mb + i (i < mb), columns k < m
  for (int idx = lane; idx < mb * m; idx += 32) {
    const int i = idx % mb, k = idx / mb;
    C v = Tr<C>::zero();
    if (i < MAXM && i <= k) v = R[i][k];
    Rout[gw * mb + i + (int64_t)k * ldR] = st_as<RO>(v);
  }
}

template <int MAXM, int K, int NW, class C, class S, class RO>
__global__ void __launch_bounds__(NW * 32)
k_tsqr_narrow(const S* __restrict__ W, int64_t rows, int64_t ld, const int* __restrict__ m_ptr,
              int m_val, RO* __restrict__ Rout, int64_t ldR, int mb, int64_t npanels, int* status,
              int normalize, XRange* xr, int xfix) {
  __shared__ C Rsh[NW][MAXM][MAXM];
  MatRows<C, S> src{W, ld, {}};
  if (!xr_begin(xr, xfix, src.rd)) return;
  const int m = m_ptr ? *m_ptr : m_val;
  const int nwb = blockDim.x >> 5;
  if (m < 1 || m > MAXM || m > mb || nwb > NW) {
    if (threadIdx.x == 0 && status) atomicOr(status, DEV_ERR_SHAPE);
    return;
  }
  const int w = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * nwb + w;
  const int64_t nwt = (int64_t)gridDim.x * nwb;
  narrow_body<MAXM, K>(src, Rsh[w], rows, m, Rout, ldR, mb, gw * npanels / nwt,
                       (gw + 1) * npanels / nwt, gw, normalize);
  xr_end(xr, xfix, src.rd);
}

}  // namespace tt
