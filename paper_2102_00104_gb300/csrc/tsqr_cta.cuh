// tsqr_cta.cuh -- CTA-cooperative TSQR level kernel (Alg. 6 panels, Sec. 3.2).
//
// One CTA folds a contiguous range of row panels into one triangle R (a flat
// tree), then writes R as one block of the stacked output, exactly like the
// warp kernels, but the whole CTA works on each panel:
//
//   thread layout  lane = cg + CG * rgl   (cg: column group, rgl: row group in the warp)
//                  rg   = warp * (32/CG) + rgl
//   a thread holds rows  r0 + rg + RG*q  (q < RL)  and columns  cg + CG*c  (c < CL)
//   of the panel in registers (PR = RG * RL rows, m <= CG * CL columns).
//
// Column j of Alg. 6 then costs, per thread: a broadcast of the pivot column
// inside the row group (shuffles), the partial dot products of the pivot with
// the thread's columns over its rows, a reduction over the row groups (warp
// shuffles, then one partial per warp in shared memory), and the rank-1 update
// of the thread's columns.  Columns are dealt cyclically to the column groups,
// so every lane keeps working as the active triangle shrinks.  One thread per
// column k ("D-thread", k mod blockDim) sums the warp partials, forms the
// branch-free reflector of Alg. 6 lines 4-7 from D_j = M_j . M_j and R_jj, and
// the coefficient c_k = (piv R_jk + M_j . M_k) / t, and updates R_jk; R is kept
// packed (upper triangle, row-major) in shared memory (or, for m too large for
// it, in an L2-resident global slice per CTA).  Two __syncthreads per column.
#pragma once
#include "tsqr_kernels.cuh"

namespace tt {

// packed upper triangle, row-major: row j starts at j*m - j*(j-1)/2 (holds columns j..m-1)
__device__ __forceinline__ int packed_row(int j, int m) { return j * m - (j * (j - 1)) / 2; }

template <int CG, int CL, int RL, int NW, int MINB, bool RG_MEM, class C, class S, class RO>
__global__ void __launch_bounds__(NW * 32, MINB)
k_tsqr_cta(const S* __restrict__ W, int64_t rows, int64_t ld, const int* __restrict__ m_ptr,
           int m_val, int mmax, RO* __restrict__ Rout, int64_t ldR, int mb, int64_t npanels,
           C* __restrict__ Rglob, int* status, XRange* xr, int xfix) {
  XRead<C, S> rd;
  if (!xr_begin(xr, xfix, rd)) return;
  constexpr int RGW = 32 / CG;
  constexpr int RG = NW * RGW;
  constexpr int PR = RG * RL;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = m_ptr ? *m_ptr : m_val;
  if (m < 1 || m > CG * CL || m > mmax || m > mb || blockDim.x != NW * 32) {
    if (threadIdx.x == 0 && status) atomicOr(status, DEV_ERR_SHAPE);
    return;
  }
  // packed triangle of m_max: in shared memory, or (RG_MEM, large m) in a per-CTA
  // slice of global memory that stays resident in L2
  C* R = RG_MEM ? Rglob + (size_t)blockIdx.x * ((size_t)mmax * (mmax + 1) / 2)
                : reinterpret_cast<C*>(smem_raw);
  C* red = RG_MEM ? reinterpret_cast<C*>(smem_raw) : R + (size_t)mmax * (mmax + 1) / 2;
  C* Cc = red + (size_t)NW * mmax;                        // coefficients c_k
  const int tid = threadIdx.x, nt = NW * 32;
  const int w = tid >> 5, lane = tid & 31;
  const int cg = lane % CG, rgl = lane / CG;
  const int rg = w * RGW + rgl;
  const int tri = m * (m + 1) / 2;
  for (int i = tid; i < tri; i += nt) R[i] = Tr<C>::zero();
  __syncthreads();
  const C eps = Tr<C>::eps();
  const int64_t p0 = (int64_t)blockIdx.x * npanels / gridDim.x;
  const int64_t p1 = (int64_t)(blockIdx.x + 1) * npanels / gridDim.x;
  for (int64_t p = p0; p < p1; ++p) {
    C a[RL][CL];
    {
      // every load of the panel first, then the conversions (which may branch)
      S raw[RL][CL];
#pragma unroll
      for (int q = 0; q < RL; ++q) {
        const int64_t row = p * PR + rg + RG * q;
#pragma unroll
        for (int c = 0; c < CL; ++c) {
          const int k = cg + CG * c;
          raw[q][c] = (row < rows && k < m) ? W[row + (int64_t)k * ld] : S{};
        }
      }
#pragma unroll
      for (int q = 0; q < RL; ++q) {
        const int64_t row = p * PR + rg + RG * q;
#pragma unroll
        for (int c = 0; c < CL; ++c) {
          const int k = cg + CG * c;
          a[q][c] = (row < rows && k < m) ? rd(raw[q][c]) : Tr<C>::zero();
        }
      }
    }
    for (int j = 0; j < m; ++j) {
      const int cgj = j % CG, cj = j / CG;
      // pivot column values of this thread's rows (owner lane: same row group, cg = j mod CG)
      C pv[RL];
#pragma unroll
      for (int q = 0; q < RL; ++q) pv[q] = Tr<C>::zero();
#pragma unroll
      for (int c = 0; c < CL; ++c)
        if (c == cj) {
#pragma unroll
          for (int q = 0; q < RL; ++q) pv[q] = a[q][c];
        }
#pragma unroll
      for (int q = 0; q < RL; ++q) pv[q] = shfl_idx(pv[q], cgj + CG * rgl);
      // partial dots over this thread's rows, reduced over the row groups of the warp
#pragma unroll
      for (int c = 0; c < CL; ++c) {
        if (CG * c + CG - 1 >= j) {  // some column of this chunk is still active (warp-uniform)
          C sacc = mul(pv[0], a[0][c]);
#pragma unroll
          for (int q = 1; q < RL; ++q) sacc = fmac(pv[q], a[q][c], sacc);
#pragma unroll
          for (int o = CG; o < 32; o <<= 1) sacc = add(sacc, shfl_xor(sacc, o));
          const int k = cg + CG * c;
          if (rgl == 0 && k >= j && k < m) red[w * mmax + k] = sacc;
        }
      }
      __syncthreads();
      // D-threads: totals, reflector, coefficients, row j of R (thread k - j handles column k;
      // thread 0 handles the pivot and writes R_jj = alpha only after the barrier, because
      // every D-thread reads the old R_jj)
      C alpha_keep = Tr<C>::zero();
      for (int k = j + tid; k < m; k += nt) {
        // pairwise sums of the NW warp partials (short dependency chains)
        C pk[NW], pj[NW];
#pragma unroll
        for (int ww = 0; ww < NW; ++ww) {
          pk[ww] = red[ww * mmax + k];
          pj[ww] = red[ww * mmax + j];
        }
#pragma unroll
        for (int h = NW / 2; h > 0; h >>= 1)
#pragma unroll
          for (int ww = 0; ww < h; ++ww) {
            pk[ww] = add(pk[ww], pk[ww + h]);
            pj[ww] = add(pj[ww], pj[ww + h]);
          }
        const C dk = pk[0], dj = pj[0];
        const int rj = packed_row(j, m);
        const C rjj = R[rj];
        const Refl<C> h = householder(rjj, dj, eps);
        const C alpha = h.alpha, piv = h.piv;
        if (k == j) {
          alpha_keep = alpha;
        } else {
          const C rjk = R[rj + (k - j)];
          const C ck = mul(fmac(piv, rjk, dk), h.rt);
          R[rj + (k - j)] = fnmac(ck, piv, rjk);
          Cc[k] = ck;
        }
      }
      __syncthreads();
      if (tid == 0) R[packed_row(j, m)] = alpha_keep;
      // rank-1 update of this thread's columns k > j
#pragma unroll
      for (int c = 0; c < CL; ++c) {
        if (CG * c + CG - 1 > j) {
          const int k = cg + CG * c;
          const C ck = (k > j && k < m) ? Cc[k] : Tr<C>::zero();
#pragma unroll
          for (int q = 0; q < RL; ++q) a[q][c] = fnmac(ck, pv[q], a[q][c]);
        }
      }
    }
  }
  __syncthreads();
  xr_end(xr, xfix, rd);
  for (int idx = tid; idx < mb * m; idx += nt) {
    const int i = idx % mb, k = idx / mb;
    C v = Tr<C>::zero();
    if (i < m && i <= k) v = R[packed_row(i, m) + (k - i)];
    Rout[(int64_t)blockIdx.x * mb + i + (int64_t)k * ldR] = st_as<RO>(v);
  }
}

}  // namespace tt
