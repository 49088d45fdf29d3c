// tsqr_merge.cu -- upper TSQR levels as a binary tree of triangle-on-triangle merges
// (the reduction tree of Sec. 3.2: R <- R of the QR of [R_a; R_b]).
//
// Above the first level the input of a level is a stack of upper-triangular R blocks.
// Folding them with the panel kernels treats the zeros below every diagonal as data;
// for wide m that costs ~4 m^3 flops per merged pair and, with several R's per CTA,
// leaves few CTAs for a long serial chain.  Here one CTA merges one pair and uses the
// structure: the reflector of column j (Alg. 6, pivot R_a[j][j], panel part the
// column of R_b) has nonzeros only in R_a's row j and in R_b's rows 0..j, so step j
// touches R_a's row j (which is final afterwards: the merged R's row j) and R_b's
// rows 0..j of the columns right of j -- about m^3 / 6 multiply-adds per pair.
//
//   R_b is copied once into a packed column-major triangle (scratch, L2-resident).
//   Lane l of a warp holds rows l + 32 q of the columns it works on; a step's dot
//   products reduce inside the warp (reduce-scatter over CH columns at once).
//   Warp 0 works one column ahead: in step j it applies reflector j to column j+1 and
//   forms reflector j+1 into the other of two shared-memory slots, while the other
//   warps update columns j+2 .. m-1.  One CTA barrier per column; no spin waits.
//
// The reflector and the column update use the same scaled, branch-free form of Alg. 6
// as the level kernels (householder() in arith.cuh): t = ||x||^2 + R_jj^2,
// alpha = -+sqrt(t), t -= alpha R_jj, piv = R_jj - alpha,
// c_k = (piv R_jk + x . y_k) / t, R_jk -= c_k piv, y_k -= c_k x.
#include "tsqr_col.cuh"

namespace tt {

namespace {

// packed upper triangle, column-major: column k keeps rows 0..k from offset k(k+1)/2
__device__ __forceinline__ int64_t tcol(int k) { return (int64_t)k * (k + 1) / 2; }

// Reflector from column values y (rows lane + 32 q; zero beyond the pivot row) and the
// pivot entry rjj: writes y, piv and 1/t to the slot and returns alpha (the new R_jj).
template <int QMAX, class C>
__device__ __forceinline__ C make_reflector(C (&y)[QMAX], C rjj, C* slot, int lane, C eps) {
  auto acc = lz(Tr<C>::zero());
#pragma unroll
  for (int q = 0; q < QMAX; ++q) {
    y[q] = renorm(y[q]);
    acc = lz_fmac(y[q], y[q], acc);
  }
  const C D = colk::warp_allsum(lz_fin(acc));
  const Refl<C> h = householder(rjj, D, eps);
#pragma unroll
  for (int q = 0; q < QMAX; ++q) slot[lane + 32 * q] = y[q];
  if (lane == 0) {
    slot[32 * QMAX] = h.piv;
    slot[32 * QMAX + 1] = h.rt;
  }
  return h.alpha;
}

template <int QMAX, int CH, int NW, class C, class S>
__global__ void __launch_bounds__(NW * 32, 1)
k_tsqr_merge(const S* __restrict__ Rin, int64_t ldi, int64_t nblk, int mb,
             const int* __restrict__ m_ptr, int m_val, int mmax, C* __restrict__ Rout,
             int64_t ldo, C* __restrict__ scr, int* status) {
  constexpr int L = colk::ilog2(CH);
  constexpr int SL = 32 * QMAX + 2;
  __shared__ C slots[2 * SL];
  const int m = m_ptr ? *m_ptr : m_val;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  constexpr int NT = NW * 32;
  if (m < 1 || m > mmax || m > mb || m > 32 * QMAX || blockDim.x != NT) {
    if (tid == 0 && status) atomicOr(status, DEV_ERR_SHAPE);
    return;
  }
  const int64_t pq = blockIdx.x;
  const S* Ra = Rin + 2 * pq * mb;  // Ra[i + k * ldi]
  C* Ro = Rout + pq * mb;           // Ro[i + k * ldo]
  if (2 * pq + 1 >= nblk) {
    // odd block out: passed up unchanged
    for (int t = tid; t < mb * m; t += NT) {
      const int i = t % mb, k = t / mb;
      Ro[i + (int64_t)k * ldo] =
          (i < m && i <= k) ? ld_as<C>(Ra[i + (int64_t)k * ldi]) : Tr<C>::zero();
    }
    return;
  }
  const S* Rb = Ra + mb;
  C* B = scr + pq * tcol(mmax);
  // the output block's zeros (below the diagonal, rows >= m); row j is written in step j
  for (int t = tid; t < mb * m; t += NT) {
    const int i = t % mb, k = t / mb;
    if (i >= m || i > k) Ro[i + (int64_t)k * ldo] = Tr<C>::zero();
  }
  for (int k = w; k < m; k += NW)
    for (int i = lane; i <= k; i += 32) B[tcol(k) + i] = ld_as<C>(Rb[i + (int64_t)k * ldi]);
  const C eps = Tr<C>::eps();
  __syncthreads();
  if (w == 0) {
    C y[QMAX];
#pragma unroll
    for (int q = 0; q < QMAX; ++q) y[q] = (q == 0 && lane == 0) ? B[0] : Tr<C>::zero();
    const C alpha = make_reflector<QMAX>(y, ld_as<C>(Ra[0]), slots, lane, eps);
    if (lane == 0) Ro[0] = alpha;
  }
  __syncthreads();

#pragma unroll 1
  for (int j = 0; j < m; ++j) {
    const C* sl = slots + (j & 1) * SL;
    const C piv = sl[32 * QMAX], rt = sl[32 * QMAX + 1];
    const int nq = (j >> 5) + 1;  // row blocks q holding rows <= j
    C x[QMAX];
#pragma unroll
    for (int q = 0; q < QMAX; ++q) x[q] = sl[lane + 32 * q];
    if (w == 0 && j + 1 < m) {
      // look-ahead: column j+1, then reflector j+1
      const int k = j + 1;
      C y[QMAX];
      auto acc = lz(Tr<C>::zero());
#pragma unroll
      for (int q = 0; q < QMAX; ++q) {
        const int i = lane + 32 * q;
        y[q] = (q < nq && i <= j) ? B[tcol(k) + i] : Tr<C>::zero();
        acc = lz_fmac(x[q], y[q], acc);
      }
      const C d = colk::warp_allsum(lz_fin(acc));
      const C r = ld_as<C>(Ra[j + (int64_t)k * ldi]);
      const C c = mul(fmac(piv, r, d), rt);
      if (lane == 0) Ro[j + (int64_t)k * ldo] = fnmac(c, piv, r);
#pragma unroll
      for (int q = 0; q < QMAX; ++q) y[q] = fnmac_nr(c, x[q], y[q]);
      // row k of R_b enters with reflector k, still as copied
#pragma unroll
      for (int q = 0; q < QMAX; ++q)
        if (lane + 32 * q == k) y[q] = B[tcol(k) + k];
      const C alpha = make_reflector<QMAX>(y, ld_as<C>(Ra[k + (int64_t)k * ldi]),
                                           slots + (k & 1) * SL, lane, eps);
      if (lane == 0) Ro[k + (int64_t)k * ldo] = alpha;
    }
    // columns j+2 .. m-1 in chunks of CH; chunk c goes to warp (c + 1) mod NW
    const int k0 = j + 2;
    const int nch = m > k0 ? (m - k0 + CH - 1) / CH : 0;
    for (int c = (w + NW - 1) % NW; c < nch; c += NW) {
      const int kb = k0 + c * CH;
      C y[CH][QMAX];
      C s[CH];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int k = kb + u;
        auto acc = lz(Tr<C>::zero());
#pragma unroll
        for (int q = 0; q < QMAX; ++q) {
          const int i = lane + 32 * q;
          y[u][q] = (k < m && q < nq && i <= j) ? B[tcol(k) + i] : Tr<C>::zero();
          acc = lz_fmac(x[q], y[u][q], acc);
        }
        s[u] = lz_fin(acc);
      }
      const C tot = colk::butterfly<CH>(s, lane);
      const int ku = kb + (lane >> (5 - L));
      C ck = Tr<C>::zero();
      if (ku < m) {
        const C r = ld_as<C>(Ra[j + (int64_t)ku * ldi]);
        ck = mul(fmac(piv, r, tot), rt);
        if ((lane & ((1 << (5 - L)) - 1)) == 0) Ro[j + (int64_t)ku * ldo] = fnmac(ck, piv, r);
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const C cb = shfl_idx(ck, u << (5 - L));
        const int k = kb + u;
        if (k < m) {
#pragma unroll
          for (int q = 0; q < QMAX; ++q) {
            const int i = lane + 32 * q;
            if (q < nq && i <= j) B[tcol(k) + i] = fnmac_nr(cb, x[q], y[u][q]);
          }
        }
      }
    }
    __syncthreads();
  }
}

template <int QMAX, int CH, int NW, class C, class S>
cudaError_t run_merge(const TsqrLevel& L, const void* Rin, int64_t ldi, const int* m_dev,
                      void* Rout, int64_t ldo, void* scr, int* status, cudaStream_t s) {
  const int64_t nblk = L.rows / L.mb;
  k_tsqr_merge<QMAX, CH, NW, C, S><<<(unsigned)L.ctas, NW * 32, 0, s>>>(
      static_cast<const S*>(Rin), ldi, nblk, L.mb, m_dev, L.mval, L.mmax, static_cast<C*>(Rout),
      ldo, static_cast<C*>(scr), status);
  return cudaGetLastError();
}

template <class C, class S>
cudaError_t run_merge_typed(const TsqrLevel& L, const void* Rin, int64_t ldi, const int* m_dev,
                            void* Rout, int64_t ldo, void* scr, int* status, cudaStream_t s) {
  if (L.mmax <= 128) return run_merge<4, 8, 16, C, S>(L, Rin, ldi, m_dev, Rout, ldo, scr, status, s);
  if (L.mmax <= 256) return run_merge<8, 4, 16, C, S>(L, Rin, ldi, m_dev, Rout, ldo, scr, status, s);
  if (L.mmax <= 512) return run_merge<16, 2, 16, C, S>(L, Rin, ldi, m_dev, Rout, ldo, scr, status, s);
  return cudaErrorInvalidValue;
}

}  // namespace

bool tsqr_merge_ok(int m_max, Fmt in, Fmt comp) {
  if (m_max < 2 || m_max > kMaxM) return false;
  if (comp == Fmt::DF) return in == Fmt::DF || in == Fmt::F32;
  if (comp == Fmt::F64) return in == Fmt::F64;
  return false;
}

size_t tsqr_merge_scratch(int m_max, Fmt comp, int64_t ctas) {
  return (size_t)ctas * ((size_t)m_max * (m_max + 1) / 2) * fmt_bytes(comp);
}

cudaError_t launch_tsqr_merge(const TsqrLevel& L, const void* Rin, int64_t ldi, const int* m_dev,
                              void* Rout, int64_t ldo, void* scr, int* status, cudaStream_t s) {
  if (L.rows % L.mb != 0 || L.ctas != (L.rows / L.mb + 1) / 2) return cudaErrorInvalidValue;
  if (L.comp == Fmt::DF && L.in == Fmt::DF)
    return run_merge_typed<df, df>(L, Rin, ldi, m_dev, Rout, ldo, scr, status, s);
  if (L.comp == Fmt::DF && L.in == Fmt::F32)
    return run_merge_typed<df, float>(L, Rin, ldi, m_dev, Rout, ldo, scr, status, s);
  if (L.comp == Fmt::F64 && L.in == Fmt::F64)
    return run_merge_typed<double, double>(L, Rin, ldi, m_dev, Rout, ldo, scr, status, s);
  return cudaErrorInvalidValue;
}

}  // namespace tt
