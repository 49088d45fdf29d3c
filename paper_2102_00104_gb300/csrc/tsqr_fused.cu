// tsqr_fused.cu -- W^(i-1) = reshape(W^(i) V_r) (Alg. 2 line 11, TSMM of Sec. 4.1.2) fused
// with the first TSQR level of the next step (Alg. 2 line 5, Alg. 6 panels) when that step
// is narrow (m_{i-1} = n_{i-1} r_{i-1} <= 8) and m_i <= 8: the steps of r_max = 1 (and of
// r_max = 2 on n_j = 4 tensors).
//
// Row a of the next unfolding W^(i-1) (rows R' = rows_i / n_{i-1}) holds, at column
// b + n_{i-1} c, entry (a + b R', c) of Y = W^(i) V_r (rows_i x r, column-major: the
// reshape is a view).  The lane that folds row a into its warp's R computes these m_{i-1}
// entries from the n_{i-1} rows a + b R' of W^(i) and V_r (shared memory), writes them to
// Y -- the next step's W V_r reads it -- and keeps them in registers for the panel, so the
// next step's first TSQR level does not read W^(i-1) back from memory.
#include "tsqr_narrow.cuh"

namespace tt {

namespace {

template <int MI, class C, class S, class SO>
struct ProdRows {
  const S* W;       // W^(i): rows_i x mi, column-major, leading dimension ldw
  int64_t ldw;
  int64_t Rp;       // rows of W^(i-1)
  int n, r, mi;     // mi <= MI
  const C* Vs;      // V_r in shared memory: Vs[kk + mi c]
  SO* Y;            // W^(i-1) as Y = W^(i) V_r (rows_i x r, leading dimension ldy)
  int64_t ldy;
  XRead<C, S> rd;   // the input reader of W^(i) (exponent shift when W^(i) is X)
  template <int MAXM>
  __device__ __forceinline__ void row(int64_t a, bool ok, int m, C (&out)[MAXM]) {
#pragma unroll
    for (int kp = 0; kp < MAXM; ++kp) {
      const bool live = ok && kp < m;
      const int b = kp % n, c = kp / n;
      const int64_t ri = live ? a + (int64_t)b * Rp : 0;
      // the row's loads first, then the conversions and the product
      S raw[MI];
#pragma unroll
      for (int kk = 0; kk < MI; ++kk) raw[kk] = (live && kk < mi) ? W[ri + (int64_t)kk * ldw] : S{};
      const C* vc = Vs + (size_t)(live ? c : 0) * mi;
      auto acc = lz(Tr<C>::zero());
#pragma unroll
      for (int kk = 0; kk < MI; ++kk)
        if (kk < mi) acc = lz_fmac(rd(raw[kk]), vc[kk], acc);
      const C y = lz_fin(acc);
      if (live) Y[ri + (int64_t)c * ldy] = st_as<SO>(y);
      out[kp] = live ? y : Tr<C>::zero();
    }
  }
};

template <int MAXM, int K, int NW, int MI, class C, class S, class VS, class SO>
__global__ void __launch_bounds__(NW * 32)
k_tsmm_tsqr_narrow(const S* __restrict__ W, int64_t ldw, const int* __restrict__ mi_ptr, int mi_max,
                   const VS* __restrict__ V, int ldV, int n, int64_t Rp,
                   const int* __restrict__ m_ptr, const int* __restrict__ r_ptr, int r_max,
                   SO* __restrict__ Y, int64_t ldy, C* __restrict__ Rout, int64_t ldR, int mb,
                   int64_t npanels, int* status, int normalize, const XRange* xr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ C Rsh[NW][MAXM][MAXM];
  C* Vs = reinterpret_cast<C*>(smem_raw);
  const int mi = *mi_ptr, m = *m_ptr, r = *r_ptr;
  const int nwb = blockDim.x >> 5;
  if (mi < 1 || mi > mi_max || mi > MI || r < 1 || r > r_max || m != n * r || m > MAXM || m > mb ||
      nwb > NW) {
    if (threadIdx.x == 0 && status) atomicOr(status, DEV_ERR_SHAPE);
    return;
  }
  for (int idx = threadIdx.x; idx < mi * r; idx += blockDim.x) {
    const int kk = idx % mi, c = idx / mi;
    Vs[idx] = ld_as<C>(V[kk + (size_t)c * ldV]);
  }
  __syncthreads();
  ProdRows<MI, C, S, SO> src{W, ldw, Rp, n, r, mi, Vs, Y, ldy, {}};
  src.rd.set(xr ? xr->k : 0, xr != nullptr);
  const int w = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * nwb + w;
  const int64_t nwt = (int64_t)gridDim.x * nwb;
  narrow_body<MAXM, K>(src, Rsh[w], Rp, m, Rout, ldR, mb, gw * npanels / nwt,
                       (gw + 1) * npanels / nwt, gw, normalize);
}

template <int MAXM, int K, class C, class S, class VS, class SO>
cudaError_t run_k(const TsqrLevel& L, const void* W, int64_t ldw, const int* mi_dev, int mi_max,
                  const void* V, int ldV, int n, const int* m_dev, const int* r_dev, int r_max,
                  void* Y, void* Rout, int64_t ldR, int* status, const XRange* xr, cudaStream_t s) {
  constexpr int NW = 4;
  if (L.nw < 1 || L.nw > NW) return cudaErrorInvalidValue;
  const size_t smem = (size_t)mi_max * r_max * sizeof(C);
  auto kern = k_tsmm_tsqr_narrow<MAXM, K, NW, kFusedMaxMi, C, S, VS, SO>;
  kern<<<(unsigned)L.ctas, L.nw * 32, smem, s>>>(
      static_cast<const S*>(W), ldw, mi_dev, mi_max, static_cast<const VS*>(V), ldV, n, L.rows,
      m_dev, r_dev, r_max, static_cast<SO*>(Y), ldw, static_cast<C*>(Rout), ldR, L.mb, L.panels,
      status, tune_get("tsqr.narrow_norm", 1), xr);
  return cudaGetLastError();
}

template <class C, class S, class VS, class SO>
cudaError_t run_typed(const TsqrLevel& L, const void* W, int64_t ldw, const int* mi_dev,
                      int mi_max, const void* V, int ldV, int n, const int* m_dev, const int* r_dev,
                      int r_max, void* Y, void* Rout, int64_t ldR, int* status, const XRange* xr,
                      cudaStream_t s) {
#define TT_FUSED(MX, KK)                                                                    \
  if (L.maxm == MX && L.pr == 32 * KK)                                                      \
    return run_k<MX, KK, C, S, VS, SO>(L, W, ldw, mi_dev, mi_max, V, ldV, n, m_dev, r_dev,  \
                                       r_max, Y, Rout, ldR, status, xr, s);
  TT_FUSED(4, 8) TT_FUSED(8, 4)
#undef TT_FUSED
  return cudaErrorInvalidValue;
}

}  // namespace

bool tsmm_tsqr_fusable(const TsqrLevel& next, Fmt in, Fmt comp, Fmt vfmt, Fmt inter, int mi_max,
                       int r_max) {
  // opt-in: measured slower than the two launches it replaces (r_max = 1 on 8^10: 17.5 ms
  // for the fused step-10 launch against 4.0 + 1.0 ms)
  if (tune_get("fuse.tsmm_tsqr", 0) == 0) return false;
  if (next.kind != 0 || next.chunks > 1 || next.comp != comp || next.in != inter) return false;
  // the default narrow layout with m_{i-1} <= 8 only
  if (next.maxm > 8 || next.pr != 32 * (32 / next.maxm)) return false;
  if (mi_max < 1 || mi_max > kFusedMaxMi || r_max < 1 || r_max > 16) return false;
  const bool df_form = comp == Fmt::DF && vfmt == Fmt::DF && inter == Fmt::DF &&
                       (in == Fmt::F64 || in == Fmt::DF);
  const bool f64_form = comp == Fmt::F64 && vfmt == Fmt::F64 && inter == Fmt::F64 && in == Fmt::F64;
  const bool f32_form = comp == Fmt::F32 && vfmt == Fmt::DF && inter == Fmt::F32 && in == Fmt::F32;
  return df_form || f64_form || f32_form;
}

cudaError_t launch_tsmm_tsqr(const TsqrLevel& next, Fmt in, Fmt vfmt, const void* W, int64_t ldw,
                             const int* mi_dev, int mi_max, const void* V, int ldV, int n,
                             const int* m_dev, const int* r_dev, int r_max, void* Y, void* Rout,
                             int64_t ldR, int* status, const XRange* xr, cudaStream_t s) {
  const Fmt comp = next.comp;
  if (comp == Fmt::DF && in == Fmt::F64)
    return run_typed<df, double, df, df>(next, W, ldw, mi_dev, mi_max, V, ldV, n, m_dev, r_dev,
                                         r_max, Y, Rout, ldR, status, xr, s);
  if (comp == Fmt::DF && in == Fmt::DF)
    return run_typed<df, df, df, df>(next, W, ldw, mi_dev, mi_max, V, ldV, n, m_dev, r_dev,
                                     r_max, Y, Rout, ldR, status, xr, s);
  if (comp == Fmt::F64)
    return run_typed<double, double, double, double>(next, W, ldw, mi_dev, mi_max, V, ldV, n,
                                                     m_dev, r_dev, r_max, Y, Rout, ldR, status,
                                                     xr, s);
  if (comp == Fmt::F32 && vfmt == Fmt::DF)
    return run_typed<float, float, df, float>(next, W, ldw, mi_dev, mi_max, V, ldV, n, m_dev,
                                              r_dev, r_max, Y, Rout, ldR, status, xr, s);
  return cudaErrorInvalidValue;
}

}  // namespace tt
