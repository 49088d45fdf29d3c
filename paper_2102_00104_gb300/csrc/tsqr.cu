// tsqr.cu -- instantiation and launch of the TSQR level kernels.
#include "tsqr_narrow.cuh"

namespace tt {

namespace {

template <int MAXM, int K, class C, class S, class RO>
cudaError_t run_narrow_k(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev, void* Rout,
                         int64_t ldR, int* status, cudaStream_t s) {
  constexpr int NW = 4;
  if (L.nw < 1 || L.nw > NW) return cudaErrorInvalidValue;
  k_tsqr_narrow<MAXM, K, NW, C, S, RO><<<(unsigned)L.ctas, L.nw * 32, 0, s>>>(
      static_cast<const S*>(W), L.rows, ld, m_dev, L.mval, static_cast<RO*>(Rout), ldR, L.mb,
      L.panels, status, tune_get("tsqr.narrow_norm", 1), L.xr, L.xfix);
  return cudaGetLastError();
}

// rows per lane K = panel rows / 32: 64 / MAXM or 32 / MAXM (fewer registers, more warps)
template <int MAXM, class C, class S, class RO>
cudaError_t run_narrow(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev, void* Rout,
                       int64_t ldR, int* status, cudaStream_t s) {
  if (L.pr == 32 * (64 / MAXM))
    return run_narrow_k<MAXM, 64 / MAXM, C, S, RO>(L, W, ld, m_dev, Rout, ldR, status, s);
  if (L.pr == 32 * (32 / MAXM))
    return run_narrow_k<MAXM, 32 / MAXM, C, S, RO>(L, W, ld, m_dev, Rout, ldR, status, s);
  return cudaErrorInvalidValue;
}

template <int NCH, class C, class S, class RO>
cudaError_t run_wide(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev, void* Rout,
                     int64_t ldR, void* Rscr, int* status, cudaStream_t s) {
  auto kern = k_tsqr_wide<NCH, C, S, RO>;
  if (L.smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L.smem);
    if (e != cudaSuccess) return e;
  }
  const int mstr = (L.mmax | 1);
  kern<<<(unsigned)L.ctas, L.nw * 32, L.smem, s>>>(static_cast<const S*>(W), L.rows, ld, m_dev,
                                                  L.mval, L.pr, mstr, static_cast<C*>(Rscr), L.mmax,
                                                  static_cast<RO*>(Rout), ldR, L.mb, L.panels,
                                                  status, L.xr, L.xfix);
  return cudaGetLastError();
}

template <class C, class S, class RO>
cudaError_t run_typed(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev, void* Rout,
                      int64_t ldR, void* Rscr, int* status, cudaStream_t s) {
  if (L.kind == 0) {
    switch (L.maxm) {
      case 4: return run_narrow<4, C, S, RO>(L, W, ld, m_dev, Rout, ldR, status, s);
      case 8: return run_narrow<8, C, S, RO>(L, W, ld, m_dev, Rout, ldR, status, s);
      case 16: return run_narrow<16, C, S, RO>(L, W, ld, m_dev, Rout, ldR, status, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (L.maxm / 32) {
    case 1: return run_wide<1, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 2: return run_wide<2, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 4: return run_wide<4, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 8: return run_wide<8, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 16: return run_wide<16, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

size_t tsqr_wide_scratch_bytes(const TsqrLevel& L) {
  if (L.kind == 2) return tsqr_cta_scratch(L.mmax, L.comp, L.cfg, L.ctas);
  if (L.kind == 4) return tsqr_cols_scratch(L.mmax, L.ctas);
  if (L.kind == 5) return tsqr_merge_scratch(L.mmax, L.comp, L.ctas);
  if (L.kind == 6) return tsqr_blk_scratch(L.mmax, L.ctas);
  if (L.kind != 1) return 0;  // kinds 0 and 3 keep R in registers / shared memory
  return (size_t)L.warps * L.mmax * L.mmax * fmt_bytes(L.comp);
}

cudaError_t launch_tsqr_level(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev,
                              void* Rout, int64_t ldR, void* Rscr, int* status, cudaStream_t s) {
  if (L.kind == 2) return launch_tsqr_cta(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
  if (L.kind == 3) return launch_tsqr_col(L, W, ld, m_dev, Rout, ldR, status, s);
  if (L.kind == 4) return launch_tsqr_cols(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
  if (L.kind == 5) return launch_tsqr_merge(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
  if (L.kind == 6) return launch_tsqr_blk(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
  if (L.in == Fmt::F64 && L.comp == Fmt::DF && L.out == Fmt::DF)
    return run_typed<df, double, df>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
  if (L.in == Fmt::DF && L.comp == Fmt::DF && L.out == Fmt::DF)
    return run_typed<df, df, df>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
  if (L.in == Fmt::F64 && L.comp == Fmt::F64 && L.out == Fmt::F64)
    return run_typed<double, double, double>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
  if (L.in == Fmt::F32 && L.comp == Fmt::F32 && L.out == Fmt::F32)
    return run_typed<float, float, float>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
  if (L.in == Fmt::F32 && L.comp == Fmt::DF && L.out == Fmt::DF)
    return run_typed<df, float, df>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
  return cudaErrorInvalidValue;
}

}  // namespace tt
