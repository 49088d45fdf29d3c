// tsqr_cols.cu -- layouts, choice and launch of the shared-memory-panel TSQR kernel
// (float-float, 160 < m <= 512).
#include <cstdio>

#include "tsqr_cols.cuh"

namespace tt {

namespace {

constexpr int kNW = 16, kCH = 4;

template <int PRL, class S>
cudaError_t run_cols(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev, void* Rout,
                     int64_t ldR, void* Rscr, int* status, cudaStream_t s) {
  auto kern = k_tsqr_cols<kNW, kCH, PRL, df, S, df>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)L.ctas, kNW * 32, L.smem, s>>>(static_cast<const S*>(W), L.rows, ld, m_dev,
                                                 L.mval, L.mmax, static_cast<df*>(Rout), ldR, L.mb,
                                                 L.panels, static_cast<df*>(Rscr), status, L.xr,
                                                 L.xfix);
  return cudaGetLastError();
}

template <class S>
cudaError_t run_prl(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev, void* Rout,
                    int64_t ldR, void* Rscr, int* status, cudaStream_t s) {
  switch (L.cfg) {
    case 1: return run_cols<1, S>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 2: return run_cols<2, S>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 3: return run_cols<3, S>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

size_t tsqr_cols_smem(int m_max, int prl) {
  return 64 + (2 * (size_t)(32 * prl + 2) + (size_t)m_max * 32 * prl) * sizeof(df);
}

// rows per lane (the layout id) for m_max, or -1: float-float arithmetic, FP64 or
// float-float input, the largest panel whose columns fit in 227 KB of shared memory
int tsqr_cols_pick(int m_max, Fmt in, Fmt comp, Fmt out, int* pr, int* nw, int* per_sm) {
  if (tune_get("tsqr.cols", 1) == 0) return -1;
  if (comp != Fmt::DF || out != Fmt::DF || (in != Fmt::F64 && in != Fmt::DF)) return -1;
  if (m_max <= 160 || m_max > kNW * kCH * 8) return -1;
  for (int prl = 3; prl >= 1; --prl)
    if (tsqr_cols_smem(m_max, prl) <= 227 * 1024) {
      *pr = 32 * prl;
      *nw = kNW;
      *per_sm = 1;
      return prl;
    }
  return -1;
}

size_t tsqr_cols_scratch(int m_max, int64_t ctas) {
  return (size_t)ctas * ((size_t)m_max * (m_max + 1) / 2) * sizeof(df);
}

cudaError_t launch_tsqr_cols(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev,
                             void* Rout, int64_t ldR, void* Rscr, int* status, cudaStream_t s) {
  if (L.in == Fmt::F64) return run_prl<double>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
  if (L.in == Fmt::DF) return run_prl<df>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
  return cudaErrorInvalidValue;
}

}  // namespace tt
