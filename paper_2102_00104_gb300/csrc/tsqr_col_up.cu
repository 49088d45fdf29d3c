// tsqr_col_up.cu -- column-owned TSQR kernel for the upper tree levels
// (float-float partial R's) and for the native FP64 arithmetic.
#include "tsqr_col.cuh"

namespace tt {

cudaError_t tsqr_col_upper(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev,
                           void* Rout, int64_t ldR, int* status, cudaStream_t s) {
  if (L.in == Fmt::DF && L.comp == Fmt::DF && L.out == Fmt::DF)
    return colk::run_df_tuned<df>(L, W, ld, m_dev, Rout, ldR, status, s);
  if (L.in == Fmt::F64 && L.comp == Fmt::F64 && L.out == Fmt::F64) {
    // the autotuner's alternative layouts (ids 5-9) for native FP64 as well
    using colk::run_col;
    using D = double;
    switch (L.cfg) {
      case 5: return run_col<12, 6, 8, 1, D, D, D>(L, W, ld, m_dev, Rout, ldR, status, s);
      case 6: return run_col<16, 4, 4, 1, D, D, D>(L, W, ld, m_dev, Rout, ldR, status, s);
      case 7: return run_col<16, 5, 6, 1, D, D, D>(L, W, ld, m_dev, Rout, ldR, status, s);
      case 8: return run_col<8, 8, 4, 2, D, D, D>(L, W, ld, m_dev, Rout, ldR, status, s);
      case 9: return run_col<8, 4, 8, 2, D, D, D>(L, W, ld, m_dev, Rout, ldR, status, s);
      default: return colk::run_default<D, D, D>(L, W, ld, m_dev, Rout, ldR, status, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace tt
