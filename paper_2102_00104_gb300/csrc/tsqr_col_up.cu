// tsqr_col_up.cu -- column-owned TSQR kernel for the upper tree levels
// (float-float partial R's) and for the native FP64 arithmetic.
#include "tsqr_col.cuh"

namespace tt {

cudaError_t tsqr_col_upper(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev,
                           void* Rout, int64_t ldR, int* status, cudaStream_t s) {
  if (L.in == Fmt::DF && L.comp == Fmt::DF && L.out == Fmt::DF)
    return colk::run_df_tuned<df>(L, W, ld, m_dev, Rout, ldR, status, s);
  if (L.in == Fmt::F64 && L.comp == Fmt::F64 && L.out == Fmt::F64)
    return colk::run_default<double, double, double>(L, W, ld, m_dev, Rout, ldR, status, s);
  return cudaErrorInvalidValue;
}

}  // namespace tt
