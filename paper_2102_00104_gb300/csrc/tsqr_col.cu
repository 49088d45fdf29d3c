// tsqr_col.cu -- layouts, choice and launch of the column-owned TSQR level kernel
// (first level of the FP64 and FP32 forms; see tsqr_col_up.cu for the rest).
#include <cstdio>

#include "tsqr_col.cuh"
#include "tt_svd.h"

namespace tt {

namespace {

struct ColCfg {
  int nw, clw, prl, minb;
};

// (warps, column slots per warp, rows per lane, CTAs per SM) per layout id.
// ids 0-9: 8-byte arithmetic (float-float, FP64); 0-4 are the defaults per m
// bucket (m <= 32, 64, 80, 128, 160), 5-9 alternatives for the autotuner.
// ids 10-14: FP32 panels (two 8-warp CTAs per SM measured best up to m = 64:
// the FP32 reflector chain is short).  Panels of 256 rows with 16 warps measured best for
// m = 64 on GB300: the column step is bound by the reflector chain of the
// look-ahead warp, so rows per panel (work per chain) count more than warps.
const ColCfg kCol[15] = {
    {16, 2, 8, 1},  {16, 4, 8, 1}, {16, 5, 4, 1}, {16, 8, 4, 1}, {20, 8, 3, 1},
    {12, 6, 8, 1},  {16, 4, 4, 1}, {16, 5, 6, 1}, {8, 8, 4, 2},  {8, 4, 8, 2},
    {8, 4, 16, 2},  {8, 8, 8, 2},  {16, 8, 8, 1}, {16, 16, 4, 1}, {32, 10, 3, 1}};

using colk::run_col;

cudaError_t run_f32(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev, void* Rout,
                    int64_t ldR, int* status, cudaStream_t s) {
  using C = float;
  switch (L.cfg) {
    case 10: return run_col<8, 4, 16, 2, C, C, C>(L, W, ld, m_dev, Rout, ldR, status, s);
    case 11: return run_col<8, 8, 8, 2, C, C, C>(L, W, ld, m_dev, Rout, ldR, status, s);
    case 12: return run_col<16, 8, 8, 1, C, C, C>(L, W, ld, m_dev, Rout, ldR, status, s);
    case 13: return run_col<16, 16, 4, 1, C, C, C>(L, W, ld, m_dev, Rout, ldR, status, s);
    case 14: return run_col<32, 10, 3, 1, C, C, C>(L, W, ld, m_dev, Rout, ldR, status, s);
    default: return cudaErrorInvalidValue;
  }
}

bool usable(int id, int m_max) { return kCol[id].nw > 0 && kCol[id].nw * kCol[id].clw >= m_max; }

}  // namespace

int tsqr_col_pick(int m_max, Fmt in, Fmt comp, Fmt out, int* pr, int* nw, int* per_sm) {
  if (tune_get("tsqr.col", 1) == 0) return -1;
  int id = -1;
  const bool f32 = in == Fmt::F32 && comp == Fmt::F32 && out == Fmt::F32;
  const bool dfin = in == Fmt::F64 && comp == Fmt::DF && out == Fmt::DF;
  const bool dfup = in == Fmt::DF && comp == Fmt::DF && out == Fmt::DF;
  const bool f64 = in == Fmt::F64 && comp == Fmt::F64 && out == Fmt::F64;
  if (f32) {
    if (m_max <= 32) id = 10;
    else if (m_max <= 64) id = 11;
    else if (m_max <= 128) id = 12;
    else if (m_max <= 256) id = 13;
    else if (m_max <= 320) id = 14;
  } else if (dfin || dfup || f64) {
    if (m_max <= 32) id = 0;
    else if (m_max <= 64) id = 1;
    else if (m_max <= 80) id = 2;
    else if (m_max <= 128) id = 3;
    else if (m_max <= 160) id = 4;
    if ((dfin || dfup) && id >= 0) {
      // the autotuner may keep the row-group kernel for a bucket ("tsqr.col.<bucket>" = 0)
      char off[32];
      snprintf(off, sizeof(off), "tsqr.col.%d", id);
      if (tune_get(off, 1) == 0) return -1;
      // autotuned layout for this bucket ("tsqr.colcfg.<bucket>"), if it covers m
      char key[32];
      snprintf(key, sizeof(key), "tsqr.colcfg.%d", id);
      const int ov = tune_get(key, -1);
      if (ov >= 0 && ov <= 9 && usable(ov, m_max)) id = ov;
    } else if (f64 && id >= 0) {
      // native FP64: its own layout per bucket ("tsqr.colcfg64.<bucket>")
      char key[32];
      snprintf(key, sizeof(key), "tsqr.colcfg64.%d", id);
      const int ov = tune_get(key, -1);
      if (ov >= 0 && ov <= 9 && usable(ov, m_max)) id = ov;
    }
  }
  if (id < 0) return -1;
  *pr = 32 * kCol[id].prl;
  *nw = kCol[id].nw;
  *per_sm = kCol[id].minb;
  return id;
}

size_t tsqr_col_smem(int m_max, Fmt comp, int id) {
  // mbarriers and abort flag (64 bytes), packed R, two pivot slots
  const size_t tri = (size_t)m_max * (m_max + 1) / 2;
  return 64 + (tri + 2 * (size_t)(32 * kCol[id].prl + 2)) * fmt_bytes(comp);
}

cudaError_t launch_tsqr_col(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev,
                            void* Rout, int64_t ldR, int* status, cudaStream_t s) {
  if (L.in == Fmt::F64 && L.comp == Fmt::DF && L.out == Fmt::DF)
    return colk::run_df_tuned<double>(L, W, ld, m_dev, Rout, ldR, status, s);
  if ((L.in == Fmt::DF && L.comp == Fmt::DF && L.out == Fmt::DF) ||
      (L.in == Fmt::F64 && L.comp == Fmt::F64 && L.out == Fmt::F64))
    return tsqr_col_upper(L, W, ld, m_dev, Rout, ldR, status, s);
  if (L.in == Fmt::F32 && L.comp == Fmt::F32 && L.out == Fmt::F32)
    return run_f32(L, W, ld, m_dev, Rout, ldR, status, s);
  return cudaErrorInvalidValue;
}

}  // namespace tt

// ---- self-test of the bounded waits -----------------------------------------------------
namespace tt {
namespace {
// waits on an mbarrier that nothing arrives at, with the wait helper of the column-owned
// TSQR kernels and a short limit; the wait gives up and the kernel records DEV_ERR_TIMEOUT
__global__ void k_wait_selftest(int* status, long long limit) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) colk::mbar_init(&bar, 1);
  __syncthreads();
  if (!colk::mbar_wait(&bar, 0, limit) && threadIdx.x == 0) atomicOr(status, DEV_ERR_TIMEOUT);
}
}  // namespace
}  // namespace tt

extern "C" tt_status tt_wait_selftest(void* work, int64_t limit_cycles, void* stream) {
  using namespace tt;
  if (!work || ((uintptr_t)work & 255) || limit_cycles < 1000 || limit_cycles > kWaitCycles)
    return TT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(work, 0, sizeof(int), s) != cudaSuccess) return TT_ECUDA;
  k_wait_selftest<<<1, 32, 0, s>>>(static_cast<int*>(work), (long long)limit_cycles);
  return cudaGetLastError() == cudaSuccess ? TT_OK : TT_ECUDA;
}
