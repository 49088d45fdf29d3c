// tsqr_cta.cu -- instantiation and launch of the CTA-cooperative TSQR kernel.
#include <cstdio>

#include "tsqr_cta.cuh"

namespace tt {

namespace {

constexpr int kNW = 8;

template <int CG, int CL, int RL, int MINB, class C, class S, class RO, bool RGM = false>
cudaError_t run_cta(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev, void* Rout,
                    int64_t ldR, void* Rscr, int* status, cudaStream_t s) {
  auto kern = k_tsqr_cta<CG, CL, RL, kNW, MINB, RGM, C, S, RO>;
  if (L.smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<(unsigned)L.ctas, kNW * 32, L.smem, s>>>(static_cast<const S*>(W), L.rows, ld, m_dev,
                                                  L.mval, L.mmax, static_cast<RO*>(Rout), ldR,
                                                  L.mb, L.panels, static_cast<C*>(Rscr), status,
                                                  L.xr, L.xfix);
  return cudaGetLastError();
}

// layouts for 8-byte arithmetic (float-float, FP64): ids 0-5; m <= 128 keeps <= 128
// registers per thread so that two CTAs share an SM
template <class C, class S, class RO>
cudaError_t run_cfg(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev, void* Rout,
                    int64_t ldR, void* Rscr, int* status, cudaStream_t s) {
  switch (L.cfg) {
    case 0: return run_cta<8, 4, 8, 2, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 1: return run_cta<8, 8, 4, 2, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 2: return run_cta<8, 10, 4, 2, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 3: return run_cta<16, 8, 4, 2, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 4: return run_cta<16, 10, 6, 1, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 5: return run_cta<32, 7, 8, 1, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 6: return run_cta<32, 10, 6, 1, C, S, RO, true>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 7: return run_cta<32, 16, 4, 1, C, S, RO, true>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    // alternative layouts for the autotuner
    case 16: return run_cta<16, 4, 8, 2, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 17: return run_cta<16, 5, 8, 2, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 18: return run_cta<8, 8, 8, 1, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 19: return run_cta<32, 2, 16, 2, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 20: return run_cta<32, 3, 12, 2, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    default: return cudaErrorInvalidValue;
  }
}

// layouts for FP32 panels: ids 8-15
template <class C, class S, class RO>
cudaError_t run_cfg_f32(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev,
                        void* Rout, int64_t ldR, void* Rscr, int* status, cudaStream_t s) {
  switch (L.cfg) {
    case 8: return run_cta<8, 4, 16, 2, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 9: return run_cta<8, 8, 8, 2, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 10: return run_cta<8, 10, 6, 2, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 11: return run_cta<16, 8, 8, 2, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 12: return run_cta<16, 10, 6, 2, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 13: return run_cta<32, 7, 8, 2, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 14: return run_cta<32, 8, 8, 1, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    case 15: return run_cta<32, 10, 6, 1, C, S, RO>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// (CG, CL, RL, CTAs per SM) per configuration id; rows per panel = (8 warps * 32 / CG) * RL
static const int kCfg[21][4] = {{8, 4, 8, 2},  {8, 8, 4, 2},  {8, 10, 4, 2}, {16, 8, 4, 2},
                                {16, 10, 6, 1}, {32, 7, 8, 1}, {32, 10, 6, 1}, {32, 16, 4, 1},
                                {8, 4, 16, 2}, {8, 8, 8, 2},  {8, 10, 6, 2}, {16, 8, 8, 2},
                                {16, 10, 6, 2}, {32, 7, 8, 2}, {32, 8, 8, 1}, {32, 10, 6, 1},
                                {16, 4, 8, 2}, {16, 5, 8, 2}, {8, 8, 8, 1}, {32, 2, 16, 2},
                                {32, 3, 12, 2}};

int tsqr_cta_pick(int m_max, Fmt comp, int* pr, int* nw, int* per_sm) {
  int id = -1;
  if (m_max <= 32) id = 0;
  else if (m_max <= 64) id = 1;
  else if (m_max <= 80) id = 2;
  else if (m_max <= 128) id = 3;
  else if (m_max <= 160) id = 4;
  else if (m_max <= 224) id = 5;
  else if (comp == Fmt::F32 && m_max <= 256) id = 6;
  else if (comp == Fmt::F32 && m_max <= 320) id = 7;
  else if (comp != Fmt::F32 && m_max <= 320) id = 6;   // R in global memory
  else if (comp != Fmt::F32 && m_max <= 512) id = 7;   // R in global memory
  if (id < 0) return -1;
  if (comp == Fmt::F32) {
    id += 8;
  } else {
    // autotuned layout for this bucket ("tsqr.cfg.<bucket id>"), if it covers m
    char key[32];
    snprintf(key, sizeof(key), "tsqr.cfg.%d", id);
    const int ov = tune_get(key, -1);
    if (ov >= 16 && ov <= 20 && kCfg[ov][0] * kCfg[ov][1] >= m_max) id = ov;
  }
  *pr = (kNW * 32 / kCfg[id][0]) * kCfg[id][2];
  *nw = kNW;
  *per_sm = kCfg[id][3];
  return id;
}

bool tsqr_cta_r_global(int id) { return id == 6 || id == 7; }

size_t tsqr_cta_smem(int m_max, Fmt comp, int id) {
  const size_t tri = tsqr_cta_r_global(id) ? 0 : (size_t)m_max * (m_max + 1) / 2;
  return (tri + (size_t)(kNW + 1) * m_max) * fmt_bytes(comp);
}

size_t tsqr_cta_scratch(int m_max, Fmt comp, int id, int64_t ctas) {
  if (!tsqr_cta_r_global(id)) return 0;
  return (size_t)ctas * ((size_t)m_max * (m_max + 1) / 2) * fmt_bytes(comp);
}

cudaError_t launch_tsqr_cta(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev,
                            void* Rout, int64_t ldR, void* Rscr, int* status, cudaStream_t s) {
  if (L.in == Fmt::F64 && L.comp == Fmt::DF && L.out == Fmt::DF)
    return run_cfg<df, double, df>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
  if (L.in == Fmt::DF && L.comp == Fmt::DF && L.out == Fmt::DF)
    return run_cfg<df, df, df>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
  if (L.in == Fmt::F64 && L.comp == Fmt::F64 && L.out == Fmt::F64)
    return run_cfg<double, double, double>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
  if (L.in == Fmt::F32 && L.comp == Fmt::DF && L.out == Fmt::DF)
    return run_cfg<df, float, df>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
  if (L.in == Fmt::F32 && L.comp == Fmt::F32 && L.out == Fmt::F32)
    return run_cfg_f32<float, float, float>(L, W, ld, m_dev, Rout, ldR, Rscr, status, s);
  return cudaErrorInvalidValue;
}

}  // namespace tt
