// driver.cu -- host side of the engine: planning, workspace layout, the step
// loop of Alg. 2 and the C ABI declared in include/tt_svd.h.
//
// Step i (d..2) of Alg. 2 on one stream, with every data-dependent size kept in
// device memory (DevState) so nothing waits for the host:
//   TSQR levels (line 5) -> Jacobi SVD of R (line 6) -> rank choice (lines 7-8)
//   -> core T^(i) from V (line 9) -> W^(i-1) = W^(i) V_r (line 11)
// and at the end T^(1) = W^(1) (line 13).  Grids are sized for the worst-case
// rank r_k = min(r_max, n_1..n_k, n_{k+1}..n_d).
#include <algorithm>
#include <atomic>
#include <map>
#include <string>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "engine.h"
#include "tt_svd.h"

namespace tt {

static int g_nsm = 0;
static size_t g_smem_optin = 0;
static std::mutex g_props_mu;

static void load_props() {
  std::lock_guard<std::mutex> lk(g_props_mu);
  if (g_nsm) return;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) == cudaSuccess) {
    g_nsm = p.multiProcessorCount;
    g_smem_optin = p.sharedMemPerBlockOptin;
  } else {
    g_nsm = 152;
    g_smem_optin = 227 * 1024;
  }
}
int num_sms() { load_props(); return g_nsm; }
size_t max_smem_optin() { load_props(); return g_smem_optin; }

static inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// ---- tuning parameters (set by the autotuner through tt_tune_set) ---------------------
static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune;

int tune_get(const char* key, int dflt) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(key);
  return it == g_tune.end() ? dflt : it->second;
}

// ---- measurement: launch counter and optional per-kernel CUDA events -----------------
static std::atomic<long long> g_launches{0};

namespace prof {
struct Rec {
  int kind, step;
  double bytes, flops;
  cudaEvent_t a, b;
  const int* info_dev;  // optional device int read back with the record (Jacobi sweeps)
};
static std::mutex mu;
static bool on = false;
static std::vector<Rec> recs;
static std::vector<cudaEvent_t> pool;
static size_t pool_used = 0;

static cudaEvent_t take() {
  if (pool_used == pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    pool.push_back(e);
  }
  return pool[pool_used++];
}

// records an event pair around the kernels issued while it is alive
struct Scope {
  bool active = false;
  cudaStream_t s;
  Rec r;
  Scope(int kind, int step, double bytes, double flops, cudaStream_t st,
        const int* info = nullptr) : s(st) {
    std::lock_guard<std::mutex> lk(mu);
    if (!on) return;
    r.kind = kind; r.step = step; r.bytes = bytes; r.flops = flops; r.info_dev = info;
    r.a = take(); r.b = take();
    if (!r.a || !r.b) return;
    cudaEventRecord(r.a, s);
    active = true;
  }
  ~Scope() {
    if (!active) return;
    cudaEventRecord(r.b, s);
    std::lock_guard<std::mutex> lk(mu);
    recs.push_back(r);
  }
};
}  // namespace prof

// ---- TSQR plan --------------------------------------------------------------------
static TsqrLevel make_level(int64_t rows, int m_max, Fmt in, Fmt comp, Fmt out, bool first,
                            int nsm, int64_t ctas_override) {
  TsqrLevel L{};
  L.rows = rows;
  L.mmax = m_max;
  L.mval = m_max;
  L.mb = m_max;
  L.in = in;
  L.comp = comp;
  L.out = out;
  if (!first && m_max >= tune_get("tsqr.merge_m", 96) && tsqr_merge_ok(m_max, in, comp) &&
      rows % m_max == 0) {
    // stacked triangles: binary tree of structured pairwise merges
    const int64_t nblk = rows / m_max;
    L.kind = 5;
    L.maxm = m_max;
    L.nw = 16;
    L.pr = m_max;
    L.panels = nblk;
    L.ctas = (nblk + 1) / 2;
    L.warps = L.ctas;
    L.smem = 0;
    return L;
  }
  int64_t warps_cap;
  int cta_pr = 0, cta_nw = 0, cta_per_sm = 1;
  int cta_kind = 3;
  int cta_cfg = -1;
  // native FP64, 16 < m <= 512: the blocked kernel ("tsqr.blk64" up to m = 80, "tsqr.blkw" above)
  if (in == Fmt::F64 && comp == Fmt::F64 && out == Fmt::F64 && m_max > 16 && m_max <= 512 &&
      tune_get("tsqr.blk64", 1) != 0 && (m_max <= 80 || tune_get("tsqr.blkw", 1) != 0) &&
      (m_max <= 64 || tune_get("tsqr.blk80", 1) != 0)) {
    cta_kind = 6;
    cta_cfg = 0;
    cta_pr = tsqr_blk_rows(m_max);
    cta_nw = 8;
    cta_per_sm = tsqr_blk_per_sm(m_max);
  }
  if (cta_cfg < 0 && m_max > 16) cta_cfg = tsqr_col_pick(m_max, in, comp, out, &cta_pr, &cta_nw, &cta_per_sm);
  if (cta_cfg < 0) {
    cta_kind = 4;
    cta_cfg = tsqr_cols_pick(m_max, in, comp, out, &cta_pr, &cta_nw, &cta_per_sm);
  }
  if (cta_cfg < 0) {
    cta_kind = 2;
    cta_cfg = m_max > 16 ? tsqr_cta_pick(m_max, comp, &cta_pr, &cta_nw, &cta_per_sm) : -1;
  }
  if (cta_cfg >= 0) {
    // CTA-cooperative panels: one partial R per CTA
    L.kind = cta_kind;
    L.cfg = cta_cfg;
    L.maxm = m_max;
    L.pr = cta_pr;
    L.nw = cta_nw;
    L.smem = cta_kind == 6   ? tsqr_blk_smem(m_max)
             : cta_kind == 3 ? tsqr_col_smem(m_max, comp, cta_cfg)
             : cta_kind == 4 ? tsqr_cols_smem(m_max, cta_cfg)
                             : tsqr_cta_smem(m_max, comp, cta_cfg);
    L.panels = (rows + L.pr - 1) / L.pr;
    int64_t ctas;
    if (first) {
      // the tree over the partial R's costs ~P m^3 against rows m^2 for this level:
      // keep P <= rows / (4 m) so the tree stays a fraction of the work.  With the merge
      // tree (m^3 / 6 per pair, log2 P deep) more and shorter first-level panels pay.
      const bool merges = m_max >= tune_get("tsqr.merge_m", 96);
      // rows per CTA >= q4 m / 4 (measured best: m rows for m >= 200, 2 m below)
      // (FP32 panels at m >= 200: 8x fewer first-level R's than float-float and FP64 -- the
      // FP32 panels are cheap, the float-float tree above them is not: measured on the
      // 8^10 FP32 form at r_max = 32, 128.6 ms against 138.0 ms with the float-float setting)
      const int q_def = m_max >= 200 ? (comp == Fmt::F32 ? tune_get("tsqr.pcap_q32", 32) : 4) : 8;
      const int64_t q4 = merges ? std::max(1, tune_get("tsqr.pcap_q", q_def)) : 16;
      const int64_t p_cap = std::max<int64_t>(1, 4 * rows / (q4 * (int64_t)m_max));
      ctas = std::min<int64_t>(std::min<int64_t>(L.panels, (int64_t)nsm * cta_per_sm), p_cap);
      if (ctas_override > 0) ctas = std::min<int64_t>(L.panels, ctas_override);
    } else {
      // upper levels: enough panels per CTA that a level shrinks the R count >= 4x
      const int64_t ppc = std::max<int64_t>(2, (4 * (int64_t)L.mb + L.pr - 1) / L.pr);
      ctas = (L.panels + ppc - 1) / ppc;
    }
    if (ctas < 1) ctas = 1;
    L.ctas = ctas;
    L.warps = ctas;
    return L;
  }
  if (m_max <= 16) {
    L.kind = 0;
    L.maxm = m_max <= 4 ? 4 : (m_max <= 8 ? 8 : 16);
    // rows per lane 32 / maxm (or 64 / maxm, "tsqr.narrow_k"), 4 CTAs of 4 warps per SM:
    // measured on GB300 for 8^10 at r_max = 1 (first step 2^27 x 8), 19.7 ms per TT-SVD
    // against 20.2 ms with 64 / maxm and 2 CTAs per SM (both without renormalisation)
    L.pr = 32 * ((tune_get("tsqr.narrow_k", 32) == 64 ? 64 : 32) / L.maxm);
    L.smem = 0;
    warps_cap = (int64_t)nsm * tune_get("tsqr.narrow_cpsm", 4) * 4;
  } else {
    L.kind = 1;
    int nch = 1;
    while (32 * nch < m_max) nch *= 2;
    L.maxm = 32 * nch;
    const size_t es = fmt_bytes(comp);
    const int mstr = m_max | 1;
    const size_t budget = 200 * 1024;
    int nw = 4, pr = 128;
    bool ok = false;
    for (int w = 4; w >= 1 && !ok; w /= 2)
      for (int p = 128; p >= 32 && !ok; p /= 2)
        if ((size_t)w * p * mstr * es <= budget) { nw = w; pr = p; ok = true; }
    if (!ok) { nw = 1; pr = 32; }
    L.pr = pr;
    L.nw = nw;
    L.smem = (size_t)nw * pr * mstr * es;
    const int per_sm = L.smem <= 100 * 1024 ? 2 : 1;
    warps_cap = (int64_t)nsm * per_sm * nw;
  }
  L.panels = (rows + L.pr - 1) / L.pr;
  int64_t warps;
  if (first) {
    warps = std::min<int64_t>(L.panels, warps_cap);
    if (ctas_override > 0) warps = std::min<int64_t>(L.panels, ctas_override * (L.kind ? L.nw : 4));
  } else {
    // upper levels: every warp folds at least 8 panels or 8 stacked R blocks, so the
    // number of partial R's drops by 8x or more per level
    const int64_t nblocks = (rows + L.mb - 1) / L.mb;
    const int64_t units = std::min<int64_t>(L.panels, nblocks);
    warps = std::max<int64_t>(1, std::min<int64_t>(warps_cap, (units + 7) / 8));
  }
  if (warps < 1) warps = 1;
  const int nwmax = L.kind == 0 ? 4 : L.nw;
  L.nw = (int)std::min<int64_t>(nwmax, warps);
  L.ctas = (warps + L.nw - 1) / L.nw;
  L.warps = L.ctas * L.nw;
  return L;
}

static std::vector<TsqrLevel> plan_tsqr(int64_t rows, int m_max, Fmt in, Fmt comp1, Fmt comp2,
                                        int nsm, int64_t ctas_override, int chunks = 1) {
  std::vector<TsqrLevel> lv;
  Fmt cur = in;
  int64_t r = rows;
  bool first = true;
  for (int guard = 0; guard < 24; ++guard) {
    const Fmt comp = first ? comp1 : comp2;
    const Fmt out = comp;  // partial R's are stored in the arithmetic of their level
    if (first && chunks > 1) {
      // first level in row blocks (input streamed in): every block is launched on its own
      // with the whole grid and writes its own partial R's
      const int64_t crows = (rows + chunks - 1) / chunks;
      TsqrLevel L = make_level(crows, m_max, cur, comp, out, true, nsm, ctas_override);
      {
        L.chunks = (int)((rows + crows - 1) / crows);
        L.chunk_rows = crows;
        L.chunk_parts = L.warps;
        L.rows = rows;
        L.warps = L.chunk_parts * L.chunks;
        lv.push_back(L);
        r = L.warps * L.mb;
        cur = out;
        first = false;
        if (L.warps == 1) return lv;
        continue;
      }
    }
    TsqrLevel L = make_level(r, m_max, cur, comp, out, first, nsm, ctas_override);
    lv.push_back(L);
    if (L.warps == 1) return lv;
    r = L.warps * L.mb;
    cur = out;
    first = false;
  }
  lv.clear();  // no single R after the level limit: the caller reports TT_ENOTIMPL
  return lv;
}

// ---- whole-call plan -----------------------------------------------------------------
struct StepPlan {
  int i;
  int64_t rows;
  int m_max;
  int r_max_out;
  bool elide;
  bool wide = false;  // rows < m: Jacobi on W^T directly, no TSQR (Sec. 3.1.2, R = [R_1; 0])
  Fmt in_fmt;
  int out_buf;   // -1: none (elided)
  std::vector<TsqrLevel> levels;
  TsmmCfg tsmm;
};

struct Plan {
  int d;
  int64_t n[TT_MAX_D];
  int r_max;
  double tol;
  tt_dtype dt;
  int in_chunks = 1;   // > 1: X arrives from the host in row blocks of the first active step
  Fmt xfmt, inter, comp_tsqr1, comp_tsqr2, comp_svd, comp_tsmm;
  std::vector<StepPlan> steps;
  int r_worst[TT_MAX_D + 1];
  // workspace offsets
  size_t off_state, off_W[2], off_R[2], off_Rscr, off_A, off_V, off_Vout, off_sig, total;
  size_t szW[2], szR, szRscr, szJ, szVout;
  int ldA, m_all_max;
};

static void worst_ranks(int d, const int64_t* n, int r_max, int* r) {
  r[0] = 1;
  r[d] = 1;
  for (int k = 1; k < d; ++k) {
    double left = 1, right = 1;
    for (int a = 0; a < k; ++a) left *= (double)n[a];
    for (int a = k; a < d; ++a) right *= (double)n[a];
    double v = std::min<double>((double)r_max, std::min(left, right));
    r[k] = (int)v;
  }
}

static tt_status validate(int d, const int64_t* n, int r_max, double tol) {
  if (d < 1 || d > TT_MAX_D || !n || r_max < 1 || !(tol >= 0.0) || !std::isfinite(tol))
    return TT_EINVAL;
  double total = 1;
  for (int i = 0; i < d; ++i) {
    if (n[i] < 1) return TT_EINVAL;
    total *= (double)n[i];
  }
  if (total > 9.0e18) return TT_EINVAL;
  return TT_OK;
}

static tt_status build_plan(int d, const int64_t* n, int r_max, double tol, tt_dtype dt,
                            const tt_opts* opts, Plan& P, int in_chunks = 1) {
  tt_status st = validate(d, n, r_max, tol);
  if (st != TT_OK) return st;
  if (dt != TT_F64 && dt != TT_F32) return TT_EINVAL;
  const tt_arith ar = opts ? opts->arith : TT_ARITH_AUTO;
  const bool no_elide = opts && opts->no_elide;
  const int64_t ctas_override = opts ? opts->tsqr_ctas : 0;
  P.d = d;
  for (int i = 0; i < d; ++i) P.n[i] = n[i];
  P.r_max = r_max;
  P.tol = tol;
  P.dt = dt;
  P.in_chunks = std::max(1, in_chunks);
  if (dt == TT_F32) {
    P.xfmt = Fmt::F32; P.inter = Fmt::F32;
    P.comp_tsqr1 = Fmt::F32; P.comp_tsqr2 = Fmt::DF; P.comp_svd = Fmt::DF; P.comp_tsmm = Fmt::F32;
  } else if (ar == TT_ARITH_F64) {
    P.xfmt = Fmt::F64; P.inter = Fmt::F64;
    P.comp_tsqr1 = P.comp_tsqr2 = P.comp_svd = P.comp_tsmm = Fmt::F64;
  } else {
    P.xfmt = Fmt::F64; P.inter = Fmt::DF;
    P.comp_tsqr1 = P.comp_tsqr2 = P.comp_svd = P.comp_tsmm = Fmt::DF;
  }
  worst_ranks(d, n, r_max, P.r_worst);
  const int nsm = num_sms();
  P.steps.clear();
  int64_t nbar = 1;
  for (int i = 0; i < d; ++i) nbar *= n[i];
  int64_t rows = d >= 1 ? nbar / n[d - 1] : 1;
  Fmt cur = P.xfmt;
  int par = 0;
  P.szW[0] = P.szW[1] = 0;
  P.szR = 0;
  P.szRscr = 0;
  P.m_all_max = 1;
  size_t wide_g = 0;  // the wide Jacobi's working copy where it leaves shared memory
  for (int i = d; i >= 2; --i) {
    StepPlan S;
    S.i = i;
    S.rows = rows;
    const int64_t m64 = n[i - 1] * (int64_t)P.r_worst[i];
    if (m64 > kMaxM) return TT_ENOTIMPL;
    S.m_max = (int)m64;
    S.r_max_out = P.r_worst[i - 1];
    S.elide = (tol == 0.0) && !no_elide && std::min<int64_t>(r_max, rows) >= S.m_max;
    S.in_fmt = cur;
    S.out_buf = -1;
    P.m_all_max = std::max(P.m_all_max, S.m_max);
    if (!S.elide) {
      const bool first_active = P.szR == 0;  // no TSQR planned yet
      S.wide = !first_active && rows < S.m_max && tune_get("svd.wide", 1) &&
               jacobi_wide_fits(P.comp_svd, (int)rows, S.m_max);
      if (S.wide) wide_g = std::max(wide_g, jacobi_wide_gbytes(P.comp_svd, (int)rows, S.m_max));
      if (!S.wide) {
        S.levels = plan_tsqr(rows, S.m_max, cur, P.comp_tsqr1, P.comp_tsqr2, nsm, ctas_override,
                             first_active ? P.in_chunks : 1);
        if (S.levels.empty()) return TT_ENOTIMPL;
      }
      for (auto& L : S.levels) {
        P.szR = std::max(P.szR, (size_t)L.warps * L.mb * S.m_max * fmt_bytes(L.out));
        P.szRscr = std::max(P.szRscr, tsqr_wide_scratch_bytes(L));
      }
      S.tsmm = plan_tsmm(cur, P.comp_tsmm, P.comp_svd, P.inter, S.m_max, S.r_max_out, rows, nsm);
      S.out_buf = par;
      P.szW[par] = std::max(P.szW[par], (size_t)rows * S.r_max_out * fmt_bytes(P.inter));
      par ^= 1;
      cur = P.inter;
    }
    P.steps.push_back(S);
    rows /= n[i - 2];
  }
  const int mp = P.m_all_max + (P.m_all_max & 1);
  P.ldA = mp;
  P.szJ = std::max(jacobi_scratch_bytes(P.comp_svd, P.m_all_max), wide_g);
  P.szVout = (size_t)mp * mp * fmt_bytes(P.comp_svd);
  size_t off = 0;
  P.off_state = off; off += align256(sizeof(DevState));
  P.off_W[0] = off; off += align256(P.szW[0]);
  P.off_W[1] = off; off += align256(P.szW[1]);
  P.off_R[0] = off; off += align256(P.szR);
  P.off_R[1] = off; off += align256(P.szR);
  P.off_Rscr = off; off += align256(P.szRscr);
  P.off_A = off; off += align256(P.szJ);
  P.off_V = P.off_A + P.szJ / 2;
  P.off_Vout = off; off += align256(P.szVout);
  P.off_sig = off; off += align256((size_t)mp * sizeof(double));
  P.total = off;
  return TT_OK;
}

// ---- thick-bounds variant (Alg. 3) -----------------------------------------------------
// line 1: the smallest k with m = n_{d-k+1}...n_d >= max(m_min, r_est / f1_min)
static int thick_k(int d, const int64_t* n, double m_min, double f1_min, double r_est) {
  double m = 1;
  for (int k = 1; k <= d; ++k) {
    m *= (double)n[d - k];
    if (m >= std::max(m_min, r_est / f1_min)) return k;
  }
  return d;
}

struct ThickPlan {
  int k = 0, d1 = 0, d2 = 0;
  int64_t n1[TT_MAX_D], n2[TT_MAX_D];
  Plan P1, P2;
  int a = 0, b = 0, r1 = 0, rho1 = 0;
  size_t off_w1 = 0, off_w2 = 0, off_tbar = 0, off_s0 = 0, off_told = 0, off_r1 = 0, off_r2 = 0,
         off_e = 0, total = 0;
};

// TT_OK with T.k >= 2: the thick plan; TT_OK with T.k < 2: the plain algorithm applies
static tt_status build_thick(int d, const int64_t* n, int r_max, double tol, tt_dtype dt,
                             const tt_opts* opts, ThickPlan& T) {
  tt_status st = validate(d, n, r_max, tol);
  if (st != TT_OK) return st;
  const double f1 = opts->thick_f1_min > 0 ? opts->thick_f1_min : 0.5;
  const double rest = opts->thick_r_est > 0 ? opts->thick_r_est : r_max;
  const int k = thick_k(d, n, opts->thick_m_min, f1, rest);
  T.k = k;
  if (k <= 1 || k >= d) return TT_OK;
  if (tol != 0.0) return TT_ENOTIMPL;
  tt_opts o = *opts;
  o.thick_m_min = 0;
  T.d1 = d - k + 1;
  T.d2 = k + 1;
  int64_t m = 1;
  for (int i = d - k; i < d; ++i) m *= n[i];
  for (int i = 0; i < d - k; ++i) T.n1[i] = n[i];
  T.n1[d - k] = m;
  if ((st = build_plan(T.d1, T.n1, r_max, 0.0, dt, &o, T.P1)) != TT_OK) return st;
  T.a = T.P1.r_worst[d - k - 1];
  T.b = (int)n[d - k - 1];
  T.r1 = T.P1.r_worst[d - k];
  T.n2[0] = T.r1;
  for (int i = 1; i <= k; ++i) T.n2[i] = n[d - k + i - 1];
  // the recovery decomposes the FP64 core T_bar, whatever the storage of X
  if ((st = build_plan(T.d2, T.n2, r_max, 0.0, TT_F64, &o, T.P2)) != TT_OK) return st;
  T.rho1 = T.P2.r_worst[1];
  size_t off = 0;
  T.off_w1 = off; off += align256(T.P1.total);
  T.off_w2 = off; off += align256(T.P2.total);
  T.off_tbar = off; off += align256((size_t)T.r1 * m * sizeof(double));
  T.off_s0 = off; off += align256((size_t)T.r1 * T.rho1 * sizeof(double));
  T.off_told = off; off += align256((size_t)T.a * T.b * T.r1 * sizeof(double));
  T.off_r1 = off; off += align256((size_t)(T.d1 + 1) * sizeof(int64_t));
  T.off_r2 = off; off += align256((size_t)(T.d2 + 1) * sizeof(int64_t));
  T.off_e = off; off += align256(2 * sizeof(double));
  T.total = off;
  return TT_OK;
}

// ---- two-sided variant (Alg. 4) ------------------------------------------------------
// The work tensor Z has the shape (r_L, n_a, ..., n_b, r_R) in Fortran order.  A right
// step on b is the one-sided step; a left step on a transposes the (r_L n_a) x rest
// unfolding, runs the same TSQR + SVD + W*V_r on it and transposes the product back.
struct TsStep {
  bool right = true, elide = false;
  int dim = 0;          // 1-based dimension whose core the step writes
  int64_t rows = 0;     // rows of the tall matrix of the step
  int m = 0, r = 0;
  Fmt in = Fmt::F64;    // format of Z before the step
  std::vector<TsqrLevel> levels;
  TsmmCfg tsmm{};
  int zin = -1, zout = -1;  // Z buffers (-1: X)
};

struct TsPlan {
  int d = 0, mid = 0, rl = 1, rr = 1;
  int64_t n[TT_MAX_D];
  int64_t ranks[TT_MAX_D + 1];
  Fmt xfmt, inter, comp_tsqr1, comp_tsqr2, comp_svd, comp_tsmm;
  std::vector<TsStep> steps;
  int zfinal = -1;
  Fmt zfmt_final = Fmt::F64;
  int ldA = 2, m_all_max = 1;
  size_t szZ[2] = {0, 0}, szT = 0, szY = 0, szR = 0, szRscr = 0, szJ = 0, szVout = 0;
  size_t off_state = 0, off_Z[2] = {0, 0}, off_T = 0, off_Y = 0, off_R[2] = {0, 0}, off_Rscr = 0,
         off_A = 0, off_V = 0, off_Vout = 0, off_sig = 0, off_e = 0, total = 0;
};

static tt_status build_two_sided(int d, const int64_t* n, int r_max, double tol, tt_dtype dt,
                                 const tt_opts* opts, TsPlan& T) {
  tt_status st = validate(d, n, r_max, tol);
  if (st != TT_OK) return st;
  if (dt != TT_F64 && dt != TT_F32) return TT_EINVAL;
  if (tol != 0.0 || (opts && opts->thick_m_min > 0)) return TT_ENOTIMPL;
  // the arithmetic of the one-sided plan
  Plan P;
  tt_opts o = opts ? *opts : tt_opts{};
  o.two_sided = 0;
  if ((st = build_plan(d, n, r_max, tol, dt, &o, P)) != TT_OK) return st;
  T.d = d;
  for (int i = 0; i < d; ++i) T.n[i] = n[i];
  T.xfmt = P.xfmt; T.inter = P.inter; T.comp_tsqr1 = P.comp_tsqr1; T.comp_tsqr2 = P.comp_tsqr2;
  T.comp_svd = P.comp_svd; T.comp_tsmm = P.comp_tsmm;
  for (int i = 0; i <= d; ++i) T.ranks[i] = 1;
  const int nsm = num_sms();
  int a = 1, b = d, rL = 1, rR = 1, t = 0, zcur = -1;
  Fmt cur = T.xfmt;
  auto prod = [&](int lo, int hi) {  // n_lo ... n_hi (1-based, inclusive), 1 if empty
    int64_t v = 1;
    for (int i = lo; i <= hi; ++i) v *= n[i - 1];
    return v;
  };
  while (a < b) {
    TsStep S;
    S.right = (t % 2 == 0);
    S.in = cur;
    S.zin = zcur;
    if (S.right) {
      S.dim = b;
      S.rows = (int64_t)rL * prod(a, b - 1);
      const int64_t m64 = n[b - 1] * (int64_t)rR;
      if (m64 > kMaxM) return TT_ENOTIMPL;
      S.m = (int)m64;
      S.r = (int)std::min<int64_t>(r_max, std::min<int64_t>(S.rows, S.m));
      S.elide = std::min<int64_t>(r_max, S.rows) >= S.m;
    } else {
      S.dim = a;
      S.rows = prod(a + 1, b) * (int64_t)rR;
      const int64_t m64 = (int64_t)rL * n[a - 1];
      if (m64 > kMaxM) return TT_ENOTIMPL;
      S.m = (int)m64;
      S.r = (int)std::min<int64_t>(r_max, std::min<int64_t>(S.rows, S.m));
      S.elide = std::min<int64_t>(r_max, S.rows) >= S.m;
    }
    T.m_all_max = std::max(T.m_all_max, S.m);
    if (!S.elide) {
      S.levels = plan_tsqr(S.rows, S.m, cur, T.comp_tsqr1, T.comp_tsqr2, nsm, 0);
      if (S.levels.empty()) return TT_ENOTIMPL;
      for (auto& L : S.levels) {
        T.szR = std::max(T.szR, (size_t)L.warps * L.mb * S.m * fmt_bytes(L.out));
        T.szRscr = std::max(T.szRscr, tsqr_wide_scratch_bytes(L));
      }
      S.tsmm = plan_tsmm(cur, T.comp_tsmm, T.comp_svd, T.inter, S.m, S.r, S.rows, nsm);
      S.zout = zcur == 0 ? 1 : 0;
      T.szZ[S.zout] = std::max(T.szZ[S.zout], (size_t)S.rows * S.r * fmt_bytes(T.inter));
      if (!S.right) {
        T.szT = std::max(T.szT, (size_t)S.rows * S.m * fmt_bytes(cur));
        T.szY = std::max(T.szY, (size_t)S.rows * S.r * fmt_bytes(T.inter));
      }
      zcur = S.zout;
      cur = T.inter;
    }
    if (S.right) {
      T.ranks[b - 1] = S.r;
      rR = S.r;
      --b;
    } else {
      T.ranks[a] = S.r;
      rL = S.r;
      ++a;
    }
    T.steps.push_back(S);
    ++t;
  }
  T.mid = a;
  T.rl = rL;
  T.rr = rR;
  T.zfinal = zcur;
  T.zfmt_final = cur;
  const int mp = T.m_all_max + (T.m_all_max & 1);
  T.ldA = mp;
  T.szJ = jacobi_scratch_bytes(T.comp_svd, T.m_all_max);
  T.szVout = (size_t)mp * mp * fmt_bytes(T.comp_svd);
  size_t off = 0;
  T.off_state = off; off += align256(sizeof(DevState));
  T.off_Z[0] = off; off += align256(T.szZ[0]);
  T.off_Z[1] = off; off += align256(T.szZ[1]);
  T.off_T = off; off += align256(T.szT);
  T.off_Y = off; off += align256(T.szY);
  T.off_R[0] = off; off += align256(T.szR);
  T.off_R[1] = off; off += align256(T.szR);
  T.off_Rscr = off; off += align256(T.szRscr);
  T.off_A = off; off += align256(T.szJ);
  T.off_V = T.off_A + T.szJ / 2;
  T.off_Vout = off; off += align256(T.szVout);
  T.off_sig = off; off += align256((size_t)mp * sizeof(double));
  T.off_e = off; off += align256(sizeof(double));
  T.total = off;
  return TT_OK;
}

// last CUDA failure seen by a tt_* call on this thread (tt_last_error)
static thread_local char g_last_err[256] = "";
static void note_err(cudaError_t e, const char* what, int line) {
  snprintf(g_last_err, sizeof(g_last_err), "%s (%s) at driver.cu:%d: %s", cudaGetErrorName(e),
           cudaGetErrorString(e), line, what);
}
static tt_status cuda_err_at(cudaError_t e, const char* what, int line) {
  if (e == cudaSuccess) return TT_OK;
  note_err(e, what, line);
  return TT_ECUDA;
}
#define cuda_err(x) cuda_err_at((x), #x, __LINE__)
void set_last_error_text(const char* text) { snprintf(g_last_err, sizeof(g_last_err), "%s", text); }
#define TT_CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { note_err(e_, #x, __LINE__); return TT_ECUDA; } } while (0)

static void sigma_layout(int d, const int64_t* n, const int* rw, int64_t* stride, int64_t* count) {
  int64_t s = 1;
  int64_t rows = 1;
  for (int a = 0; a < d - 1; ++a) rows *= n[a];
  for (int i = d; i >= 2; --i) {
    const int64_t m = n[i - 1] * (int64_t)rw[i];
    s = std::max<int64_t>(s, std::min<int64_t>(m, rows));
    rows /= n[i - 2];
  }
  *stride = s;
  *count = s * std::max(d - 1, 0);
}

// row blocks of the first TSQR level when X is copied in from the host
constexpr int kDefaultInChunks = 16;

// X arriving from the host: the copy stream and one event per row block of the first level
struct HostIn {
  const char* X_host = nullptr;
  cudaStream_t cs = nullptr;
  std::vector<cudaEvent_t> ev;
};

// largest encoded exponent (engine.h, XRange) of a strided sample of a host array
template <class T>
static int host_sample_enc(const T* X, int64_t count) {
  const int64_t ns = std::min<int64_t>(count, 4096);
  const int64_t stride = ns > 0 ? count / ns : 1;
  int best = 0;
  for (int64_t j = 0; j < ns; ++j) {
    const double x = (double)X[j * stride];
    int e = 0;
    if (!std::isfinite(x)) e = kXrNonfinite;
    else if (x != 0.0) {
      int ex = 0;
      std::frexp(x, &ex);  // |x| = f 2^ex with f in [0.5, 1)
      e = ex - 1 + kXrBias;
    }
    best = std::max(best, e);
  }
  return best;
}

static tt_status run_plan(const Plan& P, const void* X, double* const* cores_out,
                          int64_t* ranks_out, double* sigma_out, double* err2_out, void* work,
                          cudaStream_t s, HostIn* hin = nullptr) {
  char* wb = static_cast<char*>(work);
  DevState* st = reinterpret_cast<DevState*>(wb + P.off_state);
  int* status = &st->status;
  const int d = P.d;
  int64_t sig_stride = 0, sig_count = 0;
  sigma_layout(d, P.n, P.r_worst, &sig_stride, &sig_count);
  TT_CK(launch_init_state(st, d, P.n, s));
  // FP64 input in float-float and FP32 input: the exponent shift of X (engine.h, XRange)
  XRange* xr = (P.comp_tsqr1 == Fmt::DF || P.xfmt == Fmt::F32) ? &st->xr : nullptr;
  bool first_active = true;
  if (xr) {
    int64_t nbar = 1;
    for (int a = 0; a < d; ++a) nbar *= P.n[a];
    if (hin && hin->X_host) {
      const void* xh = hin->X_host;
      const int enc = P.xfmt == Fmt::F32 ? host_sample_enc(static_cast<const float*>(xh), nbar)
                                         : host_sample_enc(static_cast<const double*>(xh), nbar);
      TT_CK(launch_range_set_sample(xr, enc, s));
    } else {
      TT_CK(launch_range_sample(P.xfmt, X, nbar, xr, s));
    }
    ++g_launches;
  }
  if (hin && hin->X_host) {
    // X is copied in row blocks by the first TSQR level when that level reads it;
    // otherwise (every step elided) in one piece here
    bool streamed = false;
    for (const StepPlan& S : P.steps)
      if (!S.elide) {
        streamed = !S.levels.empty() && S.levels[0].chunks > 1;
        break;
      }
    if (!streamed) {
      size_t nb = fmt_bytes(P.xfmt);
      for (int a = 0; a < d; ++a) nb *= (size_t)P.n[a];
      TT_CK(cudaMemcpyAsync(const_cast<void*>(X), hin->X_host, nb, cudaMemcpyHostToDevice, s));
    }
  }
  ++g_launches;
  const void* cur = X;
  Fmt cur_fmt = P.xfmt;
  int64_t rows = 1;
  for (int a = 0; a < d - 1; ++a) rows *= P.n[a];
  const double tol2 = (d > 1) ? P.tol * P.tol / (double)(d - 1) : 0.0;
  bool first_level_done = false;  // the previous step's fused W V_r wrote this step's level 0
  for (size_t si = 0; si < P.steps.size(); ++si) {
    const StepPlan& S = P.steps[si];
    const StepPlan* next = si + 1 < P.steps.size() ? &P.steps[si + 1] : nullptr;
    const int i = S.i;
    double* sig_step = sigma_out ? sigma_out + (int64_t)(d - i) * sig_stride : nullptr;
    if (S.elide) {
      TT_CK(launch_core_identity(S.m_max, cores_out[i - 1], s));
      if (sig_step) { TT_CK(launch_fill_nan(sig_step, sig_stride, s)); ++g_launches; }
      // record r_{i-1} = m_i and m_{i-1} = n_{i-1} m_i on the device
      TT_CK(launch_set_rank(st, i, (int)P.n[i - 2], S.m_max, s));
      g_launches += 2;
      rows /= P.n[i - 2];
      continue;
    }
    double* sig = reinterpret_cast<double*>(wb + P.off_sig);
    void* Vout = wb + P.off_Vout;
    const double mm = (double)S.m_max;
    if (S.wide) {
      prof::Scope ps(2, i, (double)rows * mm * fmt_bytes(cur_fmt), 0.0, s, &st->sweeps[i]);
      TT_CK(launch_jacobi_wide(P.comp_svd, cur_fmt, cur, rows, (int)rows, &st->m[i], S.m_max, sig,
                               Vout, P.ldA, status, &st->sweeps[i], wb + P.off_A, s));
      ++g_launches;
    } else {
      // TSQR levels
      const void* lin = cur;
      int64_t lld = rows;
      void* Rfin = nullptr;
      int64_t ldRfin = 0;
      Fmt rfmt = Fmt::DF;
      for (size_t l = 0; l < S.levels.size(); ++l) {
        TsqrLevel L = S.levels[l];
        void* Rout = wb + P.off_R[l & 1];
        const int64_t ldR = L.warps * L.mb;
        // one launch of level L, or of each of its row blocks (xfix: the re-run pass)
        auto launch_level = [&](int xfix) -> tt_status {
          L.xfix = xfix;
          if (L.chunks > 1) {
            // first level in row blocks: block c (rows r0..r1 of every column) is copied from
            // the host when X comes from there, and its launch waits only for that copy
            const size_t es = fmt_bytes(L.in);
            for (int c = 0; c < L.chunks; ++c) {
              const int64_t r0 = (int64_t)c * L.chunk_rows;
              const int64_t r1 = std::min<int64_t>(L.rows, r0 + L.chunk_rows);
              if (!xfix && hin && hin->X_host && lin == X) {
                TT_CK(cudaMemcpy2DAsync(static_cast<char*>(const_cast<void*>(X)) + r0 * es, lld * es,
                                        hin->X_host + r0 * es, lld * es, (size_t)(r1 - r0) * es,
                                        (size_t)S.m_max, cudaMemcpyHostToDevice, hin->cs));
                TT_CK(cudaEventRecord(hin->ev[c], hin->cs));
                TT_CK(cudaStreamWaitEvent(s, hin->ev[c], 0));
              }
              TsqrLevel Lc = L;
              Lc.rows = r1 - r0;
              Lc.panels = (Lc.rows + L.pr - 1) / L.pr;
              Lc.chunks = 1;
              Lc.warps = L.chunk_parts;
              char* Rc = static_cast<char*>(Rout) + (size_t)c * L.chunk_parts * L.mb * fmt_bytes(L.out);
              TT_CK(launch_tsqr_level(Lc, static_cast<const char*>(lin) + r0 * es, lld, &st->m[i], Rc,
                                      ldR, wb + P.off_Rscr, status, s));
              ++g_launches;
            }
            return TT_OK;
          }
          TT_CK(launch_tsqr_level(L, lin, lld, &st->m[i], Rout, ldR, wb + P.off_Rscr, status, s));
          ++g_launches;
          return TT_OK;
        };
        if (l == 0 && first_level_done) {
          // written by the previous step's fused W V_r (tsqr_fused.cu)
        } else {
          prof::Scope ps(l == 0 ? 0 : 1, i, (double)L.rows * mm * fmt_bytes(L.in),
                         2.0 * (double)L.rows * mm * mm, s);
          if (xr && first_active && l == 0) L.xr = xr;  // this level reads X
          const tt_status e = launch_level(0);
          if (e != TT_OK) return e;
        }
        if (L.xr) {
          // keep the shift, or run the level again with the shift of the largest entry it met
          // (that launch returns at once when the shift was kept)
          prof::Scope ps(5, i, 0.0, 0.0, s);
          TT_CK(launch_range_decide(xr, s));
          ++g_launches;
          const tt_status e = launch_level(1);
          if (e != TT_OK) return e;
        }
        lin = Rout;
        lld = ldR;
        Rfin = Rout;
        ldRfin = ldR;
        rfmt = L.out;
      }
      // small SVD of R
      {
        prof::Scope ps(2, i, 2.0 * mm * mm * fmt_bytes(P.comp_svd), 0.0, s, &st->sweeps[i]);
        TT_CK(launch_jacobi(P.comp_svd, rfmt, Rfin, ldRfin, &st->m[i], S.m_max, wb + P.off_A,
                            wb + P.off_V, P.ldA, sig, Vout, P.ldA, status, &st->sweeps[i], s));
        ++g_launches;
      }
    }
    // rank choice, core
    {
      prof::Scope ps(3, i, mm * S.r_max_out * 8.0, 0.0, s);
      TT_CK(launch_truncate(sig, rows, i, (int)P.n[i - 2], P.r_max, tol2, st, sig_step, nullptr, s));
      TT_CK(launch_core(P.comp_svd, Vout, P.ldA, st, i, cores_out[i - 1], s));
      g_launches += 2;
    }
    // W^(i-1) = W^(i) V_r, fused with the first TSQR level of step i-1 when that is narrow
    void* Y = wb + P.off_W[S.out_buf];
    const bool fuse = next && !next->elide && !next->wide && !next->levels.empty() &&
                      tsmm_tsqr_fusable(next->levels[0], cur_fmt, P.comp_tsmm, P.comp_svd, P.inter,
                                        S.m_max, S.r_max_out);
    first_level_done = false;
    if (fuse) {
      const TsqrLevel& L0 = next->levels[0];
      const double rr = (double)S.r_max_out, mn = (double)next->m_max;
      prof::Scope ps(6, i, (double)rows * (mm * fmt_bytes(cur_fmt) + rr * fmt_bytes(P.inter)),
                     2.0 * (double)rows * mm * rr + 2.0 * (double)L0.rows * mn * mn, s);
      TT_CK(launch_tsmm_tsqr(L0, cur_fmt, P.comp_svd, cur, rows, &st->m[i], S.m_max, Vout, P.ldA,
                             (int)P.n[i - 2], &st->m[i - 1], &st->r[i - 1], S.r_max_out, Y,
                             wb + P.off_R[0], L0.warps * L0.mb, status,
                             (xr && first_active) ? xr : nullptr, s));
      ++g_launches;
      first_level_done = true;
    } else {
      const double rr = (double)S.r_max_out;
      prof::Scope ps(4, i, (double)rows * (mm * fmt_bytes(S.in_fmt) + rr * fmt_bytes(P.inter)),
                     2.0 * (double)rows * mm * rr, s);
      TsmmCfg tc = S.tsmm;
      if (xr && first_active) tc.xr = xr;
      TT_CK(launch_tsmm(tc, cur, rows, rows, &st->m[i], Vout, P.ldA, &st->r[i - 1], Y, rows,
                        status, s));
      ++g_launches;
    }
    first_active = false;
    cur = Y;
    cur_fmt = P.inter;
    rows /= P.n[i - 2];
  }
  // T^(1) = W^(1): n_1 x r_1 (worst case converted; only r_0 n_1 r_1 entries are meaningful)
  const int64_t cnt = P.n[0] * (int64_t)P.r_worst[1];
  // a W that went through the shifted pipeline carries the factor 2^-k; X itself does not
  TT_CK(launch_convert_to_f64(cur_fmt, cur, cnt, cores_out[0], s, cur == X ? nullptr : xr));
  TT_CK(launch_finish(st, d, ranks_out, err2_out, s));
  g_launches += 2;
  return TT_OK;
}

// Alg. 4: the steps in the order d, 1, d-1, 2, ..., then the middle core
static tt_status run_two_sided(const TsPlan& T, const void* X, double* const* cores_out,
                               int64_t* ranks_out, double* err2_out, void* work, cudaStream_t s) {
  char* wb = static_cast<char*>(work);
  DevState* st = reinterpret_cast<DevState*>(wb + T.off_state);
  int* status = &st->status;
  double* e = reinterpret_cast<double*>(wb + T.off_e);
  double* sig = reinterpret_cast<double*>(wb + T.off_sig);
  void* Vout = wb + T.off_Vout;
  TT_CK(launch_init_state(st, T.d, T.n, s));
  TT_CK(launch_zero(e, s));
  g_launches += 2;
  // FP64 input in float-float and FP32 input: the exponent shift of X (engine.h, XRange)
  XRange* xr = (T.comp_tsqr1 == Fmt::DF || T.xfmt == Fmt::F32) ? &st->xr : nullptr;
  if (xr) {
    int64_t nbar = 1;
    for (int a = 0; a < T.d; ++a) nbar *= T.n[a];
    TT_CK(launch_range_sample(T.xfmt, X, nbar, xr, s));
    ++g_launches;
  }
  bool first_active = true;
  auto zptr = [&](int z) -> const void* { return z < 0 ? X : (const void*)(wb + T.off_Z[z]); };
  for (const TsStep& S : T.steps) {
    double* core = cores_out[S.dim - 1];
    if (S.elide) {
      TT_CK(launch_core_identity(S.m, core, s));
      ++g_launches;
      continue;
    }
    const void* Z = zptr(S.zin);
    const void* W = Z;
    if (!S.right) {
      // the tall matrix of a left step: the transpose of the (r_L n_a) x rest unfolding
      TT_CK(launch_transpose(fmt_bytes(S.in), Z, S.m, S.rows, wb + T.off_T, s));
      ++g_launches;
      W = wb + T.off_T;
    }
    const void* lin = W;
    int64_t lld = S.rows;
    const void* Rfin = nullptr;
    int64_t ldRfin = 0;
    Fmt rfmt = Fmt::DF;
    for (size_t l = 0; l < S.levels.size(); ++l) {
      TsqrLevel L = S.levels[l];
      void* Rout = wb + T.off_R[l & 1];
      const int64_t ldR = L.warps * L.mb;
      {
        prof::Scope ps(l == 0 ? 0 : 1, S.dim, (double)L.rows * S.m * fmt_bytes(L.in),
                       2.0 * (double)L.rows * S.m * S.m, s);
        if (xr && first_active && l == 0) L.xr = xr;  // this level reads X (or its transpose)
        TT_CK(launch_tsqr_level(L, lin, lld, nullptr, Rout, ldR, wb + T.off_Rscr, status, s));
        ++g_launches;
      }
      if (L.xr) {
        // keep the shift, or run the level again with the shift of the largest entry it met
        prof::Scope ps(5, S.dim, 0.0, 0.0, s);
        TT_CK(launch_range_decide(xr, s));
        L.xfix = 1;
        TT_CK(launch_tsqr_level(L, lin, lld, nullptr, Rout, ldR, wb + T.off_Rscr, status, s));
        g_launches += 2;
      }
      lin = Rout;
      lld = ldR;
      Rfin = Rout;
      ldRfin = ldR;
      rfmt = L.out;
    }
    {
      prof::Scope ps(2, S.dim, 2.0 * S.m * S.m * fmt_bytes(T.comp_svd), 0.0, s);
      TT_CK(launch_jacobi(T.comp_svd, rfmt, Rfin, ldRfin, nullptr, S.m, wb + T.off_A, wb + T.off_V,
                          T.ldA, sig, Vout, T.ldA, status, nullptr, s));
      ++g_launches;
    }
    TT_CK(launch_core_side(T.comp_svd, !S.right, Vout, T.ldA, S.m, S.r, core, s));
    TT_CK(launch_add_discarded(sig, S.m, S.r, e, s));
    g_launches += 2;
    void* Zout = wb + T.off_Z[S.zout];
    void* Y = S.right ? Zout : (void*)(wb + T.off_Y);
    {
      prof::Scope ps(4, S.dim, (double)S.rows * (S.m * fmt_bytes(S.in) + S.r * fmt_bytes(T.inter)),
                     2.0 * (double)S.rows * S.m * S.r, s);
      TsmmCfg tc = S.tsmm;
      if (xr && first_active) tc.xr = xr;
      TT_CK(launch_tsmm(tc, W, S.rows, S.rows, nullptr, Vout, T.ldA, nullptr, Y, S.rows, status, s));
      ++g_launches;
    }
    first_active = false;
    if (!S.right) {
      // back to the (r, n_{a+1}, ..., r_R) layout of Z
      TT_CK(launch_transpose(fmt_bytes(T.inter), Y, S.rows, S.r, Zout, s));
      ++g_launches;
    }
  }
  const int64_t cnt = (int64_t)T.rl * T.n[T.mid - 1] * T.rr;
  // the middle core carries the factor 2^-k of the shifted pipeline unless it is X itself
  TT_CK(launch_convert_to_f64(T.zfmt_final, zptr(T.zfinal), cnt, cores_out[T.mid - 1], s,
                              T.zfinal < 0 ? nullptr : xr));
  TT_CK(launch_put_ranks(T.ranks, T.d + 1, ranks_out, e, err2_out, s, xr));
  g_launches += 2;
  return TT_OK;
}

// Alg. 3: lines 2-3 (reduced decomposition), line 4 (recovery of the combined cores and
// absorption of the recovered first core), ranks and discarded energy of the joined train
static tt_status run_thick(const ThickPlan& T, const void* X, double* const* cores_out,
                           int64_t* ranks_out, double* err2_out, void* work, cudaStream_t s) {
  char* wb = static_cast<char*>(work);
  const int d = T.d1 + T.k - 1, k = T.k;
  double* tbar = reinterpret_cast<double*>(wb + T.off_tbar);
  double* s0 = reinterpret_cast<double*>(wb + T.off_s0);
  double* told = reinterpret_cast<double*>(wb + T.off_told);
  int64_t* r1 = reinterpret_cast<int64_t*>(wb + T.off_r1);
  int64_t* r2 = reinterpret_cast<int64_t*>(wb + T.off_r2);
  double* e = reinterpret_cast<double*>(wb + T.off_e);
  double* c1[TT_MAX_D];
  for (int i = 0; i < d - k; ++i) c1[i] = cores_out[i];
  c1[d - k] = tbar;
  tt_status st = run_plan(T.P1, X, c1, r1, nullptr, e, wb + T.off_w1, s);
  if (st != TT_OK) return st;
  double* c2[TT_MAX_D];
  c2[0] = s0;
  for (int i = 1; i <= k; ++i) c2[i] = cores_out[d - k + i - 1];
  if ((st = run_plan(T.P2, tbar, c2, r2, nullptr, e + 1, wb + T.off_w2, s)) != TT_OK) return st;
  double* left = cores_out[d - k - 1];
  TT_CK(cudaMemcpyAsync(told, left, (size_t)T.a * T.b * T.r1 * sizeof(double), cudaMemcpyDeviceToDevice, s));
  TT_CK(launch_merge_core(told, s0, T.a * T.b, T.r1, T.rho1, left, s));
  TT_CK(launch_join_ranks(r1, d - k, r2, k, ranks_out, e, err2_out, s));
  g_launches += 2;
  return TT_OK;
}

}  // namespace tt

using namespace tt;

extern "C" {

const char* tt_status_str(tt_status s) {
  switch (s) {
    case TT_OK: return "ok";
    case TT_EINVAL: return "invalid argument";
    case TT_ENOMEM: return "workspace too small or budget exceeded";
    case TT_ECUDA: return "CUDA error";
    case TT_ETIMEOUT: return "timed out";
    case TT_ENOTIMPL: return "not implemented for these arguments";
    case TT_ECANCELLED: return "cancelled";
    case TT_ENUMERIC: return "numerical failure (no convergence or non-finite value)";
  }
  return "unknown status";
}

const char* tt_last_error(void) { return g_last_err; }

tt_status tt_range_rule(int sample_exp, int seen_exp, int* k_try, int* redo, int* k) {
  if (!k_try || !redo || !k) return TT_EINVAL;
  auto enc = [](int e) { return e == TT_RANGE_NONE ? 0 : e + kXrBias; };
  if ((sample_exp != TT_RANGE_NONE && (sample_exp < -1200 || sample_exp > 1100)) ||
      (seen_exp != TT_RANGE_NONE && (seen_exp < -1200 || seen_exp > 1100)))
    return TT_EINVAL;
  *k_try = xr_shift_for(enc(sample_exp));
  *redo = xr_needs_redo(*k_try, enc(seen_exp)) ? 1 : 0;
  *k = *redo ? xr_shift_for(enc(seen_exp)) : *k_try;
  return TT_OK;
}

tt_status tt_tune_set(const char* key, int value) {
  if (!key || !*key) return TT_EINVAL;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (value < 0) g_tune.erase(key);
  else g_tune[key] = value;
  return TT_OK;
}

tt_status tt_profile(int enable) {
  std::lock_guard<std::mutex> lk(prof::mu);
  prof::on = enable != 0;
  prof::recs.clear();
  prof::pool_used = 0;
  return TT_OK;
}

tt_status tt_profile_read(int max, int* n, int* kinds, int* steps, double* ms, double* bytes,
                          double* flops, int* info) {
  if (max < 0 || !n) return TT_EINVAL;
  std::lock_guard<std::mutex> lk(prof::mu);
  *n = (int)prof::recs.size();
  const int k = std::min<int>(max, (int)prof::recs.size());
  for (int j = 0; j < k; ++j) {
    const prof::Rec& r = prof::recs[j];
    if (cudaEventSynchronize(r.b) != cudaSuccess) return TT_ECUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return TT_ECUDA;
    if (kinds) kinds[j] = r.kind;
    if (steps) steps[j] = r.step;
    if (ms) ms[j] = t;
    if (bytes) bytes[j] = r.bytes;
    if (flops) flops[j] = r.flops;
    if (info) {
      int v = -1;
      if (r.info_dev && cudaMemcpy(&v, r.info_dev, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return TT_ECUDA;
      info[j] = v;
    }
  }
  return TT_OK;
}

tt_status tt_stats(int64_t* launches) {
  if (!launches) return TT_EINVAL;
  *launches = g_launches.load();
  return TT_OK;
}

tt_status tt_query(int d, const int64_t* n, int r_max, double tol, tt_dtype dt,
                   size_t* core_bytes, size_t* work_bytes) {
  // the largest workspace over every tt_opts variant (elision on/off, float-float
  // or native FP64 arithmetic), so that any options fit a tt_query-sized buffer
  Plan P;
  tt_status st = build_plan(d, n, r_max, tol, dt, nullptr, P);
  if (st != TT_OK) return st;
  size_t total = P.total;
  for (int ne = 0; ne <= 1; ++ne)
    for (int ar = (int)TT_ARITH_DF; ar <= (int)TT_ARITH_F64; ++ar) {
      tt_opts o{};
      o.arith = (tt_arith)ar;
      o.no_elide = ne;
      Plan Q;
      if (build_plan(d, n, r_max, tol, dt, &o, Q) == TT_OK) total = std::max(total, Q.total);
    }
  if (core_bytes) {
    size_t cb = 0;
    for (int i = 1; i <= d; ++i) cb += (size_t)P.r_worst[i - 1] * n[i - 1] * P.r_worst[i] * 8;
    *core_bytes = cb;
  }
  if (work_bytes) *work_bytes = total;
  return TT_OK;
}

tt_status tt_query_ex(int d, const int64_t* n, int r_max, double tol, tt_dtype dt,
                      const tt_opts* opts, size_t* core_bytes, size_t* work_bytes) {
  tt_status st = tt_query(d, n, r_max, tol, dt, core_bytes, work_bytes);
  if (st != TT_OK || !opts) return st;
  if (opts->two_sided) {
    TsPlan T;
    if ((st = build_two_sided(d, n, r_max, tol, dt, opts, T)) != TT_OK) return st;
    if (work_bytes) *work_bytes = std::max(*work_bytes, T.total);
    return TT_OK;
  }
  if (opts->thick_m_min <= 0) return st;
  ThickPlan T;
  if ((st = build_thick(d, n, r_max, tol, dt, opts, T)) != TT_OK) return st;
  if (T.k >= 2 && work_bytes) *work_bytes = std::max(*work_bytes, T.total);
  return TT_OK;
}

tt_status tt_core_caps(int d, const int64_t* n, int r_max, int64_t* caps, int64_t* sigma_stride,
                       int64_t* sigma_count) {
  tt_status st = validate(d, n, r_max, 0.0);
  if (st != TT_OK) return st;
  int rw[TT_MAX_D + 1];
  worst_ranks(d, n, r_max, rw);
  if (caps)
    for (int i = 1; i <= d; ++i) caps[i - 1] = (int64_t)rw[i - 1] * n[i - 1] * rw[i];
  int64_t a = 0, b = 0;
  sigma_layout(d, n, rw, &a, &b);
  if (sigma_stride) *sigma_stride = a;
  if (sigma_count) *sigma_count = b;
  return TT_OK;
}

tt_status tt_svd_ex(const void* X, tt_dtype dt, int d, const int64_t* n, int r_max, double tol,
                    double* const* cores_out, int64_t* ranks_out, double* sigma_out,
                    double* err2_out, void* work, size_t work_bytes, void* stream,
                    const tt_opts* opts) {
  if (!X || !cores_out || !work) return TT_EINVAL;
  for (int i = 0; i < d && i < TT_MAX_D; ++i)
    if (!cores_out[i]) return TT_EINVAL;
  if (((uintptr_t)work & 255) != 0) return TT_EINVAL;
  if (opts && opts->two_sided) {
    if (sigma_out) return TT_EINVAL;
    TsPlan T;
    tt_status st = build_two_sided(d, n, r_max, tol, dt, opts, T);
    if (st != TT_OK) return st;
    if (work_bytes < T.total) return TT_ENOMEM;
    return run_two_sided(T, X, cores_out, ranks_out, err2_out, work, (cudaStream_t)stream);
  }
  if (opts && opts->thick_m_min > 0) {
    if (opts->thick_m_min < 0 || opts->thick_f1_min < 0 || opts->thick_r_est < 0) return TT_EINVAL;
    ThickPlan T;
    tt_status st = build_thick(d, n, r_max, tol, dt, opts, T);
    if (st != TT_OK) return st;
    if (T.k >= 2) {
      if (sigma_out) return TT_EINVAL;
      if (work_bytes < T.total) return TT_ENOMEM;
      return run_thick(T, X, cores_out, ranks_out, err2_out, work, (cudaStream_t)stream);
    }
  }
  Plan P;
  tt_status st = build_plan(d, n, r_max, tol, dt, opts, P);
  if (st != TT_OK) return st;
  if (work_bytes < P.total) return TT_ENOMEM;
  return run_plan(P, X, cores_out, ranks_out, sigma_out, err2_out, work, (cudaStream_t)stream);
}

}  // extern "C"

namespace tt {
// Rough device time of one tt_svd (seconds) for scheduling batches: float-float TSQR at
// ~2 TFLOP/s, one-sided Jacobi ~10 sweeps of m rounds at ~1.5 us, W*V_r at ~2 TFLOP/s.
double job_cost_estimate(int d, const int64_t* n, int r_max, double tol, int dt) {
  Plan P;
  if (build_plan(d, n, r_max, tol, (tt_dtype)dt, nullptr, P) != TT_OK) return 0.0;
  double t = 0.0;
  for (const StepPlan& S : P.steps) {
    if (S.elide) continue;
    const double m = S.m_max, rows = (double)S.rows;
    t += 2.0 * rows * m * m / 2e12 + 10.0 * m * 1.5e-6 + 2.0 * rows * m * S.r_max_out / 2e12 + 20e-6;
  }
  return t;
}
}  // namespace tt

extern "C" {

tt_status tt_query_from_host(int d, const int64_t* n, int r_max, double tol, tt_dtype dt,
                             int chunks, size_t* work_bytes) {
  if (chunks < 0 || chunks > 4096 || !work_bytes) return TT_EINVAL;
  const int K = chunks ? chunks : kDefaultInChunks;
  Plan P;
  tt_status st = build_plan(d, n, r_max, tol, dt, nullptr, P, K);
  if (st != TT_OK) return st;
  size_t total = P.total;
  for (int ne = 0; ne <= 1; ++ne)
    for (int ar = (int)TT_ARITH_DF; ar <= (int)TT_ARITH_F64; ++ar) {
      tt_opts o{};
      o.arith = (tt_arith)ar;
      o.no_elide = ne;
      Plan Q;
      if (build_plan(d, n, r_max, tol, dt, &o, Q, K) == TT_OK) total = std::max(total, Q.total);
    }
  *work_bytes = total;
  return TT_OK;
}

tt_status tt_svd_from_host(const void* X_host, void* X_dev, tt_dtype dt, int d, const int64_t* n,
                           int r_max, double tol, int chunks, double* const* cores_out,
                           int64_t* ranks_out, double* sigma_out, double* err2_out, void* work,
                           size_t work_bytes, void* stream, const tt_opts* opts) {
  if (!X_host || !X_dev || !cores_out || !work || chunks < 0 || chunks > 4096) return TT_EINVAL;
  for (int i = 0; i < d && i < TT_MAX_D; ++i)
    if (!cores_out[i]) return TT_EINVAL;
  if (((uintptr_t)work & 255) != 0) return TT_EINVAL;
  Plan P;
  tt_status st = build_plan(d, n, r_max, tol, dt, opts, P, chunks ? chunks : kDefaultInChunks);
  if (st != TT_OK) return st;
  if (work_bytes < P.total) return TT_ENOMEM;
  const cudaStream_t s = (cudaStream_t)stream;
  int nev = 0;
  for (const StepPlan& S : P.steps)
    if (!S.elide) {
      nev = S.levels.empty() ? 0 : S.levels[0].chunks;
      break;
    }
  HostIn hin;
  hin.X_host = static_cast<const char*>(X_host);
  // the copy stream forks from `stream` (so it also follows earlier work that reads X_dev)
  // and joins it through the per-block events; stream and events are released when done
  cudaEvent_t fork = nullptr;
  tt_status ret = TT_OK;
  if (cuda_err(cudaStreamCreateWithFlags(&hin.cs, cudaStreamNonBlocking)) != TT_OK) return TT_ECUDA;
  hin.ev.assign(std::max(nev, 0), nullptr);
  bool ok = cuda_err(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming)) == TT_OK;
  for (auto& e : hin.ev)
    ok = ok && cuda_err(cudaEventCreateWithFlags(&e, cudaEventDisableTiming)) == TT_OK;
  ok = ok && cuda_err(cudaEventRecord(fork, s)) == TT_OK;
  ok = ok && cuda_err(cudaStreamWaitEvent(hin.cs, fork, 0)) == TT_OK;
  ret = ok ? run_plan(P, X_dev, cores_out, ranks_out, sigma_out, err2_out, work, s, &hin) : TT_ECUDA;
  for (auto& e : hin.ev)
    if (e) cudaEventDestroy(e);
  if (fork) cudaEventDestroy(fork);
  cudaStreamDestroy(hin.cs);
  return ret;
}

tt_status tt_svd(const void* X, tt_dtype dt, int d, const int64_t* n, int r_max, double tol,
                 double* const* cores_out, int64_t* ranks_out, double* sigma_out,
                 double* err2_out, void* work, size_t work_bytes, void* stream) {
  return tt_svd_ex(X, dt, d, n, r_max, tol, cores_out, ranks_out, sigma_out, err2_out, work,
                   work_bytes, stream, nullptr);
}

tt_status tt_last_device_status(const void* work, void* stream) {
  if (!work) return TT_EINVAL;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return TT_ECUDA;
  int v = 0;
  if (cudaMemcpy(&v, work, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return TT_ECUDA;
  if (v & DEV_ERR_SHAPE) return TT_EINVAL;
  if (v & DEV_ERR_TIMEOUT) return TT_ETIMEOUT;
  if (v & (DEV_SVD_NOCONV | DEV_NONFINITE)) return TT_ENUMERIC;
  return TT_OK;
}

// ---- building blocks ------------------------------------------------------------------
static Fmt tsqr_comp2(tt_dtype) { return Fmt::DF; }

// the TSQR levels of tt_tsqr / tt_tsqr_ex: FP64 input in float-float, or all levels in
// native FP64 (native = true)
static std::vector<TsqrLevel> tsqr_api_plan(int64_t rows, int m, tt_dtype dt, bool native) {
  const Fmt in = dt == TT_F32 ? Fmt::F32 : Fmt::F64;
  const Fmt c1 = dt == TT_F32 ? Fmt::F32 : (native ? Fmt::F64 : Fmt::DF);
  return plan_tsqr(rows, m, in, c1, native ? Fmt::F64 : tsqr_comp2(dt), num_sms(), 0);
}

tt_status tt_tsqr_query(int64_t rows, int m, tt_dtype dt, size_t* work_bytes) {
  if (rows < 1 || m < 1 || m > kMaxM || (dt != TT_F64 && dt != TT_F32) || !work_bytes)
    return TT_EINVAL;
  size_t szR = 0, scr = 0;
  // FP64 input: room for either arithmetic (tt_tsqr_ex)
  for (int native = 0; native <= (dt == TT_F64 ? 1 : 0); ++native) {
    auto lv = tsqr_api_plan(rows, m, dt, native != 0);
    if (lv.empty()) return TT_ENOTIMPL;
    for (auto& L : lv) {
      szR = std::max(szR, (size_t)L.warps * L.mb * m * fmt_bytes(L.out));
      scr = std::max(scr, tsqr_wide_scratch_bytes(L));
    }
  }
  *work_bytes = align256(256) + 2 * align256(szR) + align256(scr);
  return TT_OK;
}

tt_status tt_tsqr_ex(const void* W, tt_dtype dt, int64_t rows, int m, int64_t ld, double* R_out,
                     void* work, size_t work_bytes, tt_arith arith, void* stream) {
  size_t need = 0;
  tt_status st = tt_tsqr_query(rows, m, dt, &need);
  if (st != TT_OK) return st;
  if (!W || !R_out || !work || ld < rows || ((uintptr_t)work & 255) ||
      (arith != TT_ARITH_AUTO && arith != TT_ARITH_DF && arith != TT_ARITH_F64))
    return TT_EINVAL;
  if (work_bytes < need) return TT_ENOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  const Fmt in = dt == TT_F32 ? Fmt::F32 : Fmt::F64;
  const bool native = dt == TT_F64 && arith == TT_ARITH_F64;
  auto lv = tsqr_api_plan(rows, m, dt, native);
  size_t szR = 0;
  for (auto& L : lv) szR = std::max(szR, (size_t)L.warps * L.mb * m * fmt_bytes(L.out));
  char* wb = static_cast<char*>(work);
  // the first 256 bytes: the status word, then the exponent range of W (FP64 input)
  int* status = reinterpret_cast<int*>(wb);
  XRange* xr = reinterpret_cast<XRange*>(wb + 16);
  TT_CK(cudaMemsetAsync(wb, 0, 256, s));
  // (a strided W: the first pass starts unshifted and is redone if that was wrong; native
  // FP64 needs no exponent shift)
  if (ld == rows && !native) TT_CK(launch_range_sample(in, W, rows * (int64_t)m, xr, s));
  char* R0 = wb + align256(256);
  char* R1 = R0 + align256(szR);
  char* scr = R1 + align256(szR);
  const void* lin = W;
  int64_t lld = ld;
  void* Rfin = nullptr;
  int64_t ldRfin = 0;
  Fmt rf = Fmt::DF;
  for (size_t l = 0; l < lv.size(); ++l) {
    void* Rout = (l & 1) ? R1 : R0;
    const int64_t ldR = lv[l].warps * lv[l].mb;
    TsqrLevel L = lv[l];
    if (l == 0 && !native) L.xr = xr;
    TT_CK(launch_tsqr_level(L, lin, lld, nullptr, Rout, ldR, scr, status, s));
    ++g_launches;
    if (L.xr) {
      TT_CK(launch_range_decide(xr, s));
      L.xfix = 1;
      TT_CK(launch_tsqr_level(L, lin, lld, nullptr, Rout, ldR, scr, status, s));
      g_launches += 2;
    }
    lin = Rout;
    lld = ldR;
    Rfin = Rout;
    ldRfin = ldR;
    rf = lv[l].out;
  }
  // R of W = 2^k times the R of the shifted W (k = 0 for native FP64: xr is zeroed)
  g_launches += native ? 1 : 2;  // the sample and the copy
  return cuda_err(launch_copy_mat_f64(rf, Rfin, ldRfin, m, m, 1, R_out, m, s, xr));
}

tt_status tt_tsqr(const void* W, tt_dtype dt, int64_t rows, int m, int64_t ld, double* R_out,
                  void* work, size_t work_bytes, void* stream) {
  return tt_tsqr_ex(W, dt, rows, m, ld, R_out, work, work_bytes, TT_ARITH_DF, stream);
}

tt_status tt_small_svd_query(int m, size_t* work_bytes) {
  if (m < 1 || m > kMaxM || !work_bytes) return TT_EINVAL;
  const int mp = m + (m & 1);
  *work_bytes = align256(256) + align256(jacobi_scratch_bytes(Fmt::DF, m)) +
                align256((size_t)mp * mp * fmt_bytes(Fmt::DF));
  return TT_OK;
}

tt_status tt_small_svd(const double* R, int m, double* sigma, double* V, void* work,
                       size_t work_bytes, void* stream) {
  size_t need = 0;
  tt_status st = tt_small_svd_query(m, &need);
  if (st != TT_OK) return st;
  if (!R || !sigma || !V || !work || ((uintptr_t)work & 255)) return TT_EINVAL;
  if (work_bytes < need) return TT_ENOMEM;
  cudaStream_t s = (cudaStream_t)stream;
  const int mp = m + (m & 1);
  char* wb = static_cast<char*>(work);
  int* status = reinterpret_cast<int*>(wb);
  TT_CK(cudaMemsetAsync(status, 0, sizeof(int), s));
  char* A = wb + align256(256);
  const size_t szJ = jacobi_scratch_bytes(Fmt::DF, m);
  char* Vw = A + szJ / 2;
  char* Vout = A + align256(szJ);
  TT_CK(launch_jacobi(Fmt::DF, Fmt::F64, R, m, nullptr, m, A, Vw, mp, sigma, Vout, mp, status,
                      nullptr, s));
  g_launches += 2;
  return cuda_err(launch_copy_mat_f64(Fmt::DF, Vout, mp, m, m, 0, V, m, s));
}

tt_status tt_tsmm_ex(const void* W, tt_dtype dt, int64_t rows, int m, int64_t ld, const double* V,
                     int k, double* Y, int64_t ldy, tt_arith arith, void* stream) {
  if (arith != TT_ARITH_F64 || dt != TT_F64)
    return tt_tsmm(W, dt, rows, m, ld, V, k, Y, ldy, stream);
  if (!W || !V || !Y || rows < 1 || m < 1 || m > kMaxM || k < 1 || k > m || ld < rows || ldy < rows)
    return TT_EINVAL;
  // the native FP64 form's product (FP64-accurate tensor-core splitting where m >= 16)
  TsmmCfg c = plan_tsmm(Fmt::F64, Fmt::F64, Fmt::F64, Fmt::F64, m, k, rows, num_sms());
  ++g_launches;
  return cuda_err(launch_tsmm(c, W, rows, ld, nullptr, V, m, nullptr, Y, ldy, nullptr,
                              (cudaStream_t)stream));
}

tt_status tt_tsmm(const void* W, tt_dtype dt, int64_t rows, int m, int64_t ld, const double* V,
                  int k, double* Y, int64_t ldy, void* stream) {
  if (!W || !V || !Y || rows < 1 || m < 1 || m > kMaxM || k < 1 || k > m || ld < rows ||
      ldy < rows || (dt != TT_F64 && dt != TT_F32))
    return TT_EINVAL;
  const Fmt in = dt == TT_F32 ? Fmt::F32 : Fmt::F64;
  const Fmt comp = dt == TT_F32 ? Fmt::F32 : Fmt::DF;
  TsmmCfg c = plan_tsmm(in, comp, Fmt::F64, Fmt::F64, m, k, rows, num_sms());
  ++g_launches;
  return cuda_err(launch_tsmm(c, W, rows, ld, nullptr, V, m, nullptr, Y, ldy, nullptr,
                              (cudaStream_t)stream));
}

tt_status tt_gen_uniform(void* out, tt_dtype dt, int64_t count, uint64_t seed, int64_t start,
                         void* stream) {
  if (!out || count < 0 || start < 0 || (dt != TT_F64 && dt != TT_F32)) return TT_EINVAL;
  return cuda_err(launch_gen_uniform(out, dt == TT_F32 ? Fmt::F32 : Fmt::F64, count, seed, start,
                                     (cudaStream_t)stream));
}

}  // extern "C"
