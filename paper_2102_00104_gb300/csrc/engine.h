// engine.h -- internal interface between the host driver and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

namespace tt {

// element formats in device memory
enum class Fmt : int { F64 = 0, DF = 1, F32 = 2 };
inline size_t fmt_bytes(Fmt f) { return f == Fmt::F32 ? 4 : 8; }

// device status word values (bit flags)
enum : int {
  DEV_OK = 0,
  DEV_ERR_SHAPE = 1,      // a kernel saw a shape outside what it was launched for
  DEV_SVD_NOCONV = 2,     // Jacobi SVD hit its sweep limit
  DEV_NONFINITE = 4,      // a non-finite singular value appeared
  DEV_ERR_TIMEOUT = 8,    // a bounded in-kernel wait gave up (the kernel returned early)
};

// wait limit of in-kernel spin-waits, in SM clock cycles (~2 s at 2 GHz)
constexpr long long kWaitCycles = 4000000000LL;

// Exponent range of an FP64 input read in float-float.  Float-float has FP32's
// exponent range, so X is read as X * 2^-k with an exact power of two k chosen from its
// largest magnitude; sigma, the discarded energy and the last core are scaled back.
// A strided sample of X gives k_try; the first TSQR level reads with k_try and records
// the largest exponent it meets; when that lies far above the sample, the level is run
// again with the shift of the true largest magnitude (redo = 1).  Every later reader of
// X uses k.  Exponents are stored encoded so that all-zero bytes mean "none seen":
// enc = e + kXrBias for a finite nonzero value 2^e <= |x| < 2^(e+1), kXrNonfinite for
// infinity and NaN.
struct XRange {
  int sample;  // largest encoded exponent of the strided sample
  int seen;    // largest encoded exponent met by the first pass of the first TSQR level
  int redo;    // 1: the first level runs again with k
  int k;       // the shift of every other reader of X, and of the results
};
constexpr int kXrBias = 2048;
constexpr int kXrNonfinite = 8192;
constexpr int kXrWindow = 40;      // entries up to 2^40 after the shift keep every sum of
                                   // squares inside FP32's range for up to 2^46 rows
// shift that brings the largest magnitude (encoded exponent) into [0.5, 1); 0 when
// nothing nonzero and finite was seen
__host__ __device__ inline int xr_shift_for(int enc) {
  return (enc <= 0 || enc >= kXrNonfinite) ? 0 : enc - kXrBias + 1;
}
// the first pass read with k_try; true when its largest entry left the safe window
// (above it: sums of squares could overflow; below it: they could underflow -- the
// latter only when no sample was taken)
__host__ __device__ inline bool xr_needs_redo(int k_try, int seen) {
  if (seen <= 0 || seen >= kXrNonfinite) return false;
  const int top = seen - kXrBias - k_try;
  return top > kXrWindow || top < -kXrWindow;
}

// per-call device state (lives in the workspace)
struct DevState {
  int status;
  int pad_;
  XRange xr;
  int first_done;              // 1 once delta has been fixed (Alg. 2 line 7)
  double delta2;
  double err2;
  int m[40];                   // m[i] = columns of W^(i) (1-based step index)
  int r[40];                   // r[0..d]
  int sweeps[40];              // Jacobi sweeps used at step i (diagnostics)
};

constexpr int kMaxM = 512;     // widest unfolding handled

// rough device time (s) of one tt_svd with these arguments, for batch scheduling
double job_cost_estimate(int d, const int64_t* n, int r_max, double tol, int dt);

// ---- TSQR ---------------------------------------------------------------------
// One TSQR level: every warp runs a flat tree of Alg. 6 panels over its share of
// the rows of W (rows x m, leading dimension ld, format in) and writes its R
// (m x m, zero below the diagonal) as a block of `mb` rows of the stacked
// column-major output (ldR = warps * mb rows).
struct TsqrLevel {
  int kind;          // 0 = narrow (warp, register panels), 1 = wide (warp, smem panels),
                     // 2 = CTA-cooperative (register panels, R in shared memory),
                     // 3 = column-owned CTA kernel (one barrier per column, look-ahead),
                     // 4 = column-owned with the panel in shared memory (wide m),
                     // 5 = pairwise merge of the stacked triangles (upper levels only),
                     // 6 = blocked native-FP64 kernel (tensor-core trailing updates)
  int cfg;           // kind 2: layout id (see tsqr_cta.cu); kind 3: see tsqr_col.cu
  int maxm;          // narrow: 4/8/16 ; wide: 32*chunks (template bound)
  int mmax;          // worst-case m of this level (<= maxm)
  int mval;          // m passed by value when the device pointer is null
  int mb;            // rows of one R block in the stacked output
  int pr;            // panel rows per warp
  int nw;            // warps per CTA
  int64_t ctas;
  int64_t warps;     // total warps = partial R count
  int64_t rows;      // rows of this level's input
  int64_t panels;
  size_t smem;       // dynamic smem per CTA
  Fmt in, comp, out;
  XRange* xr = nullptr;       // first level of FP64 input in float-float: exponent shift
  int xfix = 0;               // 1: the re-run of that level (returns at once unless xr->redo)
  int chunks = 1;            // first level only: launched once per row block of chunk_rows
  int64_t chunk_rows = 0;    // rows with the full grid; each block writes chunk_parts partial
  int64_t chunk_parts = 0;   // R's, so warps = chunks * chunk_parts
};

cudaError_t launch_tsqr_level(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev,
                              void* Rout, int64_t ldR, void* Rscr, int* status, cudaStream_t s);
size_t tsqr_wide_scratch_bytes(const TsqrLevel& L);
// kind 2: layout id for m_max (or -1 if R does not fit in shared memory), rows per panel, warps
int tsqr_cta_pick(int m_max, Fmt comp, int* pr, int* nw, int* per_sm);
size_t tsqr_cta_smem(int m_max, Fmt comp, int id);
// global-memory R scratch needed by layout `id` for `ctas` CTAs (0 if R sits in shared memory)
size_t tsqr_cta_scratch(int m_max, Fmt comp, int id, int64_t ctas);
// kind 3: layout id for m_max and the level's formats (or -1), rows per panel, warps, CTAs per SM
int tsqr_col_pick(int m_max, Fmt in, Fmt comp, Fmt out, int* pr, int* nw, int* per_sm);
size_t tsqr_col_smem(int m_max, Fmt comp, int id);
cudaError_t launch_tsqr_col(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev,
                            void* Rout, int64_t ldR, int* status, cudaStream_t s);
// kind 6: the blocked native-FP64 kernel (compact-WY blocks of 8 reflectors, trailing
// updates on the tensor cores), 16 < m <= 512: rows per panel, CTAs per SM, shared memory
// and (m > 80: R in a global slice per CTA) scratch bytes per layout
size_t tsqr_blk_smem(int m_max);
int tsqr_blk_rows(int m_max);
int tsqr_blk_per_sm(int m_max);
size_t tsqr_blk_scratch(int m_max, int64_t ctas);
cudaError_t launch_tsqr_blk(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev,
                            void* Rout, int64_t ldR, void* Rscr, int* status, cudaStream_t s);
// kind 4 (shared-memory panels, R in an L2-resident global slice per CTA): rows per lane or -1
int tsqr_cols_pick(int m_max, Fmt in, Fmt comp, Fmt out, int* pr, int* nw, int* per_sm);
size_t tsqr_cols_smem(int m_max, int prl);
size_t tsqr_cols_scratch(int m_max, int64_t ctas);
cudaError_t launch_tsqr_cols(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev,
                             void* Rout, int64_t ldR, void* Rscr, int* status, cudaStream_t s);
// kind 5 (tsqr_merge.cu): one CTA merges two stacked R blocks with a structured Alg. 6 sweep
bool tsqr_merge_ok(int m_max, Fmt in, Fmt comp);
size_t tsqr_merge_scratch(int m_max, Fmt comp, int64_t ctas);
cudaError_t launch_tsqr_merge(const TsqrLevel& L, const void* Rin, int64_t ldi, const int* m_dev,
                              void* Rout, int64_t ldo, void* scr, int* status, cudaStream_t s);
cudaError_t launch_tsqr_cta(const TsqrLevel& L, const void* W, int64_t ld, const int* m_dev,
                            void* Rout, int64_t ldR, void* Rscr, int* status, cudaStream_t s);

// ---- small SVD ------------------------------------------------------------------
// One-sided Jacobi of the m x m matrix R (format rin, leading dimension ldR);
// writes sigma (descending, FP64) and V (format comp, column-major, ldV).
// m_dev may be null: then m = m_max.
cudaError_t launch_jacobi(Fmt comp, Fmt rin, const void* R, int64_t ldR, const int* m_dev,
                          int m_max, void* Ag, void* Vg, int ldA, double* sigma, void* Vout,
                          int ldV, int* status, int* sweeps_out, cudaStream_t s);
size_t jacobi_scratch_bytes(Fmt comp, int m_max);
// wide unfolding W (rows x m, rows < m, format win, leading dimension ldW): sigma and the
// right singular vectors from one-sided Jacobi on W^T, no TSQR (one CTA, W^T in shared memory)
bool jacobi_wide_fits(Fmt comp, int rows, int m_max);
cudaError_t launch_jacobi_wide(Fmt comp, Fmt win, const void* W, int64_t ldW, int rows,
                               const int* m_dev, int m_max, double* sigma, void* Vout, int ldV,
                               int* status, int* sweeps_out, void* gscr, cudaStream_t s);
// global scratch for the wide Jacobi's working copy when it does not fit shared memory (else 0)
size_t jacobi_wide_gbytes(Fmt comp, int rows, int m_max);
// cluster form (svd_cluster.cu): cluster size for m (0 = single CTA) and its launch
int jacobi_cluster_plan(Fmt comp, int m_max, int* npl_out);
// block-cyclic cluster kernel: cluster size (0 if it does not apply) and columns per block
int jacobi_block_plan(Fmt comp, int m_max, int* npl_out);
cudaError_t launch_jacobi_block(Fmt comp, Fmt rin, const void* R, int64_t ldR, const int* m_dev,
                                int m_max, int nc, int npl, double* sigma, void* Vout, int ldV,
                                int* status, int* sweeps_out, cudaStream_t s);
int jacobi_cluster_npl(Fmt comp, int m_max, int nc);
// Vg / ldVg: global scratch (ldVg >= m_max, m_max columns) for V when A and V do not both fit
// in the cluster's shared memory
cudaError_t launch_jacobi_cluster(Fmt comp, Fmt rin, const void* R, int64_t ldR, const int* m_dev,
                                  int m_max, int nc, int npl, double* sigma, void* Vout, int ldV,
                                  int* status, int* sweeps_out, void* Vg, int ldVg, cudaStream_t s);
bool jacobi_cluster_vg(Fmt comp, int m_max, int npl);

// ---- rank choice / cores --------------------------------------------------------
cudaError_t launch_truncate(const double* sigma, int64_t rows, int step_i, int n_next,
                            int r_max, double tol2_over_dm1, DevState* st,
                            double* sigma_out_step, int64_t* ranks_out, cudaStream_t s);
cudaError_t launch_core(Fmt vfmt, const void* V, int ldV, const DevState* st, int step_i,
                        double* core, cudaStream_t s);
cudaError_t launch_core_identity(int m, double* core, cudaStream_t s);
cudaError_t launch_set_rank(DevState* st, int step_i, int n_next, int r, cudaStream_t s);
// dst(i, k) = src(i, k) as FP64 for i < rows, k < cols (zero below the diagonal if upper)
cudaError_t launch_copy_mat_f64(Fmt f, const void* src, int64_t lds, int rows, int cols, int upper,
                                double* dst, int64_t ldd, cudaStream_t s,
                                const XRange* xr = nullptr);
cudaError_t launch_merge_core(const double* Told, const double* S0, int ab, int r, int rho,
                              double* Tnew, cudaStream_t s);
cudaError_t launch_join_ranks(const int64_t* r1, int p, const int64_t* r2, int q, int64_t* out,
                              const double* e12, double* err2_out, cudaStream_t s);
// two-sided TT-SVD (two_sided.cu)
constexpr int TT_MAX_RANKS = 40;
cudaError_t launch_transpose(size_t elem, const void* in, int64_t P, int64_t Q, void* out,
                             cudaStream_t s);
cudaError_t launch_core_side(Fmt vfmt, bool left, const void* V, int ldV, int m, int r, double* core,
                             cudaStream_t s);
cudaError_t launch_add_discarded(const double* sigma, int cnt, int r, double* e, cudaStream_t s);
cudaError_t launch_zero(double* e, cudaStream_t s);
// err2_out = e[0] * 2^(2 xr->k) (xr may be null)
cudaError_t launch_put_ranks(const int64_t* ranks, int count, int64_t* ranks_out, const double* e,
                             double* err2_out, cudaStream_t s, const XRange* xr = nullptr);
// dst = src * 2^xr->k (xr may be null: no scaling)
cudaError_t launch_convert_to_f64(Fmt f, const void* src, int64_t count, double* dst,
                                  cudaStream_t s, const XRange* xr = nullptr);
// the exponent range of X from a strided sample (sets k_try = k, seen, redo), and the
// decision after the first pass of the first TSQR level
cudaError_t launch_range_sample(Fmt f, const void* X, int64_t count, XRange* xr, cudaStream_t s);
cudaError_t launch_range_decide(XRange* xr, cudaStream_t s);
// xr->sample = enc (a sample taken on the host, for input that is still in host memory)
cudaError_t launch_range_set_sample(XRange* xr, int enc, cudaStream_t s);
cudaError_t launch_fill_nan(double* dst, int64_t count, cudaStream_t s);
cudaError_t launch_init_state(DevState* st, int d, const int64_t* n_host, cudaStream_t s);
cudaError_t launch_finish(const DevState* st, int d, int64_t* ranks_out, double* err2_out,
                          cudaStream_t s);

// ---- TSMM ----------------------------------------------------------------------
// Y (rows x r, ldy, format out) = W (rows x m, ld, format in) * V(:, 0:r)
// (V format vfmt, ldV); m = m_dev[0], r = r_dev[0]; comp = arithmetic.
struct TsmmCfg {
  int kind;         // 0 = shared-memory tile of W, 1 = register-blocked (V in shared memory),
                    // 2 = tensor cores, Ozaki splitting (float-float form), mma.sync,
                    // 3 = the same on tcgen05, 4 = the warp-specialised tcgen05 pipeline
                    // for an FP64 W (tsmm_ws.cu; kind 2 where W cannot be mapped)
  int cpt;          // kind 1: output columns per thread and pass
  Fmt in, comp, vfmt, out;
  int m_max, r_max;
  int tr;           // rows per tile
  int rc;           // kind 0: columns of V held in shared memory at a time; kind 2: tile buffers
  int mstr;         // smem row stride (elements)
  size_t smem;
  int64_t ctas;
  const XRange* xr = nullptr;  // FP64 input in float-float: W is read as W * 2^-xr->k
  // kind 4: the kind-2 launch used where the tensor map of W cannot be made
  int fb_rc = 1;
  size_t fb_smem = 0;
  int64_t fb_ctas = 1;
};
TsmmCfg plan_tsmm(Fmt in, Fmt comp, Fmt vfmt, Fmt out, int m_max, int r_max, int64_t rows,
                  int num_sms);
// the tensor-core form (tsmm_oz.cu): usable for these formats and sizes?
bool tsmm_oz_ok(Fmt in, Fmt comp, Fmt vfmt, Fmt out, int m_max, int r_max);
size_t tsmm_oz_smem(int m_max, int r_max, int nbuf, bool x64 = false);
cudaError_t launch_tsmm_oz(const TsmmCfg& c, const void* W, int64_t rows, int64_t ld,
                           const int* m_dev, const void* V, int ldV, const int* r_dev, void* Y,
                           int64_t ldy, int* status, cudaStream_t s);
// the same splitting on tcgen05 (tsmm_tc.cu)
bool tsmm_tc_ok(Fmt in, Fmt comp, Fmt vfmt, Fmt out, int m_max, int r_max);
size_t tsmm_tc_smem(int m_max, int r_max);
cudaError_t launch_tsmm_tc(const TsmmCfg& c, const void* W, int64_t rows, int64_t ld,
                           const int* m_dev, const void* V, int ldV, const int* r_dev, void* Y,
                           int64_t ldy, int* status, cudaStream_t s);
// an FP64 W on a warp-specialised tcgen05 pipeline with TMA tile loads (tsmm_ws.cu)
bool tsmm_ws_ok(Fmt in, Fmt comp, Fmt vfmt, Fmt out, int m_max, int r_max);
size_t tsmm_ws_smem(int m_max);
cudaError_t launch_tsmm_ws(const TsmmCfg& c, const void* W, int64_t rows, int64_t ld,
                           const int* m_dev, const void* V, int ldV, const int* r_dev, void* Y,
                           int64_t ldy, int* status, cudaStream_t s, bool* used);
cudaError_t launch_tsmm(const TsmmCfg& c, const void* W, int64_t rows, int64_t ld,
                        const int* m_dev, const void* V, int ldV, const int* r_dev, void* Y,
                        int64_t ldy, int* status, cudaStream_t s);

// ---- W V_r fused with the next step's first (narrow) TSQR level (tsqr_fused.cu) ----------
constexpr int kFusedMaxMi = 8;     // widest W^(i) (its m) of the fused product
// can step i's product feed the first level `next` of step i-1 directly?  (formats: in =
// W^(i), comp = arithmetic, vfmt = V, inter = W^(i-1))
bool tsmm_tsqr_fusable(const TsqrLevel& next, Fmt in, Fmt comp, Fmt vfmt, Fmt inter, int mi_max,
                       int r_max);
// Y = W^(i) V_r (rows_i = next.rows * n rows, leading dimension ldw, also of Y) and the partial
// R's of the next step's first level (as launch_tsqr_level would write them); mi = m_i,
// m = m_{i-1} = n r and r = r_{i-1} are device values.
cudaError_t launch_tsmm_tsqr(const TsqrLevel& next, Fmt in, Fmt vfmt, const void* W, int64_t ldw,
                             const int* mi_dev, int mi_max, const void* V, int ldV, int n,
                             const int* m_dev, const int* r_dev, int r_max, void* Y, void* Rout,
                             int64_t ldR, int* status, const XRange* xr, cudaStream_t s);

// ---- generator -------------------------------------------------------------------
cudaError_t launch_gen_uniform(void* out, Fmt f, int64_t count, uint64_t seed, int64_t start,
                               cudaStream_t s);

// tuning parameter set through tt_tune_set (dflt if unset)
int tune_get(const char* key, int dflt);

// sets the text returned by tt_last_error on the calling thread
void set_last_error_text(const char* text);

// device properties (cached)
int num_sms();
size_t max_smem_optin();

}  // namespace tt
