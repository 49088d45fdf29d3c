/*
 * tt_svd.h -- C ABI of a single-GPU (GB300, sm_103a) TT-SVD engine.
 *
 * The engine computes the truncated tensor-train SVD of a dense tensor core by
 * core, right to left, as in Alg. 2 (optimized TSQR TT-SVD, Sec. 3.1.2 of
 * Roehrig-Zoellner, Thies, Basermann, "Performance of the low-rank tensor-train
 * SVD (TT-SVD) for large dense tensors on modern multi-core CPUs"):
 *   per step i = d..2:  R of a Q-less tall-skinny QR of the unfolding W^(i)
 *   (blockwise Householder, Alg. 6, plus a reduction tree over the partial R
 *   factors, Sec. 3.2); the small SVD of R (Eq. QR_trick); the rank choice of
 *   Alg. 2 line 8; the core T^(i) from V (line 9); and the product W^(i) V_r
 *   written as the next unfolding (line 11).
 *
 * Conventions shared by all calls
 * -------------------------------
 * - Tensors are dense and Fortran ordered (n_1 fastest, Sec. 3.1.2 "Memory
 *   layout"), i.e. a C-ordered array of shape (n_d, ..., n_1).  No padding.
 * - All data pointers are DEVICE pointers unless a parameter says "host".
 *   The caller owns every buffer; the library never allocates device memory
 *   in these calls (the serve entry points allocate inside their budget).
 * - Calls are asynchronous on `stream` (a cudaStream_t passed as void*; NULL =
 *   legacy default stream).  Results are valid after the stream synchronises.
 * - Argument errors are detected on the host before anything is launched and
 *   return TT_EINVAL (nothing is written).  CUDA launch errors return
 *   TT_ECUDA.  Device-side failures set a status word in the workspace that
 *   tt_last_device_status() reads back.  No kernel traps or asserts.
 * - Cores are written in FP64 for both storage precisions: core i (1-based)
 *   has shape (r_{i-1}, n_i, r_i) in Fortran order, r_0 = r_d = 1.
 * - Maximum order d is TT_MAX_D.
 */
#ifndef TT_SVD_H
#define TT_SVD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TT_MAX_D 32

typedef enum {
  TT_OK = 0,
  TT_EINVAL = 1,     /* bad argument (checked on the host, nothing launched) */
  TT_ENOMEM = 2,     /* workspace too small / budget exceeded */
  TT_ECUDA = 3,      /* a CUDA call failed */
  TT_ETIMEOUT = 4,   /* a bounded device-side or host-side wait ran out */
  TT_ENOTIMPL = 5,   /* combination not supported */
  TT_ECANCELLED = 6, /* request cancelled (server shut down) */
  TT_ENUMERIC = 7,   /* device-side numerical failure: the Jacobi SVD hit its sweep
                        limit or a singular value was not finite */
  TT_EAGAIN = 8      /* tt_serve_poll: the request has not finished yet */
} tt_status;

/* Storage precision of the input tensor X.  TT_F64: FP64 tensor.  TT_F32: the
 * FP32 form (FP32 storage, FP32 Householder panels and FP32 W*V_r; the R
 * reduction tree, the small SVD and the rank choice run in FP64-class
 * arithmetic).  */
typedef enum { TT_F64 = 0, TT_F32 = 1 } tt_dtype;

/* Internal arithmetic of the FP64 form.  TT_ARITH_DF: float-float (two FP32
 * words, about 48 significant bits) for all bulk work -- GB300 runs FP32 FMAs
 * about 70x faster than FP64 FMAs.  TT_ARITH_F64: native FP64 everywhere.
 * TT_ARITH_AUTO = TT_ARITH_DF.  Ignored for TT_F32 inputs. */
typedef enum { TT_ARITH_AUTO = 0, TT_ARITH_DF = 1, TT_ARITH_F64 = 2 } tt_arith;

typedef struct {
  tt_arith arith;      /* see tt_arith */
  int no_elide;        /* 1: run every step even when V would be square (see tt_svd) */
  int tsqr_ctas;       /* 0 = auto; else number of CTAs of the first TSQR level */
  /* Thick-bounds variant (Alg. 3, Sec. 3.1.3), off when thick_m_min = 0: the k
   * right-most dimensions are combined, with k the smallest count such that
   * m = n_{d-k+1}...n_d >= max(thick_m_min, r_est / thick_f1_min) (r_est =
   * thick_r_est, or r_max when 0); the reshaped tensor is decomposed by Alg. 2
   * and the cores of the combined dimensions are recovered by Alg. 2 applied to
   * the last core T_bar reshaped to (r, n_{d-k+1}, ..., n_d), whose first core
   * is absorbed into the core to its left.  Only tol = 0 (TT_ENOTIMPL
   * otherwise); sigma_out must be NULL; err2_out receives the reduced
   * decomposition's discarded sigma^2 plus the recovery's (the latter relative
   * to the orthonormal T_bar).  k <= 1 or k = d is the plain algorithm. */
  int thick_m_min;
  double thick_f1_min; /* > 0; 0.5 when 0 */
  int thick_r_est;
  /* 1: two-sided variant (Alg. 4, Sec. 3.1.3): cores alternately at the right and
   * at the left end (i = d, 1, d-1, 2, ...), each by the TSQR + small SVD + W*V_r
   * step; a left step works on the transposed left unfolding (an explicit
   * transpose before and after it).  Core T^(i) of a left step has orthonormal
   * columns in its (r_{i-1} n_i) x r_i matricization; the middle core carries the
   * norm.  Only tol = 0 (TT_ENOTIMPL otherwise); sigma_out must be NULL; not
   * combined with thick_m_min. */
  int two_sided;
} tt_opts;

/* ---- sizing ---------------------------------------------------------------
 * tt_query: bytes needed for all d cores together (worst case, each core
 * r_{i-1} n_i r_i doubles with r_k = min(r_max, n_1..n_k, n_{k+1}..n_d)) and
 * for the workspace of tt_svd with these arguments.  `n` is a host array of d
 * positive extents.  Returns TT_EINVAL for d < 1, d > TT_MAX_D, n_i < 1,
 * r_max < 1 or tol < 0. */
tt_status tt_query(int d, const int64_t* n, int r_max, double tol, tt_dtype dt,
                   size_t* core_bytes, size_t* work_bytes);

/* tt_query for the given options (opts may be NULL): the thick-bounds variant
 * needs the workspaces of both of its decompositions. */
tt_status tt_query_ex(int d, const int64_t* n, int r_max, double tol, tt_dtype dt,
                      const tt_opts* opts, size_t* core_bytes, size_t* work_bytes);

/* Worst-case element count of each core (host array caps[d]) and of the
 * sigma_out buffer (*sigma_count): sigma_out holds, for step i = d..2 in that
 * order, min(rows_i, n_i r_i) singular values at offset
 * (d - i) * (*sigma_stride). */
tt_status tt_core_caps(int d, const int64_t* n, int r_max, int64_t* caps,
                       int64_t* sigma_stride, int64_t* sigma_count);

/* ---- the hot path -----------------------------------------------------------
 * tt_svd: truncated TT-SVD of X (Alg. 2).
 *   X          device, n_1*...*n_d elements of type dt, Fortran order, read only
 *   r_max      maximal TT rank (>= 1)
 *   tol        epsilon of Alg. 2: delta = tol / sqrt(d-1) * ||Sigma_first||_F
 *              (line 7); tol = 0 disables tolerance truncation
 *   cores_out  HOST array of d DEVICE pointers; core i receives
 *              r_{i-1} * n_i * r_i doubles (caller-allocated, >= caps[i-1])
 *   ranks_out  device int64[d+1]: r_0..r_d
 *   sigma_out  optional (NULL) device doubles, layout of tt_core_caps; entries of
 *              an elided step are set to NaN
 *   err2_out   optional (NULL) device double: sum over all steps of the
 *              discarded sigma^2 (the a-posteriori error bound squared)
 *   work       device workspace of at least tt_query's work_bytes, 256-byte aligned
 * Step elision: when tol == 0 and min(r_max, rows_i) >= n_i r_i, V would be a
 * square orthogonal matrix; the step is skipped (core = identity, W^(i-1) is a
 * view of W^(i)).  Ranks, later singular values and the approximation are
 * unchanged; only the gauge of that core differs.  opts->no_elide disables it.
 * Range: any finite X.  In the float-float and FP32 arithmetics (FP32's exponent range) X
 * is read as X 2^-k with k from its largest magnitude (tt_range_rule), and sigma_out,
 * err2_out and the core that carries the norm are scaled back by 2^k, 2^2k and 2^k;
 * results are correct wherever they are representable in FP64 (err2 of a tensor whose
 * squared norm is below DBL_MIN underflows). */
tt_status tt_svd(const void* X, tt_dtype dt, int d, const int64_t* n, int r_max, double tol,
                 double* const* cores_out, int64_t* ranks_out, double* sigma_out,
                 double* err2_out, void* work, size_t work_bytes, void* stream);

/* tt_svd with options (opts may be NULL = defaults). */
tt_status tt_svd_ex(const void* X, tt_dtype dt, int d, const int64_t* n, int r_max, double tol,
                    double* const* cores_out, int64_t* ranks_out, double* sigma_out,
                    double* err2_out, void* work, size_t work_bytes, void* stream,
                    const tt_opts* opts);

/* tt_svd_from_host: tt_svd_ex with X in HOST memory (n_1*...*n_d elements of type
 * dt, Fortran order; pinned memory for the copy to overlap, pageable memory works
 * but serialises).  The library copies X into X_dev (caller-owned device buffer of
 * the same size) on an internal stream forked from `stream`, in `chunks` row blocks
 * of the first unfolding that is not elided (0 = 16 blocks), and runs the first TSQR
 * level (Alg. 2 line 5, Sec. 3.2) on each block as soon as that block has arrived;
 * the partial R's of all blocks enter the same reduction tree, so the result equals
 * tt_svd_ex up to the order of the tree.  When every step is elided X is copied in
 * one piece.  work: at least tt_query_from_host's work_bytes (256-byte aligned).
 * Asynchronous on `stream`: X_host must stay valid and unchanged until `stream`
 * has passed this call.  Argument errors: TT_EINVAL (null pointers, chunks outside
 * 0..4096); TT_ENOMEM if work_bytes is too small; TT_ECUDA if the copy stream
 * cannot be created. */
tt_status tt_query_from_host(int d, const int64_t* n, int r_max, double tol, tt_dtype dt,
                             int chunks, size_t* work_bytes);
tt_status tt_svd_from_host(const void* X_host, void* X_dev, tt_dtype dt, int d, const int64_t* n,
                           int r_max, double tol, int chunks, double* const* cores_out,
                           int64_t* ranks_out, double* sigma_out, double* err2_out, void* work,
                           size_t work_bytes, void* stream, const tt_opts* opts);

/* Reads the device status word left by the last tt_svd* call that used `work`
 * (synchronising `stream` first).  TT_OK if no device-side failure was seen. */
tt_status tt_last_device_status(const void* work, void* stream);

/* ---- building blocks (each one step of the path; used by the tests) ---------
 * tt_tsqr: R factor of the Q-less TSQR of W (rows x m, column-major, leading
 *   dimension ld >= rows) -- Alg. 6 panels in a flat tree per warp (Sec. 3.2)
 *   and further levels of the same kernel over the stacked partial R's.
 *   R_out: device m*m doubles, column-major, upper triangular (R is unique up
 *   to the signs of its rows).  dt = storage type of W.  work: tt_tsqr_query.
 *   1 <= m <= 512. */
tt_status tt_tsqr_query(int64_t rows, int m, tt_dtype dt, size_t* work_bytes);
tt_status tt_tsqr(const void* W, tt_dtype dt, int64_t rows, int m, int64_t ld, double* R_out,
                  void* work, size_t work_bytes, void* stream);
/* tt_tsqr in a chosen arithmetic: TT_ARITH_F64 with dt = TT_F64 runs every level in native
 *   FP64 (the native FP64 form of tt_svd; up to m = 64 the first level may take the blocked
 *   kernel, tuning key tsqr.blk64); any other arith is tt_tsqr.  Same workspace
 *   (tt_tsqr_query covers both arithmetics). */
tt_status tt_tsqr_ex(const void* W, tt_dtype dt, int64_t rows, int m, int64_t ld, double* R_out,
                     void* work, size_t work_bytes, tt_arith arith, void* stream);

/* tt_small_svd: R = U Sigma V^T for a square m x m matrix R (column-major,
 *   device doubles) by one-sided Jacobi (Eq. QR_trick needs Sigma and V only).
 *   sigma: device m doubles, descending.  V: device m*m doubles, column-major.
 *   work: tt_small_svd_query.  1 <= m <= 512. */
tt_status tt_small_svd_query(int m, size_t* work_bytes);
tt_status tt_small_svd(const double* R, int m, double* sigma, double* V, void* work,
                       size_t work_bytes, void* stream);

/* tt_small_svd_noalloc: tt_small_svd for callers that cannot allocate device
 *   memory.  The paper has no counterpart; this is a convenience of the library.
 *   Who needs it: code that must not call cudaMalloc/cudaFree -- for example a
 *   component whose device memory belongs to the application's own pool
 *   allocator, or a loop where an allocation's implicit device synchronisation
 *   would stall other streams -- and plain-C callers with no workspace at hand.
 *   It takes the same R, m, sigma and V as tt_small_svd (caller-owned device
 *   buffers) but no workspace: its scratch (~1.5 MiB) is a static device array
 *   inside the library, reserved on every GPU that loads the library until the
 *   process exits.  Limits and rules:
 *   - m must be in [1, 256]; larger m returns TT_EINVAL (tt_last_error says why).
 *   - The first call on a device looks up the scratch address for that device
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - All calls share the one scratch array: calls that can overlap on the GPU
 *     (different streams without ordering between them) race; order them.
 *   - A device-side failure (Jacobi sweep limit, non-finite value) is reported
 *     by sigma[0] = NaN, since there is no workspace status word to read.
 *   It calls no cudaMalloc, cudaFree or allocating library routine. */
tt_status tt_small_svd_noalloc(const double* R, int m, double* sigma, double* V, void* stream);

/* tt_tsmm: Y = W V (Sec. 4.1.2 TSMM; with the unpadded layouts used here the
 *   reshape of Alg. 2 line 11 is a view of Y).  W: rows x m (ld), storage dt;
 *   V: device m x k doubles column-major (ldv = m); Y: device rows x k doubles
 *   column-major with leading dimension ldy >= rows.  Arithmetic as the
 *   matching tt_svd form (float-float for TT_F64, FP32 for TT_F32), in FP32's
 *   exponent range: W's row maxima and the outputs must lie within [2^-100, 2^100]
 *   in magnitude for the stated accuracy (tt_svd scales its input into that window
 *   first; the building block does not), smaller rows lose digits or flush to zero.
 *   tt_tsmm_ex with TT_ARITH_F64 takes any finite FP64 input. */
tt_status tt_tsmm(const void* W, tt_dtype dt, int64_t rows, int m, int64_t ld, const double* V,
                  int k, double* Y, int64_t ldy, void* stream);

/* tt_tsmm in a chosen arithmetic: TT_ARITH_F64 with an FP64 W gives the native FP64 form's
 *   product -- for m >= 16 the FP64-accurate tensor-core splitting (seven bf16-exact digits
 *   per value taken from the FP64 bits, 28 digit products per level set, exact level sums
 *   combined in integers and rounded once to FP64: normwise error about 2^-53 of
 *   sum_k |W_ik||V_kj|), else FP64 multiply-adds; any other arith is tt_tsmm. */
tt_status tt_tsmm_ex(const void* W, tt_dtype dt, int64_t rows, int m, int64_t ld, const double* V,
                     int k, double* Y, int64_t ldy, tt_arith arith, void* stream);

/* tt_gen_uniform: entries start..start+count-1 of the i.i.d. uniform[0,1)
 *   stream of `seed` (Philox4x32-10, Salmon et al. SC'11; entry e is built from
 *   block e/2 with counter (lo32(e/2), hi32(e/2), 0, 0) and key (lo32(seed),
 *   hi32(seed)); a double from words x, y is ((x>>5)*2^26 + (y>>6)) * 2^-53).
 *   dt = TT_F64 writes doubles, TT_F32 writes the same values rounded to float. */
tt_status tt_gen_uniform(void* out, tt_dtype dt, int64_t count, uint64_t seed, int64_t start,
                         void* stream);

/* ---- batched form -----------------------------------------------------------
 * Many independent TT-SVDs in one call; each job has the semantics of tt_svd.
 * The jobs are spread over a pool of library-owned CUDA streams that are forked
 * from `stream` and joined back into it with events, so the call is
 * asynchronous on `stream` and can be captured into one CUDA graph.  The
 * workspace holds one slice per job (tt_batched_query); jobs never share
 * buffers.  Jobs are started largest first. */
typedef struct {
  const void* X;            /* device input, Fortran order */
  tt_dtype dtype;
  int d;
  int64_t n[TT_MAX_D];
  int r_max;
  double tol;
  double* cores_out[TT_MAX_D];  /* device pointers, caps from tt_core_caps */
  int64_t* ranks_out;       /* device int64[d+1] */
  double* sigma_out;        /* optional */
  double* err2_out;         /* optional */
  int* status_out;          /* optional device int: the job's device status word */
} tt_job;

tt_status tt_batched_query(int batch, const tt_job* jobs, size_t* work_bytes);
tt_status tt_svd_batched(int batch, const tt_job* jobs, void* work, size_t work_bytes,
                         void* stream);

/* ---- serve form -------------------------------------------------------------
 * Continuous batching.  A host scheduler thread admits queued requests (FIFO)
 * into slots -- one CUDA stream each -- whenever a slot is free and the
 * request's accounted memory (input + cores + workspace) fits in what is left
 * of hbm_budget_bytes; requests that arrive while others run start as soon as a
 * slot and memory free up, and their kernels overlap on the device.  The server
 * owns one workspace arena (arena_bytes, allocated at creation and
 * sub-allocated first-fit); inputs and outputs stay caller-owned and must stay
 * valid until the request is done.  All waits are bounded; nothing spins on the
 * device. */
typedef struct tt_server tt_server;
typedef struct {
  int max_inflight;         /* slots (concurrent requests on the device), >= 1 */
  size_t arena_bytes;       /* workspace arena; 0 = a quarter of the budget */
  double timeout_s;         /* limit for a blocking tt_serve_poll (0 = 60 s) */
  int policy;               /* admission order: TT_SERVE_FIFO (0) or TT_SERVE_SHORTEST (1) */
  double max_wait_s;        /* TT_SERVE_SHORTEST: a request queued this long is admitted
                               next regardless of its size (0 = 1 s) */
} tt_serve_opts;
/* Admission order.  FIFO: in arrival order.  SHORTEST: the queued request with the least
 * estimated device work (the plan's TSQR, small-SVD and W V_r costs) first, except that
 * the oldest request goes first once it has waited max_wait_s (no request waits
 * indefinitely while smaller ones keep arriving).  Both stop at the first request the
 * budget or the arena cannot take yet. */
enum { TT_SERVE_FIFO = 0, TT_SERVE_SHORTEST = 1 };
typedef struct {
  tt_status status;         /* TT_OK, a launch error, TT_ENUMERIC, TT_ECANCELLED ... */
  double t_submit, t_start, t_done;   /* steady-clock seconds: queued, admitted, seen done */
} tt_job_result;

tt_status tt_serve_create(size_t hbm_budget_bytes, const tt_serve_opts* opts, tt_server** out);
/* Queue a request (the tt_job is copied); returns TT_ENOMEM if it can never fit the
 * budget or arena.  ready_stream: the caller's stream (cudaStream_t as void*, NULL = the
 * legacy default stream) on which the request's input and output buffers are written
 * or cleared; the server records an event on it at submission, and the request's kernels
 * wait for that event, so work queued on ready_stream before the submit is complete
 * before the request reads X or writes its outputs.  Work queued later on ready_stream
 * is not ordered with the request: poll until it is done before touching its buffers. */
tt_status tt_serve_submit(tt_server* s, const tt_job* job, void* ready_stream, uint64_t* ticket);
/* TT_OK with *out filled when the request is done; TT_EAGAIN if not yet (wait = 0);
 * with wait != 0 blocks up to timeout_s, then TT_ETIMEOUT.  A finished ticket may be
 * polled again until it is released. */
tt_status tt_serve_poll(tt_server* s, uint64_t ticket, int wait, tt_job_result* out);
/* Forget a finished request (its result can no longer be polled), so that a long-running
 * server keeps no record per past request.  TT_EAGAIN if it has not finished, TT_EINVAL
 * for an unknown or already released ticket. */
tt_status tt_serve_release(tt_server* s, uint64_t ticket);
/* Stops admission, cancels queued requests (TT_ECANCELLED), waits (bounded) for
 * running ones, frees the arena and streams. */
tt_status tt_serve_destroy(tt_server* s);

/* ---- measurement -----------------------------------------------------------
 * tt_profile(1) makes every later tt_svd* call record CUDA events around its
 * kernels (on the call's stream) together with each kernel's algorithmic bytes
 * and flops; tt_profile(0) stops; both clear earlier records.  tt_profile_read
 * synchronises the recorded events and returns up to `max` records:
 * kinds[k] (0 TSQR first level, 1 TSQR upper levels, 2 SVD of R, 3 rank choice
 * and core, 4 W*V_r, 5 the exponent-range decision and the re-run of the first level
 * that it may ask for, 6 W*V_r of step i fused with the first TSQR level of step i-1),
 * steps[k] (the step index i), ms[k], bytes[k], flops[k],
 * info[k] (Jacobi sweeps for kind 2 -- valid while the workspace of that call is
 * untouched -- else -1).  *n receives the number of records available.  Any
 * output array may be NULL. */
tt_status tt_profile(int enable);
tt_status tt_profile_read(int max, int* n, int* kinds, int* steps, double* ms, double* bytes,
                          double* flops, int* info);

/* Arithmetic peak of this GPU, measured: kind 0 = FP32 FMA, 1 = FP64 FMA, 2 = the lazy
 * float-float multiply-add of the float-float dot products (one FP64-equivalent FMA),
 * 3 = the FP64 tensor-core MMA (mma.sync m8n8k4, f64).
 * *flops_per_s = 2 x multiply-adds per second over every SM (8 CTAs of 256 threads per
 * SM, 8 independent chains per thread, a warm-up run, then one timed run of ~10 ms with
 * CUDA events on `stream`).  Synchronises `stream`.  TT_EINVAL for another kind. */
tt_status tt_fma_rate(int kind, double* flops_per_s, void* stream);

/* Self-test of the bounded device waits (failure detection without a fault): launches one
 * CTA that waits, with the wait helper of the column-owned TSQR kernels, on an mbarrier
 * that nothing arrives at; after limit_cycles SM clock cycles (1000 .. 4e9) the wait gives
 * up and the kernel records DEV_ERR_TIMEOUT in the status word at the start of `work`
 * (device, 256-byte aligned, >= 256 bytes), which tt_last_device_status(work, stream)
 * then reports as TT_ETIMEOUT.  The context stays usable.  Asynchronous on `stream`. */
tt_status tt_wait_selftest(void* work, int64_t limit_cycles, void* stream);

/* Number of kernels this library has launched since it was loaded. */
tt_status tt_stats(int64_t* launches);

/* Tuning parameters, process-wide: kernel and layout choices read when a plan is built
 * (set by the autotuner, paper_2102_00104_gb300/autotune.py, and by the Python
 * binding's TT_TUNE="key=value,..." environment variable).  value < 0 removes a key, so
 * its default applies again.  Results never depend on these settings beyond rounding.
 * Keys (default in brackets):
 *   TSQR (Alg. 6 panels, Sec. 3.2)
 *     "tsqr.col" [1]          column-owned first-level kernel for 16 < m <= 160; 0: row-group kernel
 *     "tsqr.col.<b>" [1]      the same per m bucket b (0: m <= 32, 1: <= 64, 2: <= 80,
 *                             3: <= 128, 4: <= 160), float-float form
 *     "tsqr.colcfg64.<b>" [-] the same for the native FP64 arithmetic
 *     "tsqr.colcfg.<b>" [-]   column-owned layout 0..9 (warps, columns per warp, rows per
 *                             lane) for bucket b; ignored when it cannot hold m
 *     "tsqr.cols" [1]         shared-memory panel kernel for 160 < m <= 512; 0: row-group kernel
 *     "tsqr.merge_m" [96]     smallest m whose upper tree levels use the triangle-merge kernel
 *     "tsqr.pcap_q" [4 or 8]  first-level partial R's at most rows / (q m / 4) when merging
 *     "tsqr.narrow_k" [32]    narrow kernel (m <= 16): 32 or 64 panel rows per lane x MAXM
 *     "tsqr.narrow_cpsm" [4]  narrow kernel: CTAs of 4 warps per SM
 *     "tsqr.narrow_norm" [1]  narrow kernel: renormalise the float-float pairs after each update
 *   small SVD of R (one-sided Jacobi)
 *     "svd.block" [1]         block-cyclic cluster Jacobi for m > 48
 *     "svd.block_nc" [0]      force its cluster size (2..16; other values: cost model)
 *     "svd.cluster" [1]       ring-ordered cluster Jacobi where the block form does not fit
 *     "svd.g" [16]            single-CTA Jacobi: lanes per column pair (8, 16 or 32)
 *     "svd.wide" [1]          wide steps (rows < m): Jacobi on the columns of W^T, no TSQR
 *     "svd.wide_g" [8..32]    lanes per column pair of the wide Jacobi
 *   W V_r (Sec. 4.1.2)
 *     "tsmm.oz" [1]           Ozaki-split tensor-core product: 0 never, 1 where float-float is
 *                             ALU-bound (m >= 16 and m r >= 6 (m + r)), 2 wherever it applies
 *     "tsmm.oz_nbuf" [1]      tile buffers per CTA of that kernel (1 or 2)
 *     "tsmm.tc" [0]           1: the tcgen05 form of the same product where it applies
 *   fusion (Alg. 2 lines 11 and 5)
 *     "fuse.tsmm_tsqr" [0]    1: W V_r of step i computes the next unfolding inside the first
 *                             TSQR level of step i-1 when that level is narrow (m_{i-1} <= 8,
 *                             m_i <= 8); 0: separate launches (measured faster)
 *   batched form
 *     "batched.streams" [64]  streams of tt_svd_batched (1..128) */
tt_status tt_tune_set(const char* key, int value);

/* The exponent-range rule of the FP64 form in float-float arithmetic, for tests.
 * Float-float has FP32's exponent range, so tt_svd reads an FP64 X as X 2^-k (k an exact
 * power-of-two shift) and scales sigma_out, err2_out and the core that carries the norm
 * back by 2^k; entries below 2^-62 times the largest one are read as zero (their squares
 * would leave FP32's range), which changes no singular value by more than
 * 2^-62 sqrt(n_1...n_d) max|x| (2^-47 max|x| for 2^30 entries).  Arguments:
 * floor(log2 max|x|) of a strided sample of X and of all of X (what the first TSQR
 * level, Alg. 2 line 5, meets), TT_RANGE_NONE when nothing nonzero and finite was seen.
 * Outputs: the shift of the first pass (*k_try), whether that level runs again (*redo),
 * and the shift every later step and the results use (*k).  Pure host computation. */
#define TT_RANGE_NONE (-100000)
tt_status tt_range_rule(int sample_exp, int seen_exp, int* k_try, int* redo, int* k);

const char* tt_status_str(tt_status s);

/* Text of the last CUDA failure (TT_ECUDA) seen by a tt_* call on the calling
 * thread: the CUDA error name and message and the failing call.  Empty if none. */
const char* tt_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TT_SVD_H */
