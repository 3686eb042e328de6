/*
 * topk_eigs.h - C ABI of the GB300 (sm_103a) Top-K sparse eigensolver.
 *
 * Method: Sgherzi, Parravicini & Santambrogio, "A Mixed Precision, Multi-GPU
 * Design for Large-scale Top-K Sparse Eigenproblems", arXiv 2201.07498.
 * A Lanczos phase (Algorithm 1, Section III) builds an orthonormal Krylov
 * basis V = [v_1..v_m] of the symmetric matrix M from an L2-normalised
 * random start vector, with full reorthogonalisation, and a tridiagonal
 * T = tridiag(alpha_1..alpha_m; beta_2..beta_m); a Jacobi phase (Section III,
 * Fig. 1) diagonalises T; eigenvectors of M are V times the eigenvectors of
 * T (Section III).  The K eigenpairs "largest in modulo" (Section I) are
 * returned.  Precision follows Section III-A: matrix values, arithmetic and
 * vector storage can differ ("FDF" = float values, double arithmetic, float
 * vectors; "DDD" = all double).
 *
 * Conventions shared by every entry point
 *   - Every call returns a te_status; nothing aborts.  te_last_error() gives a
 *     thread-local message for the last failing call on this thread.
 *   - The caller owns every buffer it passes; the library never frees them.
 *     Work memory is allocated inside the call (or the plan) and freed before
 *     return (or at te_plan_destroy), into the library's device memory pool,
 *     which keeps it for the next call (te_set_memory_cache).
 *   - Device pointers are CUDA device (or managed) memory of the current
 *     device.  "Host" outputs may be pageable or pinned.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls that
 *     return results to the host synchronise that stream once, at the end.
 *   - Matrices are square (n x n), symmetric (Lanczos requires it; the solver
 *     does not check it, te_check_symmetric does), stored as CSR with int64
 *     row pointers (n+1 entries,
 *     row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz) and int32 column
 *     indices in [0, n).  Column order within a row is free.
 *   - Dense results are column-major: eigenvector k occupies
 *     eigvecs[k*n .. k*n+n-1].
 *   - On an error found before the device work starts (arguments, CSR,
 *     allocation) the outputs are left untouched; after a device-side failure
 *     (TE_ERR_TIMEOUT, TE_ERR_NOT_CONVERGED) eigenvector buffers the kernels
 *     write directly (device or pinned host) may hold partial results.
 */
#ifndef TOPK_EIGS_H
#define TOPK_EIGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TE_OK = 0,
  TE_ERR_INVALID_ARG = 1,    /* bad sizes, NULL pointers, malformed CSR */
  TE_ERR_OUT_OF_MEMORY = 2,  /* device allocation failed or over budget */
  TE_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  TE_ERR_BREAKDOWN = 4,      /* the Krylov space could not be extended */
  TE_ERR_NOT_CONVERGED = 5,  /* the Jacobi sweeps hit their limit */
  TE_ERR_TIMEOUT = 6,        /* a bounded device-side wait expired */
  TE_ERR_UNSUPPORTED = 7     /* a valid but unimplemented combination */
} te_status;

/* element types (Section III-A's precision letters) */
typedef enum { TE_F64 = 0, TE_F32 = 1, TE_BF16 = 2, TE_FP8_E4M3 = 3 } te_dtype;

/* (matrix values, arithmetic, vector storage).  Supported:
 *   DDD = {TE_F64, TE_F64, TE_F64}: plain binary64 on the FP64 pipe.
 *   FDD = {TE_F32, TE_F64, TE_F64}: as DDD with binary32 matrix values
 *         (converted exactly to binary64 as they are read).
 *   FDF = {TE_F32, TE_F64, TE_F32}: binary32 matrix values and Lanczos
 *         vectors; every product and sum of the SpMV, the
 *         reorthogonalisation and the Ritz contraction is carried in
 *         double-float (about 48 significant bits) on the FP32 pipes, and
 *         cross-block sums in binary64.
 *   BDF = {TE_BF16, TE_F64, TE_F32}: as FDF with bfloat16 matrix values.
 *   8DF = {TE_FP8_E4M3, TE_F64, TE_F32}: as FDF with FP8 E4M3 matrix values
 *         and one binary32 scale per row (scale_r = max_j |a_rj| / 448).
 *   BDF and 8DF are built from binary64 values (te_csr.values_f64 = 1); the
 *   library rounds them (see te_quantize).  With te_options.refine the
 *   selected Ritz values are refined against the binary64 values. */
typedef struct {
  int32_t values;
  int32_t arithmetic;
  int32_t vectors;
} te_precision;

#define TE_DEVICE 0 /* CSR arrays live in device memory */
#define TE_HOST 1   /* CSR arrays live in host memory (copied in by the call) */

typedef struct {
  int64_t n;              /* rows = columns, >= 1, < 2^31 */
  int64_t nnz;            /* stored entries, >= 0 */
  const int64_t* row_ptr; /* n + 1 */
  const int32_t* col_idx; /* nnz */
  const void* values;     /* nnz elements: binary64 if values_f64, else of type
                             precision.values */
  const float* row_scale; /* reserved for scaled 8-bit values; must be NULL */
  int32_t where;          /* TE_DEVICE or TE_HOST */
  int32_t values_f64;     /* 0: `values` already have type precision.values.
                             1: `values` are binary64; the library rounds them to
                             precision.values (to nearest, ties to even) when it
                             builds its copy of the matrix, and keeps the binary64
                             values when refinement is requested. */
} te_csr;

#define TE_WHICH_LARGEST_MAGNITUDE 0 /* |theta| descending; ties: positive, then index */
#define TE_WHICH_LARGEST_ALGEBRAIC 1 /* theta descending; ties: lower index */

#define TE_REORTH_FULL 0 /* full reorthogonalisation every step (Algorithm 1): classical
                            Gram-Schmidt applied twice, three passes over the basis */
#define TE_REORTH_NONE 1 /* three-term recurrence only (Section IV-D's comparison) */
#define TE_REORTH_DELAYED 2 /* full reorthogonalisation with the second sweep of each new
                            vector delayed into the next step (two passes over the basis
                            per step; the same vectors up to rounding) */

typedef struct {
  uint64_t seed;    /* SplitMix64 seed: start vector = stream 0, restart r = stream r */
  const double* v1; /* optional raw start vector (n, device); NULL = draw from seed */
  int32_t which;    /* TE_WHICH_* */
  int32_t use_graph; /* plans: capture the whole solve as one CUDA graph (default 1) */
  size_t device_budget_bytes; /* 0 = no limit on the work memory */
  int32_t reorth;   /* TE_REORTH_FULL (default), TE_REORTH_NONE or TE_REORTH_DELAYED */
  int32_t refine;   /* 1: after the Ritz vectors, replace each selected Ritz value by
                       the binary64 Rayleigh quotient u'Mu/u'u of its vector against
                       the binary64 matrix, and its residual by the true residual
                       ||Mu - theta u|| / ||u||.  Needs A->values_f64 = 1.  Costs K
                       binary64 SpMVs; with eigvecs NULL the plan keeps its own
                       vectors.  Default 0. */
  size_t matrix_budget_bytes; /* 0 (default): the plan's copy of the matrix lives in device
                       memory.  Otherwise, when that copy (about nnz * (4 + value bytes))
                       would exceed this many bytes, a TE_HOST matrix stays in pinned
                       host memory and every SpMV streams it in row blocks through two
                       device buffers of at most matrix_budget_bytes / 2 each: the copy
                       of the next block (on a second stream) overlaps the SpMV of the
                       current one.  Binary64 or binary32 values only (DDD, FDD, FDF);
                       no refinement.  A TE_DEVICE matrix over the budget is an error
                       (TE_ERR_OUT_OF_MEMORY). */
  int32_t autotune; /* 1: at plan creation, build the SpMV layout with a few settings of
                       its window (rows sorted together) and piece length, time each
                       on this matrix and keep the fastest (te_plan_layout reports it);
                       resident plans only.  0 (default): window 2048, pieces of 64. */
  int32_t order;    /* TE_ORDER_KEEP (default) or TE_ORDER_DEGREE: the plan relabels the
                       rows (and the same columns) by length, longest first, so that the
                       SpMV's reads of the vector for the most connected columns share
                       cache lines (power-law graphs).  The matrix is M' = P M P^T for
                       that permutation P; the caller sees no difference: the start
                       vector and restart draws are indexed by the caller's rows and
                       the Ritz vectors come back in the caller's row order.
                       Eigenvalues agree with TE_ORDER_KEEP up to rounding (the sums
                       over rows run in another order).  Costs a counting sort of the
                       rows at plan creation, the permutation (8 bytes per row) and
                       the plan's own copy of the Ritz vectors (n x K binary64). */
  int32_t stall_first_pass; /* test hook for the device-side failure path, 0 (default) in
                       normal use.  1: the first pass over the basis of the plan's first
                       solve issues none of its copies, so its consumer warps' bounded
                       waits expire (after a shortened limit); the pass raises
                       TE_ERR_TIMEOUT in the status word and every kernel still returns,
                       with no copy in flight.  That solve returns TE_ERR_TIMEOUT (its
                       outputs are meaningless); the plan's later solves run normally. */
} te_options;

#define TE_ORDER_KEEP 0   /* rows in the caller's order */
#define TE_ORDER_DEGREE 1 /* rows by length, longest first (ties: caller's order) */

/* Fill `opt` with the defaults: seed 0, v1 NULL, largest magnitude, graphs on,
 * no budget, full reorthogonalisation, no refinement. */
void te_default_options(te_options* opt);

/* Thread-local message describing the last error on this thread ("" if none). */
const char* te_last_error(void);

/* Static name of a status code. */
const char* te_status_string(te_status s);

/* Bytes of device work memory a plan for (A, K, krylov_steps, p) allocates,
 * excluding a device copy of a host CSR.  Returns 0 for invalid arguments. */
size_t te_workspace_bytes(const te_csr* A, int32_t K, int32_t krylov_steps, te_precision p);

/*
 * One complete Top-K solve (Algorithm 1 + Jacobi + Ritz vectors, Section III):
 *   K            number of eigenpairs, 1 <= K <= krylov_steps
 *   krylov_steps m, the Lanczos steps (size of T), K <= m <= min(n, 64)
 *   eigvals      K doubles, host or device: the selected Ritz values
 *   eigvecs      n*K doubles (column-major), host or device, or NULL to skip
 *                the Ritz-vector contraction.  Device memory and pinned host
 *                memory the device can address (cudaHostAlloc, or registered)
 *                are written by the kernels directly; pageable host memory
 *                is filled from a device copy at the end
 *   residuals    K doubles, host or device, or NULL: the Ritz residual
 *                estimates |beta_{m+1} * y_k[m]| (= ||M u_k - theta_k u_k|| in
 *                exact arithmetic), or with opt->refine the true residuals
 *                ||M u_k - theta_k u_k|| / ||u_k|| in binary64
 * With A->where == TE_HOST the matrix is copied to the device inside the call.
 * Synchronises `stream` before returning.  TE_ERR_BREAKDOWN is returned (with
 * all outputs written) when a restart could not produce a new direction.
 */
te_status te_topk_eigs(const te_csr* A, int32_t K, int32_t krylov_steps, te_precision p,
                       const te_options* opt, double* eigvals, double* eigvecs,
                       double* residuals, void* stream);

/* ---- plans: reuse the analysis, work memory and CUDA graph across solves ---- */
typedef struct te_plan te_plan;

/* Analyse A (row partition for the SpMV, CSR validation), allocate the work
 * memory and, with opt->use_graph, capture the solve as a CUDA graph.  A
 * TE_HOST matrix is copied into plan-owned device memory; a TE_DEVICE matrix
 * is referenced (it must outlive the plan and not change).  *out is NULL on
 * error. */
te_status te_plan_create(const te_csr* A, int32_t K, int32_t krylov_steps, te_precision p,
                         const te_options* opt, void* stream, te_plan** out);

/* Run one solve on `stream`.  v1: optional raw start vector (n, device) that
 * overrides the plan's option for this solve; outputs as in te_topk_eigs. */
te_status te_plan_solve(te_plan* plan, const double* v1, double* eigvals, double* eigvecs,
                        double* residuals, void* stream);

/* Launch one solve on `stream` without waiting for it: eigenvalues go to the
 * device buffer `eigvals_dev` (K doubles) and Ritz vectors to `eigvecs_dev`
 * (or NULL).  The caller synchronises; te_plan_status then reports the
 * device-side status of the last finished solve. */
te_status te_plan_launch(te_plan* plan, const double* v1, double* eigvals_dev,
                         double* eigvecs_dev, void* stream);
te_status te_plan_status(te_plan* plan);

/* Kernel kinds reported by te_plan_profile. */
#define TE_KIND_SPMV 0       /* SpMV of Algorithm 1 (with the long-row finalize) */
#define TE_KIND_DOT 1        /* first Gram-Schmidt sweep: dots against the basis */
#define TE_KIND_AXPY_DOT 2   /* first update fused with the second sweep's dots */
#define TE_KIND_AXPY_STORE 3 /* second update, norms (beta), next basis vector */
#define TE_KIND_RESTART 4    /* restart passes (return at once unless a breakdown) */
#define TE_KIND_JACOBI 5     /* Jacobi phase, selection, Ritz coefficients */
#define TE_KIND_RITZ 6       /* Ritz-vector contraction V * Y */
#define TE_KIND_OTHER 7      /* solve set-up and start-vector pass */
#define TE_KIND_REFINE 8     /* binary64 Rayleigh-quotient refinement (SpMVs + reductions) */
#define TE_NUM_KINDS 9

/* Run one solve on `stream` without the CUDA graph, timing every kernel with
 * CUDA events recorded on `stream`, and synchronise.  For each kind k:
 * ms[k] = summed kernel time, launches[k] = kernel count, bytes[k] = the
 * algorithmic bytes those launches must move (SpMV: nnz*(4+value bytes) +
 * 8(n+1) + n*(vector bytes) + 8n; basis passes: the basis columns they read
 * plus the n-vectors they read and write; Ritz: m basis columns + 8nK).
 * Arrays have TE_NUM_KINDS entries; any may be NULL. */
te_status te_plan_profile(te_plan* plan, double* ms, int32_t* launches, double* bytes,
                          void* stream);

/* Number of kernels one solve launches (graph nodes when captured). */
int32_t te_plan_kernel_count(const te_plan* plan);

/* The SpMV layout of the plan: rows sorted together (window) and the longest
 * piece a row is cut into (vmax). */
te_status te_plan_layout(const te_plan* plan, int32_t* window, int32_t* vmax);

/* Row blocks each SpMV streams from host memory (0: the matrix is resident). */
int64_t te_plan_stream_blocks(const te_plan* plan);

void te_plan_destroy(te_plan* plan);

/* ---- device memory of plans (no counterpart in the paper: runtime support) ----
 * Plans (and te_topk_eigs, te_lanczos, the autotuner and the serving engine's
 * per-class tuning) take their device memory from a stream-ordered memory pool
 * per device that the library owns.  Memory a plan frees stays reserved by the
 * pool and serves the next plan without the driver mapping pages again; the
 * pool returns it to the driver when an allocation finds the device full, when
 * te_release_cached_memory is called, or, past the release threshold set by
 * te_set_memory_cache, at the next synchronisation.  Other allocators in the
 * process (PyTorch's, for example) do not see the reserved memory as free. */

/* Release threshold of every device's pool, in bytes (default UINT64_MAX: keep
 * all freed memory; 0: return it at every synchronisation). */
te_status te_set_memory_cache(uint64_t keep_bytes);

/* Return every unused block of every pool to the driver.  Memory held by live
 * plans is not affected. */
te_status te_release_cached_memory(void);

/* The pool of `device`: bytes reserved from the driver and bytes held by live
 * allocations (both 0 before the first plan on that device).
 * TE_ERR_INVALID_ARG for a NULL output or a device index outside [0, 64). */
te_status te_memory_cached(int32_t device, uint64_t* reserved_bytes, uint64_t* used_bytes);

/* ---- single phases, for testing and for callers composing their own solver ---- */

/* y = M x with the solver's SpMV (Algorithm 1, SpMV step).  x: n elements of
 * type p.vectors (device); y: n doubles (device).  A must be TE_DEVICE; with
 * A->values_f64 the values are rounded to p.values first, as in a plan. */
te_status te_spmv(const te_csr* A, te_precision p, const void* x, double* y, void* stream);

/* The Lanczos phase alone (Algorithm 1): writes alpha[0..m-1] and
 * beta[0..m] (beta[0] = beta_1 = 0, beta[i] = beta_{i+1}; host arrays) and,
 * if `basis` is not NULL, the basis V as n x m doubles (device, column-major).
 * `restarts` (host, may be NULL) receives the number of breakdown restarts. */
te_status te_lanczos(const te_csr* A, int32_t krylov_steps, te_precision p,
                     const te_options* opt, double* alpha, double* beta, double* basis,
                     int32_t* restarts, void* stream);

/* The Jacobi phase alone on T = tridiag(alpha; beta[1..m-1]) (Section III):
 * alpha (m) and beta (m+1, beta[0] ignored) are device arrays; theta
 * receives all m eigenvalues in selection order (`which`), Y (m x m,
 * column-major, device) the matching unit eigenvectors of T, each with its
 * largest-magnitude entry positive.  sweeps (host, may be NULL) receives the
 * number of sweeps.  m <= 64. */
te_status te_tridiag_eigs(int32_t m, const double* alpha, const double* beta, int32_t which,
                          double* theta, double* Y, int32_t* sweeps, void* stream);

/* y = M x like te_spmv, but without allocating any device memory: for callers
 * that cannot call cudaMalloc (for instance when another allocator already
 * owns the device memory, or when a serving loop must not take the
 * allocator's locks and latency).  The paper has no counterpart; it exists
 * for such callers.  Work memory is one fixed 4 MiB __device__ array inside
 * the library, shared by all calls on a device, which limits nnz to
 * 131072 * 2048 (DDD) or 131072 * 4096 (FDF); larger matrices get
 * TE_ERR_INVALID_ARG.  The first call on each device looks up the array's
 * device address (do that first call before any stream capture); the
 * address is kept for the life of the process, so a program that resets a
 * device (cudaDeviceReset) must not call this entry point on it afterwards.
 * Calls that overlap on the GPU (other streams, other host threads) race on
 * the array and must be serialised by the caller.  A must be TE_DEVICE with
 * values_f64 = 0 (there is no room to round the values); x has n elements of
 * type p.vectors; y receives n doubles.  A column index outside [0, n) or a
 * malformed row_ptr (row_ptr[0] != 0, decreasing, row_ptr[n] != nnz) is
 * found on the device and returns TE_ERR_INVALID_ARG (y is then
 * meaningless).  The work grows with n as well as nnz (every row is
 * visited).  Synchronises `stream`. */
te_status te_spmv_noalloc(const te_csr* A, te_precision p, const void* x, double* y,
                          void* stream);

/* Round binary64 CSR values (A: TE_DEVICE, values_f64 = 1) to a storage type,
 * on the device, in CSR order, as the plans do (Section III-A's reduced
 * precisions): round to nearest, ties to even, from the binary64 value
 * directly; a zero result is +0.
 *   to = TE_F32:      out = nnz floats.
 *   to = TE_BF16:     out = nnz uint16 bfloat16 codes (8 significant bits).
 *   to = TE_FP8_E4M3: out = nnz uint8 E4M3 codes (bias 7, largest finite 448,
 *                     no infinities) and row_scale = n floats:
 *                     scale_r = binary32(max_j |a_rj| / 448), 1 for an
 *                     all-zero row; code = round(a / scale_r) saturated at 448;
 *                     the stored matrix entry is scale_r * value(code).
 * row_scale must be given for TE_FP8_E4M3 and only then.  Values must be
 * finite with magnitude below 2^127.  Synchronises `stream`. */
te_status te_quantize(const te_csr* A, int32_t to, void* out, float* row_scale, void* stream);

/* Measure the rate (reads per second) at which the GPU serves random 4-byte
 * reads from a device table of table_elems floats (the bound of an SpMV whose
 * column indices are random: one scattered read of x per non-zero).  Best of
 * two timed launches after one warm-up, CUDA events on `stream`.  Not part of
 * the paper's method: a measurement for the SpMV's roofline. */
te_status te_probe_gather(int64_t table_elems, void* stream, double* gathers_per_s);

/* Gram matrix G = U^T U of K vectors (U: n x K, column-major, device), summed
 * in binary64 in a fixed order; G (K x K, row-major) is written to host memory.
 * For the orthogonality metric of Section IV-D (the mean angle between pairs
 * of eigenvectors).  1 <= K <= 64.  Synchronises `stream`. */
te_status te_gram(int64_t n, int32_t K, const double* U, double* G, void* stream);

/* ---- serving engine: continuous batching of many small solves ----
 *
 * Not in the paper (a serving front end for its solver).  A server keeps up
 * to max_slots solves resident on the device, each with its own matrix
 * layout, Krylov basis and tridiagonal, and advances every resident solve by
 * one Lanczos step per te_server_step: one batched SpMV launch, one batched
 * launch per basis pass (and per restart pass), replayed as one captured
 * CUDA graph.  A solve that reaches its m-th step is finished (Jacobi, Ritz
 * vectors) and its slot and work memory are freed at once; pending requests
 * are admitted, in submission order, whenever a slot and enough memory of the
 * device pool are free, so requests that arrive while others run join the
 * next step.  Each solve is given a number of pass CTAs that depends on its
 * own size only, so its result is the same, bit for bit, whatever else runs
 * beside it.
 *
 * Forms: FDF or BDF (binary32 basis, double-float arithmetic; binary32 or
 * bfloat16 values; bfloat16 needs values_f64).  Calls on one server must not
 * overlap (one host thread at a time). */
typedef struct te_server te_server;

typedef struct {
  int32_t max_slots;          /* resident solves, 1 .. 64 */
  int32_t max_krylov_steps;   /* largest m accepted, <= 64 */
  size_t device_budget_bytes; /* device pool for resident solves and finished results */
  int32_t use_graph;          /* replay each engine step as one captured CUDA graph */
  int32_t autotune;           /* 1: tune the SpMV layout per request class (value type,
                                 log2 n, log2 mean row length): the class's first
                                 request times the autotuner's layout candidates on
                                 its own matrix (host analysis thread, its own stream
                                 and temporary device memory outside the pool) and
                                 later requests of the class use the fastest.  The
                                 choice is timing-based, so two servers may pick
                                 different layouts for a class (results then differ
                                 in the last bits).  0 (default): the default layout */
} te_server_options;

/* Create a server (allocates the pool; work is issued on a stream the server
 * owns). */
te_status te_server_create(const te_server_options* opt, te_server** out);

/* Queue one solve: A in host memory, K eigenpairs largest in modulo from
 * m = krylov_steps Lanczos steps, start vector from `seed`.  *ticket
 * identifies the request.  The server reads A's arrays when it admits the
 * request: they must stay valid and unchanged until te_server_poll reports
 * the request done.  Malformed row pointers are rejected here
 * (TE_ERR_INVALID_ARG); column indices are checked on the device at
 * admission (a request with one outside [0, n) finishes with
 * TE_ERR_INVALID_ARG before its first SpMV); a request larger than the whole
 * pool fails with TE_ERR_OUT_OF_MEMORY when it reaches the head of the queue. */
te_status te_server_submit(te_server* srv, const te_csr* A, int32_t K, int32_t krylov_steps,
                           te_precision p, uint64_t seed, int64_t* ticket);

/* One engine step: wait for the previous step, retire finished solves, launch
 * one Lanczos step of every resident solve, then admit pending requests
 * (their layouts are built behind the step; they join the batch at the next
 * step).  *live (resident + just admitted) and *pending (may be NULL) receive
 * the counts.  Returns without waiting for the launched work. */
te_status te_server_step(te_server* srv, int32_t* live, int32_t* pending);

/* *done = 1 when the request has finished: eigvals (K), residual estimates
 * (K, may be NULL) and, if eigvecs is not NULL, the n x K column-major Ritz
 * vectors are written to host memory and the request is released; the call
 * returns the request's own status.  *done = 0: nothing written. */
te_status te_server_poll(te_server* srv, int64_t ticket, int32_t* done, double* eigvals,
                         double* eigvecs, double* residuals);

/* Completion queue: up to `cap` tickets of requests that finished (with any
 * status) since the last call, in the order they finished, written to
 * tickets[]; *count receives how many.  A reported ticket is then polled
 * with te_server_poll (which returns its results at once).  Lets a client
 * poll only finished requests instead of every outstanding one. */
te_status te_server_completed(te_server* srv, int64_t* tickets, int32_t cap, int32_t* count);

/* The autotuner's choices so far (te_server_options.autotune): for up to `cap`
 * tuned request classes, the class key ((value type * 64 + floor(log2 n)) * 32
 * + floor(log2(nnz / n))), the window and the longest piece of its layout
 * (arrays may be NULL); *count receives the number of tuned classes. */
te_status te_server_classes(te_server* srv, int32_t* class_key, int32_t* window, int32_t* vmax,
                            int32_t cap, int32_t* count);

/* Resident and queued solves, pool bytes in use now and at most so far. */
te_status te_server_stats(const te_server* srv, int32_t* live, int32_t* pending,
                          size_t* pool_used, size_t* pool_peak);

/* Cumulative host seconds of the calling threads: waiting for engine steps,
 * admitting requests (pool allocation, device copies and fills), launching
 * steps, inside submit, and inside poll (copying the Ritz vectors out;
 * releasing the request).  Any output may be NULL. */
te_status te_server_timing(const te_server* srv, double* wait_s, double* admit_s,
                           double* launch_s, double* submit_s, double* poll_copy_s,
                           double* poll_free_s);

/* The analysis threads' cumulative seconds (summed over threads): building
 * request layouts, gathering a request's arrays into pinned memory, copying
 * them to the device staging area, waiting for a staging block (turn or
 * space); the requests they analysed; and the engine steps launched with the
 * number of solves those steps advanced (their ratio is the mean batch).
 * Any output may be NULL. */
te_status te_server_analysis(const te_server* srv, double* layout_s, double* gather_s,
                             double* copy_s, double* stage_wait_s, int64_t* analysed,
                             int64_t* engine_steps, int64_t* resident_steps);

void te_server_destroy(te_server* srv);

/* Host-side layout behind the SpMV (no GPU needed; row_ptr in host memory):
 * the SELL-C-sigma arrangement a plan builds (Kreutzer et al., SIAM J. Sci.
 * Comput. 2014).  Rows are cut into pieces of at most vmax entries (0: 64);
 * within each window of `window` consecutive rows (0: 2048) the pieces are
 * sorted by length (longest first) and grouped into slices of 32 lanes, each
 * slice padded to its longest piece.  Writes the slice count, the padded entry count and the
 * number of rows cut into several pieces.  Optional per-slice output
 * slice_len[nslices]; optional per-lane outputs (32 * nslices entries):
 * lane_out = the row the lane sums (>= 0), -1 - p for piece p of a cut row,
 * or INT32_MIN for an empty lane; lane_src = first CSR entry of its piece;
 * lane_len = entries of its piece.  Returns TE_ERR_INVALID_ARG for a
 * malformed row_ptr. */
te_status te_spmv_layout(const int64_t* row_ptr, int64_t n, int64_t nnz, int32_t window,
                         int32_t vmax, int64_t* nslices, int64_t* entries, int64_t* nlong_rows,
                         int32_t* slice_len, int32_t* lane_out, int64_t* lane_src,
                         int32_t* lane_len);

/* The same layout (and, with order = TE_ORDER_DEGREE, the row order of
 * te_degree_order) built on the device from row_ptr in device memory, the way
 * plans build it: for tests and analysis.  Outputs are host arrays, each
 * optional (NULL skips it); sizes as for te_spmv_layout, plus perm[n] (the
 * caller's row placed at layout row r; the identity for TE_ORDER_KEEP),
 * slice_base[nslices] (first entry of each slice), lane_row[32 * nslices]
 * (the caller's row a lane's piece belongs to, -1 for an empty lane),
 * long_rows[3 * nlong_rows] ((layout row, first partial slot, pieces) of each
 * cut row, most pieces first, ties in row order) and *nbig (cut rows with more
 * than 16 pieces).  lane_out holds layout rows (relabelled rows with
 * TE_ORDER_DEGREE) and lane_src entries of the caller's CSR.  Call once with
 * NULL arrays to learn the sizes.  Returns TE_ERR_INVALID_ARG for a malformed
 * row_ptr, TE_ERR_UNSUPPORTED when vmax > 128 or the matrix is too large for
 * the device build.  Synchronises `stream`. */
te_status te_spmv_layout_device(const int64_t* row_ptr, int64_t n, int64_t nnz, int32_t window,
                                int32_t vmax, int32_t order, int64_t* nslices, int64_t* entries,
                                int64_t* nlong_rows, int32_t* perm, int32_t* slice_len,
                                int64_t* slice_base, int32_t* lane_out, int64_t* lane_src,
                                int32_t* lane_len, int32_t* lane_row, int32_t* long_rows,
                                int32_t* nbig, void* stream);

/* Debug check of the symmetry Lanczos assumes (host only, no GPU needed; the
 * solver itself does not check it): A must be TE_HOST with binary64 values
 * (values_f64 = 1).  Duplicate entries of a row are summed and a missing
 * mirror entry counts as zero.  *max_abs_diff (may be NULL) receives
 * max |a_ij - a_ji|; returns TE_OK when that is <= tol, TE_ERR_INVALID_ARG
 * (with the value in te_last_error) otherwise or for a malformed CSR. */
te_status te_check_symmetric(const te_csr* A, double tol, double* max_abs_diff);

/* The row order of TE_ORDER_DEGREE (host only, no GPU needed): rows by
 * length, longest first, rows of equal length in increasing index order.
 * perm[r] (n, host) = the caller's row placed at r; iperm (n, host, may be
 * NULL) = its inverse.  Returns TE_ERR_INVALID_ARG for a malformed row_ptr. */
te_status te_degree_order(const int64_t* row_ptr, int64_t n, int64_t nnz, int32_t* perm,
                          int32_t* iperm);

#ifdef __cplusplus
}
#endif
#endif /* TOPK_EIGS_H */
