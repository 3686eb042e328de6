// te_internal.h - declarations shared by the CUDA translation units of the
// Top-K Lanczos eigensolver (device state layout, kernel argument blocks and
// host-side launch wrappers).  Not part of the public C ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "topk_eigs.h"

namespace te {

// Device memory of plans, layouts and temporaries (te_mem.cu): a stream-ordered
// pool per device that keeps freed blocks for the next plan.  Same contract as
// cudaMalloc / cudaFree (usable by every stream on return; the free waits for
// the device to be idle first).
cudaError_t dev_alloc(void** p, size_t bytes);
template <typename T>
cudaError_t dev_alloc(T** p, size_t bytes) {
  return dev_alloc(reinterpret_cast<void**>(p), bytes);
}
cudaError_t dev_free(void* p);
// free once the work queued on s so far is done (every user of p is on s)
cudaError_t dev_free_on(void* p, cudaStream_t s);

constexpr int MAX_M = 64;        // largest supported krylov_steps
constexpr int TILE_R = 256;      // rows per tile of the basis passes
// per-CTA partial slots: dots with the pass vector at [0, MAX_M], dots with
// the candidate column at [SLOT_D2, SLOT_D2 + MAX_M], two norms at SLOT_N
constexpr int SLOT_D2 = MAX_M + 1;
constexpr int SLOT_N = 2 * MAX_M + 2;
constexpr int PSTRIDE = 2 * MAX_M + 4;
constexpr int CONSUMERS = 256;   // compute threads of the basis passes
constexpr int PASS_THREADS = CONSUMERS + 32;  // + one producer warp
constexpr int MAX_STAGES = 32;

enum Prec : int { PREC_DDD = 0, PREC_FDF = 1 };

// Device-resident state of one solve (lives in the plan's work memory).
struct LzState {
  double s[MAX_M + 2];      // v_j = s[j] * stored column j
  double alpha[MAX_M + 1];  // alpha[i] = alpha_{i+1}
  double beta[MAX_M + 2];   // beta[0] = beta_1 = 0, beta[i] = beta_{i+1}
  double c1[MAX_M + 2];     // coefficients of the first axpy pass
  double c2[MAX_M + 2];     // coefficients of the second axpy pass
  double xscale;            // multiplier of the source vector in the first axpy
  double f2;                // delayed reorthogonalisation: coefficient of the candidate
  double bt[MAX_M + 2];     // delayed: norm of each candidate after one sweep
  int rflag[MAX_M + 2];     // delayed: column set by a restart (its beta is 0)
  double cj[MAX_M + 2];     // delayed: second-sweep coefficients of the candidate
  double anorm;             // max_j |alpha_j| + beta_j + beta_{j+1}
  double theta_sel[MAX_M];  // selected Ritz values (selection order)
  double resid_est[MAX_M];  // |beta_{m+1} y_k[m-1]|
  double C[MAX_M * MAX_M];  // Ritz coefficients C[j*K + k] = s_j sign_k Y[j][idx_k]
  int restart_flag;         // set when the last step broke down
  int restarts;             // restarts so far (random stream = restarts + 1)
  int status;               // te_status of the solve so far
  int sweeps;               // Jacobi sweeps
  unsigned int ticket;      // last-CTA counter
  int stall_armed;          // test hook (te_options.stall_first_pass): the next pass that
                            // reads the basis waits for copies that are never issued
  // per-solve inputs (written by the host before each solve)
  const double* v1;
  double* eigvecs;
  double* eigvals_out;
  double* eigvecs_user;  // with refinement: the caller's buffer (eigvecs is the plan's)
};

// Host arrays whose resize() leaves new elements default-initialised (no
// zero fill): the layout and ordering arrays are written in full by worker
// threads, which then also take the first-touch page faults in parallel.
template <typename T>
struct NoInitAlloc : std::allocator<T> {
  template <typename U>
  struct rebind {
    using other = NoInitAlloc<U>;
  };
  NoInitAlloc() = default;
  template <typename U>
  NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
  template <typename U>
  void construct(U* p) noexcept(std::is_nothrow_default_constructible<U>::value) {
    ::new (static_cast<void*>(p)) U;
  }
  template <typename U, typename... Args>
  void construct(U* p, Args&&... args) {
    ::new (static_cast<void*>(p)) U(std::forward<Args>(args)...);
  }
};
template <typename T>
using hvec = std::vector<T, NoInitAlloc<T>>;

struct LongRow {
  int32_t row, first, count, pad_;  // a row cut into `count` pieces, partials at [first, ...)
};

// SELL-C-sigma layout of the matrix for the SpMV (Kreutzer et al., SISC 2014):
// rows are cut into pieces of at most SELL_VMAX entries, the pieces of every
// window of SELL_WINDOW consecutive rows are sorted by length (longest first)
// and grouped in slices of SELL_C; a slice stores its entries column-major
// (entry k of lane i at base + k*SELL_C + i), padded with zero values to the
// length of its longest piece.
constexpr int SELL_C = 32;
constexpr int SELL_VMAX = 64;
constexpr int SELL_WINDOW = 2048;
constexpr int32_t SELL_SKIP = INT32_MIN;  // lane without a piece

struct SellSlice {
  int64_t base;  // first entry of the slice
  int32_t len;   // entries per lane (length of its longest piece)
  int32_t pad_;
};

struct SellHost {
  hvec<SellSlice> slices;
  hvec<int32_t> vout;  // per lane: row (>= 0), -1 - partial slot, or SELL_SKIP
  hvec<int64_t> vsrc;  // per lane: first CSR entry of its piece
  hvec<int32_t> vlen;  // per lane: entries of its piece
  hvec<int32_t> vrow;  // per lane: the row its piece belongs to (-1: empty lane)
  hvec<LongRow> lrows;
  int64_t entries = 0;        // padded entries
  int64_t pieces = 0;         // partial sums of cut rows
  int64_t nbig = 0;           // leading cut rows (most pieces first) summed by a whole warp
};
constexpr int SELL_BIG_PIECES = 16;  // cut rows with more pieces get a whole warp
// returns false (and a message) if row_ptr is malformed
// window: rows sorted together (sigma); vmax: longest piece (rows above are cut)
// A row order: row r of the layout is CSR row perm[r], whose entries start at
// src[r] and number len[r]
struct RowOrder {
  const int32_t* perm;
  const int64_t* src;
  const int32_t* len;
};
// ord (optional): row r of the layout is CSR row ord->perm[r] and writes output r
bool make_sell(const int64_t* rp, int64_t n, int64_t nnz, SellHost& out, std::string& err,
               int window = SELL_WINDOW, int vmax = SELL_VMAX, const RowOrder* ord = nullptr);
// row_ptr starts at 0, ends at nnz and never decreases
bool rows_valid(const int64_t* rp, int64_t n, int64_t nnz, std::string& err);
// rows by length, longest first (stable): perm[r] = row placed at r, iperm = inverse,
// src/len = that row's first entry and length
void degree_order(const int64_t* rp, int64_t n, int32_t* perm, int32_t* iperm, int64_t* src,
                  int32_t* len);

// The same layout built by kernels from a device row_ptr (te_layout_dev.cu);
// identical to make_sell / degree_order.  Order of use: count (row checks,
// the row order when `reorder`), order (when `reorder`: perm, iperm and the
// placed rows' first entries and lengths), windows (the per-window counts;
// totals = slices, padded entries, cut-row pieces, cut rows, to the host),
// emit (the slices, lane records and sorted cut rows into the caller's
// arrays).  Scratch memory is owned by the object.
struct DevLayout {
  int64_t n = 0, nnz = 0, nwin = 0;
  int window = SELL_WINDOW, vmax = SELL_VMAX;
  bool reorder = false;
  const int64_t* rp = nullptr;
  void* scratch = nullptr;
  int64_t* wc = nullptr;
  int32_t* sorted_rows = nullptr;
  int32_t* spare_rows = nullptr;
  const int64_t* view_src = nullptr;
  const int32_t* view_len = nullptr;
  const int32_t* view_perm = nullptr;
  int64_t nslices = 0, entries = 0, pieces = 0, nlrows = 0;
  // err receives the reason when the row pointers are malformed or the size
  // is not covered (cudaErrorInvalidValue is returned then)
  cudaError_t count(const int64_t* rp_dev, int64_t n, int64_t nnz, int window, int vmax,
                    bool reorder, cudaStream_t s, std::string& err);
  cudaError_t order(int32_t* perm, int32_t* iperm, int64_t* src, int32_t* len, cudaStream_t s);
  cudaError_t windows(cudaStream_t s, int64_t* totals_host);
  cudaError_t emit(SellSlice* slices, int32_t* vout, int64_t* vsrc, int32_t* vlen, int32_t* vrow,
                   LongRow* lrows, LongRow* lrows_tmp, cudaStream_t s, int* nbig_host);
  ~DevLayout();
};
bool dev_layout_fits(int64_t n, int window, int vmax);

// SpMV layout candidates (rows sorted together, longest piece) tried by the
// autotuner; the first is the default
constexpr int TUNE_N = 5;
inline constexpr int TUNE_WINDOW[TUNE_N] = {SELL_WINDOW, SELL_WINDOW, SELL_WINDOW, 256, 16384};
inline constexpr int TUNE_VMAX[TUNE_N] = {SELL_VMAX, 32, 128, SELL_VMAX, SELL_VMAX};
// Build each candidate layout of a device CSR (rp, ci, val; rph: host row
// pointers; hord / dcolmap: relabelled rows, or nullptr) in temporary
// memory, time its SpMV with CUDA events on s and set *best to the fastest
// candidate's index (te_solver.cu).
cudaError_t autotune_layout(int prec, int vk, int in_type, const int64_t* rph, const int64_t* rp,
                            const int32_t* ci, const void* val, int64_t n, int64_t nnz,
                            const RowOrder* hord, const int32_t* dcolmap, cudaStream_t s,
                            int* best);

// Device copy of a SELL layout.
struct DevSell {
  const SellSlice* slices = nullptr;
  const int32_t* vout = nullptr;
  int32_t* cols = nullptr;
  void* vals = nullptr;
  int vk = TE_F64;               // te_dtype of vals: F64, F32, BF16 or FP8_E4M3
  const float* lscale = nullptr; // FP8: per-lane scale (the row's), else nullptr
  int64_t ebase = 0;             // cols/vals hold entries [ebase, ...) of the layout
                                 // (a streamed row block); 0 when resident
  void* vpart = nullptr;  // partial sums of cut rows (8 bytes each)
  const LongRow* lrows = nullptr;
  int nslices = 0, nlrows = 0;
  int nlbig = 0;  // lrows[0, nlbig) have more than SELL_BIG_PIECES pieces
  int64_t hot = 0;  // rows by degree: gathers of x[c >= min(hot, what L1 holds)] skip L1
};

// fill the SELL layout from the CSR (a warp per slice): the column indices
// (through colmap when given: column c -> colmap[c]) and the values, in two
// kernels.  Values: in_type / out_type (te_dtype) F64 -> F64, F64 -> F32
// (round to nearest even), F32 -> F32, BF16 -> BF16, FP8_E4M3 -> FP8_E4M3
// (codes copied); for FP8 also lane_scale[lane] = row_scale[vrow[lane]] (0
// for empty lanes).  bad (optional, device): the kernels do nothing when *bad
// is non-zero (the column check, earlier on s, found an invalid index).
cudaError_t launch_sell_fill_cols(const int32_t* ci, const SellSlice* slices, const int64_t* vsrc,
                                  const int32_t* vlen, int nslices, int32_t* cols,
                                  const int32_t* colmap, const int* bad, cudaStream_t s);
cudaError_t launch_sell_fill_vals(int in_type, int out_type, const void* val,
                                  const SellSlice* slices, const int64_t* vsrc,
                                  const int32_t* vlen, int nslices, void* vals,
                                  const int32_t* vrow, const float* row_scale, float* lane_scale,
                                  const int* bad, cudaStream_t s);
// the same arrays built on the host (in_type F64 or F32 -> vk F64 or F32);
// false if a column index lies outside [0, n)
bool build_sell_host(const SellHost& H, const int32_t* ci, const void* val, int in_type, int vk,
                     int64_t n, const int32_t* colmap, int32_t* cols, void* vals);
// binary64 CSR values -> `to` (TE_F32, TE_BF16 codes, TE_FP8_E4M3 codes with
// per-row scales); round to nearest, ties to even (te_quant.cu)
cudaError_t launch_quantize(int to, const int64_t* rp, const double* val, int64_t n, int64_t nnz,
                            void* out, float* row_scale, cudaStream_t s);
cudaError_t spmv_prepare();  // once per process/device, outside stream capture

// SpMV: y = A x.  out_f64: write binary64 (else the precision's vector type).
// Rows without entries are not written (the caller keeps them zero).
cudaError_t launch_spmv(int prec, const DevSell& S, const void* x, void* y, bool out_f64,
                        cudaStream_t s);
cudaError_t launch_validate_cols(const int32_t* ci, int64_t nnz, int64_t n, int* flag,
                                 cudaStream_t s);

// ---- basis passes ----
enum PassMode : int {
  MODE_DOT = 0,
  MODE_AXPY_DOT = 1,
  MODE_AXPY_STORE = 2,
  MODE_RITZ = 3,
  MODE_DCGS_DOT = 4,    // delayed: dots of every column with y and with the candidate
  MODE_DCGS_UPDATE = 5  // delayed: finish the candidate column, form the next one
};
enum XSource : int { X_VEC = 0, X_RANDOM = 1, X_V1 = 2 };
enum Finalize : int {
  FIN_DOT_STEP = 0,
  FIN_DOT_RESTART = 1,
  FIN_AXPYDOT = 2,       // second-sweep coefficients (restart passes)
  FIN_STORE_STEP = 3,
  FIN_STORE_RESTART = 4,
  FIN_STORE_INIT = 5,
  FIN_NONE = 6,
  FIN_AXPYDOT_STEP = 7,  // second-sweep coefficients and alpha = h1_i + h2_i
  FIN_DOT_NOREORTH = 8,  // alpha_i alone and the three-term coefficients
  FIN_STORE_NOREORTH = 9, // beta_{i+1} of the three-term update (source scaled by s_i)
  FIN_DCGS_DOT = 10,       // delayed: rho, beta_i, alpha_i and the update coefficients
  FIN_DCGS_UPDATE = 11     // delayed: norm and scale of the next candidate, breakdown
};

struct PassArgs {
  const void* V;     // stored basis: element (r, c) at (r / TILE_R) * tstride + c * cstride + r % TILE_R
  void* Vmut;        // same buffer, for the column written by AXPY_STORE
  int64_t ld;        // padded rows
  int64_t tstride;   // elements from a tile to the next tile of the same column
  int64_t cstride;   // elements from a column to the next (TILE_R: tile-major)
  void* xcopy;       // optional: the column a pass stores, also written contiguously
  const void* cand;  // delayed form: the candidate (column nb-1 of the pass) is read from
                     // this contiguous copy, and a new candidate is written only there
  const int32_t* perm;  // optional: row r of the vectors is the caller's row perm[r]
  double* urows;     // RITZ, optional: write the vectors by rows (K rounded up to even
                     // per row) here instead of by columns to st->eigvecs
  int64_t n;         // true rows
  int nb;            // basis columns read by this pass: col0 .. col0 + nb - 1
  int col0;          // first basis column read (0 unless reorthogonalisation is off)
  int exact_tail;    // FDF phase A: the last exact_tail columns in double-float
  int col_out;       // column written by AXPY_STORE (the next candidate in DCGS_UPDATE)
  int col_fix;       // DCGS_UPDATE: the candidate column rewritten as final
  int step;          // Lanczos step (0-based)
  int m;             // krylov steps of the solve
  int K;             // eigenpairs (RITZ)
  int xsrc;          // XSource
  int fin;           // Finalize
  int only_on_restart;  // exit at once unless st->restart_flag is set
  int stall;         // test hook: honour st->stall_armed (a plan with stall_first_pass)
  const void* xvec;  // source vector (precision's vector type), X_VEC
  void* wout;        // AXPY_DOT: output vector
  uint64_t seed;
  double tol;        // breakdown tolerance (relative to anorm)
  LzState* st;
  void* partials;    // gridDim.x * PSTRIDE slots
};

struct PassLaunch {
  int grid = 0;
  size_t smem = 0;
  size_t region = 0;  // bytes of the stage buffers
  int stages = 0;
};
// configure a pass kernel for `max_cols` basis columns (and K Ritz vectors);
// returns the launch shape
cudaError_t pass_config(int prec, int mode, int max_cols, int K, int num_sms, PassLaunch& out);
cudaError_t launch_pass(int prec, int mode, const PassArgs& a, const PassLaunch& L,
                        cudaStream_t s);

// ---- Jacobi phase ----
struct JacobiArgs {
  const double* alpha;  // m
  const double* beta;   // m+1 (beta[1..m-1] off-diagonal, beta[m] = beta_{m+1})
  const double* s;      // column scales (for Ritz coefficients), or nullptr
  int m, K, which;
  double* theta_out;    // K (selection order)
  double* Y_out;        // optional m x K column-major (sign-fixed eigenvectors)
  double* C_out;        // optional Ritz coefficients C[j*K+k]
  double* resid_out;    // optional residual estimates
  double* eigvals_dev;  // optional copy of theta_out
  LzState* st;          // status / sweeps (may be nullptr)
  int* sweeps_out;      // optional
  int* status_out;      // optional
};
cudaError_t jacobi_prepare();  // once per process/device, outside stream capture
cudaError_t launch_jacobi(const JacobiArgs& a, cudaStream_t s);

// ---- Rayleigh-quotient refinement and Gram matrix ----
// For Ritz vector k (st->eigvecs + k*n) and y = M u_k (binary64): replaces
// st->theta_sel[k] by the Rayleigh quotient theta + u'r/u'u (r = y - theta u)
// and st->resid_est[k] by ||y - theta' u|| / ||u||; also writes
// st->eigvals_out[k] when set.  `partials`: grid * 4 doubles.
cudaError_t launch_refine(LzState* st, const double* y, int64_t n, int k, double* partials,
                          int grid, cudaStream_t s);
int refine_grid(int num_sms);
// copy `count` doubles from src to st->eigvecs_user (no-op when it is NULL)
cudaError_t launch_copy_out(LzState* st, const double* src, size_t count, int grid,
                            cudaStream_t s);
// st->eigvecs_user[k*n + v] = src[k*n + iperm[v]] for k < K, v < n: Ritz
// vectors of the relabelled rows back in the caller's row order (no-op when
// eigvecs_user is NULL)
cudaError_t launch_copy_out_perm(LzState* st, const double* src, int64_t n, int K,
                                 const int32_t* iperm, int grid, cudaStream_t s);
// the same from vectors stored by rows: st->eigvecs_user[k*n + v] =
// src[iperm[v] * Kr + k], Kr = K rounded up to even
cudaError_t launch_copy_out_rows(LzState* st, const double* src, int64_t n, int K,
                                 const int32_t* iperm, int grid, cudaStream_t s);
// G[a*K + b] = u_a . u_b (device), per-block partials in `partials`
// (grid * K*(K+1)/2 doubles)
cudaError_t launch_gram(const double* U, int64_t n, int K, double* partials, int grid,
                        double* G, cudaStream_t s);

// ---- serving engine: one launch per phase for every live solve ----
constexpr int SRV_MAX_SLOTS = 64;  // solves resident at once
constexpr int SRV_MAX_CTAS = 32;   // pass CTAs per solve (fixed by its size alone)

// one live solve (FDF arithmetic: binary32 basis, binary32 or bfloat16 values)
struct BatchSlot {
  const SellSlice* slices;
  const int32_t* vout;
  const int32_t* cols;
  const void* vals;
  const LongRow* lrows;
  void* vpart;
  void* V;         // basis, n_pad x (m+1) binary32
  void* ytil;      // SpMV output (double-float pairs)
  void* w;         // first-sweep result
  void* partials;  // ncta * PSTRIDE slots
  LzState* st;
  int64_t n, n_pad;
  uint64_t seed;
  double tol;
  int vk, nslices, nlrows, m, K, step, ncta, pad_;
};
// the live solves of one engine step, with prefix offsets into the global
// slice, cut-row and pass-block enumerations
struct BatchTable {
  int nslots, pad_;
  int64_t slice_off[SRV_MAX_SLOTS + 1];
  int64_t lrow_off[SRV_MAX_SLOTS + 1];
  int item_off[SRV_MAX_SLOTS + 1];
  BatchSlot slot[SRV_MAX_SLOTS];
};
// persistent grids of the batched SpMV (8 warps a block) and finaliser: as
// many blocks as fit on num_sms SMs at once (te_spmv.cu)
cudaError_t batch_spmv_grids(int num_sms, int* spmv_blocks, int* fin_blocks);
// y_s = M_s v_{s, step_s} for every slot (te_spmv.cu)
cudaError_t launch_batch_spmv(const BatchTable* T, int spmv_blocks, int fin_blocks,
                              cudaStream_t s);
// passes of the Lanczos step of every slot; restart = the breakdown passes
// (te_reorth.cu); L: the launch configuration for the engine's largest m
cudaError_t launch_batch_pass(int mode, const BatchTable* T, int restart, const PassLaunch& L,
                              cudaStream_t s);
cudaError_t batch_pass_prepare(const PassLaunch& L);  // outside stream capture
// per-solve set-up kernel of a plan (te_solver.cu)
cudaError_t launch_solve_begin(LzState* st, const double* v1, double* eigvecs, double* eigvals,
                               double* plan_vecs, cudaStream_t s);
double breakdown_tolerance(int prec);

// ---- small utilities ----
// record the thread-local message returned by te_last_error()
void set_last_error(const std::string& msg);
cudaError_t launch_basis_to_f64(int prec, const void* V, int64_t tstride, int64_t cstride,
                                int64_t n, int cols, const double* s_dev, const int32_t* iperm,
                                double* out, cudaStream_t st);

}  // namespace te
