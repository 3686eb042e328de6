// te_solver.cu - host driver and C ABI of the Top-K Lanczos eigensolver.
//
// A plan owns the analysis of one matrix (SpMV row partition, validation),
// the work memory (Lanczos basis, vectors, device state) and, optionally, the
// whole solve captured as one CUDA graph: init pass, m Lanczos steps (SpMV,
// three basis passes, three restart passes that exit at once unless the step
// broke down), the Jacobi kernel and the Ritz contraction.  Scalars (alpha,
// beta, coefficients, breakdown flag) never leave the device during a solve;
// the only host synchronisation is the final read of the eigenvalues and the
// status word.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "te_internal.h"
#include "topk_eigs.h"

using namespace te;

namespace {

thread_local std::string g_err;

te_status fail(te_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

te_status cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return e == cudaErrorMemoryAllocation ? TE_ERR_OUT_OF_MEMORY : TE_ERR_CUDA;
}

#define TE_CK(call, what)                              \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// binary64 vectors and arithmetic with binary64 or binary32 values (DDD, FDD),
// or binary32 vectors with double-float arithmetic and binary32, bfloat16 or
// FP8 E4M3 values (FDF, BDF, 8DF)
int prec_of(te_precision p) {
  if ((p.values == TE_F64 || p.values == TE_F32) && p.arithmetic == TE_F64 &&
      p.vectors == TE_F64)
    return PREC_DDD;
  if ((p.values == TE_F32 || p.values == TE_BF16 || p.values == TE_FP8_E4M3) &&
      p.arithmetic == TE_F64 && p.vectors == TE_F32)
    return PREC_FDF;
  return -1;
}
size_t basis_elt(int prec) { return prec == PREC_DDD ? 8 : 4; }
size_t elt_of(int dtype) {
  return dtype == TE_F64 ? 8 : dtype == TE_F32 ? 4 : dtype == TE_BF16 ? 2 : 1;
}

double breakdown_tol(int prec) { return prec == PREC_DDD ? 1e-12 : 1e-6; }

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Pinned host memory the device can address (cudaHostAlloc'd or registered):
// the device-side pointer, else NULL.  Kernels then write results straight
// into it (over NVLink-C2C on Grace-Blackwell) with no device staging copy.
void* mapped_host_ptr(void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

struct Work {
  // byte offsets inside one allocation
  size_t V = 0, ytil = 0, xcur = 0, perm = 0, iperm = 0, w = 0, partials = 0, st = 0, Uint = 0, slices = 0, vout = 0,
         scols = 0, svals = 0, svals64 = 0, lscale = 0, lrows = 0, vpart = 0, flag = 0,
         total = 0;
};

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// sizes of the SELL layout of the SpMV (see te_internal.h)
struct SellSizes {
  size_t slices = 0, entries = 0, lrows = 0, pieces = 0;
};

// refine: room for the plan's own Ritz vectors (n x K) and, for a
// mixed-precision form, a binary64 copy of the SELL values; reorder: the row
// permutation both ways and the plan's own Ritz vectors (relabelled rows)
Work layout(int prec, int vk, int64_t n_pad, int m, int grid, const SellSizes& z,
            bool refine = false, int64_t n = 0, int K = 0, bool reorder = false) {
  Work w;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = al256(off + bytes);
    return o;
  };
  w.V = take((size_t)n_pad * (size_t)(m + 1) * basis_elt(prec));
  w.ytil = take((size_t)n_pad * 8);
  w.xcur = take((size_t)n_pad * basis_elt(prec));
  w.w = take((size_t)n_pad * 8);
  w.partials = take((size_t)grid * PSTRIDE * 8);
  w.st = take(sizeof(LzState));
  // by rows (K rounded up to even) for relabelled rows without refinement
  const size_t kcols = (reorder && !refine) ? (size_t)((K + 1) & ~1) : (size_t)K;
  w.Uint = (refine || reorder) ? take((size_t)n * kcols * 8) : 0;
  w.perm = reorder ? take((size_t)n * 4) : 0;
  w.iperm = reorder ? take((size_t)n * 4) : 0;
  w.slices = take(std::max<size_t>(z.slices, 1) * sizeof(SellSlice));
  w.vout = take(std::max<size_t>(z.slices, 1) * SELL_C * sizeof(int32_t));
  w.scols = take(std::max<size_t>(z.entries, 1) * sizeof(int32_t));
  w.svals = take(std::max<size_t>(z.entries, 1) * elt_of(vk));
  w.svals64 = (refine && vk != TE_F64) ? take(std::max<size_t>(z.entries, 1) * 8) : 0;
  w.lscale = vk == TE_FP8_E4M3 ? take(std::max<size_t>(z.slices, 1) * SELL_C * 4) : 0;
  w.lrows = take(std::max<size_t>(z.lrows, 1) * sizeof(LongRow));
  w.vpart = take(std::max<size_t>(z.pieces, 1) * 8);
  w.flag = take(16);
  w.total = off;
  return w;
}

int64_t pad_rows(int64_t n) { return (n + TILE_R - 1) / TILE_R * TILE_R; }

te_status check_args(const te_csr* A, int32_t K, int32_t m, te_precision p) {
  if (!A) return fail(TE_ERR_INVALID_ARG, "A is NULL");
  if (A->n < 1 || A->n >= (int64_t)1 << 31) return fail(TE_ERR_INVALID_ARG, "n out of range");
  if (A->nnz < 0) return fail(TE_ERR_INVALID_ARG, "nnz < 0");
  if (!A->row_ptr || !A->col_idx || (!A->values && A->nnz > 0))
    return fail(TE_ERR_INVALID_ARG, "CSR arrays must not be NULL");
  if (A->row_scale) return fail(TE_ERR_UNSUPPORTED, "row_scale is reserved (must be NULL)");
  if (A->where != TE_DEVICE && A->where != TE_HOST)
    return fail(TE_ERR_INVALID_ARG, "where must be TE_DEVICE or TE_HOST");
  if (A->values_f64 != 0 && A->values_f64 != 1)
    return fail(TE_ERR_INVALID_ARG, "values_f64 must be 0 or 1");
  if (prec_of(p) < 0)
    return fail(TE_ERR_UNSUPPORTED, "precision must be DDD, FDD, FDF, BDF (bfloat16 values) or "
                                    "8DF (FP8 E4M3 values)");
  if ((p.values == TE_BF16 || p.values == TE_FP8_E4M3) && A->values_f64 != 1)
    return fail(TE_ERR_INVALID_ARG,
                "bfloat16 and FP8 storage is built from binary64 values (values_f64 = 1)");
  if (K < 1) return fail(TE_ERR_INVALID_ARG, "K must be >= 1");
  if (m < K) return fail(TE_ERR_INVALID_ARG, "krylov_steps must be >= K");
  if (m > MAX_M) return fail(TE_ERR_UNSUPPORTED, "krylov_steps must be <= 64");
  if ((int64_t)m > A->n) return fail(TE_ERR_INVALID_ARG, "krylov_steps must be <= n");
  return TE_OK;
}

std::once_flag g_prep_once;
cudaError_t g_prep_err = cudaSuccess;

// kernel attributes (dynamic shared memory) are set once, before any capture
cudaError_t prepare_kernels() {
  std::call_once(g_prep_once, [] {
    g_prep_err = jacobi_prepare();
    if (g_prep_err == cudaSuccess) g_prep_err = spmv_prepare();
  });
  return g_prep_err;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

void te::set_last_error(const std::string& msg) { g_err = msg; }

struct te_plan {
  int prec = 0;
  int64_t n = 0, n_pad = 0, nnz = 0;
  int K = 0, m = 0;
  int in_type = TE_F64;  // type of the caller's values (TE_F64 or the precision's)
  int vk = TE_F64;       // storage type of the plan's copy of the values
  bool refine = false, noreorth = false, delayed = false;
  int sell_window = SELL_WINDOW, sell_vmax = SELL_VMAX;  // the SpMV layout's parameters
  te_options opt{};
  const int64_t* rp = nullptr;
  const int32_t* ci = nullptr;
  const void* val = nullptr;
  void* owned_csr = nullptr;
  int dev = 0, num_sms = 0;
  DevSell sell;
  DevSell sell64;  // binary64 values for the refinement (same layout)
  // streamed matrix: the SELL arrays stay in pinned host memory and every
  // SpMV copies them block by block into two device buffers
  struct Block {
    int first_slice, nslices;
    int64_t ebase, entries;
  };
  bool streaming = false;
  std::vector<Block> blocks;
  int64_t cap_entries = 0;     // entries per device buffer
  int32_t* hcols = nullptr;    // pinned host layout
  void* hvals = nullptr;
  cudaStream_t cs = nullptr;   // copy stream
  cudaEvent_t ev_ready[2] = {nullptr, nullptr}, ev_free[2] = {nullptr, nullptr};
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  double* ubase = nullptr;  // with refinement or reordering: the plan's Ritz vectors (n x K)
  bool reorder = false;     // rows relabelled by degree (te_options.order)
  int32_t* dperm = nullptr;   // solver row r = caller row dperm[r] (device)
  int32_t* diperm = nullptr;  // its inverse
  Work W;
  char* work = nullptr;
  LzState* st = nullptr;
  PassLaunch Ldot, Laxd, Lsto, Lritz, Lddot, Ldupd;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int nkernels = 0;
  // profiling: when set, every launch is bracketed by events of kind `kind`
  struct Prof {
    bool on = false;
    cudaStream_t s = nullptr;
    std::vector<cudaEvent_t> ev;  // pairs
    std::vector<int> kind;
    std::vector<double> bytes;
  } prof;
  struct HostRes {
    int restart_flag, restarts, status, sweeps;  // same order as in LzState
    double theta[MAX_M];
    double resid[MAX_M];
  };
  HostRes* hres = nullptr;  // pinned
};

namespace {

void* at(te_plan* P, size_t off) { return P->work + off; }

// A host-built layout's slice records, lane outputs and cut-row records
// (small) to the device, then synchronise (streamed plans keep the rest in
// host memory)
cudaError_t upload_meta(const SellHost& H, const DevSell& D, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (!H.slices.empty()) {
    e = cudaMemcpyAsync(const_cast<SellSlice*>(D.slices), H.slices.data(),
                        H.slices.size() * sizeof(SellSlice), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(const_cast<int32_t*>(D.vout), H.vout.data(),
                          H.vout.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess && !H.lrows.empty())
    e = cudaMemcpyAsync(const_cast<LongRow*>(D.lrows), H.lrows.data(),
                        H.lrows.size() * sizeof(LongRow), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

// Fill the SELL arrays from a device CSR, given the lane records (first CSR
// entry and length of every lane's piece, and its row for FP8): the columns,
// then the values, rounded or quantised (in_type: the caller's value type,
// binary64 when the storage type D.vk differs), and optionally a second value
// array with the binary64 values (vals64, for the refinement).  The columns
// wait for ev_cols and the values for ev_vals (when given: the arrival of the
// CSR's column and value arrays); bad: see launch_sell_fill_cols.
// Temporaries are freed before returning (the stream is synchronised).
cudaError_t fill_sell(int in_type, const DevSell& D, const int64_t* rp, const int32_t* ci,
                      const void* val, int64_t n, int64_t nnz, const int64_t* dsrc,
                      const int32_t* dlen, const int32_t* drow, void* vals64, float* lane_scale,
                      const int32_t* colmap, cudaStream_t s, cudaEvent_t ev_cols = nullptr,
                      cudaEvent_t ev_vals = nullptr, const int* bad = nullptr) {
  const bool quant = D.vk == TE_BF16 || D.vk == TE_FP8_E4M3;
  const bool fp8 = D.vk == TE_FP8_E4M3;
  void* q = nullptr;
  float* rscale = nullptr;
  cudaError_t e = cudaSuccess;
  if (quant) e = dev_alloc(&q, std::max<size_t>(nnz, 1) * elt_of(D.vk));
  if (e == cudaSuccess && fp8) e = dev_alloc(&rscale, std::max<int64_t>(n, 1) * sizeof(float));
  if (e == cudaSuccess && ev_cols) e = cudaStreamWaitEvent(s, ev_cols, 0);
  if (e == cudaSuccess)
    e = launch_sell_fill_cols(ci, D.slices, dsrc, dlen, D.nslices, D.cols, colmap, bad, s);
  if (e == cudaSuccess && ev_vals) e = cudaStreamWaitEvent(s, ev_vals, 0);
  if (e == cudaSuccess && quant)
    e = launch_quantize(D.vk, rp, static_cast<const double*>(val), n, nnz, q, rscale, s);
  if (e == cudaSuccess)
    e = launch_sell_fill_vals(quant ? D.vk : in_type, D.vk, quant ? q : val, D.slices, dsrc, dlen,
                              D.nslices, D.vals, drow, rscale, fp8 ? lane_scale : nullptr, bad,
                              s);
  if (e == cudaSuccess && vals64)
    e = launch_sell_fill_vals(TE_F64, TE_F64, val, D.slices, dsrc, dlen, D.nslices, vals64,
                              nullptr, nullptr, nullptr, bad, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (q) dev_free(q);
  if (rscale) dev_free(rscale);
  return e;
}

// The SELL copy of a device CSR from a host-built layout: its records and
// lane map uploaded, then filled (fill_sell).
cudaError_t upload_sell(int in_type, const SellHost& H, const int64_t* rp, const int32_t* ci,
                        const void* val, int64_t n, int64_t nnz, const DevSell& D, void* vals64,
                        float* lane_scale, const int32_t* colmap, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (!H.slices.empty()) {
    e = cudaMemcpyAsync(const_cast<SellSlice*>(D.slices), H.slices.data(),
                        H.slices.size() * sizeof(SellSlice), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(const_cast<int32_t*>(D.vout), H.vout.data(),
                          H.vout.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess && !H.lrows.empty())
    e = cudaMemcpyAsync(const_cast<LongRow*>(D.lrows), H.lrows.data(),
                        H.lrows.size() * sizeof(LongRow), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess || H.slices.empty()) return e;
  const bool fp8 = D.vk == TE_FP8_E4M3;
  // lane -> CSR piece map (and row): needed only while building
  int64_t* dsrc = nullptr;
  int32_t* dlen = nullptr;
  int32_t* drow = nullptr;
  e = dev_alloc(&dsrc, H.vsrc.size() * sizeof(int64_t));
  if (e == cudaSuccess) e = dev_alloc(&dlen, H.vlen.size() * sizeof(int32_t));
  if (e == cudaSuccess && fp8) e = dev_alloc(&drow, H.vrow.size() * sizeof(int32_t));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dsrc, H.vsrc.data(), H.vsrc.size() * sizeof(int64_t),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dlen, H.vlen.data(), H.vlen.size() * sizeof(int32_t),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && fp8)
    e = cudaMemcpyAsync(drow, H.vrow.data(), H.vrow.size() * sizeof(int32_t),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = fill_sell(in_type, D, rp, ci, val, n, nnz, dsrc, dlen, drow, vals64, lane_scale, colmap,
                  s);
  dev_free(dsrc);
  dev_free(dlen);
  if (drow) dev_free(drow);
  return e;
}

}  // namespace

// Build each candidate layout of the device CSR (rp, ci, val) in temporary
// memory, time its SpMV (CUDA events on s, after two warm-up calls), and
// return the index of the fastest.
cudaError_t te::autotune_layout(int prec, int vk, int in_type, const int64_t* rph, const int64_t* rp,
                            const int32_t* ci, const void* val, int64_t n, int64_t nnz,
                            const RowOrder* hord, const int32_t* dcolmap, cudaStream_t s,
                            int* best) {
  *best = 0;
  float best_ms = 0.f;
  const size_t xelt = prec == PREC_DDD ? 8 : 4;
  for (int c = 0; c < TUNE_N; ++c) {
    SellHost H;
    std::string err;
    if (!make_sell(rph, n, nnz, H, err, TUNE_WINDOW[c], TUNE_VMAX[c], hord))
      return cudaErrorInvalidValue;
    const size_t b_sl = al256(std::max<size_t>(H.slices.size(), 1) * sizeof(SellSlice));
    const size_t b_vo = al256(std::max<size_t>(H.vout.size(), 1) * 4);
    const size_t b_co = al256(std::max<size_t>((size_t)H.entries, 1) * 4);
    const size_t b_va = al256(std::max<size_t>((size_t)H.entries, 1) * elt_of(vk));
    const size_t b_lr = al256(std::max<size_t>(H.lrows.size(), 1) * sizeof(LongRow));
    const size_t b_vp = al256(std::max<size_t>((size_t)H.pieces, 1) * 8);
    const size_t b_ls = vk == TE_FP8_E4M3 ? b_vo : 0;
    const size_t b_x = al256((size_t)n * xelt), b_y = al256((size_t)n * 8);
    char* buf = nullptr;
    cudaError_t e = dev_alloc(&buf, b_sl + b_vo + b_co + b_va + b_lr + b_vp + b_ls + b_x + b_y);
    if (e != cudaSuccess) return e;
    DevSell D;
    size_t off = 0;
    D.slices = reinterpret_cast<SellSlice*>(buf);
    D.vout = reinterpret_cast<int32_t*>(buf + (off += b_sl));
    D.cols = reinterpret_cast<int32_t*>(buf + (off += b_vo));
    D.vals = buf + (off += b_co);
    D.lrows = reinterpret_cast<LongRow*>(buf + (off += b_va));
    D.vpart = buf + (off += b_lr);
    float* ls = b_ls ? reinterpret_cast<float*>(buf + (off += b_vp)) : nullptr;
    if (!b_ls) off += b_vp;
    void* x = buf + (off += b_ls);
    void* y = buf + off + b_x;
    D.vk = vk;
    D.lscale = ls;
    D.nslices = (int)H.slices.size();
    D.nlrows = (int)H.lrows.size();
    D.nlbig = (int)H.nbig;
    e = cudaMemsetAsync(x, 0, b_x + b_y, s);
    if (e == cudaSuccess)
      e = upload_sell(in_type, H, rp, ci, val, n, nnz, D, nullptr, ls, dcolmap, s);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int it = 0; it < 2 && e == cudaSuccess; ++it) e = launch_spmv(prec, D, x, y, false, s);
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (int it = 0; it < 5 && e == cudaSuccess; ++it) e = launch_spmv(prec, D, x, y, false, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(buf);
    if (e != cudaSuccess) return e;
    if (c == 0 || ms < best_ms) {
      best_ms = ms;
      *best = c;
    }
  }
  return cudaSuccess;
}

namespace {

// The plan stores the basis tile-major: tile t of column c at
// (t * (m + 1) + c) * TILE_R, so that a pass moves the columns of a tile with
// one bulk copy.  The SpMV reads the newest column from a contiguous copy.
int64_t basis_tstride(const te_plan* P) { return (int64_t)(P->m + 1) * TILE_R; }

PassArgs base_args(te_plan* P) {
  PassArgs a;
  memset(&a, 0, sizeof(a));
  a.V = at(P, P->W.V);
  a.Vmut = at(P, P->W.V);
  a.ld = P->n_pad;
  a.tstride = basis_tstride(P);
  a.cstride = TILE_R;
  a.xcopy = at(P, P->W.xcur);
  a.perm = P->dperm;
  a.n = P->n;
  a.m = P->m;
  a.K = P->K;
  a.seed = P->opt.seed;
  a.tol = breakdown_tol(P->prec);
  a.st = P->st;
  a.partials = at(P, P->W.partials);
  a.fin = FIN_NONE;
  a.stall = P->opt.stall_first_pass != 0;
  return a;
}

// profiling helpers: bracket a launch with two events when profiling is on
cudaError_t prof_begin(te_plan* P, cudaStream_t s) {
  if (!P->prof.on) return cudaSuccess;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return e;
  P->prof.ev.push_back(e0);
  P->prof.ev.push_back(e1);
  return cudaEventRecord(e0, s);
}
cudaError_t prof_end(te_plan* P, cudaStream_t s, int kind, double bytes) {
  if (!P->prof.on) return cudaSuccess;
  P->prof.kind.push_back(kind);
  P->prof.bytes.push_back(bytes);
  return cudaEventRecord(P->prof.ev.back(), s);
}

double pass_bytes(te_plan* P, int mode, const PassArgs& a) {
  const double n = (double)P->n, sb = (double)basis_elt(P->prec);
  const double vcols = (double)a.nb * n * sb;
  switch (mode) {
    case MODE_DOT: return vcols + n * 8.0;
    case MODE_AXPY_DOT: return vcols + 2.0 * n * 8.0;
    case MODE_AXPY_STORE: return vcols + n * 8.0 + n * sb;
    case MODE_DCGS_DOT: return vcols + n * 8.0;
    case MODE_DCGS_UPDATE: return vcols + n * 8.0 + 2.0 * n * sb;
    default: return vcols + n * 8.0 * (double)P->K;
  }
}

cudaError_t pass(te_plan* P, int mode, const PassArgs& a, cudaStream_t s) {
  const PassLaunch& L = mode == MODE_DOT           ? P->Ldot
                        : mode == MODE_AXPY_DOT    ? P->Laxd
                        : mode == MODE_AXPY_STORE  ? P->Lsto
                        : mode == MODE_DCGS_DOT    ? P->Lddot
                        : mode == MODE_DCGS_UPDATE ? P->Ldupd
                                                   : P->Lritz;
  P->nkernels++;
  cudaError_t e = prof_begin(P, s);
  if (e != cudaSuccess) return e;
  e = launch_pass(P->prec, mode, a, L, s);
  if (e != cudaSuccess) return e;
  int kind = (mode == MODE_DOT || mode == MODE_DCGS_DOT)            ? TE_KIND_DOT
             : mode == MODE_AXPY_DOT                                  ? TE_KIND_AXPY_DOT
             : (mode == MODE_AXPY_STORE || mode == MODE_DCGS_UPDATE) ? TE_KIND_AXPY_STORE
                                                                      : TE_KIND_RITZ;
  if (a.only_on_restart) kind = TE_KIND_RESTART;
  if (a.fin == FIN_STORE_INIT) kind = TE_KIND_OTHER;
  return prof_end(P, s, kind, a.only_on_restart ? 0.0 : pass_bytes(P, mode, a));
}

// y = M x for the solve.  A streamed matrix: fork the copy stream, then per
// row block b (device buffer b % 2): the copy waits until the SpMV of block
// b - 2 has released the buffer, the SpMV of block b waits for its copy; the
// cut-row finaliser runs once all blocks are done.  The same sequence is
// captured into the plan's graph (event record / wait become graph edges).
cudaError_t enqueue_spmv(te_plan* P, const void* x, void* y, bool out_f64, cudaStream_t s) {
  if (!P->streaming) {
    P->nkernels += 1 + (P->sell.nlrows > 0 ? 1 : 0);
    return launch_spmv(P->prec, P->sell, x, y, out_f64, s);
  }
  cudaError_t e;
  const size_t elt = elt_of(P->vk);
  int32_t* dcols = static_cast<int32_t*>(at(P, P->W.scols));
  char* dvals = static_cast<char*>(at(P, P->W.svals));
  if ((e = cudaEventRecord(P->ev_fork, s)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(P->cs, P->ev_fork, 0)) != cudaSuccess) return e;
  for (size_t b = 0; b < P->blocks.size(); ++b) {
    const te_plan::Block& B = P->blocks[b];
    const int u = (int)(b & 1);
    int32_t* bc = dcols + (size_t)u * P->cap_entries;
    char* bv = dvals + (size_t)u * P->cap_entries * elt;
    if (b >= 2 && (e = cudaStreamWaitEvent(P->cs, P->ev_free[u], 0)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(bc, P->hcols + B.ebase, (size_t)B.entries * 4,
                             cudaMemcpyHostToDevice, P->cs)) != cudaSuccess)
      return e;
    if ((e = cudaMemcpyAsync(bv, static_cast<char*>(P->hvals) + (size_t)B.ebase * elt,
                             (size_t)B.entries * elt, cudaMemcpyHostToDevice, P->cs)) !=
        cudaSuccess)
      return e;
    if ((e = cudaEventRecord(P->ev_ready[u], P->cs)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s, P->ev_ready[u], 0)) != cudaSuccess) return e;
    DevSell V = P->sell;
    V.slices = P->sell.slices + B.first_slice;
    V.vout = P->sell.vout + (size_t)B.first_slice * SELL_C;
    V.nslices = B.nslices;
    V.nlrows = 0;
    V.nlbig = 0;
    V.cols = bc;
    V.vals = bv;
    V.ebase = B.ebase;
    P->nkernels += 1;
    if ((e = launch_spmv(P->prec, V, x, y, out_f64, s)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(P->ev_free[u], s)) != cudaSuccess) return e;
  }
  if ((e = cudaEventRecord(P->ev_join, P->cs)) != cudaSuccess) return e;
  if ((e = cudaStreamWaitEvent(s, P->ev_join, 0)) != cudaSuccess) return e;
  if (P->sell.nlrows > 0) {
    DevSell V = P->sell;
    V.nslices = 0;  // the finaliser alone
    P->nkernels += 1;
    if ((e = launch_spmv(P->prec, V, x, y, out_f64, s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Enqueue the Lanczos phase (Algorithm 1): init + m steps.
cudaError_t enqueue_lanczos(te_plan* P, cudaStream_t s) {
  cudaError_t e;
  // v_1 = normalised start vector (stored unnormalised, scale s_0)
  {
    PassArgs a = base_args(P);
    a.nb = 0;
    a.col_out = 0;
    a.xsrc = X_V1;
    a.fin = FIN_STORE_INIT;
    a.step = 0;
    if ((e = pass(P, MODE_AXPY_STORE, a, s)) != cudaSuccess) return e;
  }
  for (int i = 0; i < P->m; ++i) {
    const void* xi = at(P, P->W.xcur);  // column i, written by the pass that formed it
    if ((e = prof_begin(P, s)) != cudaSuccess) return e;
    e = enqueue_spmv(P, xi, at(P, P->W.ytil), false, s);
    if (e != cudaSuccess) return e;
    {
      const double n = (double)P->n, nnz = (double)P->nnz;
      const double bytes = nnz * (4.0 + (double)elt_of(P->vk)) + 8.0 * (n + 1.0) +
                           n * (double)basis_elt(P->prec) + n * 8.0 +
                           (P->vk == TE_FP8_E4M3 ? 4.0 * n : 0.0);
      if ((e = prof_end(P, s, TE_KIND_SPMV, bytes)) != cudaSuccess) return e;
    }
    PassArgs a = base_args(P);
    a.step = i;
    a.xsrc = X_VEC;
    a.xvec = at(P, P->W.ytil);
    if (P->delayed) {
      // full reorthogonalisation with the candidate's second sweep delayed:
      // the SpMV ran on candidate column i; one pass takes the dots of every
      // column with y and with the candidate, one pass finishes column i and
      // forms the next candidate (column i+1)
      a.nb = i + 1;
      a.fin = FIN_DCGS_DOT;
      a.cand = at(P, P->W.xcur);  // the candidate lives in the contiguous copy
      if ((e = pass(P, MODE_DCGS_DOT, a, s)) != cudaSuccess) return e;
      a.col_out = i + 1;
      a.col_fix = i;
      a.fin = FIN_DCGS_UPDATE;
      if ((e = pass(P, MODE_DCGS_UPDATE, a, s)) != cudaSuccess) return e;
    } else if (P->noreorth) {
      // three-term recurrence only: alpha_i from v_i alone, then
      // w / s_i = ytilde - alpha_i stored_i - (beta_i s_{i-1} / s_i) stored_{i-1}
      a.col0 = i;
      a.nb = 1;
      a.fin = FIN_DOT_NOREORTH;
      if ((e = pass(P, MODE_DOT, a, s)) != cudaSuccess) return e;
      a.col0 = i > 0 ? i - 1 : 0;
      a.nb = i > 0 ? 2 : 1;
      a.exact_tail = a.nb;
      a.col_out = i + 1;
      a.fin = FIN_STORE_NOREORTH;
      if ((e = pass(P, MODE_AXPY_STORE, a, s)) != cudaSuccess) return e;
    } else {
      a.nb = i + 1;
      a.fin = FIN_DOT_STEP;
      if ((e = pass(P, MODE_DOT, a, s)) != cudaSuccess) return e;
      a.wout = at(P, P->W.w);
      a.fin = FIN_AXPYDOT_STEP;
      a.exact_tail = 2;  // alpha_i v_i and beta_i v_{i-1}
      if ((e = pass(P, MODE_AXPY_DOT, a, s)) != cudaSuccess) return e;
      a.xvec = at(P, P->W.w);
      a.col_out = i + 1;
      a.fin = FIN_STORE_STEP;
      a.exact_tail = 0;  // second-sweep coefficients are all small
      if ((e = pass(P, MODE_AXPY_STORE, a, s)) != cudaSuccess) return e;
    }
    if (i + 1 < P->m) {
      // restart from a fresh random vector if this step broke down
      PassArgs r = base_args(P);
      r.nb = i + 1;
      r.exact_tail = i + 1;  // a random vector: every coefficient may be large
      r.step = i;
      r.only_on_restart = 1;
      r.xsrc = X_RANDOM;
      r.fin = FIN_DOT_RESTART;
      if ((e = pass(P, MODE_DOT, r, s)) != cudaSuccess) return e;
      r.wout = at(P, P->W.w);
      r.fin = FIN_AXPYDOT;
      if ((e = pass(P, MODE_AXPY_DOT, r, s)) != cudaSuccess) return e;
      r.xsrc = X_VEC;
      r.xvec = at(P, P->W.w);
      r.col_out = i + 1;
      r.fin = FIN_STORE_RESTART;
      if ((e = pass(P, MODE_AXPY_STORE, r, s)) != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

cudaError_t enqueue_solve(te_plan* P, cudaStream_t s) {
  P->nkernels = 0;
  cudaError_t e = enqueue_lanczos(P, s);
  if (e != cudaSuccess) return e;
  JacobiArgs j;
  memset(&j, 0, sizeof(j));
  j.alpha = P->st->alpha;
  j.beta = P->st->beta;
  j.s = P->st->s;
  j.m = P->m;
  j.K = P->K;
  j.which = P->opt.which;
  j.theta_out = P->st->theta_sel;
  j.C_out = P->st->C;
  j.resid_out = P->st->resid_est;
  j.st = P->st;
  P->nkernels++;
  if ((e = prof_begin(P, s)) != cudaSuccess) return e;
  if ((e = launch_jacobi(j, s)) != cudaSuccess) return e;
  if ((e = prof_end(P, s, TE_KIND_JACOBI, 0.0)) != cudaSuccess) return e;
  PassArgs a = base_args(P);
  a.nb = P->m;
  a.fin = FIN_NONE;
  if (P->reorder && !P->refine) a.urows = P->ubase;  // stored by rows, gathered below
  if ((e = pass(P, MODE_RITZ, a, s)) != cudaSuccess) return e;
  const int rgrid = refine_grid(P->num_sms);
  if (!P->refine) {
    if (!P->reorder) return cudaSuccess;
    // the Ritz vectors of the relabelled rows, back in the caller's order
    P->nkernels++;
    if ((e = prof_begin(P, s)) != cudaSuccess) return e;
    if ((e = launch_copy_out_rows(P->st, P->ubase, P->n, P->K, P->diperm, rgrid * 4, s)) !=
        cudaSuccess)
      return e;
    return prof_end(P, s, TE_KIND_RITZ, (16.0 + 4.0 / P->K) * (double)P->n * P->K);
  }
  // binary64 Rayleigh-quotient refinement: y = M u_k, then the reduction
  double* y = static_cast<double*>(at(P, P->W.ytil));
  double* part = static_cast<double*>(at(P, P->W.partials));
  for (int k = 0; k < P->K; ++k) {
    P->nkernels += 2 + (P->sell64.nlrows > 0 ? 1 : 0);
    if ((e = prof_begin(P, s)) != cudaSuccess) return e;
    e = launch_spmv(PREC_DDD, P->sell64, P->ubase + (size_t)k * P->n, y, true, s);
    if (e != cudaSuccess) return e;
    if ((e = launch_refine(P->st, y, P->n, k, part, rgrid, s)) != cudaSuccess) return e;
    const double n = (double)P->n, nnz = (double)P->nnz;
    if ((e = prof_end(P, s, TE_KIND_REFINE, nnz * 12.0 + 8.0 * (n + 1.0) + 8.0 * n * 3.0)) !=
        cudaSuccess)
      return e;
  }
  // the refined vectors stay the Ritz vectors: hand them to the caller's buffer
  P->nkernels++;
  if ((e = prof_begin(P, s)) != cudaSuccess) return e;
  e = P->reorder ? launch_copy_out_perm(P->st, P->ubase, P->n, P->K, P->diperm, rgrid * 4, s)
                 : launch_copy_out(P->st, P->ubase, (size_t)P->n * P->K, rgrid * 4, s);
  if (e != cudaSuccess) return e;
  return prof_end(P, s, TE_KIND_REFINE, 16.0 * (double)P->n * P->K);
}

__global__ void solve_begin_kernel(LzState* st, const double* v1, double* eigvecs,
                                   double* eigvals, double* plan_vecs) {
  st->v1 = v1;
  // with refinement (or relabelled rows) the Ritz vectors go to the plan's
  // buffer (the refinement SpMVs read them at a fixed address) and are
  // copied out at the end
  st->eigvecs = plan_vecs ? plan_vecs : eigvecs;
  st->eigvecs_user = plan_vecs ? eigvecs : nullptr;
  st->eigvals_out = eigvals;
  st->status = 0;
  st->restarts = 0;
  st->restart_flag = 0;
  st->sweeps = 0;
  st->ticket = 0;
}

}  // namespace

cudaError_t te::launch_solve_begin(LzState* st, const double* v1, double* eigvecs, double* eigvals,
                                   double* plan_vecs, cudaStream_t s) {
  solve_begin_kernel<<<1, 1, 0, s>>>(st, v1, eigvecs, eigvals, plan_vecs);
  return cudaGetLastError();
}
double te::breakdown_tolerance(int prec) { return breakdown_tol(prec); }

namespace {

te_status plan_begin(te_plan* P, const double* v1, double* eigvecs_dev, double* eigvals_dev,
                     cudaStream_t s) {
  // refinement and relabelled rows keep the Ritz vectors in the plan's own
  // buffer (copied out to the caller's at the end)
  const bool own = P->refine || (P->reorder && eigvecs_dev != nullptr);
  solve_begin_kernel<<<1, 1, 0, s>>>(P->st, v1 ? v1 : P->opt.v1, eigvecs_dev, eigvals_dev,
                                     own ? P->ubase : nullptr);
  TE_CK(cudaGetLastError(), "solve_begin launch");
  return TE_OK;
}

}  // namespace

extern "C" {

void te_default_options(te_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->seed = 0;
  opt->v1 = nullptr;
  opt->which = TE_WHICH_LARGEST_MAGNITUDE;
  opt->use_graph = 1;
  opt->device_budget_bytes = 0;
}

const char* te_last_error(void) { return g_err.c_str(); }

const char* te_status_string(te_status s) {
  switch (s) {
    case TE_OK: return "TE_OK";
    case TE_ERR_INVALID_ARG: return "TE_ERR_INVALID_ARG";
    case TE_ERR_OUT_OF_MEMORY: return "TE_ERR_OUT_OF_MEMORY";
    case TE_ERR_CUDA: return "TE_ERR_CUDA";
    case TE_ERR_BREAKDOWN: return "TE_ERR_BREAKDOWN";
    case TE_ERR_NOT_CONVERGED: return "TE_ERR_NOT_CONVERGED";
    case TE_ERR_TIMEOUT: return "TE_ERR_TIMEOUT";
    case TE_ERR_UNSUPPORTED: return "TE_ERR_UNSUPPORTED";
  }
  return "TE_ERR_UNKNOWN";
}

size_t te_workspace_bytes(const te_csr* A, int32_t K, int32_t krylov_steps, te_precision p) {
  if (check_args(A, K, krylov_steps, p) != TE_OK) return 0;
  const int prec = prec_of(p);
  // an upper bound of the SELL layout without reading the matrix: every
  // window pads at most SELL_C * SELL_VMAX entries to sort order and one
  // partial slice
  const size_t windows = (size_t)((A->n + SELL_WINDOW - 1) / SELL_WINDOW);
  SellSizes z;
  z.pieces = (size_t)(A->nnz / SELL_VMAX + 1);
  z.slices = (size_t)((A->n + z.pieces) / SELL_C + windows + 1);
  z.entries = (size_t)A->nnz + windows * 2 * SELL_C * SELL_VMAX;
  z.lrows = (size_t)(A->nnz / SELL_VMAX + 1);
  Work w = layout(prec, p.values, pad_rows(A->n), krylov_steps, 1024, z);
  return w.total;
}

void te_plan_destroy(te_plan* P) {
  if (!P) return;
  for (cudaEvent_t e : {P->ev_ready[0], P->ev_ready[1], P->ev_free[0], P->ev_free[1], P->ev_fork,
                        P->ev_join})
    if (e) cudaEventDestroy(e);
  if (P->cs) cudaStreamDestroy(P->cs);
  if (P->hcols) cudaFreeHost(P->hcols);
  if (P->hvals) cudaFreeHost(P->hvals);
  if (P->gexec) cudaGraphExecDestroy(P->gexec);
  if (P->cap) cudaStreamDestroy(P->cap);
  if (P->work) dev_free(P->work);
  if (P->owned_csr) dev_free(P->owned_csr);
  if (P->hres) cudaFreeHost(P->hres);
  delete P;
}

te_status te_plan_create(const te_csr* A, int32_t K, int32_t krylov_steps, te_precision p,
                         const te_options* opt_in, void* stream, te_plan** out) {
  if (!out) return fail(TE_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  te_status st0 = check_args(A, K, krylov_steps, p);
  if (st0 != TE_OK) return st0;
  te_options opt;
  if (opt_in) opt = *opt_in;
  else te_default_options(&opt);
  if (opt.which != TE_WHICH_LARGEST_MAGNITUDE && opt.which != TE_WHICH_LARGEST_ALGEBRAIC)
    return fail(TE_ERR_INVALID_ARG, "which must be TE_WHICH_*");
  if (opt.reorth != TE_REORTH_FULL && opt.reorth != TE_REORTH_NONE &&
      opt.reorth != TE_REORTH_DELAYED)
    return fail(TE_ERR_INVALID_ARG, "reorth must be TE_REORTH_FULL, _NONE or _DELAYED");
  if (opt.refine != 0 && opt.refine != 1) return fail(TE_ERR_INVALID_ARG, "refine must be 0 or 1");
  if (opt.order != TE_ORDER_KEEP && opt.order != TE_ORDER_DEGREE)
    return fail(TE_ERR_INVALID_ARG, "order must be TE_ORDER_KEEP or TE_ORDER_DEGREE");
  if (opt.stall_first_pass != 0 && opt.stall_first_pass != 1)
    return fail(TE_ERR_INVALID_ARG, "stall_first_pass must be 0 or 1");
  const int in_type = A->values_f64 ? TE_F64 : p.values;
  if (opt.refine && in_type != TE_F64)
    return fail(TE_ERR_INVALID_ARG,
                "refinement needs the binary64 values (values_f64 = 1, or a binary64 form)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  if (prepare_kernels() != cudaSuccess) return cuda_fail(g_prep_err, "kernel set-up");
  if (A->where == TE_DEVICE &&
      !(aligned16(A->row_ptr) && aligned16(A->col_idx) && aligned16(A->values)))
    return fail(TE_ERR_INVALID_ARG, "device CSR arrays must be 16-byte aligned");

  te_plan* P = new te_plan();
  struct Guard {
    te_plan*& p;
    bool keep = false;
    ~Guard() {
      if (!keep) te_plan_destroy(p);
    }
  } guard{P};

  P->prec = prec_of(p);
  P->n = A->n;
  P->nnz = A->nnz;
  P->n_pad = pad_rows(A->n);
  P->K = K;
  P->m = krylov_steps;
  P->opt = opt;
  P->in_type = in_type;
  P->vk = p.values;
  P->refine = opt.refine != 0;
  P->noreorth = opt.reorth == TE_REORTH_NONE;
  P->delayed = opt.reorth == TE_REORTH_DELAYED;
  P->reorder = opt.order == TE_ORDER_DEGREE;
  TE_CK(cudaGetDevice(&P->dev), "cudaGetDevice");
  TE_CK(cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->dev),
        "device attribute");

  // a host matrix that stays resident: its copy to the device starts now and
  // overlaps the analysis below.  The row pointers come first on `s`; the
  // columns and values follow on a second stream, which `s` waits for only
  // where they are read (the column check and the layout fill).
  struct SideCopy {
    cudaStream_t cs = nullptr;
    cudaEvent_t cols_done = nullptr;  // the column indices have arrived
    cudaEvent_t done = nullptr;       // columns and values have arrived
    ~SideCopy() {
      if (cs) {
        cudaStreamSynchronize(cs);
        cudaStreamDestroy(cs);
      }
      if (cols_done) cudaEventDestroy(cols_done);
      if (done) cudaEventDestroy(done);
    }
  } side;
  if (A->where == TE_HOST && opt.matrix_budget_bytes == 0) {
    const size_t e_in = in_type == TE_F64 ? 8 : 4;
    const size_t brp = al256(sizeof(int64_t) * (A->n + 1)), bci = al256(sizeof(int32_t) * A->nnz);
    TE_CK(dev_alloc(&P->owned_csr, brp + bci + al256(e_in * A->nnz)), "allocate device CSR");
    char* b = static_cast<char*>(P->owned_csr);
    TE_CK(cudaMemcpyAsync(b, A->row_ptr, sizeof(int64_t) * (A->n + 1), cudaMemcpyHostToDevice, s),
          "copy row_ptr");
    if (A->nnz > 0) {
      TE_CK(cudaStreamCreateWithFlags(&side.cs, cudaStreamNonBlocking), "create copy stream");
      TE_CK(cudaEventCreateWithFlags(&side.done, cudaEventDisableTiming), "create event");
      TE_CK(cudaEventCreateWithFlags(&side.cols_done, cudaEventDisableTiming), "create event");
      TE_CK(cudaMemcpyAsync(b + brp, A->col_idx, sizeof(int32_t) * A->nnz, cudaMemcpyHostToDevice,
                            side.cs),
            "copy col_idx");
      TE_CK(cudaEventRecord(side.cols_done, side.cs), "record");
      TE_CK(cudaMemcpyAsync(b + brp + bci, A->values, e_in * A->nnz, cudaMemcpyHostToDevice,
                            side.cs),
            "copy values");
      TE_CK(cudaEventRecord(side.done, side.cs), "record");
    }
    P->rp = reinterpret_cast<const int64_t*>(b);
    P->ci = reinterpret_cast<const int32_t*>(b + brp);
    P->val = b + brp + bci;
  }

  // The SpMV layout (and the row order) is built by kernels from the device
  // row pointers when the matrix ends up resident with the default layout;
  // a streamed matrix or the autotuner's trial layouts use the host build.
  const bool dev_build = !opt.autotune && (A->where == TE_DEVICE || opt.matrix_budget_bytes == 0) &&
                         dev_layout_fits(A->n, SELL_WINDOW, SELL_VMAX);
  DevLayout DL;
  char* dtmp = nullptr;  // device build: the row order and the placed rows' first entries
  struct TmpFree {
    char*& p;
    ~TmpFree() {
      if (p) dev_free(p);
    }
  } dtmp_guard{dtmp};
  int32_t *dperm_t = nullptr, *diperm_t = nullptr, *dlen_t = nullptr;
  int64_t* dsrc_t = nullptr;
  int64_t dtot[4] = {0, 0, 0, 0};
  if (dev_build) {
    const int64_t* rpd = A->where == TE_DEVICE ? A->row_ptr : P->rp;
    std::string derr;
    cudaError_t e = DL.count(rpd, A->n, A->nnz, SELL_WINDOW, SELL_VMAX, P->reorder, s, derr);
    if (e == cudaErrorInvalidValue && !derr.empty())
      return fail(TE_ERR_INVALID_ARG, "malformed CSR: " + derr);
    TE_CK(e, "row order on the device");
    if (P->reorder) {
      const size_t nn = (size_t)A->n;
      TE_CK(dev_alloc(&dtmp, nn * (4 + 4 + 4) + al256(nn * 8) + 256), "allocate the row order");
      dsrc_t = reinterpret_cast<int64_t*>(dtmp);
      dperm_t = reinterpret_cast<int32_t*>(dtmp + al256(nn * 8));
      diperm_t = dperm_t + nn;
      dlen_t = diperm_t + nn;
      TE_CK(DL.order(dperm_t, diperm_t, dsrc_t, dlen_t, s), "row order on the device");
    }
    TE_CK(DL.windows(s, dtot), "layout counts on the device");
  }
  // row pointers on the host for the partition
  hvec<int64_t> rp_host;
  const int64_t* rph = A->row_ptr;
  if (A->where == TE_DEVICE && !dev_build) {
    rp_host.resize((size_t)A->n + 1);
    TE_CK(cudaMemcpyAsync(rp_host.data(), A->row_ptr, sizeof(int64_t) * (A->n + 1),
                          cudaMemcpyDeviceToHost, s),
          "copy row_ptr to host");
    TE_CK(cudaStreamSynchronize(s), "sync");
    rph = rp_host.data();
  }
  SellHost sell;
  std::string perr;
  // relabelled rows: the solver's row r is the caller's row hperm[r]
  hvec<int32_t> hperm, hiperm, hlen;
  hvec<int64_t> hsrc;
  RowOrder ord{nullptr, nullptr, nullptr};
  if (P->reorder && !dev_build) {
    if (!rows_valid(rph, A->n, A->nnz, perr))
      return fail(TE_ERR_INVALID_ARG, "malformed CSR: " + perr);
    hperm.resize((size_t)A->n);
    hiperm.resize((size_t)A->n);
    hsrc.resize((size_t)A->n);
    hlen.resize((size_t)A->n);
    degree_order(rph, A->n, hperm.data(), hiperm.data(), hsrc.data(), hlen.data());
    ord = RowOrder{hperm.data(), hsrc.data(), hlen.data()};
  }
  const RowOrder* hp = P->reorder ? &ord : nullptr;
  if (!dev_build && !make_sell(rph, A->n, A->nnz, sell, perr, SELL_WINDOW, SELL_VMAX, hp))
    return fail(TE_ERR_INVALID_ARG, "malformed CSR: " + perr);
  // the layout's sizes, from either build (the autotuner may rebuild the host
  // layout below and updates them)
  int64_t l_slices = dev_build ? dtot[0] : (int64_t)sell.slices.size();
  int64_t l_entries = dev_build ? dtot[1] : sell.entries;
  int64_t l_pieces = dev_build ? dtot[2] : sell.pieces;
  int64_t l_lrows = dev_build ? dtot[3] : (int64_t)sell.lrows.size();

  // launch shapes of the basis passes
  TE_CK(pass_config(P->prec, MODE_DOT, P->m, P->K, P->num_sms, P->Ldot), "configure dot pass");
  TE_CK(pass_config(P->prec, MODE_AXPY_DOT, P->m, P->K, P->num_sms, P->Laxd),
        "configure axpy pass");
  TE_CK(pass_config(P->prec, MODE_AXPY_STORE, P->m, P->K, P->num_sms, P->Lsto),
        "configure store pass");
  TE_CK(pass_config(P->prec, MODE_RITZ, P->m, P->K, P->num_sms, P->Lritz),
        "configure ritz pass");
  if (P->delayed) {
    TE_CK(pass_config(P->prec, MODE_DCGS_DOT, P->m, P->K, P->num_sms, P->Lddot),
          "configure dot pass");
    TE_CK(pass_config(P->prec, MODE_DCGS_UPDATE, P->m, P->K, P->num_sms, P->Ldupd),
          "configure update pass");
  }
  // a small basis has fewer tiles than the persistent grid has CTAs: one CTA
  // per tile then (idle CTAs would only lengthen the last CTA's reduction)
  const int tiles = (int)std::min<int64_t>(P->n_pad / TILE_R, INT32_MAX);
  for (PassLaunch* L : {&P->Ldot, &P->Laxd, &P->Lsto, &P->Lritz, &P->Lddot, &P->Ldupd})
    if (L->grid > tiles) L->grid = std::max(tiles, 1);
  const int grid = std::max(std::max(P->Ldot.grid, P->Laxd.grid),
                            std::max(P->Lsto.grid, P->Lritz.grid));

  // a matrix whose layout exceeds matrix_budget_bytes stays in pinned host
  // memory and is streamed in row blocks (whole slices) of at most half the
  // budget each
  const size_t velt = elt_of(P->vk);
  P->streaming = opt.matrix_budget_bytes > 0 &&
                 (size_t)l_entries * (4 + velt) > opt.matrix_budget_bytes;
  if (P->streaming) {
    if (A->where != TE_HOST)
      return fail(TE_ERR_OUT_OF_MEMORY,
                  "the matrix layout exceeds matrix_budget_bytes; only a TE_HOST matrix can be "
                  "streamed");
    if (P->vk != TE_F64 && P->vk != TE_F32)
      return fail(TE_ERR_UNSUPPORTED, "a streamed matrix holds binary64 or binary32 values");
    if (P->refine)
      return fail(TE_ERR_UNSUPPORTED, "refinement is not available with a streamed matrix");
    P->cap_entries = (int64_t)(opt.matrix_budget_bytes / 2 / (4 + velt)) / 64 * 64;
    te_plan::Block cur{0, 0, 0, 0};
    for (size_t i = 0; i < sell.slices.size(); ++i) {
      const int64_t ent = (int64_t)SELL_C * sell.slices[i].len;
      if (ent > P->cap_entries)
        return fail(TE_ERR_INVALID_ARG, "matrix_budget_bytes is too small to hold one slice");
      if (cur.entries + ent > P->cap_entries) {
        P->blocks.push_back(cur);
        cur = te_plan::Block{(int)i, 0, sell.slices[i].base, 0};
      }
      cur.nslices += 1;
      cur.entries += ent;
    }
    if (cur.nslices > 0) P->blocks.push_back(cur);
  }

  if (opt.autotune && !P->streaming) {
    // the device CSR the candidates are built from (a host matrix is copied
    // for the trials); its columns are checked before any SpMV reads them
    if (side.done) TE_CK(cudaStreamWaitEvent(s, side.done, 0), "wait for the matrix copy");
    const size_t in_elt = in_type == TE_F64 ? 8 : 4;
    const int64_t* drp = A->row_ptr;
    const int32_t* dci = A->col_idx;
    const void* dval = A->values;
    char* tmp = nullptr;
    if (P->owned_csr) {
      drp = P->rp;
      dci = P->ci;
      dval = P->val;
    } else if (A->where == TE_HOST) {
      const size_t brp = al256(sizeof(int64_t) * (A->n + 1)), bci = al256(4 * (size_t)A->nnz);
      TE_CK(dev_alloc(&tmp, brp + bci + in_elt * (size_t)A->nnz + 256), "allocate tuning CSR");
      TE_CK(cudaMemcpyAsync(tmp, A->row_ptr, sizeof(int64_t) * (A->n + 1), cudaMemcpyHostToDevice,
                            s),
            "copy row_ptr");
      TE_CK(cudaMemcpyAsync(tmp + brp, A->col_idx, 4 * (size_t)A->nnz, cudaMemcpyHostToDevice, s),
            "copy col_idx");
      TE_CK(cudaMemcpyAsync(tmp + brp + bci, A->values, in_elt * (size_t)A->nnz,
                            cudaMemcpyHostToDevice, s),
            "copy values");
      drp = reinterpret_cast<const int64_t*>(tmp);
      dci = reinterpret_cast<const int32_t*>(tmp + brp);
      dval = tmp + brp + bci;
    }
    int* flag = nullptr;
    int32_t* tmap = nullptr;  // the column relabelling, for the trial layouts
    cudaError_t e = dev_alloc(&flag, sizeof(int));
    if (e == cudaSuccess && P->reorder) e = dev_alloc(&tmap, sizeof(int32_t) * A->n);
    if (e == cudaSuccess && P->reorder)
      e = cudaMemcpyAsync(tmap, hiperm.data(), sizeof(int32_t) * A->n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_validate_cols(dci, A->nnz, A->n, flag, s);
    int hflag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (flag) dev_free(flag);
    int best = 0;
    if (e == cudaSuccess && !hflag)
      e = autotune_layout(P->prec, P->vk, in_type, rph, drp, dci, dval, A->n, A->nnz, hp, tmap, s,
                          &best);
    if (tmp) dev_free(tmp);
    if (tmap) dev_free(tmap);
    if (e != cudaSuccess) return cuda_fail(e, "autotune the SpMV layout");
    if (hflag) return fail(TE_ERR_INVALID_ARG, "malformed CSR: a column index is outside [0, n)");
    P->sell_window = TUNE_WINDOW[best];
    P->sell_vmax = TUNE_VMAX[best];
    if (best != 0 && !make_sell(rph, A->n, A->nnz, sell, perr, P->sell_window, P->sell_vmax, hp))
      return fail(TE_ERR_INVALID_ARG, "malformed CSR: " + perr);
    l_slices = (int64_t)sell.slices.size();
    l_entries = sell.entries;
    l_pieces = sell.pieces;
    l_lrows = (int64_t)sell.lrows.size();
  }

  SellSizes zs;
  zs.slices = (size_t)l_slices;
  zs.entries = P->streaming ? (size_t)(2 * P->cap_entries) : (size_t)l_entries;
  zs.lrows = (size_t)l_lrows;
  zs.pieces = (size_t)l_pieces;
  P->W = layout(P->prec, P->vk, P->n_pad, P->m, grid, zs, P->refine, P->n, P->K, P->reorder);
  const size_t in_elt = in_type == TE_F64 ? 8 : 4;
  size_t csr_bytes = 0;
  if (A->where == TE_HOST && !P->streaming)
    csr_bytes = al256(sizeof(int64_t) * (A->n + 1)) + al256(sizeof(int32_t) * A->nnz) +
                al256(in_elt * A->nnz);
  if (opt.device_budget_bytes > 0 && P->W.total + csr_bytes > opt.device_budget_bytes)
    return fail(TE_ERR_OUT_OF_MEMORY, "work memory exceeds device_budget_bytes");

  TE_CK(dev_alloc(&P->work, P->W.total), "allocate work memory");
  TE_CK(cudaMallocHost(&P->hres, sizeof(te_plan::HostRes)), "allocate pinned result buffer");
  P->st = static_cast<LzState*>(at(P, P->W.st));

  if (P->streaming) {
    // the host layout, built once; the solve copies it block by block
    TE_CK(cudaHostAlloc(reinterpret_cast<void**>(&P->hcols),
                        std::max<size_t>((size_t)sell.entries, 1) * 4, cudaHostAllocDefault),
          "allocate pinned layout");
    TE_CK(cudaHostAlloc(&P->hvals, std::max<size_t>((size_t)sell.entries, 1) * velt,
                        cudaHostAllocDefault),
          "allocate pinned layout");
    if (!build_sell_host(sell, A->col_idx, A->values, in_type, P->vk, A->n,
                         P->reorder ? hiperm.data() : nullptr, P->hcols, P->hvals))
      return fail(TE_ERR_INVALID_ARG, "malformed CSR: a column index is outside [0, n)");
    TE_CK(cudaStreamCreateWithFlags(&P->cs, cudaStreamNonBlocking), "create copy stream");
    for (cudaEvent_t* e : {&P->ev_ready[0], &P->ev_ready[1], &P->ev_free[0], &P->ev_free[1],
                           &P->ev_fork, &P->ev_join})
      TE_CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming), "create event");
  } else if (P->owned_csr) {
    // copied at the start
  } else if (A->where == TE_HOST) {
    TE_CK(dev_alloc(&P->owned_csr, csr_bytes), "allocate device CSR");
    char* b = static_cast<char*>(P->owned_csr);
    int64_t* drp = reinterpret_cast<int64_t*>(b);
    int32_t* dci = reinterpret_cast<int32_t*>(b + al256(sizeof(int64_t) * (A->n + 1)));
    void* dval = b + al256(sizeof(int64_t) * (A->n + 1)) + al256(sizeof(int32_t) * A->nnz);
    TE_CK(cudaMemcpyAsync(drp, A->row_ptr, sizeof(int64_t) * (A->n + 1),
                          cudaMemcpyHostToDevice, s),
          "copy row_ptr");
    if (A->nnz > 0) {
      TE_CK(cudaMemcpyAsync(dci, A->col_idx, sizeof(int32_t) * A->nnz, cudaMemcpyHostToDevice,
                            s),
            "copy col_idx");
      TE_CK(cudaMemcpyAsync(dval, A->values, in_elt * A->nnz, cudaMemcpyHostToDevice, s),
            "copy values");
    }
    P->rp = drp;
    P->ci = dci;
    P->val = dval;
  } else {
    P->rp = A->row_ptr;
    P->ci = A->col_idx;
    P->val = A->values;
  }

  // zero the solver vectors and state (the padded rows of V, y and w and the
  // empty rows of y must stay zero); the SELL arrays are written below
  TE_CK(cudaMemsetAsync(P->work, 0, P->W.slices, s), "clear work memory");
  if (opt.stall_first_pass) {
    // test hook: arm the stall of the first basis pass (solve_begin keeps it)
    static const int one = 1;
    TE_CK(cudaMemcpyAsync(&P->st->stall_armed, &one, sizeof(int), cudaMemcpyHostToDevice, s),
          "arm the stall hook");
    TE_CK(cudaStreamSynchronize(s), "arm the stall hook");
  }
  // A host matrix still arriving with a device-built layout: the layout's
  // emission runs during the copy, the column check and the columns' fill
  // wait only for the column indices, the values' fill for the values.
  const bool arriving = dev_build && side.done != nullptr;
  int* dflag = static_cast<int*>(at(P, P->W.flag));
  if (!arriving && side.done) TE_CK(cudaStreamWaitEvent(s, side.done, 0), "wait for the matrix copy");
  if (!P->streaming && !arriving) {
    // column indices must lie in [0, n)
    TE_CK(cudaMemsetAsync(dflag, 0, sizeof(int), s), "clear flag");
    TE_CK(launch_validate_cols(P->ci, P->nnz, P->n, dflag, s), "validate columns");
    int hflag = 0;
    TE_CK(cudaMemcpyAsync(&hflag, dflag, sizeof(int), cudaMemcpyDeviceToHost, s), "read flag");
    TE_CK(cudaStreamSynchronize(s), "plan setup");
    if (hflag) return fail(TE_ERR_INVALID_ARG, "malformed CSR: a column index is outside [0, n)");
  }
  if (P->reorder) {
    P->dperm = static_cast<int32_t*>(at(P, P->W.perm));
    P->diperm = static_cast<int32_t*>(at(P, P->W.iperm));
    const cudaMemcpyKind k = dev_build ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    TE_CK(cudaMemcpyAsync(P->dperm, dev_build ? (const void*)dperm_t : (const void*)hperm.data(),
                          sizeof(int32_t) * A->n, k, s),
          "place the row order");
    TE_CK(cudaMemcpyAsync(P->diperm,
                          dev_build ? (const void*)diperm_t : (const void*)hiperm.data(),
                          sizeof(int32_t) * A->n, k, s),
          "place the row order");
    if (!dev_build) TE_CK(cudaStreamSynchronize(s), "place the row order");
  }
  // the SELL copy of the matrix that the solve streams
  P->sell.slices = static_cast<SellSlice*>(at(P, P->W.slices));
  P->sell.vout = static_cast<int32_t*>(at(P, P->W.vout));
  P->sell.cols = static_cast<int32_t*>(at(P, P->W.scols));
  P->sell.vals = at(P, P->W.svals);
  P->sell.lrows = static_cast<LongRow*>(at(P, P->W.lrows));
  P->sell.vpart = at(P, P->W.vpart);
  P->sell.nslices = (int)l_slices;
  P->sell.nlrows = (int)l_lrows;
  P->sell.nlbig = (int)sell.nbig;  // (the device build sets it below)
  void* vals64 = P->W.svals64 ? at(P, P->W.svals64) : nullptr;
  P->sell.vk = P->vk;
  P->sell.hot = P->reorder ? P->n : 0;  // the first columns are the most connected
  P->sell.lscale = P->W.lscale ? static_cast<const float*>(at(P, P->W.lscale)) : nullptr;
  if (P->streaming) {
    TE_CK(upload_meta(sell, P->sell, s), "upload the SELL layout");
  } else if (dev_build) {
    // the lane records and the slices come from the device build; the cut
    // rows are sorted there (most pieces first)
    const size_t lanes = (size_t)std::max<int64_t>(l_slices, 1) * SELL_C;
    const bool fp8 = P->vk == TE_FP8_E4M3;
    char* lt = nullptr;
    const size_t bytes = al256(lanes * 8) + al256(lanes * 4) + (fp8 ? al256(lanes * 4) : 0) +
                         al256((size_t)std::max<int64_t>(l_lrows, 1) * sizeof(LongRow));
    TE_CK(dev_alloc(&lt, bytes), "allocate the lane records");
    struct LtFree {
      char* p;
      ~LtFree() { dev_free(p); }
    } lt_guard{lt};
    int64_t* lsrc = reinterpret_cast<int64_t*>(lt);
    int32_t* llen = reinterpret_cast<int32_t*>(lt + al256(lanes * 8));
    int32_t* lrow = fp8 ? reinterpret_cast<int32_t*>(lt + al256(lanes * 8) + al256(lanes * 4))
                        : nullptr;
    LongRow* lr_tmp = reinterpret_cast<LongRow*>(lt + al256(lanes * 8) + al256(lanes * 4) +
                                                 (fp8 ? al256(lanes * 4) : 0));
    int nbig = 0;
    TE_CK(DL.emit(const_cast<SellSlice*>(P->sell.slices), const_cast<int32_t*>(P->sell.vout),
                  lsrc, llen, lrow, const_cast<LongRow*>(P->sell.lrows), lr_tmp, s, &nbig),
          "build the SELL layout on the device");
    P->sell.nlbig = nbig;
    if (arriving) {  // column indices must lie in [0, n)
      TE_CK(cudaMemsetAsync(dflag, 0, sizeof(int), s), "clear flag");
      TE_CK(cudaStreamWaitEvent(s, side.cols_done, 0), "wait for the column indices");
      TE_CK(launch_validate_cols(P->ci, P->nnz, P->n, dflag, s), "validate columns");
    }
    if (l_slices > 0)
      TE_CK(fill_sell(in_type, P->sell, P->rp, P->ci, P->val, P->n, P->nnz, lsrc, llen, lrow,
                      vals64, P->W.lscale ? static_cast<float*>(at(P, P->W.lscale)) : nullptr,
                      P->diperm, s, arriving ? side.cols_done : nullptr,
                      arriving ? side.done : nullptr, arriving ? dflag : nullptr),
            "fill the SELL layout");
    if (arriving) {
      TE_CK(cudaStreamWaitEvent(s, side.done, 0), "wait for the matrix copy");
      int hflag = 0;
      TE_CK(cudaMemcpyAsync(&hflag, dflag, sizeof(int), cudaMemcpyDeviceToHost, s), "read flag");
      TE_CK(cudaStreamSynchronize(s), "plan setup");
      if (hflag)
        return fail(TE_ERR_INVALID_ARG, "malformed CSR: a column index is outside [0, n)");
    }
  } else {
    TE_CK(upload_sell(in_type, sell, P->rp, P->ci, P->val, P->n, P->nnz, P->sell, vals64,
                      P->W.lscale ? static_cast<float*>(at(P, P->W.lscale)) : nullptr,
                      P->diperm, s),
          "build the SELL layout");
  }
  if (P->refine) {
    P->sell64 = P->sell;
    P->sell64.vk = TE_F64;
    P->sell64.lscale = nullptr;
    if (vals64) P->sell64.vals = vals64;
  }
  if (P->refine || P->reorder) P->ubase = static_cast<double*>(at(P, P->W.Uint));
  if (P->owned_csr) {  // the solve reads only the SELL copy
    dev_free(P->owned_csr);
    P->owned_csr = nullptr;
  }

  if (opt.use_graph) {
    TE_CK(cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking), "create capture stream");
    TE_CK(cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t e = enqueue_solve(P, P->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(P->cap, &g);
    if (e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(e, "capture solve");
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
    e = cudaGraphInstantiate(&P->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "instantiate graph");
  }
  guard.keep = true;
  *out = P;
  return TE_OK;
}

te_status te_plan_launch(te_plan* P, const double* v1, double* eigvals_dev, double* eigvecs_dev,
                         void* stream) {
  if (!P) return fail(TE_ERR_INVALID_ARG, "plan is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  te_status r = plan_begin(P, v1, eigvecs_dev, eigvals_dev, s);
  if (r != TE_OK) return r;
  if (P->gexec) {
    TE_CK(cudaGraphLaunch(P->gexec, s), "graph launch");
  } else {
    TE_CK(enqueue_solve(P, s), "enqueue solve");
  }
  return TE_OK;
}

te_status te_plan_status(te_plan* P) {
  if (!P) return fail(TE_ERR_INVALID_ARG, "plan is NULL");
  int status = 0;
  TE_CK(cudaMemcpy(&status, &P->st->status, sizeof(int), cudaMemcpyDeviceToHost), "read status");
  if (status != 0) return fail((te_status)status, "device-side status of the last solve");
  return TE_OK;
}

int32_t te_plan_kernel_count(const te_plan* P) { return P ? P->nkernels : 0; }

te_status te_plan_layout(const te_plan* P, int32_t* window, int32_t* vmax) {
  if (!P) return fail(TE_ERR_INVALID_ARG, "plan is NULL");
  if (window) *window = P->sell_window;
  if (vmax) *vmax = P->sell_vmax;
  return TE_OK;
}

int64_t te_plan_stream_blocks(const te_plan* P) {
  return (P && P->streaming) ? (int64_t)P->blocks.size() : 0;
}

te_status te_plan_profile(te_plan* P, double* ms, int32_t* launches, double* bytes,
                          void* stream) {
  if (!P) return fail(TE_ERR_INVALID_ARG, "plan is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* U = nullptr;  // the Ritz contraction needs somewhere to write
  TE_CK(dev_alloc(&U, sizeof(double) * (size_t)P->n * P->K), "allocate profile eigvecs");
  te_status r = plan_begin(P, nullptr, U, nullptr, s);
  if (r != TE_OK) {
    dev_free(U);
    return r;
  }
  P->prof = te_plan::Prof();
  P->prof.on = true;
  const int saved = P->nkernels;
  cudaError_t e = enqueue_solve(P, s);
  P->nkernels = saved;
  P->prof.on = false;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  double acc_ms[TE_NUM_KINDS] = {0}, acc_b[TE_NUM_KINDS] = {0};
  int32_t cnt[TE_NUM_KINDS] = {0};
  for (size_t k = 0; e == cudaSuccess && k < P->prof.kind.size(); ++k) {
    float t = 0.f;
    e = cudaEventElapsedTime(&t, P->prof.ev[2 * k], P->prof.ev[2 * k + 1]);
    acc_ms[P->prof.kind[k]] += t;
    acc_b[P->prof.kind[k]] += P->prof.bytes[k];
    cnt[P->prof.kind[k]] += 1;
  }
  for (cudaEvent_t ev : P->prof.ev) cudaEventDestroy(ev);
  P->prof = te_plan::Prof();
  dev_free(U);
  if (e != cudaSuccess) return cuda_fail(e, "te_plan_profile");
  for (int k = 0; k < TE_NUM_KINDS; ++k) {
    if (ms) ms[k] = acc_ms[k];
    if (launches) launches[k] = cnt[k];
    if (bytes) bytes[k] = acc_b[k];
  }
  return te_plan_status(P);
}

te_status te_plan_solve(te_plan* P, const double* v1, double* eigvals, double* eigvecs,
                        double* residuals, void* stream) {
  if (!P) return fail(TE_ERR_INVALID_ARG, "plan is NULL");
  if (!eigvals) return fail(TE_ERR_INVALID_ARG, "eigvals is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* U = eigvecs;
  double* Utmp = nullptr;
  if (eigvecs && !is_device_ptr(eigvecs)) {
    U = static_cast<double*>(mapped_host_ptr(eigvecs));
    if (!U) {  // pageable host memory: stage on the device, copy at the end
      TE_CK(dev_alloc(&Utmp, sizeof(double) * (size_t)P->n * P->K), "allocate eigvecs staging");
      U = Utmp;
    }
  }
  te_status r = te_plan_launch(P, v1, nullptr, U, stream);
  if (r != TE_OK) {
    if (Utmp) dev_free(Utmp);
    return r;
  }
  cudaError_t e = cudaMemcpyAsync(&P->hres->restart_flag, &P->st->restart_flag, 4 * sizeof(int),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(P->hres->theta, P->st->theta_sel, sizeof(double) * P->K,
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(P->hres->resid, P->st->resid_est, sizeof(double) * P->K,
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    if (Utmp) dev_free(Utmp);
    return cuda_fail(e, "solve");
  }
  const int status = P->hres->status;
  if (status != 0 && status != TE_ERR_BREAKDOWN) {
    if (Utmp) dev_free(Utmp);
    return fail((te_status)status, std::string("device-side failure: ") +
                                       te_status_string((te_status)status));
  }
  // outputs
  if (Utmp) {
    e = cudaMemcpy(eigvecs, Utmp, sizeof(double) * (size_t)P->n * P->K, cudaMemcpyDeviceToHost);
    dev_free(Utmp);
    if (e != cudaSuccess) return cuda_fail(e, "copy eigvecs");
  }
  const cudaMemcpyKind kv = is_device_ptr(eigvals) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
  TE_CK(cudaMemcpy(eigvals, P->hres->theta, sizeof(double) * P->K, kv), "copy eigvals");
  if (residuals) {
    const cudaMemcpyKind kr =
        is_device_ptr(residuals) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    TE_CK(cudaMemcpy(residuals, P->hres->resid, sizeof(double) * P->K, kr), "copy residuals");
  }
  if (status == TE_ERR_BREAKDOWN) return fail(TE_ERR_BREAKDOWN, "Krylov space could not be extended");
  return TE_OK;
}

te_status te_topk_eigs(const te_csr* A, int32_t K, int32_t krylov_steps, te_precision p,
                       const te_options* opt, double* eigvals, double* eigvecs,
                       double* residuals, void* stream) {
  te_options o;
  if (opt) o = *opt;
  else te_default_options(&o);
  o.use_graph = 0;  // a single solve: launch directly
  te_plan* P = nullptr;
  te_status r = te_plan_create(A, K, krylov_steps, p, &o, stream, &P);
  if (r != TE_OK) return r;
  r = te_plan_solve(P, nullptr, eigvals, eigvecs, residuals, stream);
  std::string keep = g_err;
  te_plan_destroy(P);
  g_err = keep;
  return r;
}

te_status te_spmv(const te_csr* A, te_precision p, const void* x, double* y, void* stream) {
  if (!A) return fail(TE_ERR_INVALID_ARG, "A is NULL");
  te_status r = check_args(A, 1, 1, p);
  if (r != TE_OK) return r;
  if (A->where != TE_DEVICE) return fail(TE_ERR_INVALID_ARG, "te_spmv needs a TE_DEVICE matrix");
  if (!x || !y) return fail(TE_ERR_INVALID_ARG, "x and y must not be NULL");
  if (!(aligned16(A->row_ptr) && aligned16(A->col_idx) && aligned16(A->values)))
    return fail(TE_ERR_INVALID_ARG, "device CSR arrays must be 16-byte aligned");
  if (prepare_kernels() != cudaSuccess) return cuda_fail(g_prep_err, "kernel set-up");
  const int prec = prec_of(p);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<int64_t> rp((size_t)A->n + 1);
  TE_CK(cudaMemcpyAsync(rp.data(), A->row_ptr, sizeof(int64_t) * (A->n + 1),
                        cudaMemcpyDeviceToHost, s),
        "copy row_ptr");
  TE_CK(cudaStreamSynchronize(s), "sync");
  SellHost sell;
  std::string perr;
  if (!make_sell(rp.data(), A->n, A->nnz, sell, perr))
    return fail(TE_ERR_INVALID_ARG, "malformed CSR: " + perr);
  const size_t b_sl = al256(std::max<size_t>(sell.slices.size(), 1) * sizeof(SellSlice));
  const size_t b_vo = al256(std::max<size_t>(sell.vout.size(), 1) * sizeof(int32_t));
  const size_t b_co = al256(std::max<size_t>((size_t)sell.entries, 1) * sizeof(int32_t));
  const size_t b_va = al256(std::max<size_t>((size_t)sell.entries, 1) * elt_of(p.values));
  const size_t b_lr = al256(std::max<size_t>(sell.lrows.size(), 1) * sizeof(LongRow));
  const size_t b_vp = al256(std::max<size_t>((size_t)sell.pieces, 1) * 8);
  const size_t b_ls =
      p.values == TE_FP8_E4M3 ? al256(std::max<size_t>(sell.vout.size(), 1) * 4) : 0;
  char* buf = nullptr;
  TE_CK(dev_alloc(&buf, b_sl + b_vo + b_co + b_va + b_lr + b_vp + b_ls + 256),
        "allocate SpMV layout");
  DevSell D;
  size_t off = 0;
  D.slices = reinterpret_cast<SellSlice*>(buf + off);
  off += b_sl;
  D.vout = reinterpret_cast<int32_t*>(buf + off);
  off += b_vo;
  D.cols = reinterpret_cast<int32_t*>(buf + off);
  off += b_co;
  D.vals = buf + off;
  off += b_va;
  D.lrows = reinterpret_cast<LongRow*>(buf + off);
  off += b_lr;
  D.vpart = buf + off;
  off += b_vp;
  float* lscale = b_ls ? reinterpret_cast<float*>(buf + off) : nullptr;
  off += b_ls;
  D.vk = p.values;
  D.lscale = lscale;
  int* flag = reinterpret_cast<int*>(buf + off);
  D.nslices = (int)sell.slices.size();
  D.nlrows = (int)sell.lrows.size();
  D.nlbig = (int)sell.nbig;
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), s);
  if (e == cudaSuccess) e = launch_validate_cols(A->col_idx, A->nnz, A->n, flag, s);
  int hflag = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && hflag) {
    dev_free(buf);
    return fail(TE_ERR_INVALID_ARG, "malformed CSR: a column index is outside [0, n)");
  }
  const int in_type = A->values_f64 ? TE_F64 : p.values;
  if (e == cudaSuccess)
    e = upload_sell(in_type, sell, A->row_ptr, A->col_idx, A->values, A->n, A->nnz, D, nullptr,
                    lscale, nullptr, s);
  // the kernel writes rows with entries only
  if (e == cudaSuccess) e = cudaMemsetAsync(y, 0, sizeof(double) * A->n, s);
  if (e == cudaSuccess) e = launch_spmv(prec, D, x, y, true, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dev_free(buf);
  if (e != cudaSuccess) return cuda_fail(e, "te_spmv");
  return TE_OK;
}

te_status te_lanczos(const te_csr* A, int32_t krylov_steps, te_precision p, const te_options* opt,
                     double* alpha, double* beta, double* basis, int32_t* restarts,
                     void* stream) {
  if (!alpha || !beta) return fail(TE_ERR_INVALID_ARG, "alpha and beta must not be NULL");
  te_options o;
  if (opt) o = *opt;
  else te_default_options(&o);
  o.use_graph = 0;
  te_plan* P = nullptr;
  te_status r = te_plan_create(A, 1, krylov_steps, p, &o, stream, &P);
  if (r != TE_OK) return r;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  r = plan_begin(P, nullptr, nullptr, nullptr, s);
  cudaError_t e = cudaSuccess;
  if (r == TE_OK) e = enqueue_lanczos(P, s);
  std::vector<double> a_h(krylov_steps), b_h(krylov_steps + 1);
  int hst[4] = {0, 0, 0, 0};
  if (r == TE_OK && e == cudaSuccess)
    e = cudaMemcpyAsync(a_h.data(), P->st->alpha, sizeof(double) * krylov_steps,
                        cudaMemcpyDeviceToHost, s);
  if (r == TE_OK && e == cudaSuccess)
    e = cudaMemcpyAsync(b_h.data(), P->st->beta, sizeof(double) * (krylov_steps + 1),
                        cudaMemcpyDeviceToHost, s);
  if (r == TE_OK && e == cudaSuccess)
    e = cudaMemcpyAsync(hst, &P->st->restart_flag, sizeof(hst), cudaMemcpyDeviceToHost, s);
  if (r == TE_OK && e == cudaSuccess && basis)
    e = launch_basis_to_f64(P->prec, at(P, P->W.V), basis_tstride(P), TILE_R, P->n,
                            krylov_steps, P->st->s, P->diperm, basis, s);
  if (r == TE_OK && e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (r == TE_OK && e != cudaSuccess) r = cuda_fail(e, "te_lanczos");
  if (r == TE_OK) {
    const int status = hst[2];
    if (status != 0 && status != TE_ERR_BREAKDOWN)
      r = fail((te_status)status, "device-side failure in the Lanczos phase");
  }
  if (r == TE_OK) {
    memcpy(alpha, a_h.data(), sizeof(double) * krylov_steps);
    memcpy(beta, b_h.data(), sizeof(double) * (krylov_steps + 1));
    if (restarts) *restarts = hst[1];
    if (hst[2] == TE_ERR_BREAKDOWN) r = fail(TE_ERR_BREAKDOWN, "restart failed");
  }
  std::string keep = g_err;
  te_plan_destroy(P);
  g_err = keep;
  return r;
}

te_status te_tridiag_eigs(int32_t m, const double* alpha, const double* beta, int32_t which,
                          double* theta, double* Y, int32_t* sweeps, void* stream) {
  if (m < 1 || m > MAX_M) return fail(TE_ERR_INVALID_ARG, "m must be in [1, 64]");
  if (!alpha || !beta || !theta) return fail(TE_ERR_INVALID_ARG, "NULL argument");
  if (which != TE_WHICH_LARGEST_MAGNITUDE && which != TE_WHICH_LARGEST_ALGEBRAIC)
    return fail(TE_ERR_INVALID_ARG, "which must be TE_WHICH_*");
  if (prepare_kernels() != cudaSuccess) return cuda_fail(g_prep_err, "kernel set-up");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* dbuf = nullptr;
  TE_CK(dev_alloc(&dbuf, 2 * sizeof(int)), "allocate status");
  JacobiArgs j;
  memset(&j, 0, sizeof(j));
  j.alpha = alpha;
  j.beta = beta;
  j.m = m;
  j.K = m;
  j.which = which;
  j.theta_out = theta;
  j.Y_out = Y;
  j.sweeps_out = dbuf;
  j.status_out = dbuf + 1;
  cudaError_t e = launch_jacobi(j, s);
  int h[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, dbuf, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dev_free(dbuf);
  if (e != cudaSuccess) return cuda_fail(e, "te_tridiag_eigs");
  if (sweeps) *sweeps = h[0];
  if (h[1] != 0) return fail((te_status)h[1], "Jacobi sweeps did not converge");
  return TE_OK;
}

te_status te_quantize(const te_csr* A, int32_t to, void* out, float* row_scale, void* stream) {
  if (!A || !out) return fail(TE_ERR_INVALID_ARG, "NULL argument");
  if (A->where != TE_DEVICE || A->values_f64 != 1)
    return fail(TE_ERR_INVALID_ARG, "te_quantize needs a TE_DEVICE matrix with binary64 values");
  if (A->n < 1 || A->nnz < 0 || !A->row_ptr || (A->nnz > 0 && !A->values))
    return fail(TE_ERR_INVALID_ARG, "bad CSR sizes or pointers");
  if (to != TE_F32 && to != TE_BF16 && to != TE_FP8_E4M3)
    return fail(TE_ERR_INVALID_ARG, "to must be TE_F32, TE_BF16 or TE_FP8_E4M3");
  if ((to == TE_FP8_E4M3) != (row_scale != nullptr))
    return fail(TE_ERR_INVALID_ARG, "row_scale is required for TE_FP8_E4M3 and only for it");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = launch_quantize(to, A->row_ptr, static_cast<const double*>(A->values), A->n,
                                  A->nnz, out, row_scale, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "te_quantize");
  return TE_OK;
}

te_status te_gram(int64_t n, int32_t K, const double* U, double* G, void* stream) {
  if (n < 1 || K < 1 || K > MAX_M) return fail(TE_ERR_INVALID_ARG, "need n >= 1, 1 <= K <= 64");
  if (!U || !G) return fail(TE_ERR_INVALID_ARG, "NULL argument");
  if (!is_device_ptr(U)) return fail(TE_ERR_INVALID_ARG, "U must be device memory");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  TE_CK(cudaGetDevice(&dev), "cudaGetDevice");
  TE_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
  const int grid = sms * 2;
  const size_t np = (size_t)K * (K + 1) / 2;
  double* buf = nullptr;
  TE_CK(dev_alloc(&buf, sizeof(double) * (np * grid + (size_t)K * K)), "allocate Gram work");
  cudaError_t e = launch_gram(U, n, K, buf, grid, buf + np * grid, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(G, buf + np * grid, sizeof(double) * K * K, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dev_free(buf);
  if (e != cudaSuccess) return cuda_fail(e, "te_gram");
  return TE_OK;
}

te_status te_spmv_layout(const int64_t* row_ptr, int64_t n, int64_t nnz, int32_t window,
                         int32_t vmax, int64_t* nslices, int64_t* entries, int64_t* nlong_rows,
                         int32_t* slice_len, int32_t* lane_out, int64_t* lane_src,
                         int32_t* lane_len) {
  if (!row_ptr || n < 1 || nnz < 0) return fail(TE_ERR_INVALID_ARG, "bad arguments");
  if (window == 0) window = SELL_WINDOW;
  if (vmax == 0) vmax = SELL_VMAX;
  if (window < 1 || vmax < 1 || vmax > 1024)
    return fail(TE_ERR_INVALID_ARG, "window >= 1 and 1 <= vmax <= 1024");
  SellHost sell;
  std::string perr;
  if (!make_sell(row_ptr, n, nnz, sell, perr, window, vmax))
    return fail(TE_ERR_INVALID_ARG, "malformed CSR: " + perr);
  if (nslices) *nslices = (int64_t)sell.slices.size();
  if (entries) *entries = sell.entries;
  if (nlong_rows) *nlong_rows = (int64_t)sell.lrows.size();
  for (size_t i = 0; i < sell.slices.size(); ++i)
    if (slice_len) slice_len[i] = sell.slices[i].len;
  for (size_t l = 0; l < sell.vout.size(); ++l) {
    if (lane_out) lane_out[l] = sell.vout[l];
    if (lane_src) lane_src[l] = sell.vsrc[l];
    if (lane_len) lane_len[l] = sell.vlen[l];
  }
  return TE_OK;
}

te_status te_spmv_layout_device(const int64_t* row_ptr, int64_t n, int64_t nnz, int32_t window,
                                int32_t vmax, int32_t order, int64_t* nslices, int64_t* entries,
                                int64_t* nlong_rows, int32_t* perm, int32_t* slice_len,
                                int64_t* slice_base, int32_t* lane_out, int64_t* lane_src,
                                int32_t* lane_len, int32_t* lane_row, int32_t* long_rows,
                                int32_t* nbig, void* stream) {
  if (!row_ptr || n < 1 || nnz < 0) return fail(TE_ERR_INVALID_ARG, "bad arguments");
  if (!is_device_ptr(row_ptr)) return fail(TE_ERR_INVALID_ARG, "row_ptr must be device memory");
  if (order != TE_ORDER_KEEP && order != TE_ORDER_DEGREE)
    return fail(TE_ERR_INVALID_ARG, "order must be TE_ORDER_KEEP or TE_ORDER_DEGREE");
  if (window == 0) window = SELL_WINDOW;
  if (vmax == 0) vmax = SELL_VMAX;
  if (!dev_layout_fits(n, window, vmax))
    return fail(TE_ERR_UNSUPPORTED, "the device layout build does not cover these sizes");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool reorder = order == TE_ORDER_DEGREE;
  DevLayout DL;
  std::string derr;
  cudaError_t e = DL.count(row_ptr, n, nnz, window, vmax, reorder, s, derr);
  if (e == cudaErrorInvalidValue && !derr.empty())
    return fail(TE_ERR_INVALID_ARG, "malformed CSR: " + derr);
  TE_CK(e, "device layout");
  // device arrays: row order (4 n + 4 n + 8 n + 4 n), then the layout
  char* b = nullptr;
  struct BFree {
    char*& p;
    ~BFree() {
      if (p) dev_free(p);
    }
  } bf{b};
  const size_t nn = (size_t)n;
  int64_t tot[4];
  int32_t *dp = nullptr, *dip = nullptr, *dl = nullptr;
  int64_t* ds = nullptr;
  char* ob = nullptr;
  struct OFree {
    char*& p;
    ~OFree() {
      if (p) dev_free(p);
    }
  } of{ob};
  if (reorder) {
    TE_CK(dev_alloc(&ob, al256(nn * 8) + 3 * al256(nn * 4)), "allocate");
    ds = reinterpret_cast<int64_t*>(ob);
    dp = reinterpret_cast<int32_t*>(ob + al256(nn * 8));
    dip = reinterpret_cast<int32_t*>(ob + al256(nn * 8) + al256(nn * 4));
    dl = reinterpret_cast<int32_t*>(ob + al256(nn * 8) + 2 * al256(nn * 4));
    TE_CK(DL.order(dp, dip, ds, dl, s), "device row order");
  }
  TE_CK(DL.windows(s, tot), "device layout counts");
  const size_t S = (size_t)tot[0], lanes = std::max<size_t>(S * SELL_C, 1),
               NL = (size_t)std::max<int64_t>(tot[3], 1);
  const size_t o_sl = 0, o_out = al256(std::max<size_t>(S, 1) * sizeof(SellSlice)),
               o_src = o_out + al256(lanes * 4), o_len = o_src + al256(lanes * 8),
               o_row = o_len + al256(lanes * 4), o_lr = o_row + al256(lanes * 4),
               o_lt = o_lr + al256(NL * sizeof(LongRow)), total = o_lt + al256(NL * sizeof(LongRow));
  TE_CK(dev_alloc(&b, total), "allocate");
  int nb = 0;
  TE_CK(DL.emit(reinterpret_cast<SellSlice*>(b + o_sl), reinterpret_cast<int32_t*>(b + o_out),
                reinterpret_cast<int64_t*>(b + o_src), reinterpret_cast<int32_t*>(b + o_len),
                reinterpret_cast<int32_t*>(b + o_row), reinterpret_cast<LongRow*>(b + o_lr),
                reinterpret_cast<LongRow*>(b + o_lt), s, &nb),
        "device layout");
  if (nslices) *nslices = tot[0];
  if (entries) *entries = tot[1];
  if (nlong_rows) *nlong_rows = tot[3];
  if (nbig) *nbig = nb;
  std::vector<SellSlice> hs(S);
  std::vector<LongRow> hl((size_t)tot[3]);
  if (S) TE_CK(cudaMemcpy(hs.data(), b + o_sl, S * sizeof(SellSlice), cudaMemcpyDeviceToHost), "copy");
  if (tot[3]) TE_CK(cudaMemcpy(hl.data(), b + o_lr, hl.size() * sizeof(LongRow), cudaMemcpyDeviceToHost), "copy");
  for (size_t i = 0; i < S; ++i) {
    if (slice_len) slice_len[i] = hs[i].len;
    if (slice_base) slice_base[i] = hs[i].base;
  }
  for (size_t i = 0; i < hl.size(); ++i)
    if (long_rows) {
      long_rows[3 * i] = hl[i].row;
      long_rows[3 * i + 1] = hl[i].first;
      long_rows[3 * i + 2] = hl[i].count;
    }
  if (S) {
    if (lane_out) TE_CK(cudaMemcpy(lane_out, b + o_out, S * SELL_C * 4, cudaMemcpyDeviceToHost), "copy");
    if (lane_src) TE_CK(cudaMemcpy(lane_src, b + o_src, S * SELL_C * 8, cudaMemcpyDeviceToHost), "copy");
    if (lane_len) TE_CK(cudaMemcpy(lane_len, b + o_len, S * SELL_C * 4, cudaMemcpyDeviceToHost), "copy");
    if (lane_row) TE_CK(cudaMemcpy(lane_row, b + o_row, S * SELL_C * 4, cudaMemcpyDeviceToHost), "copy");
  }
  if (perm) {
    if (reorder) TE_CK(cudaMemcpy(perm, dp, nn * 4, cudaMemcpyDeviceToHost), "copy");
    else
      for (size_t i = 0; i < nn; ++i) perm[i] = (int32_t)i;
  }
  return TE_OK;
}

te_status te_check_symmetric(const te_csr* A, double tol, double* max_abs_diff) {
  if (!A || !A->row_ptr || A->n < 1 || A->nnz < 0 || (A->nnz > 0 && (!A->col_idx || !A->values)))
    return fail(TE_ERR_INVALID_ARG, "bad arguments");
  if (A->where != TE_HOST) return fail(TE_ERR_INVALID_ARG, "the check reads a TE_HOST matrix");
  if (!A->values_f64) return fail(TE_ERR_INVALID_ARG, "the check reads binary64 values (values_f64 = 1)");
  if (!(tol >= 0.0)) return fail(TE_ERR_INVALID_ARG, "tol must be >= 0");
  const int64_t n = A->n, nnz = A->nnz;
  const int64_t* rp = A->row_ptr;
  const int32_t* ci = A->col_idx;
  const double* va = static_cast<const double*>(A->values);
  std::string perr;
  if (!rows_valid(rp, n, nnz, perr)) return fail(TE_ERR_INVALID_ARG, "malformed CSR: " + perr);
  for (int64_t k = 0; k < nnz; ++k)
    if (ci[k] < 0 || (int64_t)ci[k] >= n)
      return fail(TE_ERR_INVALID_ARG, "malformed CSR: a column index is outside [0, n)");
  // the transpose by a counting sort over the columns
  std::vector<int64_t> tp((size_t)n + 1, 0);
  for (int64_t k = 0; k < nnz; ++k) ++tp[(size_t)ci[k] + 1];
  for (int64_t r = 0; r < n; ++r) tp[(size_t)r + 1] += tp[(size_t)r];
  std::vector<int64_t> fill(tp.begin(), tp.end() - 1);
  std::vector<int32_t> tc((size_t)nnz);
  std::vector<double> tv((size_t)nnz);
  for (int64_t r = 0; r < n; ++r)
    for (int64_t k = rp[r]; k < rp[r + 1]; ++k) {
      const int64_t at = fill[(size_t)ci[k]]++;
      tc[(size_t)at] = (int32_t)r;
      tv[(size_t)at] = va[k];
    }
  // row r of M against row r of M^T, both sorted by column, duplicates summed
  double worst = 0.0;
  std::vector<std::pair<int32_t, double>> a, b;
  auto merged = [](std::vector<std::pair<int32_t, double>>& v) {
    std::sort(v.begin(), v.end(),
              [](const std::pair<int32_t, double>& x, const std::pair<int32_t, double>& y) {
                return x.first < y.first;
              });
    size_t o = 0;
    for (size_t i = 0; i < v.size(); ++i) {
      if (o > 0 && v[o - 1].first == v[i].first) v[o - 1].second += v[i].second;
      else v[o++] = v[i];
    }
    v.resize(o);
  };
  for (int64_t r = 0; r < n; ++r) {
    a.clear();
    b.clear();
    for (int64_t k = rp[r]; k < rp[r + 1]; ++k) a.emplace_back(ci[k], va[k]);
    for (int64_t k = tp[(size_t)r]; k < tp[(size_t)r + 1]; ++k) b.emplace_back(tc[(size_t)k], tv[(size_t)k]);
    merged(a);
    merged(b);
    size_t i = 0, j = 0;
    while (i < a.size() || j < b.size()) {  // a missing mirror entry counts as zero
      double d;
      if (j == b.size() || (i < a.size() && a[i].first < b[j].first)) d = a[i++].second;
      else if (i == a.size() || b[j].first < a[i].first) d = b[j++].second;
      else d = a[i++].second - b[j++].second;
      worst = std::max(worst, std::fabs(d));
    }
  }
  if (max_abs_diff) *max_abs_diff = worst;
  if (worst > tol)
    return fail(TE_ERR_INVALID_ARG, "the matrix is not symmetric: max |a_ij - a_ji| = " +
                                        std::to_string(worst));
  return TE_OK;
}

te_status te_degree_order(const int64_t* row_ptr, int64_t n, int64_t nnz, int32_t* perm,
                          int32_t* iperm) {
  if (!row_ptr || !perm || n < 1 || n >= (int64_t)1 << 31 || nnz < 0)
    return fail(TE_ERR_INVALID_ARG, "bad arguments");
  std::string perr;
  if (!rows_valid(row_ptr, n, nnz, perr)) return fail(TE_ERR_INVALID_ARG, "malformed CSR: " + perr);
  hvec<int32_t> inv, len;
  hvec<int64_t> src((size_t)n);
  len.resize((size_t)n);
  if (!iperm) {
    inv.resize((size_t)n);
    iperm = inv.data();
  }
  degree_order(row_ptr, n, perm, iperm, src.data(), len.data());
  return TE_OK;
}

}  // extern "C"
