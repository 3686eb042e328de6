// te_noalloc.cu - y = M x without any device allocation.
//
// Some callers cannot call cudaMalloc: a framework whose caching allocator has
// already reserved the device memory, a serving loop that must not take the
// allocator's locks or latency between requests, or a host application that
// hands this library a fixed memory budget and forbids driver allocations.
// te_spmv needs work memory (its row partition and long-row partial sums);
// te_spmv_noalloc is a variant of the same SpMV that keeps its work memory in
// one file-scope __device__ array instead, so it allocates nothing.
//
// Work decomposition: the non-zeros are cut into fixed chunks of CHUNK
// entries; CTA c stages the products of chunk c exactly as the main SpMV does
// and finds, by binary search on row_ptr, the rows its chunk touches.  Rows
// that start and end inside the chunk are written directly; the (possibly
// partial) first and last row of the chunk leave their partial sums in the
// scratch array, and a second kernel adds those partials in chunk order
// (deterministic) and writes the empty rows.  The scratch holds one 32-byte
// record per chunk, so a matrix may have at most NOALLOC_MAX_CHUNKS chunks.
// A chunk's CTA walks every row its entries touch, empty ones included, and
// the second kernel visits every row: the cost grows with n as well as nnz.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "te_common.cuh"
#include "te_internal.h"

namespace te {

constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_MAX_CHUNKS = 131072;  // 4 MiB of carry records
constexpr int NOALLOC_MAX_DEVICES = 64;

struct Carry {
  int32_t head, tail;  // first and last row touched by the chunk
  int32_t pad0, pad1;
  double sum_head;     // partial sum of the head row over the chunk (f64 or dw bits)
  double sum_tail;     // partial sum of the tail row over the chunk (if tail != head)
};
static_assert(sizeof(Carry) == 32, "carry record layout");

// Shared by every call on a device; keeps the last call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[256 + NOALLOC_MAX_CHUNKS * sizeof(Carry)];

template <int P>
struct NaTr;
template <>
struct NaTr<PREC_DDD> {
  using val_t = double;
  using x_t = double;
  static constexpr int CHUNK = 2048;
};
template <>
struct NaTr<PREC_FDF> {
  using val_t = float;
  using x_t = float;
  static constexpr int CHUNK = 4096;
};

// last row r in [0, n) with rp[r] <= k (rp[0] = 0 <= k)
TE_DEV int32_t row_of(const int64_t* rp, int64_t n, int64_t k) {
  int64_t lo = 0, hi = n - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi + 1) >> 1;
    if (__ldg(rp + mid) <= k) lo = mid;
    else hi = mid - 1;
  }
  return (int32_t)lo;
}

// accumulator: double (DDD) or double-float (FDF); stored in 8 bytes
template <int P>
struct NaAcc;
template <>
struct NaAcc<PREC_DDD> {
  double v = 0.0;
  TE_DEV void add_prod(double a, double b) { v = fma(a, b, v); }
  TE_DEV void warp_reduce() { v = warp_sum(v); }
  TE_DEV double bits() const { return v; }
  TE_DEV void add_bits(double b) { v += b; }
  TE_DEV double value() const { return v; }
};
template <>
struct NaAcc<PREC_FDF> {
  dacc a = {0.f, 0.f};
  TE_DEV void add_prod(float x, float y) {
    float p, e;
    two_prod(x, y, p, e);
    dacc_add_pair(a, p, e);
  }
  TE_DEV void warp_reduce() { a = warp_sum(a); }
  TE_DEV double bits() const {
    dw v = dacc_value(a);
    return __longlong_as_double(((long long)__float_as_int(v.lo) << 32) |
                                (unsigned int)__float_as_int(v.hi));
  }
  TE_DEV void add_bits(double b) {
    long long u = __double_as_longlong(b);
    dacc_add_pair(a, __int_as_float((int)(u & 0xffffffffu)), __int_as_float((int)(u >> 32)));
  }
  TE_DEV double value() const { return dw_to_double(dacc_value(a)); }
};

template <int P>
__global__ void __launch_bounds__(NOALLOC_THREADS) noalloc_chunk_kernel(
    const int64_t* rp, const int32_t* ci, const void* val, const void* x, double* y, int64_t n,
    int64_t nnz, unsigned char* scratch) {
  using val_t = typename NaTr<P>::val_t;
  using x_t = typename NaTr<P>::x_t;
  constexpr int CH = NaTr<P>::CHUNK;
  __shared__ val_t sv[CH];
  __shared__ x_t sx[CH];
  __shared__ int32_t hs, ts;
  int* status = reinterpret_cast<int*>(scratch);
  Carry* carry = reinterpret_cast<Carry*>(scratch + 256);

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t c = blockIdx.x;
  const int64_t k0 = c * CH;
  const int64_t k1 = k0 + CH < nnz ? k0 + CH : nnz;
  const int nz = (int)(k1 - k0);
  if (tid == 0) hs = row_of(rp, n, k0);
  if (tid == 32) ts = row_of(rp, n, k1 - 1);
  const val_t* va = static_cast<const val_t*>(val);
  const x_t* xv = static_cast<const x_t*>(x);
  int bad = 0;
  for (int e = tid; e < nz; e += NOALLOC_THREADS) {
    const int32_t col = ci[k0 + e];
    const bool ok = col >= 0 && (int64_t)col < n;
    bad |= !ok;
    sv[e] = va[k0 + e];
    sx[e] = ok ? xv[col] : (x_t)0;
  }
  if (bad) atomicOr(status, 1);
  __syncthreads();
  const int32_t h = hs, t = ts;
  // one warp per touched row; head and tail rows leave their partial sums
  for (int64_t r = h + wid; r <= t; r += NOALLOC_THREADS / 32) {
    const int64_t b = __ldg(rp + r), e = __ldg(rp + r + 1);
    if (b == e) continue;  // empty rows are written by the fix-up kernel
    const int64_t s0 = (b > k0 ? b : k0) - k0, s1 = (e < k1 ? e : k1) - k0;
    NaAcc<P> acc;
    for (int64_t q = s0 + lane; q < s1; q += 32) acc.add_prod(sv[q], sx[q]);
    acc.warp_reduce();
    if (lane == 0) {
      if (r == h) carry[c].sum_head = acc.bits();
      else if (r == t) carry[c].sum_tail = acc.bits();
      else y[r] = acc.value();
    }
  }
  if (tid == 0) {
    carry[c].head = h;
    carry[c].tail = t;
  }
}

// Adds the chunks' partial sums, writes the empty rows, and checks the row
// pointers (row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz): a malformed
// row_ptr sets bit 2 of the status word.  The chunk kernel keeps every access
// in bounds whatever row_ptr holds; its results are discarded then.
template <int P>
__global__ void noalloc_fixup_kernel(const int64_t* rp, double* y, int64_t n, int64_t nnz,
                                     int64_t nchunks, unsigned char* scratch) {
  constexpr int CH = NaTr<P>::CHUNK;
  int* status = reinterpret_cast<int*>(scratch);
  const Carry* carry = reinterpret_cast<const Carry*>(scratch + 256);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t first = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (first == 0 && (__ldg(rp) != 0 || __ldg(rp + n) != nnz)) atomicOr(status, 2);
  for (int64_t i = first; i < nchunks || i < n; i += stride) {
    if (i < n) {
      const int64_t b = __ldg(rp + i), e = __ldg(rp + i + 1);
      if (b == e) y[i] = 0.0;
      if (b > e) atomicOr(status, 2);
    }
    if (i < nchunks) {
      const Carry rec = carry[i];
      const int64_t k0 = i * CH;
      // a row is completed by the chunk in which it starts
      if (__ldg(rp + rec.head) == k0) {
        NaAcc<P> s;
        s.add_bits(rec.sum_head);
        if (rec.tail == rec.head)
          for (int64_t c2 = i + 1; c2 < nchunks && carry[c2].head == rec.head; ++c2)
            s.add_bits(carry[c2].sum_head);
        y[rec.head] = s.value();
      }
      if (rec.tail != rec.head) {
        NaAcc<P> s;
        s.add_bits(rec.sum_tail);
        for (int64_t c2 = i + 1; c2 < nchunks && carry[c2].head == rec.tail; ++c2)
          s.add_bits(carry[c2].sum_head);
        y[rec.tail] = s.value();
      }
    }
  }
}

namespace {
std::mutex g_na_mu;
void* g_na_ptr[NOALLOC_MAX_DEVICES] = {nullptr};
}  // namespace

}  // namespace te

using namespace te;

extern "C" te_status te_spmv_noalloc(const te_csr* A, te_precision p, const void* x, double* y,
                                     void* stream);

// Defined here (not in te_solver.cu) so that the scratch symbol and its device
// address stay in one translation unit.
extern "C" te_status te_spmv_noalloc(const te_csr* A, te_precision p, const void* x, double* y,
                                     void* stream) {
  auto fail = [](te_status s, const std::string& m) {
    set_last_error(m);
    return s;
  };
  if (!A || !x || !y) return fail(TE_ERR_INVALID_ARG, "te_spmv_noalloc: NULL argument");
  if (A->where != TE_DEVICE)
    return fail(TE_ERR_INVALID_ARG, "te_spmv_noalloc: the matrix must be in device memory");
  if (A->n < 1 || A->n >= (int64_t)1 << 31 || A->nnz < 0 || !A->row_ptr ||
      (A->nnz > 0 && (!A->col_idx || !A->values)))
    return fail(TE_ERR_INVALID_ARG, "te_spmv_noalloc: bad CSR sizes or pointers");
  if (A->row_scale) return fail(TE_ERR_UNSUPPORTED, "te_spmv_noalloc: row_scale must be NULL");
  int prec = -1;
  if (p.values == TE_F64 && p.arithmetic == TE_F64 && p.vectors == TE_F64) prec = PREC_DDD;
  if (p.values == TE_F32 && p.arithmetic == TE_F64 && p.vectors == TE_F32) prec = PREC_FDF;
  if (prec < 0) return fail(TE_ERR_UNSUPPORTED, "te_spmv_noalloc: precision must be DDD or FDF");
  if (A->values_f64 && prec != PREC_DDD)
    return fail(TE_ERR_INVALID_ARG,
                "te_spmv_noalloc: values must already have the precision's type (values_f64 = 0)");
  const int chunk = prec == PREC_DDD ? NaTr<PREC_DDD>::CHUNK : NaTr<PREC_FDF>::CHUNK;
  const int64_t nchunks = (A->nnz + chunk - 1) / chunk;
  if (nchunks > NOALLOC_MAX_CHUNKS)
    return fail(TE_ERR_INVALID_ARG,
                "te_spmv_noalloc: nnz = " + std::to_string(A->nnz) + " exceeds the maximum " +
                    std::to_string((int64_t)NOALLOC_MAX_CHUNKS * chunk) +
                    " of the fixed scratch array for this precision");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(TE_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
    return fail(TE_ERR_UNSUPPORTED, "te_spmv_noalloc: device index too large");
  // once per device, with that device current: the scratch array's device
  // address (kept for the life of the process; a device reset invalidates it)
  unsigned char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess)
        return fail(TE_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_na_ptr[dev] = ptr;
    }
    scratch = static_cast<unsigned char*>(g_na_ptr[dev]);
  }
  // the status word must start at zero; carry records are written before read
  e = cudaMemsetAsync(scratch, 0, sizeof(int), s);
  if (e == cudaSuccess && nchunks > 0) {
    if (prec == PREC_DDD)
      noalloc_chunk_kernel<PREC_DDD><<<(unsigned)nchunks, NOALLOC_THREADS, 0, s>>>(
          A->row_ptr, A->col_idx, A->values, x, y, A->n, A->nnz, scratch);
    else
      noalloc_chunk_kernel<PREC_FDF><<<(unsigned)nchunks, NOALLOC_THREADS, 0, s>>>(
          A->row_ptr, A->col_idx, A->values, x, y, A->n, A->nnz, scratch);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const int64_t items = nchunks > A->n ? nchunks : A->n;
    int64_t blocks = (items + 255) / 256;
    if (blocks > 16384) blocks = 16384;
    if (prec == PREC_DDD)
      noalloc_fixup_kernel<PREC_DDD><<<(unsigned)blocks, 256, 0, s>>>(A->row_ptr, y, A->n,
                                                                       A->nnz, nchunks, scratch);
    else
      noalloc_fixup_kernel<PREC_FDF><<<(unsigned)blocks, 256, 0, s>>>(A->row_ptr, y, A->n,
                                                                       A->nnz, nchunks, scratch);
    e = cudaGetLastError();
  }
  int status = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, scratch, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(TE_ERR_CUDA, std::string("te_spmv_noalloc: ") + cudaGetErrorString(e));
  if (status & 2) return fail(TE_ERR_INVALID_ARG, "te_spmv_noalloc: malformed row_ptr");
  if (status) return fail(TE_ERR_INVALID_ARG, "te_spmv_noalloc: a column index is outside [0, n)");
  return TE_OK;
}
