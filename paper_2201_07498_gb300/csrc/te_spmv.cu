// te_spmv.cu - the SpMV step of Algorithm 1 (v_t <- M v_i) for sm_103a.
//
// Design ("CSR-stream" row blocks, after Greathouse & Daga, SC'14, re-planned
// for this GPU): the host packs consecutive rows into blocks of at most
// TNNZ non-zeros and SPMV_RMAX rows; rows longer than TNNZ/4 are cut into
// TNNZ-sized chunks handled by separate CTAs and summed by a second kernel.
// Each CTA
//   1. streams its non-zeros (column, value) with coalesced loads marked
//      L2 evict-first, so the gathered vector stays resident in L2,
//   2. gathers x[col] and stages the products in shared memory (FDF: the
//      exact product as a float pair; DDD: value and x as doubles),
//   3. reduces every row with a power-of-two group of lanes sized to the
//      block's mean row length (fixed shuffle tree: deterministic).
// FDF sums products in double-float (Dot2 of Ogita, Rump & Oishi);
// DDD uses binary64 FMA.
#include "te_common.cuh"
#include "te_internal.h"

namespace te {

template <int P>
struct SpmvTr;
template <>
struct SpmvTr<PREC_DDD> {
  using val_t = double;
  using x_t = double;
  using acc_t = double;
  static constexpr int TNNZ = 2048;
};
template <>
struct SpmvTr<PREC_FDF> {
  using val_t = float;
  using x_t = float;
  using acc_t = dacc;
  static constexpr int TNNZ = 4096;
};

int spmv_tile_nnz(int prec) {
  return prec == PREC_DDD ? SpmvTr<PREC_DDD>::TNNZ : SpmvTr<PREC_FDF>::TNNZ;
}

bool make_partition(const int64_t* rp, int64_t n, int64_t nnz, int tnnz, Partition& out,
                    std::string& err) {
  out.blocks.clear();
  out.chunks.clear();
  out.lrows.clear();
  if (rp[0] != 0) {
    err = "row_ptr[0] must be 0";
    return false;
  }
  for (int64_t r = 0; r < n; ++r) {
    if (rp[r + 1] < rp[r]) {
      err = "row_ptr must be non-decreasing (row " + std::to_string(r) + ")";
      return false;
    }
  }
  if (rp[n] != nnz) {
    err = "row_ptr[n] != nnz";
    return false;
  }
  const int64_t long_thresh = tnnz / 4;
  int64_t r = 0;
  while (r < n) {
    int64_t L = rp[r + 1] - rp[r];
    if (L > long_thresh) {
      LongRow lr;
      lr.row = (int32_t)r;
      lr.first = (int32_t)out.chunks.size();
      lr.count = (int32_t)((L + tnnz - 1) / tnnz);
      lr.pad_ = 0;
      for (int32_t c = 0; c < lr.count; ++c) {
        LongChunk ch;
        ch.k0 = rp[r] + (int64_t)c * tnnz;
        ch.k1 = ch.k0 + tnnz < rp[r + 1] ? ch.k0 + tnnz : rp[r + 1];
        ch.row = (int32_t)r;
        ch.pad_ = 0;
        out.chunks.push_back(ch);
      }
      out.lrows.push_back(lr);
      ++r;
      continue;
    }
    int64_t start = r, nz = 0;
    while (r < n && r - start < SPMV_RMAX) {
      int64_t Lr = rp[r + 1] - rp[r];
      if (Lr > long_thresh || nz + Lr > tnnz) break;
      nz += Lr;
      ++r;
    }
    out.blocks.push_back(make_int2((int)start, (int)r));
  }
  return true;
}

struct SpmvArgs {
  const int64_t* rp;
  const int32_t* ci;
  const void* val;
  const void* x;
  void* y;
  const int2* blocks;
  const LongChunk* chunks;
  void* lpart;
  int nshort;
};

template <int P>
TE_DEV void acc_zero(typename SpmvTr<P>::acc_t& a) {
  if constexpr (P == PREC_FDF) a = dacc_zero();
  else a = 0.0;
}

template <int P, bool F64OUT>
TE_DEV void store_row(void* y, int64_t r, const typename SpmvTr<P>::acc_t& a) {
  if constexpr (P == PREC_FDF) {
    dw v = dacc_value(a);
    if constexpr (F64OUT) static_cast<double*>(y)[r] = dw_to_double(v);
    else static_cast<float2*>(y)[r] = dw_to_f2(v);
  } else {
    static_cast<double*>(y)[r] = a;
  }
}

template <int P, bool F64OUT>
__global__ void __launch_bounds__(SPMV_THREADS) spmv_kernel(SpmvArgs a) {
  using Tr = SpmvTr<P>;
  using val_t = typename Tr::val_t;
  using x_t = typename Tr::x_t;
  using acc_t = typename Tr::acc_t;
  constexpr int TN = Tr::TNNZ;
  constexpr int ITEMS = TN / SPMV_THREADS;
  // FDF: exact products (p, e); DDD: value and gathered x
  __shared__ __align__(16) unsigned char smraw[TN * (P == PREC_FDF ? 8 : 16)];
  __shared__ acc_t red[SPMV_THREADS / 32];

  const int tid = threadIdx.x;
  const int b = blockIdx.x;
  const bool is_long = b >= a.nshort;
  int64_t k0, k1;
  int r0 = 0, r1 = 0;
  if (!is_long) {
    int2 blk = a.blocks[b];
    r0 = blk.x;
    r1 = blk.y;
    k0 = a.rp[r0];
    k1 = a.rp[r1];
  } else {
    LongChunk c = a.chunks[b - a.nshort];
    k0 = c.k0;
    k1 = c.k1;
  }
  const int nz = (int)(k1 - k0);
  const uint64_t pol = policy_evict_first();
  const int32_t* ci = a.ci + k0;
  const val_t* va = static_cast<const val_t*>(a.val) + k0;
  const x_t* x = static_cast<const x_t*>(a.x);

  // phase 1: stream (col, val), gather x, stage
  int cidx[ITEMS];
  val_t vv[ITEMS];
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    int e = j * SPMV_THREADS + tid;
    if (e < nz) {
      cidx[j] = ld_stream_i32(ci + e, pol);
      if constexpr (P == PREC_FDF) vv[j] = ld_stream_f32(va + e, pol);
      else vv[j] = ld_stream_f64(va + e, pol);
    }
  }
  x_t xv[ITEMS];
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    int e = j * SPMV_THREADS + tid;
    if (e < nz) xv[j] = __ldg(x + cidx[j]);
  }
#pragma unroll
  for (int j = 0; j < ITEMS; ++j) {
    int e = j * SPMV_THREADS + tid;
    if (e < nz) {
      if constexpr (P == PREC_FDF) {
        float p, q;
        two_prod(vv[j], xv[j], p, q);
        reinterpret_cast<float2*>(smraw)[e] = make_float2(p, q);
      } else {
        reinterpret_cast<double*>(smraw)[e] = vv[j];
        reinterpret_cast<double*>(smraw)[TN + e] = xv[j];
      }
    }
  }
  __syncthreads();

  auto add_elem = [&](acc_t& acc, int e) {
    if constexpr (P == PREC_FDF) {
      float2 pe = reinterpret_cast<const float2*>(smraw)[e];
      dacc_add_pair(acc, pe.x, pe.y);
    } else {
      acc = fma(reinterpret_cast<const double*>(smraw)[e],
                reinterpret_cast<const double*>(smraw)[TN + e], acc);
    }
  };

  if (!is_long) {
    // phase 2: rows of the block, `tpr` lanes per row
    const int R = r1 - r0;
    if (R <= 0) return;
    const int half_mean = nz / (2 * R);
    int tpr = 1;
    while (tpr < 32 && tpr * 2 <= half_mean) tpr *= 2;
    const int groups = SPMV_THREADS / tpr;
    const int g = tid / tpr, sub = tid % tpr;
    for (int base = 0; base < R; base += groups) {
      const int rr = base + g;
      const bool valid = rr < R;
      acc_t acc;
      acc_zero<P>(acc);
      if (valid) {
        const int r = r0 + rr;
        const int e0 = (int)(__ldg(a.rp + r) - k0), e1 = (int)(__ldg(a.rp + r + 1) - k0);
        for (int e = e0 + sub; e < e1; e += tpr) add_elem(acc, e);
      }
      acc = group_sum(acc, tpr);
      if (valid && sub == 0) store_row<P, F64OUT>(a.y, (int64_t)(r0 + rr), acc);
    }
  } else {
    // long-row chunk: whole-CTA sum, one partial per chunk
    acc_t acc;
    acc_zero<P>(acc);
    for (int e = tid; e < nz; e += SPMV_THREADS) add_elem(acc, e);
    acc = warp_sum(acc);
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
      acc_t t = red[0];
#pragma unroll
      for (int w = 1; w < SPMV_THREADS / 32; ++w) {
        if constexpr (P == PREC_FDF) t = dacc_merge(t, red[w]);
        else t += red[w];
      }
      const int c = b - a.nshort;
      if constexpr (P == PREC_FDF)
        static_cast<float2*>(a.lpart)[c] = dw_to_f2(dacc_value(t));
      else
        static_cast<double*>(a.lpart)[c] = t;
    }
  }
}

// one warp per long row: sum its chunk partials in order of a fixed tree
template <int P, bool F64OUT>
__global__ void spmv_long_finalize(const LongRow* lrows, int nl, const void* lpart, void* y) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= nl) return;
  LongRow lr = lrows[w];
  typename SpmvTr<P>::acc_t acc;
  acc_zero<P>(acc);
  for (int c = lane; c < lr.count; c += 32) {
    if constexpr (P == PREC_FDF) {
      float2 v = static_cast<const float2*>(lpart)[lr.first + c];
      dacc_add_pair(acc, v.x, v.y);
    } else {
      acc += static_cast<const double*>(lpart)[lr.first + c];
    }
  }
  acc = warp_sum(acc);
  if (lane == 0) store_row<P, F64OUT>(y, lr.row, acc);
}

template <int P, bool F64OUT>
static cudaError_t launch_spmv_t(const SpmvArgs& a, const DevPartition& Pt, cudaStream_t s) {
  const int grid = Pt.nshort + Pt.nchunks;
  if (grid > 0) spmv_kernel<P, F64OUT><<<grid, SPMV_THREADS, 0, s>>>(a);
  if (Pt.nlrows > 0) {
    const int threads = 256;
    const int blocks = (Pt.nlrows * 32 + threads - 1) / threads;
    spmv_long_finalize<P, F64OUT><<<blocks, threads, 0, s>>>(Pt.lrows, Pt.nlrows, Pt.lpart, a.y);
  }
  return cudaGetLastError();
}

cudaError_t launch_spmv(int prec, const int64_t* rp, const int32_t* ci, const void* val,
                        const void* x, void* y, int64_t n, const DevPartition& Pt,
                        bool out_f64, cudaStream_t s) {
  (void)n;
  SpmvArgs a;
  a.rp = rp;
  a.ci = ci;
  a.val = val;
  a.x = x;
  a.y = y;
  a.blocks = Pt.blocks;
  a.chunks = Pt.chunks;
  a.lpart = Pt.lpart;
  a.nshort = Pt.nshort;
  if (prec == PREC_DDD) return launch_spmv_t<PREC_DDD, true>(a, Pt, s);
  if (out_f64) return launch_spmv_t<PREC_FDF, true>(a, Pt, s);
  return launch_spmv_t<PREC_FDF, false>(a, Pt, s);
}

__global__ void validate_cols_kernel(const int32_t* ci, int64_t nnz, int64_t n, int* flag) {
  int bad = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x) {
    int32_t c = ci[k];
    bad |= (c < 0 || (int64_t)c >= n);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

cudaError_t launch_validate_cols(const int32_t* ci, int64_t nnz, int64_t n, int* flag,
                                 cudaStream_t s) {
  if (nnz <= 0) return cudaSuccess;
  int64_t blocks = (nnz + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  validate_cols_kernel<<<(int)blocks, 256, 0, s>>>(ci, nnz, n, flag);
  return cudaGetLastError();
}

}  // namespace te
