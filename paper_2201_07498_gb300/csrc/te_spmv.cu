// te_spmv.cu - the SpMV step of Algorithm 1 (v_t <- M v_i) for sm_103a.
//
// Partition ("CSR-stream" row blocks, after Greathouse & Daga, SC'14): the
// host packs consecutive rows into blocks of at most TNNZ non-zeros and
// SPMV_RMAX rows; a row longer than TNNZ/4 is cut into TNNZ-sized chunks whose
// partial sums a second kernel adds in order.  Every block becomes a 32-byte
// descriptor holding its non-zero range and row range.
//
// Each block's non-empty rows are also listed as 32-bit records (row offset,
// end offset), and for every thread's run the record of its first row: the
// kernel reads 4 bytes per non-empty row instead of the row pointers, and
// never touches empty rows (the caller keeps them zero).
//
// Kernel: one CTA of 256 threads per descriptor.  The block's non-zeros are
// split into aligned runs of IPT consecutive entries (IPT = 32 for binary32
// values, 16 for binary64), one run per thread, loaded in two halves with
// 128-bit vector loads marked L2 evict-first so that the gathered vector
// stays resident in L2.  Each thread gathers x[col] for its run and walks it
// once; when it crosses a row end it parks the row's sum in shared memory
// (one store and one shared load: cheap even when the lanes of a warp close
// rows at different entries).  A row that crosses thread boundaries leaves
// one partial per thread; a segmented scan (warp shuffles, then one
// cross-warp step, in a fixed order: deterministic) adds them into the
// thread that closes it.  All row sums then leave in one converged, row-order
// pass of stores.  FDF forms every product exactly as a float pair and sums in
// double-float (Dot2 of Ogita, Rump & Oishi); DDD uses binary64 FMA.  The CSR
// arrays must be 16-byte aligned.
#include <type_traits>

#include "te_common.cuh"
#include "te_internal.h"

namespace te {

template <int P>
struct SpmvTr;
// a run of IPT entries is processed as IPT/H halves of H entries
template <>
struct SpmvTr<PREC_DDD> {
  using val_t = double;
  using x_t = double;
  using acc_t = double;
  static constexpr int IPT = 16;
  static constexpr int H = 8;
  static constexpr int TNNZ = SPMV_T * IPT - IPT;  // room for the alignment of the runs
};
template <>
struct SpmvTr<PREC_FDF> {
  using val_t = float;
  using x_t = float;
  using acc_t = dacc;
  static constexpr int IPT = 32;
  static constexpr int H = 16;
  static constexpr int TNNZ = SPMV_T * IPT - IPT;
};

static int spmv_ipt(int prec) { return prec == PREC_DDD ? SpmvTr<PREC_DDD>::IPT : SpmvTr<PREC_FDF>::IPT; }

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

void make_descriptors(int prec, const Partition& P, const int64_t* rp,
                      std::vector<SpmvDesc>& out, std::vector<uint16_t>& runrow,
                      std::vector<uint32_t>& rowrec) {
  const int64_t ipt = spmv_ipt(prec);
  out.clear();
  rowrec.clear();
  out.reserve(P.blocks.size() + P.chunks.size());
  runrow.assign((P.blocks.size() + P.chunks.size()) * SPMV_T, 0);
  for (size_t b = 0; b < P.blocks.size(); ++b) {
    const int2 bl = P.blocks[b];
    SpmvDesc d;
    d.k0 = rp[bl.x];
    d.nz = (int32_t)(rp[bl.y] - rp[bl.x]);
    d.r0 = bl.x;
    d.r1 = bl.y;
    d.lslot = -1;
    d.pad_ = 0;
    d.meta = (int64_t)rowrec.size();
    for (int r = bl.x; r < bl.y; ++r)
      if (rp[r + 1] > rp[r])
        rowrec.push_back(((uint32_t)(rp[r + 1] - d.k0) << 16) | (uint32_t)(r - bl.x));
    d.nrows = (int32_t)(rowrec.size() - d.meta);
    out.push_back(d);
    // merge the runs' first entries with the row ends
    const int64_t k1 = d.k0 + d.nz, base = d.k0 / ipt * ipt;
    int j = 0;
    for (int t = 0; t < SPMV_T; ++t) {
      int64_t e = base + (int64_t)t * ipt;
      if (e < d.k0) e = d.k0;
      if (e >= k1) break;
      while (j + 1 < d.nrows && (int64_t)(rowrec[d.meta + j] >> 16) + d.k0 <= e) ++j;
      runrow[b * SPMV_T + t] = (uint16_t)j;
    }
  }
  for (size_t c = 0; c < P.chunks.size(); ++c) {
    const LongChunk& ch = P.chunks[c];
    SpmvDesc d;
    d.k0 = ch.k0;
    d.nz = (int32_t)(ch.k1 - ch.k0);
    d.r0 = ch.row;
    d.r1 = ch.row + 1;
    d.lslot = (int32_t)c;
    d.pad_ = 0;
    d.meta = (int64_t)rowrec.size();
    d.nrows = 1;  // one row: every run starts in record 0
    rowrec.push_back((uint32_t)d.nz << 16);
    out.push_back(d);
  }
}

struct SpmvArgs {
  const int64_t* rp;
  const int32_t* ci;
  const void* val;
  const void* x;
  void* y;
  const SpmvDesc* desc;
  const uint16_t* runrow;
  const uint32_t* rowrec;
  void* lpart;
  int64_t n, nnz;
  int ndesc;
};

template <int P>
TE_DEV void acc_zero(typename SpmvTr<P>::acc_t& a) {
  if constexpr (P == PREC_FDF) a = dacc_zero();
  else a = 0.0;
}
template <int P>
TE_DEV typename SpmvTr<P>::acc_t acc_add(typename SpmvTr<P>::acc_t a,
                                         typename SpmvTr<P>::acc_t b) {
  if constexpr (P == PREC_FDF) return dacc_merge(a, b);
  else return a + b;
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

// 16-byte streaming loads (no L1 allocation, L2 evict-first)
TE_DEV int4 ld_stream_v4i(const int32_t* p, uint64_t pol) {
  int4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p), "l"(pol));
  return v;
}
TE_DEV float4 ld_stream_v4f(const float* p, uint64_t pol) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p), "l"(pol));
  return v;
}
TE_DEV double2 ld_stream_v2d(const double* p, uint64_t pol) {
  double2 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;"
               : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(pol));
  return v;
}

template <int P, bool F64OUT>
__global__ void __launch_bounds__(SPMV_T, 3) spmv_kernel(SpmvArgs a) {
  using Tr = SpmvTr<P>;
  using val_t = typename Tr::val_t;
  using x_t = typename Tr::x_t;
  using acc_t = typename Tr::acc_t;
  constexpr int IPT = Tr::IPT, H = Tr::H;
  __shared__ uint16_t rend_s[SPMV_RMAX + 1];  // end offset of each non-empty row
  __shared__ uint16_t rid_s[SPMV_RMAX];       // its row offset in the block
  __shared__ acc_t outv[SPMV_RMAX];           // its sum
  __shared__ int32_t wkey[SPMV_T / 32];       // last open row record of each warp
  __shared__ acc_t wval[SPMV_T / 32];         // its partial within the warp

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const SpmvDesc d = a.desc[blockIdx.x];
  const int64_t k0 = d.k0, k1 = d.k0 + d.nz;
  const int NR = d.nrows;
  const uint64_t pol = policy_evict_first();
  const int j0 = a.runrow[(size_t)blockIdx.x * SPMV_T + tid];
  for (int j = tid; j < NR; j += SPMV_T) {
    const uint32_t rec = __ldg(a.rowrec + d.meta + j);
    rend_s[j] = (uint16_t)(rec >> 16);
    rid_s[j] = (uint16_t)(rec & 0xffffu);
  }
  if (tid == 0) rend_s[NR] = 0xffffu;  // sentinel past the last row

  // this thread's run [rs, rs + IPT), aligned to IPT entries
  const int64_t rs = (k0 / IPT) * IPT + (int64_t)tid * IPT;
  const int rel0 = (int)(rs - k0);  // block-relative position of the run's first entry
  const int lo = rel0 > 0 ? rel0 : 0;
  const int hi = rel0 + IPT < d.nz ? rel0 + IPT : d.nz;
  const bool any = lo < hi;
  const bool full = any && rel0 >= 0 && rel0 + IPT <= d.nz && rs + IPT <= a.nnz;
  const x_t* x = static_cast<const x_t*>(a.x);

  // load one half of the run (entries h0 .. h0 + H)
  auto load_half = [&](int h0, int32_t* col, val_t* val) {
    if (full) {
#pragma unroll
      for (int q = 0; q < H; q += 4) {
        int4 c4 = ld_stream_v4i(a.ci + rs + h0 + q, pol);
        col[q] = c4.x; col[q + 1] = c4.y; col[q + 2] = c4.z; col[q + 3] = c4.w;
      }
      if constexpr (P == PREC_FDF) {
#pragma unroll
        for (int q = 0; q < H; q += 4) {
          float4 v4 = ld_stream_v4f(static_cast<const float*>(a.val) + rs + h0 + q, pol);
          val[q] = v4.x; val[q + 1] = v4.y; val[q + 2] = v4.z; val[q + 3] = v4.w;
        }
      } else {
#pragma unroll
        for (int q = 0; q < H; q += 2) {
          double2 v2 = ld_stream_v2d(static_cast<const double*>(a.val) + rs + h0 + q, pol);
          val[q] = v2.x; val[q + 1] = v2.y;
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < H; ++q) {
        const int e = rel0 + h0 + q;
        if (e >= lo && e < hi) {
          col[q] = a.ci[rs + h0 + q];
          val[q] = static_cast<const val_t*>(a.val)[rs + h0 + q];
        } else {
          col[q] = -1;
          val[q] = (val_t)0;
        }
      }
    }
  };
  int32_t colA[H], colB[H];
  val_t valA[H], valB[H];
  x_t xA[H], xB[H];
  if (any) {
    load_half(0, colA, valA);
    load_half(H, colB, valB);
  }
  // all gathers of the run go out before any of them is consumed
#pragma unroll
  for (int q = 0; q < H; ++q) {
    xA[q] = (any && (full || colA[q] >= 0)) ? __ldg(x + colA[q]) : (x_t)0;
    xB[q] = (any && (full || colB[q] >= 0)) ? __ldg(x + colB[q]) : (x_t)0;
  }
  __syncthreads();  // row records complete

  // walk the run once; a row that ends inside it stores its (partial) sum in
  // outv; the first row may have begun in an earlier run (it is completed
  // after the scan), the last may continue into a later one (it is scanned)
  int j = j0;
  int rend = any ? rend_s[j] : 0xffff;
  const int rstart0 = (any && j > 0) ? rend_s[j - 1] : 0;
  const bool cont = any && rstart0 < lo;  // the first row began in an earlier run
  bool head_closed = false;               // ... and ends in this run
  acc_t acc;
  acc_zero<P>(acc);
  auto walk = [&](int h0, const val_t* val, const x_t* xv, auto fullc) {
    constexpr bool FULL = decltype(fullc)::value;
#pragma unroll
    for (int q = 0; q < H; ++q) {
      const int e = rel0 + h0 + q;
      if (FULL || (e >= lo && e < hi)) {
        if constexpr (P == PREC_FDF) {
          float p, pe;
          two_prod(val[q], xv[q], p, pe);
          dacc_add_pair(acc, p, pe);
        } else {
          acc = fma(val[q], xv[q], acc);
        }
        if (e + 1 == rend) {  // the row ends here
          outv[j] = acc;
          if (j == j0 && cont) {
            head_closed = true;
            rid_s[j] = 0xffffu;  // completed below by this thread, not by the store loop
          }
          acc_zero<P>(acc);
          rend = rend_s[++j];
        }
      }
    }
  };
  if (any) {
    if (full) {
      walk(0, valA, xA, std::true_type{});
      walk(H, valB, xB, std::true_type{});
    } else {
      walk(0, valA, xA, std::false_type{});
      walk(H, valB, xB, std::false_type{});
    }
  }
  // the row left open at the end of the run (it began in this run or earlier)
  int open_key = -1;
  acc_t open_acc;
  acc_zero<P>(open_acc);
  if (any && j < NR && (j > 0 ? (int)rend_s[j - 1] : 0) < hi) {
    open_key = j;
    open_acc = acc;
  }

  // segmented inclusive scan of the open partials (equal keys are contiguous)
#pragma unroll
  for (int dlt = 1; dlt < 32; dlt <<= 1) {
    const int k2 = __shfl_up_sync(0xffffffffu, open_key, dlt);
    acc_t v2;
    if constexpr (P == PREC_FDF) {
      v2.s = __shfl_up_sync(0xffffffffu, open_acc.s, dlt);
      v2.c = __shfl_up_sync(0xffffffffu, open_acc.c, dlt);
    } else {
      v2 = __shfl_up_sync(0xffffffffu, open_acc, dlt);
    }
    if (lane >= dlt && open_key >= 0 && k2 == open_key) open_acc = acc_add<P>(v2, open_acc);
  }
  if (lane == 31) {
    wkey[wid] = open_key;
    wval[wid] = open_acc;
  }
  __syncthreads();
  // carry from earlier warps into this warp's first open row (nearest first)
  const int kin = wid > 0 ? wkey[wid - 1] : -1;
  acc_t carry;
  acc_zero<P>(carry);
  if (kin >= 0) {
    carry = wval[wid - 1];
    for (int w = wid - 2; w >= 0 && wkey[w] == kin; --w) carry = acc_add<P>(wval[w], carry);
  }
  if (open_key >= 0 && open_key == kin) open_acc = acc_add<P>(carry, open_acc);
  // the thread that closes a row begun earlier adds the partials ending at tid - 1
  int kprev = __shfl_up_sync(0xffffffffu, open_key, 1);
  acc_t vprev;
  if constexpr (P == PREC_FDF) {
    vprev.s = __shfl_up_sync(0xffffffffu, open_acc.s, 1);
    vprev.c = __shfl_up_sync(0xffffffffu, open_acc.c, 1);
  } else {
    vprev = __shfl_up_sync(0xffffffffu, open_acc, 1);
  }
  if (lane == 0) {  // thread tid - 1 is the last lane of the previous warp
    kprev = kin;
    vprev = carry;
  }
  auto emit = [&](int jj, int row_off, const acc_t& v) {
    if (d.lslot >= 0) {
      if constexpr (P == PREC_FDF)
        static_cast<float2*>(a.lpart)[d.lslot] = dw_to_f2(dacc_value(v));
      else
        static_cast<double*>(a.lpart)[d.lslot] = v;
    } else {
      store_row<P, F64OUT>(a.y, (int64_t)d.r0 + row_off, v);
    }
    (void)jj;
  };
  if (cont && head_closed) {
    acc_t t = outv[j0];
    if (kprev == j0) t = acc_add<P>(vprev, t);
    // the row offset of record j0 was overwritten with the skip marker
    const int row_off = (int)(__ldg(a.rowrec + d.meta + j0) & 0xffffu);
    emit(j0, row_off, t);
  }
  // every other row sum of the block, stored in row order
  for (int jj = tid; jj < NR; jj += SPMV_T) {
    const int row_off = rid_s[jj];
    if (row_off != 0xffff) emit(jj, row_off, outv[jj]);
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
  if (Pt.ndesc > 0) spmv_kernel<P, F64OUT><<<Pt.ndesc, SPMV_T, 0, s>>>(a);
  if (Pt.nlrows > 0) {
    const int threads = 256;
    const int blocks = (Pt.nlrows * 32 + threads - 1) / threads;
    spmv_long_finalize<P, F64OUT><<<blocks, threads, 0, s>>>(Pt.lrows, Pt.nlrows, Pt.lpart, a.y);
  }
  return cudaGetLastError();
}

cudaError_t spmv_prepare() { return cudaSuccess; }

cudaError_t launch_spmv(int prec, const int64_t* rp, const int32_t* ci, const void* val,
                        const void* x, void* y, int64_t n, int64_t nnz, const DevPartition& Pt,
                        bool out_f64, cudaStream_t s) {
  SpmvArgs a;
  a.rp = rp;
  a.ci = ci;
  a.val = val;
  a.x = x;
  a.y = y;
  a.desc = Pt.desc;
  a.runrow = Pt.runrow;
  a.rowrec = Pt.rowrec;
  a.lpart = Pt.lpart;
  a.n = n;
  a.nnz = nnz;
  a.ndesc = Pt.ndesc;
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
