// te_spmv.cu - the SpMV step of Algorithm 1 (v_t <- M v_i) for sm_103a.
//
// Layout: SELL-C-sigma (Kreutzer, Hager, Wellein, Fehske & Bishop, SIAM J.
// Sci. Comput. 36(5), 2014), built once per matrix by the plan.  Rows are cut
// into pieces of at most SELL_VMAX entries; within every window of SELL_WINDOW
// consecutive rows the pieces are sorted by length (longest first, a counting
// sort) and grouped into slices of SELL_C = 32, one warp per slice, one lane
// per piece.  A slice stores its column indices and values column-major
// (entry k of lane i at base + 32 k + i) padded with zero values to the
// length of its longest piece; sorting keeps that padding small even on
// power-law graphs, and keeping the sort inside windows keeps the row writes
// local.  The plan keeps this copy in HBM and the solve never re-reads the
// caller's CSR.  The arrangement (slices, lanes, cut rows) is computed on the
// device (te_layout_dev.cu) for a plan's device-resident copy, otherwise on
// the host (te_layout.cu: host-streamed matrices, autotuned plans, serving
// requests); the kernels below fill it with column indices and values.
//
// Kernel: a warp streams its slice with coalesced 128-byte loads (marked L2
// evict-first so that the gathered vector stays resident in L2), gathers
// x[col] and accumulates one piece per lane: no row-boundary logic, no
// shared memory, no barriers, every lane busy.  FDF forms each product exactly
// as a float pair and sums in double-float (Dot2 of Ogita, Rump & Oishi); DDD
// uses binary64 FMA.  Pieces of a cut row leave partial sums that a second
// kernel adds in piece order (deterministic).
#include "te_common.cuh"
#include "te_internal.h"

namespace te {

// Vin -> Vout: binary64 -> binary32 rounds to nearest even (__double2float_rn)
template <typename Vin, typename Vout>
TE_DEV Vout convert_value(Vin v) {
  if constexpr (sizeof(Vin) == 8 && sizeof(Vout) == 4) return __double2float_rn(v);
  else return (Vout)v;
}

// Device fill of the SELL arrays, a warp per slice, lane i walking its own
// piece (a contiguous run of the CSR) entry after entry and storing entry k
// of the slice's 32 lanes with one coalesced store (entry k of lane i at
// base + 32 k + i; padding: column 0, value 0).  A lane's successive loads
// fall in the sector its previous load brought into L1.  No shared memory
// and 32 registers: 64 warps per SM keep loads in flight (a shared-memory
// transpose tile with coalesced loads ran no faster at R-MAT 2^24 and
// allowed a third of the warps).  Columns and values are filled by separate
// kernels so that each can start as soon as its CSR array has arrived.
// Columns go through colmap when the rows are relabelled; values are
// converted on the way (binary64 -> binary32 rounds to nearest even).  A
// non-zero *bad (the column check found an index outside [0, n), earlier on
// the stream) makes both kernels return at once: colmap is never indexed
// with such a column.
constexpr int SELL_FILL_WARPS = 8;

__global__ void __launch_bounds__(32 * SELL_FILL_WARPS, 8)
    sell_fill_cols_kernel(const int32_t* ci, const SellSlice* slices, const int64_t* vsrc,
                          const int32_t* vlen, int nslices, int32_t* cols,
                          const int32_t* colmap, const int* bad) {
  if (bad && *bad) return;
  const int lane = threadIdx.x & 31;
  const int64_t s = (int64_t)blockIdx.x * SELL_FILL_WARPS + (threadIdx.x >> 5);
  if (s >= nslices) return;  // uniform per warp
  const SellSlice sl = slices[s];
  const int64_t t = s * SELL_C + lane;
  const int32_t* cp = ci + vsrc[t];
  const int my_len = vlen[t];
  int32_t* co = cols + sl.base + lane;
#pragma unroll 4
  for (int k = 0; k < sl.len; ++k) {
    int32_t c = 0;
    if (k < my_len) {
      const int32_t c0 = cp[k];
      c = colmap ? colmap[c0] : c0;
    }
    __stcs(co + (int64_t)k * SELL_C, c);
  }
}

template <typename Vin, typename Vout>
__global__ void __launch_bounds__(32 * SELL_FILL_WARPS, 8)
    sell_fill_vals_kernel(const Vin* val, const SellSlice* slices, const int64_t* vsrc,
                          const int32_t* vlen, int nslices, Vout* vals, const int32_t* vrow,
                          const float* row_scale, float* lane_scale, const int* bad) {
  if (bad && *bad) return;
  const int lane = threadIdx.x & 31;
  const int64_t s = (int64_t)blockIdx.x * SELL_FILL_WARPS + (threadIdx.x >> 5);
  if (s >= nslices) return;  // uniform per warp
  const SellSlice sl = slices[s];
  const int64_t t = s * SELL_C + lane;
  const Vin* vp = val + vsrc[t];
  const int my_len = vlen[t];
  if (lane_scale) {
    const int32_t r = vrow[t];
    lane_scale[t] = r >= 0 ? row_scale[r] : 0.f;
  }
  Vout* vo = vals + sl.base + lane;
#pragma unroll 4
  for (int k = 0; k < sl.len; ++k) {
    Vout v = (Vout)0;
    if (k < my_len) v = convert_value<Vin, Vout>(vp[k]);
    __stcs(vo + (int64_t)k * SELL_C, v);
  }
}

cudaError_t launch_sell_fill_cols(const int32_t* ci, const SellSlice* slices, const int64_t* vsrc,
                                  const int32_t* vlen, int nslices, int32_t* cols,
                                  const int32_t* colmap, const int* bad, cudaStream_t s) {
  if (nslices <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)(((int64_t)nslices + SELL_FILL_WARPS - 1) / SELL_FILL_WARPS);
  sell_fill_cols_kernel<<<blocks, 32 * SELL_FILL_WARPS, 0, s>>>(ci, slices, vsrc, vlen, nslices,
                                                                cols, colmap, bad);
  return cudaGetLastError();
}

cudaError_t launch_sell_fill_vals(int in_type, int out_type, const void* val,
                                  const SellSlice* slices, const int64_t* vsrc,
                                  const int32_t* vlen, int nslices, void* vals,
                                  const int32_t* vrow, const float* row_scale, float* lane_scale,
                                  const int* bad, cudaStream_t s) {
  if (nslices <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)(((int64_t)nslices + SELL_FILL_WARPS - 1) / SELL_FILL_WARPS);
#define TE_FILL(IN, OUT, TI, TO)                                                              \
  if (in_type == IN && out_type == OUT) {                                                    \
    sell_fill_vals_kernel<TI, TO><<<blocks, 32 * SELL_FILL_WARPS, 0, s>>>(                   \
        static_cast<const TI*>(val), slices, vsrc, vlen, nslices, static_cast<TO*>(vals),    \
        vrow, row_scale, lane_scale, bad);                                                   \
    return cudaGetLastError();                                                               \
  }
  TE_FILL(TE_F64, TE_F64, double, double)
  TE_FILL(TE_F64, TE_F32, double, float)
  TE_FILL(TE_F32, TE_F32, float, float)
  TE_FILL(TE_BF16, TE_BF16, uint16_t, uint16_t)
  TE_FILL(TE_FP8_E4M3, TE_FP8_E4M3, uint8_t, uint8_t)
#undef TE_FILL
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// the SpMV kernel
// ---------------------------------------------------------------------------
template <int P>
struct SpmvTr;
template <>
struct SpmvTr<PREC_DDD> {
  using val_t = double;
  using x_t = double;
  using acc_t = double;
};
template <>
struct SpmvTr<PREC_FDF> {
  using val_t = float;
  using x_t = float;
  using acc_t = dacc;
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

struct SpmvArgs {
  const SellSlice* slices;
  const int32_t* vout;
  const int32_t* cols;
  const void* vals;
  const float* lscale;  // FP8: per-lane scale
  int64_t ebase;        // first layout entry held by cols/vals
  const void* x;
  void* y;
  void* vpart;
  int nslices;
  int hot;  // gathers of x[c], c >= hot, skip L1 allocation (0: all allocate)
};

constexpr int SPMV_WPB = 8;     // warps (slices) per CTA
// with rows relabelled by degree, the first HOT_BYTES of x (the most
// connected columns) are the ones L1 keeps
constexpr int64_t HOT_BYTES = 128 << 10;
constexpr int SPMV_UNROLL = 8;  // entries per lane in flight

// stored matrix value type per te_dtype, and its streaming load + exact
// conversion to the arithmetic's input type
template <int VK>
struct VStore;
template <>
struct VStore<TE_F64> {
  using t = double;
};
template <>
struct VStore<TE_F32> {
  using t = float;
};
template <>
struct VStore<TE_BF16> {
  using t = uint16_t;
};
template <>
struct VStore<TE_FP8_E4M3> {
  using t = uint8_t;
};
template <int VK>
TE_DEV auto load_value(const typename VStore<VK>::t* p, uint64_t pol) {
  if constexpr (VK == TE_F64) return ld_stream_f64(p, pol);
  else if constexpr (VK == TE_F32) return ld_stream_f32(p, pol);
  else if constexpr (VK == TE_BF16) return bf16_to_f32(ld_stream_u16(p, pol));
  else return e4m3_to_f32(ld_stream_u8(p, pol));
}

// Reduced-precision values (BF16, FP8 codes) are exact binary32 numbers, so
// the FDF arithmetic (exact products, double-float sums) is unchanged; FP8
// rows are summed over their codes and multiplied by the row scale at the end.
// one warp sums one slice (lane = one piece); the serving engine's batched
// SpMV runs the same body on the slices of several solves
template <int P, int VK, bool F64OUT>
__device__ __forceinline__ void spmv_slice(const SpmvArgs& a, const int slice, const int lane) {
  using Tr = SpmvTr<P>;
  using val_t = typename Tr::val_t;
  using x_t = typename Tr::x_t;
  using acc_t = typename Tr::acc_t;
  using store_t = typename VStore<VK>::t;
  const SellSlice sl = a.slices[slice];
  const int32_t out = a.vout[(int64_t)slice * SELL_C + lane];
  const uint64_t pol = policy_evict_first();
  const uint64_t keep = policy_evict_last();
  const int32_t* cp = a.cols + (sl.base - a.ebase) + lane;
  const store_t* vp = static_cast<const store_t*>(a.vals) + (sl.base - a.ebase) + lane;
  const x_t* x = static_cast<const x_t*>(a.x);
  acc_t acc0, acc1;
  acc_zero<P>(acc0);
  acc_zero<P>(acc1);
  auto add = [&](acc_t& acc, val_t v, x_t xv) {
    if constexpr (P == PREC_FDF) {
      float p, e;
      two_prod(v, xv, p, e);
      dacc_add_pair(acc, p, e);
    } else {
      acc = fma(v, xv, acc);
    }
  };
  // chunks of SPMV_UNROLL entries per lane; all loads of a chunk go out
  // before its gathers, and the tail of a slice is a predicated chunk
  for (int k = 0; k < sl.len; k += SPMV_UNROLL) {
    int32_t c[SPMV_UNROLL];
    val_t v[SPMV_UNROLL];
#pragma unroll
    for (int u = 0; u < SPMV_UNROLL; ++u) {
      const bool ok = k + u < sl.len;
      c[u] = ok ? ld_stream_i32(cp + (int64_t)(k + u) * SELL_C, pol) : 0;
      v[u] = ok ? (val_t)load_value<VK>(vp + (int64_t)(k + u) * SELL_C, pol) : (val_t)0;
    }
    x_t xv[SPMV_UNROLL];
#pragma unroll
    for (int u = 0; u < SPMV_UNROLL; ++u) {  // padding reads x[0]
      if (a.hot > 0) {  // uniform: cold columns leave L1 to the hot ones
        const bool h = c[u] < a.hot;
        if constexpr (sizeof(x_t) == 4)
          xv[u] = ld_keep_f32_if<true>(x + c[u], h, keep) + ld_keep_f32_if<false>(x + c[u], !h, keep);
        else
          xv[u] = ld_keep_f64_if<true>(x + c[u], h, keep) + ld_keep_f64_if<false>(x + c[u], !h, keep);
      } else {
        if constexpr (sizeof(x_t) == 4) xv[u] = ld_keep_f32(x + c[u], keep);
        else xv[u] = ld_keep_f64(x + c[u], keep);
      }
    }
#pragma unroll
    for (int u = 0; u < SPMV_UNROLL; u += 2) {
      add(acc0, v[u], xv[u]);
      add(acc1, v[u + 1], xv[u + 1]);
    }
  }
  if constexpr (P == PREC_FDF) {
    dw r = dacc_value(dacc_merge(acc0, acc1));
    if constexpr (VK == TE_FP8_E4M3)
      r = dw_mul(r, dw{a.lscale[(int64_t)slice * SELL_C + lane], 0.f});
    if (out >= 0) {
      if constexpr (F64OUT) static_cast<double*>(a.y)[out] = dw_to_double(r);
      else static_cast<float2*>(a.y)[out] = dw_to_f2(r);
    } else if (out != SELL_SKIP) {
      static_cast<float2*>(a.vpart)[-1 - (int64_t)out] = dw_to_f2(r);
    }
  } else {
    const double r = acc0 + acc1;
    if (out >= 0) static_cast<double*>(a.y)[out] = r;
    else if (out != SELL_SKIP) static_cast<double*>(a.vpart)[-1 - (int64_t)out] = r;
  }
}

template <int P, int VK, bool F64OUT>
__global__ void __launch_bounds__(32 * SPMV_WPB) spmv_kernel(SpmvArgs a) {
  const int slice = blockIdx.x * SPMV_WPB + (threadIdx.x >> 5);
  if (slice >= a.nslices) return;
  spmv_slice<P, VK, F64OUT>(a, slice, threadIdx.x & 31);
}

// Cut rows: the first nbig rows (most pieces first) get a whole warp each:
// each lane sums a strided subset of the row's piece partials, then a fixed
// shuffle tree adds the lanes.  Every other row (at most SELL_BIG_PIECES
// pieces, most have a handful) gets one thread, which loads all its
// partials at once and sums them in the same fixed order as FIN_G lanes
// would: chain s takes pieces s, s + FIN_G, ..., then the chains are added
// as the xor tree over FIN_G lanes adds them, ((0, 2), (1, 3)).  The order
// is fixed, so the result is deterministic.
constexpr int FIN_G = 4;
constexpr int FIN_PF = 8;  // partial loads in flight per lane of a whole-warp row
static_assert(FIN_G == 4, "the per-thread merge order below is the xor tree of four lanes");
template <int P>
using part_t = typename std::conditional<P == PREC_FDF, float2, double>::type;
template <int P>
TE_DEV void acc_add_partial(typename SpmvTr<P>::acc_t& acc, const part_t<P>& v) {
  if constexpr (P == PREC_FDF) dacc_add_pair(acc, v.x, v.y);
  else acc += v;
}
template <int P>
TE_DEV typename SpmvTr<P>::acc_t acc_join(const typename SpmvTr<P>::acc_t& a,
                                         const typename SpmvTr<P>::acc_t& b) {
  if constexpr (P == PREC_FDF) return dacc_merge(a, b);
  else return a + b;
}

template <int P, bool F64OUT>
__global__ void spmv_long_finalize(const LongRow* lrows, int nl, int nbig, int big_blocks,
                                   const void* vpart, void* y) {
  using acc_t = typename SpmvTr<P>::acc_t;
  const part_t<P>* vp = static_cast<const part_t<P>*>(vpart);
  if ((int)blockIdx.x < big_blocks) {  // uniform per block
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int sub = threadIdx.x & 31;
    const bool live = g < nbig;  // every lane reaches the shuffles below
    LongRow lr{0, 0, 0, 0};
    if (live) lr = lrows[g];
    acc_t acc;
    acc_zero<P>(acc);
    // the lane's pieces in order, FIN_PF loads in flight (the most connected
    // rows have thousands of pieces, so the lanes' chains set the kernel's end)
    for (int c0 = sub; c0 < lr.count; c0 += 32 * FIN_PF) {
      part_t<P> v[FIN_PF];
#pragma unroll
      for (int u = 0; u < FIN_PF; ++u)
        if (c0 + 32 * u < lr.count) v[u] = vp[(int64_t)lr.first + c0 + 32 * u];
#pragma unroll
      for (int u = 0; u < FIN_PF; ++u)
        if (c0 + 32 * u < lr.count) acc_add_partial<P>(acc, v[u]);
    }
    acc = group_sum(acc, 32);
    if (live && sub == 0) store_row<P, F64OUT>(y, lr.row, acc);
    return;
  }
  const int64_t g = nbig + (int64_t)(blockIdx.x - big_blocks) * blockDim.x + threadIdx.x;
  if (g >= nl) return;
  const LongRow lr = lrows[g];
  part_t<P> v[SELL_BIG_PIECES];
#pragma unroll
  for (int c = 0; c < SELL_BIG_PIECES; ++c)
    if (c < lr.count) v[c] = vp[(int64_t)lr.first + c];
  acc_t ch[FIN_G];
#pragma unroll
  for (int q = 0; q < FIN_G; ++q) acc_zero<P>(ch[q]);
#pragma unroll
  for (int c = 0; c < SELL_BIG_PIECES; ++c)
    if (c < lr.count) acc_add_partial<P>(ch[c % FIN_G], v[c]);
  const acc_t acc = acc_join<P>(acc_join<P>(ch[0], ch[2]), acc_join<P>(ch[1], ch[3]));
  store_row<P, F64OUT>(y, lr.row, acc);
}

template <int P, int VK, bool F64OUT>
static cudaError_t launch_spmv_t(const SpmvArgs& a, const DevSell& S, cudaStream_t s) {
  if (S.nslices > 0)
    spmv_kernel<P, VK, F64OUT><<<(S.nslices + SPMV_WPB - 1) / SPMV_WPB, 32 * SPMV_WPB, 0, s>>>(a);
  if (S.nlrows > 0) {
    const int threads = 256;
    const int big_blocks = (int)(((int64_t)S.nlbig * 32 + threads - 1) / threads);
    const int small_blocks = (int)(((int64_t)(S.nlrows - S.nlbig) + threads - 1) / threads);
    spmv_long_finalize<P, F64OUT><<<big_blocks + small_blocks, threads, 0, s>>>(
        S.lrows, S.nlrows, S.nlbig, big_blocks, S.vpart, a.y);
  }
  return cudaGetLastError();
}

cudaError_t spmv_prepare() { return cudaSuccess; }

// ---------------------------------------------------------------------------
// serving engine: the SpMV of every live solve in one launch.  Warps walk the
// concatenated slice lists (a warp finds its solve from the prefix offsets);
// x is the solve's current basis column, y its ytilde.  Each slice is summed
// exactly as in the single-solve kernel, so a solve's result does not depend
// on which other solves share the launch.
// ---------------------------------------------------------------------------
TE_DEV int find_slot(const int64_t* off, int nslots, int64_t g) {
  int lo = 0, hi = nslots - 1;  // the last slot whose offset is <= g
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// the step's table (offsets and slot records) in shared memory: each warp
// looks up the solve of every slice it takes, so the lookups stay on chip
struct BatchCache {
  int64_t off[SRV_MAX_SLOTS + 1];
  BatchSlot slot[SRV_MAX_SLOTS];
};
static_assert(sizeof(BatchSlot) % 8 == 0, "slot records are copied as 8-byte words");
TE_DEV int load_batch_cache(BatchCache& c, const BatchTable* T, const int64_t* off) {
  const int ns = T->nslots;
  for (int i = threadIdx.x; i <= ns; i += blockDim.x) c.off[i] = off[i];
  const uint64_t* src = reinterpret_cast<const uint64_t*>(T->slot);
  uint64_t* dst = reinterpret_cast<uint64_t*>(c.slot);
  const int words = ns * (int)(sizeof(BatchSlot) / 8);
  for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  return ns;
}

__global__ void __launch_bounds__(32 * SPMV_WPB) batch_spmv_kernel(const BatchTable* T) {
  __shared__ BatchCache c;
  const int lane = threadIdx.x & 31;
  const int ns = load_batch_cache(c, T, T->slice_off);
  const int64_t total = c.off[ns];
  for (int64_t g = (int64_t)blockIdx.x * SPMV_WPB + (threadIdx.x >> 5); g < total;
       g += (int64_t)gridDim.x * SPMV_WPB) {
    const int sidx = find_slot(c.off, ns, g);
    const BatchSlot& B = c.slot[sidx];
    SpmvArgs a;
    a.slices = B.slices;
    a.vout = B.vout;
    a.cols = B.cols;
    a.vals = B.vals;
    a.lscale = nullptr;
    a.ebase = 0;
    a.x = static_cast<const float*>(B.V) + (size_t)B.step * (size_t)B.n_pad;
    a.y = B.ytil;
    a.vpart = B.vpart;
    a.nslices = B.nslices;
    a.hot = 0;
    const int slice = (int)(g - c.off[sidx]);
    if (B.vk == TE_BF16) spmv_slice<PREC_FDF, TE_BF16, false>(a, slice, lane);
    else spmv_slice<PREC_FDF, TE_F32, false>(a, slice, lane);
  }
}

// cut rows of every live solve, FIN_G lanes per row; the loop runs whole
// warps so that every lane reaches the shuffles
__global__ void batch_finalize_kernel(const BatchTable* T) {
  __shared__ BatchCache c;
  const int ns = load_batch_cache(c, T, T->lrow_off);
  const int64_t total = c.off[ns];
  const int lane = threadIdx.x & 31, sub = lane & (FIN_G - 1);
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 / FIN_G);
       w0 < total; w0 += warps * (32 / FIN_G)) {
    const int64_t g = w0 + lane / FIN_G;
    const bool live = g < total;
    LongRow lr{0, 0, 0, 0};
    const BatchSlot* B = nullptr;
    if (live) {
      const int sidx = find_slot(c.off, ns, g);
      B = &c.slot[sidx];
      lr = B->lrows[g - c.off[sidx]];
    }
    dacc acc = dacc_zero();
    for (int c = sub; c < lr.count; c += FIN_G) {
      const float2 v = static_cast<const float2*>(B->vpart)[lr.first + c];
      dacc_add_pair(acc, v.x, v.y);
    }
    acc = group_sum(acc, FIN_G);
    if (live && sub == 0) static_cast<float2*>(B->ytil)[lr.row] = dw_to_f2(dacc_value(acc));
  }
}

// persistent grids that fit on the GPU at once (a grid larger than that
// leaves a second wave of blocks to start after the first ones finish)
cudaError_t batch_spmv_grids(int num_sms, int* spmv_blocks, int* fin_blocks) {
  int a = 0, b = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, batch_spmv_kernel,
                                                                32 * SPMV_WPB, 0);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, batch_finalize_kernel, 256, 0);
  if (e != cudaSuccess) return e;
  *spmv_blocks = std::max(a, 1) * num_sms;
  *fin_blocks = std::max(b, 1) * num_sms;
  return cudaSuccess;
}

cudaError_t launch_batch_spmv(const BatchTable* T, int spmv_blocks, int fin_blocks,
                              cudaStream_t s) {
  batch_spmv_kernel<<<spmv_blocks, 32 * SPMV_WPB, 0, s>>>(T);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  batch_finalize_kernel<<<fin_blocks, 256, 0, s>>>(T);
  return cudaGetLastError();
}

cudaError_t launch_spmv(int prec, const DevSell& S, const void* x, void* y, bool out_f64,
                        cudaStream_t s) {
  SpmvArgs a;
  a.slices = S.slices;
  a.vout = S.vout;
  a.cols = S.cols;
  a.vals = S.vals;
  a.lscale = S.lscale;
  a.ebase = S.ebase;
  a.x = x;
  a.y = y;
  a.vpart = S.vpart;
  a.nslices = S.nslices;
  a.hot = (int)std::min<int64_t>(S.hot, (int64_t)(HOT_BYTES / (prec == PREC_DDD ? 8 : 4)));
  if (prec == PREC_DDD) {
    if (S.vk == TE_F64) return launch_spmv_t<PREC_DDD, TE_F64, true>(a, S, s);
    if (S.vk == TE_F32) return launch_spmv_t<PREC_DDD, TE_F32, true>(a, S, s);
    return cudaErrorInvalidValue;
  }
#define TE_SPMV_FDF(VK)                                              \
  if (S.vk == VK) {                                                  \
    if (out_f64) return launch_spmv_t<PREC_FDF, VK, true>(a, S, s);  \
    return launch_spmv_t<PREC_FDF, VK, false>(a, S, s);              \
  }
  TE_SPMV_FDF(TE_F32)
  TE_SPMV_FDF(TE_BF16)
  TE_SPMV_FDF(TE_FP8_E4M3)
#undef TE_SPMV_FDF
  return cudaErrorInvalidValue;
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
