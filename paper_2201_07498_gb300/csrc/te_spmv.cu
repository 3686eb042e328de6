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
// caller's CSR.
//
// Kernel: a warp streams its slice with coalesced 128-byte loads (marked L2
// evict-first so that the gathered vector stays resident in L2), gathers
// x[col] and accumulates one piece per lane: no row-boundary logic, no
// shared memory, no barriers, every lane busy.  FDF forms each product exactly
// as a float pair and sums in double-float (Dot2 of Ogita, Rump & Oishi); DDD
// uses binary64 FMA.  Pieces of a cut row leave partial sums that a second
// kernel adds in piece order (deterministic).
#include <algorithm>
#include <atomic>
#include <thread>

#include "te_common.cuh"
#include "te_internal.h"

namespace te {

// Windows of rows [w0, w1) into `out`, with entry offsets and cut-row piece
// slots numbered from 0 (the caller shifts them).  Row r of the layout is CSR
// row ord->perm[r] (ord NULL: row r); it writes output r.
static void sell_windows(const int64_t* rp, int64_t n, int64_t w0, int64_t w1, int window,
                         int vmax, const RowOrder* ord, SellHost& out) {
  struct Piece {
    int64_t src;
    int32_t len, out, row;
  };
  std::vector<Piece> win, sorted;
  std::vector<int64_t> pos((size_t)vmax + 2);
  for (int64_t w = w0; w < w1; ++w) {
    const int64_t r0 = w * window, r1 = std::min<int64_t>(r0 + window, n);
    win.clear();
    for (int64_t r = r0; r < r1; ++r) {
      const int64_t o = ord ? (int64_t)ord->perm[r] : r;  // the CSR row
      const int64_t first = ord ? ord->src[r] : rp[r];
      const int64_t L = ord ? (int64_t)ord->len[r] : rp[r + 1] - rp[r];
      if (L == 0) continue;  // empty rows: never written by the kernel
      if (L <= vmax) {
        win.push_back({first, (int32_t)L, (int32_t)r, (int32_t)o});
        continue;
      }
      LongRow lr;
      lr.row = (int32_t)r;
      lr.first = (int32_t)out.pieces;
      lr.count = (int32_t)((L + vmax - 1) / vmax);
      lr.pad_ = 0;
      for (int32_t c = 0; c < lr.count; ++c) {
        const int64_t s0 = first + (int64_t)c * vmax;
        const int64_t l = std::min<int64_t>(vmax, first + L - s0);
        win.push_back({s0, (int32_t)l, -1 - (int32_t)(out.pieces + c), (int32_t)o});
      }
      out.pieces += lr.count;
      out.lrows.push_back(lr);
    }
    if (win.empty()) continue;
    // stable counting sort by length, longest first
    std::fill(pos.begin(), pos.end(), 0);
    for (const Piece& p : win) ++pos[p.len];
    int64_t acc = 0;
    for (int L = vmax; L >= 1; --L) {
      const int64_t c = pos[L];
      pos[L] = acc;
      acc += c;
    }
    sorted.assign(win.size(), Piece{0, 0, 0, 0});
    for (const Piece& p : win) sorted[pos[p.len]++] = p;
    // slices of SELL_C lanes
    for (size_t i = 0; i < sorted.size(); i += SELL_C) {
      SellSlice sl;
      sl.base = out.entries;
      sl.len = sorted[i].len;
      sl.pad_ = 0;
      out.slices.push_back(sl);
      for (int l = 0; l < SELL_C; ++l) {
        if (i + l < sorted.size()) {
          out.vout.push_back(sorted[i + l].out);
          out.vsrc.push_back(sorted[i + l].src);
          out.vlen.push_back(sorted[i + l].len);
          out.vrow.push_back(sorted[i + l].row);
        } else {
          out.vout.push_back(SELL_SKIP);
          out.vsrc.push_back(0);
          out.vlen.push_back(0);
          out.vrow.push_back(-1);
        }
      }
      out.entries += (int64_t)SELL_C * sl.len;
    }
  }
}

// Threads take chunks of consecutive windows from a shared counter (the work
// of a window grows with its rows' lengths, so a row order that puts the
// longest rows first would leave one static range with most of it); the
// chunks' parts are joined in chunk order with their entry and piece
// offsets, so the result equals a sequential build.  The row pointers are
// checked (all rows) before any window is built.
bool make_sell(const int64_t* rp, int64_t n, int64_t nnz, SellHost& out, std::string& err,
               int window, int vmax, const RowOrder* ord) {
  out = SellHost();
  if (rp[0] != 0) {
    err = "row_ptr[0] must be 0";
    return false;
  }
  if (rp[n] != nnz) {
    err = "row_ptr[n] != nnz";
    return false;
  }
  const int64_t W = (n + window - 1) / window;
  unsigned nt = std::thread::hardware_concurrency();
  if (nt < 1) nt = 1;
  if (nt > 32) nt = 32;
  if ((int64_t)nt > W / 16) nt = (unsigned)std::max<int64_t>(1, W / 16);
  const int64_t nc = nt == 1 ? 1 : std::min<int64_t>(W, (int64_t)nt * 16);  // chunks
  std::vector<int64_t> bad(nt, -1);
  std::vector<SellHost> part((size_t)nc);
  std::vector<int64_t> cw((size_t)nc + 1, 0);  // chunk c: windows [cw[c], cw[c+1])
  std::atomic<int64_t> next{0};
  // the row pointers (all rows) and, for several chunks, the work of each
  // window in one pass
  std::vector<int64_t> wwork(nc > 1 ? (size_t)W : 0, 0);
  auto check = [&](unsigned t) {
    const int64_t w0 = W * t / nt, w1 = W * (t + 1) / nt;
    for (int64_t w = w0; w < w1; ++w) {
      const int64_t r0 = w * window, r1 = std::min<int64_t>(r0 + window, n);
      for (int64_t r = r0; r < r1; ++r)
        if (rp[r + 1] < rp[r]) {
          bad[t] = r;
          return;
        }
      if (nc > 1) {  // the work of a window ~ its pieces ~ rows + entries / vmax
        int64_t e = 0;
        if (ord) {
          for (int64_t r = r0; r < r1; ++r) e += ord->len[r];
        } else {
          e = rp[r1] - rp[r0];
        }
        wwork[(size_t)w] = (r1 - r0) + e / vmax;
      }
    }
  };
  auto work = [&](unsigned) {
    for (int64_t c = next++; c < nc; c = next++)
      sell_windows(rp, n, cw[(size_t)c], cw[(size_t)c + 1], window, vmax, ord, part[(size_t)c]);
  };

  auto run = [&](auto&& f) {
    if (nt == 1) {
      f(0u);
    } else {
      std::vector<std::thread> th;
      for (unsigned t = 0; t < nt; ++t) th.emplace_back(f, t);
      for (auto& x : th) x.join();
    }
  };
  run(check);
  for (unsigned t = 0; t < nt; ++t)
    if (bad[t] >= 0) {
      err = "row_ptr must be non-decreasing (row " + std::to_string(bad[t]) + ")";
      return false;
    }
  if (nc > 1) {  // chunks of equal work (a chunk holds at least one window)
    int64_t total = 0;
    for (int64_t w = 0; w < W; ++w) total += wwork[(size_t)w];
    int64_t c = 1, acc = 0;
    for (int64_t w = 0; w < W && c < nc; ++w) {
      acc += wwork[(size_t)w];
      // close chunk c-1 after window w once it holds its share of the work,
      // leaving at least one window for each later chunk
      while (c < nc && acc * nc >= total * c && W - (w + 1) >= nc - c) cw[(size_t)c++] = w + 1;
    }
    for (; c < nc; ++c) cw[(size_t)c] = W - (nc - c);
  }
  cw[(size_t)nc] = W;
  run(work);
  // join the parts
  size_t ns = 0, nl = 0, nr = 0;
  for (const SellHost& p : part) {
    ns += p.slices.size();
    nl += p.vout.size();
    nr += p.lrows.size();
  }
  out.slices.resize(ns);
  out.vout.resize(nl);
  out.vsrc.resize(nl);
  out.vlen.resize(nl);
  out.vrow.resize(nl);
  std::vector<LongRow> lrows(nr);
  std::vector<size_t> so(nc + 1, 0), lo(nc + 1, 0), ro(nc + 1, 0);
  std::vector<int64_t> eo(nc + 1, 0), po(nc + 1, 0);
  for (int64_t t = 0; t < nc; ++t) {
    so[t + 1] = so[t] + part[t].slices.size();
    lo[t + 1] = lo[t] + part[t].vout.size();
    ro[t + 1] = ro[t] + part[t].lrows.size();
    eo[t + 1] = eo[t] + part[t].entries;
    po[t + 1] = po[t] + part[t].pieces;
  }
  next = 0;
  auto join = [&](unsigned) {
    for (int64_t t = next++; t < nc; t = next++) {
      const SellHost& p = part[(size_t)t];
      for (size_t i = 0; i < p.slices.size(); ++i) {
        SellSlice sl = p.slices[i];
        sl.base += eo[t];
        out.slices[so[t] + i] = sl;
      }
      for (size_t i = 0; i < p.vout.size(); ++i) {
        int32_t v = p.vout[i];
        if (v < 0 && v != SELL_SKIP) v = -1 - (int32_t)(po[t] + (-1 - (int64_t)v));
        out.vout[lo[t] + i] = v;
        out.vsrc[lo[t] + i] = p.vsrc[i];
        out.vlen[lo[t] + i] = p.vlen[i];
        out.vrow[lo[t] + i] = p.vrow[i];
      }
      for (size_t i = 0; i < p.lrows.size(); ++i) {
        LongRow lr = p.lrows[i];
        lr.first += (int32_t)po[t];
        lrows[ro[t] + i] = lr;
      }
    }
  };
  run(join);
  out.entries = eo[nc];
  out.pieces = po[nc];
  // cut rows with the most pieces first (their finalising lanes run longest):
  // a stable counting sort by piece count
  int32_t maxc = 0;
  for (const LongRow& lr : lrows) maxc = std::max(maxc, lr.count);
  std::vector<int64_t> cpos((size_t)maxc + 2, 0);
  for (const LongRow& lr : lrows) ++cpos[lr.count];
  int64_t acc = 0;
  for (int32_t c = maxc; c >= 0; --c) {
    const int64_t k = cpos[c];
    cpos[c] = acc;
    acc += k;
  }
  out.lrows.resize(nr);
  for (const LongRow& lr : lrows) out.lrows[cpos[lr.count]++] = lr;
  out.nbig = 0;
  while (out.nbig < (int64_t)out.lrows.size() && out.lrows[out.nbig].count > SELL_BIG_PIECES)
    ++out.nbig;
  return true;
}

// Host threads for a pass over n rows (at least ~64K rows each).
static unsigned row_threads(int64_t n) {
  unsigned nt = std::thread::hardware_concurrency();
  if (nt < 1) nt = 1;
  if (nt > 32) nt = 32;
  const int64_t cap = n / 65536;
  if ((int64_t)nt > cap) nt = (unsigned)std::max<int64_t>(1, cap);
  return nt;
}
template <typename F>
static void run_threads(unsigned nt, F&& f) {
  if (nt == 1) {
    f(0u);
    return;
  }
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; ++t) th.emplace_back(f, t);
  for (auto& x : th) x.join();
}

bool rows_valid(const int64_t* rp, int64_t n, int64_t nnz, std::string& err) {
  if (rp[0] != 0) {
    err = "row_ptr[0] must be 0";
    return false;
  }
  if (rp[n] != nnz) {
    err = "row_ptr[n] != nnz";
    return false;
  }
  const unsigned nt = row_threads(n);
  std::vector<int64_t> bad(nt, -1);
  run_threads(nt, [&](unsigned t) {
    const int64_t r0 = n * t / nt, r1 = n * (t + 1) / nt;
    for (int64_t r = r0; r < r1; ++r)
      if (rp[r + 1] < rp[r]) {
        bad[t] = r;
        return;
      }
  });
  for (int64_t b : bad)
    if (b >= 0) {
      err = "row_ptr must be non-decreasing (row " + std::to_string(b) + ")";
      return false;
    }
  return true;
}

// Rows by length, longest first, ties in row order (a stable counting sort
// over the row lengths): perm[r] = the row placed at r, iperm its inverse;
// src[r] and len[r] = the first CSR entry and the length of that row, so that
// the layout reads them in order.  Threads take contiguous row ranges, each
// with its own histogram; the offsets of (length, range) follow lengths
// descending, then ranges in order, so the result equals the sequential sort.
// Sparse graphs whose degrees follow a power law then keep their
// high-degree vertices together, so that the SpMV's reads of x for those
// columns share cache lines.  The row pointers must be valid.
void degree_order(const int64_t* rp, int64_t n, int32_t* perm, int32_t* iperm, int64_t* src,
                  int32_t* len) {
  unsigned nt = row_threads(n);
  std::vector<int64_t> maxl(nt, 0);
  run_threads(nt, [&](unsigned t) {
    const int64_t r0 = n * t / nt, r1 = n * (t + 1) / nt;
    int64_t m = 0;
    for (int64_t r = r0; r < r1; ++r) m = std::max<int64_t>(m, rp[r + 1] - rp[r]);
    maxl[t] = m;
  });
  const int64_t L = *std::max_element(maxl.begin(), maxl.end()) + 1;
  // the histograms hold nt * L counts: fewer threads when rows are very long
  while (nt > 1 && (int64_t)nt * L > std::max<int64_t>(n, (int64_t)1 << 22)) --nt;
  std::vector<int64_t> cnt((size_t)nt * L, 0);  // [thread][length]
  run_threads(nt, [&](unsigned t) {
    const int64_t r0 = n * t / nt, r1 = n * (t + 1) / nt;
    int64_t* c = cnt.data() + (size_t)t * L;
    for (int64_t r = r0; r < r1; ++r) ++c[rp[r + 1] - rp[r]];
  });
  int64_t acc = 0;
  for (int64_t l = L - 1; l >= 0; --l)
    for (unsigned t = 0; t < nt; ++t) {
      int64_t& c = cnt[(size_t)t * L + l];
      const int64_t k = c;
      c = acc;
      acc += k;
    }
  run_threads(nt, [&](unsigned t) {
    const int64_t r0 = n * t / nt, r1 = n * (t + 1) / nt;
    int64_t* c = cnt.data() + (size_t)t * L;
    for (int64_t r = r0; r < r1; ++r) {
      const int64_t l = rp[r + 1] - rp[r];
      const int64_t at = c[l]++;
      perm[at] = (int32_t)r;
      iperm[r] = (int32_t)at;
      src[at] = rp[r];
      len[at] = (int32_t)l;
    }
  });
}

// Host build of the SELL arrays (for a matrix that stays in host memory and
// is streamed to the device in row blocks): the same arrangement the device
// build produces; binary64 -> binary32 rounds to nearest even.  Threads split
// the slices; the output does not depend on their number.  Returns false if a
// column index lies outside [0, n).
template <typename Vin, typename Vout>
static bool build_sell_host_t(const SellHost& H, const int32_t* ci, const Vin* val, int64_t n,
                              const int32_t* colmap, int32_t* cols, Vout* vals) {
  const int64_t S = (int64_t)H.slices.size();
  unsigned nt = std::thread::hardware_concurrency();
  if (nt < 1) nt = 1;
  if (nt > 64) nt = 64;
  std::vector<int> bad(nt, 0);
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; ++t) {
    th.emplace_back([&, t] {
      for (int64_t sl = (int64_t)t; sl < S; sl += nt) {
        const SellSlice& q = H.slices[(size_t)sl];
        for (int lane = 0; lane < SELL_C; ++lane) {
          const size_t l = (size_t)sl * SELL_C + lane;
          const int64_t src = H.vsrc[l];
          const int len = H.vlen[l];
          for (int k = 0; k < q.len; ++k) {
            const int64_t dst = q.base + (int64_t)k * SELL_C + lane;
            if (k < len) {
              const int32_t c = ci[src + k];
              const bool ok = c >= 0 && (int64_t)c < n;
              if (!ok) bad[t] = 1;
              cols[dst] = (colmap && ok) ? colmap[c] : c;
              vals[dst] = (Vout)val[src + k];
            } else {
              cols[dst] = 0;
              vals[dst] = (Vout)0;
            }
          }
        }
      }
    });
  }
  for (auto& x : th) x.join();
  for (int b : bad)
    if (b) return false;
  return true;
}

bool build_sell_host(const SellHost& H, const int32_t* ci, const void* val, int in_type, int vk,
                     int64_t n, const int32_t* colmap, int32_t* cols, void* vals) {
  if (in_type == TE_F64 && vk == TE_F64)
    return build_sell_host_t(H, ci, static_cast<const double*>(val), n, colmap, cols,
                             static_cast<double*>(vals));
  if (in_type == TE_F64 && vk == TE_F32)
    return build_sell_host_t(H, ci, static_cast<const double*>(val), n, colmap, cols,
                             static_cast<float*>(vals));
  if (in_type == TE_F32 && vk == TE_F32)
    return build_sell_host_t(H, ci, static_cast<const float*>(val), n, colmap, cols,
                             static_cast<float*>(vals));
  return false;
}

// Vin -> Vout: binary64 -> binary32 rounds to nearest even (__double2float_rn)
template <typename Vin, typename Vout>
TE_DEV Vout convert_value(Vin v) {
  if constexpr (sizeof(Vin) == 8 && sizeof(Vout) == 4) return __double2float_rn(v);
  else return (Vout)v;
}

template <typename Vin, typename Vout>
__global__ void sell_build_kernel(const int32_t* ci, const Vin* val, const SellSlice* slices,
                                  const int64_t* vsrc, const int32_t* vlen, int nslices,
                                  int32_t* cols, Vout* vals, const int32_t* vrow,
                                  const float* row_scale, float* lane_scale,
                                  const int32_t* colmap) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nslices * SELL_C) return;
  const int64_t s = t / SELL_C;
  const int lane = (int)(t % SELL_C);
  const SellSlice sl = slices[s];
  const int64_t src = vsrc[t];
  const int len = vlen[t];
  if (lane_scale) {
    const int32_t r = vrow[t];
    lane_scale[t] = r >= 0 ? row_scale[r] : 0.f;
  }
  for (int k = 0; k < sl.len; ++k) {
    const int64_t dst = sl.base + (int64_t)k * SELL_C + lane;
    if (k < len) {
      const int32_t c = ci[src + k];  // checked to lie in [0, n) before the build
      cols[dst] = colmap ? colmap[c] : c;
      vals[dst] = convert_value<Vin, Vout>(val[src + k]);
    } else {
      cols[dst] = 0;
      vals[dst] = (Vout)0;
    }
  }
}

cudaError_t launch_sell_build(int in_type, int out_type, const int32_t* ci, const void* val,
                              const SellSlice* slices, const int64_t* vsrc, const int32_t* vlen,
                              int nslices, int32_t* cols, void* vals, const int32_t* vrow,
                              const float* row_scale, float* lane_scale, const int32_t* colmap,
                              cudaStream_t s) {
  if (nslices <= 0) return cudaSuccess;
  const int64_t lanes = (int64_t)nslices * SELL_C;
  const unsigned blocks = (unsigned)((lanes + 255) / 256);
#define TE_BUILD(IN, OUT, TI, TO)                                                               \
  if (in_type == IN && out_type == OUT) {                                                      \
    sell_build_kernel<TI, TO><<<blocks, 256, 0, s>>>(ci, static_cast<const TI*>(val), slices, \
                                                     vsrc, vlen, nslices, cols,                \
                                                     static_cast<TO*>(vals), vrow, row_scale,  \
                                                     lane_scale, colmap);                      \
    return cudaGetLastError();                                                                 \
  }
  TE_BUILD(TE_F64, TE_F64, double, double)
  TE_BUILD(TE_F64, TE_F32, double, float)
  TE_BUILD(TE_F32, TE_F32, float, float)
  TE_BUILD(TE_BF16, TE_BF16, uint16_t, uint16_t)
  TE_BUILD(TE_FP8_E4M3, TE_FP8_E4M3, uint8_t, uint8_t)
#undef TE_BUILD
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

// Cut rows: the first nbig rows (most pieces first) get a whole warp each,
// the others FIN_G lanes each (most cut rows have a handful of pieces).
// Each lane sums a strided subset of the row's piece partials, then a fixed
// shuffle tree adds the lanes (deterministic).
constexpr int FIN_G = 4;
template <int P, bool F64OUT>
__global__ void spmv_long_finalize(const LongRow* lrows, int nl, int nbig, int big_blocks,
                                   const void* vpart, void* y) {
  const bool big = (int)blockIdx.x < big_blocks;  // uniform per block
  const int G = big ? 32 : FIN_G;
  const int64_t t = (int64_t)(big ? blockIdx.x : blockIdx.x - big_blocks) * blockDim.x + threadIdx.x;
  const int64_t g = (big ? 0 : nbig) + t / G;
  const int sub = threadIdx.x & (G - 1);
  const bool live = big ? (g < nbig) : (g < nl);  // every lane reaches the shuffles below
  LongRow lr{0, 0, 0, 0};
  if (live) lr = lrows[g];
  typename SpmvTr<P>::acc_t acc;
  acc_zero<P>(acc);
  for (int c = sub; c < lr.count; c += G) {
    if constexpr (P == PREC_FDF) {
      float2 v = static_cast<const float2*>(vpart)[lr.first + c];
      dacc_add_pair(acc, v.x, v.y);
    } else {
      acc += static_cast<const double*>(vpart)[lr.first + c];
    }
  }
  acc = group_sum(acc, G);
  if (live && sub == 0) store_row<P, F64OUT>(y, lr.row, acc);
}

template <int P, int VK, bool F64OUT>
static cudaError_t launch_spmv_t(const SpmvArgs& a, const DevSell& S, cudaStream_t s) {
  if (S.nslices > 0)
    spmv_kernel<P, VK, F64OUT><<<(S.nslices + SPMV_WPB - 1) / SPMV_WPB, 32 * SPMV_WPB, 0, s>>>(a);
  if (S.nlrows > 0) {
    const int threads = 256;
    const int big_blocks = (int)(((int64_t)S.nlbig * 32 + threads - 1) / threads);
    const int small_blocks =
        (int)(((int64_t)(S.nlrows - S.nlbig) * FIN_G + threads - 1) / threads);
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

__global__ void __launch_bounds__(32 * SPMV_WPB) batch_spmv_kernel(const BatchTable* T) {
  const int lane = threadIdx.x & 31;
  const int ns = T->nslots;
  const int64_t total = T->slice_off[ns];
  for (int64_t g = (int64_t)blockIdx.x * SPMV_WPB + (threadIdx.x >> 5); g < total;
       g += (int64_t)gridDim.x * SPMV_WPB) {
    const int sidx = find_slot(T->slice_off, ns, g);
    const BatchSlot& B = T->slot[sidx];
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
    const int slice = (int)(g - T->slice_off[sidx]);
    if (B.vk == TE_BF16) spmv_slice<PREC_FDF, TE_BF16, false>(a, slice, lane);
    else spmv_slice<PREC_FDF, TE_F32, false>(a, slice, lane);
  }
}

// cut rows of every live solve, FIN_G lanes per row; the loop runs whole
// warps so that every lane reaches the shuffles
__global__ void batch_finalize_kernel(const BatchTable* T) {
  const int ns = T->nslots;
  const int64_t total = T->lrow_off[ns];
  const int lane = threadIdx.x & 31, sub = lane & (FIN_G - 1);
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 / FIN_G);
       w0 < total; w0 += warps * (32 / FIN_G)) {
    const int64_t g = w0 + lane / FIN_G;
    const bool live = g < total;
    LongRow lr{0, 0, 0, 0};
    const BatchSlot* B = nullptr;
    if (live) {
      B = &T->slot[find_slot(T->lrow_off, ns, g)];
      lr = B->lrows[g - T->lrow_off[B - T->slot]];
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

cudaError_t launch_batch_spmv(const BatchTable* T, cudaStream_t s) {
  batch_spmv_kernel<<<SRV_SPMV_BLOCKS, 32 * SPMV_WPB, 0, s>>>(T);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  batch_finalize_kernel<<<SRV_FIN_BLOCKS, 256, 0, s>>>(T);
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
