// te_layout.cu - host side of the SpMV layout (SELL-C-sigma, Kreutzer,
// Hager, Wellein, Fehske & Bishop, SIAM J. Sci. Comput. 36(5), 2014): the
// row-pointer check, the relabelling of rows by length (rows by degree), the
// arrangement of row pieces into windows and slices that the device build
// (te_spmv.cu) fills with column indices and values, and the host build of
// those arrays for a matrix streamed from host memory.  Plain host code;
// every pass is split over host threads and gives the result of a sequential
// pass whatever their number.
#include <algorithm>
#include <atomic>
#include <thread>

#include "te_internal.h"

namespace te {

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

// Row r of the layout: its first CSR entry, its length and the CSR row it
// is (row r itself, or ord->perm[r] when the rows are relabelled).
struct LayoutRows {
  const int64_t* rp;
  const RowOrder* ord;
  int64_t first(int64_t r) const { return ord ? ord->src[r] : rp[r]; }
  int64_t len(int64_t r) const { return ord ? (int64_t)ord->len[r] : rp[r + 1] - rp[r]; }
  int32_t csr_row(int64_t r) const { return ord ? ord->perm[r] : (int32_t)r; }
};

// What one window of rows contributes to the layout; prefix sums of these
// give every window its offsets.
struct WinCount {
  int64_t slices, entries, pieces, lrows;
};

// Counts of window w from the histogram of its piece lengths: sorted longest
// first, the pieces fill slices of SELL_C lanes, each slice padded to its
// first (longest) piece.  hist has vmax + 1 zero entries and is left zero.
static WinCount count_window(const LayoutRows& R, int64_t n, int64_t w, int window, int vmax,
                             int64_t* hist) {
  WinCount c{0, 0, 0, 0};
  const int64_t r0 = w * window, r1 = std::min<int64_t>(r0 + window, n);
  int64_t np = 0;
  for (int64_t r = r0; r < r1; ++r) {
    const int64_t L = R.len(r);
    if (L == 0) continue;
    if (L <= vmax) {
      ++hist[L];
      ++np;
      continue;
    }
    const int64_t q = L / vmax, rem = L - q * vmax;
    hist[vmax] += q;
    if (rem) ++hist[rem];
    np += q + (rem ? 1 : 0);
    c.pieces += q + (rem ? 1 : 0);
    ++c.lrows;
  }
  // sorted positions [at, at + hist[L]) hold pieces of length L; a slice
  // starts at every multiple of SELL_C
  int64_t at = 0;
  for (int L = vmax; L >= 1; --L) {
    const int64_t h = hist[L];
    if (h == 0) continue;
    hist[L] = 0;
    const int64_t starts = (at + h + SELL_C - 1) / SELL_C - (at + SELL_C - 1) / SELL_C;
    c.entries += starts * SELL_C * L;
    at += h;
  }
  c.slices = (np + SELL_C - 1) / SELL_C;
  return c;
}

// Window w written at its offsets `at`.  Its pieces, taken in row order (a
// cut row's pieces in order, numbered from at.pieces), are placed by a
// stable counting sort on length, longest first: a histogram of the lengths
// gives each length its first sorted position, and a second walk over the
// rows writes every piece straight to its lane (sorted position p is lane
// p % SELL_C of slice at.slices + p / SELL_C).  Slices take the length of
// their first piece; lanes past the last piece are empty.  The window's cut
// rows go to lrows[at.lrows, ...).  pos has vmax + 2 entries.
static void emit_window(const LayoutRows& R, int64_t n, int64_t w, int window, int vmax,
                        const WinCount& at, SellHost& out, LongRow* lrows, int64_t* pos) {
  const int64_t r0 = w * window, r1 = std::min<int64_t>(r0 + window, n);
  std::fill(pos, pos + vmax + 2, (int64_t)0);
  int64_t np = 0;
  for (int64_t r = r0; r < r1; ++r) {
    const int64_t L = R.len(r);
    if (L == 0) continue;
    if (L <= vmax) {
      ++pos[L];
      ++np;
      continue;
    }
    const int64_t q = L / vmax, rem = L - q * vmax;
    pos[vmax] += q;
    if (rem) ++pos[rem];
    np += q + (rem ? 1 : 0);
  }
  if (np == 0) return;
  // first sorted position of each length; the slices starting in each run
  int64_t acc = 0, sidx = at.slices, e = at.entries;
  for (int L = vmax; L >= 1; --L) {
    const int64_t h = pos[L];
    pos[L] = acc;
    for (int64_t p = (acc + SELL_C - 1) / SELL_C * SELL_C; p < acc + h; p += SELL_C, ++sidx) {
      SellSlice sl;
      sl.base = e;
      sl.len = L;
      sl.pad_ = 0;
      out.slices[(size_t)sidx] = sl;
      e += (int64_t)SELL_C * L;
    }
    acc += h;
  }
  const size_t lane0 = (size_t)at.slices * SELL_C;
  auto put = [&](int64_t src, int32_t len, int32_t o, int32_t row) {
    const size_t l = lane0 + (size_t)pos[len]++;
    out.vout[l] = o;
    out.vsrc[l] = src;
    out.vlen[l] = len;
    out.vrow[l] = row;
  };
  int64_t piece = at.pieces, lr_at = at.lrows;
  for (int64_t r = r0; r < r1; ++r) {
    const int64_t L = R.len(r);
    if (L == 0) continue;  // empty rows: never written by the kernel
    const int64_t first = R.first(r);
    const int32_t o = R.csr_row(r);
    if (L <= vmax) {
      put(first, (int32_t)L, (int32_t)r, o);
      continue;
    }
    LongRow lr;
    lr.row = (int32_t)r;
    lr.first = (int32_t)piece;
    lr.count = (int32_t)((L + vmax - 1) / vmax);
    lr.pad_ = 0;
    for (int32_t c = 0; c < lr.count; ++c) {
      const int64_t s0 = first + (int64_t)c * vmax;
      const int64_t l = std::min<int64_t>(vmax, first + L - s0);
      put(s0, (int32_t)l, -1 - (int32_t)(piece + c), o);
    }
    piece += lr.count;
    lrows[lr_at++] = lr;
  }
  for (size_t l = lane0 + (size_t)np; l < (size_t)(sidx * SELL_C); ++l) {
    out.vout[l] = SELL_SKIP;
    out.vsrc[l] = 0;
    out.vlen[l] = 0;
    out.vrow[l] = -1;
  }
}

// Cut rows with the most pieces first (their finalising lanes run longest),
// ties in row order: a stable counting sort on the piece count.  Threads
// take contiguous ranges with their own histograms; the offsets of (count,
// range) follow counts descending, then ranges in order, so the result
// equals the sequential sort.
static void sort_long_rows(const hvec<LongRow>& in, hvec<LongRow>& out) {
  const int64_t nr = (int64_t)in.size();
  out.resize((size_t)nr);
  if (nr == 0) return;
  const unsigned nt = row_threads(nr);
  std::vector<int32_t> maxc(nt, 0);
  run_threads(nt, [&](unsigned t) {
    const int64_t i0 = nr * t / nt, i1 = nr * (t + 1) / nt;
    int32_t m = 0;
    for (int64_t i = i0; i < i1; ++i) m = std::max(m, in[(size_t)i].count);
    maxc[t] = m;
  });
  const int64_t C = *std::max_element(maxc.begin(), maxc.end()) + 1;
  std::vector<int64_t> cnt((size_t)nt * C, 0);  // [thread][count]
  run_threads(nt, [&](unsigned t) {
    const int64_t i0 = nr * t / nt, i1 = nr * (t + 1) / nt;
    int64_t* c = cnt.data() + (size_t)t * C;
    for (int64_t i = i0; i < i1; ++i) ++c[in[(size_t)i].count];
  });
  int64_t acc = 0;
  for (int64_t k = C - 1; k >= 0; --k)
    for (unsigned t = 0; t < nt; ++t) {
      int64_t& c = cnt[(size_t)t * C + k];
      const int64_t h = c;
      c = acc;
      acc += h;
    }
  run_threads(nt, [&](unsigned t) {
    const int64_t i0 = nr * t / nt, i1 = nr * (t + 1) / nt;
    int64_t* c = cnt.data() + (size_t)t * C;
    for (int64_t i = i0; i < i1; ++i) out[(size_t)c[in[(size_t)i].count]++] = in[(size_t)i];
  });
}

// Two passes over the windows.  The first checks the row pointers (all rows,
// before anything is built) and counts each window from the histogram of its
// piece lengths; prefix sums of the counts place every window.  The second
// writes each window straight into the final arrays (allocated without a
// zero fill), threads taking chunks of windows from a shared counter (with
// rows relabelled by degree the first windows hold most of the cut rows), so
// the result equals a sequential build whatever the thread count.
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
  const LayoutRows R{rp, ord};
  std::vector<WinCount> off((size_t)W + 1);
  std::vector<int64_t> bad(nt, -1);
  run_threads(nt, [&](unsigned t) {
    std::vector<int64_t> hist((size_t)vmax + 1, 0);
    const int64_t w0 = W * t / nt, w1 = W * (t + 1) / nt;
    for (int64_t w = w0; w < w1; ++w) {
      const int64_t r0 = w * window, r1 = std::min<int64_t>(r0 + window, n);
      for (int64_t r = r0; r < r1; ++r)
        if (rp[r + 1] < rp[r]) {
          bad[t] = r;
          return;
        }
      off[(size_t)w + 1] = count_window(R, n, w, window, vmax, hist.data());
    }
  });
  for (unsigned t = 0; t < nt; ++t)
    if (bad[t] >= 0) {
      err = "row_ptr must be non-decreasing (row " + std::to_string(bad[t]) + ")";
      return false;
    }
  off[0] = WinCount{0, 0, 0, 0};
  for (int64_t w = 0; w < W; ++w) {
    WinCount& o = off[(size_t)w + 1];
    const WinCount& p = off[(size_t)w];
    o.slices += p.slices;
    o.entries += p.entries;
    o.pieces += p.pieces;
    o.lrows += p.lrows;
  }
  const WinCount tot = off[(size_t)W];
  out.slices.resize((size_t)tot.slices);
  out.vout.resize((size_t)tot.slices * SELL_C);
  out.vsrc.resize((size_t)tot.slices * SELL_C);
  out.vlen.resize((size_t)tot.slices * SELL_C);
  out.vrow.resize((size_t)tot.slices * SELL_C);
  hvec<LongRow> lrows((size_t)tot.lrows);
  constexpr int64_t CHUNK = 4;  // windows taken at a time
  std::atomic<int64_t> next{0};
  run_threads(nt, [&](unsigned) {
    std::vector<int64_t> pos((size_t)vmax + 2);
    for (int64_t c = next++; c * CHUNK < W; c = next++)
      for (int64_t w = c * CHUNK; w < std::min<int64_t>(W, (c + 1) * CHUNK); ++w)
        emit_window(R, n, w, window, vmax, off[(size_t)w], out, lrows.data(), pos.data());
  });
  out.entries = tot.entries;
  out.pieces = tot.pieces;
  sort_long_rows(lrows, out.lrows);
  out.nbig = 0;
  while (out.nbig < (int64_t)out.lrows.size() && out.lrows[out.nbig].count > SELL_BIG_PIECES)
    ++out.nbig;
  return true;
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
  hvec<int64_t> cnt((size_t)nt * L);  // [thread][length], zeroed by its thread
  run_threads(nt, [&](unsigned t) {
    const int64_t r0 = n * t / nt, r1 = n * (t + 1) / nt;
    int64_t* c = cnt.data() + (size_t)t * L;
    std::fill(c, c + L, (int64_t)0);
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

}  // namespace te
