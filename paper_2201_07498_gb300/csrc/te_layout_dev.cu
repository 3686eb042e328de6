// te_layout_dev.cu - the SpMV layout built on the device.
//
// The same arrangement te_layout.cu computes on the host (rows relabelled by
// length, SELL-C-sigma windows, cut rows), computed by kernels from a device
// row_ptr, so that a plan's analysis costs a few kernel launches instead of
// host passes over every row.  The result is identical, element for element,
// to the host build.
//
// Row order: a stable sort of the rows by length, longest first, as an LSD
// radix sort over 8-bit digits of (Lmax - length), row index as the value.
// Each pass is a stable counting sort: a warp owns a tile of DS_TILE
// consecutive elements; it counts the tile's digits, an exclusive scan over
// (digit, tile) gives every (digit, tile) its first output position, and the
// warp then walks its tile in order, 32 elements at a time, ranking equal
// digits among the lanes with __match_any_sync so that equal keys keep their
// input order.
//
// Arrangement: a warp per window of rows.  Counting: the histogram of piece
// lengths gives the window's slices, padded entries, cut-row pieces and cut
// rows; an exclusive scan over the windows places them.  Emission: the
// window's rows are walked in order, 32 at a time; full-length pieces take
// consecutive positions of their length class (warp prefix sums), shorter
// pieces are ranked within their class with __match_any_sync, so every piece
// lands at the position a stable sort by length (longest first) gives it.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "te_common.cuh"
#include "te_internal.h"

namespace te {

namespace {

constexpr int DS_TILE = 2048;  // elements per warp and pass
constexpr int DS_WARPS = 8;    // warps per CTA
constexpr int DS_BINS = 256;
constexpr int LD_WARPS = 8;    // warps (windows) per CTA of the arrangement kernels
constexpr int LD_MAX_VMAX = 128;
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;  // elements per thread of a scan block
constexpr int SCAN_BLOCK = SCAN_THREADS * SCAN_ITEMS;
constexpr int SCAN_MAX_BLOCKS = SCAN_BLOCK;  // one block scans the block sums

TE_DEV unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <typename T>
TE_DEV T warp_isum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
TE_DEV T warp_excl_scan(T v, T* total) {
  const int lane = threadIdx.x & 31;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  *total = __shfl_sync(0xffffffffu, x, 31);
  return x - v;
}

// ---------------------------------------------------------------------------
// exclusive scan of int64 values (in place), up to SCAN_BLOCK * SCAN_MAX_BLOCKS
// elements: per-block sums, one block scanning them, per-block scans
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SCAN_THREADS) scan_sums_kernel(const int64_t* a, int64_t n,
                                                                 int64_t* sums) {
  __shared__ int64_t ws[SCAN_THREADS / 32];
  const int64_t b0 = (int64_t)blockIdx.x * SCAN_BLOCK;
  int64_t acc = 0;
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int64_t k = b0 + (int64_t)i * SCAN_THREADS + threadIdx.x;
    if (k < n) acc += a[k];
  }
  acc = warp_isum(acc);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < SCAN_THREADS / 32; ++w) t += ws[w];
    sums[blockIdx.x] = t;
  }
}

// exclusive scan of `cnt` values in one block (cnt <= SCAN_BLOCK); the total
// goes to *total
__global__ void __launch_bounds__(SCAN_THREADS) scan_one_block_kernel(int64_t* a, int64_t cnt,
                                                                      int64_t* total) {
  __shared__ int64_t ws[SCAN_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  int64_t v[SCAN_ITEMS];
  int64_t mine = 0;
  for (int i = 0; i < SCAN_ITEMS; ++i) {  // thread tid holds elements tid*ITEMS + i
    const int64_t k = (int64_t)tid * SCAN_ITEMS + i;
    v[i] = k < cnt ? a[k] : 0;
    mine += v[i];
  }
  int64_t wt;
  const int64_t ex = warp_excl_scan(mine, &wt);
  if (lane == 0) ws[wid] = wt;
  __syncthreads();
  if (wid == 0) {
    const int64_t x = lane < SCAN_THREADS / 32 ? ws[lane] : 0;
    int64_t tt;
    const int64_t e2 = warp_excl_scan(x, &tt);
    if (lane < SCAN_THREADS / 32) ws[lane] = e2;
    if (lane == 0 && total) *total = tt;
  }
  __syncthreads();
  int64_t run = ws[wid] + ex;
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int64_t k = (int64_t)tid * SCAN_ITEMS + i;
    if (k < cnt) a[k] = run;
    run += v[i];
  }
}

// block b scans its SCAN_BLOCK elements and adds the scanned block sum
__global__ void __launch_bounds__(SCAN_THREADS) scan_blocks_kernel(int64_t* a, int64_t n,
                                                                   const int64_t* sums) {
  __shared__ int64_t ws[SCAN_THREADS / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int64_t b0 = (int64_t)blockIdx.x * SCAN_BLOCK;
  int64_t v[SCAN_ITEMS];
  int64_t mine = 0;
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int64_t k = b0 + (int64_t)tid * SCAN_ITEMS + i;
    v[i] = k < n ? a[k] : 0;
    mine += v[i];
  }
  int64_t wt;
  const int64_t ex = warp_excl_scan(mine, &wt);
  if (lane == 0) ws[wid] = wt;
  __syncthreads();
  if (wid == 0) {
    const int64_t x = lane < SCAN_THREADS / 32 ? ws[lane] : 0;
    int64_t tt;
    const int64_t e2 = warp_excl_scan(x, &tt);
    if (lane < SCAN_THREADS / 32) ws[lane] = e2;
  }
  __syncthreads();
  int64_t run = sums[blockIdx.x] + ws[wid] + ex;
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int64_t k = b0 + (int64_t)tid * SCAN_ITEMS + i;
    if (k < n) a[k] = run;
    run += v[i];
  }
}

// exclusive scan of a[0, n) in place; tmp holds SCAN_MAX_BLOCKS + 1 values;
// *total (device, optional) receives the sum
cudaError_t excl_scan(int64_t* a, int64_t n, int64_t* tmp, int64_t* total, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
  if (blocks > SCAN_MAX_BLOCKS) return cudaErrorInvalidValue;
  if (blocks == 1) {
    scan_one_block_kernel<<<1, SCAN_THREADS, 0, s>>>(a, n, total);
    return cudaGetLastError();
  }
  scan_sums_kernel<<<(unsigned)blocks, SCAN_THREADS, 0, s>>>(a, n, tmp);
  scan_one_block_kernel<<<1, SCAN_THREADS, 0, s>>>(tmp, blocks, total);
  scan_blocks_kernel<<<(unsigned)blocks, SCAN_THREADS, 0, s>>>(a, n, tmp);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// row lengths, row-pointer checks, the longest row
// ---------------------------------------------------------------------------
// flag bit 1: row_ptr[0] != 0 or row_ptr[n] != nnz; bit 2: a decreasing row
__global__ void row_lengths_kernel(const int64_t* rp, int64_t n, int64_t nnz, uint32_t* key,
                                   int32_t* val, int* flag, unsigned long long* lmax) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t first = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (first == 0 && (rp[0] != 0 || rp[n] != nnz)) atomicOr(flag, 1);
  unsigned long long m = 0;
  for (int64_t r = first; r < n; r += stride) {
    const int64_t L = rp[r + 1] - rp[r];
    if (L < 0) atomicOr(flag, 2);
    const unsigned long long l = L > 0 ? (unsigned long long)L : 0ull;
    m = l > m ? l : m;
    if (key) key[r] = (uint32_t)(L > 0 ? (L < 0xffffffffll ? L : 0xffffffffll) : 0);
    if (val) val[r] = (int32_t)r;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_down_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
  }
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(lmax, m);
}

// key <- lmax - key: ascending keys = descending lengths
__global__ void flip_keys_kernel(uint32_t* key, int64_t n, uint32_t lmax) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x)
    key[r] = lmax - key[r];
}

// ---------------------------------------------------------------------------
// one stable counting-sort pass on the 8-bit digit at `shift`
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32 * DS_WARPS) ds_hist_kernel(const uint32_t* key, int64_t n,
                                                                int shift, int64_t ntiles,
                                                                int64_t* cnt) {
  __shared__ int32_t h[DS_WARPS][DS_BINS];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t = (int64_t)blockIdx.x * DS_WARPS + w;
  for (int d = lane; d < DS_BINS; d += 32) h[w][d] = 0;
  __syncwarp();
  if (t < ntiles) {
    const int64_t i0 = t * DS_TILE, i1 = i0 + DS_TILE < n ? i0 + DS_TILE : n;
    for (int64_t i = i0 + lane; i < i1; i += 32) atomicAdd(&h[w][(key[i] >> shift) & 255u], 1);
    __syncwarp();
    for (int d = lane; d < DS_BINS; d += 32) cnt[(int64_t)d * ntiles + t] = h[w][d];
  }
}

__global__ void __launch_bounds__(32 * DS_WARPS) ds_scatter_kernel(
    const uint32_t* key, const int32_t* val, uint32_t* key_out, int32_t* val_out, int64_t n,
    int shift, int64_t ntiles, const int64_t* off) {
  __shared__ int64_t base[DS_WARPS][DS_BINS];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t = (int64_t)blockIdx.x * DS_WARPS + w;
  if (t >= ntiles) return;  // uniform per warp
  for (int d = lane; d < DS_BINS; d += 32) base[w][d] = off[(int64_t)d * ntiles + t];
  __syncwarp();
  const int64_t i0 = t * DS_TILE, i1 = i0 + DS_TILE < n ? i0 + DS_TILE : n;
  for (int64_t c = i0; c < i1; c += 32) {
    const int64_t i = c + lane;
    const bool ok = i < i1;
    const uint32_t k = ok ? key[i] : 0u;
    const int d = ok ? (int)((k >> shift) & 255u) : DS_BINS;  // DS_BINS: no element
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int64_t b = ok ? base[w][d] : 0;
    __syncwarp();
    if (ok) {
      const int64_t p = b + __popc(peers & lanemask_lt());
      key_out[p] = k;
      val_out[p] = val[i];
      if (lane == __ffs(peers) - 1) base[w][d] = b + __popc(peers);
    }
    __syncwarp();
  }
}

// the row order from the sorted rows: perm, iperm, and each placed row's
// first entry and length
__global__ void order_arrays_kernel(const int32_t* sorted_rows, const int64_t* rp, int64_t n,
                                    int32_t* perm, int32_t* iperm, int64_t* src, int32_t* len) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int32_t o = sorted_rows[r];
    perm[r] = o;
    iperm[o] = (int32_t)r;
    src[r] = rp[o];
    len[r] = (int32_t)(rp[o + 1] - rp[o]);
  }
}

// ---------------------------------------------------------------------------
// the arrangement
// ---------------------------------------------------------------------------
struct RowsView {
  const int64_t* rp;     // CSR row pointers
  const int64_t* src;    // relabelled rows: first entry of row r (else nullptr)
  const int32_t* len;    // relabelled rows: length of row r
  const int32_t* perm;   // relabelled rows: the CSR row placed at r
  TE_DEV int64_t L(int64_t r) const { return src ? (int64_t)len[r] : rp[r + 1] - rp[r]; }
  TE_DEV int64_t first(int64_t r) const { return src ? src[r] : rp[r]; }
  TE_DEV int32_t csr_row(int64_t r) const { return perm ? perm[r] : (int32_t)r; }
};

// the pieces of a row: nfull pieces of length vmax, then one of length s (0:
// none); a row of length <= vmax is one piece (of length vmax when L = vmax)
TE_DEV void row_pieces(int64_t L, int vmax, int64_t& nfull, int& s) {
  if (L <= 0) {
    nfull = 0;
    s = 0;
  } else if (L <= vmax) {
    nfull = L == vmax ? 1 : 0;
    s = L == vmax ? 0 : (int)L;
  } else {
    nfull = L / vmax;
    s = (int)(L - nfull * vmax);
  }
}

// WinCount fields as four int64 arrays (slices, entries, pieces, lrows),
// one entry per window
__global__ void __launch_bounds__(32 * LD_WARPS) win_count_kernel(RowsView R, int64_t n,
                                                                  int window, int vmax,
                                                                  int64_t nwin, int64_t* wc) {
  __shared__ int64_t hist[LD_WARPS][LD_MAX_VMAX + 1];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t win = (int64_t)blockIdx.x * LD_WARPS + w;
  if (win >= nwin) return;  // uniform per warp
  for (int l = lane; l <= vmax; l += 32) hist[w][l] = 0;
  __syncwarp();
  const int64_t r0 = win * window, r1 = r0 + window < n ? r0 + window : n;
  int64_t pieces = 0, lrows = 0, np = 0;
  for (int64_t r = r0 + lane; r < r1; r += 32) {
    const int64_t L = R.L(r);
    int64_t nfull;
    int s;
    row_pieces(L, vmax, nfull, s);
    if (nfull) atomicAdd(reinterpret_cast<unsigned long long*>(&hist[w][vmax]),
                         (unsigned long long)nfull);
    if (s) atomicAdd(reinterpret_cast<unsigned long long*>(&hist[w][s]), 1ull);
    np += nfull + (s ? 1 : 0);
    if (L > vmax) {
      pieces += nfull + (s ? 1 : 0);
      lrows += 1;
    }
  }
  pieces = warp_isum(pieces);
  lrows = warp_isum(lrows);
  np = warp_isum(np);
  __syncwarp();
  if (lane == 0) {
    int64_t at = 0, entries = 0;
    for (int L = vmax; L >= 1; --L) {
      const int64_t h = hist[w][L];
      if (h == 0) continue;
      const int64_t starts = (at + h + SELL_C - 1) / SELL_C - (at + SELL_C - 1) / SELL_C;
      entries += starts * SELL_C * L;
      at += h;
    }
    wc[win] = (np + SELL_C - 1) / SELL_C;
    wc[nwin + win] = entries;
    wc[2 * nwin + win] = pieces;
    wc[3 * nwin + win] = lrows;
  }
}

// window `win` written at its offsets (the scanned counts); lrows unsorted
__global__ void __launch_bounds__(32 * LD_WARPS) win_emit_kernel(
    RowsView R, int64_t n, int window, int vmax, int64_t nwin, const int64_t* off,
    SellSlice* slices, int32_t* vout, int64_t* vsrc, int32_t* vlen, int32_t* vrow,
    LongRow* lrows) {
  __shared__ int64_t start[LD_WARPS][LD_MAX_VMAX + 1];  // first sorted position of a length
  __shared__ int64_t cntl[LD_WARPS][LD_MAX_VMAX + 1];   // pieces of a length
  __shared__ int64_t pos[LD_WARPS][LD_MAX_VMAX + 1];    // next free position of a length
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t win = (int64_t)blockIdx.x * LD_WARPS + w;
  if (win >= nwin) return;  // uniform per warp
  const int64_t at_slices = off[win], at_entries = off[nwin + win];
  const int64_t at_pieces = off[2 * nwin + win], at_lrows = off[3 * nwin + win];
  for (int l = lane; l <= vmax; l += 32) cntl[w][l] = 0;
  __syncwarp();
  const int64_t r0 = win * window, r1 = r0 + window < n ? r0 + window : n;
  for (int64_t r = r0 + lane; r < r1; r += 32) {
    int64_t nfull;
    int s;
    row_pieces(R.L(r), vmax, nfull, s);
    if (nfull) atomicAdd(reinterpret_cast<unsigned long long*>(&cntl[w][vmax]),
                         (unsigned long long)nfull);
    if (s) atomicAdd(reinterpret_cast<unsigned long long*>(&cntl[w][s]), 1ull);
  }
  __syncwarp();
  if (lane == 0) {
    int64_t acc = 0;
    for (int L = vmax; L >= 1; --L) {
      start[w][L] = acc;
      pos[w][L] = acc;
      acc += cntl[w][L];
    }
    start[w][0] = acc;  // the window's pieces
  }
  __syncwarp();
  const int64_t np = start[w][0];
  const int64_t nsl = (np + SELL_C - 1) / SELL_C;
  // slices: slice j starts at sorted position 32 j and takes the length of
  // the piece there; their entries follow one another
  int64_t ebase = at_entries;
  for (int64_t j0 = 0; j0 < nsl; j0 += 32) {
    const int64_t j = j0 + lane;
    int L = 0;
    if (j < nsl) {
      const int64_t p = j * SELL_C;
      for (int l = vmax; l >= 1; --l)
        if (cntl[w][l] > 0 && start[w][l] <= p && p < start[w][l] + cntl[w][l]) {
          L = l;
          break;
        }
    }
    int64_t tot;
    const int64_t ex = warp_excl_scan((int64_t)SELL_C * L, &tot);
    if (j < nsl) {
      SellSlice sl;
      sl.base = ebase + ex;
      sl.len = L;
      sl.pad_ = 0;
      slices[at_slices + j] = sl;
    }
    ebase += tot;
  }
  // pieces, in row order
  const int64_t lane0 = at_slices * SELL_C;
  int64_t piece_run = at_pieces, lrow_run = at_lrows;
  for (int64_t c0 = r0; c0 < r1; c0 += 32) {
    const int64_t r = c0 + lane;
    const bool ok = r < r1;
    const int64_t L = ok ? R.L(r) : 0;
    int64_t nfull;
    int s;
    row_pieces(L, vmax, nfull, s);
    const bool cut = L > vmax;
    const int64_t npc = cut ? nfull + (s ? 1 : 0) : 0;
    int64_t tf, tp, tl;
    const int64_t exf = warp_excl_scan(nfull, &tf);
    const int64_t exp_ = warp_excl_scan(npc, &tp);
    const int64_t exl = warp_excl_scan((int64_t)(cut ? 1 : 0), &tl);
    const int64_t pf = pos[w][vmax] + exf;
    const int key = s ? s : 0;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int64_t bs = s ? pos[w][s] : 0;
    __syncwarp();
    if (lane == 0) pos[w][vmax] += tf;
    if (s && lane == __ffs(peers) - 1) pos[w][s] = bs + __popc(peers);
    __syncwarp();
    const int64_t first = ok && L > 0 ? R.first(r) : 0;
    const int32_t o = ok && L > 0 ? R.csr_row(r) : -1;
    const int64_t pid = piece_run + exp_;
    // full-length pieces: a row with one writes it; the pieces of a row cut
    // into several are written by the whole warp, row by row (consecutive
    // lanes, coalesced)
    if (nfull == 1) {
      const int64_t l = lane0 + pf;
      vout[l] = cut ? (int32_t)(-1 - pid) : (int32_t)r;
      vsrc[l] = first;
      vlen[l] = vmax;
      if (vrow) vrow[l] = o;
    }
    for (unsigned many = __ballot_sync(0xffffffffu, nfull > 1); many; many &= many - 1) {
      const int src_lane = __ffs(many) - 1;
      const int64_t nf = __shfl_sync(0xffffffffu, nfull, src_lane);
      const int64_t pf_l = __shfl_sync(0xffffffffu, pf, src_lane);
      const int64_t first_l = __shfl_sync(0xffffffffu, first, src_lane);
      const int64_t pid_l = __shfl_sync(0xffffffffu, pid, src_lane);
      const int32_t o_l = __shfl_sync(0xffffffffu, o, src_lane);
      for (int64_t c = lane; c < nf; c += 32) {  // (a row cut into several pieces)
        const int64_t l = lane0 + pf_l + c;
        vout[l] = (int32_t)(-1 - (pid_l + c));
        vsrc[l] = first_l + c * vmax;
        vlen[l] = vmax;
        if (vrow) vrow[l] = o_l;
      }
    }
    if (ok && L > 0) {
      if (s) {
        const int64_t l = lane0 + bs + __popc(peers & lanemask_lt());
        vout[l] = cut ? (int32_t)(-1 - (pid + nfull)) : (int32_t)r;
        vsrc[l] = first + nfull * vmax;
        vlen[l] = s;
        if (vrow) vrow[l] = o;
      }
      if (cut) {
        LongRow lr;
        lr.row = (int32_t)r;
        lr.first = (int32_t)pid;
        lr.count = (int32_t)npc;
        lr.pad_ = 0;
        lrows[lrow_run + exl] = lr;
      }
    }
    piece_run += tp;
    lrow_run += tl;
  }
  // lanes past the last piece of the window's last slice
  for (int64_t l = lane0 + np + lane; l < lane0 + nsl * SELL_C; l += 32) {
    vout[l] = SELL_SKIP;
    vsrc[l] = 0;
    vlen[l] = 0;
    if (vrow) vrow[l] = -1;
  }
}

// keys of the cut rows for the stable sort by piece count (most first)
__global__ void lrow_keys_kernel(const LongRow* lr, int64_t nl, uint32_t cmax, uint32_t* key,
                                 int32_t* val) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nl;
       i += (int64_t)gridDim.x * blockDim.x) {
    key[i] = cmax - (uint32_t)lr[i].count;
    val[i] = (int32_t)i;
  }
}
__global__ void lrow_gather_kernel(const LongRow* in, const int32_t* idx, int64_t nl,
                                   LongRow* out, int* nbig) {
  int big = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nl;
       i += (int64_t)gridDim.x * blockDim.x) {
    const LongRow r = in[idx[i]];
    out[i] = r;
    big += r.count > SELL_BIG_PIECES;
  }
  big = warp_isum(big);
  if ((threadIdx.x & 31) == 0 && big) atomicAdd(nbig, big);
}
__global__ void lrow_cmax_kernel(const LongRow* lr, int64_t nl, unsigned int* cmax) {
  unsigned m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nl;
       i += (int64_t)gridDim.x * blockDim.x)
    m = (unsigned)lr[i].count > m ? (unsigned)lr[i].count : m;
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned y = __shfl_down_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
  }
  if ((threadIdx.x & 31) == 0 && m) atomicMax(cmax, m);
}

int grid_for(int64_t items, int threads, int cap = 16384) {
  int64_t b = (items + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

// LSD radix sort of (key, val) pairs, stable, over the low `bits` bits of
// the keys; the result ends in (k0, v0).  k1/v1: buffers of the same size;
// cnt: 256 * tiles int64; tmp: scan scratch.
cudaError_t radix_sort(uint32_t*& k0, int32_t*& v0, uint32_t*& k1, int32_t*& v1, int64_t n,
                       int bits, int64_t* cnt, int64_t* tmp, cudaStream_t s) {
  const int64_t ntiles = (n + DS_TILE - 1) / DS_TILE;
  const unsigned blocks = (unsigned)((ntiles + DS_WARPS - 1) / DS_WARPS);
  for (int shift = 0; shift < bits; shift += 8) {
    ds_hist_kernel<<<blocks, 32 * DS_WARPS, 0, s>>>(k0, n, shift, ntiles, cnt);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = excl_scan(cnt, ntiles * DS_BINS, tmp, nullptr, s);
    if (e != cudaSuccess) return e;
    ds_scatter_kernel<<<blocks, 32 * DS_WARPS, 0, s>>>(k0, v0, k1, v1, n, shift, ntiles, cnt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    std::swap(k0, k1);
    std::swap(v0, v1);
  }
  return cudaSuccess;
}

int key_bits(uint64_t m) {
  int b = 0;
  while (b < 32 && (m >> b) != 0) b += 8;
  return b;
}

}  // namespace

size_t dev_layout_scratch_bytes(int64_t n) {
  const int64_t ntiles = (n + DS_TILE - 1) / DS_TILE;
  const size_t a = (size_t)std::max<int64_t>(n, 1);
  return 4 * a * 4 + (size_t)ntiles * DS_BINS * 8 + (SCAN_MAX_BLOCKS + 1) * 8 + 4096;
}

bool dev_layout_fits(int64_t n, int window, int vmax) {
  const int64_t ntiles = (n + DS_TILE - 1) / DS_TILE;
  const int64_t nwin = (n + window - 1) / std::max(window, 1);
  return vmax >= 1 && vmax <= LD_MAX_VMAX && window >= 1 &&
         ntiles * DS_BINS <= (int64_t)SCAN_BLOCK * SCAN_MAX_BLOCKS &&
         nwin <= (int64_t)SCAN_BLOCK * SCAN_MAX_BLOCKS && n < ((int64_t)1 << 31) - 1;
}

// Stage 1: row checks, the row order (when `reorder`), and the window counts.
cudaError_t DevLayout::count(const int64_t* rp_dev, int64_t n_, int64_t nnz_, int window_,
                             int vmax_, bool reorder_, cudaStream_t s, std::string& err) {
  n = n_;
  nnz = nnz_;
  window = window_;
  vmax = vmax_;
  reorder = reorder_;
  rp = rp_dev;
  if (!dev_layout_fits(n, window, vmax)) {
    err = "the device layout build does not cover this size";
    return cudaErrorInvalidValue;
  }
  const int64_t ntiles = (n + DS_TILE - 1) / DS_TILE;
  nwin = (n + window - 1) / window;
  // scratch: keys/values (double-buffered), digit counts, scan sums, flags
  char* b = nullptr;
  const size_t a = (size_t)std::max<int64_t>(n, 1);
  const size_t bytes = 4 * a * 4 + (size_t)ntiles * DS_BINS * 8 + (SCAN_MAX_BLOCKS + 1) * 8 +
                       (size_t)4 * std::max<int64_t>(nwin, 1) * 8 + 256;
  cudaError_t e = dev_alloc(&b, bytes);
  if (e != cudaSuccess) return e;
  scratch = b;
  uint32_t* k0 = reinterpret_cast<uint32_t*>(b);
  int32_t* v0 = reinterpret_cast<int32_t*>(b + a * 4);
  uint32_t* k1 = reinterpret_cast<uint32_t*>(b + 2 * a * 4);
  int32_t* v1 = reinterpret_cast<int32_t*>(b + 3 * a * 4);
  int64_t* cnt = reinterpret_cast<int64_t*>(b + 4 * a * 4);
  int64_t* tmp = cnt + (size_t)ntiles * DS_BINS;
  wc = tmp + SCAN_MAX_BLOCKS + 1;
  unsigned char* tail = reinterpret_cast<unsigned char*>(wc + 4 * std::max<int64_t>(nwin, 1));
  int* flag = reinterpret_cast<int*>(tail);
  unsigned long long* lmax = reinterpret_cast<unsigned long long*>(tail + 8);
  e = cudaMemsetAsync(tail, 0, 64, s);
  if (e != cudaSuccess) return e;
  row_lengths_kernel<<<grid_for(n, 256), 256, 0, s>>>(rp, n, nnz, reorder ? k0 : nullptr,
                                                      reorder ? v0 : nullptr, flag, lmax);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  struct {
    int flag, pad;
    unsigned long long lmax;
  } h;
  e = cudaMemcpyAsync(&h, tail, 16, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  if (h.flag & 1) {
    err = "row_ptr[0] must be 0 and row_ptr[n] must equal nnz";
    return cudaErrorInvalidValue;
  }
  if (h.flag & 2) {
    err = "row_ptr must be non-decreasing";
    return cudaErrorInvalidValue;
  }
  if (reorder) {
    const uint32_t L = (uint32_t)std::min<unsigned long long>(h.lmax, 0xffffffffull);
    flip_keys_kernel<<<grid_for(n, 256), 256, 0, s>>>(k0, n, L);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = radix_sort(k0, v0, k1, v1, n, key_bits(L), cnt, tmp, s);
    if (e != cudaSuccess) return e;
    sorted_rows = v0;
    spare_rows = v1;
  }
  return cudaSuccess;
}

cudaError_t DevLayout::order(int32_t* perm, int32_t* iperm, int64_t* src, int32_t* len,
                             cudaStream_t s) {
  order_arrays_kernel<<<grid_for(n, 256), 256, 0, s>>>(sorted_rows, rp, n, perm, iperm, src,
                                                        len);
  view_src = src;
  view_len = len;
  view_perm = perm;
  return cudaGetLastError();
}

cudaError_t DevLayout::windows(cudaStream_t s, int64_t* totals_host) {
  RowsView R{rp, view_src, view_len, view_perm};
  const unsigned blocks = (unsigned)((nwin + LD_WARPS - 1) / LD_WARPS);
  win_count_kernel<<<blocks, 32 * LD_WARPS, 0, s>>>(R, n, window, vmax, nwin, wc);
  cudaError_t e = cudaGetLastError();
  int64_t* tmp = wc - (SCAN_MAX_BLOCKS + 1);
  int64_t* tot = reinterpret_cast<int64_t*>(reinterpret_cast<unsigned char*>(wc) +
                                            (size_t)4 * std::max<int64_t>(nwin, 1) * 8 + 16);
  for (int f = 0; f < 4 && e == cudaSuccess; ++f)
    e = excl_scan(wc + (size_t)f * nwin, nwin, tmp, tot + f, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(totals_host, tot, 4 * 8, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) {
    nslices = totals_host[0];
    entries = totals_host[1];
    pieces = totals_host[2];
    nlrows = totals_host[3];
  }
  return e;
}

cudaError_t DevLayout::emit(SellSlice* slices, int32_t* vout, int64_t* vsrc, int32_t* vlen,
                            int32_t* vrow, LongRow* lrows, LongRow* lrows_tmp, cudaStream_t s,
                            int* nbig_host) {
  RowsView R{rp, view_src, view_len, view_perm};
  const unsigned blocks = (unsigned)((nwin + LD_WARPS - 1) / LD_WARPS);
  win_emit_kernel<<<blocks, 32 * LD_WARPS, 0, s>>>(R, n, window, vmax, nwin, wc, slices, vout,
                                                   vsrc, vlen, vrow, lrows_tmp);
  cudaError_t e = cudaGetLastError();
  *nbig_host = 0;
  if (e != cudaSuccess || nlrows == 0) return e;
  // cut rows: stable sort by piece count, most first, and how many exceed
  // SELL_BIG_PIECES
  char* b = static_cast<char*>(scratch);
  const size_t a = (size_t)std::max<int64_t>(n, 1);
  uint32_t* k0 = reinterpret_cast<uint32_t*>(b);
  int32_t* v0 = reinterpret_cast<int32_t*>(b + a * 4);
  uint32_t* k1 = reinterpret_cast<uint32_t*>(b + 2 * a * 4);
  int32_t* v1 = reinterpret_cast<int32_t*>(b + 3 * a * 4);
  // (the row-order arrays in k/v are no longer needed: order() copied them)
  const int64_t ntiles = (n + DS_TILE - 1) / DS_TILE;
  int64_t* cnt = reinterpret_cast<int64_t*>(b + 4 * a * 4);
  int64_t* tmp = cnt + (size_t)ntiles * DS_BINS;
  unsigned char* tail =
      reinterpret_cast<unsigned char*>(wc + 4 * std::max<int64_t>(nwin, 1)) + 64;
  unsigned* cmax = reinterpret_cast<unsigned*>(tail);
  int* nbig = reinterpret_cast<int*>(tail + 8);
  e = cudaMemsetAsync(tail, 0, 16, s);
  if (e == cudaSuccess) {
    lrow_cmax_kernel<<<grid_for(nlrows, 256), 256, 0, s>>>(lrows_tmp, nlrows, cmax);
    e = cudaGetLastError();
  }
  unsigned hc = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, cmax, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  lrow_keys_kernel<<<grid_for(nlrows, 256), 256, 0, s>>>(lrows_tmp, nlrows, hc, k0, v0);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the cut rows are at most n: the row-order buffers and counts serve again
  e = radix_sort(k0, v0, k1, v1, nlrows, key_bits(hc), cnt, tmp, s);
  if (e != cudaSuccess) return e;
  lrow_gather_kernel<<<grid_for(nlrows, 256), 256, 0, s>>>(lrows_tmp, v0, nlrows, lrows, nbig);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  e = cudaMemcpyAsync(nbig_host, nbig, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

DevLayout::~DevLayout() {
  if (scratch) dev_free(scratch);
}

}  // namespace te
