// te_refine.cu - binary64 Rayleigh-quotient refinement of the selected Ritz
// pairs, and the Gram matrix of a set of vectors (orthogonality metric).
//
// Refinement (for the mixed-precision forms): the Ritz vector u of a Ritz
// value theta is an approximate eigenvector of M; its Rayleigh quotient
// u'Mu / u'u against the binary64 matrix is a better eigenvalue estimate
// (the error is quadratic in the vector's error), and ||Mu - theta' u|| /
// ||u|| is the reconstruction error the paper reports (Section IV-D).  The
// host runs one binary64 SpMV y = M u per vector; this kernel then reduces,
// with r = y - theta u (small, so no cancellation),
//   theta' = theta + u'r / u'u,   ||y - theta' u||^2 = r'r - (u'r)^2 / u'u.
// Per-block partial sums are added by the last block in a fixed order, so the
// result does not depend on scheduling.
#include "te_common.cuh"
#include "te_internal.h"

namespace te {

constexpr int RQ_THREADS = 256;
constexpr int RQ_WARPS = RQ_THREADS / 32;

int refine_grid(int num_sms) { return num_sms * 2; }

__global__ void __launch_bounds__(RQ_THREADS) refine_kernel(LzState* st, const double* y,
                                                            int64_t n, int k, double* partials) {
  __shared__ double red[RQ_WARPS][3];
  __shared__ int last;
  const double th = st->theta_sel[k];
  const double* u = st->eigvecs + (size_t)k * (size_t)n;
  double ur = 0.0, uu = 0.0, rr = 0.0;
  for (int64_t r = blockIdx.x * (int64_t)RQ_THREADS + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * RQ_THREADS) {
    const double uv = u[r];
    const double res = fma(-th, uv, y[r]);
    ur = fma(uv, res, ur);
    uu = fma(uv, uv, uu);
    rr = fma(res, res, rr);
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  ur = warp_sum(ur);
  uu = warp_sum(uu);
  rr = warp_sum(rr);
  if (lane == 0) {
    red[wid][0] = ur;
    red[wid][1] = uu;
    red[wid][2] = rr;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int w = 0; w < RQ_WARPS; ++w) {
      a += red[w][0];
      b += red[w][1];
      c += red[w][2];
    }
    partials[(size_t)blockIdx.x * 4 + 0] = a;
    partials[(size_t)blockIdx.x * 4 + 1] = b;
    partials[(size_t)blockIdx.x * 4 + 2] = c;
    __threadfence();
    const unsigned tk = atomicAdd(&st->ticket, 1u);
    last = (tk == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (wid == 0) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int blk = lane; blk < (int)gridDim.x; blk += 32) {
      a += __ldcg(partials + (size_t)blk * 4 + 0);
      b += __ldcg(partials + (size_t)blk * 4 + 1);
      c += __ldcg(partials + (size_t)blk * 4 + 2);
    }
    a = warp_sum(a);
    b = warp_sum(b);
    c = warp_sum(c);
    if (lane == 0) {
      double thn = th, res = 0.0;
      if (b > 0.0) {
        thn = th + a / b;
        const double q = c - a * a / b;
        res = sqrt(q > 0.0 ? q : 0.0) / sqrt(b);
      }
      st->theta_sel[k] = thn;
      st->resid_est[k] = res;
      if (st->eigvals_out) st->eigvals_out[k] = thn;
      __threadfence();
      st->ticket = 0;
    }
  }
}

cudaError_t launch_refine(LzState* st, const double* y, int64_t n, int k, double* partials,
                          int grid, cudaStream_t s) {
  refine_kernel<<<grid, RQ_THREADS, 0, s>>>(st, y, n, k, partials);
  return cudaGetLastError();
}

__global__ void copy_out_kernel(const LzState* st, const double* src, size_t count) {
  double* dst = st->eigvecs_user;
  if (dst == nullptr) return;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count;
       e += (size_t)gridDim.x * blockDim.x)
    dst[e] = src[e];
}

cudaError_t launch_copy_out(LzState* st, const double* src, size_t count, int grid,
                            cudaStream_t s) {
  copy_out_kernel<<<grid, 256, 0, s>>>(st, src, count);
  return cudaGetLastError();
}

// Thread per caller row, column by column: the writes are coalesced, the
// reads gather from one column (n doubles) at a time, which the L2 keeps.
__global__ void copy_out_perm_kernel(const LzState* st, const double* src, int64_t n, int K,
                                     const int32_t* iperm) {
  double* dst = st->eigvecs_user;
  if (dst == nullptr) return;
  for (int k = 0; k < K; ++k) {
    const double* sk = src + (size_t)k * n;
    double* dk = dst + (size_t)k * n;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
      dk[v] = sk[iperm[v]];
  }
}

cudaError_t launch_copy_out_perm(LzState* st, const double* src, int64_t n, int K,
                                 const int32_t* iperm, int grid, cudaStream_t s) {
  copy_out_perm_kernel<<<grid, 256, 0, s>>>(st, src, n, K, iperm);
  return cudaGetLastError();
}

// Thread per caller row: its K values are one contiguous row of src (read
// with 16-byte loads, up to eight in flight per thread), written to the K
// columns (coalesced across threads).
__global__ void copy_out_rows_kernel(const LzState* st, const double* __restrict__ src, int64_t n,
                                     int K, const int32_t* __restrict__ iperm) {
  double* __restrict__ dst = st->eigvecs_user;
  if (dst == nullptr) return;
  const int Kr = (K + 1) & ~1;
  constexpr int CH = 8;  // 16-byte loads of one row in flight per thread
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
       v += (int64_t)gridDim.x * blockDim.x) {
    const double2* row = reinterpret_cast<const double2*>(src + (size_t)iperm[v] * Kr);
    for (int k0 = 0; k0 < K; k0 += 2 * CH) {
      double2 t[CH];
#pragma unroll
      for (int q = 0; q < CH; ++q)
        if (k0 + 2 * q < K) t[q] = row[(k0 >> 1) + q];
#pragma unroll
      for (int q = 0; q < CH; ++q) {
        const int k = k0 + 2 * q;
        if (k < K) dst[(size_t)k * n + v] = t[q].x;
        if (k + 1 < K) dst[(size_t)(k + 1) * n + v] = t[q].y;
      }
    }
  }
}

cudaError_t launch_copy_out_rows(LzState* st, const double* src, int64_t n, int K,
                                 const int32_t* iperm, int grid, cudaStream_t s) {
  copy_out_rows_kernel<<<grid, 256, 0, s>>>(st, src, n, K, iperm);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gram matrix: G[a][b] = sum_r U[r, a] U[r, b] for a <= b (pair index p in
// row-major upper-triangle order).  Each block stages GR rows of U in shared
// memory and every thread accumulates up to GP pairs; per-block partials are
// summed over blocks in order by gram_reduce.
// ---------------------------------------------------------------------------
constexpr int GR = 32;  // rows staged per block iteration
constexpr int GT = 256;
constexpr int GP = (MAX_M * (MAX_M + 1) / 2 + GT - 1) / GT;  // pairs per thread

__global__ void __launch_bounds__(GT) gram_kernel(const double* U, int64_t n, int K,
                                                  double* partials) {
  __shared__ double tile[MAX_M][GR + 1];  // +1: pairs of a warp hit different banks
  const int np = K * (K + 1) / 2;
  int pa[GP], pb[GP];
  double acc[GP];
#pragma unroll
  for (int q = 0; q < GP; ++q) {
    acc[q] = 0.0;
    pa[q] = -1;
    pb[q] = 0;
    const int p = threadIdx.x + q * GT;
    if (p < np) {
      // invert p = a*K - a*(a-1)/2 + (b - a)
      int a = 0, base = 0;
      while (base + (K - a) <= p) {
        base += K - a;
        ++a;
      }
      pa[q] = a;
      pb[q] = a + (p - base);
    }
  }
  for (int64_t r0 = (int64_t)blockIdx.x * GR; r0 < n; r0 += (int64_t)gridDim.x * GR) {
    __syncthreads();
    for (int e = threadIdx.x; e < K * GR; e += GT) {
      const int a = e / GR, rr = e % GR;
      const int64_t r = r0 + rr;
      tile[a][rr] = r < n ? U[(size_t)a * (size_t)n + r] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < GP; ++q) {
      if (pa[q] < 0) continue;
      double t = acc[q];
      for (int rr = 0; rr < GR; ++rr) t = fma(tile[pa[q]][rr], tile[pb[q]][rr], t);
      acc[q] = t;
    }
  }
#pragma unroll
  for (int q = 0; q < GP; ++q) {
    const int p = threadIdx.x + q * GT;
    if (p < np) partials[(size_t)blockIdx.x * np + p] = acc[q];
  }
}

__global__ void gram_reduce(const double* partials, int blocks, int K, double* G) {
  const int np = K * (K + 1) / 2;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  double t = 0.0;
  for (int b = 0; b < blocks; ++b) t += partials[(size_t)b * np + p];
  int a = 0, base = 0;
  while (base + (K - a) <= p) {
    base += K - a;
    ++a;
  }
  const int bcol = a + (p - base);
  G[a * K + bcol] = t;
  G[bcol * K + a] = t;
}

cudaError_t launch_gram(const double* U, int64_t n, int K, double* partials, int grid,
                        double* G, cudaStream_t s) {
  gram_kernel<<<grid, GT, 0, s>>>(U, n, K, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int np = K * (K + 1) / 2;
  gram_reduce<<<(np + 127) / 128, 128, 0, s>>>(partials, grid, K, G);
  return cudaGetLastError();
}

}  // namespace te
