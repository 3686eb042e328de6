// te_jacobi.cu - the Jacobi phase (Section III, Fig. 1): eigen-decomposition
// of the small tridiagonal T produced by the Lanczos phase, the selection of
// the K eigenvalues largest in modulo (Section I), and the coefficients of the
// Ritz-vector contraction.
//
// The paper ran this step on the CPU because one 24x24 matrix cannot fill a
// GPU; here it stays on the device so that a solve needs no host round trip
// before the Ritz contraction.  One CTA holds T and the eigenvector matrix Y in
// shared memory and applies cyclic Jacobi with the parallel (round-robin,
// "circle method") ordering of Brent & Luk: every round rotates m/2 disjoint
// index pairs at once, T <- J^T T J (on 2x2 blocks of the upper triangle,
// mirrored), Y <- Y J.  Rotation angle (textbook
// form, e.g. Golub & Van Loan Sec. 8.5): zeta = (t_qq - t_pp) / (2 t_pq),
// t = sgn(zeta)/(|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1 + t^2), s = t c
// (evaluated as |2 t_pq| sgn(zeta) / (|d| + hypot(d, 2 t_pq)), d = t_qq - t_pp);
// a pair is rotated when |t_pq| > 1e-16 ||T||_F and the sweeps stop after
// one without rotations (which is skipped when no off-diagonal element left
// after a sweep exceeds that threshold: it could rotate nothing).
// Arithmetic is binary64.
//
// GB300 runs binary64 at two operations per SM and clock, so for m >= 40 the
// rounds are spread over a cluster of JAC_CLUSTER CTAs: every CTA keeps a full
// copy of T, computes all rotations of a round (the same values everywhere),
// updates the blocks e = rank (mod JAC_CLUSTER) and the rows of Y with the
// same residue, writes every diagonal block (they depend on the angles
// only), and pushes its updated off-diagonal blocks into the other CTAs'
// copies through distributed shared memory; one cluster barrier per round
// orders the pushes before the next round's angles (and one after the
// copies are initialised, before the first push).  Each element is
// computed by the same formula from the same inputs as in the one-CTA form,
// so both give the same bits.
#include "te_common.cuh"
#include "te_internal.h"

namespace te {

constexpr int JAC_THREADS = 256;
constexpr int JAC_MAX_SWEEPS = 100;
constexpr int JLD = MAX_M + 1;  // padded row length in shared memory
constexpr int JAC_CLUSTER = 8;  // CTAs of the cluster form (a portable cluster size)
constexpr int JAC_CLUSTER_MIN_M = 40;  // smaller T: one CTA (barriers would dominate)

TE_DEV uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// the shared::cluster address of the same location in CTA `rank` of the cluster
TE_DEV uint32_t cluster_map(uint32_t saddr, uint32_t rank) {
  uint32_t d;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(saddr), "r"(rank));
  return d;
}
TE_DEV void st_cluster_f64(uint32_t addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
// every thread of every CTA of the cluster; orders shared-memory writes
// (local and remote) before the barrier against reads after it
TE_DEV void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// position j of the round-robin schedule in round r (player 0 stays put)
TE_DEV int rr_player(int j, int r, int mm) { return j == 0 ? 0 : 1 + (j - 1 + r) % (mm - 1); }

TE_DEV bool sel_before(double a, int ia, double b, int ib, int which) {
  if (which == TE_WHICH_LARGEST_ALGEBRAIC) {
    if (a != b) return a > b;
    return ia < ib;
  }
  double fa = fabs(a), fb = fabs(b);
  if (fa != fb) return fa > fb;
  if ((a > 0) != (b > 0)) return a > 0;
  return ia < ib;
}

constexpr size_t JAC_SMEM = 2 * (size_t)MAX_M * JLD * sizeof(double);

template <int CL>
__global__ void __launch_bounds__(JAC_THREADS, 1) jacobi_kernel(JacobiArgs a) {
  extern __shared__ __align__(16) double jsm[];
  double* T = jsm;
  double* Y = jsm + MAX_M * JLD;
  __shared__ double rc[MAX_M / 2], rs[MAX_M / 2], rt[MAX_M / 2];
  __shared__ double d_pp[MAX_M / 2], d_qq[MAX_M / 2], d_pq[MAX_M / 2];
  __shared__ int rp_[MAX_M / 2], rq_[MAX_M / 2], rot[MAX_M / 2];
  __shared__ int any_rot;
  __shared__ int sel[MAX_M];
  __shared__ double thr_s;
  __shared__ double off_part[JAC_THREADS];  // the off-diagonal check's partial maxima
  // the (a, b) pair indices of block e, a <= b, row-major upper triangle
  constexpr int MAX_BLK = MAX_M / 2 * (MAX_M / 2 + 1) / 2;
  __shared__ unsigned char blk_a[MAX_BLK], blk_b[MAX_BLK];

  const int tid = threadIdx.x;
  const int m = a.m;
  const int mm = m + (m & 1);  // even size; a dummy index never rotates
  const int half = mm / 2;
  const int nblk = half * (half + 1) / 2;
  // The rotation of pair k is computed by thread (k % 4) * 32 + k / 4: the
  // pairs spread over four warps, one per scheduler, so that their binary64
  // divisions and square roots issue from all four schedulers of the SM.
  const int rk = (tid & 31) * 4 + (tid >> 5);  // the pair thread tid computes
  const bool rthread = tid < 128 && rk < half;
  // this CTA's share: blocks e = rank + i CL (i < nb_mine), rows of Y
  // r = rank + i CL (i < ny_rows); CL = 1: everything
  const int rank = CL > 1 ? (int)cluster_ctarank() : 0;
  const int nb_mine = (nblk - rank + CL - 1) / CL;
  const int ny_rows = (mm - rank + CL - 1) / CL;
  const uint32_t T_s = smem_addr(T);

  for (int e = tid; e < mm * mm; e += JAC_THREADS) {
    const int r = e / mm, c = e % mm;
    double v = 0.0;
    if (r < m && c < m) {
      if (r == c) v = a.alpha[r];
      else if (r - c == 1 || c - r == 1) v = a.beta[r > c ? r : c];
    }
    T[r * JLD + c] = v;
    Y[r * JLD + c] = (r == c) ? 1.0 : 0.0;
  }
  if (tid == 0) {
    double f = 0.0;
    for (int r = 0; r < m; ++r) f += a.alpha[r] * a.alpha[r];
    for (int r = 1; r < m; ++r) f += 2.0 * a.beta[r] * a.beta[r];
    thr_s = 1e-16 * sqrt(f);
    for (int x = 0, e = 0; x < half; ++x)
      for (int y = x; y < half; ++y, ++e) {
        blk_a[e] = (unsigned char)x;
        blk_b[e] = (unsigned char)y;
      }
  }
  __syncthreads();
  // every copy of T is initialised before any CTA pushes into another
  if constexpr (CL > 1) cluster_barrier();
  const double thr = thr_s;

  int sweep = 0;
  for (; sweep < JAC_MAX_SWEEPS; ++sweep) {
    if (tid == 0) any_rot = 0;
    __syncthreads();
    for (int round = 0; round < mm - 1; ++round) {
      if (rthread) {
        const int k = rk;
        int p = rr_player(k, round, mm), q = rr_player(mm - 1 - k, round, mm);
        if (p > q) {
          int tmp = p;
          p = q;
          q = tmp;
        }
        rp_[k] = p;
        rq_[k] = q;
        const double tpq = T[p * JLD + q];
        if (fabs(tpq) > thr) {
          const double tpp = T[p * JLD + p], tqq = T[q * JLD + q];
          // t = sgn(zeta) / (|zeta| + sqrt(1 + zeta^2)) with zeta = d / (2 t_pq),
          // d = t_qq - t_pp, multiplied through by |2 t_pq|: one hypot, one
          // division and one reciprocal square root in the dependent chain
          // (sgn(0) = +1 as before)
          const double d = tqq - tpp, two = 2.0 * tpq;
          const double sz = (d == 0.0 || (d > 0.0) == (tpq > 0.0)) ? 1.0 : -1.0;
          const double t = sz * fabs(two) / (fabs(d) + hypot(d, two));
          const double c = rsqrt(1.0 + t * t);
          rc[k] = c;
          rs[k] = t * c;
          rt[k] = t;
          d_pp[k] = tpp;
          d_qq[k] = tqq;
          d_pq[k] = tpq;
          rot[k] = 1;
          any_rot = 1;
        } else {
          rot[k] = 0;
        }
      }
      __syncthreads();
      // T <- J^T T J on 2x2 blocks: block (a, b) of pairs a <= b is
      // J_a^T T[{p_a,q_a},{p_b,q_b}] J_b, written with its mirror image (T
      // stays exactly symmetric); a rotated pair's own block takes the exact
      // post-rotation values.  Those diagonal blocks depend only on the angles
      // and every CTA writes all of them into its own copy; the off-diagonal
      // blocks are this CTA's share.  Y <- Y J in the same phase.
      for (int i = tid; i < half + nb_mine + half * ny_rows; i += JAC_THREADS) {
        if (i < half) {
          if (rot[i]) {
            const int pa = rp_[i], qa = rq_[i];
            T[pa * JLD + pa] = d_pp[i] - rt[i] * d_pq[i];
            T[qa * JLD + qa] = d_qq[i] + rt[i] * d_pq[i];
            T[pa * JLD + qa] = 0.0;
            T[qa * JLD + pa] = 0.0;
          }
        } else if (i < half + nb_mine) {
          const int e = rank + (i - half) * CL;
          const int a = blk_a[e], b = blk_b[e];
          if (a == b || (!rot[a] && !rot[b])) continue;
          const int pa = rp_[a], qa = rq_[a], pb = rp_[b], qb = rq_[b];
          double x00 = T[pa * JLD + pb], x01 = T[pa * JLD + qb];
          double x10 = T[qa * JLD + pb], x11 = T[qa * JLD + qb];
          if (rot[a]) {  // rows: J_a^T
            const double c = rc[a], sn = rs[a];
            const double y00 = c * x00 - sn * x10, y01 = c * x01 - sn * x11;
            const double y10 = sn * x00 + c * x10, y11 = sn * x01 + c * x11;
            x00 = y00; x01 = y01; x10 = y10; x11 = y11;
          }
          if (rot[b]) {  // columns: J_b
            const double c = rc[b], sn = rs[b];
            const double y00 = c * x00 - sn * x01, y01 = sn * x00 + c * x01;
            const double y10 = c * x10 - sn * x11, y11 = sn * x10 + c * x11;
            x00 = y00; x01 = y01; x10 = y10; x11 = y11;
          }
          T[pa * JLD + pb] = x00;
          T[pa * JLD + qb] = x01;
          T[qa * JLD + pb] = x10;
          T[qa * JLD + qb] = x11;
          T[pb * JLD + pa] = x00;
          T[qb * JLD + pa] = x01;
          T[pb * JLD + qa] = x10;
          T[qb * JLD + qa] = x11;
        } else {
          const int f = i - half - nb_mine, k = f / ny_rows, row = rank + (f % ny_rows) * CL;
          if (!rot[k]) continue;
          const int p = rp_[k], q = rq_[k];
          const double c = rc[k], sn = rs[k];
          const double gy = Y[row * JLD + p], hy = Y[row * JLD + q];
          Y[row * JLD + p] = c * gy - sn * hy;
          Y[row * JLD + q] = sn * gy + c * hy;
        }
      }
      __syncthreads();
      if constexpr (CL > 1) {
        // push this CTA's changed off-diagonal blocks (all eight positions,
        // the mirror included) into the other copies of T.  They hold no
        // element that any CTA reads for this round's angles (those lie in
        // the diagonal blocks), so a slower CTA may still be computing its
        // angles: one cluster barrier per round suffices.
        for (int i = tid; i < nb_mine * 8 * (CL - 1); i += JAC_THREADS) {
          const int j = i / (8 * (CL - 1)), rem = i - j * (8 * (CL - 1));
          const int el = rem / (CL - 1), rr = rem - el * (CL - 1);
          const int e = rank + j * CL;
          const int a = blk_a[e], b = blk_b[e];
          if (a == b || (!rot[a] && !rot[b])) continue;
          const int pa = rp_[a], qa = rq_[a], pb = rp_[b], qb = rq_[b];
          const int ra = (el & 2) ? qa : pa, cb = (el & 1) ? qb : pb;
          const int off = (el < 4) ? ra * JLD + cb : cb * JLD + ra;
          const int dst = rr < rank ? rr : rr + 1;
          st_cluster_f64(cluster_map(T_s + (uint32_t)off * 8u, (uint32_t)dst), T[off]);
        }
        cluster_barrier();
      }
    }
    if (!any_rot) break;
    // When no |t_pq| off the diagonal exceeds thr, the next sweep's first
    // round rotates nothing, so T stays as it is and no later round rotates
    // either: that sweep is skipped (same bits, and the same sweep count).
    // The CTAs of a cluster hold the same T and all take the same decision.
    {
      double mx = 0.0;
      for (int e = tid; e < m * m; e += JAC_THREADS) {
        const int r = e / m, c = e - r * m;
        if (r != c) mx = fmax(mx, fabs(T[r * JLD + c]));
      }
      off_part[tid] = mx;
      __syncthreads();
      for (int w = JAC_THREADS / 2; w > 0; w >>= 1) {
        if (tid < w) off_part[tid] = fmax(off_part[tid], off_part[tid + w]);
        __syncthreads();
      }
      if (off_part[0] <= thr) {
        ++sweep;
        break;
      }
    }
    __syncthreads();
  }
  if constexpr (CL > 1) {
    // the rows of Y into CTA 0, which selects and writes the outputs
    const uint32_t Y0 = cluster_map(smem_addr(Y), 0u);
    if (rank != 0)
      for (int i = tid; i < ny_rows * mm; i += JAC_THREADS) {
        const int row = rank + (i / mm) * CL, c = i % mm;
        st_cluster_f64(Y0 + (uint32_t)(row * JLD + c) * 8u, Y[row * JLD + c]);
      }
    cluster_barrier();
    if (rank != 0) return;
  }

  // selection: rank of each Ritz value under the selection order
  if (tid < m) {
    const double th = T[tid * JLD + tid];
    int rank = 0;
    for (int l = 0; l < m; ++l)
      if (l != tid && sel_before(T[l * JLD + l], l, th, tid, a.which)) ++rank;
    sel[rank] = tid;
  }
  __syncthreads();
  double* eigvals_dev = a.eigvals_dev;
  if (a.st != nullptr) eigvals_dev = a.st->eigvals_out;
  // one warp per selected pair: sign, outputs, Ritz coefficients
  const int wid = tid >> 5, lane = tid & 31;
  for (int k = wid; k < a.K; k += JAC_THREADS / 32) {
    const int j = sel[k];
    // largest-magnitude entry of y (lowest index on ties)
    double best = -1.0;
    int bi = m;
    for (int r = lane; r < m; r += 32) {
      const double v = fabs(Y[r * JLD + j]);
      if (v > best || (v == best && r < bi)) {
        best = v;
        bi = r;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    const double sgn = Y[bi * JLD + j] < 0.0 ? -1.0 : 1.0;
    const double th = T[j * JLD + j];
    if (lane == 0) {
      a.theta_out[k] = th;
      if (eigvals_dev) eigvals_dev[k] = th;
      if (a.resid_out) a.resid_out[k] = fabs(a.beta[m] * Y[(m - 1) * JLD + j]);
    }
    for (int r = lane; r < m; r += 32) {
      const double y = sgn * Y[r * JLD + j];
      if (a.Y_out) a.Y_out[(size_t)k * m + r] = y;
      if (a.C_out) a.C_out[(size_t)r * a.K + k] = (a.s ? a.s[r] : 1.0) * y;
    }
  }
  if (tid == 0) {
    const int conv = sweep < JAC_MAX_SWEEPS;
    if (a.sweeps_out) *a.sweeps_out = sweep;
    if (a.status_out) *a.status_out = conv ? 0 : (int)TE_ERR_NOT_CONVERGED;
    if (a.st) {
      a.st->sweeps = sweep;
      if (!conv && a.st->status == 0) a.st->status = (int)TE_ERR_NOT_CONVERGED;
    }
  }
}

cudaError_t jacobi_prepare() {
  cudaError_t e = cudaFuncSetAttribute(jacobi_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)JAC_SMEM);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(jacobi_kernel<JAC_CLUSTER>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)JAC_SMEM);
}

cudaError_t launch_jacobi(const JacobiArgs& a, cudaStream_t s) {
  if (a.m < JAC_CLUSTER_MIN_M) {
    jacobi_kernel<1><<<1, JAC_THREADS, JAC_SMEM, s>>>(a);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(JAC_CLUSTER, 1, 1);
  cfg.blockDim = dim3(JAC_THREADS, 1, 1);
  cfg.dynamicSmemBytes = JAC_SMEM;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = JAC_CLUSTER;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, jacobi_kernel<JAC_CLUSTER>, a);
}

}  // namespace te
