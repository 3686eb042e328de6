// te_reorth.cu - the passes over the Lanczos basis for sm_103a: the
// three-term update and the reorthogonalisation of Algorithm 1 (done as
// classical Gram-Schmidt applied twice), the normalisation that yields beta
// and the next basis vector, and the Ritz-vector contraction V*Y
// (Section III).
//
// One persistent kernel template serves every pass.  The basis V holds rows
// padded to a multiple of TILE_R (the padding kept at zero) in tiles of TILE_R
// rows; a solve plan stores it tile-major (the columns of one tile side by
// side, so that one bulk copy moves a tile's columns), the serving engine
// column-major.  Column j holds an unnormalised vector whose scale s_j (so
// that v_j = s_j * stored_j) lives in the device state.  A stage of the
// pipeline holds a group of G consecutive tiles (G > 1 when the tiles are
// small, so that each stage still moves tens of KB) and the pass vector's
// rows; a CTA owns every gridDim.x-th group.  One producer warp moves the
// stage into shared memory with bulk (TMA) copies into a multi-stage mbarrier
// pipeline; eight consumer warps then, tile by tile,
//   phase A (axpy):  w_r = xscale * x_r - sum_j c_j V[r, j]    (thread per row)
//   phase B (dots):  g_j += sum_r V[r, j] w_r                  (warp per column)
// so the second Gram-Schmidt sweep's dot products read the same shared-memory
// tile as the first sweep's update: one HBM read of V per fused pass.  The
// per-CTA sums go to a partial buffer; the last CTA to finish (ticket counter)
// reduces them in a fixed order and computes the next pass's coefficients,
// alpha, beta and the breakdown flag on the device - no host round trip.
//
// Precision: DDD uses binary64 FMA.  FDF stores V in binary32 and carries
// every product and sum in double-float (te_common.cuh); per-CTA partials are
// double-float, the final cross-CTA sums binary64.
#include "te_common.cuh"
#include "te_internal.h"

namespace te {

template <int P>
struct PassTr;
template <>
struct PassTr<PREC_DDD> {
  using basis_t = double;
  using vec_t = double;
  using acc_t = double;
  using coef_t = double;
  using part_t = double;
};
template <>
struct PassTr<PREC_FDF> {
  using basis_t = float;
  using vec_t = float2;
  using acc_t = dacc;
  using coef_t = float2;
  using part_t = float2;  // a double-float partial sum as stored
};

constexpr uint32_t WAIT_LIMIT = 1u << 22;
// the shortened limit of a pass stalled by the test hook (stall_first_pass)
constexpr uint32_t STALL_WAIT_LIMIT = 1u << 12;
// FDF tiles are half the size of DDD tiles: two CTAs per SM still double-buffer
__host__ __device__ constexpr int pass_ctas_per_sm(int prec) { return prec == PREC_FDF ? 2 : 1; }
constexpr int QMAX = MAX_M / (CONSUMERS / 32);  // dot columns per warp
constexpr int RITZ_KC = 8;                      // Ritz outputs per register block
constexpr int RITZ_JG = 16;                     // FDF Ritz: basis columns per binary32 partial sum
constexpr int RED_LOADS = 10;                   // partial loads per lane in flight

// Packed binary32 pairs (Blackwell's .f32x2 instructions): the low half holds
// the first value.  Each half is computed and rounded as the scalar
// instruction with the same rounding mode would.
TE_DEV uint64_t f32x2_pack(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
TE_DEV void f32x2_unpack(uint64_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
TE_DEV uint64_t f32x2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
TE_DEV uint64_t f32x2_add(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
TE_DEV uint64_t f32x2_sub(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// tile groups of a tile-major basis: stages of up to GROUP_BYTES (and at
// most half the stage region, so that two stages fit), at most GROUP_MAX
// tiles, and at least GROUP_MIN_PER_CTA groups for every CTA
constexpr uint32_t GROUP_BYTES = 48u << 10;
constexpr int GROUP_MAX = 16;
constexpr int GROUP_MIN_PER_CTA = 8;

__host__ __device__ constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct SmemPlan {
  size_t region, ws_off, coef_off, coef2_off, ritz_off, red_off, fin_off, bar_off, total;
};
// finalize scratch (doubles): copies of s, alpha, beta, the c_j, warp sums
constexpr int FIN_SCRATCH = 4 * (MAX_M + 2) + 2 * (CONSUMERS / 32) + 8;
// ritz_elems: m*K coefficients held by the Ritz pass (0 for the other passes)
__host__ __device__ inline SmemPlan smem_plan(int mode, size_t region, int ritz_elems) {
  SmemPlan p{};
  p.region = region;
  p.ws_off = align_up(region, 128);
  p.coef_off = p.ws_off + TILE_R * 8;
  p.coef2_off = p.coef_off + (MAX_M + 2) * 8;
  p.ritz_off = p.coef2_off + (MAX_M + 2) * 8;
  size_t ritz = (mode == MODE_RITZ) ? align_up((size_t)ritz_elems * 8, 128) : 0;
  p.red_off = p.ritz_off + ritz;
  p.fin_off = align_up(p.red_off + PSTRIDE * 8, 8);
  p.bar_off = p.fin_off + FIN_SCRATCH * 8;
  p.total = p.bar_off + 2 * MAX_STAGES * 8 + 16;
  return p;
}

// ---------------------------------------------------------------------------
// small helpers specialised per precision
// ---------------------------------------------------------------------------
template <int P>
TE_DEV typename PassTr<P>::acc_t zero_acc() {
  if constexpr (P == PREC_FDF) return dacc_zero();
  else return 0.0;
}
// acc += v * c
template <int P>
TE_DEV void acc_fma(typename PassTr<P>::acc_t& acc, typename PassTr<P>::basis_t v,
                    typename PassTr<P>::coef_t c) {
  if constexpr (P == PREC_FDF) dacc_fma(acc, v, c.x, c.y);
  else acc = fma(v, c, acc);
}
template <int P>
TE_DEV typename PassTr<P>::acc_t acc_merge(typename PassTr<P>::acc_t a,
                                           typename PassTr<P>::acc_t b) {
  if constexpr (P == PREC_FDF) return dacc_merge(a, b);
  else return a + b;
}
template <int P>
TE_DEV typename PassTr<P>::coef_t to_coef(double c) {
  if constexpr (P == PREC_FDF) {
    dw d = dw_from_double(c);
    return make_float2(d.hi, d.lo);
  } else {
    return c;
  }
}
template <int P>
TE_DEV typename PassTr<P>::vec_t vec_from_double(double x) {
  if constexpr (P == PREC_FDF) {
    dw d = dw_from_double(x);
    return make_float2(d.hi, d.lo);
  } else {
    return x;
  }
}
template <int P>
TE_DEV typename PassTr<P>::vec_t vec_zero() {
  if constexpr (P == PREC_FDF) return make_float2(0.f, 0.f);
  else return 0.0;
}
// partial slot (8 bytes) <-> accumulator
// per-CTA partial sums, slot-major: the CTAs' values of one slot are adjacent,
// so that the last CTA reads each slot with coalesced loads
TE_DEV size_t pidx(int slot, int cta, int ncta) { return (size_t)slot * ncta + cta; }

template <int P>
TE_DEV void put_partial(void* part, size_t idx, typename PassTr<P>::acc_t a) {
  if constexpr (P == PREC_FDF) static_cast<float2*>(part)[idx] = dw_to_f2(dacc_value(a));
  else static_cast<double*>(part)[idx] = a;
}
template <int P>
TE_DEV typename PassTr<P>::part_t load_partial(const void* part, size_t idx) {
  using T = typename PassTr<P>::part_t;
  return __ldcg(static_cast<const T*>(part) + idx);
}
template <int P>
TE_DEV void add_partial(typename PassTr<P>::acc_t& acc, typename PassTr<P>::part_t v) {
  if constexpr (P == PREC_FDF) dacc_add_pair(acc, v.x, v.y);
  else acc += v;
}
template <int P>
TE_DEV double acc_to_double(typename PassTr<P>::acc_t a) {
  if constexpr (P == PREC_FDF) return dw_to_double(dacc_value(a));
  else return a;
}

// ---------------------------------------------------------------------------
// last-CTA epilogue: turns the reduced sums into the next coefficients
// ---------------------------------------------------------------------------
// Run by every consumer thread of the last CTA (tid = 0 .. CONSUMERS-1): the
// loops over basis columns are spread over the threads, the scalar updates
// are made by thread 0.  `scr` is FIN_SCRATCH doubles of shared memory.
TE_DEV void finalize_pass(const PassArgs& a, const double* tot, double* scr, const int tid) {
  LzState* st = a.st;
  const int i = a.step;
  switch (a.fin) {
    case FIN_DOT_STEP: {
      // tot[j] = stored_j . ytilde with y = s_i ytilde = M v_i
      const double si = st->s[i];
      for (int j = tid; j < a.nb; j += CONSUMERS) {
        const double sj = st->s[j];
        const double h = sj * si * tot[j];  // v_j . M v_i (first sweep)
        st->c1[j] = h * sj;
      }
      // Algorithm 1's alpha_i = v_i . M v_i; the second sweep adds its
      // correction (FIN_AXPYDOT_STEP), so alpha keeps full accuracy even when
      // the first sweep's dots are taken in binary32 chunks
      if (tid == 0) {
        st->alpha[i] = si * si * tot[i];
        st->xscale = si;
      }
      break;
    }
    case FIN_AXPYDOT_STEP: {
      for (int j = tid; j < a.nb; j += CONSUMERS) st->c2[j] = st->s[j] * st->s[j] * tot[j];
      if (tid == 0) st->alpha[i] += st->s[i] * tot[i];  // + v_i . w after the first sweep
      break;
    }
    case FIN_DOT_RESTART: {
      for (int j = tid; j < a.nb; j += CONSUMERS) st->c1[j] = st->s[j] * st->s[j] * tot[j];
      if (tid == 0) st->xscale = 1.0;
      break;
    }
    case FIN_AXPYDOT: {
      for (int j = tid; j < a.nb; j += CONSUMERS) st->c2[j] = st->s[j] * st->s[j] * tot[j];
      break;
    }
    case FIN_STORE_STEP:
    case FIN_STORE_NOREORTH: {
      if (tid != 0) break;
      // tot[0] = ||w||^2, tot[1] = ||stored(w)||^2 (beta_{i+1} of Algorithm 1);
      // without reorthogonalisation the pass formed w / s_i
      double b = sqrt(tot[0] > 0.0 ? tot[0] : 0.0);
      if (a.fin == FIN_STORE_NOREORTH) b *= st->s[i];
      const double ns = sqrt(tot[1] > 0.0 ? tot[1] : 0.0);
      st->s[i + 1] = ns > 0.0 ? 1.0 / ns : 0.0;
      double cand = fabs(st->alpha[i]) + st->beta[i] + b;
      if (cand > st->anorm) st->anorm = cand;
      st->beta[i + 1] = b;
      st->restart_flag = 0;
      if (i + 1 < a.m && !(b > a.tol * st->anorm)) {
        st->restart_flag = 1;
        st->beta[i + 1] = 0.0;
      }
      break;
    }
    case FIN_DOT_NOREORTH: {
      if (tid != 0) break;
      // tot[0] = stored_i . ytilde: alpha_i = v_i . M v_i.  The store pass then
      // forms w / s_i = ytilde - alpha_i stored_i - (beta_i s_{i-1} / s_i) stored_{i-1}
      const double si = st->s[i];
      const double al = si * si * tot[0];
      st->alpha[i] = al;
      if (i > 0) {
        st->c2[0] = st->beta[i] * st->s[i - 1] / si;
        st->c2[1] = al;
      } else {
        st->c2[0] = al;
      }
      break;
    }
    case FIN_DCGS_DOT: {
      // Delayed second sweep of the candidate u_i = sig S_i (unit norm after
      // its first sweep): c_j = v_j . u_i, rho = ||u_i - V c||, v_i = (u_i -
      // V c) / rho.  tot[j] = S_j . ytilde, tot[nb + j] = S_j . S_i, with
      // ytilde = M S_i.  M v_j of the final columns follows the three-term
      // relation, so sum_j c_j M v_j = sum_k t_k v_k (second order in c).
      const int ni = a.nb - 1;  // = i
      constexpr int NW = CONSUMERS / 32;
      double* sv = scr;                 // s_j
      double* av = sv + (MAX_M + 2);    // alpha_j
      double* bv = av + (MAX_M + 2);    // beta_j
      double* cj = bv + (MAX_M + 2);    // c_j
      double* wred = cj + (MAX_M + 2);  // warp sums
      double* sc = wred + 2 * NW;       // scalars from thread 0
      const double sig = st->s[i];
      double pc = 0.0, ps = 0.0;
      for (int j = tid; j < ni; j += CONSUMERS) {
        const double sj = st->s[j];
        sv[j] = sj;
        av[j] = st->alpha[j];
        bv[j] = st->beta[j];
        const double c = sj * sig * tot[a.nb + j];
        cj[j] = c;
        pc = fma(c, c, pc);                // ||c||^2
        ps = fma(c * sj, tot[j], ps);      // sum_j c_j v_j . ytilde / sig
      }
      pc = warp_sum(pc);
      ps = warp_sum(ps);
      if ((tid & 31) == 0) {
        wred[tid >> 5] = pc;
        wred[NW + (tid >> 5)] = ps;
      }
      named_bar_sync(1, CONSUMERS);
      if (tid == 0) {
        double cc = 0.0, scg = 0.0;
        for (int w = 0; w < NW; ++w) {
          cc += wred[w];
          scg += wred[NW + w];
        }
        double rho = 1.0;
        if (ni > 0) {
          const double r2 = sig * sig * tot[a.nb + ni] - cc;
          rho = r2 > 0.0 ? sqrt(r2) : 0.0;
          if (!(rho > 0.0)) {
            st->status = TE_ERR_BREAKDOWN;
            rho = 1.0;
          }
        }
        const double beta_i = (ni == 0 || st->rflag[i]) ? 0.0 : st->bt[i] * rho;
        st->beta[i] = beta_i;
        st->s[i] = sig / rho;
        const double vy = (sig * tot[ni] - scg) / rho;  // v_i . ytilde
        const double t_i = ni > 0 ? cj[ni - 1] * beta_i : 0.0;
        const double al = (sig * vy - t_i) / rho;       // alpha_i = v_i . M v_i
        st->alpha[i] = al;
        const double F = t_i / rho + al;
        st->f2 = F * sig / rho;
        st->xscale = sig / rho;
        sc[0] = rho;
        sc[1] = F;
      }
      named_bar_sync(1, CONSUMERS);
      const double rho = sc[0], F = sc[1];
      for (int k = tid; k < ni; k += CONSUMERS) {
        double tk = cj[k] * av[k];
        if (k > 0) tk += cj[k - 1] * bv[k];
        if (k + 1 < ni) tk += cj[k + 1] * bv[k + 1];
        const double hk = (sig * sv[k] * tot[k] - tk) / rho;  // v_k . M v_i
        st->c1[k] = cj[k] * sv[k] / sig;
        st->c2[k] = ((tk / rho + hk) - F * cj[k] / rho) * sv[k];
      }
      break;
    }
    case FIN_DCGS_UPDATE: {
      if (tid != 0) break;
      // tot[0] = ||w||^2 (the next candidate after its first sweep), tot[1] =
      // ||stored(w)||^2; its second sweep (and final beta) comes next step
      const double b = sqrt(tot[0] > 0.0 ? tot[0] : 0.0);
      const double ns = sqrt(tot[1] > 0.0 ? tot[1] : 0.0);
      st->bt[i + 1] = b;
      st->s[i + 1] = ns > 0.0 ? 1.0 / ns : 0.0;
      st->rflag[i + 1] = 0;
      const double cand = fabs(st->alpha[i]) + st->beta[i] + b;
      if (cand > st->anorm) st->anorm = cand;
      st->restart_flag = 0;
      if (i + 1 < a.m && !(b > a.tol * st->anorm)) {
        st->restart_flag = 1;
        st->rflag[i + 1] = 1;
      }
      if (i + 1 == a.m) st->beta[i + 1] = b;  // beta_{m+1}: residual estimates
      break;
    }
    case FIN_STORE_RESTART: {
      if (tid != 0) break;
      const double b = sqrt(tot[0] > 0.0 ? tot[0] : 0.0);
      const double ns = sqrt(tot[1] > 0.0 ? tot[1] : 0.0);
      if (ns > 0.0 && b > 0.0) st->s[i + 1] = 1.0 / ns;
      else st->status = TE_ERR_BREAKDOWN;
      st->restarts += 1;
      st->restart_flag = 0;
      break;
    }
    case FIN_STORE_INIT: {
      for (int j = tid; j < MAX_M + 2; j += CONSUMERS) st->rflag[j] = 0;
      if (tid != 0) break;
      const double ns = sqrt(tot[1] > 0.0 ? tot[1] : 0.0);
      if (ns > 0.0) st->s[0] = 1.0 / ns;
      else st->status = TE_ERR_INVALID_ARG;
      st->beta[0] = 0.0;
      st->anorm = 0.0;
      st->restart_flag = 0;
      break;
    }
    default:
      break;
  }
}

// ---------------------------------------------------------------------------
// the pass kernel
// ---------------------------------------------------------------------------
// One CTA's share of a pass: CTA `cta` of `ncta` takes tiles cta, cta + ncta, ...
// (the single-solve kernel passes blockIdx.x / gridDim.x; the batched kernel
// of the serving engine maps its blocks onto the CTAs of several solves).
template <int P, int MODE>
__device__ __forceinline__ void pass_body(const PassArgs& a, size_t region, const int cta,
                                          const int ncta) {
  using Tr = PassTr<P>;
  using basis_t = typename Tr::basis_t;
  using vec_t = typename Tr::vec_t;
  using acc_t = typename Tr::acc_t;
  using coef_t = typename Tr::coef_t;
  constexpr bool HAS_AXPY = (MODE == MODE_AXPY_DOT || MODE == MODE_AXPY_STORE);
  constexpr bool HAS_DOT = (MODE == MODE_DOT || MODE == MODE_AXPY_DOT);
  constexpr bool DDOT = (MODE == MODE_DCGS_DOT);
  constexpr bool DUPD = (MODE == MODE_DCGS_UPDATE);

  extern __shared__ __align__(128) unsigned char sm[];
  LzState* st = a.st;
  if (a.only_on_restart) {
    if (*((volatile int*)&st->restart_flag) == 0) return;
  }
  const SmemPlan L = smem_plan(
      MODE, region, MODE == MODE_RITZ ? a.nb * ((a.K + RITZ_KC - 1) / RITZ_KC * RITZ_KC) : 0);
  vec_t* ws = reinterpret_cast<vec_t*>(sm + L.ws_off);
  coef_t* coef = reinterpret_cast<coef_t*>(sm + L.coef_off);
  coef_t* coef2 = reinterpret_cast<coef_t*>(sm + L.coef2_off);
  coef_t* rC = reinterpret_cast<coef_t*>(sm + L.ritz_off);
  acc_t* red = reinterpret_cast<acc_t*>(sm + L.red_off);
  double* tot = reinterpret_cast<double*>(sm + L.red_off);  // reused by the last CTA
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + L.bar_off);
  uint64_t* empty = full + MAX_STAGES;
  int* lastflag = reinterpret_cast<int*>(empty + MAX_STAGES);
  int* abortflag = lastflag + 1;

  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;
  const int64_t tiles = a.ld / TILE_R;
  const int nb = a.nb;
  // A pass vector held in memory travels with the basis tiles: the producer
  // copies its rows behind the group's columns, so that its latency is hidden
  // by the same pipeline (it is twice a column's bytes in FDF).
  const bool xst = MODE != MODE_RITZ && a.xsrc == X_VEC && nb > 0;
  const uint32_t col_bytes = (uint32_t)((size_t)nb * TILE_R * sizeof(basis_t));
  const uint32_t xbytes = xst ? (uint32_t)(TILE_R * sizeof(vec_t)) : 0u;
  // tiles per group: enough for GROUP_BYTES per stage (tile-major basis
  // only), yet at least GROUP_MIN_PER_CTA groups per CTA
  int G = 1;
  if (nb > 0 && a.cstride == TILE_R) {
    const size_t cap = region / 2 < GROUP_BYTES ? region / 2 : GROUP_BYTES;
    const int64_t gb = (int64_t)(cap / (col_bytes + xbytes));
    const int64_t gl = tiles / ((int64_t)ncta * GROUP_MIN_PER_CTA);
    int64_t g = gb < gl ? gb : gl;
    if (g > GROUP_MAX) g = GROUP_MAX;
    if (g > 1) G = (int)g;
  }
  const int64_t groups = (tiles + G - 1) / G;
  const uint32_t stage_bytes = (uint32_t)G * (col_bytes + xbytes);
  int S = 0;
  if (nb > 0) {
    S = (int)(region / stage_bytes);
    if (S > MAX_STAGES) S = MAX_STAGES;
    if (S < 1) {  // more columns than the launch was configured for
      if (threadIdx.x == 0) atomicExch(&a.st->status, (int)TE_ERR_INVALID_ARG);
      return;
    }
  }

  // test hook: a stalled pass issues no copies, so every wait of its consumers
  // expires; the last CTA disarms the hook once every CTA has read it
  const bool stall = a.stall && nb > 0 && a.fin != FIN_NONE &&
                     *((volatile int*)&st->stall_armed) != 0;
  const uint32_t wait_limit = stall ? STALL_WAIT_LIMIT : WAIT_LIMIT;
  if (tid == 0) *abortflag = 0;
  if (tid == 0 && nb > 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], CONSUMERS / 32);
    }
    fence_mbar_init();
  }
  if constexpr (MODE == MODE_AXPY_DOT) {
    for (int j = tid; j < nb; j += PASS_THREADS) coef[j] = to_coef<P>(st->c1[j]);
  }
  if constexpr (MODE == MODE_AXPY_STORE) {
    for (int j = tid; j < nb; j += PASS_THREADS) coef[j] = to_coef<P>(st->c2[j]);
  }
  if constexpr (DUPD) {
    for (int j = tid; j < nb - 1; j += PASS_THREADS) {
      coef[j] = to_coef<P>(st->c1[j]);
      coef2[j] = to_coef<P>(st->c2[j]);
    }
  }
  // Ritz coefficients C (nb x K) with the row stride padded to Kp (a multiple
  // of RITZ_KC, zeros beyond K); FDF keeps their binary32 roundings only
  const int Kp = (a.K + RITZ_KC - 1) / RITZ_KC * RITZ_KC;
  if constexpr (MODE == MODE_RITZ) {
    if (st->eigvecs == nullptr) return;  // uniform: no vectors requested
    for (int e = tid; e < nb * Kp; e += PASS_THREADS) {
      const int j = e / Kp, k = e - j * Kp;
      const double c = k < a.K ? st->C[j * a.K + k] : 0.0;
      if constexpr (P == PREC_FDF) reinterpret_cast<float*>(rC)[e] = __double2float_rn(c);
      else rC[e] = c;
    }
  }
  __syncthreads();

  const basis_t* Vg = static_cast<const basis_t*>(a.V) + (size_t)a.col0 * a.cstride;

  // ------------------------- producer warp -------------------------
  if (wid == CONSUMERS / 32) {
    if (nb > 0 && lane == 0 && !stall) {
      const uint64_t pol = policy_evict_first();
      const bool tmaj = a.cstride == TILE_R;
      int it = 0;
      bool ok = true;
      for (int64_t T = cta; T < groups; T += ncta, ++it) {
        const int s = it % S, k = it / S;
        if (k > 0 && !mbar_wait_bounded(&empty[s], (uint32_t)((k - 1) & 1), WAIT_LIMIT)) {
          atomicExch(&st->status, (int)TE_ERR_TIMEOUT);
          ok = false;
          break;
        }
        const int64_t t0 = T * G;
        const int gc = (int)(tiles - t0 < G ? tiles - t0 : G);
        mbar_arrive_expect_tx(&full[s], (uint32_t)gc * (col_bytes + xbytes));
        unsigned char* dst = sm + (size_t)s * stage_bytes;
        for (int g = 0; g < gc; ++g) {
          const basis_t* src = Vg + (t0 + g) * a.tstride;
          basis_t* d = reinterpret_cast<basis_t*>(dst + (size_t)g * col_bytes);
          if (tmaj && a.cand) {  // the final columns, then the candidate's tile
            const uint32_t vb = col_bytes - (uint32_t)(TILE_R * sizeof(basis_t));
            if (vb > 0) bulk_g2s(d, src, vb, &full[s], pol);
            bulk_g2s(d + (size_t)(nb - 1) * TILE_R,
                     static_cast<const basis_t*>(a.cand) + (t0 + g) * TILE_R,
                     (uint32_t)(TILE_R * sizeof(basis_t)), &full[s], pol);
          } else if (tmaj) {
            bulk_g2s(d, src, col_bytes, &full[s], pol);
          } else {
            for (int j = 0; j < nb; ++j)
              bulk_g2s(d + (size_t)j * TILE_R, src + (size_t)j * a.cstride,
                       (uint32_t)(TILE_R * sizeof(basis_t)), &full[s], pol);
          }
        }
        if (xst)
          bulk_g2s(dst + (size_t)G * col_bytes, static_cast<const vec_t*>(a.xvec) + t0 * TILE_R,
                   (uint32_t)gc * xbytes, &full[s], pol);
      }
      // drain: every issued copy must land before this warp retires
      const int issued = it;
      for (int s = 0; s < S && s < issued; ++s) {
        const int klast = (issued - 1 - s) / S;
        if (!mbar_wait_bounded(&full[s], (uint32_t)(klast & 1), WAIT_LIMIT)) {
          atomicExch(&st->status, (int)TE_ERR_TIMEOUT);
        }
      }
      (void)ok;
    }
    return;
  }

  // ------------------------- consumer warps -------------------------
  const double xs_d = (MODE == MODE_AXPY_DOT || DUPD) ? st->xscale : 1.0;
  coef_t xscale = to_coef<P>(xs_d);
  const coef_t fcand = to_coef<P>(DUPD ? st->f2 : 0.0);
  basis_t* Vfix = static_cast<basis_t*>(a.Vmut) + (size_t)a.col_fix * a.cstride;
  basis_t* xcopy = static_cast<basis_t*>(a.xcopy);
  const uint64_t rstream = (a.xsrc == X_V1) ? 0ull : (uint64_t)(st->restarts + 1);
  const double* v1 = st->v1;
  acc_t dots[QMAX], dots2[DDOT ? QMAX : 1];
#pragma unroll
  for (int q = 0; q < QMAX; ++q) dots[q] = zero_acc<P>();
#pragma unroll
  for (int q = 0; q < (DDOT ? QMAX : 1); ++q) dots2[q] = zero_acc<P>();
  acc_t n1 = zero_acc<P>(), n2 = zero_acc<P>();
  basis_t* Vout = static_cast<basis_t*>(a.Vmut) + (size_t)a.col_out * a.cstride;

  // the source value of a row: the pass vector, the start vector, or a
  // seeded random draw (restarts); the last two are indexed by the caller's
  // row (perm maps the solver's rows to the caller's)
  auto load_x = [&](int64_t row) {
    vec_t v = vec_zero<P>();
    if constexpr (MODE != MODE_RITZ) {
      if (a.xsrc == X_VEC) {
        v = static_cast<const vec_t*>(a.xvec)[row];
      } else if (row < a.n) {
        const int64_t orow = a.perm ? (int64_t)a.perm[row] : row;
        if (a.xsrc == X_V1 && v1 != nullptr) v = vec_from_double<P>(v1[orow]);
        else v = vec_from_double<P>(sm64_uniform_pm1(a.seed, rstream, (uint64_t)orow));
      }
    }
    return v;
  };
  int it = 0;
  for (int64_t T = cta; T < groups; T += ncta, ++it) {
    int s = 0;
    if (nb > 0) {
      s = it % S;
      if (!mbar_wait_bounded(&full[s], (uint32_t)((it / S) & 1), wait_limit)) {
        atomicExch(&st->status, (int)TE_ERR_TIMEOUT);
        *abortflag = 1;
      }
      // every consumer leaves together if any of them gave up waiting
      named_bar_sync(1, CONSUMERS);
      if (*abortflag) break;
    }
    const unsigned char* sbase = sm + (size_t)s * stage_bytes;
    const int64_t t0 = T * G;
    const int gc = (int)(tiles - t0 < G ? tiles - t0 : G);
    for (int g = 0; g < gc; ++g) {
      const int64_t t = t0 + g;
      const int64_t row = t * TILE_R + tid;
      const int64_t vrow = t * a.tstride + tid;  // this row's element of a basis column
      const basis_t* tv = reinterpret_cast<const basis_t*>(sbase + (size_t)g * col_bytes);
      const vec_t* xs = reinterpret_cast<const vec_t*>(sbase + (size_t)G * col_bytes);
      const vec_t x = xst ? xs[g * TILE_R + tid] : load_x(row);

      if constexpr (HAS_AXPY) {
        // phase A: t_r = sum_j c_j V[r, j] with four independent chains
        acc_t tacc;
        if constexpr (P == PREC_FDF) {
          // Only two coefficients can be large: those of v_i and v_{i-1} in the
          // first sweep (alpha_i and beta_i of the three-term recurrence).  The
          // others sit at the basis' loss-of-orthogonality level, as do all
          // second-sweep coefficients, so binary32 products and sums of those
          // columns add an error far below the binary32 rounding of the stored
          // result.  The host marks the trailing columns whose coefficients can
          // be large (exact_tail: 2 in the first sweep, all of them without
          // reorthogonalisation and in restarts); those are taken exactly in
          // double-float.
          const int nsmall = nb > a.exact_tail ? nb - a.exact_tail : 0;
          float f[4] = {0.f, 0.f, 0.f, 0.f};
          int j = 0;
          for (; j + 4 <= nsmall; j += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              f[u] = __fmaf_rn(tv[(size_t)(j + u) * TILE_R + tid], coef[j + u].x, f[u]);
          }
          for (; j < nsmall; ++j) f[0] = __fmaf_rn(tv[(size_t)j * TILE_R + tid], coef[j].x, f[0]);
          tacc = dacc_zero();
          dacc_add_pair(tacc, __fadd_rn(f[0], f[1]), __fadd_rn(f[2], f[3]));
          for (; j < nb; ++j) acc_fma<P>(tacc, tv[(size_t)j * TILE_R + tid], coef[j]);
        } else {
          acc_t ta[4] = {zero_acc<P>(), zero_acc<P>(), zero_acc<P>(), zero_acc<P>()};
          int j = 0;
          for (; j + 4 <= nb; j += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
              acc_fma<P>(ta[u], tv[(size_t)(j + u) * TILE_R + tid], coef[j + u]);
          }
          for (; j < nb; ++j) acc_fma<P>(ta[0], tv[(size_t)j * TILE_R + tid], coef[j]);
          tacc = acc_merge<P>(acc_merge<P>(ta[0], ta[1]), acc_merge<P>(ta[2], ta[3]));
        }
        vec_t w;
        if constexpr (P == PREC_FDF) {
          dw xv = dw_from_f2(x);
          dw sx = (MODE == MODE_AXPY_DOT) ? dw_mul(dw_from_f2(xscale), xv) : xv;
          dw wd = dw_sub(sx, dacc_value(tacc));
          w = dw_to_f2(wd);
        } else {
          w = (MODE == MODE_AXPY_DOT) ? fma(xscale, x, -tacc) : x - tacc;
        }
        if constexpr (MODE == MODE_AXPY_DOT) {
          static_cast<vec_t*>(a.wout)[row] = w;
          ws[tid] = w;
          if constexpr (P == PREC_FDF) {
            // the second-sweep dot of column i (it enters alpha_i) is exact; a
            // thread per row keeps the warps of phase B balanced
            dacc_fma(n1, tv[(size_t)(nb - 1) * TILE_R + tid], w.x, w.y);
          }
        } else {
          // store the next basis vector (unnormalised) and its two norms
          if constexpr (P == PREC_FDF) {
            Vout[vrow] = w.x;
            if (xcopy) xcopy[row] = w.x;
            dacc_fma(n1, w.x, w.x, 2.0f * w.y);
            dacc_fma(n2, w.x, w.x, 0.0f);
          } else {
            Vout[vrow] = w;
            if (xcopy) xcopy[row] = w;
            n1 = fma(w, w, n1);
          }
        }
      } else if constexpr (MODE == MODE_DOT || DDOT) {
        ws[tid] = x;
      }
      if constexpr (DDOT) {
        // the candidate's own two dots (u' y gives alpha, u' u its norm) are
        // exact; a thread per row keeps the warps of phase B balanced
        const basis_t sc = tv[(size_t)(nb - 1) * TILE_R + tid];
        if constexpr (P == PREC_FDF) {
          dacc_fma(n1, sc, x.x, x.y);
          dacc_fma(n2, sc, sc, 0.0f);
        } else {
          n1 = fma(sc, x, n1);
          n2 = fma(sc, sc, n2);
        }
      }

      if constexpr (DUPD) {
        // delayed reorthogonalisation, thread per row: the candidate column
        // (tile column nb-1) loses its components along the final columns
        // (coefficients e1, all small) and is stored back as final; the next
        // candidate is w = xscale * y - sum_k e2_k S_k - f2 * candidate, where
        // only e2 of column nb-2 (the beta term) and f2 (the alpha term) can be
        // large and are taken in double-float.
        const basis_t sc = tv[(size_t)(nb - 1) * TILE_R + tid];
        const int nj = nb - 1;
        vec_t w;
        if constexpr (P == PREC_FDF) {
          const int nsmall = nj > 1 ? nj - 1 : 0;
          float f1[4] = {0.f, 0.f, 0.f, 0.f}, g1[4] = {0.f, 0.f, 0.f, 0.f};
          int j = 0;
          for (; j + 4 <= nsmall; j += 4) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float v = tv[(size_t)(j + u) * TILE_R + tid];
              f1[u] = __fmaf_rn(v, coef[j + u].x, f1[u]);
              g1[u] = __fmaf_rn(v, coef2[j + u].x, g1[u]);
            }
          }
          for (; j < nsmall; ++j) {
            const float v = tv[(size_t)j * TILE_R + tid];
            f1[0] = __fmaf_rn(v, coef[j].x, f1[0]);
            g1[0] = __fmaf_rn(v, coef2[j].x, g1[0]);
          }
          dacc t2 = dacc_zero();
          dacc_add_pair(t2, __fadd_rn(g1[0], g1[1]), __fadd_rn(g1[2], g1[3]));
          for (; j < nj; ++j) {
            const float v = tv[(size_t)j * TILE_R + tid];
            f1[0] = __fmaf_rn(v, coef[j].x, f1[0]);
            acc_fma<P>(t2, v, coef2[j]);
          }
          acc_fma<P>(t2, sc, fcand);
          const float t1 = __fadd_rn(__fadd_rn(f1[0], f1[1]), __fadd_rn(f1[2], f1[3]));
          if (nj > 0) Vfix[vrow] = __fsub_rn(sc, t1);
          const dw sx = dw_mul(dw_from_f2(xscale), dw_from_f2(x));
          w = dw_to_f2(dw_sub(sx, dacc_value(t2)));
          if (!a.cand) Vout[vrow] = w.x;  // (the delayed form keeps it in the copy only)
          if (xcopy) xcopy[row] = w.x;
          dacc_fma(n1, w.x, w.x, 2.0f * w.y);
          dacc_fma(n2, w.x, w.x, 0.0f);
        } else {
          double t1 = 0.0, t2 = 0.0;
          for (int j = 0; j < nj; ++j) {
            const double v = tv[(size_t)j * TILE_R + tid];
            t1 = fma(v, coef[j], t1);
            t2 = fma(v, coef2[j], t2);
          }
          t2 = fma(sc, fcand, t2);
          if (nj > 0) Vfix[vrow] = sc - t1;
          w = fma(xscale, x, -t2);
          if (!a.cand) Vout[vrow] = w;
          if (xcopy) xcopy[row] = w;
          n1 = fma(w, w, n1);
        }
      }

      if constexpr (DDOT) {
        named_bar_sync(1, CONSUMERS);
        // delayed reorthogonalisation, warp per column: the dot of every column
        // with y (the first sweep of the new vector) and with the candidate
        // column nb-1 (the second sweep of the previous one).  Binary32 chunks
        // for the columns before the candidate (their errors are removed by the
        // next step's sweep); the candidate's own two dots (u' y gives alpha,
        // u' u its norm) exactly.
        const basis_t* cand = tv + (size_t)(nb - 1) * TILE_R;
        if constexpr (P == PREC_FDF) {
          float wx[TILE_R / 32], cx[TILE_R / 32];
#pragma unroll
          for (int rr = 0; rr < TILE_R / 32; ++rr) {
            wx[rr] = ws[lane + 32 * rr].x;
            cx[rr] = cand[lane + 32 * rr];
          }
#pragma unroll
          for (int q = 0; q < QMAX; ++q) {
            const int jj = wid + (CONSUMERS / 32) * q;
            if (jj >= nb - 1) break;
            const basis_t* col = tv + (size_t)jj * TILE_R;
            float c0 = 0.f, c1 = 0.f, d0 = 0.f, d1 = 0.f;
#pragma unroll
            for (int rr = 0; rr < TILE_R / 32; rr += 2) {
              const float v0 = col[lane + 32 * rr], v1 = col[lane + 32 * (rr + 1)];
              c0 = __fmaf_rn(v0, wx[rr], c0);
              c1 = __fmaf_rn(v1, wx[rr + 1], c1);
              d0 = __fmaf_rn(v0, cx[rr], d0);
              d1 = __fmaf_rn(v1, cx[rr + 1], d1);
            }
            dacc_add_pair(dots[q], c0, c1);
            dacc_add_pair(dots2[q], d0, d1);
          }
        } else {
#pragma unroll
          for (int q = 0; q < QMAX; ++q) {
            const int jj = wid + (CONSUMERS / 32) * q;
            if (jj >= nb - 1) break;
            const basis_t* col = tv + (size_t)jj * TILE_R;
#pragma unroll
            for (int rr = 0; rr < TILE_R / 32; ++rr) {
              dots[q] = fma(col[lane + 32 * rr], ws[lane + 32 * rr], dots[q]);
              dots2[q] = fma(col[lane + 32 * rr], cand[lane + 32 * rr], dots2[q]);
            }
          }
        }
      }

      if constexpr (HAS_DOT) {
        named_bar_sync(1, CONSUMERS);
        // phase B: warp `wid` owns columns wid, wid+8, ...; lanes stride rows.
        // The column loop stops at this warp's last column (uniform branch).
        // FDF sums the dots in binary32 over the tile's 8 rows per lane and
        // adds each chunk exactly.  For the first sweep the error is removed by
        // the second; for the second sweep it leaves a component of about
        // u32 |w| along V, the level of w's own binary32 rounding.  The one
        // second-sweep dot that enters alpha_i (column i, the last) keeps
        // exact products and double-float sums, and so does alpha_i's dot
        // without reorthogonalisation (no second sweep corrects it).  Each
        // lane's 8 vector values are read from shared memory once per tile.
        if constexpr (P == PREC_FDF) {
          float wx[TILE_R / 32], wy[TILE_R / 32];
#pragma unroll
          for (int rr = 0; rr < TILE_R / 32; ++rr) {
            const float2 t = ws[lane + 32 * rr];
            wx[rr] = t.x;
            wy[rr] = t.y;
          }
          // (AXPY_DOT's last column is summed thread per row above)
          const int jend = MODE == MODE_AXPY_DOT ? nb - 1 : nb;
#pragma unroll
          for (int q = 0; q < QMAX; ++q) {
            const int jj = wid + (CONSUMERS / 32) * q;
            if (jj >= jend) break;
            const basis_t* col = tv + (size_t)jj * TILE_R;
            if ((MODE == MODE_DOT && a.fin != FIN_DOT_NOREORTH) ||
                (MODE == MODE_AXPY_DOT && jj < nb - 1)) {
              float c0 = 0.f, c1 = 0.f;
#pragma unroll
              for (int rr = 0; rr < TILE_R / 32; rr += 2) {
                c0 = __fmaf_rn(col[lane + 32 * rr], wx[rr], c0);
                c1 = __fmaf_rn(col[lane + 32 * (rr + 1)], wx[rr + 1], c1);
              }
              dacc_add_pair(dots[q], c0, c1);
            } else {
              acc_t e0 = zero_acc<P>(), e1 = zero_acc<P>();
#pragma unroll
              for (int rr = 0; rr < TILE_R / 32; rr += 2) {
                dacc_fma(e0, col[lane + 32 * rr], wx[rr], wy[rr]);
                dacc_fma(e1, col[lane + 32 * (rr + 1)], wx[rr + 1], wy[rr + 1]);
              }
              dots[q] = acc_merge<P>(dots[q], acc_merge<P>(e0, e1));
            }
          }
        } else {
#pragma unroll
          for (int q = 0; q < QMAX; ++q) {
            const int jj = wid + (CONSUMERS / 32) * q;
            if (jj >= nb) break;
            const basis_t* col = tv + (size_t)jj * TILE_R;
            acc_t e0 = zero_acc<P>(), e1 = zero_acc<P>();
#pragma unroll
            for (int rr = 0; rr < TILE_R / 32; rr += 2) {
              e0 = fma(col[lane + 32 * rr], ws[lane + 32 * rr], e0);
              e1 = fma(col[lane + 32 * (rr + 1)], ws[lane + 32 * (rr + 1)], e1);
            }
            dots[q] = acc_merge<P>(dots[q], acc_merge<P>(e0, e1));
          }
        }
      }

      if constexpr (MODE == MODE_RITZ) {
        const int K = a.K;
        double* U = st->eigvecs;
        for (int k0 = 0; k0 < K; k0 += RITZ_KC) {
          acc_t ra[RITZ_KC];
#pragma unroll
          for (int kk = 0; kk < RITZ_KC; ++kk) ra[kk] = zero_acc<P>();
          if constexpr (P == PREC_FDF) {
            // binary32 partial sums over RITZ_JG basis columns, each added
            // exactly to a double-float accumulator: the error stays within a
            // small multiple of the binary32 rounding the stored basis already
            // has.  The coefficients of a column come in 16-byte broadcasts.
            // Outputs go in pairs through the packed binary32 instructions
            // (fma/add/sub .rn.f32x2): each half rounds as the scalar
            // instruction would, so the results are those of the scalar
            // form, with half the FMA and double-float addition instructions.
            const float* rh = reinterpret_cast<const float*>(rC) + k0;
            uint64_t as2[RITZ_KC / 2], ac2[RITZ_KC / 2];  // double-float (s, c) pairs
#pragma unroll
            for (int q = 0; q < RITZ_KC / 2; ++q) as2[q] = ac2[q] = 0ull;
            for (int j0 = 0; j0 < nb; j0 += RITZ_JG) {
              uint64_t f2[RITZ_KC / 2];
#pragma unroll
              for (int q = 0; q < RITZ_KC / 2; ++q) f2[q] = 0ull;
              const int j1 = j0 + RITZ_JG < nb ? j0 + RITZ_JG : nb;
#pragma unroll 4
              for (int j = j0; j < j1; ++j) {
                const float v = tv[(size_t)j * TILE_R + tid];
                const uint64_t vv = f32x2_pack(v, v);
#pragma unroll
                for (int k4 = 0; k4 < RITZ_KC; k4 += 4) {
                  const ulonglong2 c = *reinterpret_cast<const ulonglong2*>(rh + j * Kp + k4);
                  f2[k4 / 2] = f32x2_fma(vv, c.x, f2[k4 / 2]);
                  f2[k4 / 2 + 1] = f32x2_fma(vv, c.y, f2[k4 / 2 + 1]);
                }
              }
              // (s, c) += (f, 0) exactly, as dacc_add_pair does per output
#pragma unroll
              for (int q = 0; q < RITZ_KC / 2; ++q) {
                const uint64_t sn = f32x2_add(as2[q], f2[q]);
                const uint64_t bb = f32x2_sub(sn, as2[q]);
                const uint64_t es = f32x2_add(f32x2_sub(as2[q], f32x2_sub(sn, bb)),
                                              f32x2_sub(f2[q], bb));
                as2[q] = sn;
                ac2[q] = f32x2_add(ac2[q], f32x2_add(es, 0ull));
              }
            }
#pragma unroll
            for (int q = 0; q < RITZ_KC / 2; ++q) {
              f32x2_unpack(as2[q], ra[2 * q].s, ra[2 * q + 1].s);
              f32x2_unpack(ac2[q], ra[2 * q].c, ra[2 * q + 1].c);
            }
          } else {
            for (int j = 0; j < nb; ++j) {
              const basis_t v = tv[(size_t)j * TILE_R + tid];
#pragma unroll
              for (int kk = 0; kk < RITZ_KC; ++kk) acc_fma<P>(ra[kk], v, rC[j * Kp + k0 + kk]);
            }
          }
          if (row < a.n) {
            double o[RITZ_KC];
#pragma unroll
            for (int kk = 0; kk < RITZ_KC; ++kk) {
              if constexpr (P == PREC_FDF) o[kk] = dw_to_double_bits(dacc_value(ra[kk]));
              else o[kk] = ra[kk];
            }
            if (a.urows) {  // by rows: pairs of outputs as 16-byte stores
              double2* ur = reinterpret_cast<double2*>(a.urows + (size_t)row * ((K + 1) & ~1) + k0);
#pragma unroll
              for (int kk = 0; kk < RITZ_KC; kk += 2)
                if (k0 + kk < K) ur[kk >> 1] = make_double2(o[kk], o[kk + 1]);
            } else {
#pragma unroll
              for (int kk = 0; kk < RITZ_KC; ++kk)
                if (k0 + kk < K) U[(size_t)(k0 + kk) * a.n + row] = o[kk];
            }
          }
        }
      }

      if constexpr (HAS_DOT || DDOT) named_bar_sync(1, CONSUMERS);
    }  // tiles of the group
    if (nb > 0) {
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
  }

  if (a.fin == FIN_NONE) return;

  // ---- per-CTA partial sums ----
  if constexpr (HAS_DOT) {
    const int jend = (MODE == MODE_AXPY_DOT && P == PREC_FDF) ? nb - 1 : nb;
#pragma unroll
    for (int q = 0; q < QMAX; ++q) {
      const int jj = wid + (CONSUMERS / 32) * q;
      if (jj < jend) {
        acc_t v = dots[q];
        if constexpr (P == PREC_FDF) v = warp_sum(v);
        else v = warp_sum(v);
        if (lane == 0) put_partial<P>(a.partials, pidx(jj, cta, ncta), v);
      }
    }
  }
  if constexpr (DDOT) {
#pragma unroll
    for (int q = 0; q < QMAX; ++q) {
      const int jj = wid + (CONSUMERS / 32) * q;
      if (jj < nb - 1) {
        const acc_t v = warp_sum(dots[q]), v2 = warp_sum(dots2[q]);
        if (lane == 0) {
          put_partial<P>(a.partials, pidx(jj, cta, ncta), v);
          put_partial<P>(a.partials, pidx(SLOT_D2 + jj, cta, ncta), v2);
        }
      }
    }
  }
  if constexpr (MODE == MODE_AXPY_DOT && P == PREC_FDF) {
    n1 = warp_sum(n1);
    if (lane == 0) red[wid] = n1;
    named_bar_sync(1, CONSUMERS);
    if (tid == 0) {
      acc_t t1 = red[0];
      for (int w = 1; w < CONSUMERS / 32; ++w) t1 = acc_merge<P>(t1, red[w]);
      put_partial<P>(a.partials, pidx(nb - 1, cta, ncta), t1);
    }
  }
  if constexpr (MODE == MODE_AXPY_STORE || DUPD || DDOT) {
    if constexpr (P == PREC_DDD && !DDOT) n2 = n1;
    n1 = warp_sum(n1);
    n2 = warp_sum(n2);
    if (lane == 0) {
      red[2 * wid] = n1;
      red[2 * wid + 1] = n2;
    }
    named_bar_sync(1, CONSUMERS);
    if (tid == 0) {
      acc_t t1 = red[0], t2 = red[1];
      for (int w = 1; w < CONSUMERS / 32; ++w) {
        t1 = acc_merge<P>(t1, red[2 * w]);
        t2 = acc_merge<P>(t2, red[2 * w + 1]);
      }
      if constexpr (DDOT) {  // the candidate's dots, in its columns' slots
        put_partial<P>(a.partials, pidx(nb - 1, cta, ncta), t1);
        put_partial<P>(a.partials, pidx(SLOT_D2 + nb - 1, cta, ncta), t2);
      } else {
        put_partial<P>(a.partials, pidx(SLOT_N, cta, ncta), t1);
        put_partial<P>(a.partials, pidx(SLOT_N + 1, cta, ncta), t2);
      }
    }
  }

  // ---- the last CTA reduces every CTA's partials in a fixed order ----
  __threadfence();
  named_bar_sync(1, CONSUMERS);
  if (tid == 0) {
    unsigned int tk = atomicAdd(&st->ticket, 1u);
    *lastflag = (tk == (unsigned)ncta - 1) ? 1 : 0;
  }
  named_bar_sync(1, CONSUMERS);
  if (*lastflag == 0) return;
  __threadfence();
  const int slots = (MODE == MODE_AXPY_STORE || DUPD) ? 2 : (DDOT ? 2 * nb : nb);
  for (int q = wid; q < slots; q += CONSUMERS / 32) {
    const int slot = (MODE == MODE_AXPY_STORE || DUPD) ? SLOT_N + q
                     : (DDOT && q >= nb)               ? SLOT_D2 + (q - nb)
                                                       : q;
    acc_t acc = zero_acc<P>();
    // each lane adds the CTAs lane, lane + 32, ... in order; a chunk's loads
    // are all issued before its sums
    for (int b0 = 0; b0 < ncta; b0 += 32 * RED_LOADS) {
      typename Tr::part_t v[RED_LOADS];
#pragma unroll
      for (int u = 0; u < RED_LOADS; ++u) {
        const int b = b0 + lane + 32 * u;
        if (b < ncta) v[u] = load_partial<P>(a.partials, pidx(slot, b, ncta));
      }
#pragma unroll
      for (int u = 0; u < RED_LOADS; ++u)
        if (b0 + lane + 32 * u < ncta) add_partial<P>(acc, v[u]);
    }
    acc = warp_sum(acc);
    if (lane == 0) tot[q] = acc_to_double<P>(acc);
  }
  named_bar_sync(1, CONSUMERS);
  finalize_pass(a, tot, reinterpret_cast<double*>(sm + L.fin_off), tid);
  if (tid == 0) {
    st->ticket = 0;
    if (stall) st->stall_armed = 0;
  }
}

template <int P, int MODE>
__global__ void __launch_bounds__(PASS_THREADS, pass_ctas_per_sm(P)) pass_kernel(PassArgs a, size_t region) {
  pass_body<P, MODE>(a, region, (int)blockIdx.x, (int)gridDim.x);
}

// ---------------------------------------------------------------------------
// serving engine: one pass for every live solve.  Block b is CTA
// b - item_off[s] of solve s (each solve has a fixed number of CTAs that
// depends only on its size), so every solve's sums run in the same order
// whatever else shares the launch.  The arguments are those the single-solve
// plan uses at the solve's current step.
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(PASS_THREADS, pass_ctas_per_sm(PREC_FDF))
    batch_pass_kernel(const BatchTable* T, int restart, size_t region) {
  const int ns = T->nslots;
  const int item = (int)blockIdx.x;
  if (item >= T->item_off[ns]) return;
  int sidx = 0;
  while (T->item_off[sidx + 1] <= item) ++sidx;
  const BatchSlot& B = T->slot[sidx];
  const int i = B.step;
  if (restart && i + 1 >= B.m) return;  // no restart after the last step
  PassArgs a;
  memset(&a, 0, sizeof(a));
  a.V = B.V;
  a.Vmut = B.V;
  a.ld = B.n_pad;
  a.tstride = TILE_R;  // column-major
  a.cstride = B.n_pad;
  a.n = B.n;
  a.m = B.m;
  a.K = B.K;
  a.seed = B.seed;
  a.tol = B.tol;
  a.st = B.st;
  a.partials = B.partials;
  a.step = i;
  a.nb = i + 1;
  if (!restart) {
    a.xsrc = X_VEC;
    if (MODE == MODE_DOT) {
      a.xvec = B.ytil;
      a.fin = FIN_DOT_STEP;
    } else if (MODE == MODE_AXPY_DOT) {
      a.xvec = B.ytil;
      a.wout = B.w;
      a.fin = FIN_AXPYDOT_STEP;
      a.exact_tail = 2;
    } else {
      a.xvec = B.w;
      a.col_out = i + 1;
      a.fin = FIN_STORE_STEP;
      a.exact_tail = 0;
    }
  } else {
    a.only_on_restart = 1;
    a.exact_tail = i + 1;
    if (MODE == MODE_DOT) {
      a.xsrc = X_RANDOM;
      a.fin = FIN_DOT_RESTART;
    } else if (MODE == MODE_AXPY_DOT) {
      a.xsrc = X_RANDOM;
      a.wout = B.w;
      a.fin = FIN_AXPYDOT;
    } else {
      a.xsrc = X_VEC;
      a.xvec = B.w;
      a.col_out = i + 1;
      a.fin = FIN_STORE_RESTART;
    }
  }
  pass_body<PREC_FDF, MODE>(a, region, item - T->item_off[sidx], B.ncta);
}

cudaError_t batch_pass_prepare(const PassLaunch& L) {
  cudaError_t e = cudaFuncSetAttribute(batch_pass_kernel<MODE_DOT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(batch_pass_kernel<MODE_AXPY_DOT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(batch_pass_kernel<MODE_AXPY_STORE>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
  return e;
}

cudaError_t launch_batch_pass(int mode, const BatchTable* T, int restart, const PassLaunch& L,
                              cudaStream_t s) {
  const int grid = SRV_MAX_SLOTS * SRV_MAX_CTAS;
  if (mode == MODE_DOT)
    batch_pass_kernel<MODE_DOT><<<grid, PASS_THREADS, L.smem, s>>>(T, restart, L.region);
  else if (mode == MODE_AXPY_DOT)
    batch_pass_kernel<MODE_AXPY_DOT><<<grid, PASS_THREADS, L.smem, s>>>(T, restart, L.region);
  else if (mode == MODE_AXPY_STORE)
    batch_pass_kernel<MODE_AXPY_STORE><<<grid, PASS_THREADS, L.smem, s>>>(T, restart, L.region);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <int P, int MODE>
static cudaError_t config_t(int max_cols, int K, int num_sms, PassLaunch& out) {
  using basis_t = typename PassTr<P>::basis_t;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  const int ritz_elems = MODE == MODE_RITZ ? max_cols * ((K + RITZ_KC - 1) / RITZ_KC * RITZ_KC) : 0;
  // pass_ctas_per_sm CTAs per SM share the SM's shared memory (minus the
  // per-CTA reservation of 1 KB)
  const size_t fixed = smem_plan(MODE, 0, ritz_elems).total + 128;
  int persm = 0;
  e = cudaDeviceGetAttribute(&persm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e != cudaSuccess) return e;
  const size_t half = (size_t)persm / pass_ctas_per_sm(P) - 1024;
  const size_t cap = half < (size_t)optin ? half : (size_t)optin;
  size_t avail = cap > fixed ? cap - fixed : 0;
  // a stage: max_cols basis columns of a tile, plus the pass vector's rows
  const size_t per_stage = (size_t)(max_cols > 0 ? max_cols : 1) * TILE_R * sizeof(basis_t) +
                           (MODE == MODE_RITZ ? 0 : (size_t)TILE_R * 8);
  // every byte that fits: the kernel fits region / (its stage) stages, so
  // that passes over few columns keep many tiles in flight
  const size_t region = avail / 128 * 128;
  const int stages = (int)(region / per_stage);
  if (stages < 1) return cudaErrorInvalidConfiguration;
  const size_t total = smem_plan(MODE, region, ritz_elems).total;
  e = cudaFuncSetAttribute(pass_kernel<P, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)total);
  if (e != cudaSuccess) return e;
  out.grid = num_sms * pass_ctas_per_sm(P);
  out.smem = total;
  out.stages = stages;
  out.region = region;
  return cudaSuccess;
}

cudaError_t pass_config(int prec, int mode, int max_cols, int K, int num_sms, PassLaunch& out) {
#define TE_CFG(PP, MM) \
  if (prec == PP && mode == MM) return config_t<PP, MM>(max_cols, K, num_sms, out);
  TE_CFG(PREC_DDD, MODE_DOT)
  TE_CFG(PREC_DDD, MODE_AXPY_DOT)
  TE_CFG(PREC_DDD, MODE_AXPY_STORE)
  TE_CFG(PREC_DDD, MODE_RITZ)
  TE_CFG(PREC_DDD, MODE_DCGS_DOT)
  TE_CFG(PREC_DDD, MODE_DCGS_UPDATE)
  TE_CFG(PREC_FDF, MODE_DCGS_DOT)
  TE_CFG(PREC_FDF, MODE_DCGS_UPDATE)
  TE_CFG(PREC_FDF, MODE_DOT)
  TE_CFG(PREC_FDF, MODE_AXPY_DOT)
  TE_CFG(PREC_FDF, MODE_AXPY_STORE)
  TE_CFG(PREC_FDF, MODE_RITZ)
#undef TE_CFG
  return cudaErrorInvalidValue;
}

cudaError_t launch_pass(int prec, int mode, const PassArgs& a, const PassLaunch& L,
                        cudaStream_t s) {
#define TE_LAUNCH(PP, MM)                                                        \
  if (prec == PP && mode == MM) {                                                \
    pass_kernel<PP, MM><<<L.grid, PASS_THREADS, L.smem, s>>>(a, L.region);       \
    return cudaGetLastError();                                                   \
  }
  TE_LAUNCH(PREC_DDD, MODE_DOT)
  TE_LAUNCH(PREC_DDD, MODE_AXPY_DOT)
  TE_LAUNCH(PREC_DDD, MODE_AXPY_STORE)
  TE_LAUNCH(PREC_DDD, MODE_RITZ)
  TE_LAUNCH(PREC_DDD, MODE_DCGS_DOT)
  TE_LAUNCH(PREC_DDD, MODE_DCGS_UPDATE)
  TE_LAUNCH(PREC_FDF, MODE_DCGS_DOT)
  TE_LAUNCH(PREC_FDF, MODE_DCGS_UPDATE)
  TE_LAUNCH(PREC_FDF, MODE_DOT)
  TE_LAUNCH(PREC_FDF, MODE_AXPY_DOT)
  TE_LAUNCH(PREC_FDF, MODE_AXPY_STORE)
  TE_LAUNCH(PREC_FDF, MODE_RITZ)
#undef TE_LAUNCH
  return cudaErrorInvalidValue;
}

// out[j*n + v] = s_j * V(r, j) with r = iperm[v] (iperm NULL: r = v), V(r, j)
// at (r / TILE_R) * tstride + j * cstride + r % TILE_R
template <typename B>
__global__ void basis_to_f64_kernel(const B* V, int64_t tstride, int64_t cstride, int64_t n,
                                    int cols, const double* s, const int32_t* iperm,
                                    double* out) {
  const int64_t total = n * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / n, v = e - j * n;
    const int64_t r = iperm ? (int64_t)iperm[v] : v;
    out[e] = s[j] * (double)V[(r / TILE_R) * tstride + j * cstride + r % TILE_R];
  }
}

cudaError_t launch_basis_to_f64(int prec, const void* V, int64_t tstride, int64_t cstride,
                                int64_t n, int cols, const double* s_dev, const int32_t* iperm,
                                double* out, cudaStream_t st) {
  const int64_t total = n * cols;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  if (blocks < 1) blocks = 1;
  if (prec == PREC_DDD)
    basis_to_f64_kernel<double><<<(int)blocks, 256, 0, st>>>(
        static_cast<const double*>(V), tstride, cstride, n, cols, s_dev, iperm, out);
  else
    basis_to_f64_kernel<float><<<(int)blocks, 256, 0, st>>>(
        static_cast<const float*>(V), tstride, cstride, n, cols, s_dev, iperm, out);
  return cudaGetLastError();
}

}  // namespace te
