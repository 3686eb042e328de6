/*
 * oracle.c - plain FP64 CPU oracle of the Top-K sparse eigensolver.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this code.  It shares nothing with
 * the CUDA path (no headers, helpers or tables) and is deliberately simple:
 * every routine follows the paper's description step by step, in binary64.
 *
 * Paper: Sgherzi, Parravicini, Santambrogio, "A Mixed Precision, Multi-GPU
 * Design for Large-scale Top-K Sparse Eigenproblems" (arXiv 2201.07498).
 *   - oracle_spmv:        Algorithm 1, the SpMV step (v_t <- M v_i).
 *   - oracle_lanczos:     Algorithm 1 (Lanczos with MGS reorthogonalisation),
 *                         Section III.
 *   - oracle_jacobi:      the Jacobi phase on T (Section III, Fig. 1; cyclic
 *                         Jacobi after Rutishauser 1966).
 *   - oracle_select_topk: "largest in modulo" (Section I).
 *   - oracle_ritz:        eigenvectors of M as (Lanczos basis) x (eigenvectors
 *                         of T) (Section III).
 *   - oracle_lanczos_ex:  the same Lanczos with reorthogonalisation switched
 *                         off (the comparison of Section IV-D).
 *   - oracle_refine:      Rayleigh quotient u'Mu/u'u and residual of given
 *                         vectors (definition).
 *   - oracle_mean_pairwise_angle: the orthogonality metric of Section IV-D.
 *   - oracle_round_bf16, oracle_quantize_e4m3_rows: the reduced-precision
 *                         matrix values of the mixed forms (Section III-A).
 *
 * Readings where the paper is silent or garbled (listed with reasons in the
 * design notes of the repository):
 *   R1  the loop runs m = krylov_steps >= K times; the top K of the m Ritz
 *       pairs are returned.
 *   R2  "v_tmp" in the three-term update is the SpMV output v_t.
 *   R3  the odd/even ping-pong reorthogonalisation is one modified
 *       Gram-Schmidt pass of v_nxt against v_1..v_i, in order.
 *   R4  beta_1 = 0; T = tridiag(alpha_1..alpha_m; beta_2..beta_m); beta_{m+1}
 *       is kept for residual estimates.
 *   R5  "largest in modulo" = largest |theta|; ties: positive first, then
 *       lower index.  LARGEST_ALGEBRAIC is an option.
 *   R7  breakdown: if beta_{i+1} <= tol * anorm (anorm = max_j |alpha_j| +
 *       beta_j + beta_{j+1} so far) and i < m, restart from a fresh seeded
 *       vector (SplitMix64, stream 1 + restart count), orthogonalised twice by
 *       MGS against the basis, and set beta_{i+1} = 0.
 *   R8  Jacobi: cyclic-by-row; a pair is rotated when |t_pq| > 1e-16 ||T||_F;
 *       stop after a sweep with no rotation (at most max_sweeps sweeps).
 *   R9  eigenvector sign: the entry of largest magnitude of T's eigenvector y
 *       (lowest index on ties) is made positive; u = V y is not renormalised.
 *
 * Sums over n (dot products, norms) are taken in fixed blocks of 2^16
 * elements, blocks summed in order, so results do not depend on the number of
 * OpenMP threads.  Each SpMV row is summed left to right.
 *
 * A test-only switch (oracle_set_fault) plants one known mistake at a time so
 * that the test-suite can show its pins catch it.  It is off by default.
 */
#include "oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int g_fault = 0;
void oracle_set_fault(int kind) { g_fault = kind; }
int oracle_get_fault(void) { return g_fault; }

/* ---------------- SplitMix64 (Steele, Lea & Flood 2014) ---------------- */
static uint64_t om_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static double om_uniform_pm1(uint64_t seed, uint64_t stream, uint64_t i) {
  uint64_t s0 = seed ^ (stream * 0xD1B54A32D192ED03ULL);
  uint64_t x = om_mix64(s0 + (i + 1) * 0x9E3779B97F4A7C15ULL);
  return 2.0 * ((double)(x >> 11) * 0x1.0p-53) - 1.0;
}

/* ---------------- level-1 kernels in binary64 ---------------- */
#define OM_BLOCK 65536

static double om_dot(int64_t n, const double* x, const double* y) {
  int64_t nb = (n + OM_BLOCK - 1) / OM_BLOCK;
  double* part = (double*)malloc(sizeof(double) * (size_t)(nb > 0 ? nb : 1));
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < nb; ++b) {
    int64_t s = b * OM_BLOCK, e = s + OM_BLOCK < n ? s + OM_BLOCK : n;
    double acc = 0.0;
    for (int64_t k = s; k < e; ++k) acc += x[k] * y[k];
    part[b] = acc;
  }
  double tot = 0.0;
  for (int64_t b = 0; b < nb; ++b) tot += part[b];
  free(part);
  return tot;
}

static double om_norm(int64_t n, const double* x) { return sqrt(om_dot(n, x, x)); }

/* y <- y + a x */
static void om_axpy(int64_t n, double a, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < n; ++k) y[k] += a * x[k];
}

/* ---------------- SpMV (Algorithm 1, v_t <- M v_i) ---------------- */
double oracle_spmv_row(const int64_t* rp, const int32_t* ci, const double* val,
                       const double* x, int64_t r) {
  double acc = 0.0;
  for (int64_t k = rp[r]; k < rp[r + 1]; ++k) acc += val[k] * x[ci[k]];
  return acc;
}

void oracle_spmv(int64_t n, const int64_t* rp, const int32_t* ci, const double* val,
                 const double* x, double* y) {
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t r = 0; r < n; ++r) {
    if (g_fault == ORACLE_FAULT_SPMV_SKIP_LAST) {
      double acc = 0.0;
      for (int64_t k = rp[r]; k + 1 < rp[r + 1]; ++k) acc += val[k] * x[ci[k]];
      y[r] = acc;
    } else {
      y[r] = oracle_spmv_row(rp, ci, val, x, r);
    }
  }
}

/* ---------------- Lanczos with MGS reorthogonalisation ---------------- */
/* MGS pass of w against columns 0..cols-1 of V (Algorithm 1's reorthogonalisation) */
static void om_mgs(int64_t n, int32_t cols, const double* V, double* w) {
  for (int32_t j = 0; j < cols; ++j) {
    const double* vj = V + (size_t)j * (size_t)n;
    double o = om_dot(n, vj, w);
    om_axpy(n, -o, vj, w);
  }
}

int oracle_lanczos(int64_t n, const int64_t* rp, const int32_t* ci, const double* val,
                   const double* v1_raw, int32_t m, uint64_t seed, double tol,
                   double* alpha, double* beta, double* V, double* w_out,
                   int32_t* restarts_out) {
  return oracle_lanczos_ex(n, rp, ci, val, v1_raw, m, seed, tol, 1, alpha, beta, V, w_out,
                           restarts_out);
}

int oracle_lanczos_ex(int64_t n, const int64_t* rp, const int32_t* ci, const double* val,
                      const double* v1_raw, int32_t m, uint64_t seed, double tol, int32_t reorth,
                      double* alpha, double* beta, double* V, double* w_out,
                      int32_t* restarts_out) {
  if (n < 1 || m < 1 || m > n || !rp || !ci || !val || !v1_raw || !alpha || !beta || !V)
    return -1;
  double* vt = (double*)malloc(sizeof(double) * (size_t)n);
  double* w = (double*)malloc(sizeof(double) * (size_t)n);
  if (!vt || !w) { free(vt); free(w); return -2; }
  int32_t restarts = 0;

  /* v_1: the L2-normalised random input vector (Section III) */
  double nv = om_norm(n, v1_raw);
  if (!(nv > 0.0)) { free(vt); free(w); return -3; }
  for (int64_t k = 0; k < n; ++k)
    V[k] = (g_fault == ORACLE_FAULT_NO_V1_NORMALISE) ? v1_raw[k] : v1_raw[k] / nv;
  beta[0] = 0.0; /* beta_1 */
  double anorm = 0.0;

  for (int32_t i = 0; i < m; ++i) {
    const double* vi = V + (size_t)i * (size_t)n;
    const double* vim1 = i > 0 ? V + (size_t)(i - 1) * (size_t)n : NULL;
    /* SpMV step: v_t <- M v_i */
    oracle_spmv(n, rp, ci, val, vi, vt);
    /* alpha_i <- v_i . v_t */
    alpha[i] = om_dot(n, vi, vt);
    /* three-term update: v_nxt <- v_t - alpha_i v_i - beta_i v_{i-1} */
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) {
      double x = vt[k] - alpha[i] * vi[k];
      if (vim1) x -= beta[i] * vim1[k];
      w[k] = x;
    }
    if (g_fault == ORACLE_FAULT_ALPHA_SIGN) alpha[i] = -alpha[i];
    /* reorthogonalise v_nxt against v_1..v_i (one MGS pass) */
    if ((reorth || g_fault == ORACLE_FAULT_REORTH_IGNORED) && g_fault != ORACLE_FAULT_NO_REORTH)
      om_mgs(n, i + 1, V, w);
    /* start of the next iteration: beta_{i+1} <- ||v_nxt|| */
    double b = om_norm(n, w);
    double cand = fabs(alpha[i]) + beta[i] + b;
    if (cand > anorm) anorm = cand;
    beta[i + 1] = b;
    if (i + 1 < m) {
      double* vnext = V + (size_t)(i + 1) * (size_t)n;
      if (b <= tol * anorm) {
        /* R7: invariant subspace found; restart from a fresh seeded vector */
        restarts += 1;
        for (int64_t k = 0; k < n; ++k)
          w[k] = om_uniform_pm1(seed, (uint64_t)restarts, (uint64_t)k);
        om_mgs(n, i + 1, V, w);
        om_mgs(n, i + 1, V, w);
        double br = om_norm(n, w);
        if (!(br > 0.0)) { free(vt); free(w); return -4; }
        for (int64_t k = 0; k < n; ++k) vnext[k] = w[k] / br;
        beta[i + 1] = 0.0;
      } else {
        /* v_{i+1} <- v_nxt / beta_{i+1} */
        for (int64_t k = 0; k < n; ++k) vnext[k] = w[k] / b;
      }
    } else if (w_out) {
      memcpy(w_out, w, sizeof(double) * (size_t)n);
    }
  }
  if (restarts_out) *restarts_out = restarts;
  free(vt);
  free(w);
  return 0;
}

/* ---------------- cyclic Jacobi on a dense symmetric matrix ---------------- */
int oracle_jacobi(int32_t m, double* T, double* Y, double tol, int32_t max_sweeps,
                  int32_t* sweeps_out) {
  if (m < 1 || !T || !Y) return -1;
  for (int32_t r = 0; r < m; ++r)
    for (int32_t c = 0; c < m; ++c) Y[(size_t)r * m + c] = (r == c) ? 1.0 : 0.0;
  double fro = 0.0;
  for (size_t k = 0; k < (size_t)m * m; ++k) fro += T[k] * T[k];
  fro = sqrt(fro);
  const double thr = tol * fro;
  int32_t sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    int rotated = 0;
    for (int32_t p = 0; p < m - 1; ++p) {
      for (int32_t q = p + 1; q < m; ++q) {
        double tpq = T[(size_t)p * m + q];
        if (!(fabs(tpq) > thr)) continue;
        rotated = 1;
        double tpp = T[(size_t)p * m + p], tqq = T[(size_t)q * m + q];
        /* rotation annihilating t_pq: zeta = (t_qq - t_pp) / (2 t_pq),
           t = sgn(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1+t^2), s = t c */
        double zeta = (tqq - tpp) / (2.0 * tpq);
        double t;
        if (fabs(zeta) > 1e150) t = 0.5 / zeta;
        else t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double c = 1.0 / sqrt(1.0 + t * t);
        double s = t * c;
        if (g_fault == ORACLE_FAULT_JACOBI_SIGN) s = -s;
        T[(size_t)p * m + p] = tpp - t * tpq;
        T[(size_t)q * m + q] = tqq + t * tpq;
        T[(size_t)p * m + q] = 0.0;
        T[(size_t)q * m + p] = 0.0;
        for (int32_t r = 0; r < m; ++r) {
          if (r == p || r == q) continue;
          double g = T[(size_t)r * m + p], h = T[(size_t)r * m + q];
          double gp = c * g - s * h, hq = s * g + c * h;
          T[(size_t)r * m + p] = gp; T[(size_t)p * m + r] = gp;
          T[(size_t)r * m + q] = hq; T[(size_t)q * m + r] = hq;
        }
        for (int32_t r = 0; r < m; ++r) {
          double g = Y[(size_t)r * m + p], h = Y[(size_t)r * m + q];
          Y[(size_t)r * m + p] = c * g - s * h;
          Y[(size_t)r * m + q] = s * g + c * h;
        }
      }
    }
    if (!rotated) break;
  }
  if (sweeps_out) *sweeps_out = sweep;
  return sweep < max_sweeps ? 0 : 1;
}

/* ---------------- top-K selection (Section I: largest in modulo) ---------------- */
static int om_before(double a, int32_t ia, double b, int32_t ib, int32_t which) {
  if (which == ORACLE_LARGEST_ALGEBRAIC) {
    if (a != b) return a > b;
    return ia < ib;
  }
  double fa = fabs(a), fb = fabs(b);
  if (fa != fb) return fa > fb;
  if ((a > 0) != (b > 0)) return a > 0;
  return ia < ib;
}

void oracle_select_topk(int32_t m, const double* theta, int32_t K, int32_t which,
                        int32_t* idx) {
  int32_t* ord = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
  for (int32_t j = 0; j < m; ++j) ord[j] = j;
  int32_t w = (g_fault == ORACLE_FAULT_SELECT_ALGEBRAIC) ? ORACLE_LARGEST_ALGEBRAIC : which;
  /* insertion sort by the selection key (m is small) */
  for (int32_t a = 1; a < m; ++a) {
    int32_t x = ord[a], b = a - 1;
    while (b >= 0 && om_before(theta[x], x, theta[ord[b]], ord[b], w)) {
      ord[b + 1] = ord[b];
      --b;
    }
    ord[b + 1] = x;
  }
  for (int32_t k = 0; k < K; ++k) idx[k] = ord[k];
  free(ord);
}

/* ---------------- Ritz vectors (Section III: eigenvectors = V * Y) ---------------- */
void oracle_ritz(int64_t n, int32_t m, const double* V, const double* Y, int32_t K,
                 const int32_t* idx, double* U) {
  for (int32_t k = 0; k < K; ++k) {
    int32_t c = idx[k];
    /* R9: the largest-magnitude entry of y (lowest index on ties) is positive */
    int32_t jmax = 0;
    for (int32_t j = 1; j < m; ++j)
      if (fabs(Y[(size_t)j * m + c]) > fabs(Y[(size_t)jmax * m + c])) jmax = j;
    double sgn = Y[(size_t)jmax * m + c] < 0.0 ? -1.0 : 1.0;
    double* u = U + (size_t)k * (size_t)n;
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n; ++r) {
      double acc = 0.0;
      for (int32_t j = 0; j < m; ++j) {
        double yj = (g_fault == ORACLE_FAULT_RITZ_TRANSPOSE) ? Y[(size_t)c * m + j]
                                                             : Y[(size_t)j * m + c];
        acc += V[(size_t)j * (size_t)n + r] * yj;
      }
      u[r] = sgn * acc;
    }
  }
}

/* ---------------- Rayleigh quotient, residual, pairwise angles ---------------- */
void oracle_refine(int64_t n, const int64_t* rp, const int32_t* ci, const double* val,
                   int32_t K, const double* U, double* theta_out, double* resid_out) {
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  for (int32_t k = 0; k < K; ++k) {
    const double* u = U + (size_t)k * (size_t)n;
    oracle_spmv(n, rp, ci, val, u, y);
    const double uu = om_dot(n, u, u);
    const double th = om_dot(n, u, y) / (g_fault == ORACLE_FAULT_REFINE_NO_NORM ? 1.0 : uu);
    theta_out[k] = th;
    if (resid_out) {
      for (int64_t i = 0; i < n; ++i) r[i] = y[i] - th * u[i];
      resid_out[k] = om_norm(n, r) / sqrt(uu);
    }
  }
  free(y);
  free(r);
}

double oracle_mean_pairwise_angle(int64_t n, int32_t K, const double* U) {
  if (K < 2) return 0.0;
  const double pi = acos(-1.0);
  double sum = 0.0;
  int64_t pairs = 0;
  for (int32_t a = 0; a < K; ++a) {
    const double* ua = U + (size_t)a * (size_t)n;
    for (int32_t b = a + 1; b < K; ++b) {
      const double* ub = U + (size_t)b * (size_t)n;
      double d = om_dot(n, ua, ub);
      if (g_fault != ORACLE_FAULT_ANGLE_SIGNED) d = fabs(d);
      double c = d / (om_norm(n, ua) * om_norm(n, ub));
      if (c > 1.0) c = 1.0;
      sum += acos(c) * 180.0 / pi;
      pairs += 1;
    }
  }
  return sum / (double)pairs;
}

/* ---------------- rounding to the storage types ---------------- */
/* Round |x| > 0 to p significant bits, with the quantum never below 2^qmin
   (gradual underflow): x = f * 2^e with f in [0.5, 1); the quantum is
   2^(e - p), clamped; keep floor(|x| / quantum) and round up when the rest
   exceeds a half, or equals a half and the kept integer is odd. */
static double om_round_sig(double ax, int p, int qmin) {
  int e;
  (void)frexp(ax, &e);
  int qe = e - p;
  if (qe < qmin) qe = qmin;
  const double quantum = ldexp(1.0, qe);
  const double t = ax / quantum; /* exact: a power-of-two scaling */
  double f = floor(t);
  const double rest = t - f;     /* exact */
  const int up_on_tie = g_fault == ORACLE_FAULT_TIES_AWAY ? 1 : (fmod(f, 2.0) != 0.0);
  if (rest > 0.5 || (rest == 0.5 && up_on_tie)) f += 1.0;
  return f * quantum;
}

void oracle_round_bf16(int64_t count, const double* x, uint16_t* codes, double* deq) {
  for (int64_t i = 0; i < count; ++i) {
    const double ax = fabs(x[i]);
    double r = ax > 0.0 ? om_round_sig(ax, 8, -133) : 0.0;
    if (r != 0.0 && x[i] < 0.0) r = -r;
    float f = (float)r; /* exact: r has at most 8 significant bits */
    uint32_t bits;
    memcpy(&bits, &f, 4);
    if (r == 0.0) bits = 0;
    if (codes) codes[i] = (uint16_t)(bits >> 16);
    if (deq) deq[i] = r;
  }
}

double oracle_e4m3_value(uint8_t code) {
  const int e = (code >> 3) & 15, m = code & 7;
  double v = e == 0 ? ldexp((double)m, -9) : ldexp(1.0 + m / 8.0, e - 7);
  return (code & 0x80) ? -v : v;
}

static uint8_t om_e4m3_code(double x) {
  const double ax = fabs(x);
  double r = ax > 0.0 ? om_round_sig(ax, 4, -9) : 0.0;
  if (r > 448.0) r = 448.0;
  if (r == 0.0) return 0;
  int e;
  double f = frexp(r, &e); /* r = f 2^e, f in [0.5, 1) */
  uint8_t code;
  if (e - 1 < -6) {
    code = (uint8_t)(r / ldexp(1.0, -9)); /* subnormal: m * 2^-9 */
  } else {
    const int m = (int)(f * 16.0) - 8; /* 1.mmm = 2f */
    code = (uint8_t)(((e - 1 + 7) << 3) | m);
  }
  return (uint8_t)(x < 0.0 ? (code | 0x80) : code);
}

void oracle_quantize_e4m3_rows(int64_t n, const int64_t* rp, const double* val,
                               uint8_t* codes, float* scale, double* deq) {
  for (int64_t r = 0; r < n; ++r) {
    double mx = 0.0;
    for (int64_t k = rp[r]; k < rp[r + 1]; ++k)
      if (fabs(val[k]) > mx) mx = fabs(val[k]);
    const float s = mx > 0.0 ? (float)(mx / 448.0) : 1.0f;
    if (scale) scale[r] = s;
    for (int64_t k = rp[r]; k < rp[r + 1]; ++k) {
      const uint8_t c = om_e4m3_code(val[k] / (double)s);
      if (codes) codes[k] = c;
      if (deq) deq[k] = (double)s * oracle_e4m3_value(c);
    }
  }
}

/* ---------------- the whole pipeline ---------------- */
int oracle_topk_eigs(int64_t n, const int64_t* rp, const int32_t* ci, const double* val,
                     const double* v1_raw, int32_t K, int32_t m, int32_t which, uint64_t seed,
                     double* eigvals, double* U, double* residuals, double* alpha_out,
                     double* beta_out, int32_t* info) {
  return oracle_topk_eigs_ex(n, rp, ci, val, v1_raw, K, m, which, seed, 1, eigvals, U,
                             residuals, alpha_out, beta_out, info);
}

int oracle_topk_eigs_ex(int64_t n, const int64_t* rp, const int32_t* ci, const double* val,
                        const double* v1_raw, int32_t K, int32_t m, int32_t which,
                        uint64_t seed, int32_t reorth, double* eigvals, double* U,
                        double* residuals, double* alpha_out, double* beta_out, int32_t* info) {
  if (K < 1 || m < K || m > n || !eigvals) return -1;
  double* V = (double*)malloc(sizeof(double) * (size_t)n * (size_t)m);
  double* alpha = (double*)malloc(sizeof(double) * (size_t)m);
  double* beta = (double*)malloc(sizeof(double) * (size_t)(m + 1));
  double* T = (double*)calloc((size_t)m * m, sizeof(double));
  double* Y = (double*)malloc(sizeof(double) * (size_t)m * m);
  int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)K);
  int rc = -2;
  if (!V || !alpha || !beta || !T || !Y || !idx) goto done;
  int32_t restarts = 0, sweeps = 0;
  rc = oracle_lanczos_ex(n, rp, ci, val, v1_raw, m, seed, ORACLE_BREAKDOWN_TOL, reorth, alpha,
                         beta, V, NULL, &restarts);
  if (rc != 0) goto done;
  for (int32_t i = 0; i < m; ++i) {
    T[(size_t)i * m + i] = alpha[i];
    if (i + 1 < m) {
      double b = (g_fault == ORACLE_FAULT_BETA_INDEX) ? beta[i] : beta[i + 1];
      T[(size_t)i * m + i + 1] = b;
      T[(size_t)(i + 1) * m + i] = b;
    }
  }
  int jrc = oracle_jacobi(m, T, Y, ORACLE_JACOBI_TOL, ORACLE_JACOBI_MAX_SWEEPS, &sweeps);
  double* theta = (double*)malloc(sizeof(double) * (size_t)m);
  for (int32_t j = 0; j < m; ++j) theta[j] = T[(size_t)j * m + j];
  oracle_select_topk(m, theta, K, which, idx);
  for (int32_t k = 0; k < K; ++k) eigvals[k] = theta[idx[k]];
  free(theta);
  if (U || residuals) {
    double* UU = U ? U : (double*)malloc(sizeof(double) * (size_t)n * (size_t)K);
    oracle_ritz(n, m, V, Y, K, idx, UU);
    if (residuals) {
      double* r = (double*)malloc(sizeof(double) * (size_t)n);
      for (int32_t k = 0; k < K; ++k) {
        const double* u = UU + (size_t)k * (size_t)n;
        oracle_spmv(n, rp, ci, val, u, r);
        om_axpy(n, -eigvals[k], u, r);
        residuals[k] = om_norm(n, r);
      }
      free(r);
    }
    if (!U) free(UU);
  }
  if (alpha_out) memcpy(alpha_out, alpha, sizeof(double) * (size_t)m);
  if (beta_out) memcpy(beta_out, beta, sizeof(double) * (size_t)(m + 1));
  if (info) { info[0] = restarts; info[1] = sweeps; info[2] = jrc; }
  rc = jrc == 0 ? 0 : 1;
done:
  free(V); free(alpha); free(beta); free(T); free(Y); free(idx);
  return rc;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* thread count of the OpenMP regions that follow (timing only: results do
   not depend on it) */
void oracle_set_num_threads(int threads) {
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
}
