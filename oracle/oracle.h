/*
 * oracle.h - declarations of the plain FP64 CPU oracle (test infrastructure
 * only; see oracle.c).  This header belongs to the oracle alone: the CUDA
 * path never includes it.
 *
 * Layouts: CSR with int64 row pointers (n+1), int32 columns, float64 values;
 * the Lanczos basis V and the Ritz vectors U are column-major (n rows, one
 * column per vector); the small matrices T and Y are dense row-major m x m.
 */
#ifndef ORACLE_H
#define ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_LARGEST_MAGNITUDE 0
#define ORACLE_LARGEST_ALGEBRAIC 1

#define ORACLE_BREAKDOWN_TOL 1e-12
#define ORACLE_JACOBI_TOL 1e-16
#define ORACLE_JACOBI_MAX_SWEEPS 100

/* planted mistakes, for the test that shows the pins catch them */
#define ORACLE_FAULT_NONE 0
#define ORACLE_FAULT_BETA_INDEX 1
#define ORACLE_FAULT_ALPHA_SIGN 2
#define ORACLE_FAULT_NO_REORTH 3
#define ORACLE_FAULT_JACOBI_SIGN 4
#define ORACLE_FAULT_RITZ_TRANSPOSE 5
#define ORACLE_FAULT_SELECT_ALGEBRAIC 6
#define ORACLE_FAULT_SPMV_SKIP_LAST 7
#define ORACLE_FAULT_NO_V1_NORMALISE 8
#define ORACLE_FAULT_REFINE_NO_NORM 9     /* Rayleigh quotient without the 1/u'u */
#define ORACLE_FAULT_ANGLE_SIGNED 10      /* angle metric without the absolute value */
#define ORACLE_FAULT_REORTH_IGNORED 11    /* reorth = 0 still reorthogonalises */
#define ORACLE_FAULT_TIES_AWAY 12         /* rounding ties away from zero, not to even */

void oracle_set_fault(int kind);
int oracle_get_fault(void);
int oracle_num_threads(void);
void oracle_set_num_threads(int threads); /* timing only; results do not depend on it */

/* Algorithm 1, SpMV step: y = M x (each row summed left to right) */
void oracle_spmv(int64_t n, const int64_t* rp, const int32_t* ci, const double* val,
                 const double* x, double* y);
double oracle_spmv_row(const int64_t* rp, const int32_t* ci, const double* val,
                       const double* x, int64_t r);

/* Algorithm 1: m Lanczos steps with one MGS reorthogonalisation pass each.
   alpha[m], beta[m+1] (beta[0] = beta_1 = 0, beta[i] = beta_{i+1}),
   V n x m column-major; w_out (optional, n) receives the last unnormalised
   v_nxt, whose norm is beta[m].  Returns 0 on success. */
int oracle_lanczos(int64_t n, const int64_t* rp, const int32_t* ci, const double* val,
                   const double* v1_raw, int32_t m, uint64_t seed, double tol,
                   double* alpha, double* beta, double* V, double* w_out,
                   int32_t* restarts_out);

/* Lanczos with a choice of reorthogonalisation: reorth = 1 is oracle_lanczos;
   reorth = 0 keeps only Algorithm 1's SpMV, alpha and three-term update:
   the variant without reorthogonalisation of Section IV-D. */
int oracle_lanczos_ex(int64_t n, const int64_t* rp, const int32_t* ci, const double* val,
                      const double* v1_raw, int32_t m, uint64_t seed, double tol, int32_t reorth,
                      double* alpha, double* beta, double* V, double* w_out,
                      int32_t* restarts_out);

/* Rayleigh quotient and residual of K given vectors (U n x K column-major):
   theta_out[k] = u_k' M u_k / u_k' u_k and resid_out[k] = ||M u_k -
   theta_out[k] u_k|| / ||u_k||, both in binary64 (definition; the
   refinement step of the mixed-precision forms).  resid_out may be NULL. */
void oracle_refine(int64_t n, const int64_t* rp, const int32_t* ci, const double* val,
                   int32_t K, const double* U, double* theta_out, double* resid_out);

/* Mean over the pairs a < b of the angle (degrees) between u_a and u_b,
   taken sign-free: acos(|u_a . u_b| / (||u_a|| ||u_b||)) (the orthogonality
   metric of Section IV-D; 90 for an orthogonal set).  K >= 2. */
double oracle_mean_pairwise_angle(int64_t n, int32_t K, const double* U);

/* Rounding of matrix values to the storage types of the mixed forms
   (Section III-A; readings: round to nearest, ties to even, from the
   binary64 value directly; a zero result is +0).
   oracle_round_bf16: bfloat16 (8 significant bits, binary32 exponent range);
     codes[i] = the 16-bit pattern, deq[i] = its value.
   oracle_quantize_e4m3_rows: FP8 E4M3 (4 significant bits, bias 7, largest
     finite 448, no infinities) with one binary32 scale per row,
     scale_r = (binary32) (max_j |a_rj| / 448) (1 for an all-zero row);
     code = round(a / scale_r), saturated to +-448; deq = scale_r * code.
   Values are finite with |a| < 2^127. */
void oracle_round_bf16(int64_t count, const double* x, uint16_t* codes, double* deq);
void oracle_quantize_e4m3_rows(int64_t n, const int64_t* rp, const double* val,
                               uint8_t* codes, float* scale, double* deq);
double oracle_e4m3_value(uint8_t code);

/* cyclic-by-row Jacobi: T (m x m, symmetric, row-major) is diagonalised in
   place, Y receives the eigenvectors (columns).  Returns 0 if converged. */
int oracle_jacobi(int32_t m, double* T, double* Y, double tol, int32_t max_sweeps,
                  int32_t* sweeps_out);

void oracle_select_topk(int32_t m, const double* theta, int32_t K, int32_t which,
                        int32_t* idx);

/* U[:,k] = sign_k * V Y[:, idx[k]] (U n x K column-major) */
void oracle_ritz(int64_t n, int32_t m, const double* V, const double* Y, int32_t K,
                 const int32_t* idx, double* U);

/* whole solve; info[0] = restarts, info[1] = Jacobi sweeps, info[2] = Jacobi rc.
   U, residuals, alpha_out, beta_out and info may be NULL. */
int oracle_topk_eigs(int64_t n, const int64_t* rp, const int32_t* ci, const double* val,
                     const double* v1_raw, int32_t K, int32_t m, int32_t which, uint64_t seed,
                     double* eigvals, double* U, double* residuals, double* alpha_out,
                     double* beta_out, int32_t* info);
/* the same with the reorthogonalisation choice of oracle_lanczos_ex */
int oracle_topk_eigs_ex(int64_t n, const int64_t* rp, const int32_t* ci, const double* val,
                        const double* v1_raw, int32_t K, int32_t m, int32_t which,
                        uint64_t seed, int32_t reorth, double* eigvals, double* U,
                        double* residuals, double* alpha_out, double* beta_out, int32_t* info);

#ifdef __cplusplus
}
#endif
#endif
