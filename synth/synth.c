/*
 * synth.c - seeded synthetic inputs for the Top-K sparse eigensolver.
 *
 * This module only MAKES inputs: symmetric sparse matrices in CSR form and
 * raw random vectors.  It holds none of the eigensolver's arithmetic (no
 * normalisation of start vectors, no products, no reductions of the method);
 * both the CUDA path and the CPU oracle consume what it produces.
 *
 * Random numbers come from one counter-based generator, SplitMix64
 * (G. L. Steele, D. Lea, C. H. Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the i-th output (0-based) of a generator whose
 * state starts at s0 is mix64(s0 + (i+1)*GAMMA), where mix64 is the
 * published 64-bit finaliser and GAMMA = 0x9E3779B97F4A7C15.  A (seed,
 * stream) pair selects s0 = seed XOR (stream * 0xD1B54A32D192ED03).
 * Everything below is a pure function of (seed, stream, index), so results
 * do not depend on the thread count or on the machine.
 *
 * Stream numbers used here: 0 start vectors; 101/102 uniform-matrix columns /
 * values; 110 R-MAT quadrant draws; 111 R-MAT vertex permutation; 112 the
 * vertex permutation of the planted communities.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SYNTH_GAMMA 0x9E3779B97F4A7C15ULL
#define SYNTH_STREAM_MUL 0xD1B54A32D192ED03ULL

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

uint64_t synth_rng_u64(uint64_t seed, uint64_t stream, uint64_t i) {
  uint64_t s0 = seed ^ (stream * SYNTH_STREAM_MUL);
  return mix64(s0 + (i + 1) * SYNTH_GAMMA);
}

/* uniform in [0,1) with 53 random bits (exact) */
static inline double u01(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }
/* uniform in [-1,1): 2*u01 - 1 is exact in binary64 */
static inline double upm1(uint64_t x) { return 2.0 * u01(x) - 1.0; }
/* integer in [0, N) by the high half of a 64x64 product */
static inline uint64_t uint_below(uint64_t x, uint64_t N) {
  return (uint64_t)(((unsigned __int128)x * (unsigned __int128)N) >> 64);
}

/* raw start / test vector: out[i] = uniform(-1,1) draw i of (seed, stream) */
void synth_uniform_pm1(int64_t n, uint64_t seed, uint64_t stream, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) out[i] = upm1(synth_rng_u64(seed, stream, (uint64_t)i));
}

/* ------------------------------------------------------------------ */
/* CSR container                                                        */
/* ------------------------------------------------------------------ */
typedef struct synth_csr {
  int64_t n, nnz;
  int64_t* row_ptr;
  int32_t* col;
  double* val;
} synth_csr;

int64_t synth_csr_n(const synth_csr* A) { return A ? A->n : -1; }
int64_t synth_csr_nnz(const synth_csr* A) { return A ? A->nnz : -1; }

void synth_csr_free(synth_csr* A) {
  if (!A) return;
  free(A->row_ptr);
  free(A->col);
  free(A->val);
  free(A);
}

/* copy the CSR arrays into caller-owned buffers (any may be NULL) */
void synth_csr_export(const synth_csr* A, int64_t* row_ptr, int32_t* col, double* val) {
  if (!A) return;
  if (row_ptr) memcpy(row_ptr, A->row_ptr, sizeof(int64_t) * (size_t)(A->n + 1));
  const int64_t nnz = A->nnz;
  const int64_t chunk = 1 << 22;
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < nnz; s += chunk) {
    int64_t e = s + chunk < nnz ? s + chunk : nnz;
    if (col) memcpy(col + s, A->col + s, sizeof(int32_t) * (size_t)(e - s));
    if (val) memcpy(val + s, A->val + s, sizeof(double) * (size_t)(e - s));
  }
}

/* copy values rounded to binary32 (round to nearest even) */
void synth_csr_export_f32(const synth_csr* A, float* val) {
  if (!A || !val) return;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < A->nnz; ++k) val[k] = (float)A->val[k];
}

/* ------------------------------------------------------------------ */
/* Entry list -> CSR with sorted, merged columns                        */
/* ------------------------------------------------------------------ */
typedef struct {
  int32_t c;
  double v;
} cv_pair;

static int cmp_cv(const void* a, const void* b) {
  const cv_pair* x = (const cv_pair*)a;
  const cv_pair* y = (const cv_pair*)b;
  if (x->c != y->c) return x->c < y->c ? -1 : 1;
  if (x->v != y->v) return x->v < y->v ? -1 : 1;
  return 0;
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/*
 * Build a CSR from m entries (r[k], c[k], v[k]).  With v == NULL every entry
 * has weight one and duplicates collapse to a single entry of value 1;
 * otherwise duplicates are summed (in ascending value order, so the result is
 * independent of the scatter order).
 */
static synth_csr* build_csr(int64_t n, int64_t m, const int32_t* r, const int32_t* c,
                            const double* v) {
  synth_csr* A = (synth_csr*)calloc(1, sizeof(synth_csr));
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!A || !cnt) goto fail;
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < m; ++k) __atomic_fetch_add(&cnt[r[k] + 1], 1, __ATOMIC_RELAXED);
  for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
  int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int32_t* tc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  double* tv = v ? (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1)) : NULL;
  int64_t* len = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!cur || !tc || (v && !tv) || !len) {
    free(cur); free(tc); free(tv); free(len);
    goto fail;
  }
  memcpy(cur, cnt, sizeof(int64_t) * (size_t)n);
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < m; ++k) {
    int64_t p = __atomic_fetch_add(&cur[r[k]], 1, __ATOMIC_RELAXED);
    tc[p] = c[k];
    if (v) tv[p] = v[k];
  }
  free(cur);
  /* sort + merge every row in place */
#pragma omp parallel
  {
    cv_pair* buf = NULL;
    int64_t cap = 0;
#pragma omp for schedule(dynamic, 4096)
    for (int64_t i = 0; i < n; ++i) {
      int64_t b = cnt[i], e = cnt[i + 1], L = e - b;
      if (L == 0) { len[i + 1] = 0; continue; }
      if (!v) {
        qsort(tc + b, (size_t)L, sizeof(int32_t), cmp_i32);
        int64_t w = b;
        for (int64_t k = b; k < e; ++k)
          if (k == b || tc[k] != tc[w - 1]) tc[w++] = tc[k];
        len[i + 1] = w - b;
      } else {
        if (L > cap) {
          free(buf);
          cap = L;
          buf = (cv_pair*)malloc(sizeof(cv_pair) * (size_t)cap);
        }
        for (int64_t k = 0; k < L; ++k) { buf[k].c = tc[b + k]; buf[k].v = tv[b + k]; }
        qsort(buf, (size_t)L, sizeof(cv_pair), cmp_cv);
        int64_t w = 0;
        for (int64_t k = 0; k < L; ++k) {
          if (w > 0 && buf[k].c == buf[w - 1].c) buf[w - 1].v += buf[k].v;
          else buf[w++] = buf[k];
        }
        for (int64_t k = 0; k < w; ++k) { tc[b + k] = buf[k].c; tv[b + k] = buf[k].v; }
        len[i + 1] = w;
      }
    }
    free(buf);
  }
  for (int64_t i = 0; i < n; ++i) len[i + 1] += len[i];
  A->n = n;
  A->nnz = len[n];
  A->row_ptr = len;
  A->col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(A->nnz > 0 ? A->nnz : 1));
  A->val = (double*)malloc(sizeof(double) * (size_t)(A->nnz > 0 ? A->nnz : 1));
  if (!A->col || !A->val) { free(tc); free(tv); free(cnt); synth_csr_free(A); return NULL; }
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t i = 0; i < n; ++i) {
    int64_t src = cnt[i], dst = len[i], L = len[i + 1] - len[i];
    memcpy(A->col + dst, tc + src, sizeof(int32_t) * (size_t)L);
    if (v) memcpy(A->val + dst, tv + src, sizeof(double) * (size_t)L);
    else for (int64_t k = 0; k < L; ++k) A->val[dst + k] = 1.0;
  }
  free(tc);
  free(tv);
  free(cnt);
  return A;
fail:
  free(cnt);
  free(A);
  return NULL;
}

/*
 * Uniform-random symmetric matrix: row i of A draws `per_row` entries with
 * column uniform in [0, n) (stream 101) and value uniform(0,1) (stream 102);
 * duplicates are summed, then S = A + A^T (so diagonal entries double).
 */
synth_csr* synth_uniform_sym(int64_t n, int32_t per_row, uint64_t seed) {
  if (n <= 0 || per_row < 0 || n > INT32_MAX) return NULL;
  int64_t e = n * per_row, m = 2 * e;
  int32_t* r = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  int32_t* c = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  double* v = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  if (!r || !c || !v) { free(r); free(c); free(v); return NULL; }
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < e; ++k) {
    int32_t i = (int32_t)(k / per_row);
    int32_t j = (int32_t)uint_below(synth_rng_u64(seed, 101, (uint64_t)k), (uint64_t)n);
    double x = u01(synth_rng_u64(seed, 102, (uint64_t)k));
    r[2 * k] = i; c[2 * k] = j; v[2 * k] = x;
    r[2 * k + 1] = j; c[2 * k + 1] = i; v[2 * k + 1] = x;
  }
  synth_csr* A = build_csr(n, m, r, c, v);
  free(r); free(c); free(v);
  return A;
}

/*
 * Banded symmetric matrix: row i of A draws `per_row` entries with column
 * i + d, d uniform in [1, half_width] (stream 103), and value uniform(0,1)
 * (stream 104); draws past the last column are dropped, duplicates summed,
 * then S = A + A^T.  Every column of row i lies within half_width of i: a
 * mesh-like structure whose SpMV reads x with locality.
 */
synth_csr* synth_banded_sym(int64_t n, int32_t per_row, int32_t half_width, uint64_t seed) {
  if (n <= 0 || per_row < 0 || half_width < 1 || n > INT32_MAX) return NULL;
  int64_t e = n * per_row;
  int32_t* r = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * e > 0 ? 2 * e : 1));
  int32_t* c = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * e > 0 ? 2 * e : 1));
  double* v = (double*)malloc(sizeof(double) * (size_t)(2 * e > 0 ? 2 * e : 1));
  int64_t* keep = (int64_t*)malloc(sizeof(int64_t) * (size_t)(e > 0 ? e : 1));
  if (!r || !c || !v || !keep) { free(r); free(c); free(v); free(keep); return NULL; }
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < e; ++k) {
    int64_t i = k / per_row;
    int64_t j = i + 1 + (int64_t)uint_below(synth_rng_u64(seed, 103, (uint64_t)k),
                                            (uint64_t)half_width);
    keep[k] = j < n ? j : -1;
  }
  int64_t m = 0;
  for (int64_t k = 0; k < e; ++k) {
    if (keep[k] < 0) continue;
    int32_t i = (int32_t)(k / per_row), j = (int32_t)keep[k];
    double x = u01(synth_rng_u64(seed, 104, (uint64_t)k));
    r[m] = i; c[m] = j; v[m] = x; ++m;
    r[m] = j; c[m] = i; v[m] = x; ++m;
  }
  free(keep);
  synth_csr* A = build_csr(n, m, r, c, v);
  free(r); free(c); free(v);
  return A;
}

/*
 * R-MAT / Kronecker graph (Chakrabarti, Zhan & Faloutsos 2004) with
 * n = 2^scale vertices and edge_factor * n edge draws.  Each draw descends
 * `scale` levels, picking quadrant (0,0),(0,1),(1,0),(1,1) with probabilities
 * a, b, c, 1-a-b-c (stream 110, 32 random bits per level).  Vertex ids are
 * then relabelled by a seeded Fisher-Yates permutation (stream 111),
 * self-loops dropped, the graph symmetrised and duplicate edges merged
 * (weight 1).  With `normalized` the value of (i,j) becomes
 * 1/sqrt(d_i d_j) (D^{-1/2} A D^{-1/2}); isolated vertices give empty rows.
 */
synth_csr* synth_rmat_sym(int32_t scale, int32_t edge_factor, double a, double b, double c,
                          uint64_t seed, int normalized) {
  if (scale < 1 || scale > 30 || edge_factor < 0) return NULL;
  const int64_t n = (int64_t)1 << scale;
  const int64_t E = n * (int64_t)edge_factor;
  const int32_t halves = (scale + 1) / 2;
  const double tab = a + b, tabc = a + b + c;
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* r = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * E > 0 ? 2 * E : 1));
  int32_t* cc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * E > 0 ? 2 * E : 1));
  if (!perm || !r || !cc) { free(perm); free(r); free(cc); return NULL; }
  for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  for (int64_t i = n - 1; i >= 1; --i) {
    int64_t j = (int64_t)uint_below(synth_rng_u64(seed, 111, (uint64_t)i), (uint64_t)(i + 1));
    int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
  }
  int64_t kept = 0;
#pragma omp parallel
  {
#pragma omp for schedule(static) reduction(+ : kept)
    for (int64_t e = 0; e < E; ++e) {
      int64_t u = 0, w = 0;
      uint64_t x = 0;
      for (int32_t l = 0; l < scale; ++l) {
        uint32_t bits;
        if ((l & 1) == 0) {
          x = synth_rng_u64(seed, 110, (uint64_t)e * (uint64_t)halves + (uint64_t)(l >> 1));
          bits = (uint32_t)(x >> 32);
        } else {
          bits = (uint32_t)(x & 0xffffffffu);
        }
        double p = (double)bits * 0x1.0p-32;
        int64_t bit = (int64_t)1 << (scale - 1 - l);
        if (p < a) {
        } else if (p < tab) {
          w |= bit;
        } else if (p < tabc) {
          u |= bit;
        } else {
          u |= bit;
          w |= bit;
        }
      }
      int32_t pu = perm[u], pw = perm[w];
      if (pu == pw) {
        r[2 * e] = -1;
        continue;
      }
      r[2 * e] = pu; cc[2 * e] = pw;
      r[2 * e + 1] = pw; cc[2 * e + 1] = pu;
      kept += 1;
    }
  }
  free(perm);
  /* compact away self-loops (order preserving) */
  int64_t m = 0;
  for (int64_t e = 0; e < E; ++e) {
    if (r[2 * e] < 0) continue;
    r[m] = r[2 * e]; cc[m] = cc[2 * e]; ++m;
    r[m] = r[2 * e + 1]; cc[m] = cc[2 * e + 1]; ++m;
  }
  (void)kept;
  synth_csr* A = build_csr(n, m, r, cc, NULL);
  free(r); free(cc);
  if (!A) return NULL;
  if (normalized) {
    const int64_t* rp = A->row_ptr;
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t i = 0; i < n; ++i) {
      double di = (double)(rp[i + 1] - rp[i]);
      for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
        int32_t j = A->col[k];
        double dj = (double)(rp[j + 1] - rp[j]);
        A->val[k] = 1.0 / sqrt(di * dj);
      }
    }
  }
  return A;
}

/*
 * Planted communities: the uniform-random background of synth_uniform_sym
 * (`per_row` draws per row, streams 101/102, then A + A^T) plus `ncomm`
 * disjoint cliques of unit weight.  Community k (k = 0 .. ncomm-1) has
 * s_k = round(smin * ratio^(ncomm-1-k)) vertices, taken in order from a
 * seeded Fisher-Yates permutation of the vertex ids (stream 112); every pair
 * (i, j), i != j, of a community gets the entry 1 (added to a background
 * entry at the same position).  A clique of s vertices contributes an
 * eigenvalue near s - 1, so with ratio > 1 the matrix has ncomm outlying
 * eigenvalues in a geometric progression above the background's spectrum:
 * the community structure spectral clustering looks for.
 */
synth_csr* synth_planted_sym(int64_t n, int32_t per_row, int32_t ncomm, int32_t smin,
                             double ratio, uint64_t seed) {
  if (n <= 0 || per_row < 0 || ncomm < 0 || smin < 2 || !(ratio >= 1.0) || n > INT32_MAX)
    return NULL;
  int64_t* size = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ncomm > 0 ? ncomm : 1));
  if (!size) return NULL;
  int64_t members = 0, pairs = 0;
  for (int32_t k = 0; k < ncomm; ++k) {
    size[k] = (int64_t)floor((double)smin * pow(ratio, (double)(ncomm - 1 - k)) + 0.5);
    members += size[k];
    pairs += size[k] * (size[k] - 1);
  }
  if (members > n) { free(size); return NULL; }
  const int64_t e = n * per_row, m = 2 * e + pairs;
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* r = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  int32_t* c = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
  double* v = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  if (!perm || !r || !c || !v) {
    free(size); free(perm); free(r); free(c); free(v);
    return NULL;
  }
#pragma omp parallel for schedule(static)
  for (int64_t k = 0; k < e; ++k) {
    int32_t i = (int32_t)(k / per_row);
    int32_t j = (int32_t)uint_below(synth_rng_u64(seed, 101, (uint64_t)k), (uint64_t)n);
    double x = u01(synth_rng_u64(seed, 102, (uint64_t)k));
    r[2 * k] = i; c[2 * k] = j; v[2 * k] = x;
    r[2 * k + 1] = j; c[2 * k + 1] = i; v[2 * k + 1] = x;
  }
  for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  for (int64_t i = n - 1; i >= 1; --i) {
    int64_t j = (int64_t)uint_below(synth_rng_u64(seed, 112, (uint64_t)i), (uint64_t)(i + 1));
    int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
  }
  int64_t first = 0, at = 2 * e;
  for (int32_t k = 0; k < ncomm; ++k) {
    const int64_t s = size[k];
    for (int64_t a = 0; a < s; ++a)
      for (int64_t b = 0; b < s; ++b) {
        if (a == b) continue;
        r[at] = perm[first + a]; c[at] = perm[first + b]; v[at] = 1.0; ++at;
      }
    first += s;
  }
  free(size);
  free(perm);
  synth_csr* A = build_csr(n, m, r, c, v);
  free(r); free(c); free(v);
  return A;
}

/* build a CSR from caller entry triplets (duplicates summed); for tests */
synth_csr* synth_from_triplets(int64_t n, int64_t m, const int32_t* r, const int32_t* c,
                               const double* v) {
  if (n <= 0 || m < 0) return NULL;
  for (int64_t k = 0; k < m; ++k)
    if (r[k] < 0 || r[k] >= n || c[k] < 0 || c[k] >= n) return NULL;
  return build_csr(n, m, r, c, v);
}
