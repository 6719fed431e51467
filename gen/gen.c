/*
 * Seeded synthetic input generators for the CRS sparse matrix-vector multiply.
 *
 * This file produces INPUTS only: CRS matrices (row_ptr / col_idx / val) and
 * right-hand-side vectors.  It contains none of the spMVM arithmetic.  Both the
 * CPU oracle and the GPU path consume what it produces; neither shares any other
 * code with it.
 *
 * Random numbers: SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) expands a
 * (seed, stream) pair into the 256-bit state of xoshiro256** (Blackman and
 * Vigna, 2018), written here from their published descriptions.
 *   uniform01()   = (x >> 11) * 2^-53                       in [0, 1)
 *   uniform_int(n)= floor(x * n / 2^64)  (128-bit product)   in [0, n)
 *   normal()      = Box-Muller, cos branch, one normal per two uniforms
 *
 * Workloads (shapes follow the paper's test matrices, Sec. 1.3.1):
 *   laplace2d     2D 5-point Dirichlet Laplacian (4, -1), natural order.
 *   poisson3d_var 3D 7-point variable-coefficient Poisson stencil; each edge
 *                 draws u~U[0,1) once (rows in natural order, then +x, +y, +z)
 *                 and stores -(1+u) at (i,j) and (j,i); the diagonal is the sum
 *                 of |off-diagonal| of the kept neighbours (ascending column
 *                 order) plus 1e-3.  Stand-in for the sAMG matrix (N~2.2e7,
 *                 Nnzr~7).
 *   eigen_shaped  symmetric eigenproblem-shaped matrix: diagonal N(0,1); band
 *                 pairs (i,i+1), (i,i+2) kept with p; per row P scattered
 *                 symmetric partners j=i+d, d~U{-W..W}, resampled when j is out
 *                 of range, |d|<=2, or the pair exists.  Stand-in for the HMeP
 *                 matrix (N=6.2e6, Nnzr~15).
 *   powerlaw      random square matrix, row lengths from the discrete power law
 *                 P(L) ~ L^-alpha on [lmin, min(lmax, N)], distinct uniform
 *                 columns sorted ascending, values U[-1,1).
 *
 * All matrices come back with columns ascending inside each row.  Compile with
 * -ffp-contract=off so that the x86 and Arm builds draw the same numbers.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ RNG */

typedef struct { uint64_t s[4]; } gen_rng;

static uint64_t splitmix64_next(uint64_t* x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static void rng_init(gen_rng* r, uint64_t seed, uint64_t stream) {
  uint64_t x = seed ^ (0xD1B54A32D192ED03ULL * (stream + 1));
  for (int i = 0; i < 4; ++i) r->s[i] = splitmix64_next(&x);
}

static inline uint64_t rng_next(gen_rng* r) {
  uint64_t* s = r->s;
  const uint64_t result = rotl64(s[1] * 5, 7) * 9;
  const uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl64(s[3], 45);
  return result;
}

static inline double rng_uniform01(gen_rng* r) {
  return (double)(rng_next(r) >> 11) * 0x1.0p-53;
}

static inline uint64_t rng_uniform_int(gen_rng* r, uint64_t n) {
  return (uint64_t)(((unsigned __int128)rng_next(r) * n) >> 64);
}

static inline double rng_normal(gen_rng* r) {
  double u1 = 1.0 - rng_uniform01(r); /* (0, 1] */
  double u2 = rng_uniform01(r);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* ------------------------------------------------------------ CRS output */

typedef struct {
  int64_t n_rows, n_cols, nnz;
  int32_t* row_ptr; /* n_rows + 1 */
  int32_t* col_idx; /* nnz */
  double* val;      /* nnz */
} gen_csr;

void gen_free(gen_csr* m) {
  if (!m) return;
  free(m->row_ptr);
  free(m->col_idx);
  free(m->val);
  m->row_ptr = NULL;
  m->col_idx = NULL;
  m->val = NULL;
}

static int csr_alloc(gen_csr* m, int64_t n_rows, int64_t n_cols, int64_t nnz) {
  m->n_rows = n_rows;
  m->n_cols = n_cols;
  m->nnz = nnz;
  m->row_ptr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n_rows + 1));
  m->col_idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  m->val = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  if (!m->row_ptr || !m->col_idx || !m->val) {
    gen_free(m);
    return -1;
  }
  return 0;
}

/* Vector of n values uniform in [lo, hi): lo + (hi-lo)*u. */
void gen_uniform(uint64_t seed, uint64_t stream, int64_t n, double lo, double hi, double* out) {
  gen_rng r;
  rng_init(&r, seed, stream);
  for (int64_t i = 0; i < n; ++i) out[i] = lo + (hi - lo) * rng_uniform01(&r);
}

/* ------------------------------------------------- 2D 5-point Laplacian */

int gen_laplace2d(int64_t nx, int64_t ny, gen_csr* out) {
  if (nx < 1 || ny < 1 || nx * ny > INT32_MAX) return -2;
  int64_t n = nx * ny;
  int64_t nnz = 5 * n - 2 * nx - 2 * ny;
  if (nnz > INT32_MAX) return -2;
  if (csr_alloc(out, n, n, nnz)) return -1;
  int64_t p = 0;
  out->row_ptr[0] = 0;
  for (int64_t y = 0; y < ny; ++y) {
    for (int64_t x = 0; x < nx; ++x) {
      int64_t i = x + nx * y;
      if (y > 0) { out->col_idx[p] = (int32_t)(i - nx); out->val[p++] = -1.0; }
      if (x > 0) { out->col_idx[p] = (int32_t)(i - 1); out->val[p++] = -1.0; }
      out->col_idx[p] = (int32_t)i; out->val[p++] = 4.0;
      if (x < nx - 1) { out->col_idx[p] = (int32_t)(i + 1); out->val[p++] = -1.0; }
      if (y < ny - 1) { out->col_idx[p] = (int32_t)(i + nx); out->val[p++] = -1.0; }
      out->row_ptr[i + 1] = (int32_t)p;
    }
  }
  return p == nnz ? 0 : -3;
}

/* -------------------------------- 3D 7-point variable-coefficient Poisson */

int gen_poisson3d_var(int64_t n, uint64_t seed, uint64_t stream, gen_csr* out) {
  if (n < 1) return -2;
  int64_t N = n * n * n;
  int64_t nnz = 7 * N - 6 * n * n;
  if (N > INT32_MAX || nnz > INT32_MAX) return -2;
  double* ex = (double*)malloc(sizeof(double) * (size_t)N);
  double* ey = (double*)malloc(sizeof(double) * (size_t)N);
  double* ez = (double*)malloc(sizeof(double) * (size_t)N);
  if (!ex || !ey || !ez) { free(ex); free(ey); free(ez); return -1; }
  gen_rng r;
  rng_init(&r, seed, stream);
  const int64_t nn = n * n;
  /* one draw per edge, rows in natural order, then +x, +y, +z */
  for (int64_t z = 0; z < n; ++z)
    for (int64_t y = 0; y < n; ++y)
      for (int64_t x = 0; x < n; ++x) {
        int64_t i = x + n * (y + n * z);
        ex[i] = (x < n - 1) ? -(1.0 + rng_uniform01(&r)) : 0.0;
        ey[i] = (y < n - 1) ? -(1.0 + rng_uniform01(&r)) : 0.0;
        ez[i] = (z < n - 1) ? -(1.0 + rng_uniform01(&r)) : 0.0;
      }
  if (csr_alloc(out, N, N, nnz)) { free(ex); free(ey); free(ez); return -1; }
  int64_t p = 0;
  out->row_ptr[0] = 0;
  for (int64_t z = 0; z < n; ++z)
    for (int64_t y = 0; y < n; ++y)
      for (int64_t x = 0; x < n; ++x) {
        int64_t i = x + n * (y + n * z);
        double nb[6];
        int64_t nc[6];
        int k = 0;
        if (z > 0) { nc[k] = i - nn; nb[k++] = ez[i - nn]; }
        if (y > 0) { nc[k] = i - n; nb[k++] = ey[i - n]; }
        if (x > 0) { nc[k] = i - 1; nb[k++] = ex[i - 1]; }
        int lower = k;
        if (x < n - 1) { nc[k] = i + 1; nb[k++] = ex[i]; }
        if (y < n - 1) { nc[k] = i + n; nb[k++] = ey[i]; }
        if (z < n - 1) { nc[k] = i + nn; nb[k++] = ez[i]; }
        double d = 0.0;
        for (int t = 0; t < k; ++t) d += fabs(nb[t]);
        d += 1e-3;
        for (int t = 0; t < lower; ++t) { out->col_idx[p] = (int32_t)nc[t]; out->val[p++] = nb[t]; }
        out->col_idx[p] = (int32_t)i; out->val[p++] = d;
        for (int t = lower; t < k; ++t) { out->col_idx[p] = (int32_t)nc[t]; out->val[p++] = nb[t]; }
        out->row_ptr[i + 1] = (int32_t)p;
      }
  free(ex); free(ey); free(ez);
  return p == nnz ? 0 : -3;
}

/* ------------------------------------------- eigenproblem-shaped matrix */

typedef struct { uint64_t* key; uint64_t mask; } pair_set;

static inline uint64_t pair_hash(uint64_t k) {
  k ^= k >> 33; k *= 0xFF51AFD7ED558CCDULL; k ^= k >> 33; k *= 0xC4CEB9FE1A85EC53ULL; k ^= k >> 33;
  return k;
}

/* returns 1 if inserted, 0 if already present */
static int pair_set_insert(pair_set* s, uint64_t k) {
  uint64_t h = pair_hash(k) & s->mask;
  for (;;) {
    if (s->key[h] == 0) { s->key[h] = k; return 1; }
    if (s->key[h] == k) return 0;
    h = (h + 1) & s->mask;
  }
}

static void sort_row(int32_t* c, double* v, int64_t len) {
  for (int64_t a = 1; a < len; ++a) {
    int32_t cc = c[a]; double vv = v[a]; int64_t b = a - 1;
    while (b >= 0 && c[b] > cc) { c[b + 1] = c[b]; v[b + 1] = v[b]; --b; }
    c[b + 1] = cc; v[b + 1] = vv;
  }
}

int gen_eigen_shaped(int64_t N, int64_t window, int pairs_per_row, double band_p,
                     uint64_t seed, uint64_t stream, gen_csr* out) {
  if (N < 64 || N > INT32_MAX || window < 3 || pairs_per_row < 0) return -2;
  gen_rng r;
  rng_init(&r, seed, stream);
  int64_t n_band_max = 2 * N;
  int64_t n_scat = (int64_t)pairs_per_row * N;
  int64_t n_edges_max = n_band_max + n_scat;
  int32_t* ei = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_edges_max);
  int32_t* ej = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_edges_max);
  double* ev = (double*)malloc(sizeof(double) * (size_t)n_edges_max);
  double* diag = (double*)malloc(sizeof(double) * (size_t)N);
  uint64_t cap = 1;
  while (cap < (uint64_t)(2 * n_scat + 16)) cap <<= 1;
  pair_set set = { (uint64_t*)calloc(cap, sizeof(uint64_t)), cap - 1 };
  int32_t* cnt = (int32_t*)calloc((size_t)N + 1, sizeof(int32_t));
  if (!ei || !ej || !ev || !diag || !set.key || !cnt) {
    free(ei); free(ej); free(ev); free(diag); free(set.key); free(cnt);
    return -1;
  }
  /* 1. diagonal */
  for (int64_t i = 0; i < N; ++i) diag[i] = rng_normal(&r);
  /* 2. near bands: pairs (i, i+1) and (i, i+2), kept with probability band_p */
  int64_t ne = 0;
  for (int64_t i = 0; i < N; ++i)
    for (int off = 1; off <= 2; ++off) {
      if (i + off >= N) continue;
      if (rng_uniform01(&r) < band_p) {
        ei[ne] = (int32_t)i; ej[ne] = (int32_t)(i + off);
        ev[ne++] = -1.0 + 2.0 * rng_uniform01(&r);
      }
    }
  /* 3. scattered symmetric partners */
  const uint64_t span = 2 * (uint64_t)window + 1;
  for (int64_t i = 0; i < N; ++i) {
    for (int t = 0; t < pairs_per_row; ++t) {
      int64_t j;
      for (;;) {
        int64_t d = (int64_t)rng_uniform_int(&r, span) - window;
        j = i + d;
        if (j < 0 || j >= N || (d >= -2 && d <= 2)) continue;
        uint64_t lo = (uint64_t)(i < j ? i : j), hi = (uint64_t)(i < j ? j : i);
        if (!pair_set_insert(&set, lo * (uint64_t)N + hi + 1)) continue;
        break;
      }
      ei[ne] = (int32_t)i; ej[ne] = (int32_t)j;
      ev[ne++] = -1.0 + 2.0 * rng_uniform01(&r);
    }
  }
  free(set.key);
  /* assemble: each row holds its diagonal plus both ends of every edge */
  for (int64_t i = 0; i < N; ++i) cnt[i + 1] = 1;
  for (int64_t e = 0; e < ne; ++e) { cnt[ei[e] + 1]++; cnt[ej[e] + 1]++; }
  for (int64_t i = 0; i < N; ++i) cnt[i + 1] += cnt[i];
  int64_t nnz = cnt[N];
  if (csr_alloc(out, N, N, nnz)) {
    free(ei); free(ej); free(ev); free(diag); free(cnt);
    return -1;
  }
  memcpy(out->row_ptr, cnt, sizeof(int32_t) * (size_t)(N + 1));
  for (int64_t i = 0; i < N; ++i) {
    int32_t p = cnt[i]++;
    out->col_idx[p] = (int32_t)i; out->val[p] = diag[i];
  }
  for (int64_t e = 0; e < ne; ++e) {
    int32_t p = cnt[ei[e]]++;
    out->col_idx[p] = ej[e]; out->val[p] = ev[e];
    p = cnt[ej[e]]++;
    out->col_idx[p] = ei[e]; out->val[p] = ev[e];
  }
  for (int64_t i = 0; i < N; ++i)
    sort_row(out->col_idx + out->row_ptr[i], out->val + out->row_ptr[i],
             out->row_ptr[i + 1] - out->row_ptr[i]);
  free(ei); free(ej); free(ev); free(diag); free(cnt);
  return 0;
}

/* ---------------------------------------------------- power-law matrix */

/* Matrix dimension for member `stream` of a batch: round(exp(U[ln lo, ln hi))).
 * Drawn first from the member's own generator, so that gen_powerlaw with the
 * same (seed, stream) continues the same sequence. */
static int64_t draw_loguniform_dim(gen_rng* r, double lo, double hi) {
  double u = rng_uniform01(r);
  return (int64_t)llround(exp(log(lo) + (log(hi) - log(lo)) * u));
}

int64_t gen_powerlaw_dim(uint64_t seed, uint64_t stream, double lo, double hi) {
  gen_rng r;
  rng_init(&r, seed, stream);
  return draw_loguniform_dim(&r, lo, hi);
}

/* If n <= 0 the dimension is drawn log-uniformly in [dim_lo, dim_hi] first.
 * Per row: length L by inverse CDF of the truncated discrete power law, then L
 * distinct columns (rejection), sorted, then L values U[-1,1). */
int gen_powerlaw(int64_t n, double dim_lo, double dim_hi, double alpha, int64_t lmin, int64_t lmax,
                 uint64_t seed, uint64_t stream, gen_csr* out) {
  gen_rng r;
  rng_init(&r, seed, stream);
  if (n <= 0) n = draw_loguniform_dim(&r, dim_lo, dim_hi);
  if (n < 1 || n > INT32_MAX / 4 || lmin < 0) return -2;
  int64_t hi = lmax < n ? lmax : n;
  if (hi < lmin) return -2;
  int64_t nl = hi - lmin + 1;
  double* cdf = (double*)malloc(sizeof(double) * (size_t)nl);
  int32_t* len = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int64_t* stamp = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  if (!cdf || !len || !stamp) { free(cdf); free(len); free(stamp); return -1; }
  double acc = 0.0;
  for (int64_t l = lmin; l <= hi; ++l) {
    acc += (l == 0) ? 0.0 : pow((double)l, -alpha);
    cdf[l - lmin] = acc;
  }
  /* row lengths first (one uniform each), then the entries row by row */
  int64_t nnz = 0;
  for (int64_t i = 0; i < n; ++i) {
    double u = rng_uniform01(&r) * acc;
    int64_t a = 0, b = nl - 1; /* smallest index with cdf > u */
    while (a < b) { int64_t m = (a + b) / 2; if (cdf[m] > u) b = m; else a = m + 1; }
    len[i] = (int32_t)(lmin + a);
    nnz += len[i];
  }
  free(cdf);
  if (nnz > INT32_MAX || csr_alloc(out, n, n, nnz)) { free(len); free(stamp); return nnz > INT32_MAX ? -2 : -1; }
  for (int64_t i = 0; i < n; ++i) stamp[i] = -1;
  int64_t p = 0;
  out->row_ptr[0] = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t start = p;
    for (int32_t t = 0; t < len[i]; ++t) {
      int64_t c;
      do { c = (int64_t)rng_uniform_int(&r, (uint64_t)n); } while (stamp[c] == i);
      stamp[c] = i;
      out->col_idx[p++] = (int32_t)c;
    }
    for (int64_t q = start; q < p; ++q) out->val[q] = -1.0 + 2.0 * rng_uniform01(&r);
    sort_row(out->col_idx + start, out->val + start, p - start);
    out->row_ptr[i + 1] = (int32_t)p;
  }
  free(len); free(stamp);
  return 0;
}
