/*
 * ORACLE — test infrastructure only.
 *
 * Plain, slow, single-threaded FP64 reference for the CRS sparse matrix-vector
 * multiply and the index structures built around it.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may call it; the
 * library path never does.  It shares no code, header or table with the CUDA
 * library.  Compile with -O2 -ffp-contract=off and without -ffast-math: every
 * product is rounded, then added, in the order written here.
 *
 * Indices are 0-based (the paper's listing is 1-based Fortran).  The paper's
 * loop accumulates into C; here C is overwritten, i.e. the loop runs on a C
 * that starts at +0.0 (C = A*B).
 */
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* Sec. 1.2, CRS listing: for each row i, C(i) = C(i) + val(j) * B(col_idx(j))
 * for j = row_ptr(i) .. row_ptr(i+1)-1, in ascending j, starting from 0. */
void oracle_crs_spmv(int64_t n_rows, const int32_t* row_ptr, const int32_t* col_idx,
                     const double* val, const double* B, double* C) {
  for (int64_t i = 0; i < n_rows; ++i) {
    double s = 0.0;
    for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j) {
      double prod = val[j] * B[col_idx[j]];
      s = s + prod;
    }
    C[i] = s;
  }
}

/* The same loop applied to k right-hand sides at once.  B is row-major with
 * leading dimension ldb (B[col * ldb + c]), C row-major with ldc. */
void oracle_crs_spmm(int64_t n_rows, int64_t k, const int32_t* row_ptr, const int32_t* col_idx,
                     const double* val, const double* B, int64_t ldb, double* C, int64_t ldc) {
  for (int64_t i = 0; i < n_rows; ++i) {
    for (int64_t c = 0; c < k; ++c) {
      double s = 0.0;
      for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j) {
        double prod = val[j] * B[(int64_t)col_idx[j] * ldb + c];
        s = s + prod;
      }
      C[i * ldc + c] = s;
    }
  }
}

/* FP32-stored values: each val is first rounded to float (C conversion,
 * round-to-nearest-even), widened back to double, and the loop runs in FP64. */
void oracle_crs_spmm_f32val(int64_t n_rows, int64_t k, const int32_t* row_ptr,
                            const int32_t* col_idx, const double* val, const double* B,
                            int64_t ldb, double* C, int64_t ldc) {
  for (int64_t i = 0; i < n_rows; ++i) {
    for (int64_t c = 0; c < k; ++c) {
      double s = 0.0;
      for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j) {
        float v32 = (float)val[j];
        double prod = (double)v32 * B[(int64_t)col_idx[j] * ldb + c];
        s = s + prod;
      }
      C[i * ldc + c] = s;
    }
  }
}

/* The same row sums evaluated as if in twice the working precision, used to
 * attribute an error to one side when a parity check fails (it is not the
 * reference of any check).  Compensated dot product in the manner of Ogita, Rump and Oishi
 * (SIAM J. Sci. Comput. 26, 2005, "Dot2"): every product is split exactly into
 * p + e with one fused multiply-add (e = fma(a, b, -p), the rounding error of
 * p), the p are summed with Knuth's TwoSum, which yields each addition's
 * rounding error exactly, and all error terms are added to the sum at the end.
 * fma() is called explicitly; the file is compiled with -ffp-contract=off. */
static void two_sum(double a, double b, double* s, double* t) {
  const double x = a + b;
  const double z = x - a;
  *t = (a - (x - z)) + (b - z);
  *s = x;
}

void oracle_crs_spmm_dot2(int64_t n_rows, int64_t k, const int32_t* row_ptr, const int32_t* col_idx,
                          const double* val, const double* B, int64_t ldb, double* C, int64_t ldc) {
  for (int64_t i = 0; i < n_rows; ++i) {
    for (int64_t c = 0; c < k; ++c) {
      double s = 0.0, err = 0.0;
      for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j) {
        const double a = val[j], b = B[(int64_t)col_idx[j] * ldb + c];
        const double p = a * b;
        const double e = fma(a, b, -p);
        double t;
        two_sum(s, p, &s, &t);
        err = err + (t + e);
      }
      C[i * ldc + c] = s + err;
    }
  }
}

/* Error scale of the tolerance: S[i, c] = sum_j |val[j] * B[col_idx[j], c]|. */
void oracle_abs_scale(int64_t n_rows, int64_t k, const int32_t* row_ptr, const int32_t* col_idx,
                      const double* val, const double* B, int64_t ldb, double* S, int64_t lds) {
  for (int64_t i = 0; i < n_rows; ++i) {
    for (int64_t c = 0; c < k; ++c) {
      double s = 0.0;
      for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j)
        s = s + fabs(val[j] * B[(int64_t)col_idx[j] * ldb + c]);
      S[i * lds + c] = s;
    }
  }
}

/* ---------------------------------------------------------------------------
 * SELL-C-sigma (Kreutzer et al., SIAM J. Sci. Comput. 2014), the sliced ELLPACK
 * form of the same matrix.  Reading used throughout this project:
 *   1. rows are cut into windows of sigma consecutive rows; inside each window
 *      they are stably sorted by descending length (ties keep row order);
 *      perm[r] = original row at sorted position r;
 *   2. sorted rows are grouped into chunks of C; chunk c holds sorted rows
 *      [c*C, c*C + C); a last partial chunk is padded with empty rows;
 *   3. chunk_len[c] = the longest row of the chunk; chunk_ptr[c] = the element
 *      offset of chunk c = sum over earlier chunks of C * chunk_len;
 *   4. inside a chunk, storage is column-major: entry j of the row at lane t
 *      sits at chunk_ptr[c] + j*C + t;
 *   5. padding slots hold val = +0.0 and col = the row's last column (0 for an
 *      empty row, and for the padding rows of a partial chunk).
 * --------------------------------------------------------------------------- */

static int64_t rowlen(const int32_t* row_ptr, int64_t r) { return (int64_t)row_ptr[r + 1] - row_ptr[r]; }

/* Fills perm (n_rows entries); returns the stored element count
 * (sum of C * chunk_len) and, through n_chunks, the chunk count. */
int64_t oracle_sell_perm(int64_t n_rows, const int32_t* row_ptr, int64_t C, int64_t sigma,
                         int32_t* perm, int64_t* n_chunks) {
  for (int64_t r = 0; r < n_rows; ++r) perm[r] = (int32_t)r;
  if (sigma < 1) sigma = 1;
  for (int64_t w0 = 0; w0 < n_rows; w0 += sigma) {
    int64_t w1 = w0 + sigma < n_rows ? w0 + sigma : n_rows;
    /* stable insertion sort by descending length */
    for (int64_t a = w0 + 1; a < w1; ++a) {
      int32_t r = perm[a];
      int64_t len = rowlen(row_ptr, r);
      int64_t b = a - 1;
      while (b >= w0 && rowlen(row_ptr, perm[b]) < len) { perm[b + 1] = perm[b]; --b; }
      perm[b + 1] = r;
    }
  }
  int64_t nc = (n_rows + C - 1) / C;
  int64_t total = 0;
  for (int64_t c = 0; c < nc; ++c) {
    int64_t mx = 0;
    for (int64_t t = 0; t < C; ++t) {
      int64_t r = c * C + t;
      if (r < n_rows && rowlen(row_ptr, perm[r]) > mx) mx = rowlen(row_ptr, perm[r]);
    }
    total += C * mx;
  }
  *n_chunks = nc;
  return total;
}

/* Fills chunk_ptr[n_chunks+1], chunk_len[n_chunks], sell_col[total], sell_val[total]
 * for the perm from oracle_sell_perm. */
void oracle_sell_fill(int64_t n_rows, const int32_t* row_ptr, const int32_t* col_idx,
                      const double* val, int64_t C, const int32_t* perm, int64_t n_chunks,
                      int64_t* chunk_ptr, int32_t* chunk_len, int32_t* sell_col, double* sell_val) {
  int64_t off = 0;
  for (int64_t c = 0; c < n_chunks; ++c) {
    int64_t mx = 0;
    for (int64_t t = 0; t < C; ++t) {
      int64_t r = c * C + t;
      if (r < n_rows && rowlen(row_ptr, perm[r]) > mx) mx = rowlen(row_ptr, perm[r]);
    }
    chunk_ptr[c] = off;
    chunk_len[c] = (int32_t)mx;
    for (int64_t t = 0; t < C; ++t) {
      int64_t r = c * C + t;
      int64_t orig = r < n_rows ? perm[r] : -1;
      int64_t len = orig >= 0 ? rowlen(row_ptr, orig) : 0;
      int32_t last_col = 0;
      for (int64_t j = 0; j < mx; ++j) {
        int64_t slot = off + j * C + t;
        if (j < len) {
          int64_t src = row_ptr[orig] + j;
          sell_col[slot] = col_idx[src];
          sell_val[slot] = val[src];
          last_col = col_idx[src];
        } else {
          sell_col[slot] = last_col;
          sell_val[slot] = 0.0;
        }
      }
    }
    off += C * mx;
  }
  chunk_ptr[n_chunks] = off;
}

/* SELL-C-sigma product by definition of the format: for sorted row r, sum its
 * stored slots in order j = 0 .. chunk_len-1 (padding adds +0.0 * B), then
 * C[perm[r]] = s. */
void oracle_sell_spmv(int64_t n_rows, int64_t C, const int32_t* perm, int64_t n_chunks,
                      const int64_t* chunk_ptr, const int32_t* chunk_len, const int32_t* sell_col,
                      const double* sell_val, const double* B, double* Cout) {
  for (int64_t c = 0; c < n_chunks; ++c) {
    for (int64_t t = 0; t < C; ++t) {
      int64_t r = c * C + t;
      if (r >= n_rows) continue;
      double s = 0.0;
      for (int64_t j = 0; j < chunk_len[c]; ++j) {
        int64_t slot = chunk_ptr[c] + j * C + t;
        double prod = sell_val[slot] * B[sell_col[slot]];
        s = s + prod;
      }
      Cout[perm[r]] = s;
    }
  }
}

/* ---------------------------------------------------------------------------
 * Local / halo column split (Sec. 3.1, "vector mode with naive overlap", and
 * Sec. 3.2, task mode): the entries whose RHS element is available locally
 * (col < h) form the local matrix over every row; the others (col >= h) form
 * the halo matrix over the ascending list of rows that have any.  In-row entry
 * order is kept.  Column indices stay global.
 * --------------------------------------------------------------------------- */

/* Returns the halo nnz; n_halo_rows through the pointer. */
int64_t oracle_split_count(int64_t n_rows, const int32_t* row_ptr, const int32_t* col_idx,
                           int64_t h, int64_t* n_halo_rows) {
  int64_t nh = 0, hr = 0;
  for (int64_t i = 0; i < n_rows; ++i) {
    int64_t here = 0;
    for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j)
      if (col_idx[j] >= h) ++here;
    nh += here;
    if (here > 0) ++hr;
  }
  *n_halo_rows = hr;
  return nh;
}

void oracle_split_fill(int64_t n_rows, const int32_t* row_ptr, const int32_t* col_idx,
                       const double* val, int64_t h,
                       int32_t* loc_row_ptr, int32_t* loc_col, double* loc_val,
                       int32_t* halo_rows, int32_t* halo_row_ptr, int32_t* halo_col,
                       double* halo_val) {
  int64_t pl = 0, ph = 0, hr = 0;
  loc_row_ptr[0] = 0;
  halo_row_ptr[0] = 0;
  for (int64_t i = 0; i < n_rows; ++i) {
    int64_t before = ph;
    for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j) {
      if (col_idx[j] < h) {
        loc_col[pl] = col_idx[j];
        loc_val[pl++] = val[j];
      } else {
        halo_col[ph] = col_idx[j];
        halo_val[ph++] = val[j];
      }
    }
    loc_row_ptr[i + 1] = (int32_t)pl;
    if (ph > before) {
      halo_rows[hr] = (int32_t)i;
      halo_row_ptr[++hr] = (int32_t)ph;
    }
  }
}

/* Split product in the order of Sec. 3.1: first the local part writes C, then,
 * once the halo values are in, the non-local part is added to C. */
void oracle_split_spmv(int64_t n_rows, const int32_t* loc_row_ptr, const int32_t* loc_col,
                       const double* loc_val, int64_t n_halo_rows, const int32_t* halo_rows,
                       const int32_t* halo_row_ptr, const int32_t* halo_col,
                       const double* halo_val, const double* B, double* C) {
  oracle_crs_spmv(n_rows, loc_row_ptr, loc_col, loc_val, B, C);
  for (int64_t t = 0; t < n_halo_rows; ++t) {
    double s = 0.0;
    for (int64_t j = halo_row_ptr[t]; j < halo_row_ptr[t + 1]; ++j) {
      double prod = halo_val[j] * B[halo_col[j]];
      s = s + prod;
    }
    C[halo_rows[t]] = C[halo_rows[t]] + s;
  }
}

/* ---------------------------------------------------------------------------
 * Symmetric CRS (Sec. 1.3.1): a real symmetric matrix is fully described by
 * the entries on and above the diagonal, which roughly halves the stored
 * val/col_idx volume.  The paper gives no code for it; the definitions below
 * are the plain ones.
 * --------------------------------------------------------------------------- */

/* One off-diagonal entry as (r, c, key); the key is the value's bit pattern
 * with -0.0 mapped to +0.0, so that equal values compare equal. */
typedef struct {
  int64_t r, c;
  uint64_t key;
} sym_triple;

static uint64_t value_key(double v) {
  uint64_t b;
  if (v == 0.0) v = 0.0;  /* -0.0 -> +0.0 */
  memcpy(&b, &v, sizeof(b));
  return b;
}

static int triple_cmp(const void* a, const void* b) {
  const sym_triple* x = (const sym_triple*)a;
  const sym_triple* y = (const sym_triple*)b;
  if (x->r != y->r) return x->r < y->r ? -1 : 1;
  if (x->c != y->c) return x->c < y->c ? -1 : 1;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return 0;
}

/* 1 if the matrix is square and every entry strictly above the diagonal,
 * (i, j, v), is matched one to one by an entry (j, i, v) strictly below it
 * (as multisets, so duplicates must mirror one to one); else 0.  -1 if the
 * scratch allocation fails.  Entries strictly below the diagonal are listed
 * transposed, both lists are sorted and compared. */
int oracle_is_symmetric(int64_t n_rows, int64_t n_cols, const int32_t* row_ptr, const int32_t* col_idx,
                        const double* val) {
  if (n_rows != n_cols) return 0;
  int64_t nu = 0, nl = 0;
  for (int64_t i = 0; i < n_rows; ++i)
    for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j) {
      if (col_idx[j] > i) ++nu;
      if (col_idx[j] < i) ++nl;
    }
  if (nu != nl) return 0;
  sym_triple* U = (sym_triple*)malloc(sizeof(sym_triple) * (size_t)(nu > 0 ? nu : 1));
  sym_triple* L = (sym_triple*)malloc(sizeof(sym_triple) * (size_t)(nl > 0 ? nl : 1));
  if (!U || !L) {
    free(U);
    free(L);
    return -1;
  }
  int64_t pu = 0, pl = 0;
  for (int64_t i = 0; i < n_rows; ++i)
    for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j) {
      int64_t c = col_idx[j];
      if (c > i) {
        U[pu].r = i;
        U[pu].c = c;
        U[pu++].key = value_key(val[j]);
      } else if (c < i) {
        L[pl].r = c; /* transposed */
        L[pl].c = i;
        L[pl++].key = value_key(val[j]);
      }
    }
  qsort(U, (size_t)nu, sizeof(sym_triple), triple_cmp);
  qsort(L, (size_t)nl, sizeof(sym_triple), triple_cmp);
  int same = 1;
  for (int64_t t = 0; t < nu && same; ++t)
    if (triple_cmp(U + t, L + t) != 0) same = 0;
  free(U);
  free(L);
  return same;
}

/* Number of entries on or above the diagonal (col_idx >= row). */
int64_t oracle_sym_count(int64_t n_rows, const int32_t* row_ptr, const int32_t* col_idx) {
  int64_t n = 0;
  for (int64_t i = 0; i < n_rows; ++i)
    for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j)
      if (col_idx[j] >= i) ++n;
  return n;
}

/* The stored triangle: for every row, its entries with col_idx >= row, in
 * the order they have in the row. */
void oracle_sym_fill(int64_t n_rows, const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                     int32_t* u_row_ptr, int32_t* u_col, double* u_val) {
  int64_t p = 0;
  u_row_ptr[0] = 0;
  for (int64_t i = 0; i < n_rows; ++i) {
    for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j)
      if (col_idx[j] >= i) {
        u_col[p] = col_idx[j];
        u_val[p++] = val[j];
      }
    u_row_ptr[i + 1] = (int32_t)p;
  }
}

/* Product from the stored triangle, rows in order: a stored entry u(i,j)
 * adds u(i,j)*B(j) to C(i) and, when j != i, its mirror u(i,j)*B(i) to C(j).
 * C starts at +0.0. */
void oracle_sym_spmv(int64_t n_rows, const int32_t* u_row_ptr, const int32_t* u_col, const double* u_val,
                     const double* B, double* C) {
  for (int64_t i = 0; i < n_rows; ++i) C[i] = 0.0;
  for (int64_t i = 0; i < n_rows; ++i) {
    for (int64_t j = u_row_ptr[i]; j < u_row_ptr[i + 1]; ++j) {
      int64_t c = u_col[j];
      double prod = u_val[j] * B[c];
      C[i] = C[i] + prod;
      if (c != i) {
        double mirror = u_val[j] * B[i];
        C[c] = C[c] + mirror;
      }
    }
  }
}
