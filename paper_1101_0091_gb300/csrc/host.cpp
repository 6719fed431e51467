// Host-side analysis and format builders of the plan: CRS validation, the row
// blocks of CRS_STAGED, SELL-C-sigma, the local/halo split, and the feature
// vector read by the cost model.  One-time work at plan creation.
#include <algorithm>
#include <functional>
#include <cmath>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace spmv {

bool validate_csr(int64_t n_rows, int64_t n_cols, const int32_t* row_ptr, const int32_t* col, std::string* why) {
  if (n_rows < 0 || n_cols < 0) {
    *why = "negative dimension";
    return false;
  }
  if (n_rows > INT32_MAX - 1 || n_cols > INT32_MAX) {
    *why = "dimension exceeds int32 indexing";
    return false;
  }
  if (!row_ptr) {
    *why = "row_ptr is NULL";
    return false;
  }
  if (row_ptr[0] != 0) {
    *why = "row_ptr[0] != 0";
    return false;
  }
  for (int64_t i = 0; i < n_rows; ++i) {
    if (row_ptr[i + 1] < row_ptr[i]) {
      *why = "row_ptr decreases at row " + std::to_string(i);
      return false;
    }
  }
  const int64_t nnz = row_ptr[n_rows];
  if (nnz > 0 && !col) {
    *why = "col_idx is NULL";
    return false;
  }
  for (int64_t j = 0; j < nnz; ++j) {
    if (col[j] < 0 || col[j] >= n_cols) {
      *why = "col_idx[" + std::to_string(j) + "] = " + std::to_string(col[j]) + " outside [0, n_cols)";
      return false;
    }
  }
  return true;
}

bool has_special_f32(const float* v, int64_t n) {
  for (int64_t i = 0; i < n; ++i) {
    uint32_t u;
    std::memcpy(&u, v + i, 4);
    const uint32_t a = u & 0x7fffffffu;
    if (a != 0 && (a < 0x00800000u || a >= 0x7f800000u)) return true;
  }
  return false;
}

// Blocks of CRS_STAGED.  A tile block: consecutive rows of length <= long_row,
// at most rows_per_block rows and at most `tile` entries.  A warp block: up to
// 8 consecutive rows longer than long_row.  Entry b is the first row of block b
// (high bit set for a warp block); the last entry is n_rows.  The tile
// capacity is 1.25 x the entries of an average full block, rounded up to 256,
// within [512, 8192].
std::vector<uint32_t> build_row_blocks(const int32_t* row_ptr, int64_t n_rows, int rows_per_block, int long_row,
                                       int* tile_out) {
  const int64_t nnz = n_rows ? row_ptr[n_rows] : 0;
  const double nnzr = n_rows ? (double)nnz / (double)n_rows : 0.0;
  int64_t tile = (int64_t)std::ceil(1.25 * rows_per_block * std::min(nnzr, (double)long_row));
  tile = (tile + 255) / 256 * 256;
  tile = std::max<int64_t>(512, std::min<int64_t>(8192, tile));
  *tile_out = (int)tile;
  std::vector<uint32_t> blk;
  blk.reserve((size_t)(n_rows / rows_per_block + 16));
  int64_t r = 0;
  while (r < n_rows) {
    const int64_t len = row_ptr[r + 1] - row_ptr[r];
    if (len > long_row) {
      int64_t e = r;
      while (e < n_rows && e - r < kWarpRowsPerBlock && row_ptr[e + 1] - row_ptr[e] > long_row) ++e;
      blk.push_back((uint32_t)r | kBlockWarpFlag);
      r = e;
    } else {
      int64_t e = r;
      while (e < n_rows && e - r < rows_per_block) {
        const int64_t l = row_ptr[e + 1] - row_ptr[e];
        if (l > long_row || row_ptr[e + 1] - row_ptr[r] > tile) break;
        ++e;
      }
      blk.push_back((uint32_t)r);
      r = e;
    }
  }
  blk.push_back((uint32_t)n_rows);
  return blk;
}

// SELL-C-sigma: stable descending sort of row lengths inside windows of sigma
// rows, chunks of C sorted rows padded to the chunk's longest row, column-major
// inside a chunk, padding val = +0.0 with the row's last column (0 for empty
// and padding rows).
void build_sell(const HostCsr& A, int64_t C, int64_t sigma, SellHost* out) {
  const int64_t n = A.n_rows;
  const int32_t* rp = A.row_ptr.data();
  if (sigma < 1) sigma = 1;
  out->C = C;
  out->sigma = sigma;
  out->perm.resize((size_t)n);
  std::iota(out->perm.begin(), out->perm.end(), 0);
  auto len = [&](int32_t r) { return rp[r + 1] - rp[r]; };
  if (sigma > 1) {
    for (int64_t w0 = 0; w0 < n; w0 += sigma) {
      const int64_t w1 = std::min(n, w0 + sigma);
      std::stable_sort(out->perm.begin() + w0, out->perm.begin() + w1,
                       [&](int32_t a, int32_t b) { return len(a) > len(b); });
    }
  }
  const int64_t nc = (n + C - 1) / C;
  out->n_chunks = nc;
  out->chunk_len.assign((size_t)nc, 0);
  out->chunk_ptr.assign((size_t)nc + 1, 0);
  for (int64_t c = 0; c < nc; ++c) {
    int32_t mx = 0;
    for (int64_t t = 0; t < C && c * C + t < n; ++t) mx = std::max(mx, len(out->perm[c * C + t]));
    out->chunk_len[c] = mx;
    out->chunk_ptr[c + 1] = out->chunk_ptr[c] + C * mx;
  }
  out->slots = out->chunk_ptr[nc];
  out->col.assign((size_t)out->slots, 0);
  out->val.assign((size_t)out->slots, 0.0);
  for (int64_t c = 0; c < nc; ++c) {
    const int64_t base = out->chunk_ptr[c], L = out->chunk_len[c];
    for (int64_t t = 0; t < C; ++t) {
      const int64_t r = c * C + t;
      if (r >= n) break;  // padding rows keep col 0, val +0.0
      const int32_t o = out->perm[r];
      const int64_t s = rp[o], ln = rp[o + 1] - rp[o];
      int32_t last = 0;
      for (int64_t j = 0; j < L; ++j) {
        const int64_t slot = base + j * C + t;
        if (j < ln) {
          last = A.col[s + j];
          out->col[slot] = last;
          out->val[slot] = A.val[s + j];
        } else {
          out->col[slot] = last;
        }
      }
    }
  }
}

// Fraction of the stored entries of a sample of rows that consecutive rows
// gather at scattered addresses: entry (i, c) counts as regular when row i-1
// holds column c-1 or row i+1 holds column c+1 (a stencil or a band moves by
// one column per row, so a warp of consecutive rows reads consecutive B
// entries), and as scattered otherwise.  At most about 4096 rows, evenly
// spaced, so that the result is deterministic and cheap on any matrix.
double scattered_fraction(const int32_t* rp, const int32_t* col, int64_t n_rows) {
  if (n_rows < 3) return 0.0;
  const int64_t step = std::max<int64_t>(1, (n_rows - 2) / 4096);
  std::vector<int32_t> prev, next;
  int64_t total = 0, scattered = 0;
  for (int64_t i = 1; i + 1 < n_rows; i += step) {
    prev.assign(col + rp[i - 1], col + rp[i]);
    next.assign(col + rp[i + 1], col + rp[i + 2]);
    std::sort(prev.begin(), prev.end());
    std::sort(next.begin(), next.end());
    for (int32_t j = rp[i]; j < rp[i + 1]; ++j) {
      const int32_t c = col[j];
      const bool reg = std::binary_search(prev.begin(), prev.end(), c - 1) ||
                       std::binary_search(next.begin(), next.end(), c + 1);
      ++total;
      if (!reg) ++scattered;
    }
  }
  return total ? (double)scattered / (double)total : 0.0;
}

// Fill of SELL-32-sigma (nonzeros over stored slots) from the row lengths
// alone: rows sorted by descending length inside sigma-windows, 32 per chunk,
// a chunk as long as its longest row.  1.0 for an empty matrix.
double sell_fill(const int32_t* rp, int64_t n_rows, int64_t sigma) {
  if (sigma < 1) sigma = 1;
  std::vector<int32_t> len;
  int64_t slots = 0;
  for (int64_t w0 = 0; w0 < n_rows; w0 += sigma) {
    const int64_t w1 = std::min(n_rows, w0 + sigma);
    len.resize((size_t)(w1 - w0));
    for (int64_t r = w0; r < w1; ++r) len[(size_t)(r - w0)] = rp[r + 1] - rp[r];
    if (sigma > 1) std::sort(len.begin(), len.end(), std::greater<int32_t>());
    for (size_t c = 0; c < len.size(); c += kSellC) {
      int32_t mx = 0;
      for (size_t t = c; t < std::min(len.size(), c + kSellC); ++t) mx = std::max(mx, len[t]);
      slots += (int64_t)kSellC * mx;
    }
  }
  const int64_t nnz = rp[n_rows];
  return slots ? (double)nnz / (double)slots : 1.0;
}

// Local/halo split at column h (Sec. 3.1): local = entries with col < h over all
// rows, halo = entries with col >= h over the ascending list of rows that have
// any; in-row order kept, global column indices.
void build_split(const HostCsr& A, int64_t h, SplitHost* out) {
  const int64_t n = A.n_rows;
  out->h = h;
  out->loc_row_ptr.assign((size_t)n + 1, 0);
  out->halo_rows.clear();
  out->halo_row_ptr.assign(1, 0);
  out->loc_col.clear();
  out->loc_val.clear();
  out->halo_col.clear();
  out->halo_val.clear();
  for (int64_t i = 0; i < n; ++i) {
    const size_t before = out->halo_col.size();
    for (int64_t j = A.row_ptr[i]; j < A.row_ptr[i + 1]; ++j) {
      if (A.col[j] < h) {
        out->loc_col.push_back(A.col[j]);
        out->loc_val.push_back(A.val[j]);
      } else {
        out->halo_col.push_back(A.col[j]);
        out->halo_val.push_back(A.val[j]);
      }
    }
    out->loc_row_ptr[i + 1] = (int32_t)out->loc_col.size();
    if (out->halo_col.size() > before) {
      out->halo_rows.push_back((int32_t)i);
      out->halo_row_ptr.push_back((int32_t)out->halo_col.size());
    }
  }
}

// ------------------------------------------------------- symmetric CRS (Sec. 1.3.1)
// Symmetry test in O(nnz): the strictly-lower entries are transposed into a
// CRS by a stable counting sort (row j of the transpose lists (i, v) for every
// stored (i, j) with j < i, in ascending i), then each row's strictly-upper
// entries are compared with that row of the transpose: directly when they come
// in the same order (sorted columns), else after sorting both by (column,
// value key).  Values compare by bit pattern with -0.0 mapped to +0.0.
static uint64_t sym_value_key(double v) {
  if (v == 0.0) v = 0.0;
  uint64_t b;
  std::memcpy(&b, &v, sizeof(b));
  return b;
}

bool build_sym(const HostCsr& A, SymHost* out, std::string* why) {
  const int64_t n = A.n_rows;
  if (A.n_cols != n) {
    *why = "symmetric CRS needs a square matrix";
    return false;
  }
  const int32_t* rp = A.row_ptr.data();
  const int32_t* col = A.col.data();
  const double* val = A.val.data();
  std::vector<int64_t> lt_ptr(n + 1, 0);
  int64_t n_upper = 0, n_diag = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = rp[i]; j < rp[i + 1]; ++j) {
      if (col[j] < i) ++lt_ptr[col[j] + 1];
      else if (col[j] > i) ++n_upper;
      else ++n_diag;
    }
  for (int64_t r = 0; r < n; ++r) lt_ptr[r + 1] += lt_ptr[r];
  if (lt_ptr[n] != n_upper) {
    *why = "matrix is not symmetric: " + std::to_string(n_upper) + " entries above the diagonal, " +
           std::to_string(lt_ptr[n]) + " below";
    return false;
  }
  std::vector<int32_t> lt_col((size_t)n_upper);
  std::vector<uint64_t> lt_key((size_t)n_upper);
  {
    std::vector<int64_t> fill(lt_ptr.begin(), lt_ptr.end() - 1);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = rp[i]; j < rp[i + 1]; ++j)
        if (col[j] < i) {
          const int64_t q = fill[col[j]]++;
          lt_col[q] = (int32_t)i;
          lt_key[q] = sym_value_key(val[j]);
        }
  }
  std::vector<std::pair<int32_t, uint64_t>> a, b;
  for (int64_t i = 0; i < n; ++i) {
    int64_t q = lt_ptr[i], cnt = 0;
    bool in_order = true;
    for (int64_t j = rp[i]; j < rp[i + 1]; ++j) {
      if (col[j] <= i) continue;
      ++cnt;
      if (in_order && (q >= lt_ptr[i + 1] || lt_col[q] != col[j] || lt_key[q] != sym_value_key(val[j])))
        in_order = false;
      ++q;
    }
    if (cnt != lt_ptr[i + 1] - lt_ptr[i]) {
      *why = "matrix is not symmetric: row " + std::to_string(i) + " has " + std::to_string(cnt) +
             " entries above the diagonal, column " + std::to_string(i) + " has " +
             std::to_string(lt_ptr[i + 1] - lt_ptr[i]) + " below";
      return false;
    }
    if (in_order) continue;
    a.clear();
    b.clear();
    for (int64_t j = rp[i]; j < rp[i + 1]; ++j)
      if (col[j] > i) a.emplace_back(col[j], sym_value_key(val[j]));
    for (int64_t t = lt_ptr[i]; t < lt_ptr[i + 1]; ++t) b.emplace_back(lt_col[t], lt_key[t]);
    std::sort(a.begin(), a.end());
    std::sort(b.begin(), b.end());
    if (a != b) {
      *why = "matrix is not symmetric: the entries above the diagonal in row " + std::to_string(i) +
             " do not mirror those below it in column " + std::to_string(i);
      return false;
    }
  }
  out->row_ptr.assign(n + 1, 0);
  out->col.resize((size_t)(n_upper + n_diag));
  out->val.resize((size_t)(n_upper + n_diag));
  int64_t p = 0;
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = rp[i]; j < rp[i + 1]; ++j)
      if (col[j] >= i) {
        out->col[p] = col[j];
        out->val[p++] = val[j];
      }
    out->row_ptr[i + 1] = (int32_t)p;
  }
  return true;
}


// Feature vector of the cost model (34 entries); definition in the header of
// spmv_features in include/spmv.h.
void compute_features(int64_t n, int64_t n_cols, const int32_t* rp, const int32_t* col, int k, double* f) {
  constexpr int NB = 13;
  std::memset(f, 0, sizeof(double) * 34);
  const int64_t nnz = n ? rp[n] : 0;
  int64_t cnt[NB] = {0}, ent[NB] = {0};
  int64_t maxlen = 0, bw = 0, span_sum = 0, nonempty = 0;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t L = rp[i + 1] - rp[i];
    int b = 0;
    if (L > 0) {
      b = 64 - __builtin_clzll((unsigned long long)L);  // bit length = 1 + floor(log2 L)
      if (b > NB - 1) b = NB - 1;
    }
    cnt[b] += 1;
    ent[b] += L;
    maxlen = std::max(maxlen, L);
    if (L > 0) {
      int32_t lo = col[rp[i]], hi = col[rp[i]];
      for (int64_t j = rp[i]; j < rp[i + 1]; ++j) {
        lo = std::min(lo, col[j]);
        hi = std::max(hi, col[j]);
        bw = std::max<int64_t>(bw, std::llabs((long long)i - (long long)col[j]));
      }
      span_sum += hi - lo;
      nonempty += 1;
    }
  }
  if (n > 0) {
    for (int b = 0; b < NB; ++b) {
      f[b] = (double)cnt[b] / (double)n;
      f[NB + b] = nnz > 0 ? (double)ent[b] / (double)nnz : 0.0;
    }
  }
  f[26] = std::log2(1.0 + (double)n);
  f[27] = std::log2(1.0 + (double)nnz);
  const double mean = n > 0 ? (double)nnz / (double)n : 0.0;
  f[28] = mean;
  f[29] = std::log2(1.0 + (double)maxlen);
  if (n > 0) {
    double ss = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      const double d = (double)(rp[i + 1] - rp[i]) - mean;
      ss += d * d;
    }
    f[30] = std::sqrt(ss / (double)n) / (1.0 + mean);
  }
  const double denom = (double)std::max<int64_t>(1, n_cols);
  if (nnz > 0) {
    f[31] = (double)bw / denom;
    f[32] = (double)span_sum / ((double)nonempty * denom);
  }
  f[33] = std::log2((double)k);
}

}  // namespace spmv
