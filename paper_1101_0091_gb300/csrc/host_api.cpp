// Host-side format builders of the C ABI: the SELL-C-sigma, local/halo split
// and symmetric-triangle builders that plan creation and variant changes run,
// callable on host CRS arrays without a device.  Each call validates the CRS
// arrays, builds the format, and copies it out in the two-call pattern: with
// the output arrays NULL only the sizes are returned.
#include <algorithm>
#include <cstring>
#include <new>

#include "internal.h"

namespace {

using namespace spmv;

spmv_status load_host(int64_t n_rows, int64_t n_cols, const int32_t* row_ptr, const int32_t* col_idx,
                      const double* val, HostCsr* A) {
  std::string why;
  if (!validate_csr(n_rows, n_cols, row_ptr, col_idx, &why)) return fail(SPMV_ERR_CSR, why);
  const int64_t nnz = row_ptr[n_rows];
  if (nnz > 0 && !val) return fail(SPMV_ERR_ARG, "val is NULL");
  A->n_rows = n_rows;
  A->n_cols = n_cols;
  A->nnz = nnz;
  A->row_ptr.assign(row_ptr, row_ptr + n_rows + 1);
  A->col.assign(col_idx, col_idx + nnz);
  A->val.assign(val, val + nnz);
  return SPMV_OK;
}

template <typename T>
void copy_out(T* dst, const std::vector<T>& src) {
  if (dst && !src.empty()) std::memcpy(dst, src.data(), sizeof(T) * src.size());
}

}  // namespace

extern "C" {

spmv_status spmv_sell_build_host(int64_t n_rows, int64_t n_cols, const int32_t* row_ptr, const int32_t* col_idx,
                                 const double* val, int32_t sigma, int64_t* n_chunks, int64_t* n_slots,
                                 int32_t* perm, int64_t* chunk_ptr, int32_t* chunk_len, int32_t* sell_col,
                                 double* sell_val) {
  if (!n_chunks || !n_slots) return fail(SPMV_ERR_ARG, "n_chunks or n_slots is NULL");
  if (sigma < 1) return fail(SPMV_ERR_ARG, "sigma must be >= 1");
  try {
    HostCsr A;
    spmv_status st = load_host(n_rows, n_cols, row_ptr, col_idx, val, &A);
    if (st != SPMV_OK) return st;
    SellHost S;
    build_sell(A, kSellC, sigma, &S);
    *n_chunks = S.n_chunks;
    *n_slots = S.slots;
    if (!perm) return SPMV_OK;
    if (!chunk_ptr || !chunk_len || (S.slots > 0 && (!sell_col || !sell_val)))
      return fail(SPMV_ERR_ARG, "NULL output array");
    copy_out(perm, S.perm);
    copy_out(chunk_ptr, S.chunk_ptr);
    copy_out(chunk_len, S.chunk_len);
    copy_out(sell_col, S.col);
    copy_out(sell_val, S.val);
  } catch (const std::bad_alloc&) {
    return fail(SPMV_ERR_OOM, "host allocation failed");
  }
  return SPMV_OK;
}

spmv_status spmv_split_build_host(int64_t n_rows, int64_t n_cols, const int32_t* row_ptr, const int32_t* col_idx,
                                  const double* val, int64_t h, int64_t* loc_nnz, int64_t* n_halo_rows,
                                  int64_t* halo_nnz, int32_t* loc_row_ptr, int32_t* loc_col, double* loc_val,
                                  int32_t* halo_rows, int32_t* halo_row_ptr, int32_t* halo_col,
                                  double* halo_val) {
  if (!loc_nnz || !n_halo_rows || !halo_nnz) return fail(SPMV_ERR_ARG, "size output is NULL");
  if (h < 0 || h > n_cols) return fail(SPMV_ERR_ARG, "h must be in 0..n_cols");
  try {
    HostCsr A;
    spmv_status st = load_host(n_rows, n_cols, row_ptr, col_idx, val, &A);
    if (st != SPMV_OK) return st;
    SplitHost S;
    build_split(A, h, &S);
    *loc_nnz = (int64_t)S.loc_col.size();
    *n_halo_rows = (int64_t)S.halo_rows.size();
    *halo_nnz = (int64_t)S.halo_col.size();
    if (!loc_row_ptr) return SPMV_OK;
    if (!halo_row_ptr || (*loc_nnz > 0 && (!loc_col || !loc_val)) || (*n_halo_rows > 0 && !halo_rows) ||
        (*halo_nnz > 0 && (!halo_col || !halo_val)))
      return fail(SPMV_ERR_ARG, "NULL output array");
    copy_out(loc_row_ptr, S.loc_row_ptr);
    copy_out(loc_col, S.loc_col);
    copy_out(loc_val, S.loc_val);
    copy_out(halo_rows, S.halo_rows);
    copy_out(halo_row_ptr, S.halo_row_ptr);
    copy_out(halo_col, S.halo_col);
    copy_out(halo_val, S.halo_val);
  } catch (const std::bad_alloc&) {
    return fail(SPMV_ERR_OOM, "host allocation failed");
  }
  return SPMV_OK;
}

spmv_status spmv_sym_build_host(int64_t n_rows, int64_t n_cols, const int32_t* row_ptr, const int32_t* col_idx,
                                const double* val, int64_t* sym_nnz, int32_t* sym_row_ptr, int32_t* sym_col,
                                double* sym_val) {
  if (!sym_nnz) return fail(SPMV_ERR_ARG, "sym_nnz is NULL");
  try {
    HostCsr A;
    spmv_status st = load_host(n_rows, n_cols, row_ptr, col_idx, val, &A);
    if (st != SPMV_OK) return st;
    SymHost S;
    std::string why;
    if (!build_sym(A, &S, &why)) return fail(SPMV_ERR_UNSUPPORTED, "SYM: " + why);
    *sym_nnz = (int64_t)S.col.size();
    if (!sym_row_ptr) return SPMV_OK;
    if (*sym_nnz > 0 && (!sym_col || !sym_val)) return fail(SPMV_ERR_ARG, "NULL output array");
    copy_out(sym_row_ptr, S.row_ptr);
    copy_out(sym_col, S.col);
    copy_out(sym_val, S.val);
  } catch (const std::bad_alloc&) {
    return fail(SPMV_ERR_OOM, "host allocation failed");
  }
  return SPMV_OK;
}

}  // extern "C"
