/*
 * CPU node baseline: the CRS loop of Sec. 1.2 parallelised over rows with an
 * OpenMP static schedule, as in the paper's node-level runs (Sec. 2).  It is a
 * timing comparison for bench.py, not part of the library and not the oracle
 * (which stays single-threaded).  Compiled with -ffp-contract=off: every row
 * is summed in the same order and rounding as the oracle's loop.
 */
#include <stdint.h>
#include <omp.h>

void crs_omp_spmv(int64_t n_rows, const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                  const double* B, double* C) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_rows; ++i) {
    double s = 0.0;
    for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j) {
      double prod = val[j] * B[col_idx[j]];
      s = s + prod;
    }
    C[i] = s;
  }
}

int crs_omp_threads(void) { return omp_get_max_threads(); }
