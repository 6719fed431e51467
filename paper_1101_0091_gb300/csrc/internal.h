// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/spmv.h"
#include "layout.h"

namespace spmv {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
spmv_status fail(spmv_status st, const std::string& msg);
spmv_status cuda_fail(cudaError_t e, const char* what);

#define SPMV_CUDA(call)                                                   \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess) return ::spmv::cuda_fail(e_, #call);           \
  } while (0)

// ------------------------------------------------------- host copies of the formats
struct HostCsr {
  int64_t n_rows = 0, n_cols = 0, nnz = 0;
  std::vector<int32_t> row_ptr, col;
  std::vector<double> val;
};

struct SellHost {
  int64_t C = kSellC, sigma = 1, n_chunks = 0, slots = 0;
  std::vector<int32_t> perm, chunk_len, col;
  std::vector<int64_t> chunk_ptr;
  std::vector<double> val;
};

// Symmetric CRS (Sec. 1.3.1): the entries of each row with col >= row, in their order in the row.
struct SymHost {
  std::vector<int32_t> row_ptr, col;
  std::vector<double> val;
};

struct SplitHost {
  int64_t h = -1;
  std::vector<int32_t> loc_row_ptr, loc_col, halo_rows, halo_row_ptr, halo_col;
  std::vector<double> loc_val, halo_val;
};

// True if any float is subnormal, infinite or NaN (zero and normals are "plain").
bool has_special_f32(const float* v, int64_t n);

// ------------------------------------------------------- plan accessors
const CsrDev* plan_csr(spmv_handle h);              // device view of the whole matrix
const int32_t* plan_host_row_ptr(spmv_handle h);    // host copy of row_ptr
const int32_t* plan_host_col(spmv_handle h);        // host copy of col_idx
const double* plan_host_val(spmv_handle h);         // host copy of val
int plan_device(spmv_handle h);
int plan_max_k(spmv_handle h);                     // largest k accepted by spmv_apply_block
// Changes whenever the plan's kernel, its device arrays or its launch parameters change (work
// captured into a CUDA graph through the plan must be captured again).
uint64_t plan_generation(spmv_handle h);

// ------------------------------------------------------- host builders
bool validate_csr(int64_t n_rows, int64_t n_cols, const int32_t* row_ptr, const int32_t* col,
                  std::string* why);
std::vector<uint32_t> build_row_blocks(const int32_t* row_ptr, int64_t n_rows, int rows_per_block,
                                       int long_row, int* tile_out);
void build_sell(const HostCsr& A, int64_t C, int64_t sigma, SellHost* out);
void build_split(const HostCsr& A, int64_t h, SplitHost* out);
// False (reason in *why) unless A is square and symmetric in the sense of spmv_set_variant.
bool build_sym(const HostCsr& A, SymHost* out, std::string* why);
// Reverse Cuthill-McKee permutation (perm[new] = old) of a square pattern.
bool rcm_permutation(int64_t n, const int32_t* row_ptr, const int32_t* col, int32_t* perm);
// True if perm is a permutation of 0..n-1; fills inv (inv[old] = new).
bool validate_permutation(int64_t n, const int32_t* perm, std::vector<int32_t>* inv, std::string* why);
// A' = P A P^T: row r of A' is row perm[r] of A, columns relabelled by inv and sorted (stable).
void permute_csr(int64_t n, const int32_t* row_ptr, const int32_t* col, const double* val, const int32_t* perm,
                 const std::vector<int32_t>& inv, int32_t* out_row_ptr, int32_t* out_col, double* out_val);
// Default L2 prefetch distance of the row and SELL kernels, in CTAs ahead:
// three per SM.  280^3 Poisson product, CRS_L1: 0 / 76 / 152 / 228 / 304 /
// 456 / 608 CTAs ahead gave 871 / 917 / 926 / 930 / 933 / 933.5 / 933.7
// GFlop/s.
constexpr int kDefaultPrefetch = 456;

// AUTO: a matrix whose sampled entries are scattered beyond this share (see
// scattered_fraction) runs without the L2 prefetch, and runs SELL-32-256 when
// that format stores at least kAutoSellFill nonzeros per slot.
constexpr double kAutoScattered = 0.3;
constexpr double kAutoSellFill = 0.85;

// Share of a row sample's entries gathered at scattered addresses by consecutive rows (see host.cpp).
double scattered_fraction(const int32_t* row_ptr, const int32_t* col, int64_t n_rows);
// Nonzeros over stored slots of SELL-32-sigma, from the row lengths.
double sell_fill(const int32_t* row_ptr, int64_t n_rows, int64_t sigma);
void compute_features(int64_t n_rows, int64_t n_cols, const int32_t* row_ptr, const int32_t* col,
                      int k, double* f);

// ------------------------------------------------------- kernel launchers
// All launchers enqueue on `stream` and return the launch error (if any).
cudaError_t launch_crs_staged(const CsrDev& A, bool fp32, const double* B, int64_t ldb, double* C,
                              int64_t ldc, int k, bool accumulate, int* status, cudaStream_t s);
cudaError_t launch_crs_lanes(const CsrDev& A, bool fp32, int lanes, const double* B, int64_t ldb,
                             double* C, int64_t ldc, int k, cudaStream_t s);
cudaError_t launch_sell(const SellDev& S, bool fp32, const double* B, int64_t ldb, double* C,
                        int64_t ldc, int k, cudaStream_t s);
cudaError_t launch_halo(const HaloDev& H, bool fp32, const double* B, int64_t ldb, double* C,
                        int64_t ldc, int k, cudaStream_t s);
// Zeroes C[:, 0:k] on the stream, then runs the symmetric kernel.
cudaError_t launch_sym(const SymDev& S, bool fp32, const double* B, int64_t ldb, double* C, int64_t ldc,
                       int k, cudaStream_t s);

}  // namespace spmv
