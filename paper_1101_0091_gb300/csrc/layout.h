// Layout shared by the kernels and the host code: device status codes, the
// bounded-wait limit, launch constants and the device views of the formats.
#pragma once

#include <stdint.h>

namespace spmv {

// Device status word codes written by kernels (0 = fine).
enum : int { DEV_OK = 0, DEV_WAIT_TIMEOUT = 1 };

// Bounded device waits give up after this many nanoseconds of %globaltimer.
constexpr unsigned long long kWaitLimitNs = 1000000000ull;

// ------------------------------------------------------- layout constants
constexpr int kThreads = 256;        // threads per CTA of the row kernels
constexpr int kStagedRows = 256;     // rows per CRS_STAGED block (one per thread)
constexpr int kLongRow = 64;         // rows longer than this are handled warp-per-row
constexpr int kWarpRowsPerBlock = kThreads / 32;
constexpr int kSellC = 32;           // SELL chunk height
constexpr uint32_t kBlockWarpFlag = 0x80000000u;  // high bit of a row-block entry: warp-per-row block

// Device view of one CRS matrix (values in FP64 and, optionally, FP32).
struct CsrDev {
  int64_t n_rows = 0, n_cols = 0, nnz = 0;
  const int32_t* row_ptr = nullptr;
  const int32_t* col = nullptr;     // padded to a multiple of 4 entries + 4
  const double* val = nullptr;      // padded to a multiple of 2 entries + 2
  const float* val32 = nullptr;     // padded to a multiple of 4 entries + 4
  const uint32_t* blk = nullptr;    // row blocks of CRS_STAGED (n_blk + 1 entries)
  int64_t n_blk = 0;
  int tile = 0;                     // nonzero capacity of a CRS_STAGED tile
  int prefetch = 0;                 // CTAs ahead whose val/col slices are prefetched into L2 (0 = off)
  bool val32_special = false;       // val32 holds a subnormal, infinite or NaN float
};

struct SellDev {
  int64_t n_rows = 0, n_chunks = 0, slots = 0;
  int sigma = 0;
  const int32_t* perm = nullptr;
  const int64_t* chunk_ptr = nullptr;
  const int32_t* chunk_len = nullptr;
  const int32_t* col = nullptr;
  const double* val = nullptr;
  const float* val32 = nullptr;
  int prefetch = 0;                 // CTAs ahead whose slots are prefetched into L2 (0 = off)
  bool val32_special = false;
};

// Stored triangle of SPMV_SYM.
struct SymDev {
  int64_t n_rows = 0, nnz = 0;
  const int32_t* row_ptr = nullptr;
  const int32_t* col = nullptr;     // padded like CsrDev::col
  const double* val = nullptr;
  const float* val32 = nullptr;
  int prefetch = 0;
  bool val32_special = false;
};

// Halo part of a split: rows listed in `rows`, CRS over them.
struct HaloDev {
  int64_t n_rows = 0, nnz = 0;
  const int32_t* rows = nullptr;
  const int32_t* row_ptr = nullptr;
  const int32_t* col = nullptr;
  const double* val = nullptr;
  const float* val32 = nullptr;
  bool val32_special = false;
};

}  // namespace spmv
