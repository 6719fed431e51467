// C ABI of the library: plan lifecycle, the apply calls, variant switching and
// the export of built index structures.  See include/spmv.h for the contract.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>

#include "internal.h"

namespace spmv {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

spmv_status fail(spmv_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

spmv_status cuda_fail(cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return fail(SPMV_ERR_OOM, m);
  return fail(SPMV_ERR_CUDA, m);
}

// Device allocation list owned by a plan; everything is freed together.
struct DevArena {
  std::vector<void*> ptrs;
  int64_t bytes = 0;
  cudaError_t alloc(void** p, size_t n) {
    *p = nullptr;
    cudaError_t e = cudaMalloc(p, std::max<size_t>(n, 256));
    if (e == cudaSuccess) {
      ptrs.push_back(*p);
      bytes += (int64_t)std::max<size_t>(n, 256);
    }
    return e;
  }
  void release(void* p) {
    auto it = std::find(ptrs.begin(), ptrs.end(), p);
    if (it != ptrs.end()) {
      cudaFree(p);
      ptrs.erase(it);
    }
  }
  void free_all() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
    bytes = 0;
  }
};

// Upload n elements, padding the allocation by `pad` zero elements.
template <typename T>
static cudaError_t upload(DevArena& a, T** dst, const T* src, int64_t n, int64_t pad) {
  void* p;
  const size_t bytes = sizeof(T) * (size_t)(n + pad);
  cudaError_t e = a.alloc(&p, bytes);
  if (e != cudaSuccess) return e;
  e = cudaMemset(p, 0, bytes);
  if (e == cudaSuccess && n > 0) e = cudaMemcpy(p, src, sizeof(T) * (size_t)n, cudaMemcpyHostToDevice);
  *dst = static_cast<T*>(p);
  return e;
}

static int64_t pad_to(int64_t n, int64_t m) { return (m - n % m) % m + m; }

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace spmv

using namespace spmv;

struct spmv_plan {
  int device = 0;
  uint64_t generation = 0;  // bumped whenever the kernel, its arrays or its launch parameters change
  spmv_options opt{};
  int variant = SPMV_CRS_STAGED;
  // what AUTO runs: SELL-32-256 on matrices whose rows gather at scattered
  // addresses (and pack well into SELL), CRS_L1 otherwise
  double scattered = 0.0;
  double fill256 = 1.0;
  bool auto_sell = false;
  HostCsr host;
  DevArena arena;
  CsrDev A;            // the whole matrix
  bool blocks_built = false;
  // SELL
  SellHost sell_host;
  SellDev sell;
  std::vector<void*> sell_ptrs;
  // symmetric CRS triangle
  SymDev sym;
  // split
  bool has_split = false;
  SplitHost split_host;
  CsrDev local;        // local part (row blocks built for CRS_STAGED)
  HaloDev halo;
  cudaEvent_t ev_main = nullptr, ev_copy = nullptr;
  // status word and end-to-end scratch
  int* status = nullptr;
  double* d_B = nullptr;
  double* d_C = nullptr;
  int64_t scratch_k = 0;
  spmv_tuning tuning{};
  // pipelined host steps: two device buffer sets, copy-in / copy-out streams
  struct Pipe {
    double* B[2] = {nullptr, nullptr};
    double* C[2] = {nullptr, nullptr};
    int64_t k = 0;
    cudaStream_t in = nullptr, out = nullptr;
    cudaEvent_t in_done[2] = {nullptr, nullptr}, kern_done[2] = {nullptr, nullptr}, out_done[2] = {nullptr, nullptr};
    int64_t step = 0;
  } pipe;
};

static void free_pipe(spmv_plan* p) {
  auto& q = p->pipe;
  for (int s = 0; s < 2; ++s) {
    if (q.in_done[s]) cudaEventDestroy(q.in_done[s]);
    if (q.kern_done[s]) cudaEventDestroy(q.kern_done[s]);
    if (q.out_done[s]) cudaEventDestroy(q.out_done[s]);
  }
  if (q.in) cudaStreamDestroy(q.in);
  if (q.out) cudaStreamDestroy(q.out);
  q = spmv_plan::Pipe{};
}

static void apply_tuning(spmv_plan* p) {
  p->A.prefetch = p->tuning.prefetch_distance;
  p->local.prefetch = p->tuning.prefetch_distance;
  p->sell.prefetch = p->tuning.prefetch_distance;
  p->sym.prefetch = p->tuning.prefetch_distance;
}

namespace spmv {
const CsrDev* plan_csr(spmv_handle h) { return &h->A; }
const int32_t* plan_host_row_ptr(spmv_handle h) { return h->host.row_ptr.data(); }
const int32_t* plan_host_col(spmv_handle h) { return h->host.col.data(); }
const double* plan_host_val(spmv_handle h) { return h->host.val.data(); }
int plan_device(spmv_handle h) { return h->device; }
int plan_max_k(spmv_handle h) { return h->opt.max_k; }
uint64_t plan_generation(spmv_handle h) { return h->generation; }
}  // namespace spmv

static spmv_status build_blocks(spmv_plan* p, CsrDev* M, const int32_t* host_row_ptr) {
  int tile = 0;
  std::vector<uint32_t> blk = build_row_blocks(host_row_ptr, M->n_rows, kStagedRows, kLongRow, &tile);
  uint32_t* d = nullptr;
  SPMV_CUDA(upload(p->arena, &d, blk.data(), (int64_t)blk.size(), 0));
  M->blk = d;
  M->n_blk = (int64_t)blk.size() - 1;
  M->tile = tile;
  return SPMV_OK;
}

static spmv_status build_sell_dev(spmv_plan* p, int sigma) {
  if (sigma < 1) sigma = 1;
  if (p->sell.perm && p->sell.sigma == sigma) return SPMV_OK;
  for (void* q : p->sell_ptrs) p->arena.release(q);
  p->sell_ptrs.clear();
  p->sell = SellDev{};
  build_sell(p->host, kSellC, sigma, &p->sell_host);
  const SellHost& S = p->sell_host;
  int32_t *perm, *clen, *col;
  int64_t* cptr;
  double* val;
  SPMV_CUDA(upload(p->arena, &perm, S.perm.data(), (int64_t)S.perm.size(), 0));
  p->sell_ptrs.push_back(perm);
  SPMV_CUDA(upload(p->arena, &cptr, S.chunk_ptr.data(), (int64_t)S.chunk_ptr.size(), 0));
  p->sell_ptrs.push_back(cptr);
  SPMV_CUDA(upload(p->arena, &clen, S.chunk_len.data(), (int64_t)S.chunk_len.size(), 0));
  p->sell_ptrs.push_back(clen);
  SPMV_CUDA(upload(p->arena, &col, S.col.data(), S.slots, 4));
  p->sell_ptrs.push_back(col);
  SPMV_CUDA(upload(p->arena, &val, S.val.data(), S.slots, 2));
  p->sell_ptrs.push_back(val);
  p->sell.n_rows = p->host.n_rows;
  p->sell.n_chunks = S.n_chunks;
  p->sell.slots = S.slots;
  p->sell.sigma = sigma;
  p->sell.perm = perm;
  p->sell.chunk_ptr = cptr;
  p->sell.chunk_len = clen;
  p->sell.col = col;
  p->sell.val = val;
  p->sell.prefetch = p->tuning.prefetch_distance;
  if (p->opt.val_fp32) {
    std::vector<float> v32(S.val.begin(), S.val.end());
    float* d32;
    SPMV_CUDA(upload(p->arena, &d32, v32.data(), S.slots, 4));
    p->sell_ptrs.push_back(d32);
    p->sell.val32 = d32;
    p->sell.val32_special = has_special_f32(v32.data(), S.slots);
  }
  std::vector<double>().swap(p->sell_host.val);  // values live on the device; keep the index arrays
  return SPMV_OK;
}

static spmv_status upload_csr(spmv_plan* p, CsrDev* M, int64_t n_rows, int64_t n_cols, const int32_t* rp,
                              const int32_t* col, const double* val, int64_t nnz) {
  int32_t *drp, *dcol;
  double* dval;
  SPMV_CUDA(upload(p->arena, &drp, rp, n_rows + 1, 0));
  SPMV_CUDA(upload(p->arena, &dcol, col, nnz, pad_to(nnz, 4)));
  SPMV_CUDA(upload(p->arena, &dval, val, nnz, pad_to(nnz, 2)));
  M->n_rows = n_rows;
  M->n_cols = n_cols;
  M->nnz = nnz;
  M->row_ptr = drp;
  M->col = dcol;
  M->val = dval;
  if (p->opt.val_fp32) {
    std::vector<float> v32(val, val + nnz);  // round to nearest even
    float* d32;
    SPMV_CUDA(upload(p->arena, &d32, v32.data(), nnz, pad_to(nnz, 4)));
    M->val32 = d32;
    M->val32_special = has_special_f32(v32.data(), nnz);
  }
  return SPMV_OK;
}

static spmv_status build_split_dev(spmv_plan* p, int64_t h) {
  build_split(p->host, h, &p->split_host);
  const SplitHost& S = p->split_host;
  spmv_status st = upload_csr(p, &p->local, p->host.n_rows, p->host.n_cols, S.loc_row_ptr.data(),
                              S.loc_col.data(), S.loc_val.data(), (int64_t)S.loc_col.size());
  if (st != SPMV_OK) return st;
  st = build_blocks(p, &p->local, S.loc_row_ptr.data());
  if (st != SPMV_OK) return st;
  CsrDev hc;
  st = upload_csr(p, &hc, (int64_t)S.halo_rows.size(), p->host.n_cols, S.halo_row_ptr.data(), S.halo_col.data(),
                  S.halo_val.data(), (int64_t)S.halo_col.size());
  if (st != SPMV_OK) return st;
  int32_t* rows;
  SPMV_CUDA(upload(p->arena, &rows, S.halo_rows.data(), (int64_t)S.halo_rows.size(), 0));
  p->halo.n_rows = (int64_t)S.halo_rows.size();
  p->halo.nnz = (int64_t)S.halo_col.size();
  p->halo.rows = rows;
  p->halo.row_ptr = hc.row_ptr;
  p->halo.col = hc.col;
  p->halo.val = hc.val;
  p->halo.val32 = hc.val32;
  p->halo.val32_special = hc.val32_special;
  SPMV_CUDA(cudaEventCreateWithFlags(&p->ev_main, cudaEventDisableTiming));
  SPMV_CUDA(cudaEventCreateWithFlags(&p->ev_copy, cudaEventDisableTiming));
  p->has_split = true;
  return SPMV_OK;
}

static spmv_status build_sym_dev(spmv_plan* p) {
  if (p->sym.row_ptr) return SPMV_OK;
  SymHost S;
  std::string why;
  if (!build_sym(p->host, &S, &why)) return fail(SPMV_ERR_UNSUPPORTED, "SYM: " + why);
  const int64_t nnz = (int64_t)S.col.size();
  SymDev d;
  int32_t *drp, *dcol;
  double* dval;
  SPMV_CUDA(upload(p->arena, &drp, S.row_ptr.data(), p->host.n_rows + 1, 0));
  SPMV_CUDA(upload(p->arena, &dcol, S.col.data(), nnz, pad_to(nnz, 4)));
  SPMV_CUDA(upload(p->arena, &dval, S.val.data(), nnz, pad_to(nnz, 2)));
  if (p->opt.val_fp32) {
    std::vector<float> v32(S.val.begin(), S.val.end());  // round to nearest even
    float* d32;
    SPMV_CUDA(upload(p->arena, &d32, v32.data(), nnz, pad_to(nnz, 4)));
    d.val32 = d32;
    d.val32_special = has_special_f32(v32.data(), nnz);
  }
  d.n_rows = p->host.n_rows;
  d.nnz = nnz;
  d.row_ptr = drp;
  d.col = dcol;
  d.val = dval;
  d.prefetch = p->tuning.prefetch_distance;
  p->sym = d;
  return SPMV_OK;
}

static spmv_status prepare_variant(spmv_plan* p, int variant, int sigma) {
  if (variant == SPMV_VARIANT_AUTO) {
    variant = p->auto_sell ? SPMV_SELL : SPMV_CRS_L1;
    sigma = p->auto_sell ? 256 : sigma;
  }
  if (variant < SPMV_CRS_STAGED || variant >= SPMV_N_VARIANTS)
    return fail(SPMV_ERR_ARG, "unknown variant " + std::to_string(variant));
  if (variant == SPMV_CRS_STAGED && !p->blocks_built) {
    spmv_status st = build_blocks(p, &p->A, p->host.row_ptr.data());
    if (st != SPMV_OK) return st;
    p->blocks_built = true;
  }
  if (variant == SPMV_SELL) {
    spmv_status st = build_sell_dev(p, sigma);
    if (st != SPMV_OK) return st;
  }
  if (variant == SPMV_SYM) {
    spmv_status st = build_sym_dev(p);
    if (st != SPMV_OK) return st;
  }
  p->variant = variant;
  ++p->generation;
  return SPMV_OK;
}

static cudaError_t run_variant(spmv_plan* p, const CsrDev& M, int variant, const double* B, int64_t ldb,
                               double* C, int64_t ldc, int k, cudaStream_t s) {
  const bool f32 = p->opt.val_fp32 != 0;
  switch (variant) {
    case SPMV_CRS_STAGED: return launch_crs_staged(M, f32, B, ldb, C, ldc, k, false, p->status, s);
    case SPMV_CRS_L1: return launch_crs_lanes(M, f32, 1, B, ldb, C, ldc, k, s);
    case SPMV_CRS_L2: return launch_crs_lanes(M, f32, 2, B, ldb, C, ldc, k, s);
    case SPMV_CRS_L4: return launch_crs_lanes(M, f32, 4, B, ldb, C, ldc, k, s);
    case SPMV_CRS_L8: return launch_crs_lanes(M, f32, 8, B, ldb, C, ldc, k, s);
    case SPMV_CRS_L16: return launch_crs_lanes(M, f32, 16, B, ldb, C, ldc, k, s);
    case SPMV_CRS_L32: return launch_crs_lanes(M, f32, 32, B, ldb, C, ldc, k, s);
    case SPMV_SELL: return launch_sell(p->sell, f32, B, ldb, C, ldc, k, s);
    case SPMV_SYM: return launch_sym(p->sym, f32, B, ldb, C, ldc, k, s);
    default: return cudaErrorInvalidValue;
  }
}

extern "C" {

spmv_options spmv_default_options(void) {
  spmv_options o;
  std::memset(&o, 0, sizeof(o));
  o.variant = SPMV_VARIANT_AUTO;
  o.sell_sigma = 1;
  o.val_fp32 = 0;
  o.max_k = 16;
  o.split = 0;
  o.halo_begin = 0;
  return o;
}

const char* spmv_last_error(void) { return g_last_error.c_str(); }

spmv_status spmv_create(spmv_handle* out, int64_t n_rows, int64_t n_cols, int64_t nnz, const int32_t* row_ptr,
                        const int32_t* col_idx, const double* val, const spmv_options* opt) {
  if (!out) return fail(SPMV_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (nnz < 0 || nnz > INT32_MAX) return fail(SPMV_ERR_CSR, "nnz outside [0, 2^31-1]");
  std::string why;
  if (!validate_csr(n_rows, n_cols, row_ptr, col_idx, &why)) return fail(SPMV_ERR_CSR, why);
  if (row_ptr[n_rows] != nnz)
    return fail(SPMV_ERR_CSR, "row_ptr[n_rows] = " + std::to_string(row_ptr[n_rows]) + " differs from nnz = " +
                                  std::to_string(nnz));
  if (nnz > 0 && !val) return fail(SPMV_ERR_ARG, "val is NULL");
  spmv_options o = opt ? *opt : spmv_default_options();
  if (o.max_k == 0) o.max_k = 16;
  if (o.sell_sigma < 1) o.sell_sigma = 1;
  if (o.max_k < 1 || o.max_k > 16) return fail(SPMV_ERR_ARG, "max_k must be in 1..16");
  if (o.split != 0 && o.split != 1) return fail(SPMV_ERR_ARG, "split must be 0 or 1");
  if (o.reserved != 0) return fail(SPMV_ERR_ARG, "reserved option field must be 0");
  if (o.split && (o.halo_begin < 0 || o.halo_begin > n_cols)) return fail(SPMV_ERR_ARG, "halo_begin outside [0, n_cols]");
  std::unique_ptr<spmv_plan> p;
  try {
    p.reset(new spmv_plan());
    p->host.n_rows = n_rows;
    p->host.n_cols = n_cols;
    p->host.nnz = nnz;
    p->host.row_ptr.assign(row_ptr, row_ptr + n_rows + 1);
    p->host.col.assign(col_idx, col_idx + nnz);
    p->host.val.assign(val, val + nnz);
  } catch (const std::bad_alloc&) {
    return fail(SPMV_ERR_OOM, "host allocation failed");
  }
  p->opt = o;
  // Scattered gathers are bound by the SM's requests to L2, not by HBM: there
  // the L2 prefetch of the matrix slices ahead only adds requests (SELL-32-256
  // on the eigenproblem-shaped matrix: 306 -> 287 us without it).
  p->scattered = scattered_fraction(p->host.row_ptr.data(), p->host.col.data(), n_rows);
  p->fill256 = sell_fill(p->host.row_ptr.data(), n_rows, 256);
  p->auto_sell = p->scattered > kAutoScattered && p->fill256 >= kAutoSellFill;
  p->tuning.prefetch_distance = p->scattered > kAutoScattered ? 0 : kDefaultPrefetch;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  auto cleanup = [&](spmv_status st) {
    if (p->ev_main) cudaEventDestroy(p->ev_main);
    if (p->ev_copy) cudaEventDestroy(p->ev_copy);
    p->arena.free_all();
    return st;
  };
  spmv_status st = upload_csr(p.get(), &p->A, n_rows, n_cols, p->host.row_ptr.data(), p->host.col.data(),
                              p->host.val.data(), nnz);
  if (st != SPMV_OK) return cleanup(st);
  int* status;
  e = upload(p->arena, &status, (const int*)nullptr, 0, 4);
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "status word"));
  p->status = status;
  if (o.split) {
    st = build_split_dev(p.get(), o.halo_begin);
    if (st != SPMV_OK) return cleanup(st);
  }
  st = prepare_variant(p.get(), o.variant, o.sell_sigma);
  if (st != SPMV_OK) return cleanup(st);
  apply_tuning(p.get());
  *out = p.release();
  return SPMV_OK;
}

spmv_status spmv_destroy(spmv_handle h) {
  if (!h) return SPMV_OK;
  DeviceGuard g(h->device);
  cudaDeviceSynchronize();
  if (h->ev_main) cudaEventDestroy(h->ev_main);
  if (h->ev_copy) cudaEventDestroy(h->ev_copy);
  free_pipe(h);
  h->arena.free_all();
  delete h;
  return SPMV_OK;
}

spmv_status spmv_apply_host_async(spmv_handle h, const double* B_host, int32_t k, double* C_host, void* stream) {
  if (!h) return fail(SPMV_ERR_ARG, "handle is NULL");
  if (k < 1 || k > h->opt.max_k) return fail(SPMV_ERR_ARG, "k out of range 1..max_k");
  if ((!B_host && h->host.n_cols > 0) || (!C_host && h->host.n_rows > 0)) return fail(SPMV_ERR_ARG, "NULL buffer");
  DeviceGuard g(h->device);
  auto& q = h->pipe;
  if (q.k < k) {  // (re)allocate both buffer sets for this k
    if (q.in) {
      SPMV_CUDA(cudaStreamSynchronize(q.in));
      SPMV_CUDA(cudaStreamSynchronize(q.out));
    }
    for (int s = 0; s < 2; ++s) {
      if (q.B[s]) h->arena.release(q.B[s]);
      if (q.C[s]) h->arena.release(q.C[s]);
      q.B[s] = q.C[s] = nullptr;
    }
    q.k = 0;
    for (int s = 0; s < 2; ++s) {
      void *b, *c;
      SPMV_CUDA(h->arena.alloc(&b, sizeof(double) * (size_t)(h->host.n_cols * k)));
      q.B[s] = (double*)b;
      SPMV_CUDA(h->arena.alloc(&c, sizeof(double) * (size_t)(h->host.n_rows * k)));
      q.C[s] = (double*)c;
    }
    q.k = k;
  }
  if (!q.in) {
    SPMV_CUDA(cudaStreamCreateWithFlags(&q.in, cudaStreamNonBlocking));
    SPMV_CUDA(cudaStreamCreateWithFlags(&q.out, cudaStreamNonBlocking));
    for (int s = 0; s < 2; ++s) {
      SPMV_CUDA(cudaEventCreateWithFlags(&q.in_done[s], cudaEventDisableTiming));
      SPMV_CUDA(cudaEventCreateWithFlags(&q.kern_done[s], cudaEventDisableTiming));
      SPMV_CUDA(cudaEventCreateWithFlags(&q.out_done[s], cudaEventDisableTiming));
    }
  }
  const int s = (int)(q.step & 1);
  cudaStream_t cs = (cudaStream_t)stream;
  // copy in once the product two steps back has finished reading this buffer set
  SPMV_CUDA(cudaStreamWaitEvent(q.in, q.kern_done[s], 0));
  SPMV_CUDA(cudaMemcpyAsync(q.B[s], B_host, sizeof(double) * (size_t)(h->host.n_cols * k), cudaMemcpyHostToDevice,
                            q.in));
  SPMV_CUDA(cudaEventRecord(q.in_done[s], q.in));
  // multiply once the operand is in and the result two steps back has been copied out
  SPMV_CUDA(cudaStreamWaitEvent(cs, q.in_done[s], 0));
  SPMV_CUDA(cudaStreamWaitEvent(cs, q.out_done[s], 0));
  spmv_status st = spmv_apply_block(h, q.B[s], k, k, q.C[s], k, stream);
  if (st != SPMV_OK) return st;
  SPMV_CUDA(cudaEventRecord(q.kern_done[s], cs));
  SPMV_CUDA(cudaStreamWaitEvent(q.out, q.kern_done[s], 0));
  SPMV_CUDA(cudaMemcpyAsync(C_host, q.C[s], sizeof(double) * (size_t)(h->host.n_rows * k), cudaMemcpyDeviceToHost,
                            q.out));
  SPMV_CUDA(cudaEventRecord(q.out_done[s], q.out));
  q.step += 1;
  return SPMV_OK;
}

spmv_status spmv_host_sync(spmv_handle h) {
  if (!h) return fail(SPMV_ERR_ARG, "handle is NULL");
  DeviceGuard g(h->device);
  if (h->pipe.in) {
    SPMV_CUDA(cudaStreamSynchronize(h->pipe.in));
    SPMV_CUDA(cudaStreamSynchronize(h->pipe.out));
  }
  return SPMV_OK;
}

spmv_status spmv_apply_block(spmv_handle h, const double* B_dev, int32_t k, int64_t ldb, double* C_dev,
                             int64_t ldc, void* stream) {
  if (!h) return fail(SPMV_ERR_ARG, "handle is NULL");
  if (k < 1 || k > h->opt.max_k) return fail(SPMV_ERR_ARG, "k out of range 1..max_k");
  if (ldb < k || ldc < k) return fail(SPMV_ERR_ARG, "ldb and ldc must be >= k");
  if (h->host.n_rows == 0) return SPMV_OK;
  if (!C_dev || (!B_dev && h->host.n_cols > 0)) return fail(SPMV_ERR_ARG, "B or C is NULL");
  DeviceGuard g(h->device);
  cudaError_t e = run_variant(h, h->A, h->variant, B_dev, ldb, C_dev, ldc, k, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return SPMV_OK;
}

spmv_status spmv_apply(spmv_handle h, const double* B_dev, double* C_dev, void* stream) {
  return spmv_apply_block(h, B_dev, 1, 1, C_dev, 1, stream);
}

spmv_status spmv_apply_split(spmv_handle h, double* B_dev, const double* B_halo_pinned, double* C_dev,
                             void* main_stream, void* copy_stream) {
  if (!h) return fail(SPMV_ERR_ARG, "handle is NULL");
  if (!h->has_split) return fail(SPMV_ERR_UNSUPPORTED, "plan was built without a split (options.split = 0)");
  if (h->host.n_rows == 0) return SPMV_OK;
  const int64_t hb = h->split_host.h, nhalo = h->host.n_cols - hb;
  if (!C_dev || !B_dev || (nhalo > 0 && !B_halo_pinned)) return fail(SPMV_ERR_ARG, "NULL buffer");
  DeviceGuard g(h->device);
  cudaStream_t ms = (cudaStream_t)main_stream, cs = (cudaStream_t)copy_stream;
  const bool f32 = h->opt.val_fp32 != 0;
  if (nhalo > 0) {
    if (cs != ms) {
      // the copy must not overwrite B before earlier work on the main stream is done with it
      SPMV_CUDA(cudaEventRecord(h->ev_main, ms));
      SPMV_CUDA(cudaStreamWaitEvent(cs, h->ev_main, 0));
    }
    SPMV_CUDA(cudaMemcpyAsync(B_dev + hb, B_halo_pinned, sizeof(double) * (size_t)nhalo, cudaMemcpyHostToDevice,
                              cs));
    if (cs != ms) SPMV_CUDA(cudaEventRecord(h->ev_copy, cs));
  }
  // local pass: the plan's CRS kernel (SELL and SYM plans have no local copy in
  // their format, so they run CRS_L1 here)
  const int lv = h->variant >= SPMV_CRS_STAGED && h->variant <= SPMV_CRS_L32 ? h->variant : SPMV_CRS_L1;
  cudaError_t e = run_variant(h, h->local, lv, B_dev, 1, C_dev, 1, 1, ms);
  if (e != cudaSuccess) return cuda_fail(e, "local kernel launch");
  if (nhalo > 0 && cs != ms) SPMV_CUDA(cudaStreamWaitEvent(ms, h->ev_copy, 0));
  e = launch_halo(h->halo, f32, B_dev, 1, C_dev, 1, 1, ms);
  if (e != cudaSuccess) return cuda_fail(e, "halo kernel launch");
  return SPMV_OK;
}

spmv_status spmv_apply_host(spmv_handle h, const double* B_host, int32_t k, double* C_host, void* stream) {
  if (!h) return fail(SPMV_ERR_ARG, "handle is NULL");
  if (k < 1 || k > h->opt.max_k) return fail(SPMV_ERR_ARG, "k out of range 1..max_k");
  if ((!B_host && h->host.n_cols > 0) || (!C_host && h->host.n_rows > 0)) return fail(SPMV_ERR_ARG, "NULL buffer");
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  if (h->scratch_k < k) {
    if (h->d_B) h->arena.release(h->d_B);
    if (h->d_C) h->arena.release(h->d_C);
    h->d_B = h->d_C = nullptr;
    h->scratch_k = 0;
    void *b, *c;
    SPMV_CUDA(h->arena.alloc(&b, sizeof(double) * (size_t)(h->host.n_cols * k)));
    h->d_B = (double*)b;
    SPMV_CUDA(h->arena.alloc(&c, sizeof(double) * (size_t)(h->host.n_rows * k)));
    h->d_C = (double*)c;
    h->scratch_k = k;
  }
  SPMV_CUDA(cudaMemcpyAsync(h->d_B, B_host, sizeof(double) * (size_t)(h->host.n_cols * k), cudaMemcpyHostToDevice,
                            s));
  spmv_status st = spmv_apply_block(h, h->d_B, k, k, h->d_C, k, stream);
  if (st != SPMV_OK) return st;
  SPMV_CUDA(cudaMemcpyAsync(C_host, h->d_C, sizeof(double) * (size_t)(h->host.n_rows * k), cudaMemcpyDeviceToHost,
                            s));
  SPMV_CUDA(cudaStreamSynchronize(s));
  return SPMV_OK;
}

spmv_status spmv_set_variant(spmv_handle h, int32_t variant, int32_t sell_sigma) {
  if (!h) return fail(SPMV_ERR_ARG, "handle is NULL");
  DeviceGuard g(h->device);
  return prepare_variant(h, variant, sell_sigma);
}

spmv_status spmv_set_tuning(spmv_handle h, const spmv_tuning* t) {
  if (!h || !t) return fail(SPMV_ERR_ARG, "NULL argument");
  if (t->prefetch_distance < 0) return fail(SPMV_ERR_ARG, "prefetch_distance must be >= 0");
  h->tuning = *t;
  apply_tuning(h);
  ++h->generation;
  return SPMV_OK;
}

spmv_status spmv_get_tuning(spmv_handle h, spmv_tuning* t) {
  if (!h || !t) return fail(SPMV_ERR_ARG, "NULL argument");
  *t = h->tuning;
  return SPMV_OK;
}

spmv_status spmv_get_info(spmv_handle h, spmv_info* info) {
  if (!h || !info) return fail(SPMV_ERR_ARG, "NULL argument");
  std::memset(info, 0, sizeof(*info));
  info->n_rows = h->host.n_rows;
  info->n_cols = h->host.n_cols;
  info->nnz = h->host.nnz;
  info->variant = h->variant;
  info->sell_sigma = h->sell.perm ? h->sell.sigma : 0;
  info->sell_slots = h->sell.perm ? h->sell.slots : 0;
  info->sell_chunks = h->sell.perm ? h->sell.n_chunks : 0;
  info->n_halo_rows = h->has_split ? h->halo.n_rows : 0;
  info->halo_nnz = h->has_split ? h->halo.nnz : 0;
  info->n_row_blocks = h->A.n_blk;
  info->tile_nnz = h->A.tile;
  info->val_fp32 = h->opt.val_fp32;
  info->device_bytes = h->arena.bytes;
  info->sym_nnz = h->sym.row_ptr ? h->sym.nnz : 0;
  info->scattered = h->scattered;
  info->sell256_fill = h->fill256;
  return SPMV_OK;
}

spmv_status spmv_check(spmv_handle h, void* stream) {
  if (!h) return fail(SPMV_ERR_ARG, "handle is NULL");
  DeviceGuard g(h->device);
  SPMV_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  int word = 0;
  SPMV_CUDA(cudaMemcpy(&word, h->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (word != DEV_OK) {
    SPMV_CUDA(cudaMemset(h->status, 0, sizeof(int)));
    return fail(SPMV_ERR_DEVICE, "a CRS_STAGED block gave up waiting for its bulk copy (device status " +
                                     std::to_string(word) + ")");
  }
  return SPMV_OK;
}

spmv_status spmv_sell_export(spmv_handle h, int32_t* perm, int64_t* chunk_ptr, int32_t* chunk_len,
                             int32_t* sell_col, double* sell_val) {
  if (!h) return fail(SPMV_ERR_ARG, "handle is NULL");
  if (!h->sell.perm) return fail(SPMV_ERR_UNSUPPORTED, "no SELL arrays built (set_variant SELL first)");
  DeviceGuard g(h->device);
  const SellDev& S = h->sell;
  if (perm) SPMV_CUDA(cudaMemcpy(perm, S.perm, sizeof(int32_t) * (size_t)S.n_rows, cudaMemcpyDeviceToHost));
  if (chunk_ptr)
    SPMV_CUDA(cudaMemcpy(chunk_ptr, S.chunk_ptr, sizeof(int64_t) * (size_t)(S.n_chunks + 1), cudaMemcpyDeviceToHost));
  if (chunk_len)
    SPMV_CUDA(cudaMemcpy(chunk_len, S.chunk_len, sizeof(int32_t) * (size_t)S.n_chunks, cudaMemcpyDeviceToHost));
  if (sell_col) SPMV_CUDA(cudaMemcpy(sell_col, S.col, sizeof(int32_t) * (size_t)S.slots, cudaMemcpyDeviceToHost));
  if (sell_val) SPMV_CUDA(cudaMemcpy(sell_val, S.val, sizeof(double) * (size_t)S.slots, cudaMemcpyDeviceToHost));
  return SPMV_OK;
}

spmv_status spmv_select(spmv_handle h, spmv_model_handle m, int32_t k, const int32_t* variants,
                        const int32_t* sigmas, int32_t* choice, void* stream) {
  if (!h || !m || !variants || !sigmas || !choice) return fail(SPMV_ERR_ARG, "NULL argument");
  if (k < 1 || k > h->opt.max_k) return fail(SPMV_ERR_ARG, "k out of range 1..max_k");
  int32_t n_in = 0, n_hidden = 0, n_out = 0;
  int64_t n_params = 0;
  int32_t steps = 0;
  spmv_status st = spmv_model_info(m, &n_in, &n_hidden, &n_out, &n_params, &steps);
  if (st != SPMV_OK) return st;
  if (n_in != 34) return fail(SPMV_ERR_ARG, "the model must take the 34 matrix features");
  double f[34];
  compute_features(h->host.n_rows, h->host.n_cols, h->host.row_ptr.data(), h->host.col.data(), k, f);
  int32_t o = 0;
  st = spmv_model_select(m, f, 1, &o, nullptr, stream);
  if (st != SPMV_OK) return st;
  DeviceGuard g(h->device);
  st = prepare_variant(h, variants[o], sigmas[o]);
  if (st != SPMV_OK) return st;
  *choice = o;
  return SPMV_OK;
}

spmv_status spmv_autotune(spmv_handle h, int32_t k, const double* B_dev, int64_t ldb, double* C_dev, int64_t ldc,
                          const int32_t* variants, const int32_t* sigmas, int32_t n, int32_t reps, int32_t* best,
                          float* times_ms, void* stream) {
  if (!h || !variants || !sigmas || !best || n < 1 || reps < 1) return fail(SPMV_ERR_ARG, "bad argument");
  if (k < 1 || k > h->opt.max_k || ldb < k || ldc < k) return fail(SPMV_ERR_ARG, "bad k, ldb or ldc");
  if (h->host.n_rows > 0 && (!C_dev || (!B_dev && h->host.n_cols > 0))) return fail(SPMV_ERR_ARG, "NULL buffer");
  DeviceGuard g(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int keep_variant = h->variant, keep_sigma = h->sell.perm ? h->sell.sigma : 1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SPMV_CUDA(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(ce, "cudaEventCreate");
  }
  std::vector<float> med((size_t)n, INFINITY), t((size_t)reps);
  int arg = -1;
  spmv_status st = SPMV_OK;
  for (int i = 0; i < n && st == SPMV_OK; ++i) {
    if (prepare_variant(h, variants[i], sigmas[i]) != SPMV_OK) continue;  // not buildable for this matrix
    cudaError_t e = run_variant(h, h->A, h->variant, B_dev, ldb, C_dev, ldc, k, s);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
      e = cudaEventRecord(e0, s);
      if (e == cudaSuccess) e = run_variant(h, h->A, h->variant, B_dev, ldb, C_dev, ldc, k, s);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t[(size_t)r], e0, e1);
    }
    if (e != cudaSuccess) {
      st = cuda_fail(e, "autotune launch");
      break;
    }
    std::vector<float> sorted(t);
    std::sort(sorted.begin(), sorted.end());
    med[(size_t)i] = sorted[sorted.size() / 2];
    if (arg < 0 || med[(size_t)i] < med[(size_t)arg]) arg = i;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != SPMV_OK) return st;
  if (times_ms) std::memcpy(times_ms, med.data(), sizeof(float) * (size_t)n);
  if (arg < 0) {
    prepare_variant(h, keep_variant, keep_sigma);
    return fail(SPMV_ERR_UNSUPPORTED, "no candidate variant could be built for this matrix");
  }
  st = prepare_variant(h, variants[arg], sigmas[arg]);
  if (st != SPMV_OK) return st;
  *best = arg;
  return SPMV_OK;
}

spmv_status spmv_sym_export(spmv_handle h, int32_t* row_ptr, int32_t* col, double* val) {
  if (!h) return fail(SPMV_ERR_ARG, "handle is NULL");
  if (!h->sym.row_ptr) return fail(SPMV_ERR_UNSUPPORTED, "no SYM triangle built (set_variant SYM first)");
  DeviceGuard g(h->device);
  const SymDev& S = h->sym;
  if (row_ptr)
    SPMV_CUDA(cudaMemcpy(row_ptr, S.row_ptr, sizeof(int32_t) * (size_t)(S.n_rows + 1), cudaMemcpyDeviceToHost));
  if (col && S.nnz) SPMV_CUDA(cudaMemcpy(col, S.col, sizeof(int32_t) * (size_t)S.nnz, cudaMemcpyDeviceToHost));
  if (val && S.nnz) SPMV_CUDA(cudaMemcpy(val, S.val, sizeof(double) * (size_t)S.nnz, cudaMemcpyDeviceToHost));
  return SPMV_OK;
}

spmv_status spmv_split_export(spmv_handle h, int32_t* loc_row_ptr, int32_t* loc_col, double* loc_val,
                              int32_t* halo_rows, int32_t* halo_row_ptr, int32_t* halo_col, double* halo_val) {
  if (!h) return fail(SPMV_ERR_ARG, "handle is NULL");
  if (!h->has_split) return fail(SPMV_ERR_UNSUPPORTED, "plan was built without a split (options.split = 0)");
  DeviceGuard g(h->device);
  const CsrDev& L = h->local;
  const HaloDev& H = h->halo;
  auto d2h = [](void* dst, const void* src, size_t bytes) {
    return (dst && bytes) ? cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost) : cudaSuccess;
  };
  SPMV_CUDA(d2h(loc_row_ptr, L.row_ptr, sizeof(int32_t) * (size_t)(L.n_rows + 1)));
  SPMV_CUDA(d2h(loc_col, L.col, sizeof(int32_t) * (size_t)L.nnz));
  SPMV_CUDA(d2h(loc_val, L.val, sizeof(double) * (size_t)L.nnz));
  SPMV_CUDA(d2h(halo_rows, H.rows, sizeof(int32_t) * (size_t)H.n_rows));
  SPMV_CUDA(d2h(halo_row_ptr, H.row_ptr, sizeof(int32_t) * (size_t)(H.n_rows + 1)));
  SPMV_CUDA(d2h(halo_col, H.col, sizeof(int32_t) * (size_t)H.nnz));
  SPMV_CUDA(d2h(halo_val, H.val, sizeof(double) * (size_t)H.nnz));
  return SPMV_OK;
}

spmv_status spmv_features(int64_t n_rows, int64_t n_cols, const int32_t* row_ptr, const int32_t* col_idx,
                          int32_t k, double* out) {
  if (!out) return fail(SPMV_ERR_ARG, "out is NULL");
  if (k < 1) return fail(SPMV_ERR_ARG, "k must be >= 1");
  std::string why;
  if (!validate_csr(n_rows, n_cols, row_ptr, col_idx, &why)) return fail(SPMV_ERR_CSR, why);
  compute_features(n_rows, n_cols, row_ptr, col_idx, k, out);
  return SPMV_OK;
}

}  // extern "C"
