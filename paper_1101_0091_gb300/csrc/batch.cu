// Batched products over many uneven matrices in one persistent launch,
// replayed from a CUDA graph, and the autotuner of its launch configuration.
//
// Work list: items (matrix, rows, lanes per row L).  A persistent grid of
// SMs x ctas_per_sm CTAs runs; each warp takes items either round-robin
// (static) or from an atomic counter reset by the graph before the kernel
// (dynamic).  Inside an item, groups of L lanes share a row (Sec. 1.2 loop per
// lane over a strided subset of the row, FP64 FMAs, xor-shuffle sum when L > 1),
// 32/L rows per pass.  Fixed policies cut each member's rows into contiguous
// ranges.  The adaptive policy bins rows by exact length (a counting sort), so
// that the 32 rows of a warp pass have equal length and no lane idles on the
// FP64 pipe; rows up to 32 entries get one lane, longer rows about 32 entries
// per lane; inside a member, longer rows come first.  The sorted policy (the
// default) puts the rows of up to kSortedMaxLen entries into a length-sorted
// SELL-32 copy and the longer ones into adaptive items.  Items keep member order,
// which keeps the B blocks being gathered resident in L2.  No CTA ever waits
// for another.
#include <algorithm>
#include <cstring>
#include <vector>

#include "batch_kernel.cuh"
#include "internal.h"

namespace spmv {

static int policy_lanes(int policy) {
  switch (policy) {
    case SPMV_BATCH_L1: return 1;
    case SPMV_BATCH_L2: return 2;
    case SPMV_BATCH_L4: return 4;
    case SPMV_BATCH_L8: return 8;
    case SPMV_BATCH_L32: return 32;
    default: return 0;  // adaptive
  }
}

// Lanes for a row of `len` entries under the adaptive policy: at most about 32
// entries per lane (fewer lanes keep the shuffle adds on the FP64 pipe few).
static int adaptive_lanes(int64_t len) {
  int L = 1;
  while (L < 32 && (int64_t)L * 32 < len) L <<= 1;
  return L;
}

// Items of about item_nnz work units (a row counts max(len, 1)) and at most
// 64 warp passes.  Contiguous rows [p0, p1) (mode 0), or positions [p0, p1) of
// the row list, all of length len (mode 1).
static void cut_items(const int32_t* rp, int64_t p0, int64_t p1, int mat, int L, int mode, int64_t len,
                      int item_nnz, std::vector<BatchItem>& out) {
  const int64_t rows_cap = (int64_t)(32 / L) * 64;
  int64_t s = p0, work = 0;
  for (int64_t p = p0; p < p1; ++p) {
    if (p > s && (work >= item_nnz || p - s >= rows_cap)) {
      out.push_back(BatchItem{mat, (int32_t)s, (int32_t)p, (int32_t)len, (int16_t)L, (int16_t)mode, 0, 0});
      s = p;
      work = 0;
    }
    work += mode == 1 ? std::max<int64_t>(len, 1) : (mode == 2 ? len : std::max<int64_t>(rp[p + 1] - rp[p], 1));
  }
  if (p1 > s) out.push_back(BatchItem{mat, (int32_t)s, (int32_t)p1, (int32_t)len, (int16_t)L, (int16_t)mode, 0, 0});
}

// Rows of at most this many entries go to the length-sorted SELL-32 copy
// (sorted policy, one lane per row, coalesced slots); longer rows to
// multi-lane CRS items.  Of 32 / 64 / 96 / 128, 64 gave the fastest
// power-law batch (rows of 33-64 entries ran at 0.69 of the FP64 peak as
// two-lane CRS items and at 0.96 in the sorted copy).
constexpr int kSortedMaxLen = 64;

// Length-sorted SELL-32 copy of the rows with at most kSortedMaxLen entries (sorted
// policy), appended for one member: rows by descending length (stable), 32 per
// chunk, chunk length = its first (longest) row, column-major slots, padding
// val +0.0 with the row's last column (0 for empty and padding rows).
struct SortedSell {
  std::vector<int64_t> chunk_ptr{0};
  std::vector<int32_t> chunk_len, perm, col;
  std::vector<double> val;
};

static void append_sorted_sell(const int32_t* rp, const int32_t* col, const double* val, int64_t n_rows,
                               SortedSell& S, int64_t* first_chunk, int64_t* n_chunks) {
  int64_t cnt[kSortedMaxLen + 2] = {0};
  for (int64_t r = 0; r < n_rows; ++r) {
    const int64_t len = rp[r + 1] - rp[r];
    if (len <= kSortedMaxLen) cnt[kSortedMaxLen - len + 1]++;
  }
  for (int i = 1; i < kSortedMaxLen + 2; ++i) cnt[i] += cnt[i - 1];
  const int64_t n_short = cnt[kSortedMaxLen + 1];
  std::vector<int32_t> order((size_t)n_short);
  for (int64_t r = 0; r < n_rows; ++r) {
    const int64_t len = rp[r + 1] - rp[r];
    if (len <= kSortedMaxLen) order[(size_t)cnt[kSortedMaxLen - len]++] = (int32_t)r;
  }
  *first_chunk = (int64_t)S.chunk_len.size();
  *n_chunks = (n_short + 31) / 32;
  for (int64_t i = 0; i < n_short; i += 32) {
    const int32_t clen = rp[order[i] + 1] - rp[order[i]];
    const int64_t base = S.chunk_ptr.back();
    S.col.resize((size_t)(base + 32 * clen), 0);
    S.val.resize((size_t)(base + 32 * clen), 0.0);
    for (int t = 0; t < 32; ++t) {
      const int32_t r = (i + t < n_short) ? order[(size_t)(i + t)] : -1;
      S.perm.push_back(r);
      const int64_t len = r >= 0 ? rp[r + 1] - rp[r] : 0;
      int32_t last = 0;
      for (int64_t j = 0; j < clen; ++j) {
        const int64_t slot = base + j * 32 + t;
        if (j < len) {
          last = col[rp[r] + j];
          S.col[(size_t)slot] = last;
          S.val[(size_t)slot] = val[rp[r] + j];
        } else {
          S.col[(size_t)slot] = last;
        }
      }
    }
    S.chunk_len.push_back(clen);
    S.chunk_ptr.push_back(base + 32 * (int64_t)clen);
  }
}

// Items over chunks [c0, c0 + nc) of the sorted copy, about item_nnz slots each.
// (An item never mixes chunk lengths, so it carries the length and the first
// slot and the kernel needs no per-chunk metadata.)
static void cut_chunk_items(const SortedSell& S, int64_t c0, int64_t nc, int mat, int item_nnz,
                            std::vector<BatchItem>& out) {
  int64_t s = c0, work = 0;
  auto emit = [&](int64_t e) {
    out.push_back(BatchItem{mat, (int32_t)s, (int32_t)e, S.chunk_len[(size_t)s], (int16_t)1, (int16_t)3, 0,
                            S.chunk_ptr[(size_t)s]});
  };
  for (int64_t c = c0; c < c0 + nc; ++c) {
    if (c > s && (work >= item_nnz || S.chunk_len[(size_t)c] != S.chunk_len[(size_t)s])) {
      emit(c);
      s = c;
      work = 0;
    }
    work += std::max<int64_t>(32 * (int64_t)S.chunk_len[(size_t)c], 32);
  }
  if (c0 + nc > s) emit(c0 + nc);
}

void build_batch_items(const int32_t* rp, int64_t n_rows, int mat, int policy, int item_nnz,
                       std::vector<BatchItem>& out, std::vector<int2>& rowlist) {
  const int fixed = policy_lanes(policy);
  if (fixed) {
    cut_items(rp, 0, n_rows, mat, fixed, 0, 0, item_nnz, out);
    return;
  }
  const bool long_only = policy == SPMV_BATCH_SORTED;  // short rows live in the sorted SELL copy
  // counting sort of the rows by descending length (ascending row inside a length)
  int64_t maxlen = 0;
  for (int64_t r = 0; r < n_rows; ++r) maxlen = std::max<int64_t>(maxlen, rp[r + 1] - rp[r]);
  std::vector<int64_t> start((size_t)maxlen + 2, 0);
  for (int64_t r = 0; r < n_rows; ++r) start[(size_t)(maxlen - (rp[r + 1] - rp[r])) + 1]++;
  for (size_t i = 1; i < start.size(); ++i) start[i] += start[i - 1];
  const int64_t base = (int64_t)rowlist.size();
  rowlist.resize((size_t)(base + n_rows));
  std::vector<int64_t> fill(start.begin(), start.end() - 1);
  for (int64_t r = 0; r < n_rows; ++r) {
    const int64_t len = rp[r + 1] - rp[r];
    rowlist[(size_t)(base + fill[(size_t)(maxlen - len)]++)] = make_int2((int)r, (int)rp[r]);
  }
  // rows of up to 32 entries: one item family per exact length (one lane per
  // row, no divergence); longer rows: one family per lane count, lengths within
  // a factor of two of each other (few rows per length, which would leave
  // most lanes of a pass idle)
  int64_t d = 0;
  while (d <= maxlen) {
    const int64_t len = maxlen - d;
    const int L = adaptive_lanes(len);
    int64_t e = d + 1;
    if (len > 32)
      while (e <= maxlen && adaptive_lanes(maxlen - e) == L && maxlen - e > 32) ++e;
    const int64_t p0 = start[(size_t)d], p1 = start[(size_t)e];
    if (p1 > p0 && !(long_only && len <= kSortedMaxLen))
      cut_items(rp, base + p0, base + p1, mat, L, len > 32 ? 2 : 1, len, item_nnz, out);
    d = e;
  }
}

}  // namespace spmv

using namespace spmv;

struct spmv_batch_plan {
  int device = 0;
  int num_sms = 0;
  int k = 1;
  std::vector<spmv_handle> plans;
  std::vector<int32_t> policies;
  spmv_batch_config cfg{};
  std::vector<BatchMat> h_mats;
  BatchMat* d_mats = nullptr;
  BatchItem* d_items = nullptr;
  int2* d_rowlist = nullptr;
  int64_t n_items = 0;
  int64_t n_chunk_items = 0;  // sorted-chunk items in the list
  int* d_counter = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // recorded on the caller's stream after every replay: set_io waits on it
  // before it rewrites the member table a replay in flight may still read
  cudaEvent_t ev_last = nullptr;
  // pipelined host path: two device buffer sets, each with its own member table
  // and graph; copy-in and copy-out streams; events per set
  struct Pipe {
    double* B[2] = {nullptr, nullptr};
    double* C[2] = {nullptr, nullptr};
    BatchMat* mats[2] = {nullptr, nullptr};
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaStream_t in = nullptr, out = nullptr;
    cudaEvent_t in_done[2] = {nullptr, nullptr}, kern_done[2] = {nullptr, nullptr}, out_done[2] = {nullptr, nullptr};
    std::vector<int64_t> b_off, c_off;  // member offsets (doubles) inside a set
    bool vec = false;
    int64_t step = 0;
  } pipe;
  bool io_set = false;
  bool vec = false;  // 16-byte loads/stores of right-hand-side rows
  // length-sorted SELL copy of the sorted-policy members (rebuilt when the policies change)
  std::vector<int32_t> sell_policies;
  SortedSell sell_host;
  std::vector<int64_t> sell_first, sell_count;
  BatchSell sell{};
  std::vector<void*> sell_ptrs;
};

static void free_sell(spmv_batch_plan* b) {
  for (void* p : b->sell_ptrs) cudaFree(p);
  b->sell_ptrs.clear();
  b->sell = BatchSell{};
}

// Build (when the policies changed) and upload the sorted SELL copy.
static spmv_status ensure_sell(spmv_batch_plan* b) {
  if (b->sell_policies == b->policies && (b->sell.perm || b->sell_host.chunk_len.empty())) return SPMV_OK;
  free_sell(b);
  b->sell_host = SortedSell{};
  const size_t n = b->plans.size();
  b->sell_first.assign(n, 0);
  b->sell_count.assign(n, 0);
  for (size_t m = 0; m < n; ++m)
    if (b->policies[m] == SPMV_BATCH_SORTED)
      append_sorted_sell(plan_host_row_ptr(b->plans[m]), plan_host_col(b->plans[m]), plan_host_val(b->plans[m]),
                         plan_csr(b->plans[m])->n_rows, b->sell_host, &b->sell_first[m], &b->sell_count[m]);
  b->sell_policies = b->policies;
  const SortedSell& S = b->sell_host;
  if (S.chunk_len.empty()) return SPMV_OK;
  auto up = [&](const void* src, size_t bytes, void** dst) -> cudaError_t {
    cudaError_t e = cudaMalloc(dst, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return e;
    b->sell_ptrs.push_back(*dst);
    return bytes ? cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) : cudaSuccess;
  };
  void *cp, *cl, *pm, *co, *va;
  SPMV_CUDA(up(S.chunk_ptr.data(), sizeof(int64_t) * S.chunk_ptr.size(), &cp));
  SPMV_CUDA(up(S.chunk_len.data(), sizeof(int32_t) * S.chunk_len.size(), &cl));
  SPMV_CUDA(up(S.perm.data(), sizeof(int32_t) * S.perm.size(), &pm));
  SPMV_CUDA(up(S.col.data(), sizeof(int32_t) * S.col.size(), &co));
  SPMV_CUDA(up(S.val.data(), sizeof(double) * S.val.size(), &va));
  b->sell = BatchSell{(const int64_t*)cp, (const int32_t*)cl, (const int32_t*)pm, (const int32_t*)co,
                      (const double*)va};
  // the entries now live on the device; keep the chunk lengths for cutting items
  std::vector<int32_t>().swap(b->sell_host.col);
  std::vector<double>().swap(b->sell_host.val);
  std::vector<int32_t>().swap(b->sell_host.perm);
  return SPMV_OK;
}

static void free_graph(spmv_batch_plan* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// Graph of one batched product over member table `mats`: counter reset +
// persistent kernel (the rows-only variant when the list holds no sorted chunks).
static spmv_status capture_graph(spmv_batch_plan* b, BatchMat* mats, bool vec, cudaGraph_t* graph,
                                 cudaGraphExec_t* exec) {
  int grid = b->num_sms * b->cfg.ctas_per_sm;
  int dynamic = b->cfg.schedule ? 1 : 0;
  int n_items = (int)b->n_items;
  int k = b->k;
  void* a_all[] = {(void*)&mats,    (void*)&b->d_items,   (void*)&n_items, (void*)&b->d_rowlist,
                   (void*)&b->sell, (void*)&b->d_counter, (void*)&dynamic, (void*)&k};
  void* a_rows[] = {(void*)&mats,         (void*)&b->d_items, (void*)&n_items, (void*)&b->d_rowlist,
                    (void*)&b->d_counter, (void*)&dynamic,    (void*)&k};
  const bool chunks = b->n_chunk_items > 0;
  SPMV_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e1 = cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->cap_stream);
  cudaError_t e2 = cudaLaunchKernel(chunks ? batch_kernel(b->k, vec) : batch_rows_kernel(b->k, vec), dim3(grid),
                                    dim3(kBatchThreads), chunks ? a_all : a_rows, 0, b->cap_stream);
  cudaError_t e3 = cudaStreamEndCapture(b->cap_stream, graph);
  if (e1 != cudaSuccess) return cuda_fail(e1, "graph memset node");
  if (e2 != cudaSuccess) return cuda_fail(e2, "graph kernel node");
  if (e3 != cudaSuccess) return cuda_fail(e3, "cudaStreamEndCapture");
  SPMV_CUDA(cudaGraphInstantiate(exec, *graph, 0));
  return SPMV_OK;
}

static void free_pipe_graphs(spmv_batch_plan* b) {
  for (int s = 0; s < 2; ++s) {
    if (b->pipe.exec[s]) cudaGraphExecDestroy(b->pipe.exec[s]);
    if (b->pipe.graph[s]) cudaGraphDestroy(b->pipe.graph[s]);
    b->pipe.exec[s] = nullptr;
    b->pipe.graph[s] = nullptr;
  }
}

static spmv_status build_graph(spmv_batch_plan* b) {
  free_graph(b);
  free_pipe_graphs(b);  // the pipelined path captures its own again on its next step
  return capture_graph(b, b->d_mats, b->vec, &b->graph, &b->exec);
}

// (Re)build the work list and the graph.
static spmv_status rebuild(spmv_batch_plan* b) {
  spmv_status st = ensure_sell(b);
  if (st != SPMV_OK) return st;
  std::vector<BatchItem> items;
  std::vector<int2> rowlist;
  for (size_t m = 0; m < b->plans.size(); ++m) {
    if (b->policies[m] == SPMV_BATCH_SORTED && b->sell_count[m] > 0)
      cut_chunk_items(b->sell_host, b->sell_first[m], b->sell_count[m], (int)m, b->cfg.item_nnz, items);
    build_batch_items(plan_host_row_ptr(b->plans[m]), plan_csr(b->plans[m])->n_rows, (int)m, b->policies[m],
                      b->cfg.item_nnz, items, rowlist);
  }
  if (items.size() > (size_t)INT32_MAX || rowlist.size() > (size_t)INT32_MAX)
    return fail(SPMV_ERR_ARG, "too many work items");
  // Items stay in member order (inside a member, longest rows first): the warps
  // in flight then work on a few neighbouring members whose B blocks fit in L2,
  // instead of gathering at random from every member's B in DRAM.
  b->n_chunk_items = std::count_if(items.begin(), items.end(), [](const BatchItem& it) { return it.mode == 3; });
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_rowlist) cudaFree(b->d_rowlist);
  b->d_items = nullptr;
  b->d_rowlist = nullptr;
  b->n_items = (int64_t)items.size();
  SPMV_CUDA(cudaMalloc(&b->d_items, sizeof(BatchItem) * std::max<size_t>(items.size(), 1)));
  if (!items.empty())
    SPMV_CUDA(cudaMemcpy(b->d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice));
  SPMV_CUDA(cudaMalloc(&b->d_rowlist, sizeof(int2) * std::max<size_t>(rowlist.size(), 1)));
  if (!rowlist.empty())
    SPMV_CUDA(cudaMemcpy(b->d_rowlist, rowlist.data(), sizeof(int2) * rowlist.size(), cudaMemcpyHostToDevice));
  return build_graph(b);
}

static spmv_status check_config(const spmv_batch_config* c) {
  if (c->item_nnz < 64 || c->item_nnz > (1 << 20)) return fail(SPMV_ERR_ARG, "item_nnz out of range 64..2^20");
  if (c->schedule != 0 && c->schedule != 1) return fail(SPMV_ERR_ARG, "schedule must be 0 or 1");
  if (c->ctas_per_sm < 1 || c->ctas_per_sm > 8) return fail(SPMV_ERR_ARG, "ctas_per_sm out of range 1..8");
  return SPMV_OK;
}

// Set up the pipelined host path on first use: two device sets of every
// member's B and C back to back (ld = k), a member table and a graph per set,
// the copy streams and the events.
static spmv_status pipe_setup(spmv_batch_plan* b) {
  auto& q = b->pipe;
  const size_t n = b->plans.size();
  if (q.b_off.empty()) {
    q.b_off.assign(n + 1, 0);
    q.c_off.assign(n + 1, 0);
    for (size_t m = 0; m < n; ++m) {
      q.b_off[m + 1] = q.b_off[m] + plan_csr(b->plans[m])->n_cols * b->k;
      q.c_off[m + 1] = q.c_off[m] + b->h_mats[m].n_rows * b->k;
    }
    SPMV_CUDA(cudaStreamCreateWithFlags(&q.in, cudaStreamNonBlocking));
    SPMV_CUDA(cudaStreamCreateWithFlags(&q.out, cudaStreamNonBlocking));
    for (int s = 0; s < 2; ++s) {
      SPMV_CUDA(cudaMalloc(&q.B[s], sizeof(double) * (size_t)std::max<int64_t>(q.b_off[n], 2)));
      SPMV_CUDA(cudaMalloc(&q.C[s], sizeof(double) * (size_t)std::max<int64_t>(q.c_off[n], 2)));
      SPMV_CUDA(cudaMalloc(&q.mats[s], sizeof(BatchMat) * n));
      SPMV_CUDA(cudaEventCreateWithFlags(&q.in_done[s], cudaEventDisableTiming));
      SPMV_CUDA(cudaEventCreateWithFlags(&q.kern_done[s], cudaEventDisableTiming));
      SPMV_CUDA(cudaEventCreateWithFlags(&q.out_done[s], cudaEventDisableTiming));
      std::vector<BatchMat> t(b->h_mats);
      for (size_t m = 0; m < n; ++m) {
        t[m].B = q.B[s] + q.b_off[m];
        t[m].C = q.C[s] + q.c_off[m];
        t[m].ldb = b->k;
        t[m].ldc = b->k;
      }
      SPMV_CUDA(cudaMemcpy(q.mats[s], t.data(), sizeof(BatchMat) * n, cudaMemcpyHostToDevice));
    }
    // every member's block starts at a multiple of k doubles from a 256-byte aligned base
    q.vec = b->k % 2 == 0;
  }
  for (int s = 0; s < 2; ++s)
    if (!q.exec[s]) {
      spmv_status st = capture_graph(b, q.mats[s], q.vec, &q.graph[s], &q.exec[s]);
      if (st != SPMV_OK) return st;
    }
  return SPMV_OK;
}

// Copies of consecutive members whose host blocks follow one another merge
// into one copy (the device blocks of a set are back to back).
template <class DevOf, class HostOf, class LenOf>
static cudaError_t copy_members(size_t n, DevOf dev_of, HostOf host_of, LenOf len_of, bool to_device,
                                cudaStream_t s) {
  size_t m = 0;
  while (m < n) {
    if (len_of(m) == 0) {
      ++m;
      continue;
    }
    char* d = (char*)dev_of(m);
    char* h = (char*)host_of(m);
    size_t bytes = len_of(m), e = m + 1;
    while (e < n && len_of(e) > 0 && (char*)host_of(e) == h + bytes && (char*)dev_of(e) == d + bytes)
      bytes += len_of(e++);
    cudaError_t err = to_device ? cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, s)
                                : cudaMemcpyAsync(h, d, bytes, cudaMemcpyDeviceToHost, s);
    if (err != cudaSuccess) return err;
    m = e;
  }
  return cudaSuccess;
}

extern "C" {

spmv_batch_config spmv_batch_default_config(void) {
  spmv_batch_config c;
  std::memset(&c, 0, sizeof(c));
  c.item_nnz = 1024;
  c.schedule = 1;
  c.ctas_per_sm = kBatchCtasPerSm;
  return c;
}

spmv_status spmv_batch_create(spmv_batch_handle* out, int32_t count, const spmv_handle* plans, int32_t k,
                              const int32_t* policies, const spmv_batch_config* cfg) {
  if (!out) return fail(SPMV_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (count < 1 || !plans) return fail(SPMV_ERR_ARG, "count must be >= 1 with a plan array");
  if (k < 1 || k > 16) return fail(SPMV_ERR_ARG, "k out of range 1..16");
  spmv_batch_config c = cfg ? *cfg : spmv_batch_default_config();
  spmv_status st = check_config(&c);
  if (st != SPMV_OK) return st;
  const int dev = plan_device(plans[0]);
  for (int m = 0; m < count; ++m) {
    if (!plans[m]) return fail(SPMV_ERR_ARG, "NULL plan in the batch");
    if (plan_device(plans[m]) != dev) return fail(SPMV_ERR_ARG, "batch members on different devices");
    if (policies && (policies[m] < 0 || policies[m] >= SPMV_BATCH_N_POLICIES))
      return fail(SPMV_ERR_ARG, "unknown batch policy");
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != dev) SPMV_CUDA(cudaSetDevice(dev));
  auto* b = new spmv_batch_plan();
  b->device = dev;
  b->k = k;
  b->cfg = c;
  b->plans.assign(plans, plans + count);
  b->policies.assign(count, SPMV_BATCH_SORTED);
  if (policies) b->policies.assign(policies, policies + count);
  auto bail = [&](spmv_status s) {
    spmv_batch_destroy(b);
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    return s;
  };
  cudaError_t e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return bail(cuda_fail(e, "cudaDeviceGetAttribute"));
  b->h_mats.resize(count);
  for (int m = 0; m < count; ++m) {
    const CsrDev* A = plan_csr(plans[m]);
    b->h_mats[m] = BatchMat{A->row_ptr, A->col, A->val, nullptr, nullptr, k, k, A->n_rows};
  }
  e = cudaMalloc(&b->d_mats, sizeof(BatchMat) * count);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_mats, b->h_mats.data(), sizeof(BatchMat) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(int) * 4);
  if (e == cudaSuccess) e = cudaMemset(b->d_counter, 0, sizeof(int) * 4);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_last, cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(cuda_fail(e, "batch allocation"));
  st = rebuild(b);
  if (st != SPMV_OK) return bail(st);
  if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  *out = b;
  return SPMV_OK;
}

spmv_status spmv_batch_set_io(spmv_batch_handle b, const double* const* B_ptrs, const int64_t* ldb,
                              double* const* C_ptrs, const int64_t* ldc) {
  if (!b || !B_ptrs || !C_ptrs) return fail(SPMV_ERR_ARG, "NULL argument");
  for (size_t m = 0; m < b->h_mats.size(); ++m) {
    const int64_t lb = ldb ? ldb[m] : b->k, lc = ldc ? ldc[m] : b->k;
    if (lb < b->k || lc < b->k) return fail(SPMV_ERR_ARG, "ldb/ldc must be >= k");
    if (!C_ptrs[m] && b->h_mats[m].n_rows > 0) return fail(SPMV_ERR_ARG, "NULL C pointer");
    if (!B_ptrs[m] && plan_csr(b->plans[m])->nnz > 0)
      return fail(SPMV_ERR_ARG, "NULL B pointer of member " + std::to_string(m) + " (it has nonzeros)");
  }
  // a replay enqueued earlier (on any stream) may still read the table: wait for it
  SPMV_CUDA(cudaEventSynchronize(b->ev_last));
  bool vec = (b->k % 2 == 0);
  for (size_t m = 0; m < b->h_mats.size(); ++m) {
    const int64_t lb = ldb ? ldb[m] : b->k, lc = ldc ? ldc[m] : b->k;
    b->h_mats[m].B = B_ptrs[m];
    b->h_mats[m].C = C_ptrs[m];
    b->h_mats[m].ldb = lb;
    b->h_mats[m].ldc = lc;
    vec = vec && (lb % 2 == 0) && (lc % 2 == 0) && ((uintptr_t)B_ptrs[m] % 16 == 0) &&
          ((uintptr_t)C_ptrs[m] % 16 == 0);
  }
  SPMV_CUDA(cudaMemcpy(b->d_mats, b->h_mats.data(), sizeof(BatchMat) * b->h_mats.size(), cudaMemcpyHostToDevice));
  if (vec != b->vec || !b->exec) {
    b->vec = vec;
    spmv_status st = build_graph(b);
    if (st != SPMV_OK) return st;
  }
  b->io_set = true;
  return SPMV_OK;
}

spmv_status spmv_batch_apply(spmv_batch_handle b, void* stream) {
  if (!b) return fail(SPMV_ERR_ARG, "batch is NULL");
  if (!b->io_set) return fail(SPMV_ERR_ARG, "spmv_batch_set_io was not called");
  SPMV_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
  SPMV_CUDA(cudaEventRecord(b->ev_last, (cudaStream_t)stream));
  return SPMV_OK;
}

spmv_status spmv_batch_apply_host(spmv_batch_handle b, const double* const* B_host, double* const* C_host,
                                  void* stream) {
  if (!b || !B_host || !C_host) return fail(SPMV_ERR_ARG, "NULL argument");
  if (!b->io_set) return fail(SPMV_ERR_ARG, "spmv_batch_set_io was not called");
  const size_t n = b->plans.size();
  std::vector<int64_t> n_cols(n);
  for (size_t m = 0; m < n; ++m) {
    const BatchMat& M = b->h_mats[m];
    if (M.ldb != b->k || M.ldc != b->k) return fail(SPMV_ERR_ARG, "the host path needs set_io with ldb = ldc = k");
    spmv_info info;
    spmv_status st = spmv_get_info(b->plans[m], &info);
    if (st != SPMV_OK) return st;
    n_cols[m] = info.n_cols;
    if ((n_cols[m] > 0 && !B_host[m]) || (M.n_rows > 0 && !C_host[m])) return fail(SPMV_ERR_ARG, "NULL host buffer");
  }
  cudaStream_t s = (cudaStream_t)stream;
  // members whose blocks follow one another both on the host and on the device
  // (one allocation cut into views) move in one copy: a copy per member costs
  // its own setup, which dominates for many small members
  auto copy_runs = [&](auto dst_of, auto src_of, auto len_of, cudaMemcpyKind kind) -> cudaError_t {
    size_t m = 0;
    while (m < n) {
      if (len_of(m) == 0) {
        ++m;
        continue;
      }
      char* dst = (char*)dst_of(m);
      const char* src = (const char*)src_of(m);
      size_t bytes = len_of(m);
      size_t e = m + 1;
      while (e < n && len_of(e) > 0 && (char*)dst_of(e) == dst + bytes && (const char*)src_of(e) == src + bytes)
        bytes += len_of(e++);
      cudaError_t err = cudaMemcpyAsync(dst, src, bytes, kind, s);
      if (err != cudaSuccess) return err;
      m = e;
    }
    return cudaSuccess;
  };
  const size_t kb = sizeof(double) * (size_t)b->k;
  SPMV_CUDA(copy_runs([&](size_t m) { return (void*)b->h_mats[m].B; }, [&](size_t m) { return (const void*)B_host[m]; },
                      [&](size_t m) { return kb * (size_t)n_cols[m]; }, cudaMemcpyHostToDevice));
  SPMV_CUDA(cudaGraphLaunch(b->exec, s));
  SPMV_CUDA(cudaEventRecord(b->ev_last, s));
  SPMV_CUDA(copy_runs([&](size_t m) { return (void*)C_host[m]; }, [&](size_t m) { return (const void*)b->h_mats[m].C; },
                      [&](size_t m) { return kb * (size_t)b->h_mats[m].n_rows; }, cudaMemcpyDeviceToHost));
  return SPMV_OK;
}

spmv_status spmv_batch_apply_host_async(spmv_batch_handle b, const double* const* B_host, double* const* C_host,
                                        void* stream) {
  if (!b || !B_host || !C_host) return fail(SPMV_ERR_ARG, "NULL argument");
  const size_t n = b->plans.size();
  for (size_t m = 0; m < n; ++m)
    if ((plan_csr(b->plans[m])->n_cols > 0 && !B_host[m]) || (b->h_mats[m].n_rows > 0 && !C_host[m]))
      return fail(SPMV_ERR_ARG, "NULL host buffer of member " + std::to_string(m));
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != b->device) SPMV_CUDA(cudaSetDevice(b->device));
  spmv_status st = pipe_setup(b);
  if (st != SPMV_OK) return st;
  auto& q = b->pipe;
  const int s = (int)(q.step & 1);
  cudaStream_t ks = (cudaStream_t)stream;
  const size_t kb = sizeof(double) * (size_t)b->k;
  // set s is free for new B once the launch two steps back has read it
  SPMV_CUDA(cudaStreamWaitEvent(q.in, q.kern_done[s], 0));
  SPMV_CUDA(copy_members(
      n, [&](size_t m) { return (void*)(q.B[s] + q.b_off[m]); }, [&](size_t m) { return (void*)B_host[m]; },
      [&](size_t m) { return kb * (size_t)plan_csr(b->plans[m])->n_cols; }, true, q.in));
  SPMV_CUDA(cudaEventRecord(q.in_done[s], q.in));
  // the launch waits for its B and for the copy-out of the step that last used C of set s
  SPMV_CUDA(cudaStreamWaitEvent(ks, q.in_done[s], 0));
  SPMV_CUDA(cudaStreamWaitEvent(ks, q.out_done[s], 0));
  SPMV_CUDA(cudaGraphLaunch(q.exec[s], ks));
  SPMV_CUDA(cudaEventRecord(q.kern_done[s], ks));
  SPMV_CUDA(cudaEventRecord(b->ev_last, ks));
  SPMV_CUDA(cudaStreamWaitEvent(q.out, q.kern_done[s], 0));
  SPMV_CUDA(copy_members(
      n, [&](size_t m) { return (void*)(q.C[s] + q.c_off[m]); }, [&](size_t m) { return (void*)C_host[m]; },
      [&](size_t m) { return kb * (size_t)b->h_mats[m].n_rows; }, false, q.out));
  SPMV_CUDA(cudaEventRecord(q.out_done[s], q.out));
  ++q.step;
  if (prev >= 0 && prev != b->device) cudaSetDevice(prev);
  return SPMV_OK;
}

spmv_status spmv_batch_host_sync(spmv_batch_handle b) {
  if (!b) return fail(SPMV_ERR_ARG, "batch is NULL");
  if (b->pipe.in) SPMV_CUDA(cudaStreamSynchronize(b->pipe.in));
  if (b->pipe.out) SPMV_CUDA(cudaStreamSynchronize(b->pipe.out));
  return SPMV_OK;
}

spmv_status spmv_batch_apply_separate(spmv_batch_handle b, void* stream) {
  if (!b) return fail(SPMV_ERR_ARG, "batch is NULL");
  if (!b->io_set) return fail(SPMV_ERR_ARG, "spmv_batch_set_io was not called");
  for (size_t m = 0; m < b->plans.size(); ++m) {
    const BatchMat& M = b->h_mats[m];
    spmv_status st = spmv_apply_block(b->plans[m], M.B, b->k, M.ldb, M.C, M.ldc, stream);
    if (st != SPMV_OK) return st;
  }
  return SPMV_OK;
}

spmv_status spmv_batch_set_config(spmv_batch_handle b, const spmv_batch_config* cfg) {
  if (!b || !cfg) return fail(SPMV_ERR_ARG, "NULL argument");
  spmv_status st = check_config(cfg);
  if (st != SPMV_OK) return st;
  b->cfg = *cfg;
  return rebuild(b);
}

spmv_status spmv_batch_get_config(spmv_batch_handle b, spmv_batch_config* cfg) {
  if (!b || !cfg) return fail(SPMV_ERR_ARG, "NULL argument");
  *cfg = b->cfg;
  return SPMV_OK;
}

spmv_status spmv_batch_set_policies(spmv_batch_handle b, const int32_t* policies) {
  if (!b || !policies) return fail(SPMV_ERR_ARG, "NULL argument");
  for (size_t m = 0; m < b->plans.size(); ++m)
    if (policies[m] < 0 || policies[m] >= SPMV_BATCH_N_POLICIES) return fail(SPMV_ERR_ARG, "unknown batch policy");
  b->policies.assign(policies, policies + b->plans.size());
  return rebuild(b);
}

spmv_status spmv_batch_autotune(spmv_batch_handle b, void* stream, int32_t reps, spmv_batch_config* best,
                                float* times_ms) {
  if (!b) return fail(SPMV_ERR_ARG, "batch is NULL");
  if (!b->io_set) return fail(SPMV_ERR_ARG, "spmv_batch_set_io was not called");
  if (reps < 1) reps = 1;
  cudaStream_t s = (cudaStream_t)stream;
  const int item_opts[5] = {256, 512, 1024, 2048, 4096};
  const int sched_opts[2] = {0, 1};
  const int cta_opts[2] = {4, kBatchCtasPerSm};
  cudaEvent_t e0, e1;
  SPMV_CUDA(cudaEventCreate(&e0));
  SPMV_CUDA(cudaEventCreate(&e1));
  spmv_batch_config keep = b->cfg, win = b->cfg;
  float win_t = 1e30f;
  int idx = 0;
  spmv_status st = SPMV_OK;
  std::vector<float> ts((size_t)reps);
  for (int io = 0; io < 5 && st == SPMV_OK; ++io)
    for (int so = 0; so < 2 && st == SPMV_OK; ++so)
      for (int co = 0; co < 2 && st == SPMV_OK; ++co, ++idx) {
        spmv_batch_config c = keep;
        c.item_nnz = item_opts[io];
        c.schedule = sched_opts[so];
        c.ctas_per_sm = cta_opts[co];
        b->cfg = c;
        st = rebuild(b);
        if (st != SPMV_OK) break;
        cudaGraphLaunch(b->exec, s);  // warm-up
        for (int r = 0; r < reps; ++r) {
          cudaEventRecord(e0, s);
          cudaGraphLaunch(b->exec, s);
          cudaEventRecord(e1, s);
          cudaError_t e = cudaEventSynchronize(e1);
          if (e != cudaSuccess) {
            st = cuda_fail(e, "autotune timing");
            break;
          }
          cudaEventElapsedTime(&ts[r], e0, e1);
        }
        if (st != SPMV_OK) break;
        std::vector<float> sorted = ts;
        std::sort(sorted.begin(), sorted.end());
        const float med = sorted[sorted.size() / 2];
        if (times_ms) times_ms[idx] = med;
        if (med < win_t) {
          win_t = med;
          win = c;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->cfg = (st == SPMV_OK) ? win : keep;
  spmv_status st2 = rebuild(b);
  if (st != SPMV_OK) return st;
  if (st2 != SPMV_OK) return st2;
  if (best) *best = win;
  return SPMV_OK;
}

spmv_status spmv_batch_info(spmv_batch_handle b, int64_t* n_items, int64_t* total_rows, int64_t* total_nnz) {
  if (!b) return fail(SPMV_ERR_ARG, "batch is NULL");
  int64_t rows = 0, nnz = 0;
  for (spmv_handle p : b->plans) {
    rows += plan_csr(p)->n_rows;
    nnz += plan_csr(p)->nnz;
  }
  if (n_items) *n_items = b->n_items;
  if (total_rows) *total_rows = rows;
  if (total_nnz) *total_nnz = nnz;
  return SPMV_OK;
}

spmv_status spmv_batch_destroy(spmv_batch_handle b) {
  if (!b) return SPMV_OK;
  cudaDeviceSynchronize();
  free_graph(b);
  free_pipe_graphs(b);
  {
    auto& q = b->pipe;
    for (int s2 = 0; s2 < 2; ++s2) {
      if (q.B[s2]) cudaFree(q.B[s2]);
      if (q.C[s2]) cudaFree(q.C[s2]);
      if (q.mats[s2]) cudaFree(q.mats[s2]);
      if (q.in_done[s2]) cudaEventDestroy(q.in_done[s2]);
      if (q.kern_done[s2]) cudaEventDestroy(q.kern_done[s2]);
      if (q.out_done[s2]) cudaEventDestroy(q.out_done[s2]);
    }
    if (q.in) cudaStreamDestroy(q.in);
    if (q.out) cudaStreamDestroy(q.out);
  }
  if (b->ev_last) cudaEventDestroy(b->ev_last);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_rowlist) cudaFree(b->d_rowlist);
  if (b->d_mats) cudaFree(b->d_mats);
  free_sell(b);
  if (b->d_counter) cudaFree(b->d_counter);
  delete b;
  return SPMV_OK;
}

}  // extern "C"
