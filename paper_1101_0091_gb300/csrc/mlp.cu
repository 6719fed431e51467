// Cost model: a small MLP that predicts, from a matrix's feature vector, the
// log run time of every kernel variant, so that a plan (or a batch member) can
// run the variant with the smallest prediction.  Forward, backward and Adam are
// hand-written FP32 kernels (the network is tiny: no tensor cores needed).
//
//   Xn = (X - mean) * inv_std
//   H1 = relu(Xn W1^T + b1),  H2 = relu(H1 W2^T + b2),  Y = H2 W3^T + b3
//   loss = sum(mask * (Y - T)^2) / sum(mask)
//   Adam (Kingma and Ba, 2015) on all parameters.
//
// Every reduction runs in a fixed order (one thread per output, or one CTA),
// so results are deterministic.  Parameter layout (host and device):
// W1[H*F], b1[H], W2[H*H], b2[H], W3[V*H], b3[V].
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "internal.h"

namespace spmv {

__global__ void k_normalize(const float* __restrict__ X, const float* __restrict__ mean,
                            const float* __restrict__ inv_std, int M, int F, float* __restrict__ Xn) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M * F) {
    const int f = i % F;
    Xn[i] = (X[i] - mean[f]) * inv_std[f];
  }
}

// Z[m, o] = b[o] + sum_i X[m, i] W[o, i]; H = relu(Z) when H != nullptr.
__global__ void k_linear(const float* __restrict__ X, const float* __restrict__ W, const float* __restrict__ b,
                         int M, int In, int Out, float* __restrict__ Z, float* __restrict__ H) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * Out) return;
  const int m = i / Out, o = i % Out;
  float s = b[o];
  const float* x = X + (size_t)m * In;
  const float* w = W + (size_t)o * In;
  for (int t = 0; t < In; ++t) s = fmaf(x[t], w[t], s);
  Z[i] = s;
  if (H) H[i] = s > 0.f ? s : 0.f;
}

// One CTA: sum(mask), sum(mask * (Y - T)^2), then dY = 2 mask (Y - T) / sum(mask).
__global__ void k_loss(const float* __restrict__ Y, const float* __restrict__ T, const float* __restrict__ mask,
                       int n, float* __restrict__ dY, float* __restrict__ loss) {
  __shared__ float s_m[1024], s_l[1024];
  const int tid = threadIdx.x;
  float am = 0.f, al = 0.f;
  for (int i = tid; i < n; i += blockDim.x) {
    if (mask[i] != 0.f) {  // masked entries may hold any target value
      const float d = Y[i] - T[i];
      am += mask[i];
      al += mask[i] * d * d;
    }
  }
  s_m[tid] = am;
  s_l[tid] = al;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (tid < s) {
      s_m[tid] += s_m[tid + s];
      s_l[tid] += s_l[tid + s];
    }
    __syncthreads();
  }
  const float denom = s_m[0] > 0.f ? s_m[0] : 1.f;
  if (tid == 0 && loss) *loss = s_l[0] / denom;
  if (dY)
    for (int i = tid; i < n; i += blockDim.x) dY[i] = mask[i] != 0.f ? 2.f * mask[i] * (Y[i] - T[i]) / denom : 0.f;
}

// dW[o, i] = sum_m dZ[m, o] Hin[m, i];  db[o] = sum_m dZ[m, o].
__global__ void k_grad_w(const float* __restrict__ dZ, const float* __restrict__ Hin, int M, int In, int Out,
                         float* __restrict__ dW, float* __restrict__ db) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < Out * In) {
    const int o = i / In, t = i % In;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s = fmaf(dZ[(size_t)m * Out + o], Hin[(size_t)m * In + t], s);
    dW[i] = s;
  } else if (i < Out * In + Out) {
    const int o = i - Out * In;
    float s = 0.f;
    for (int m = 0; m < M; ++m) s += dZ[(size_t)m * Out + o];
    db[o] = s;
  }
}

// dZin[m, i] = (sum_o dZ[m, o] W[o, i]) * (Zin[m, i] > 0).
__global__ void k_backprop(const float* __restrict__ dZ, const float* __restrict__ W, const float* __restrict__ Zin,
                           int M, int In, int Out, float* __restrict__ dZin) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M * In) return;
  const int m = i / In, t = i % In;
  float s = 0.f;
  for (int o = 0; o < Out; ++o) s = fmaf(dZ[(size_t)m * Out + o], W[(size_t)o * In + t], s);
  dZin[i] = Zin[i] > 0.f ? s : 0.f;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float a = b1 * m1[i] + (1.f - b1) * gi;
  const float v = b2 * m2[i] + (1.f - b2) * gi * gi;
  m1[i] = a;
  m2[i] = v;
  p[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
}

static unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace spmv

using namespace spmv;

struct spmv_model {
  int F = 0, H = 0, V = 0;
  int64_t n_params = 0;
  int device = 0;
  int step = 0;
  float* params = nullptr;  // device
  float* m1 = nullptr;
  float* m2 = nullptr;
  float* grad = nullptr;
  float* mean = nullptr;
  float* inv_std = nullptr;
  std::vector<float> h_mean, h_inv_std;
  // activations (capacity cap rows)
  int cap = 0;
  float *Xn = nullptr, *Z1 = nullptr, *H1 = nullptr, *Z2 = nullptr, *H2 = nullptr, *Y = nullptr, *dY = nullptr,
        *dZ2 = nullptr, *dZ1 = nullptr, *Xs = nullptr, *loss = nullptr;
  float* W1() const { return params; }
  float* b1() const { return params + (size_t)H * F; }
  float* W2() const { return b1() + H; }
  float* b2() const { return W2() + (size_t)H * H; }
  float* W3() const { return b2() + H; }
  float* b3() const { return W3() + (size_t)V * H; }
};

static int64_t n_params_of(int F, int H, int V) { return (int64_t)H * F + H + (int64_t)H * H + H + (int64_t)V * H + V; }

static void free_acts(spmv_model* m) {
  for (float** p : {&m->Xn, &m->Z1, &m->H1, &m->Z2, &m->H2, &m->Y, &m->dY, &m->dZ2, &m->dZ1, &m->Xs})
    if (*p) cudaFree(*p), *p = nullptr;
  m->cap = 0;
}

static spmv_status ensure_cap(spmv_model* m, int M) {
  if (M <= m->cap) return SPMV_OK;
  free_acts(m);
  const size_t F = m->F, H = m->H, V = m->V, Mc = (size_t)M;
  SPMV_CUDA(cudaMalloc(&m->Xn, sizeof(float) * Mc * F));
  SPMV_CUDA(cudaMalloc(&m->Xs, sizeof(float) * Mc * F));
  SPMV_CUDA(cudaMalloc(&m->Z1, sizeof(float) * Mc * H));
  SPMV_CUDA(cudaMalloc(&m->H1, sizeof(float) * Mc * H));
  SPMV_CUDA(cudaMalloc(&m->Z2, sizeof(float) * Mc * H));
  SPMV_CUDA(cudaMalloc(&m->H2, sizeof(float) * Mc * H));
  SPMV_CUDA(cudaMalloc(&m->Y, sizeof(float) * Mc * V));
  SPMV_CUDA(cudaMalloc(&m->dY, sizeof(float) * Mc * V));
  SPMV_CUDA(cudaMalloc(&m->dZ2, sizeof(float) * Mc * H));
  SPMV_CUDA(cudaMalloc(&m->dZ1, sizeof(float) * Mc * H));
  m->cap = M;
  return SPMV_OK;
}

static cudaError_t forward(spmv_model* m, const float* X, int M, cudaStream_t s) {
  k_normalize<<<blocks((int64_t)M * m->F), 256, 0, s>>>(X, m->mean, m->inv_std, M, m->F, m->Xn);
  k_linear<<<blocks((int64_t)M * m->H), 256, 0, s>>>(m->Xn, m->W1(), m->b1(), M, m->F, m->H, m->Z1, m->H1);
  k_linear<<<blocks((int64_t)M * m->H), 256, 0, s>>>(m->H1, m->W2(), m->b2(), M, m->H, m->H, m->Z2, m->H2);
  k_linear<<<blocks((int64_t)M * m->V), 256, 0, s>>>(m->H2, m->W3(), m->b3(), M, m->H, m->V, m->Y, nullptr);
  return cudaGetLastError();
}

extern "C" {

spmv_status spmv_model_create(spmv_model_handle* out, int32_t n_in, int32_t n_hidden, int32_t n_out,
                              const float* params) {
  if (!out || !params) return fail(SPMV_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (n_in < 1 || n_hidden < 1 || n_out < 1 || n_in > 4096 || n_hidden > 4096 || n_out > 4096)
    return fail(SPMV_ERR_ARG, "layer sizes out of range 1..4096");
  auto* m = new spmv_model();
  m->F = n_in;
  m->H = n_hidden;
  m->V = n_out;
  m->n_params = n_params_of(n_in, n_hidden, n_out);
  cudaGetDevice(&m->device);
  auto bail = [&](spmv_status st) {
    spmv_model_destroy(m);
    return st;
  };
  const size_t pb = sizeof(float) * (size_t)m->n_params;
  cudaError_t e = cudaMalloc(&m->params, pb);
  if (e == cudaSuccess) e = cudaMalloc(&m->m1, pb);
  if (e == cudaSuccess) e = cudaMalloc(&m->m2, pb);
  if (e == cudaSuccess) e = cudaMalloc(&m->grad, pb);
  if (e == cudaSuccess) e = cudaMalloc(&m->mean, sizeof(float) * n_in);
  if (e == cudaSuccess) e = cudaMalloc(&m->inv_std, sizeof(float) * n_in);
  if (e == cudaSuccess) e = cudaMalloc(&m->loss, sizeof(float) * 4);
  if (e != cudaSuccess) return bail(cuda_fail(e, "model allocation"));
  m->h_mean.assign(n_in, 0.f);
  m->h_inv_std.assign(n_in, 1.f);
  e = cudaMemcpy(m->mean, m->h_mean.data(), sizeof(float) * n_in, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m->inv_std, m->h_inv_std.data(), sizeof(float) * n_in, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bail(cuda_fail(e, "model upload"));
  spmv_status st = spmv_model_set_params(m, params);
  if (st != SPMV_OK) return bail(st);
  *out = m;
  return SPMV_OK;
}

spmv_status spmv_model_info(spmv_model_handle m, int32_t* n_in, int32_t* n_hidden, int32_t* n_out,
                            int64_t* n_params, int32_t* adam_steps) {
  if (!m) return fail(SPMV_ERR_ARG, "model is NULL");
  if (n_in) *n_in = m->F;
  if (n_hidden) *n_hidden = m->H;
  if (n_out) *n_out = m->V;
  if (n_params) *n_params = m->n_params;
  if (adam_steps) *adam_steps = m->step;
  return SPMV_OK;
}

spmv_status spmv_model_set_params(spmv_model_handle m, const float* params) {
  if (!m || !params) return fail(SPMV_ERR_ARG, "NULL argument");
  const size_t pb = sizeof(float) * (size_t)m->n_params;
  SPMV_CUDA(cudaMemcpy(m->params, params, pb, cudaMemcpyHostToDevice));
  SPMV_CUDA(cudaMemset(m->m1, 0, pb));
  SPMV_CUDA(cudaMemset(m->m2, 0, pb));
  m->step = 0;
  return SPMV_OK;
}

spmv_status spmv_model_get_params(spmv_model_handle m, float* params) {
  if (!m || !params) return fail(SPMV_ERR_ARG, "NULL argument");
  SPMV_CUDA(cudaMemcpy(params, m->params, sizeof(float) * (size_t)m->n_params, cudaMemcpyDeviceToHost));
  return SPMV_OK;
}

spmv_status spmv_model_set_normalizer(spmv_model_handle m, const float* mean, const float* inv_std) {
  if (!m || !mean || !inv_std) return fail(SPMV_ERR_ARG, "NULL argument");
  m->h_mean.assign(mean, mean + m->F);
  m->h_inv_std.assign(inv_std, inv_std + m->F);
  SPMV_CUDA(cudaMemcpy(m->mean, mean, sizeof(float) * m->F, cudaMemcpyHostToDevice));
  SPMV_CUDA(cudaMemcpy(m->inv_std, inv_std, sizeof(float) * m->F, cudaMemcpyHostToDevice));
  return SPMV_OK;
}

spmv_status spmv_model_forward(spmv_model_handle m, const float* X_dev, int32_t M, float* Y_dev, void* stream) {
  if (!m || !X_dev || !Y_dev || M < 1) return fail(SPMV_ERR_ARG, "bad argument");
  spmv_status st = ensure_cap(m, M);
  if (st != SPMV_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = forward(m, X_dev, M, s);
  if (e != cudaSuccess) return cuda_fail(e, "forward");
  SPMV_CUDA(cudaMemcpyAsync(Y_dev, m->Y, sizeof(float) * (size_t)M * m->V, cudaMemcpyDeviceToDevice, s));
  return SPMV_OK;
}

spmv_status spmv_model_loss_grad(spmv_model_handle m, const float* X_dev, const float* T_dev, const float* mask_dev,
                                 int32_t M, float* loss_dev, float* grad_dev, void* stream) {
  if (!m || !X_dev || !T_dev || !mask_dev || M < 1) return fail(SPMV_ERR_ARG, "bad argument");
  spmv_status st = ensure_cap(m, M);
  if (st != SPMV_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  float* g = grad_dev ? grad_dev : m->grad;
  cudaError_t e = forward(m, X_dev, M, s);
  if (e != cudaSuccess) return cuda_fail(e, "forward");
  const int F = m->F, H = m->H, V = m->V;
  k_loss<<<1, 1024, 0, s>>>(m->Y, T_dev, mask_dev, M * V, m->dY, loss_dev ? loss_dev : m->loss);
  float* gW1 = g;
  float* gb1 = gW1 + (size_t)H * F;
  float* gW2 = gb1 + H;
  float* gb2 = gW2 + (size_t)H * H;
  float* gW3 = gb2 + H;
  float* gb3 = gW3 + (size_t)V * H;
  k_grad_w<<<blocks((int64_t)V * H + V), 256, 0, s>>>(m->dY, m->H2, M, H, V, gW3, gb3);
  k_backprop<<<blocks((int64_t)M * H), 256, 0, s>>>(m->dY, m->W3(), m->Z2, M, H, V, m->dZ2);
  k_grad_w<<<blocks((int64_t)H * H + H), 256, 0, s>>>(m->dZ2, m->H1, M, H, H, gW2, gb2);
  k_backprop<<<blocks((int64_t)M * H), 256, 0, s>>>(m->dZ2, m->W2(), m->Z1, M, H, H, m->dZ1);
  k_grad_w<<<blocks((int64_t)H * F + H), 256, 0, s>>>(m->dZ1, m->Xn, M, F, H, gW1, gb1);
  SPMV_CUDA(cudaGetLastError());
  return SPMV_OK;
}

spmv_status spmv_model_adam_step(spmv_model_handle m, const float* grad_dev, float lr, float beta1, float beta2,
                                 float eps, void* stream) {
  if (!m) return fail(SPMV_ERR_ARG, "model is NULL");
  m->step += 1;
  const float c1 = 1.f - std::pow(beta1, (float)m->step), c2 = 1.f - std::pow(beta2, (float)m->step);
  k_adam<<<blocks(m->n_params), 256, 0, (cudaStream_t)stream>>>(m->params, grad_dev ? grad_dev : m->grad, m->m1,
                                                                 m->m2, (int)m->n_params, lr, beta1, beta2, eps, c1,
                                                                 c2);
  SPMV_CUDA(cudaGetLastError());
  return SPMV_OK;
}

spmv_status spmv_model_train_step(spmv_model_handle m, const float* X_dev, const float* T_dev, const float* mask_dev,
                                  int32_t M, float lr, float* loss_dev, void* stream) {
  spmv_status st = spmv_model_loss_grad(m, X_dev, T_dev, mask_dev, M, loss_dev, nullptr, stream);
  if (st != SPMV_OK) return st;
  return spmv_model_adam_step(m, nullptr, lr, 0.9f, 0.999f, 1e-8f, stream);
}

spmv_status spmv_model_select_guarded(spmv_model_handle m, const double* features, int32_t M, int32_t fallback,
                                      float margin, int32_t* choice, float* predicted, void* stream) {
  if (!m || !features || !choice || M < 1) return fail(SPMV_ERR_ARG, "bad argument");
  if (fallback >= m->V) return fail(SPMV_ERR_ARG, "fallback output out of range");
  if (!(margin >= 0.0f)) return fail(SPMV_ERR_ARG, "margin must be >= 0");
  spmv_status st = ensure_cap(m, M);
  if (st != SPMV_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<float> xf((size_t)M * m->F);
  for (size_t i = 0; i < xf.size(); ++i) xf[i] = (float)features[i];
  SPMV_CUDA(cudaMemcpyAsync(m->Xs, xf.data(), sizeof(float) * xf.size(), cudaMemcpyHostToDevice, s));
  cudaError_t e = forward(m, m->Xs, M, s);
  if (e != cudaSuccess) return cuda_fail(e, "forward");
  std::vector<float> y((size_t)M * m->V);
  SPMV_CUDA(cudaMemcpyAsync(y.data(), m->Y, sizeof(float) * y.size(), cudaMemcpyDeviceToHost, s));
  SPMV_CUDA(cudaStreamSynchronize(s));
  for (int32_t i = 0; i < M; ++i) {
    const float* yi = y.data() + (size_t)i * m->V;
    int best = 0;
    for (int v = 1; v < m->V; ++v)
      if (yi[v] < yi[best]) best = v;
    // the guard: leave the fallback only for a predicted gain above the margin
    if (fallback >= 0 && !(yi[best] < yi[fallback] - margin)) best = fallback;
    choice[i] = best;
  }
  if (predicted) std::memcpy(predicted, y.data(), sizeof(float) * y.size());
  return SPMV_OK;
}

spmv_status spmv_model_select(spmv_model_handle m, const double* features, int32_t M, int32_t* choice,
                              float* predicted, void* stream) {
  return spmv_model_select_guarded(m, features, M, -1, 0.0f, choice, predicted, stream);
}

// Checkpoint: magic, sizes, Adam step, normalizer, parameters, Adam moments.
spmv_status spmv_model_save(spmv_model_handle m, const char* path) {
  if (!m || !path) return fail(SPMV_ERR_ARG, "NULL argument");
  const size_t n = (size_t)m->n_params;
  std::vector<float> p(n), a(n), v(n);
  SPMV_CUDA(cudaMemcpy(p.data(), m->params, sizeof(float) * n, cudaMemcpyDeviceToHost));
  SPMV_CUDA(cudaMemcpy(a.data(), m->m1, sizeof(float) * n, cudaMemcpyDeviceToHost));
  SPMV_CUDA(cudaMemcpy(v.data(), m->m2, sizeof(float) * n, cudaMemcpyDeviceToHost));
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(SPMV_ERR_ARG, std::string("cannot open ") + path);
  const int32_t hdr[5] = {0x4d4c5031, m->F, m->H, m->V, m->step};
  bool ok = std::fwrite(hdr, sizeof(hdr), 1, f) == 1;
  ok = ok && std::fwrite(m->h_mean.data(), sizeof(float), m->F, f) == (size_t)m->F;
  ok = ok && std::fwrite(m->h_inv_std.data(), sizeof(float), m->F, f) == (size_t)m->F;
  ok = ok && std::fwrite(p.data(), sizeof(float), n, f) == n;
  ok = ok && std::fwrite(a.data(), sizeof(float), n, f) == n;
  ok = ok && std::fwrite(v.data(), sizeof(float), n, f) == n;
  ok = (std::fclose(f) == 0) && ok;
  return ok ? SPMV_OK : fail(SPMV_ERR_ARG, std::string("write failed: ") + path);
}

spmv_status spmv_model_load(spmv_model_handle* out, const char* path) {
  if (!out || !path) return fail(SPMV_ERR_ARG, "NULL argument");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(SPMV_ERR_ARG, std::string("cannot open ") + path);
  int32_t hdr[5];
  if (std::fread(hdr, sizeof(hdr), 1, f) != 1 || hdr[0] != 0x4d4c5031 || hdr[1] < 1 || hdr[2] < 1 || hdr[3] < 1 ||
      hdr[1] > 4096 || hdr[2] > 4096 || hdr[3] > 4096) {
    std::fclose(f);
    return fail(SPMV_ERR_ARG, std::string("not a model checkpoint: ") + path);
  }
  const int F = hdr[1], H = hdr[2], V = hdr[3];
  const size_t n = (size_t)n_params_of(F, H, V);
  std::vector<float> mean(F), inv(F), p(n), a(n), v(n);
  bool ok = std::fread(mean.data(), sizeof(float), F, f) == (size_t)F;
  ok = ok && std::fread(inv.data(), sizeof(float), F, f) == (size_t)F;
  ok = ok && std::fread(p.data(), sizeof(float), n, f) == n;
  ok = ok && std::fread(a.data(), sizeof(float), n, f) == n;
  ok = ok && std::fread(v.data(), sizeof(float), n, f) == n;
  std::fclose(f);
  if (!ok) return fail(SPMV_ERR_ARG, std::string("truncated checkpoint: ") + path);
  spmv_model_handle m;
  spmv_status st = spmv_model_create(&m, F, H, V, p.data());
  if (st != SPMV_OK) return st;
  st = spmv_model_set_normalizer(m, mean.data(), inv.data());
  if (st == SPMV_OK) {
    cudaError_t e = cudaMemcpy(m->m1, a.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->m2, v.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) st = cuda_fail(e, "checkpoint upload");
  }
  if (st != SPMV_OK) {
    spmv_model_destroy(m);
    return st;
  }
  m->step = hdr[4];
  *out = m;
  return SPMV_OK;
}

spmv_status spmv_model_destroy(spmv_model_handle m) {
  if (!m) return SPMV_OK;
  cudaDeviceSynchronize();
  free_acts(m);
  for (float* p : {m->params, m->m1, m->m2, m->grad, m->mean, m->inv_std, m->loss})
    if (p) cudaFree(p);
  delete m;
  return SPMV_OK;
}

}  // extern "C"
