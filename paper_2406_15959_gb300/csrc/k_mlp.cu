// The learned interface warm start (include/elm_mlp.h): an MLP with GELU activations,
// trained by kernels of our own: the layers' GEMMs with their fused epilogues on the tensor
// cores at FP32 accuracy (three TF32 products of a hi/lo split, launch_tf32x3_gemm in
// k_ozaki.cu), column sums, a deterministic MSE reduction, Adam.  Sizes are small
// (64 -> 512 -> 512 -> n_Gamma, batches of a few hundred).
#include "elm_ddm.h"
#include "elm_mlp.h"
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <random>
#include <string>
#include <vector>

namespace elmddm {

namespace {

// db[j] = sum_i D[i][j] (D rows x cols, row-major): one thread per column, fixed order.
__global__ void k_colsum(const float* __restrict__ D, int rows, int cols, float* __restrict__ db) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cols) return;
  float s = 0.f;
  for (int i = 0; i < rows; ++i) s += D[(size_t)i * cols + j];
  db[j] = s;
}

// dY = 2 (Y - T) / n and per-block partial sums of (Y - T)^2 / n (n = rows * cols).
__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ Y, const float* __restrict__ T,
                                             long long n, float* __restrict__ dY, float* __restrict__ part) {
  __shared__ float red[256];
  float s = 0.f;
  const float inv = 1.0f / (float)n;
  for (long long e = blockIdx.x * 256ll + threadIdx.x; e < n; e += (long long)gridDim.x * 256) {
    const float d = Y[e] - T[e];
    dY[e] = 2.0f * d * inv;
    s = fmaf(d, d, s);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0] * inv;
}

// loss = sum of the partials (one thread, fixed order: deterministic).
__global__ void k_sum_parts(const float* __restrict__ part, int n, float* __restrict__ loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += part[i];
    *loss = s;
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr_t, float b1, float b2, float eps) {
  for (long long i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (long long)gridDim.x * 256) {
    const float gi = g[i];
    const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr_t * mi / (sqrtf(vi) + eps);
  }
}

constexpr int MSE_BLOCKS = 256;

}  // namespace
}  // namespace elmddm

using namespace elmddm;

struct elm_mlp {
  int din = 0, dh = 0, dout = 0, max_batch = 0;
  cudaStream_t st = nullptr;
  int64_t np = 0;
  float *params = nullptr, *grads = nullptr, *am = nullptr, *av = nullptr;
  float *z1 = nullptr, *a1 = nullptr, *z2 = nullptr, *a2 = nullptr, *y = nullptr;
  float *dy = nullptr, *d2 = nullptr, *d1 = nullptr, *part = nullptr, *loss = nullptr;
  float* work = nullptr;        // split planes of the tensor-core GEMMs
  size_t work_floats = 0;
  unsigned* status = nullptr;   // bounded waits of the GEMM kernels (ST_TIMEOUT)
  int step = 0;
  std::vector<void*> allocs;
  std::string err;
  // parameter views
  float *W1 = nullptr, *b1 = nullptr, *W2 = nullptr, *b2 = nullptr, *W3 = nullptr, *b3 = nullptr;
};

namespace {

std::string g_mlp_error;

int mfail(elm_mlp* m, int code, const std::string& msg) {
  if (m) m->err = msg; else g_mlp_error = msg;
  return code;
}

bool malloc_f(elm_mlp* m, float** p, size_t n) {
  void* q = nullptr;
  if (cudaMalloc(&q, (n ? n : 1) * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  m->allocs.push_back(q);
  *p = static_cast<float*>(q);
  return true;
}

int check_launch(elm_mlp* m, const char* where) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return mfail(m, ELM_DDM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return ELM_DDM_OK;
}

// C (M x N, row-major) = op(A) op(B) with the layer epilogue epi: A, B row-major with leading
// dimensions lda, ldb, transposed when ta / tb (op(A) M x K, op(B) K x N).
cudaError_t gemm(elm_mlp* m, bool ta, bool tb, int epi, int M, int N, int K, const float* A, int lda,
                 const float* B, int ldb, float* C, int ldc, const float* bias = nullptr, float* Z = nullptr,
                 int ldz = 0) {
  return launch_tf32x3_gemm(M, N, K, A, ta ? 1 : lda, ta ? lda : 1, B, tb ? ldb : 1, tb ? 1 : ldb, C, ldc, epi,
                            bias, Z, ldz, m->work, m->work_floats, m->status, m->st);
}

// the largest split workspace of the layers' GEMMs at batch size B
size_t gemm_work(int din, int dh, int dout, int B) {
  const int shapes[8][3] = {{B, dh, din}, {B, dh, dh}, {B, dout, dh}, {dh, dout, B},
                            {B, dh, dout}, {dh, dh, B}, {B, dh, dh}, {din, dh, B}};
  size_t w = 0;
  for (const auto& sh : shapes) w = std::max(w, tf32x3_work_floats(sh[0], sh[1], sh[2]));
  return w;
}

// forward through the three layers; keeps z1, a1, z2, a2 for the backward pass
cudaError_t forward(elm_mlp* m, const float* x, int B, float* y) {
  cudaError_t e = gemm(m, false, false, 1, B, m->dh, m->din, x, m->din, m->W1, m->dh, m->a1, m->dh, m->b1, m->z1, m->dh);
  if (e == cudaSuccess)
    e = gemm(m, false, false, 1, B, m->dh, m->dh, m->a1, m->dh, m->W2, m->dh, m->a2, m->dh, m->b2, m->z2, m->dh);
  if (e == cudaSuccess) e = gemm(m, false, false, 2, B, m->dout, m->dh, m->a2, m->dh, m->W3, m->dout, y, m->dout, m->b3);
  return e;
}

// loss and gradients of the MSE with respect to every parameter (into m->grads)
cudaError_t backward(elm_mlp* m, const float* x, const float* t, int B) {
  const long long n = (long long)B * m->dout;
  k_mse<<<MSE_BLOCKS, 256, 0, m->st>>>(m->y, t, n, m->dy, m->part); count_launch();
  k_sum_parts<<<1, 32, 0, m->st>>>(m->part, MSE_BLOCKS, m->loss); count_launch();
  float* gW1 = m->grads;
  float* gb1 = gW1 + (size_t)m->din * m->dh;
  float* gW2 = gb1 + m->dh;
  float* gb2 = gW2 + (size_t)m->dh * m->dh;
  float* gW3 = gb2 + m->dh;
  float* gb3 = gW3 + (size_t)m->dh * m->dout;
  // layer 3: dW3 = a2^T dy, db3 = colsum(dy), d2 = (dy W3^T) * g'(z2)
  cudaError_t e = gemm(m, true, false, 0, m->dh, m->dout, B, m->a2, m->dh, m->dy, m->dout, gW3, m->dout);
  k_colsum<<<(m->dout + 255) / 256, 256, 0, m->st>>>(m->dy, B, m->dout, gb3); count_launch();
  if (e == cudaSuccess)
    e = gemm(m, false, true, 3, B, m->dh, m->dout, m->dy, m->dout, m->W3, m->dout, m->d2, m->dh, nullptr, m->z2, m->dh);
  // layer 2
  if (e == cudaSuccess) e = gemm(m, true, false, 0, m->dh, m->dh, B, m->a1, m->dh, m->d2, m->dh, gW2, m->dh);
  k_colsum<<<(m->dh + 255) / 256, 256, 0, m->st>>>(m->d2, B, m->dh, gb2); count_launch();
  if (e == cudaSuccess)
    e = gemm(m, false, true, 3, B, m->dh, m->dh, m->d2, m->dh, m->W2, m->dh, m->d1, m->dh, nullptr, m->z1, m->dh);
  // layer 1
  if (e == cudaSuccess) e = gemm(m, true, false, 0, m->din, m->dh, B, x, m->din, m->d1, m->dh, gW1, m->dh);
  k_colsum<<<(m->dh + 255) / 256, 256, 0, m->st>>>(m->d1, B, m->dh, gb1); count_launch();
  return e;
}

}  // namespace

extern "C" {

int elm_mlp_create(int d_in, int d_hidden, int d_out, int max_batch, uint64_t seed, void* stream,
                   elm_mlp** out) {
  if (!out) return mfail(nullptr, ELM_DDM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (d_in < 1 || d_hidden < 1 || d_out < 1 || max_batch < 1)
    return mfail(nullptr, ELM_DDM_ERR_ARG, "sizes must be >= 1");
  elm_mlp* m = new elm_mlp;
  m->din = d_in; m->dh = d_hidden; m->dout = d_out; m->max_batch = max_batch;
  m->st = static_cast<cudaStream_t>(stream);
  m->np = (int64_t)d_in * d_hidden + d_hidden + (int64_t)d_hidden * d_hidden + d_hidden +
          (int64_t)d_hidden * d_out + d_out;
  const size_t hb = (size_t)max_batch * d_hidden, ob = (size_t)max_batch * d_out;
  bool ok = malloc_f(m, &m->params, m->np) && malloc_f(m, &m->grads, m->np) && malloc_f(m, &m->am, m->np) &&
            malloc_f(m, &m->av, m->np) && malloc_f(m, &m->z1, hb) && malloc_f(m, &m->a1, hb) &&
            malloc_f(m, &m->z2, hb) && malloc_f(m, &m->a2, hb) && malloc_f(m, &m->y, ob) &&
            malloc_f(m, &m->dy, ob) && malloc_f(m, &m->d2, hb) && malloc_f(m, &m->d1, hb) &&
            malloc_f(m, &m->part, MSE_BLOCKS) && malloc_f(m, &m->loss, 1);
  m->work_floats = gemm_work(d_in, d_hidden, d_out, max_batch);
  ok = ok && malloc_f(m, &m->work, m->work_floats) && malloc_f(m, reinterpret_cast<float**>(&m->status), 1);
  if (!ok) {
    for (void* p : m->allocs) cudaFree(p);
    delete m;
    return mfail(nullptr, ELM_DDM_ERR_OOM, "device allocation failed");
  }
  m->W1 = m->params;
  m->b1 = m->W1 + (size_t)d_in * d_hidden;
  m->W2 = m->b1 + d_hidden;
  m->b2 = m->W2 + (size_t)d_hidden * d_hidden;
  m->W3 = m->b2 + d_hidden;
  m->b3 = m->W3 + (size_t)d_hidden * d_out;
  // Glorot-uniform weights, zero biases
  std::vector<float> h(m->np, 0.f);
  std::mt19937_64 rng(seed);
  auto fill = [&](size_t off, int fin, int fout) {
    const float a = std::sqrt(6.0f / (float)(fin + fout));
    std::uniform_real_distribution<float> U(-a, a);
    for (size_t i = 0; i < (size_t)fin * fout; ++i) h[off + i] = U(rng);
  };
  fill(0, d_in, d_hidden);
  fill((size_t)(m->W2 - m->params), d_hidden, d_hidden);
  fill((size_t)(m->W3 - m->params), d_hidden, d_out);
  cudaError_t e = cudaMemcpy(m->params, h.data(), m->np * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->am, 0, m->np * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->av, 0, m->np * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->status, 0, sizeof(unsigned));
  if (e != cudaSuccess) {
    for (void* p : m->allocs) cudaFree(p);
    delete m;
    return mfail(nullptr, ELM_DDM_ERR_CUDA, cudaGetErrorString(e));
  }
  *out = m;
  return ELM_DDM_OK;
}

int elm_mlp_param_count(const elm_mlp* m, int64_t* count) {
  if (!m || !count) return ELM_DDM_ERR_ARG;
  *count = m->np;
  return ELM_DDM_OK;
}

int elm_mlp_get_params(elm_mlp* m, float* dst) {
  if (!m) return ELM_DDM_ERR_ARG;
  if (!dst) return mfail(m, ELM_DDM_ERR_ARG, "get_params: NULL dst");
  cudaError_t e = cudaMemcpyAsync(dst, m->params, m->np * sizeof(float), cudaMemcpyDeviceToDevice, m->st);
  return e == cudaSuccess ? ELM_DDM_OK : mfail(m, ELM_DDM_ERR_CUDA, cudaGetErrorString(e));
}

int elm_mlp_set_params(elm_mlp* m, const float* src) {
  if (!m) return ELM_DDM_ERR_ARG;
  if (!src) return mfail(m, ELM_DDM_ERR_ARG, "set_params: NULL src");
  cudaError_t e = cudaMemcpyAsync(m->params, src, m->np * sizeof(float), cudaMemcpyDeviceToDevice, m->st);
  return e == cudaSuccess ? ELM_DDM_OK : mfail(m, ELM_DDM_ERR_CUDA, cudaGetErrorString(e));
}

int elm_mlp_forward(elm_mlp* m, const float* x, int batch, float* y) {
  if (!m) return ELM_DDM_ERR_ARG;
  if (!x || !y) return mfail(m, ELM_DDM_ERR_ARG, "forward: NULL pointer");
  if (batch < 1 || batch > m->max_batch) return mfail(m, ELM_DDM_ERR_ARG, "forward: batch out of range");
  const cudaError_t e = forward(m, x, batch, y);
  if (e != cudaSuccess) return mfail(m, ELM_DDM_ERR_CUDA, std::string("forward: ") + cudaGetErrorString(e));
  return check_launch(m, "forward");
}

int elm_mlp_gradient(elm_mlp* m, const float* x, const float* target, int batch, float* loss, float* grad) {
  if (!m) return ELM_DDM_ERR_ARG;
  if (!x || !target) return mfail(m, ELM_DDM_ERR_ARG, "gradient: NULL pointer");
  if (batch < 1 || batch > m->max_batch) return mfail(m, ELM_DDM_ERR_ARG, "gradient: batch out of range");
  cudaError_t e = forward(m, x, batch, m->y);
  if (e == cudaSuccess) e = backward(m, x, target, batch);
  if (e != cudaSuccess) return mfail(m, ELM_DDM_ERR_CUDA, std::string("gradient: ") + cudaGetErrorString(e));
  if (loss) e = cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToDevice, m->st);
  if (e == cudaSuccess && grad)
    e = cudaMemcpyAsync(grad, m->grads, m->np * sizeof(float), cudaMemcpyDeviceToDevice, m->st);
  if (e != cudaSuccess) return mfail(m, ELM_DDM_ERR_CUDA, cudaGetErrorString(e));
  return check_launch(m, "gradient");
}

int elm_mlp_train_step(elm_mlp* m, const float* x, const float* target, int batch, float lr, float* loss) {
  if (!m) return ELM_DDM_ERR_ARG;
  if (!(lr > 0.f) || !std::isfinite(lr)) return mfail(m, ELM_DDM_ERR_ARG, "train_step: lr must be > 0");
  int rc = elm_mlp_gradient(m, x, target, batch, loss, nullptr);
  if (rc) return rc;
  m->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float lr_t = lr * std::sqrt(1.0f - std::pow(b2, (float)m->step)) / (1.0f - std::pow(b1, (float)m->step));
  const int blocks = (int)std::min<int64_t>((m->np + 255) / 256, 4096);
  k_adam<<<blocks, 256, 0, m->st>>>(m->params, m->grads, m->am, m->av, m->np, lr_t, b1, b2, 1e-8f); count_launch();
  return check_launch(m, "train_step");
}

int elm_mlp_check(elm_mlp* m) {
  if (!m) return ELM_DDM_ERR_ARG;
  unsigned st = 0;
  cudaError_t e = cudaStreamSynchronize(m->st);
  if (e == cudaSuccess) e = cudaMemcpy(&st, m->status, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && st) e = cudaMemset(m->status, 0, sizeof(unsigned));
  if (e != cudaSuccess) return mfail(m, ELM_DDM_ERR_CUDA, cudaGetErrorString(e));
  if (st) return mfail(m, ELM_DDM_ERR_TIMEOUT, "a tensor-core GEMM wait gave up (its results are not valid)");
  return ELM_DDM_OK;
}

int elm_mlp_destroy(elm_mlp* m) {
  if (!m) return ELM_DDM_ERR_ARG;
  cudaStreamSynchronize(m->st);
  for (void* p : m->allocs) cudaFree(p);
  delete m;
  return ELM_DDM_OK;
}

const char* elm_mlp_last_error(const elm_mlp* m) { return m ? m->err.c_str() : g_mlp_error.c_str(); }

}  // extern "C"
