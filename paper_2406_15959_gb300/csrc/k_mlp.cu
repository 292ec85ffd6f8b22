// The learned interface warm start (include/elm_mlp.h): an MLP with GELU activations,
// trained by FP32 kernels of our own (tiled GEMM with fused epilogues, column sums, a
// deterministic MSE reduction, Adam).  Sizes are small (64 -> 512 -> 512 -> n_Gamma,
// batches of a few hundred), so a 64x64-tile SIMT GEMM on the FP32 pipe (~70 TFLOP/s)
// keeps an epoch at tens of milliseconds.
#include "elm_ddm.h"
#include "elm_mlp.h"
#include "common.cuh"

#include <cmath>
#include <random>
#include <string>
#include <vector>

namespace elmddm {

namespace {

constexpr int GT = 64;  // output tile
constexpr int GK = 16;  // k step

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// C (M x N) = op(A) op(B) with a fused epilogue; row-major, op(A) M x K, op(B) K x N.
//   EPI 0: C = AB           EPI 1: Z = AB + bias, C = gelu(Z)
//   EPI 2: C = AB + bias    EPI 3: C = AB * gelu'(Z)
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256) k_sgemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                               const float* __restrict__ B, int ldb, float* __restrict__ C,
                                               int ldc, const float* __restrict__ bias, float* __restrict__ Z,
                                               int ldz) {
  __shared__ float As[GK][GT + 4];
  __shared__ float Bs[GK][GT + 4];
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  const int i0 = blockIdx.y * GT, j0 = blockIdx.x * GT;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  for (int k0 = 0; k0 < K; k0 += GK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = t + 256 * q;
      int i, k;
      if (TA) { i = e & 63; k = e >> 6; } else { k = e & 15; i = e >> 4; }
      const int gi = i0 + i, gk = k0 + k;
      float v = 0.f;
      if (gi < M && gk < K) v = TA ? A[(size_t)gk * lda + gi] : A[(size_t)gi * lda + gk];
      As[k][i] = v;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = t + 256 * q;
      int j, k;
      if (TB) { k = e & 15; j = e >> 4; } else { j = e & 63; k = e >> 6; }
      const int gj = j0 + j, gk = k0 + k;
      float v = 0.f;
      if (gj < N && gk < K) v = TB ? B[(size_t)gj * ldb + gk] : B[(size_t)gk * ldb + gj];
      Bs[k][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < GK; ++k) {
      float av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[k][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[k][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int gi = i0 + ty + 16 * a;
    if (gi >= M) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int gj = j0 + tx + 16 * b;
      if (gj >= N) continue;
      float v = acc[a][b];
      if (EPI == 1) {
        v += bias[gj];
        Z[(size_t)gi * ldz + gj] = v;
        v = gelu(v);
      } else if (EPI == 2) {
        v += bias[gj];
      } else if (EPI == 3) {
        v *= gelu_grad(Z[(size_t)gi * ldz + gj]);
      }
      C[(size_t)gi * ldc + gj] = v;
    }
  }
}

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

template <bool TA, bool TB, int EPI>
void sgemm(cudaStream_t st, int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C,
           int ldc, const float* bias = nullptr, float* Z = nullptr, int ldz = 0) {
  dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT);
  k_sgemm<TA, TB, EPI><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, Z, ldz); count_launch();
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

// forward through the three layers; keeps z1, a1, z2, a2 for the backward pass
void forward(elm_mlp* m, const float* x, int B, float* y) {
  sgemm<false, false, 1>(m->st, B, m->dh, m->din, x, m->din, m->W1, m->dh, m->a1, m->dh, m->b1, m->z1, m->dh);
  sgemm<false, false, 1>(m->st, B, m->dh, m->dh, m->a1, m->dh, m->W2, m->dh, m->a2, m->dh, m->b2, m->z2, m->dh);
  sgemm<false, false, 2>(m->st, B, m->dout, m->dh, m->a2, m->dh, m->W3, m->dout, y, m->dout, m->b3);
}

// loss and gradients of the MSE with respect to every parameter (into m->grads)
void backward(elm_mlp* m, const float* x, const float* t, int B) {
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
  sgemm<true, false, 0>(m->st, m->dh, m->dout, B, m->a2, m->dh, m->dy, m->dout, gW3, m->dout);
  k_colsum<<<(m->dout + 255) / 256, 256, 0, m->st>>>(m->dy, B, m->dout, gb3); count_launch();
  sgemm<false, true, 3>(m->st, B, m->dh, m->dout, m->dy, m->dout, m->W3, m->dout, m->d2, m->dh, nullptr, m->z2, m->dh);
  // layer 2
  sgemm<true, false, 0>(m->st, m->dh, m->dh, B, m->a1, m->dh, m->d2, m->dh, gW2, m->dh);
  k_colsum<<<(m->dh + 255) / 256, 256, 0, m->st>>>(m->d2, B, m->dh, gb2); count_launch();
  sgemm<false, true, 3>(m->st, B, m->dh, m->dh, m->d2, m->dh, m->W2, m->dh, m->d1, m->dh, nullptr, m->z1, m->dh);
  // layer 1
  sgemm<true, false, 0>(m->st, m->din, m->dh, B, x, m->din, m->d1, m->dh, gW1, m->dh);
  k_colsum<<<(m->dh + 255) / 256, 256, 0, m->st>>>(m->d1, B, m->dh, gb1); count_launch();
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
  forward(m, x, batch, y);
  return check_launch(m, "forward");
}

int elm_mlp_gradient(elm_mlp* m, const float* x, const float* target, int batch, float* loss, float* grad) {
  if (!m) return ELM_DDM_ERR_ARG;
  if (!x || !target) return mfail(m, ELM_DDM_ERR_ARG, "gradient: NULL pointer");
  if (batch < 1 || batch > m->max_batch) return mfail(m, ELM_DDM_ERR_ARG, "gradient: batch out of range");
  forward(m, x, batch, m->y);
  backward(m, x, target, batch);
  cudaError_t e = cudaSuccess;
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

int elm_mlp_destroy(elm_mlp* m) {
  if (!m) return ELM_DDM_ERR_ARG;
  cudaStreamSynchronize(m->st);
  for (void* p : m->allocs) cudaFree(p);
  delete m;
  return ELM_DDM_OK;
}

const char* elm_mlp_last_error(const elm_mlp* m) { return m ? m->err.c_str() : g_mlp_error.c_str(); }

}  // extern "C"
