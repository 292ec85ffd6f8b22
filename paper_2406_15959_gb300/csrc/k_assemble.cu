// Step (a): batched assembly of the local collocation blocks (Section 3), and the
// evaluation of the trained local networks at arbitrary points.
//
// For subdomain s and hidden neuron j, with t = tanh(w_j . x + b_j):
//   interior rows          L phi_j = -Laplacian phi_j = 2 |w_j|^2 t (1 - t^2), or for
//                          L = -div(rho grad) (Section 4, variable coefficient)
//                          2 rho |w_j|^2 t (1 - t^2) - (grad rho . w_j)(1 - t^2)
//   boundary/interface     phi_j = t
//   A^s (interface rows)   d phi_j / d n = (w_j . n)(1 - t^2)
// The kernel also writes the m_Gamma "interface identity" columns J = E^T next to
// K^s (row mi+mb+k of column n+k is 1), so that the Householder QR applies Q^T to
// them and leaves Q_G^T in rows 0..n-1 of those columns.
#include "common.cuh"

namespace elmddm {

namespace {

constexpr int AR = 64;  // rows per block
constexpr int AC = 32;  // columns per block

__global__ void __launch_bounds__(256) k_assemble(double* __restrict__ K, long long kstride, int ld,
                                                  int ncap, double* __restrict__ Amat,
                                                  long long astride, int mgld,
                                                  const double* __restrict__ xy,
                                                  const double* __restrict__ nrm, int m_max,
                                                  const int* __restrict__ cnt,
                                                  const double* __restrict__ W,
                                                  const double* __restrict__ bias, int n,
                                                  const double* __restrict__ coef,
                                                  unsigned* status) {
  const int s = blockIdx.z;
  const int r = blockIdx.x * AR + threadIdx.x;
  const int c0 = blockIdx.y * AC;
  const int mi = cnt[3 * s], mb = cnt[3 * s + 1], mg = cnt[3 * s + 2];
  const int row0g = mi + mb, ms = row0g + mg;

  __shared__ double sw[AC][3];
  const int tl = threadIdx.y * AR + threadIdx.x;
  if (tl < AC) {
    const int c = c0 + tl;
    double wx = 0, wy = 0, bb = 0;
    if (c < n) {
      wx = W[((size_t)s * n + c) * 2];
      wy = W[((size_t)s * n + c) * 2 + 1];
      bb = bias[(size_t)s * n + c];
    }
    sw[tl][0] = wx; sw[tl][1] = wy; sw[tl][2] = bb;
  }
  __syncthreads();
  if (r >= ld) return;

  double px = 0, py = 0, nx = 0, ny = 0;
  double rho = 1.0, rx = 0.0, ry = 0.0;  // coefficient and its gradient (interior rows)
  if (r < ms) {
    px = xy[((size_t)s * m_max + r) * 2];
    py = xy[((size_t)s * m_max + r) * 2 + 1];
    if (coef && r < mi) {
      const double* cr = coef + ((size_t)s * m_max + r) * 3;
      rho = cr[0]; rx = cr[1]; ry = cr[2];
      if (!isfinite(rho) || !isfinite(rx) || !isfinite(ry)) atomicOr(status, ST_NONFINITE);
    }
    if (r >= row0g) {
      nx = nrm[((size_t)s * m_max + r) * 2];
      ny = nrm[((size_t)s * m_max + r) * 2 + 1];
    }
  }
  double* Ks = K + (size_t)s * kstride;
  double* As = Amat + (size_t)s * astride;
  bool bad = false;
#pragma unroll
  for (int q = 0; q < AC / 4; ++q) {
    const int cl = threadIdx.y + 4 * q;
    const int c = c0 + cl;
    if (c >= ncap) break;
    double v = 0.0;
    if (c < n) {
      if (r < ms) {
        const double wx = sw[cl][0], wy = sw[cl][1];
        const double z = fma(wx, px, fma(wy, py, sw[cl][2]));
        const double t = tanh(z);
        const double d1 = 1.0 - t * t;
        bad |= !isfinite(z);
        if (r < mi) {
          v = 2.0 * fma(wx, wx, wy * wy) * t * d1;
          if (coef) v = fma(rho, v, -fma(rx, wx, ry * wy) * d1);
        } else {
          v = t;
        }
        if (r >= row0g) As[(r - row0g) + (size_t)c * mgld] = fma(wx, nx, wy * ny) * d1;
      }
    } else if (c - n < mg) {
      v = (r == row0g + (c - n)) ? 1.0 : 0.0;
    }
    Ks[r + (size_t)c * ld] = v;
  }
  if (bad) atomicOr(status, ST_NONFINITE);
}

// One warp per point.
__global__ void __launch_bounds__(256) k_eval(const double* __restrict__ W,
                                              const double* __restrict__ bias, int N, int n,
                                              int npts, const double* __restrict__ xy,
                                              const int* __restrict__ owner,
                                              const double* __restrict__ c,
                                              double* __restrict__ u, double* __restrict__ grad) {
  const int lane = threadIdx.x & 31;
  const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (p >= npts) return;
  const int s = owner[p];
  if (s < 0 || s >= N) {
    if (lane == 0) {
      u[p] = __longlong_as_double(0x7ff8000000000000ll);
      if (grad) grad[2 * p] = grad[2 * p + 1] = u[p];
    }
    return;
  }
  const double x = xy[2 * p], y = xy[2 * p + 1];
  const double* Ws = W + (size_t)s * n * 2;
  const double* bs = bias + (size_t)s * n;
  const double* cs = c + (size_t)s * n;
  double su = 0, sx = 0, sy = 0;
  for (int j = lane; j < n; j += 32) {
    const double wx = Ws[2 * j], wy = Ws[2 * j + 1];
    const double t = tanh(fma(wx, x, fma(wy, y, bs[j])));
    const double cj = cs[j];
    su = fma(cj, t, su);
    const double d = cj * (1.0 - t * t);
    sx = fma(d, wx, sx);
    sy = fma(d, wy, sy);
  }
  su = warp_sum(su);
  sx = warp_sum(sx);
  sy = warp_sum(sy);
  if (lane == 0) {
    u[p] = su;
    if (grad) { grad[2 * p] = sx; grad[2 * p + 1] = sy; }
  }
}

}  // namespace

cudaError_t launch_assemble(double* K, long long kstride, int ld, int ncap, double* Amat,
                            long long astride, int mgld, const double* xy, const double* nrm,
                            int m_max, const int* cnt, const double* W, const double* b, int N,
                            int n, const double* coef, unsigned* status, cudaStream_t st) {
  dim3 grid((ld + AR - 1) / AR, (ncap + AC - 1) / AC, N);
  k_assemble<<<grid, dim3(AR, 4), 0, st>>>(K, kstride, ld, ncap, Amat, astride, mgld, xy, nrm,
                                           m_max, cnt, W, b, n, coef, status); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_eval(const double* W, const double* b, int N, int n, int npts,
                        const double* xy, const int* owner, const double* c, double* u,
                        double* grad, cudaStream_t st) {
  if (npts <= 0) return cudaSuccess;
  k_eval<<<(npts + 7) / 8, 256, 0, st>>>(W, b, N, n, npts, xy, owner, c, u, grad); count_launch();
  return cudaGetLastError();
}

}  // namespace elmddm
