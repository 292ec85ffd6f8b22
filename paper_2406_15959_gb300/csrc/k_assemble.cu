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
//
// tanh costs some 30 FP64 operations, and the FP64 pipe (2 per clock per SM) bounds
// this step.  The paper's collocation points are tensor grids and edge lines, so a
// subdomain has few distinct x and y coordinates, and
//   E = exp(2 z) = exp(2 (w_x (x - c_x) + z_c)) * exp(2 w_y (y - c_y)),
//   z_c = w . c + b (c the centre of the subdomain's coordinates),
// factors into per-neuron tables over those coordinates (k_exp_tables).  Then with
// r = 1 / (E + 1)
//   t = (E - 1) r,   1 - t^2 = 4 E r^2,
// one product and one reciprocal per entry instead of a tanh (the reciprocal by a
// third-order iteration from an FP32 seed, rcp_newton: three FP64 FMAs, within 2 ulp).  Accuracy: E carries the
// relative error of the two factors (a few ulp plus the rounding of their centred
// arguments), E - 1 is exact near E = 1, so t has an absolute error of a few ulp times
// the argument's magnitude -- no more than tanh(w . x + b) itself, whose argument rounds
// at the scale of |w| |x| with x uncentred.  The y factor is kept within exp(+-600)
// (larger arguments store NaN), so an overflowing product means z > 50 and saturates
// (t = 1, 1 - t^2 = 0), an underflowing one means t = -1, and a product that is not a
// number (such a y factor, or non-finite parameters) falls back to tanh(z).
#include "common.cuh"

namespace elmddm {

namespace {

constexpr int AR = 64;  // rows per block
constexpr int AC = 32;  // columns per block

// Factor tables of subdomain s = blockIdx.y: Tx[s][j][ix] = exp(2 (w_x (x_ix - c_x) + z_c))
// and Ty[s][j][iy] = exp(2 w_y (y_iy - c_y)), over its distinct coordinates.
__global__ void __launch_bounds__(256) k_exp_tables(const double* __restrict__ W,
                                                    const double* __restrict__ bias, int n,
                                                    const AsmTables tb) {
  const int s = blockIdx.y;
  const int per = tb.nxmax + tb.nymax;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * per) return;
  const int j = (int)(idx / per), i = (int)(idx % per);
  const double wx = W[((size_t)s * n + j) * 2], wy = W[((size_t)s * n + j) * 2 + 1];
  const double cx = tb.ctr[2 * s], cy = tb.ctr[2 * s + 1];
  if (i < tb.nxmax) {
    if (i >= tb.nxy[2 * s]) return;
    const double zc = fma(wx, cx, fma(wy, cy, bias[(size_t)s * n + j]));
    const double x = tb.xs[(size_t)s * tb.nxmax + i];
    tb.Tx[((size_t)s * n + j) * tb.nxmax + i] = exp(2.0 * fma(wx, x - cx, zc));
  } else {
    const int iy = i - tb.nxmax;
    if (iy >= tb.nxy[2 * s + 1]) return;
    const double y = tb.ys[(size_t)s * tb.nymax + iy];
    // beyond |arg| = 600 the product could pair an overflow with a compensating
    // underflow: a NaN entry sends that neuron's entries to tanh(z)
    const double arg = 2.0 * wy * (y - cy);
    tb.Ty[((size_t)s * n + j) * tb.nymax + iy] =
        fabs(arg) <= 600.0 ? exp(arg) : __longlong_as_double(0x7ff8000000000000ll);
  }
}

template <bool TAB>
__global__ void __launch_bounds__(256) k_assemble(double* __restrict__ K, long long kstride, int ld,
                                                  int ncap, double* __restrict__ Amat,
                                                  long long astride, int mgld,
                                                  const double* __restrict__ xy,
                                                  const double* __restrict__ nrm, int m_max,
                                                  const int* __restrict__ cnt,
                                                  const double* __restrict__ W,
                                                  const double* __restrict__ bias, int n,
                                                  const double* __restrict__ coef,
                                                  const AsmTables tb, unsigned* status,
                                                  const int* __restrict__ nsub) {
  const int s = blockIdx.z;
  const int r = blockIdx.x * AR + threadIdx.x;
  const int c0 = blockIdx.y * AC;
  const int mi = cnt[3 * s], mb = cnt[3 * s + 1], mg = cnt[3 * s + 2];
  const int row0g = mi + mb, ms = row0g + mg;   // rows with collocation points
  const int ns = nsub ? nsub[s] : n;            // columns ns .. n-1: pad neurons

  __shared__ double sw[AC][4];  // w_x, w_y, b, 2 |w|^2
  const int tl = threadIdx.y * AR + threadIdx.x;
  if (tl < AC) {
    const int c = c0 + tl;
    double wx = 0, wy = 0, bb = 0;
    if (c < n) {
      wx = W[((size_t)s * n + c) * 2];
      wy = W[((size_t)s * n + c) * 2 + 1];
      bb = bias[(size_t)s * n + c];
    }
    sw[tl][0] = wx; sw[tl][1] = wy; sw[tl][2] = bb; sw[tl][3] = 2.0 * fma(wx, wx, wy * wy);
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
  int ix = 0, iy = 0;
  if (TAB && r < ms) {
    const int pk = tb.rix[(size_t)s * m_max + r];
    ix = pk & 0xFFFF;
    iy = pk >> 16;
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
    if (c >= ns && c < n) {
      v = (r == ms + (c - ns)) ? 1.0 : 0.0;  // identity column on pad row ms + (c - ns)
    } else if (c < n) {
      if (r < ms) {
        const double wx = sw[cl][0], wy = sw[cl][1];
        double t, d1;
        bool direct = !TAB;
        if (TAB) {
          const double a = tb.Tx[((size_t)s * n + c) * tb.nxmax + ix];
          const double b = tb.Ty[((size_t)s * n + c) * tb.nymax + iy];
          const double E = a * b;
          if (E < 1e300) {
            const double rr = rcp_newton(E + 1.0);  // E + 1 in [1, 1e300]: the iteration's fast path
            t = (E - 1.0) * rr;
            d1 = 4.0 * rr * (E * rr);
          } else if (E >= 1e300) {
            t = 1.0;
            d1 = 0.0;
          } else {
            direct = true;
          }
        }
        if (direct) {
          const double z = fma(wx, px, fma(wy, py, sw[cl][2]));
          t = tanh(z);
          d1 = 1.0 - t * t;
          bad |= !isfinite(z);
        }
        if (r < mi) {
          v = sw[cl][3] * t * d1;
          if (coef) v = fma(rho, v, -fma(rx, wx, ry * wy) * d1);
        } else {
          v = t;
        }
        if (Amat && r >= row0g) As[(r - row0g) + (size_t)c * mgld] = fma(wx, nx, wy * ny) * d1;
      }
    } else if (c - n < mg) {
      v = (r == row0g + (c - n)) ? 1.0 : 0.0;
    }
    Ks[r + (size_t)c * ld] = v;
  }
  if (bad) atomicOr(status, ST_NONFINITE);
}

// Explicit A-rows (the corner rule of the remark in Section 3: one row per edge through a
// cross point, with that edge's normal): row f of A^s sits at collocation row frow[s][f]
// with normal fnrm[s][f]; A[f][c] = (w_c . n)(1 - t^2), t = tanh(w_c . x + b_c).  A thread
// per (row, 8 columns), rows fastest so the column-major stores coalesce.
__global__ void __launch_bounds__(256) k_flux_rows(double* __restrict__ A, long long astride, int mfld,
                                                   const int* __restrict__ mf, const int* __restrict__ frow,
                                                   const double* __restrict__ fnrm,
                                                   const double* __restrict__ xy, int m_max,
                                                   const double* __restrict__ W,
                                                   const double* __restrict__ bias, int n,
                                                   const int* __restrict__ nsub, unsigned* status) {
  const int s = blockIdx.z;
  const int f = blockIdx.x * 32 + threadIdx.x;
  if (f >= mf[s]) return;
  const int ns = nsub ? nsub[s] : n;
  const size_t q = (size_t)s * mfld + f;
  const int r = frow[q];
  const double px = xy[((size_t)s * m_max + r) * 2], py = xy[((size_t)s * m_max + r) * 2 + 1];
  const double nx = fnrm[2 * q], ny = fnrm[2 * q + 1];
  double* As = A + (size_t)s * astride;
  bool bad = false;
  for (int c = blockIdx.y * 64 + threadIdx.y; c < min(ns, (int)(blockIdx.y + 1) * 64); c += 8) {
    const double wx = W[((size_t)s * n + c) * 2], wy = W[((size_t)s * n + c) * 2 + 1];
    const double z = fma(wx, px, fma(wy, py, bias[(size_t)s * n + c]));
    const double t = tanh(z);
    bad |= !isfinite(z);
    As[f + (size_t)c * mfld] = fma(wx, nx, wy * ny) * (1.0 - t * t);
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

// Copy of one kind of row (0 interior, 1 boundary, 2 interface points, 3 interface
// normals) of every subdomain into out [N][kmax][2], zero-padded past each count.
__global__ void k_get_points(const double* __restrict__ xy, const double* __restrict__ nrm, int m_max,
                             const int* __restrict__ cnt, int kind, int kmax, double* __restrict__ out) {
  const int s = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kmax) return;
  const int mi = cnt[3 * s], mb = cnt[3 * s + 1], mg = cnt[3 * s + 2];
  const int k = kind > 2 ? 2 : kind;
  const int off = k == 0 ? 0 : (k == 1 ? mi : mi + mb), count = k == 0 ? mi : (k == 1 ? mb : mg);
  const double* src = kind == 3 ? nrm : xy;
  double a = 0.0, b = 0.0;
  if (i < count) {
    a = src[((size_t)s * m_max + off + i) * 2];
    b = src[((size_t)s * m_max + off + i) * 2 + 1];
  }
  out[((size_t)s * kmax + i) * 2] = a;
  out[((size_t)s * kmax + i) * 2 + 1] = b;
}

// Warp per column: E = biased exponent of 1.0001 sqrt(sum of squares) over the rows.
__global__ void __launch_bounds__(256) k_colexp(const double* __restrict__ K, long long kstride, int ld,
                                               int ncap, const int* __restrict__ ms, int* __restrict__ colexp) {
  const int s = blockIdx.y, lane = threadIdx.x & 31;
  const int j = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (j >= ncap) return;
  const int m = ms[s];
  const double* col = K + (size_t)s * kstride + (size_t)j * ld;
  double acc = 0.0;
  for (int r = lane; r < m; r += 32) acc = fma(col[r], col[r], acc);
  acc = warp_sum(acc);
  if (lane == 0) {
    const double b = sqrt(acc) * 1.0001;
    colexp[(size_t)s * ncap + j] = acc > 0.0 ? (int)((__double_as_longlong(b) >> 52) & 0x7FF) : 0;
  }
}

}  // namespace

cudaError_t launch_colexp(const double* K, long long kstride, int ld, int ncap, const int* ms, int N,
                          int* colexp, cudaStream_t st) {
  k_colexp<<<dim3((ncap + 7) / 8, N), 256, 0, st>>>(K, kstride, ld, ncap, ms, colexp); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_get_points(const double* xy, const double* nrm, int m_max, const int* cnt, int N,
                              int kind, int kmax, double* out, cudaStream_t st) {
  if (kmax <= 0 || N <= 0) return cudaSuccess;
  k_get_points<<<dim3((kmax + 127) / 128, N), 128, 0, st>>>(xy, nrm, m_max, cnt, kind, kmax, out);
  count_launch();
  return cudaGetLastError();
}

// Tikhonov rows of subdomain s (one CTA): lambda = alpha * the largest column norm of K^s
// over its collocation rows and real columns, then K[ms + (n - n_s) + j][j] = lambda for
// j < n_s (the rows were written as zeros by the assembly).
__global__ void __launch_bounds__(256) k_ridge_rows(double* __restrict__ K, long long kstride, int ld,
                                                   const int* __restrict__ cnt, const int* __restrict__ nsub,
                                                   int n, double alpha) {
  const int s = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ms = cnt[3 * s] + cnt[3 * s + 1] + cnt[3 * s + 2], ns = nsub[s];
  double* Ks = K + (size_t)s * kstride;
  __shared__ double wmax[8];
  double mx = 0.0;
  for (int j = warp; j < ns; j += 8) {
    double a = 0.0;
    for (int r = lane; r < ms; r += 32) a = fma(Ks[r + (size_t)j * ld], Ks[r + (size_t)j * ld], a);
    a = warp_sum(a);
    mx = fmax(mx, a);
  }
  if (lane == 0) wmax[warp] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < 8; ++w) m = fmax(m, wmax[w]);
    wmax[0] = alpha * sqrt(m);
  }
  __syncthreads();
  const double lam = wmax[0];
  const int r0 = ms + (n - ns);
  for (int j = threadIdx.x; j < ns; j += 256) Ks[(r0 + j) + (size_t)j * ld] = lam;
}

cudaError_t launch_ridge_rows(double* K, long long kstride, int ld, const int* cnt, const int* nsub, int N, int n,
                              double alpha, cudaStream_t st) {
  k_ridge_rows<<<N, 256, 0, st>>>(K, kstride, ld, cnt, nsub, n, alpha); count_launch();
  return cudaGetLastError();
}

__global__ void k_zero_pad_theta(double* __restrict__ W, double* __restrict__ b, const int* __restrict__ nsub,
                                 int n) {
  const int s = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n || j < nsub[s]) return;
  W[((size_t)s * n + j) * 2] = 0.0;
  W[((size_t)s * n + j) * 2 + 1] = 0.0;
  b[(size_t)s * n + j] = 0.0;
}

cudaError_t launch_zero_pad_theta(double* W, double* b, const int* nsub, int N, int n, cudaStream_t st) {
  k_zero_pad_theta<<<dim3((n + 127) / 128, N), 128, 0, st>>>(W, b, nsub, n); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_assemble(double* K, long long kstride, int ld, int ncap, double* Amat,
                            long long astride, int mgld, const double* xy, const double* nrm,
                            int m_max, const int* cnt, const double* W, const double* b, int N,
                            int n, const double* coef, const AsmTables* tb, unsigned* status,
                            cudaStream_t st, const int* nsub) {
  dim3 grid((ld + AR - 1) / AR, (ncap + AC - 1) / AC, N);
  if (tb && tb->rix) {
    const long long per = (long long)n * (tb->nxmax + tb->nymax);
    if (per > 0) {
      k_exp_tables<<<dim3((unsigned)((per + 255) / 256), N), 256, 0, st>>>(W, b, n, *tb); count_launch();
    }
    k_assemble<true><<<grid, dim3(AR, 4), 0, st>>>(K, kstride, ld, ncap, Amat, astride, mgld, xy, nrm,
                                                   m_max, cnt, W, b, n, coef, *tb, status, nsub);
    count_launch();
  } else {
    k_assemble<false><<<grid, dim3(AR, 4), 0, st>>>(K, kstride, ld, ncap, Amat, astride, mgld, xy, nrm,
                                                    m_max, cnt, W, b, n, coef, AsmTables{}, status, nsub);
    count_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_flux_rows(double* A, long long astride, int mfld, const int* mf, int mfmax,
                             const int* frow, const double* fnrm, const double* xy, int m_max,
                             const double* W, const double* b, int N, int n, const int* nsub,
                             unsigned* status, cudaStream_t st) {
  if (mfmax <= 0 || N <= 0) return cudaSuccess;
  k_flux_rows<<<dim3((mfmax + 31) / 32, (n + 63) / 64, N), dim3(32, 8), 0, st>>>(
      A, astride, mfld, mf, frow, fnrm, xy, m_max, W, b, n, nsub, status);
  count_launch();
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
