// Step (b): batched blocked Householder QR of the local matrices [K^s | J], the
// triangular solve Y_s = A^s R_s^{-1}, and the per-subdomain kernels of the RHS path
// and of step (d) (q_s = Q_s^T F^s, interface vectors, back-solve).
//
// Householder QR (not the normal equations the paper writes for K^+, Section 3) is
// used because the tanh feature matrices are numerically rank deficient
// (min|R_ii|/max|R_ii| ~ 1e-19 on the 8x8 Poisson workload); Q_G must come from the
// reflectors themselves, since forming it as K_G R^{-1} loses all accuracy.
//
// Reflectors follow the LAPACK convention: H_j = I - tau_j v_j v_j^T, v_j(j) = 1,
// stored below the diagonal of K; each panel of QR_NB columns keeps the upper
// triangular T with H_1 ... H_nb = I - V T V^T, so Q^T = I - V T^T V^T per panel.
#include "common.cuh"

#include <cooperative_groups.h>

namespace elmddm {

namespace {

// One block per subdomain: factor the panel of columns [k0, k0+nbe) over rows [k0, m_s)
// (the fallback for panels whose rows do not fit in the shared memory of an 8-CTA cluster).
__global__ void __launch_bounds__(256) k_panel_qr(double* __restrict__ K, long long kstride, int ld,
                                                  const int* __restrict__ ms_arr, int k0, int nbe,
                                                  double* __restrict__ tau_out, int n,
                                                  double* __restrict__ Vp, long long vstride,
                                                  unsigned* status, int vrow0) {
  const int s = blockIdx.x;
  double* A = K + (size_t)s * kstride;
  const int m = ms_arr[s];
  __shared__ double red[33];
  __shared__ double wred[8][32];
  __shared__ double d[32];
  __shared__ double stau[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned bits = 0;
  __syncthreads();

  for (int j = 0; j < nbe; ++j) {
    const int c = k0 + j;
    double* ac = A + (size_t)c * ld;
    // Norm of the part below the diagonal.
    double p = 0.0;
    for (int r = c + 1 + tid; r < m; r += 256) {
      const double v = ac[r];
      p = fma(v, v, p);
    }
    p = block_sum(p, red);
    const double alpha = (c < m) ? ac[c] : 0.0;
    double beta, tau, scal;
    if (p == 0.0) {
      tau = 0.0; beta = alpha; scal = 1.0;
    } else {
      beta = -copysign(sqrt(fma(alpha, alpha, p)), alpha);
      tau = (beta - alpha) / beta;
      scal = 1.0 / (alpha - beta);
    }
    if (tid == 0) {
      if (beta == 0.0) bits |= ST_RANK;
      if (!isfinite(beta)) bits |= ST_NONFINITE;
    }
    if (p != 0.0)
      for (int r = c + 1 + tid; r < m; r += 256) ac[r] *= scal;
    __syncthreads();

    // d_k = v_j . (column k0+k) over rows >= c: for k > j the w of H_j applied to column k
    double acc[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) acc[k] = 0.0;
    for (int r = c + 1 + tid; r < m; r += 256) {
      const double v = ac[r];
      const double* row = A + r + (size_t)k0 * ld;
#pragma unroll
      for (int k = 0; k < 32; ++k)
        if (k < nbe && k != j) acc[k] = fma(v, row[(size_t)k * ld], acc[k]);
    }
    const double ws = warp_transpose_sum32(acc);
    wred[warp][lane] = ws;
    __syncthreads();
    if (tid < 32) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < 8; ++w) t += wred[w][tid];
      if (tid < nbe && tid != j && c < m) t += A[c + (size_t)(k0 + tid) * ld];
      d[tid] = t;
    }
    __syncthreads();

    if (tau != 0.0) {
      for (int r = c + tid; r < m; r += 256) {
        const double tv = tau * ((r == c) ? 1.0 : ac[r]);
        double* row = A + r + (size_t)k0 * ld;
        for (int k = j + 1; k < nbe; ++k) row[(size_t)k * ld] = fma(-tv, d[k], row[(size_t)k * ld]);
      }
    }
    if (tid == 0) {
      stau[j] = tau;
      if (c < m) ac[c] = beta;
    }
    __syncthreads();
  }

  if (tid < nbe) tau_out[(size_t)s * n + k0 + tid] = stau[tid];
  double* V = Vp + (size_t)s * vstride;
  const int rows = m - k0;
  if (rows > 0) {
    for (int e = tid; e < rows * nbe; e += 256) {
      const int r = k0 + e % rows, j = e / rows;
      const double v = r < k0 + j ? 0.0 : (r == k0 + j ? 1.0 : A[r + (size_t)(k0 + j) * ld]);
      V[r + (size_t)j * ld] = v;
    }
  }
  // rows [vrow0, k0) of these columns of V: zero, for a reflector block that starts above
  for (int e = tid; e < (k0 - vrow0) * nbe; e += 256)
    V[vrow0 + e % (k0 - vrow0) + (size_t)(e / (k0 - vrow0)) * ld] = 0.0;
  if (tid == 0 && bits) atomicOr(status, bits);
}

// Y = A R^{-1} for a tile of 32 rows of Y (one subdomain), in place over A.
__global__ void __launch_bounds__(256) k_trsm_y(double* __restrict__ Y, long long ystride, int mgld,
                                                const double* __restrict__ K, long long kstride,
                                                int ld, const int* __restrict__ mg_arr, int n) {
  const int s = blockIdx.y, i0 = blockIdx.x * 32;
  const int mg = mg_arr[s];
  if (i0 >= mg) return;
  double* Ys = Y + (size_t)s * ystride;
  const double* R = K + (size_t)s * kstride;
  __shared__ double sY[32][33];
  __shared__ double sR[32][33];
  const int t = threadIdx.x, ri = t & 31, cg = (t >> 5) * 4;
  const bool row_ok = (i0 + ri) < mg;
  for (int jb = 0; jb < n; jb += 32) {
    const int nbj = min(32, n - jb);
    double acc[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int cc = jb + cg + q;
      acc[q] = (row_ok && cc < n) ? Ys[(i0 + ri) + (size_t)cc * mgld] : 0.0;
    }
    for (int l0 = 0; l0 < jb; l0 += 32) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int e = t + 256 * q, r = e & 31, cc = e >> 5;
        sY[r][cc] = (i0 + r < mg) ? Ys[(i0 + r) + (size_t)(l0 + cc) * mgld] : 0.0;
        sR[r][cc] = (jb + cc < n) ? R[(l0 + r) + (size_t)(jb + cc) * ld] : 0.0;
      }
      __syncthreads();
#pragma unroll 8
      for (int l = 0; l < 32; ++l) {
        const double y = sY[ri][l];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q] = fma(-y, sR[l][cg + q], acc[q]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) sY[ri][cg + q] = acc[q];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = t + 256 * q, r = e & 31, cc = e >> 5;
      sR[r][cc] = (r <= cc && cc < nbj) ? R[(jb + r) + (size_t)(jb + cc) * ld] : 0.0;
    }
    __syncthreads();
    if (t < 32) {
      for (int c2 = 0; c2 < nbj; ++c2) {
        double x = sY[ri][c2];
        for (int l = 0; l < c2; ++l) x = fma(-sY[ri][l], sR[l][c2], x);
        sY[ri][c2] = x / sR[c2][c2];
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int cc = jb + cg + q;
      if (row_ok && cc < n) Ys[(i0 + ri) + (size_t)cc * mgld] = sY[ri][cg + q];
    }
    __syncthreads();
  }
}

// Diagonal step of the blocked Y R = A solve: for the 64 columns c0.. of Y (already
// updated with the blocks to their left), Y_b <- Y_b R_bb^{-1} by substitution, one row of
// Y per thread.  The thread's row and R_bb live in shared memory (row stride 65: the
// threads' own-row reads are conflict-free, R reads are broadcasts); columns past n are
// padded with an identity block.
constexpr int TRSMY_NB = 64;
__global__ void __launch_bounds__(64) k_trsm_y_diag(double* __restrict__ Y, long long ystride, int mgld,
                                                    const double* __restrict__ K, long long kstride,
                                                    int ld, const int* __restrict__ mg_arr, int n,
                                                    int c0) {
  extern __shared__ double trsmy_smem[];
  double (*sR)[TRSMY_NB + 1] = reinterpret_cast<double (*)[TRSMY_NB + 1]>(trsmy_smem);
  double (*sy)[TRSMY_NB + 1] = reinterpret_cast<double (*)[TRSMY_NB + 1]>(trsmy_smem + TRSMY_NB * (TRSMY_NB + 1));
  __shared__ double rdg[TRSMY_NB];
  const int s = blockIdx.y, i0 = blockIdx.x * 64, t = threadIdx.x;
  const int mg = mg_arr[s];
  if (i0 >= mg) return;
  const int nbe = min(TRSMY_NB, n - c0);
  const double* R = K + (size_t)s * kstride;
  double* Ys = Y + (size_t)s * ystride;
  for (int e = t; e < TRSMY_NB * TRSMY_NB; e += 64) {
    const int r = e % TRSMY_NB, c = e / TRSMY_NB;
    double v = (r == c) ? 1.0 : 0.0;
    if (r <= c && c < nbe) v = R[(c0 + r) + (size_t)(c0 + c) * ld];
    sR[r][c] = v;
    sy[r][c] = (i0 + r < mg && c < nbe) ? Ys[(i0 + r) + (size_t)(c0 + c) * mgld] : 0.0;
  }
  __syncthreads();
  rdg[t] = 1.0 / sR[t][t];
  __syncthreads();
  for (int c = 0; c < nbe; ++c) {
    double x = sy[t][c];
#pragma unroll 8
    for (int k = 0; k < c; ++k) x = fma(-sy[t][k], sR[k][c], x);
    sy[t][c] = x * rdg[c];
  }
  __syncthreads();
  for (int e = t; e < TRSMY_NB * TRSMY_NB; e += 64) {
    const int r = e % TRSMY_NB, c = e / TRSMY_NB;
    if (i0 + r < mg && c < nbe) Ys[(i0 + r) + (size_t)(c0 + c) * mgld] = sy[r][c];
  }
}

// X[r][s][row] = F^s: f/g on interior and boundary rows, zero elsewhere.
__global__ void k_load_rhs(double* __restrict__ X, const double* __restrict__ rhs, int N,
                           int m_max, int ld, const int* __restrict__ cnt, unsigned* status) {
  const int s = blockIdx.y, rh = blockIdx.z;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= ld) return;
  const int mb_end = cnt[3 * s] + cnt[3 * s + 1];
  double v = 0.0;
  if (row < mb_end) {
    v = rhs[((size_t)rh * N + s) * m_max + row];
    if (!isfinite(v)) atomicOr(status, ST_NONFINITE);
  }
  X[((size_t)rh * N + s) * ld + row] = v;
}

// x <- Q^T x for each subdomain and right-hand side, panel by panel (x -= V T^T V^T x),
// with a cluster of AQ_CL CTAs per (subdomain, right-hand side) so that every SM's FP64
// pipe takes part (one CTA per subdomain left most SMs idle).
// The 32-row groups of x are dealt round-robin to the CTAs (group g to CTA g % AQ_CL),
// which keeps the shrinking active rows (r >= k0) balanced; each row stays with one
// thread for both phases of a panel, so x needs no synchronisation.  Per panel: the
// CTA's 32 partial dot products V^T x (warp transpose-sums, then the warps' sums), one
// cluster barrier, every CTA adds the AQ_CL partials through distributed shared memory
// (double-buffered by panel parity, so one barrier per panel suffices), w2 = T^T w with
// all threads, and x -= V w2 on the CTA's rows.
constexpr int AQ_CL = 4;
__global__ void __cluster_dims__(AQ_CL, 1, 1) __launch_bounds__(256)
    k_apply_qt_cl(double* __restrict__ X, const double* __restrict__ K, long long kstride, int ld,
                  const int* __restrict__ ms_arr, int N, int n, const double* __restrict__ Tb,
                  long long tstride) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int c = (int)cluster.block_rank();
  const int s = blockIdx.y, rh = blockIdx.z;
  const int m = ms_arr[s];
  double* x = X + ((size_t)rh * N + s) * ld;
  const double* A = K + (size_t)s * kstride;
  const double* Ts = Tb + (size_t)s * tstride;
  __shared__ double wred[8][32];
  __shared__ double part[2][32];  // this CTA's partial V^T x, by panel parity
  __shared__ double w[32], w2p[8][32], w2[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ngroups = (m + 31) / 32;
  for (int k0 = 0, pan = 0; k0 < n; k0 += 32, ++pan) {
    const int nbe = min(32, n - k0), par = pan & 1;
    // owned groups g >= k0 / 32 with g % AQ_CL == c; warp w takes every 8th of them
    int g0 = k0 / 32;
    g0 += (c - g0 % AQ_CL + AQ_CL) % AQ_CL;
    double acc[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) acc[k] = 0.0;
    for (int g = g0 + warp * AQ_CL; g < ngroups; g += 8 * AQ_CL) {
      const int r = g * 32 + lane;
      if (r >= m) continue;
      const double xr = x[r];
      const double* row = A + r + (size_t)k0 * ld;
      if (r >= k0 + 32) {
#pragma unroll
        for (int k = 0; k < 32; ++k)
          if (k < nbe) acc[k] = fma(row[(size_t)k * ld], xr, acc[k]);
      } else {  // the panel's own 32 rows: unit diagonal, zeros above
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          if (k < nbe) {
            if (r > k0 + k) acc[k] = fma(row[(size_t)k * ld], xr, acc[k]);
            else if (r == k0 + k) acc[k] += xr;
          }
        }
      }
    }
    const double ws = warp_transpose_sum32(acc);
    wred[warp][lane] = ws;
    __syncthreads();
    if (tid < 32) {
      double t = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) t += wred[q][tid];
      part[par][tid] = t;
    }
    cluster.sync();
    if (tid < 32) {
      double t = 0.0;
#pragma unroll
      for (int q = 0; q < AQ_CL; ++q) t += cluster.map_shared_rank(&part[par][0], q)[tid];
      w[tid] = tid < nbe ? t : 0.0;
    }
    __syncthreads();
    {  // w2 = T^T w, T upper triangular: w2_i = sum_{j <= i} T[j][i] w_j, 4 terms per thread
      const int i = lane, j0 = warp * 4;
      const double* Tk = Ts + (size_t)pan * 1024;
      double t = 0.0;
#pragma unroll
      for (int j = j0; j < j0 + 4; ++j)
        if (j <= i) t = fma(Tk[j + 32 * i], w[j], t);
      w2p[warp][i] = t;
    }
    __syncthreads();
    if (tid < 32) {
      double t = 0.0;
#pragma unroll
      for (int q = 0; q < 8; ++q) t += w2p[q][tid];
      w2[tid] = t;
    }
    __syncthreads();
    for (int g = g0 + warp * AQ_CL; g < ngroups; g += 8 * AQ_CL) {
      const int r = g * 32 + lane;
      if (r >= m) continue;
      double xr = x[r];
      const double* row = A + r + (size_t)k0 * ld;
      if (r >= k0 + 32) {
#pragma unroll
        for (int k = 0; k < 32; ++k)
          if (k < nbe) xr = fma(-row[(size_t)k * ld], w2[k], xr);
      } else {
        for (int k = 0; k < nbe; ++k) {
          const double v = r > k0 + k ? row[(size_t)k * ld] : (r == k0 + k ? 1.0 : 0.0);
          xr = fma(-v, w2[k], xr);
        }
      }
      x[r] = xr;
    }
    __syncthreads();
  }
  cluster.sync();  // no CTA leaves while another may still read its partials
}

// gq = Q_G q and hq = Y q for each subdomain / right-hand side.  A block takes IV_GROWS
// rows of gq, a warp each with lanes over the contiguous columns of Q_G^T, and IV_HROWS
// rows of hq, a lane each (Y is column-major, so a warp reads 32 consecutive rows of one
// column) with the n columns split over the 8 warps and summed in shared memory.  Both
// loops issue 4 loads before their first FMA.
constexpr int IV_GROWS = 8;
constexpr int IV_HROWS = 32;
__global__ void __launch_bounds__(256) k_iface_vecs(const double* __restrict__ X,
                                                    const double* __restrict__ K, long long kstride,
                                                    int ld, const double* __restrict__ Y,
                                                    long long ystride, int mgld,
                                                    const int* __restrict__ mg_arr, int mfld,
                                                    const int* __restrict__ mf_arr, int N, int n,
                                                    double* __restrict__ gq,
                                                    double* __restrict__ hq) {
  __shared__ double part[8][IV_HROWS];
  const int s = blockIdx.x, rh = blockIdx.y, b = blockIdx.z;
  const int mg = mg_arr[s], mf = mf_arr[s];
  const double* q = X + ((size_t)rh * N + s) * ld;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = b * IV_GROWS + warp;
  if (i < mg) {
    const double* row = K + (size_t)s * kstride + (size_t)n * ld + (size_t)i * ld;  // row i of Q_G
    double a = 0.0;
    int j = lane;
    for (; j + 96 < n; j += 128) {
      const double r0 = row[j], r1 = row[j + 32], r2 = row[j + 64], r3 = row[j + 96];
      const double q0 = q[j], q1 = q[j + 32], q2 = q[j + 64], q3 = q[j + 96];
      a = fma(r0, q0, a);
      a = fma(r1, q1, a);
      a = fma(r2, q2, a);
      a = fma(r3, q3, a);
    }
    for (; j < n; j += 32) a = fma(row[j], q[j], a);
    a = warp_sum(a);
    if (lane == 0) gq[((size_t)rh * N + s) * mgld + i] = a;
  }
  if (b * IV_HROWS >= mf) return;  // uniform over the block
  const int r = b * IV_HROWS + lane;
  double acc = 0.0;
  if (r < mf) {
    const double* col = Y + (size_t)s * ystride + r;
    const int j1 = (int)(((long long)n * (warp + 1)) / 8);
    int j = (int)(((long long)n * warp) / 8);
    for (; j + 3 < j1; j += 4) {
      const double y0 = col[(size_t)j * mfld], y1 = col[(size_t)(j + 1) * mfld];
      const double y2 = col[(size_t)(j + 2) * mfld], y3 = col[(size_t)(j + 3) * mfld];
      acc = fma(y0, q[j], acc);
      acc = fma(y1, q[j + 1], acc);
      acc = fma(y2, q[j + 2], acc);
      acc = fma(y3, q[j + 3], acc);
    }
    for (; j < j1; ++j) acc = fma(col[(size_t)j * mfld], q[j], acc);
  }
  part[warp][lane] = acc;
  __syncthreads();
  if (warp == 0 && r < mf) {
    double t = part[0][lane];
#pragma unroll
    for (int w = 1; w < 8; ++w) t += part[w][lane];
    hq[((size_t)rh * N + s) * mfld + r] = t;
  }
}

// out[g] (+)= the sum of a[s][l] over the (s, l) pairs of entry g (2 to kmax of them).
__global__ void k_gather2(const int* __restrict__ map, int kmax, int n, int ldv, int N,
                          const double* __restrict__ a, double* __restrict__ out, int accumulate) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x, rh = blockIdx.y;
  if (g >= n) return;
  const int* m = map + (size_t)2 * kmax * g;
  double v = a[((size_t)rh * N + m[0]) * ldv + m[1]] + a[((size_t)rh * N + m[2]) * ldv + m[3]];
  for (int q = 2; q < kmax && m[2 * q] >= 0; ++q) v += a[((size_t)rh * N + m[2 * q]) * ldv + m[2 * q + 1]];
  double* o = out + (size_t)rh * n + g;
  *o = accumulate ? *o + v : v;
}

// dst[r][g] = src[r][idx[g]].
__global__ void k_gather_perm(const int* __restrict__ idx, int n, const double* __restrict__ src,
                              double* __restrict__ dst) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x, rh = blockIdx.y;
  if (g < n) dst[(size_t)rh * n + g] = src[(size_t)rh * n + idx[g]];
}

// z_s = M_s^T (P_s h) (warp per column of M_s; P_s = E_s without explicit flux rows).
__global__ void __launch_bounds__(256) k_mt_h(const double* __restrict__ M, long long mstride, int mfld,
                                              const int* __restrict__ mf_arr,
                                              const int* __restrict__ mg_arr,
                                              const int* __restrict__ ffd,
                                              const double* __restrict__ h, int n_flux, int N, int mgld,
                                              double* __restrict__ z) {
  const int s = blockIdx.x, rh = blockIdx.y;
  const int mg = mg_arr[s], mf = mf_arr[s];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.z * 8 + warp;
  if (i >= mg) return;
  const double* col = M + (size_t)s * mstride + (size_t)i * mfld;  // column i of M_s
  const int* fds = ffd + (size_t)s * mfld;
  const double* hh = h + (size_t)rh * n_flux;
  double a = 0.0;
  int k = lane;
  for (; k + 96 < mf; k += 128) {  // 4 loads in flight, summed in the same order
    const double m0 = col[k], m1 = col[k + 32], m2 = col[k + 64], m3 = col[k + 96];
    const int f0 = fds[k], f1 = fds[k + 32], f2 = fds[k + 64], f3 = fds[k + 96];
    a = fma(m0, hh[f0], a);
    a = fma(m1, hh[f1], a);
    a = fma(m2, hh[f2], a);
    a = fma(m3, hh[f3], a);
  }
  for (; k < mf; k += 32) a = fma(col[k], hh[fds[k]], a);
  a = warp_sum(a);
  if (lane == 0) z[((size_t)rh * N + s) * mgld + i] = a;
}

// c^s = R^{-1} (q + Q_G^T E_s u), one block per (subdomain, right-hand side).
__global__ void __launch_bounds__(256) k_backsolve(const double* __restrict__ X,
                                                   const double* __restrict__ K, long long kstride,
                                                   int ld, const int* __restrict__ mg_arr,
                                                   const int* __restrict__ ifc_dof, int mgld,
                                                   const double* __restrict__ u, int n_gamma, int N,
                                                   int n, double* __restrict__ cout) {
  extern __shared__ double v[];
  const int s = blockIdx.x, rh = blockIdx.y;
  const int mg = mg_arr[s];
  const double* q = X + ((size_t)rh * N + s) * ld;
  const double* A = K + (size_t)s * kstride;
  const double* QGt = A + (size_t)n * ld;
  const int* dofs = ifc_dof + (size_t)s * mgld;
  const double* uu = u + (size_t)rh * n_gamma;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int j = tid; j < n; j += 256) {
    double a = q[j];
    for (int i = 0; i < mg; ++i) a = fma(QGt[j + (size_t)i * ld], uu[dofs[i]], a);
    v[j] = a;
  }
  __syncthreads();
  for (int jb = ((n - 1) / 32) * 32; jb >= 0; jb -= 32) {
    const int nbj = min(32, n - jb);
    if (warp == 0) {
      for (int j = jb + nbj - 1; j >= jb; --j) {
        const double cj = v[j] / A[j + (size_t)j * ld];
        __syncwarp();
        if (lane == 0) v[j] = cj;
        if (lane < j - jb) v[jb + lane] = fma(-A[(jb + lane) + (size_t)j * ld], cj, v[jb + lane]);
        __syncwarp();
      }
    }
    __syncthreads();
    for (int i = tid; i < jb; i += 256) {
      double t = v[i];
      for (int l = 0; l < nbj; ++l) t = fma(-A[i + (size_t)(jb + l) * ld], v[jb + l], t);
      v[i] = t;
    }
    __syncthreads();
  }
  double* co = cout + ((size_t)rh * N + s) * n;
  for (int j = tid; j < n; j += 256) co[j] = v[j];
}


// k_backsolve with a cluster of AQ_CL CTAs per (subdomain, right-hand side).  Entry j of
// v and the rows of R it heads belong to CTA (j / 32) % AQ_CL.  Each CTA forms its own
// entries of v = q + Q_G^T E u_Gamma, then for each 32-column block of R from the last:
// the owning CTA solves the block's triangle (one warp, multiplying by the stored
// reciprocals of R's diagonal), one cluster barrier, every CTA reads the block's 32
// results from the owner's shared memory and updates its own entries above the block.
// The owner of the next block has applied every earlier block before it starts, since
// it reads them after the barriers in order.
__global__ void __cluster_dims__(AQ_CL, 1, 1) __launch_bounds__(256)
    k_backsolve_cl(const double* __restrict__ X, const double* __restrict__ K, long long kstride,
                   int ld, const int* __restrict__ mg_arr, const int* __restrict__ ifc_dof, int mgld,
                   const double* __restrict__ u, int n_gamma, int N, int n, double* __restrict__ cout) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int c = (int)cluster.block_rank();
  extern __shared__ double bs_smem[];
  double* v = bs_smem;            // [n]: this CTA's entries (others unused)
  double* rinv = bs_smem + n;     // [n]: 1 / R_jj for this CTA's entries
  double* ug = bs_smem + 2 * n;   // [mg]: u_Gamma at this subdomain's interface rows
  __shared__ double cb[32];
  const int s = blockIdx.y, rh = blockIdx.z;
  const int mg = mg_arr[s];
  const double* q = X + ((size_t)rh * N + s) * ld;
  const double* A = K + (size_t)s * kstride;
  const double* QGt = A + (size_t)n * ld;
  const int* dofs = ifc_dof + (size_t)s * mgld;
  const double* uu = u + (size_t)rh * n_gamma;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ng32 = (n + 31) / 32;
  for (int i = tid; i < mg; i += 256) ug[i] = uu[dofs[i]];
  __syncthreads();
  // owned entry number e -> j = ((e / 32) * AQ_CL + c) * 32 + e % 32
  const int owned = ((ng32 - c + AQ_CL - 1) / AQ_CL) * 32;
  for (int e = tid; e < owned; e += 256) {
    const int j = ((e / 32) * AQ_CL + c) * 32 + (e % 32);
    if (j >= n) continue;
    double a = q[j];
    for (int i = 0; i < mg; ++i) a = fma(QGt[j + (size_t)i * ld], ug[i], a);
    v[j] = a;
    rinv[j] = 1.0 / A[j + (size_t)j * ld];
  }
  __syncthreads();
  for (int jb = (ng32 - 1) * 32; jb >= 0; jb -= 32) {
    const int nbj = min(32, n - jb), own = (jb / 32) % AQ_CL;
    if (c == own && warp == 0) {
      for (int j = jb + nbj - 1; j >= jb; --j) {
        const double cj = v[j] * rinv[j];
        __syncwarp();
        if (lane == 0) v[j] = cj;
        if (lane < j - jb) v[jb + lane] = fma(-A[(jb + lane) + (size_t)j * ld], cj, v[jb + lane]);
        __syncwarp();
      }
    }
    cluster.sync();
    if (tid < 32) cb[tid] = tid < nbj ? cluster.map_shared_rank(v, own)[jb + tid] : 0.0;
    __syncthreads();
    // this CTA's entries above the block
    const int owned_above = ((jb / 32 - c + AQ_CL - 1) / AQ_CL) * 32;
    for (int e = tid; e < owned_above; e += 256) {
      const int i = ((e / 32) * AQ_CL + c) * 32 + (e % 32);
      double t = v[i];
      const double* Ar = A + i + (size_t)jb * ld;
#pragma unroll 8
      for (int l = 0; l < nbj; ++l) t = fma(-Ar[(size_t)l * ld], cb[l], t);
      v[i] = t;
    }
    __syncthreads();
  }
  double* co = cout + ((size_t)rh * N + s) * n;
  for (int e = tid; e < owned; e += 256) {
    const int j = ((e / 32) * AQ_CL + c) * 32 + (e % 32);
    if (j < n) co[j] = v[j];
  }
  cluster.sync();  // no CTA leaves while another may still read its results
}

constexpr int PLD = 33;    // shared-memory row stride of the panel chunk (doubles)

// Cluster variant of the panel factorisation: the PCL CTAs of a cluster share one
// subdomain's panel, each holding a contiguous slice of its rows in shared memory.
// Column j of the panel takes two phases over the CTA's rows, with the threads mapped to
// (column, row subset) pairs of the columns still active, so that no FP64 work goes to
// columns already factored and the cross-thread reduction is one add per partial:
//   phase 1: for the active columns k = j .. nbe-1, y_k = sum of x_r a_k(r) over the rows
//            strictly below the diagonal row c = k0 + j (k = j gives sigma = |x_below|^2);
//            partials are summed within each warp (lanes 32 apart modulo the column
//            count hold the same column), across the 8 warps, then across the cluster
//            through distributed shared memory in a fixed order, so every CTA computes the
//            identical reflector;
//   then     beta = -sign(alpha) sqrt(alpha^2 + sigma),  tau = (beta - alpha) / beta,
//            v = (x - beta e_c) / (alpha - beta),  v^T a_k = a_k(c) + y_k / (alpha - beta);
//   phase 2: a_k -= tau v (v^T a_k) for k > j on the rows from c down, written as
//            a_k(c) -= tau (v^T a_k) and a_k(r) -= [tau (v^T a_k) / (alpha - beta)] x_r,
//            so column j itself is scaled into v only once, when the panel is written back.
// The compact-WY factor T is not formed here: the products v_l^T v_j (l < j) it needs come
// out of the next W1 = V^T A2 product as its first rows (k_form_t).  T = double is the
// FP64 path; T = float gives the low-precision factorisation of the mixed-precision mode
// (the FP32 pipe is some 60 times the FP64 pipe; every value stays FP32 until the panel
// is written back as FP64).
template <int PCL, typename T>
__global__ void __cluster_dims__(PCL, 1, 1) __launch_bounds__(256)
    k_panel_qr_cl(double* __restrict__ K, long long kstride, int ld, const int* __restrict__ ms_arr,
                  int k0, int nbe, double* __restrict__ tau_out, int n, double* __restrict__ Vp,
                  long long vstride, unsigned* status, int s_off, int vrow0) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int q = (int)cluster.block_rank();
  const int s = s_off + blockIdx.y;
  double* A = K + (size_t)s * kstride;
  const int m = ms_arr[s];
  const int mp = m - k0;
  const int rows_per = (mp + PCL - 1) / PCL;
  const int r0 = k0 + q * rows_per;                     // first global row of this chunk
  const int nr = max(0, min(rows_per, m - r0));         // rows held here
  extern __shared__ __align__(16) unsigned char panel_smem[];
  T* P = reinterpret_cast<T*>(panel_smem);              // [rows_per][PLD]
  __shared__ T red[2][64];                         // [parity]: y_k, a_k(c) by column slot
  __shared__ T wred[8][32];                        // per warp, by column slot
  __shared__ T cf[32], cfs[32];                    // tau v^T a_k, and divided by (alpha - beta)
  __shared__ T stau[32], sscal[32];                // tau_j, 1 / (alpha_j - beta_j)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int k = 0; k < nbe; ++k)
    for (int r = tid; r < nr; r += 256) P[r * PLD + k] = (T)A[(r0 + r) + (size_t)(k0 + k) * ld];
  unsigned bits = 0;
  __syncthreads();

  int par = 0;
  for (int j = 0; j < nbe; ++j) {
    const int c = k0 + j;
    const int cl = c - r0;                   // local row of c (valid if 0 <= cl < nr)
    const bool own_c = cl >= 0 && cl < nr;
    const int na = nbe - j;                  // active columns j .. nbe-1, slot = k - j
    {
      const int P1 = 256 / na;
      T acc = 0;
      if (tid < P1 * na) {
        const int col = j + tid % na, p = tid / na;
        for (int r = max(0, cl + 1) + p; r < nr; r += P1) acc = fma(P[r * PLD + j], P[r * PLD + col], acc);
      }
      // lanes l and l + na hold the same column (thread index modulo na)
      for (int o = na; o < 32; o <<= 1) {
        const T v = __shfl_down_sync(0xffffffffu, acc, o);
        if (lane + o < 32) acc += v;
      }
      if (lane < na) wred[warp][(32 * warp + lane) % na] = acc;
    }
    __syncthreads();
    if (warp == 0) {
      T t = 0;
      if (lane < na) {
#pragma unroll
        for (int w = 0; w < 8; ++w) t += wred[w][lane];
      }
      red[par][lane] = t;
      red[par][32 + lane] = (own_c && lane < na) ? P[cl * PLD + j + lane] : (T)0;
    }
    cluster.sync();
    if (warp == 0) {
      T y = 0, rc = 0;
#pragma unroll
      for (int qq = 0; qq < PCL; ++qq) {
        const T* rr = cluster.map_shared_rank(&red[par][0], qq);
        y += rr[lane];
        rc += rr[32 + lane];
      }
      const T alpha = __shfl_sync(0xffffffffu, rc, 0);
      const T ss = __shfl_sync(0xffffffffu, y, 0);
      T beta, tau, scal;
      if (ss == (T)0) {
        tau = 0; beta = alpha; scal = 1;
      } else {
        beta = -copysign(sqrt(fma(alpha, alpha, ss)), alpha);
        tau = (beta - alpha) / beta;
        scal = (T)1 / (alpha - beta);
      }
      const T td = tau * fma(scal, y, rc);  // tau v^T a_k for slot `lane`
      cf[lane] = td;
      cfs[lane] = td * scal;
      if (lane == 0) {
        stau[j] = tau;
        sscal[j] = scal;
        if (q == 0) {
          if (beta == (T)0) bits |= ST_RANK;
          if (!isfinite(beta)) bits |= ST_NONFINITE;
        }
        if (own_c) P[cl * PLD + j] = beta;  // row c: R_jj (read as alpha above)
      }
    }
    __syncthreads();
    const int nu = na - 1;                   // columns j+1 .. nbe-1
    if (nu > 0 && stau[j] != (T)0) {
      const int P2 = 256 / nu;
      if (tid < P2 * nu) {
        const int sl = 1 + tid % nu, col = j + sl, p = tid / nu;
        const T b = cfs[sl];
        if (own_c && p == 0) P[cl * PLD + col] -= cf[sl];
        for (int r = max(0, cl + 1) + p; r < nr; r += P2)
          P[r * PLD + col] = fma(-b, P[r * PLD + j], P[r * PLD + col]);
      }
    }
    __syncthreads();
    par ^= 1;
  }

  // R on and above the diagonal, the reflectors (x scaled into v) below it; V explicit
  double* V = Vp + (size_t)s * vstride;
  for (int k = 0; k < nbe; ++k) {
    const T sc = sscal[k];
    for (int r = tid; r < nr; r += 256) {
      const int gr = r0 + r;
      T tv = P[r * PLD + k];
      if (gr > k0 + k) tv *= sc;
      const double v = (double)tv;
      A[gr + (size_t)(k0 + k) * ld] = v;
      V[gr + (size_t)k * ld] = gr < k0 + k ? 0.0 : (gr == k0 + k ? 1.0 : v);
    }
  }
  if (q == 0) {
    // rows [vrow0, k0) of these columns of V: zero, for a reflector block that starts above
    for (int e = tid; e < (k0 - vrow0) * nbe; e += 256)
      V[vrow0 + e % (k0 - vrow0) + (size_t)(e / (k0 - vrow0)) * ld] = 0.0;
    if (tid < nbe) tau_out[(size_t)s * n + k0 + tid] = (double)stau[tid];
    if (tid == 0 && bits) atomicOr(status, bits);
  }
  cluster.sync();  // peers may still read this CTA's reduction slots
}

// Compact-WY factor of one panel, H_0 ... H_{nb-1} = I - V T V^T (T upper triangular), by
// the forward column recurrence T_jj = tau_j, T(0:j, j) = -tau_j T(0:j, 0:j) g_j with
// g_j(l) = v_l^T v_j, l < j: the first nb rows of the panel's W1 product (G[l * 32 + j]).
// One CTA of 128 threads per subdomain: G and tau are staged in shared memory, and each
// row i of T is shared by 4 threads (every fourth term of the sum, added by shuffles), so
// a column of the recurrence costs a few dependent FMAs.
__global__ void __launch_bounds__(128) k_form_t(const double* __restrict__ G, long long gstride,
                                               const double* __restrict__ tau, int n, int k0, int nbe,
                                               double* __restrict__ Tout, long long tstride) {
  const int s = blockIdx.x, t = threadIdx.x, i = t >> 2, qd = t & 3;
  __shared__ double T[32][33];
  __shared__ double Gs[32][33];
  __shared__ double ts[32];
  const double* Gp = G + (size_t)s * gstride;
  for (int e = t; e < 32 * 32; e += 128) {
    const int l = e >> 5, j = e & 31;
    Gs[l][j] = (l < nbe && j < nbe) ? Gp[e] : 0.0;
    T[l][j] = 0.0;
  }
  if (t < 32) ts[t] = t < nbe ? tau[(size_t)s * n + k0 + t] : 0.0;
  __syncthreads();
  for (int j = 0; j < nbe; ++j) {
    double p = 0.0;
    if (i < j)
      for (int l = i + qd; l < j; l += 4) p = fma(T[i][l], Gs[l][j], p);
    p += __shfl_xor_sync(0xffffffffu, p, 1);
    p += __shfl_xor_sync(0xffffffffu, p, 2);
    if (qd == 0) {
      if (i < j) T[i][j] = -ts[j] * p;
      else if (i == j) T[j][j] = ts[j];
    }
    __syncthreads();
  }
  double* Tp = Tout + (size_t)s * tstride;
  for (int e = t; e < 32 * 32; e += 128) Tp[e] = T[e & 31][e >> 5];
}

// Compact-WY factor of a block of w <= 128 columns spanning several panels, for the
// trailing update of a two-level blocked QR: the forward recurrence of k_form_t,
// T(i, j) = -tau_j sum_{l=i}^{j-1} T(i, l) g_j(l) for j > i, T(i, i) = tau_i, over the
// block's Gram matrix (g_j(l) = v_l^T v_j = G[j][l]).  Row i of T needs only row i's
// earlier entries, so rows are independent: the 8-row groups of a subdomain are dealt
// round-robin to FTW_RS CTAs (the heavy first rows spread over both), a warp owns one
// group with 4 threads per row (each summing every fourth term, 2 shuffles per entry; the
// groups are paired heavy with light on each SM sub-partition), and
// no block barrier is needed after G is staged.  The FP64 work, w^3 / 6 per subdomain, is
// what bounds it; a warp's rows differ by at most 7 in length, so its lanes stay busy.
constexpr int FTW_MAX = 128;
constexpr int FTW_RS = 2;                      // CTAs per subdomain
constexpr int FTW_GLD = FTW_MAX + 1;           // padded row of the staged Gram matrix
constexpr int FTW_ROWS = FTW_MAX / FTW_RS;     // rows of T per CTA
constexpr int FTW_SMEM = (FTW_MAX * FTW_GLD + FTW_ROWS * FTW_MAX + FTW_MAX) * (int)sizeof(double);
static_assert(FTW_ROWS == 64, "8 warps x 8 rows per CTA");

__global__ void __launch_bounds__(256) k_form_t_wide(const double* __restrict__ G, long long gstride, int gld,
                                                    const double* __restrict__ tau, int n, int k0, int w,
                                                    double* __restrict__ Tw, long long twstride, int tld,
                                                    double* __restrict__ Td, long long tdstride, int dcol) {
  extern __shared__ double ftw_smem[];
  double* Gs = ftw_smem;                        // [w][FTW_GLD]: row j holds g_j
  double* Tr = Gs + FTW_MAX * FTW_GLD;          // [FTW_ROWS][FTW_MAX]: this CTA's rows of T
  double* ts = Tr + FTW_ROWS * FTW_MAX;         // [FTW_MAX]
  const int s = blockIdx.x, q = blockIdx.y, t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const double* Gp = G + (size_t)s * gstride;
  for (int e = t; e < w * w; e += 256) {
    const int j = e / w, l = e % w;
    Gs[j * FTW_GLD + l] = Gp[(size_t)j * gld + l];
  }
  if (t < FTW_MAX) ts[t] = t < w ? tau[(size_t)s * n + k0 + t] : 0.0;
  __syncthreads();
  // warp -> 8-row group, 4 threads per row.  This CTA's groups are q, q + FTW_RS, ...
  // (heaviest first); warps w and w + 4 share an SM sub-partition's quarter of the FP64
  // pipe, so warp w < 4 takes the w-th heaviest and warp w + 4 the w-th lightest group.
  const int rank = warp < 4 ? warp : 11 - warp;
  const int grp = rank * FTW_RS + q, r8 = lane >> 2, qd = lane & 3;
  const int i = grp * 8 + r8, slot = warp * 8 + r8;
  double* Ti = Tr + slot * FTW_MAX;
  const bool live = i < w;
  if (live && qd == 0) Ti[i] = ts[i];
  __syncwarp();
  const int j0 = grp * 8 + 1;                   // first j any row of the group needs
  for (int j = j0; j < w; ++j) {
    double acc = 0.0;
    if (live)
      for (int l = i + qd; l < j; l += 4) acc = fma(Ti[l], Gs[j * FTW_GLD + l], acc);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (live && j > i && qd == 0) Ti[j] = -ts[j] * acc;
    __syncwarp();
  }
  if (live) {
    double* Tp = Tw + (size_t)s * twstride;
    for (int j = qd; j < w; j += 4) Tp[(size_t)j * tld + i] = j < i ? 0.0 : Ti[j];
    // the last panel's diagonal 32-block (rows and columns dcol .. dcol + 31)
    if (i >= dcol && i < dcol + 32) {
      double* Dp = Td + (size_t)s * tdstride;
      for (int c = qd; c < 32; c += 4) {
        const int j = dcol + c;
        Dp[(size_t)c * 32 + (i - dcol)] = (j < w && j >= i) ? Ti[j] : 0.0;
      }
    }
  }
  // rows of the diagonal block beyond w (a last panel narrower than 32): zero
  if (q == 0 && t < 32 && dcol + t >= w) {
    double* Dp = Td + (size_t)s * tdstride;
    for (int c = 0; c < 32; ++c) Dp[(size_t)c * 32 + t] = 0.0;
  }
}

}  // namespace

cudaError_t launch_panel_qr(double* K, long long kstride, int ld, const int* ms, int N, int k0,
                            int nbe, double* tau, int n, double* Vp, long long vstride, unsigned* status,
                            cudaStream_t st, bool fp32, int pcl_pref, int vrow0) {
  if (vrow0 < 0 || vrow0 > k0) return cudaErrorInvalidValue;
  // the cluster variant keeps 1/PCL of the rows (up to ld - k0) in shared memory: 4 CTAs
  // per subdomain, or 8 when a quarter of the rows does not fit.  (Splitting the launch
  // into a full wave of 4-CTA clusters and a remainder of 5-CTA clusters measured slower:
  // a cluster has to fit in one GPC, so fewer clusters run at once than SMs / size.)  The
  // FP32 panel needs half the space per row and takes 2 CTAs where they suffice.
  constexpr int kMax = 180 * 1024;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* f) {
      if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kMax);
    };
    set((const void*)k_panel_qr_cl<4, double>); set((const void*)k_panel_qr_cl<8, double>);
    set((const void*)k_panel_qr_cl<2, float>); set((const void*)k_panel_qr_cl<4, float>);
    set((const void*)k_panel_qr_cl<8, float>);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  auto smem = [&](int pcl, size_t bytes) { return (size_t)((ld - k0 + pcl - 1) / pcl) * PLD * bytes; };
#define ELM_PANEL(PCL_, T_)                                                                          \
  k_panel_qr_cl<PCL_, T_><<<dim3(PCL_, N), 256, smem(PCL_, sizeof(T_)), st>>>(K, kstride, ld, ms, k0, nbe, \
                                                                          tau, n, Vp, vstride, status, 0, vrow0)
  if (fp32) {
    if (smem(2, 4) <= kMax) ELM_PANEL(2, float);
    else if (smem(4, 4) <= kMax) ELM_PANEL(4, float);
    else if (smem(8, 4) <= kMax) ELM_PANEL(8, float);
    else return cudaErrorInvalidValue;  // rows beyond the low-precision panel's shared memory
  } else if (pcl_pref == 8 && smem(8, 8) <= kMax) {
    ELM_PANEL(8, double);  // a tile choice: twice the SMs per subdomain (small batches)
  } else if (smem(4, 8) <= kMax) {
    ELM_PANEL(4, double);
  } else if (smem(8, 8) <= kMax) {
    ELM_PANEL(8, double);
  } else {
    k_panel_qr<<<N, 256, 0, st>>>(K, kstride, ld, ms, k0, nbe, tau, n, Vp, vstride, status, vrow0);
  }
#undef ELM_PANEL
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_form_t(const double* G, long long gstride, const double* tau, int n, int k0, int nbe,
                          int N, double* T, long long tstride, cudaStream_t st) {
  k_form_t<<<N, 128, 0, st>>>(G, gstride, tau, n, k0, nbe, T, tstride); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_form_t_wide(const double* G, long long gstride, int gld, const double* tau, int n,
                               int k0, int w, int N, double* Tw, long long twstride, int tld,
                               double* Td, long long tdstride, int dcol, cudaStream_t st) {
  if (w <= 0 || w > FTW_MAX || tld < w || gld < w || dcol < 0 || dcol >= w) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_form_t_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, FTW_SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_form_t_wide<<<dim3(N, FTW_RS), 256, FTW_SMEM, st>>>(G, gstride, gld, tau, n, k0, w, Tw, twstride, tld, Td,
                                                        tdstride, dcol);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_trsm_y(double* Y, long long ystride, int mgld, const double* K,
                          long long kstride, int ld, const int* mg, int mgmax, int N, int n,
                          cudaStream_t st) {
  if (mgmax <= 0) return cudaSuccess;
  k_trsm_y<<<dim3((mgmax + 31) / 32, N), 256, 0, st>>>(Y, ystride, mgld, K, kstride, ld, mg, n); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_trsm_y_diag(double* Y, long long ystride, int mgld, const double* K,
                               long long kstride, int ld, const int* mg, int mgmax, int N, int n,
                               int c0, cudaStream_t st) {
  if (mgmax <= 0 || c0 >= n) return cudaSuccess;
  const int smem = 2 * TRSMY_NB * (TRSMY_NB + 1) * (int)sizeof(double);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_trsm_y_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_trsm_y_diag<<<dim3((mgmax + 63) / 64, N), 64, smem, st>>>(Y, ystride, mgld, K, kstride, ld, mg, n, c0); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_load_rhs(double* X, const double* rhs, int N, int m_max, int ld,
                            const int* cnt, int nrhs, unsigned* status, cudaStream_t st) {
  k_load_rhs<<<dim3((ld + 255) / 256, N, nrhs), 256, 0, st>>>(X, rhs, N, m_max, ld, cnt, status); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_apply_qt(double* X, const double* K, long long kstride, int ld,
                            const int* ms, int N, int n, const double* T, long long tstride,
                            int nrhs, cudaStream_t st) {
  k_apply_qt_cl<<<dim3(AQ_CL, N, nrhs), 256, 0, st>>>(X, K, kstride, ld, ms, N, n, T, tstride); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_iface_vecs(const double* X, const double* K, long long kstride, int ld,
                              const double* Y, long long ystride, int mgld, const int* mg, int mfld,
                              const int* mf, int N, int n, int nrhs, double* gq, double* hq,
                              cudaStream_t st) {
  const int zg = (mgld + IV_GROWS - 1) / IV_GROWS, zh = (mfld + IV_HROWS - 1) / IV_HROWS;
  const int zb = zg > zh ? zg : zh;
  if (N <= 0 || nrhs <= 0 || zb <= 0) return cudaSuccess;
  k_iface_vecs<<<dim3(N, nrhs, zb), 256, 0, st>>>(X, K, kstride, ld, Y, ystride, mgld, mg, mfld, mf, N, n,
                                                  gq, hq); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_gather2(const int* map, int kmax, int n, int ldv, int N, const double* a,
                           double* out, int accumulate, int nrhs, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (kmax < 2) return cudaErrorInvalidValue;
  k_gather2<<<dim3((n + 255) / 256, nrhs), 256, 0, st>>>(map, kmax, n, ldv, N, a, out,
                                                         accumulate); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_gather_perm(const int* idx, int n, const double* src, double* dst, int nrhs,
                               cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_gather_perm<<<dim3((n + 255) / 256, nrhs), 256, 0, st>>>(idx, n, src, dst); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_mt_h(const double* M, long long mstride, int mfld, const int* mf, const int* mg,
                        const int* ffd, const double* h, int n_flux, int N, int mgld, int nrhs,
                        double* z, cudaStream_t st) {
  if (N <= 0 || nrhs <= 0 || mgld <= 0) return cudaSuccess;
  k_mt_h<<<dim3(N, nrhs, (mgld + 7) / 8), 256, 0, st>>>(M, mstride, mfld, mf, mg, ffd, h, n_flux, N, mgld, z);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_backsolve(const double* X, const double* K, long long kstride, int ld,
                             const int* mg, const int* ifc_dof, int mgld, const double* u,
                             int n_gamma, int N, int n, int nrhs, double* c, cudaStream_t st) {
  // v, 1 / R_jj and u_Gamma at the interface rows (mgld >= every subdomain's m_Gamma)
  const size_t smem = (2 * (size_t)n + (size_t)mgld) * sizeof(double);
  if (smem > 227 * 1024) {
    const size_t sm1 = (size_t)n * sizeof(double);
    if (sm1 > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_backsolve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sm1);
      if (e != cudaSuccess) return e;
    }
    k_backsolve<<<dim3(N, nrhs), 256, sm1, st>>>(X, K, kstride, ld, mg, ifc_dof, mgld, u, n_gamma,
                                                 N, n, c); count_launch();
    return cudaGetLastError();
  }
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_backsolve_cl, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_backsolve_cl<<<dim3(AQ_CL, N, nrhs), 256, smem, st>>>(X, K, kstride, ld, mg, ifc_dof, mgld, u,
                                                          n_gamma, N, n, c); count_launch();
  return cudaGetLastError();
}

}  // namespace elmddm
