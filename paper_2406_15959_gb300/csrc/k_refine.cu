// Mixed-precision mode: FP64 residuals of the system that defines the method's result and
// the pieces of its correction that the low-precision factors do not already provide.
//
// The result (c, u_Gamma) of Section 3 solves Eq. (3.4), whose second block carries
// K^+ = (K^T K)^{-1} K^T.  With w = (K^T K)^{-1} A^T A c (so K^{+T} A^T A c = K w), Eq. (3.4)
// is equivalent to the block system in (c, w, u) without any K^+:
//   K^T K c + K^T B u          = K^T F          (the local least-squares problems)
//   K^T K w - A^T A c          = 0
//   B^T K c - B^T K w + B^T B u = B^T F          (the interface condition)
// Its residual needs only products with the FP64 K^s, A^s and the index maps, which the
// kernels below compute; the correction is solved with the low-precision R, Q_G, Y, M and
// the FP64 Cholesky factor of the (low-precision) Schur matrix by the elimination of
// Eq. (3.5).  B^s = [0; 0; -E_s] and F^s = 0 on interface rows throughout.
#include "common.cuh"

namespace elmddm {

namespace {

// Per subdomain s and right-hand side: e = F - K c + [0; 0; E u] (the residual of
// K c + B u = F), kw = K w over the rows, and z = -(e + K w) on the interface rows: the
// third residual block is sum_s E_s^T z_s.  One thread per row; c and w staged in
// shared memory.
__global__ void __launch_bounds__(256) k_resid_rows(const double* __restrict__ K, long long kstride, int ld,
                                                   int n, const int* __restrict__ ms,
                                                   const int* __restrict__ cnt,
                                                   const int* __restrict__ ifc_dof, int mgld,
                                                   const double* __restrict__ F, const double* __restrict__ c,
                                                   const double* __restrict__ w, const double* __restrict__ u,
                                                   int ng, int N, double* __restrict__ e,
                                                   double* __restrict__ kw, double* __restrict__ z) {
  extern __shared__ double rr_sh[];
  const int s = blockIdx.y, rh = blockIdx.z;
  const size_t cv = ((size_t)rh * N + s) * n, xv = ((size_t)rh * N + s) * ld;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    rr_sh[j] = c[cv + j];
    rr_sh[n + j] = w[cv + j];
  }
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= ms[s]) return;
  const double* Kr = K + (size_t)s * kstride + r;
  double a = 0.0, b = 0.0;
#pragma unroll 4
  for (int j = 0; j < n; ++j) {
    const double k = Kr[(size_t)j * ld];
    a = fma(k, rr_sh[j], a);
    b = fma(k, rr_sh[n + j], b);
  }
  const int i0 = cnt[3 * s] + cnt[3 * s + 1];
  double ev = F[xv + r] - a;
  if (r >= i0 && r < i0 + cnt[3 * s + 2]) {  // interface rows (pad rows follow them)
    const int li = r - i0;
    ev += u[(size_t)rh * ng + ifc_dof[(size_t)s * mgld + li]];
    z[((size_t)rh * N + s) * mgld + li] = -(ev + b);
  }
  e[xv + r] = ev;
  kw[xv + r] = b;
}

// r1 = K^T e and t = K^T kw per column of K (warp per column; e and kw of the subdomain
// staged in shared memory).
__global__ void __launch_bounds__(256) k_resid_cols(const double* __restrict__ K, long long kstride, int ld,
                                                   int n, const int* __restrict__ ms,
                                                   const double* __restrict__ e, const double* __restrict__ kw,
                                                   int N, double* __restrict__ r1, double* __restrict__ t) {
  extern __shared__ double rc_sh[];
  const int s = blockIdx.y, rh = blockIdx.z, m = ms[s];
  const size_t xv = ((size_t)rh * N + s) * ld;
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    rc_sh[r] = e[xv + r];
    rc_sh[ld + r] = kw[xv + r];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, j = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (j >= n) return;
  const double* Kc = K + (size_t)s * kstride + (size_t)j * ld;
  double a = 0.0, b = 0.0;
  for (int r = lane; r < m; r += 32) {
    const double k = Kc[r];
    a = fma(k, rc_sh[r], a);
    b = fma(k, rc_sh[ld + r], b);
  }
  a = warp_sum(a);
  b = warp_sum(b);
  if (lane == 0) {
    r1[((size_t)rh * N + s) * n + j] = a;
    t[((size_t)rh * N + s) * n + j] = b;
  }
}

// out = A^s x_s at the interface rows (thread per row; A column-major, leading dim mgld).
__global__ void __launch_bounds__(128) k_amul(const double* __restrict__ A, long long astride, int mgld,
                                             const int* __restrict__ mg, int n, const double* __restrict__ x,
                                             int N, double* __restrict__ out) {
  const int s = blockIdx.y, rh = blockIdx.z;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= mg[s]) return;
  const double* As = A + (size_t)s * astride + i;
  const double* xs = x + ((size_t)rh * N + s) * n;
  double a = 0.0;
  for (int j = 0; j < n; ++j) a = fma(As[(size_t)j * mgld], xs[j], a);
  out[((size_t)rh * N + s) * mgld + i] = a;
}

// out = A^s^T (E_s g) + sg * t per column of A^s (warp per column); with r1 given, also
// d = r1 - out.
__global__ void __launch_bounds__(256) k_atmul(const double* __restrict__ A, long long astride, int mgld,
                                              const int* __restrict__ mg, const int* __restrict__ ifc_dof,
                                              int n, const double* __restrict__ g, int ng,
                                              const double* __restrict__ t, double sg,
                                              const double* __restrict__ r1, int N, double* __restrict__ out,
                                              double* __restrict__ d) {
  const int s = blockIdx.y, rh = blockIdx.z, lane = threadIdx.x & 31;
  const int j = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (j >= n) return;
  const int m = mg[s];
  const double* Ac = A + (size_t)s * astride + (size_t)j * mgld;
  const int* dofs = ifc_dof + (size_t)s * mgld;
  const double* gg = g + (size_t)rh * ng;
  double a = 0.0;
  for (int i = lane; i < m; i += 32) a = fma(Ac[i], gg[dofs[i]], a);
  a = warp_sum(a);
  if (lane == 0) {
    const size_t o = ((size_t)rh * N + s) * n + j;
    const double v = fma(sg, t[o], a);
    out[o] = v;
    if (r1) d[o] = r1[o] - v;
  }
}

// p = R^{-T} v per subdomain and vector (R upper triangular, R_ij at K[i + j * ld]; v and
// p of length n, v at v + (vec * N + s) * vs, p at p + (vec * N + s) * ps).  One CTA per
// (subdomain, vector), x in shared memory; 32-column blocks: the block's entries take the
// dot products with the entries already solved (column j of R above the block is
// contiguous; 8 warps, a column each), then warp 0 solves the block's triangle by
// columns (lane jj holds entry jj and R's column jj in registers).
__global__ void __launch_bounds__(256) k_rt_solve(const double* __restrict__ K, long long kstride, int ld,
                                                 int n, const double* __restrict__ v, long long vs,
                                                 double* __restrict__ p, long long ps, int N) {
  extern __shared__ double rt_sh[];
  const int s = blockIdx.x, vec = blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* R = K + (size_t)s * kstride;
  const double* vv = v + ((size_t)vec * N + s) * vs;
  for (int j = tid; j < n; j += 256) rt_sh[j] = vv[j];
  __syncthreads();
  for (int jb = 0; jb < n; jb += 32) {
    const int nbj = min(32, n - jb);
    for (int jj = warp; jj < nbj; jj += 8) {
      const double* Rc = R + (size_t)(jb + jj) * ld;
      double a = 0.0;
      for (int i = lane; i < jb; i += 32) a = fma(Rc[i], rt_sh[i], a);
      a = warp_sum(a);
      if (lane == 0) rt_sh[jb + jj] -= a;
    }
    __syncthreads();
    if (warp == 0) {
      double rc[32];
      const double* Rc = R + (size_t)(jb + lane) * ld + jb;
#pragma unroll
      for (int ii = 0; ii < 32; ++ii) rc[ii] = (lane < nbj && ii <= lane) ? Rc[ii] : 0.0;
      double x = lane < nbj ? rt_sh[jb + lane] : 0.0;
      const double rinv = lane < nbj ? 1.0 / R[(size_t)(jb + lane) * ld + jb + lane] : 0.0;
#pragma unroll
      for (int ii = 0; ii < 32; ++ii) {
        double xi = __shfl_sync(0xffffffffu, x * rinv, ii);  // entry ii is final once reached
        if (lane == ii) x = xi;
        if (lane > ii) x = fma(-rc[ii], xi, x);
      }
      if (lane < nbj) rt_sh[jb + lane] = x;
    }
    __syncthreads();
  }
  double* pp = p + ((size_t)vec * N + s) * ps;
  for (int j = tid; j < n; j += 256) pp[j] = rt_sh[j];
}

// c += dc, w += dw (nc entries per right-hand side), u += du (ng per right-hand side);
// nrm[4 rh ..] = max |du|, max |u|, max |dc|, max |c| after the update (as bit patterns:
// non-negative doubles order like them, NaN above everything).
__global__ void k_refine_update(double* __restrict__ c, const double* __restrict__ dc, double* __restrict__ w,
                                const double* __restrict__ dw, long long nc, double* __restrict__ u,
                                const double* __restrict__ du, int ng, unsigned long long* __restrict__ nrm) {
  const int rh = blockIdx.y;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nc) {
    const size_t o = (size_t)rh * nc + i;
    const double d = dc[o], cn = c[o] + d;
    c[o] = cn;
    w[o] += dw[o];
    atomicMax(nrm + 4 * rh + 2, (unsigned long long)__double_as_longlong(fabs(d)));
    atomicMax(nrm + 4 * rh + 3, (unsigned long long)__double_as_longlong(fabs(cn)));
  }
  if (i < ng) {
    const size_t o = (size_t)rh * ng + i;
    const double d = du[o];
    const double un = u[o] + d;
    u[o] = un;
    atomicMax(nrm + 4 * rh, (unsigned long long)__double_as_longlong(fabs(d)));
    atomicMax(nrm + 4 * rh + 1, (unsigned long long)__double_as_longlong(fabs(un)));
  }
}

}  // namespace

cudaError_t launch_resid_rows(const double* K, long long kstride, int ld, int n, const int* ms, const int* cnt,
                              const int* ifc_dof, int mgld, const double* F, const double* c, const double* w,
                              const double* u, int ng, int N, int mmax, int nrhs, double* e, double* kw,
                              double* z, cudaStream_t st) {
  const size_t smem = 2 * (size_t)n * sizeof(double);
  static int attr = 0;
  if (smem > 48 * 1024 && smem > (size_t)attr) {
    cudaError_t er = cudaFuncSetAttribute(k_resid_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (er != cudaSuccess) return er;
    attr = (int)smem;
  }
  k_resid_rows<<<dim3((mmax + 255) / 256, N, nrhs), 256, smem, st>>>(K, kstride, ld, n, ms, cnt, ifc_dof, mgld,
                                                                     F, c, w, u, ng, N, e, kw, z);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_resid_cols(const double* K, long long kstride, int ld, int n, const int* ms, const double* e,
                              const double* kw, int N, int nrhs, double* r1, double* t, cudaStream_t st) {
  const size_t smem = 2 * (size_t)ld * sizeof(double);
  static int attr = 0;
  if (smem > 48 * 1024 && smem > (size_t)attr) {
    cudaError_t er = cudaFuncSetAttribute(k_resid_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (er != cudaSuccess) return er;
    attr = (int)smem;
  }
  k_resid_cols<<<dim3((n + 7) / 8, N, nrhs), 256, smem, st>>>(K, kstride, ld, n, ms, e, kw, N, r1, t);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_amul(const double* A, long long astride, int mgld, const int* mg, int mgmax, int n,
                        const double* x, int N, int nrhs, double* out, cudaStream_t st) {
  if (mgmax <= 0) return cudaSuccess;
  k_amul<<<dim3((mgmax + 127) / 128, N, nrhs), 128, 0, st>>>(A, astride, mgld, mg, n, x, N, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_atmul(const double* A, long long astride, int mgld, const int* mg, const int* ifc_dof, int n,
                         const double* g, int ng, const double* t, double sg, const double* r1, int N, int nrhs,
                         double* out, double* d, cudaStream_t st) {
  k_atmul<<<dim3((n + 7) / 8, N, nrhs), 256, 0, st>>>(A, astride, mgld, mg, ifc_dof, n, g, ng, t, sg, r1, N, out,
                                                      d);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_rt_solve(const double* K, long long kstride, int ld, int n, const double* v, long long vs,
                            double* p, long long ps, int N, int nvec, cudaStream_t st) {
  const size_t smem = (size_t)n * sizeof(double);
  static int attr = 0;
  if (smem > 48 * 1024 && smem > (size_t)attr) {
    cudaError_t er = cudaFuncSetAttribute(k_rt_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (er != cudaSuccess) return er;
    attr = (int)smem;
  }
  k_rt_solve<<<dim3(N, nvec), 256, smem, st>>>(K, kstride, ld, n, v, vs, p, ps, N);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_refine_update(double* c, const double* dc, double* w, const double* dw, long long nc, double* u,
                                 const double* du, int ng, int nrhs, unsigned long long* nrm, cudaStream_t st) {
  const long long top = nc > ng ? nc : ng;
  k_refine_update<<<dim3((unsigned)((top + 255) / 256), nrhs), 256, 0, st>>>(c, dc, w, dw, nc, u, du, ng, nrm);
  count_launch();
  return cudaGetLastError();
}

}  // namespace elmddm
