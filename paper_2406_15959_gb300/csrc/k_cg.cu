// Conjugate gradients on the Schur system of Eq. (3.5), the solver the paper uses for
// the interface problem (Section 4: CG to a relative residual of 1e-9).  S is applied
// without being formed, from the stored local pieces:
//     S p = sum_s E_s^T D_s E_s p + M^T (M p),   M p = sum_s E_s^T M_s E_s p,
// i.e. per subdomain two dense products with D_s and M_s, one with M_s^T, and two
// local -> global sums (launch_gather2, every interface unknown has two owners).
#include "common.cuh"

namespace elmddm {

namespace {

// z_s = D_s E_s p and w_s = M_s E_s p.  Block (row chunk of 64, s, rhs), 256 threads:
// 64 rows x 4 column phases; a warp reads 32 consecutive rows of a column (coalesced).
__global__ void __launch_bounds__(256) k_schur_apply1(const double* __restrict__ D,
                                                      const double* __restrict__ M, long long mstride,
                                                      int mgld, const int* __restrict__ mg_arr,
                                                      const int* __restrict__ ifc_dof,
                                                      const double* __restrict__ p, int ng, int N,
                                                      double* __restrict__ zl, double* __restrict__ wl) {
  extern __shared__ double cg_smem[];
  double* ps = cg_smem;                          // [mgld]
  __shared__ double red[2][4][64];
  const int s = blockIdx.y, rh = blockIdx.z, i0 = blockIdx.x * 64;
  const int mg = mg_arr[s];
  if (i0 >= mg) return;
  const int tid = threadIdx.x, tx = tid & 63, ty = tid >> 6;
  const int* dofs = ifc_dof + (size_t)s * mgld;
  const double* pp = p + (size_t)rh * ng;
  for (int k = tid; k < mg; k += 256) ps[k] = pp[dofs[k]];
  __syncthreads();
  const double* Ds = D + (size_t)s * mstride;
  const double* Ms = M + (size_t)s * mstride;
  const int i = i0 + tx;
  double a = 0.0, b = 0.0;
  if (i < mg)
    for (int j = ty; j < mg; j += 4) {
      const double pj = ps[j];
      a = fma(Ds[i + (size_t)j * mgld], pj, a);
      b = fma(Ms[i + (size_t)j * mgld], pj, b);
    }
  red[0][ty][tx] = a;
  red[1][ty][tx] = b;
  __syncthreads();
  if (ty == 0 && i < mg) {
    const size_t o = ((size_t)rh * N + s) * mgld + i;
    zl[o] = red[0][0][tx] + red[0][1][tx] + red[0][2][tx] + red[0][3][tx];
    wl[o] = red[1][0][tx] + red[1][1][tx] + red[1][2][tx] + red[1][3][tx];
  }
}

// z_s += M_s^T E_s w.  Block (16 columns, s, rhs), 8 warps, warp per column of M_s
// (contiguous in memory), lanes over its rows.
__global__ void __launch_bounds__(256) k_schur_apply2(const double* __restrict__ M, long long mstride,
                                                      int mgld, const int* __restrict__ mg_arr,
                                                      const int* __restrict__ ifc_dof,
                                                      const double* __restrict__ w, int ng, int N,
                                                      double* __restrict__ zl) {
  extern __shared__ double cg_smem[];
  double* ws = cg_smem;                          // [mgld]
  const int s = blockIdx.y, rh = blockIdx.z, c0 = blockIdx.x * 16;
  const int mg = mg_arr[s];
  if (c0 >= mg) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int* dofs = ifc_dof + (size_t)s * mgld;
  const double* ww = w + (size_t)rh * ng;
  for (int k = tid; k < mg; k += 256) ws[k] = ww[dofs[k]];
  __syncthreads();
  const double* Ms = M + (size_t)s * mstride;
  for (int i = c0 + warp; i < min(c0 + 16, mg); i += 8) {
    double a = 0.0;
    for (int k = lane; k < mg; k += 32) a = fma(Ms[k + (size_t)i * mgld], ws[k], a);
    a = warp_sum(a);
    if (lane == 0) zl[((size_t)rh * N + s) * mgld + i] += a;
  }
}

// Start of (preconditioned) CG from x (zero or the caller's guess, with q = S x already
// formed): r = b - q, z = M^{-1} r, p = z; rr = r^T r, rz = r^T z, bb = b^T b.  M is the
// Jacobi preconditioner diag(S) (dinv = its inverse) or the identity (dinv = NULL).
// One block per right-hand side.
__global__ void __launch_bounds__(1024) k_pcg_init(const double* __restrict__ b, const double* __restrict__ q,
                                                   double* __restrict__ r, double* __restrict__ p,
                                                   const double* __restrict__ dinv, CgState* __restrict__ st,
                                                   int ng, int has_x0, double tol2) {
  __shared__ double red[33];
  const int rh = blockIdx.x, tid = threadIdx.x;
  const size_t o = (size_t)rh * ng;
  double bb = 0.0, rr = 0.0, rz = 0.0;
  for (int g = tid; g < ng; g += blockDim.x) {
    const double bv = b[o + g];
    const double rg = has_x0 ? bv - q[o + g] : bv;
    const double zg = dinv ? rg * dinv[g] : rg;
    r[o + g] = rg;
    p[o + g] = zg;
    bb = fma(bv, bv, bb);
    rr = fma(rg, rg, rr);
    rz = fma(rg, zg, rz);
  }
  bb = block_sum(bb, red);
  rr = block_sum(rr, red);
  rz = block_sum(rz, red);
  if (tid == 0) {
    st[rh].rr = rr;
    st[rh].rz = rz;
    st[rh].bb = bb;
    st[rh].iters = 0;
    st[rh].done = !isfinite(rr) || !isfinite(rz) ? 2 : (rr <= tol2 * bb ? 1 : 0);
  }
}

// One (preconditioned) CG step for every right-hand side not yet converged:
// alpha = rz / p^T q, x += alpha p, r -= alpha q, z = M^{-1} r, beta = r^T z / rz,
// p = z + beta p.  done = 1 once r^T r <= tol^2 b^T b (the true residual of the
// recurrence, not the preconditioned one); done = 2 if p^T q <= 0 (S not positive
// definite in floating point) or a quantity is not finite.
__global__ void __launch_bounds__(1024) k_pcg_update(double* __restrict__ x, double* __restrict__ r,
                                                     double* __restrict__ p, const double* __restrict__ q,
                                                     const double* __restrict__ dinv,
                                                     CgState* __restrict__ st, int ng, double tol2) {
  __shared__ double red[33];
  const int rh = blockIdx.x, tid = threadIdx.x;
  if (st[rh].done) return;
  const double rz_old = st[rh].rz, bb = st[rh].bb;
  const size_t o = (size_t)rh * ng;
  double pq = 0.0;
  for (int g = tid; g < ng; g += blockDim.x) pq = fma(p[o + g], q[o + g], pq);
  pq = block_sum(pq, red);
  if (!(pq > 0.0) || !isfinite(pq)) {
    if (tid == 0) st[rh].done = 2;
    return;
  }
  const double alpha = rz_old / pq;
  double rr = 0.0, rz = 0.0;
  for (int g = tid; g < ng; g += blockDim.x) {
    x[o + g] = fma(alpha, p[o + g], x[o + g]);
    const double rg = fma(-alpha, q[o + g], r[o + g]);
    r[o + g] = rg;
    rr = fma(rg, rg, rr);
    rz = fma(rg, dinv ? rg * dinv[g] : rg, rz);
  }
  rr = block_sum(rr, red);
  rz = block_sum(rz, red);
  const double beta = rz / rz_old;
  for (int g = tid; g < ng; g += blockDim.x) {
    const double zg = dinv ? r[o + g] * dinv[g] : r[o + g];
    p[o + g] = fma(beta, p[o + g], zg);
  }
  if (tid == 0) {
    st[rh].rr = rr;
    st[rh].rz = rz;
    st[rh].iters += 1;
    if (!isfinite(rr) || !isfinite(rz)) st[rh].done = 2;
    else if (rr <= tol2 * bb) st[rh].done = 1;
  }
}

// dst[idx[g]] = src[g] for every right-hand side (caller order -> internal order).
__global__ void k_scatter_perm(const int* __restrict__ idx, int n, const double* __restrict__ src,
                               double* __restrict__ dst) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x, rh = blockIdx.y;
  if (g < n) dst[(size_t)rh * n + idx[g]] = src[(size_t)rh * n + g];
}

// dinv[i] = 1 / S[i, i] (the Jacobi preconditioner; S column-major, ld n).
__global__ void k_diag_inv(const double* __restrict__ S, int n, double* __restrict__ dinv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dinv[i] = 1.0 / S[i + (size_t)i * n];
}

// ---- block-Jacobi preconditioner: the inverse of S's diagonal block of every interface
// edge (the unknowns of one edge are consecutive in the internal order) ----

// Inverse of one edge's diagonal block (len <= BJ_MAX), from the lower triangle of S, by
// Gauss-Jordan elimination in place without pivoting (S is SPD, so every pivot of its
// principal blocks is positive): for every k, row k is divided by the pivot and column k
// eliminated from every other row, the identity's column k built in its place.  One CTA
// per edge, the block in shared memory.  A pivot that is not positive flags ST_NOT_SPD.
constexpr int BJ_MAX = 128;
__global__ void __launch_bounds__(256) k_block_inv(const double* __restrict__ S, int ng,
                                                   const int* __restrict__ off, const int* __restrict__ len,
                                                   const long long* __restrict__ ioff, double* __restrict__ inv,
                                                   unsigned* status) {
  extern __shared__ double bj_smem[];
  const int e = blockIdx.x, t = threadIdx.x;
  const int o = off[e], n = len[e], ld = n + 1;
  double* a = bj_smem;  // [n][n + 1]
  __shared__ double prow[BJ_MAX + 1], pcol[BJ_MAX + 1];
  __shared__ int bad;
  for (int q = t; q < n * n; q += 256) {
    const int i = q / n, j = q % n;
    const int r = max(i, j), c = min(i, j);
    a[i * ld + j] = S[(o + r) + (size_t)(o + c) * ng];
  }
  if (t == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    const double piv = a[k * ld + k];
    if (t == 0 && !(piv > 0.0)) bad = 1;
    const double rp = piv > 0.0 ? 1.0 / piv : 0.0;
    // pivot row scaled (the identity's entry at k becomes 1 / piv) and column k saved
    for (int j = t; j < n; j += 256) {
      prow[j] = j == k ? rp : a[k * ld + j] * rp;
      pcol[j] = a[j * ld + k];
    }
    __syncthreads();
    for (int q = t; q < n * n; q += 256) {
      const int i = q / n, j = q % n;
      if (i == k) a[i * ld + j] = prow[j];
      else a[i * ld + j] = (j == k ? 0.0 : a[i * ld + j]) - pcol[i] * prow[j];
    }
    __syncthreads();
  }
  double* out = inv + ioff[e];
  for (int q = t; q < n * n; q += 256) out[q] = a[(q / n) * ld + q % n];
  if (t == 0 && bad) atomicOr(status, ST_NOT_SPD);
}

// z = B^{-1} r on every edge's unknowns, B the block-diagonal part of S.  Block (edge,
// right-hand side), one thread per row of the edge's inverse (row-major, contiguous).
__global__ void __launch_bounds__(BJ_MAX) k_bj_apply(const double* __restrict__ inv, const int* __restrict__ off,
                                                    const int* __restrict__ len,
                                                    const long long* __restrict__ ioff,
                                                    const double* __restrict__ r, double* __restrict__ z, int ng) {
  __shared__ double rs[BJ_MAX];
  const int e = blockIdx.x, rh = blockIdx.y, t = threadIdx.x;
  const int o = off[e], n = len[e];
  const double* rr = r + (size_t)rh * ng + o;
  if (t < n) rs[t] = rr[t];
  __syncthreads();
  if (t < n) {
    const double* row = inv + ioff[e] + (size_t)t * n;
    double acc = 0.0;
    for (int j = 0; j < n; ++j) acc = fma(row[j], rs[j], acc);
    z[(size_t)rh * ng + o + t] = acc;
  }
}

// First half of a CG step with a preconditioner applied by separate launches:
// alpha = rz / p^T q, x += alpha p, r -= alpha q, rr = r^T r.
__global__ void __launch_bounds__(1024) k_pcg_step_a(double* __restrict__ x, double* __restrict__ r,
                                                     const double* __restrict__ p, const double* __restrict__ q,
                                                     CgState* __restrict__ st, int ng) {
  __shared__ double red[33];
  const int rh = blockIdx.x, tid = threadIdx.x;
  if (st[rh].done) return;
  const size_t o = (size_t)rh * ng;
  double pq = 0.0;
  for (int g = tid; g < ng; g += blockDim.x) pq = fma(p[o + g], q[o + g], pq);
  pq = block_sum(pq, red);
  if (!(pq > 0.0) || !isfinite(pq)) {
    if (tid == 0) st[rh].done = 2;
    return;
  }
  const double alpha = st[rh].rz / pq;
  double rr = 0.0;
  for (int g = tid; g < ng; g += blockDim.x) {
    x[o + g] = fma(alpha, p[o + g], x[o + g]);
    const double rg = fma(-alpha, q[o + g], r[o + g]);
    r[o + g] = rg;
    rr = fma(rg, rg, rr);
  }
  rr = block_sum(rr, red);
  if (tid == 0) st[rh].rr = rr;
}

// Second half, with z = M^{-1} r already formed: beta = r^T z / rz, p = z + beta p (and at
// the start, first = 1: p = z); the stopping rule and the breakdown flags as in
// k_pcg_update.
__global__ void __launch_bounds__(1024) k_pcg_step_b(const double* __restrict__ r, const double* __restrict__ z,
                                                     double* __restrict__ p, CgState* __restrict__ st, int ng,
                                                     double tol2, int first) {
  __shared__ double red[33];
  const int rh = blockIdx.x, tid = threadIdx.x;
  if (st[rh].done) return;
  const size_t o = (size_t)rh * ng;
  double rz = 0.0;
  for (int g = tid; g < ng; g += blockDim.x) rz = fma(r[o + g], z[o + g], rz);
  rz = block_sum(rz, red);
  const double beta = first ? 0.0 : rz / st[rh].rz;
  for (int g = tid; g < ng; g += blockDim.x) p[o + g] = first ? z[o + g] : fma(beta, p[o + g], z[o + g]);
  if (tid == 0) {
    const double rr = st[rh].rr, bb = st[rh].bb;
    st[rh].rz = rz;
    if (!first) st[rh].iters += 1;
    if (!isfinite(rr) || !isfinite(rz)) st[rh].done = 2;
    else if (rr <= tol2 * bb) st[rh].done = 1;
  }
}

}  // namespace

cudaError_t launch_schur_apply(const double* D, const double* M, long long mstride, int mgld,
                               const int* mg, int mgmax, const int* ifc_dof, const int* dofmap,
                               const double* p, double* q, double* zl, double* wl, double* wg,
                               int ng, int N, int nrhs, cudaStream_t st) {
  if (ng <= 0 || mgmax <= 0) return cudaSuccess;
  const size_t smem = (size_t)mgld * sizeof(double);
  k_schur_apply1<<<dim3((mgmax + 63) / 64, N, nrhs), 256, smem, st>>>(D, M, mstride, mgld, mg, ifc_dof,
                                                                     p, ng, N, zl, wl); count_launch();
  cudaError_t e = launch_gather2(dofmap, GRP_MAX, ng, mgld, N, wl, wg, 0, nrhs, st);
  if (e != cudaSuccess) return e;
  k_schur_apply2<<<dim3((mgmax + 15) / 16, N, nrhs), 256, smem, st>>>(M, mstride, mgld, mg, ifc_dof, wg,
                                                                     ng, N, zl); count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_gather2(dofmap, GRP_MAX, ng, mgld, N, zl, q, 0, nrhs, st);
}

cudaError_t launch_pcg_init(const double* b, const double* q, double* r, double* p, const double* dinv,
                            CgState* state, int ng, int nrhs, int has_x0, double tol2, cudaStream_t st) {
  k_pcg_init<<<nrhs, 1024, 0, st>>>(b, q, r, p, dinv, state, ng, has_x0, tol2); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pcg_update(double* x, double* r, double* p, const double* q, const double* dinv,
                              CgState* state, int ng, int nrhs, double tol2, cudaStream_t st) {
  k_pcg_update<<<nrhs, 1024, 0, st>>>(x, r, p, q, dinv, state, ng, tol2); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_block_inv(const double* S, int ng, const int* off, const int* len, const long long* ioff,
                             int nedges, int maxlen, double* inv, unsigned* status, cudaStream_t st) {
  if (nedges <= 0) return cudaSuccess;
  if (maxlen > BJ_MAX) return cudaErrorInvalidValue;
  const int smem = maxlen * (maxlen + 1) * (int)sizeof(double);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_block_inv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         BJ_MAX * (BJ_MAX + 1) * (int)sizeof(double));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_block_inv<<<nedges, 256, smem, st>>>(S, ng, off, len, ioff, inv, status); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_bj_apply(const double* inv, const int* off, const int* len, const long long* ioff, int nedges,
                            const double* r, double* z, int ng, int nrhs, cudaStream_t st) {
  if (nedges <= 0) return cudaSuccess;
  k_bj_apply<<<dim3(nedges, nrhs), BJ_MAX, 0, st>>>(inv, off, len, ioff, r, z, ng); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pcg_step_a(double* x, double* r, const double* p, const double* q, CgState* state, int ng,
                              int nrhs, cudaStream_t st) {
  k_pcg_step_a<<<nrhs, 1024, 0, st>>>(x, r, p, q, state, ng); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_pcg_step_b(const double* r, const double* z, double* p, CgState* state, int ng, int nrhs,
                              double tol2, int first, cudaStream_t st) {
  k_pcg_step_b<<<nrhs, 1024, 0, st>>>(r, z, p, state, ng, tol2, first); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_scatter_perm(const int* idx, int n, const double* src, double* dst, int nrhs,
                                cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_scatter_perm<<<dim3((n + 255) / 256, nrhs), 256, 0, st>>>(idx, n, src, dst); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_diag_inv(const double* S, int n, double* dinv, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_diag_inv<<<(n + 255) / 256, 256, 0, st>>>(S, n, dinv); count_launch();
  return cudaGetLastError();
}

}  // namespace elmddm
