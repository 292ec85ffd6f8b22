// Step (c): blocked right-looking Cholesky S = L L^T of the Schur matrix of Eq. (3.5)
// (the paper states the system is SPD), and the blocked triangular solves that give
// u_Gamma.  The trailing SYRK update of the factorisation goes through launch_gemm.
#include "common.cuh"
#include "digits.cuh"

#include <cuda_bf16.h>

namespace elmddm {

namespace {

constexpr int NB = CHOL_NB;

// Unblocked Cholesky of the nb x nb diagonal block at (k, k), in shared memory, one
// barrier per pivot.  Step j works with the unscaled column j (a_ij, i > j, final at this
// point) and the multipliers t_i = a_ij / d_j, d_j = a_jj:
//   a_ik -= t_i a_kj   for j < k <= i   (= l_ij l_kj);
// at the end l_jj = sqrt(d_j) and l_ij = a_ij / l_jj.
//
// FP64 arithmetic is the scarce resource (2 FMA per clock per SM, a quarter of that for
// the warps of one SM sub-partition), and the pivot reciprocal is a long dependent chain.
// So step j is split between a look-ahead warp and the rest:
//   warp 0:      makes column c = j+1 final (applies column j to it), forms d_c, its
//                reciprocal and the multipliers t^(c) (double-buffered in shared memory);
//                it keeps column j and t^(j) in registers (lane l: rows l and l + 32), so
//                its chain reads shared memory once per step (the new column);
//   warps 1..15: the trailing triangle (columns >= 2) in registers, about four entries per
//                thread dealt round-robin over the column-major enumeration (so the active
//                entries stay spread over all threads as the triangle shrinks); step j
//                applies column j to the entries of columns >= j+2 and writes column j+2's
//                entries to shared memory, where warp 0 takes it as the next look-ahead.
// Every entry sees the same FMAs in the same order as in the plain right-looking
// elimination.  The reciprocal's latency hides behind the bulk update.  (Panels of 8
// columns factored by one warp in registers measured slower: the whole chain then runs on
// one sub-partition's quarter of the FP64 pipe; two pivots per barrier too.)
constexpr int POTRF_THREADS = 512;
constexpr int POTRF_BULK = POTRF_THREADS - 32;
constexpr int POTRF_E = (NB - 2) * (NB - 1) / 2;                     // entries (i, k), 2 <= k <= i < NB
constexpr int POTRF_PER = (POTRF_E + POTRF_BULK - 1) / POTRF_BULK;   // per bulk thread

__global__ void __launch_bounds__(POTRF_THREADS) k_potrf_diag(double* __restrict__ S, int ld, int k, int nb,
                                                              unsigned* status) {
  __shared__ double a[NB][NB + 1];
  __shared__ double piv[NB], rl[NB], tcol[2][NB];  // d_j, 1/sqrt(d_j), t^(j) (by parity of j)
  __shared__ int bad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < NB * NB; e += POTRF_THREADS) {
    const int i = e % NB, j = e / NB;
    a[i][j] = (i < nb && j < nb && i >= j) ? S[(k + i) + (size_t)(k + j) * ld] : 0.0;
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  // a pivot that is not positive (not SPD) is flagged and replaced by 1 so the loop ends
  auto checked = [&](double d) {
    const long long db = __double_as_longlong(d);
    if (db <= 0 || (db >> 52) >= 0x7FF) {  // positive and finite: sign clear, not zero, exponent < 2047
      if (lane == 0) bad = 1;
      return 1.0;
    }
    return d;
  };
  if (warp == 0) {
    const int r0 = lane, r1 = lane + 32;
    double tj0 = 0.0, tj1 = 0.0, cj0 = 0.0, cj1 = 0.0;  // t^(j), column j at rows r0, r1
    if (nb > 0) {  // column 0
      cj0 = a[r0][0];
      cj1 = a[r1][0];
      const double d = checked(__shfl_sync(0xffffffffu, cj0, 0));
      if (lane == 0) piv[0] = d;
      const double rd = rcp_newton(d);
      if (r0 > 0 && r0 < nb) { tj0 = cj0 * rd; tcol[0][r0] = tj0; }
      if (r1 < nb) { tj1 = cj1 * rd; tcol[0][r1] = tj1; }
    }
    for (int j = 0; j + 1 < nb; ++j) {
      const int c = j + 1;
      double x0 = (r0 >= c && r0 < nb) ? a[r0][c] : 0.0;
      double x1 = (r1 >= c && r1 < nb) ? a[r1][c] : 0.0;
      const double acj = __shfl_sync(0xffffffffu, c < 32 ? cj0 : cj1, c & 31);
      if (r0 >= c && r0 < nb) x0 = fma(-tj0, acj, x0);
      if (r1 >= c && r1 < nb) x1 = fma(-tj1, acj, x1);
      const double d = checked(__shfl_sync(0xffffffffu, c < 32 ? x0 : x1, c & 31));
      const double rd = rcp_newton(d);
      double* tn = tcol[c & 1];
      if (r0 > c && r0 < nb) { tj0 = x0 * rd; tn[r0] = tj0; }
      if (r1 > c && r1 < nb) { tj1 = x1 * rd; tn[r1] = tj1; }
      if (r0 >= c && r0 < nb) a[r0][c] = x0;
      if (r1 >= c && r1 < nb) a[r1][c] = x1;
      if (lane == 0) piv[c] = d;
      cj0 = x0;
      cj1 = x1;
      __syncthreads();
    }
  } else {
    const int bt = tid - 32;
    int ei[POTRF_PER], ek[POTRF_PER];
    double v[POTRF_PER];
#pragma unroll
    for (int q = 0; q < POTRF_PER; ++q) {
      const int e = bt + POTRF_BULK * q;
      ei[q] = -1;
      ek[q] = NB;
      v[q] = 0.0;
      if (e < POTRF_E) {  // column-major over k = 2 .. NB-1, rows i = k .. NB-1
        int kk = 2, base = 0;
        while (base + (NB - kk) <= e) { base += NB - kk; ++kk; }
        const int i = kk + (e - base);
        if (i < nb && kk < nb) { ei[q] = i; ek[q] = kk; v[q] = a[i][kk]; }
      }
    }
    for (int j = 0; j + 1 < nb; ++j) {
      const double* t = tcol[j & 1];
#pragma unroll
      for (int q = 0; q < POTRF_PER; ++q) {
        if (ei[q] >= 0 && ek[q] >= j + 2) {
          v[q] = fma(-t[ei[q]], a[ek[q]][j], v[q]);
          if (ek[q] == j + 2) a[ei[q]][ek[q]] = v[q];
        }
      }
      __syncthreads();
    }
  }
  if (tid < nb) rl[tid] = 1.0 / sqrt(piv[tid]);
  __syncthreads();
  for (int e = tid; e < NB * NB; e += POTRF_THREADS) {
    const int i = e % NB, j = e / NB;
    if (i >= nb || j >= nb || i < j) continue;
    S[(k + i) + (size_t)(k + j) * ld] = i == j ? sqrt(piv[j]) : a[i][j] * rl[j];
  }
  if (tid == 0 && bad) atomicOr(status, ST_NOT_SPD);
}

// Inverses of all diagonal blocks of the finished factor, one block per CTA: column c of
// X = L_kk^{-1} by forward substitution, x_rc = (delta_rc - sum_{c<=l<r} l_rl x_lc) / l_rr,
// one thread per column.  Used by the triangular solves of the solve phase; runs once
// after the factorisation, off its critical path.
__global__ void __launch_bounds__(NB) k_tri_inv(const double* __restrict__ S, int ld, int n,
                                               double* __restrict__ inv) {
  extern __shared__ double tinv_smem[];
  double (*L)[NB + 1] = reinterpret_cast<double (*)[NB + 1]>(tinv_smem);
  double (*X)[NB + 1] = reinterpret_cast<double (*)[NB + 1]>(tinv_smem + NB * (NB + 1));
  __shared__ double rd[NB];
  const int t = threadIdx.x, k = blockIdx.x * NB, nb = min(NB, n - k);
  for (int e = t; e < NB * NB; e += NB) {
    const int i = e % NB, j = e / NB;
    L[i][j] = (i < nb && j < nb && i >= j) ? S[(k + i) + (size_t)(k + j) * ld] : (i == j ? 1.0 : 0.0);
  }
  __syncthreads();
  rd[t] = 1.0 / L[t][t];
  __syncthreads();
  for (int r = 0; r < NB; ++r) {
    double v = r == t ? 1.0 : 0.0;
    for (int l = t; l < r; ++l) v = fma(-L[r][l], X[l][t], v);
    X[r][t] = r >= t ? v * rd[r] : 0.0;
  }
  __syncthreads();
  double* out = inv + (size_t)blockIdx.x * NB * NB;
  for (int e = t; e < NB * NB; e += NB) {
    const int i = e % NB, j = e / NB;
    out[i + j * NB] = (i < nb && j < nb) ? X[i][j] : 0.0;
  }
}

// L21 = A21 L11^{-T} by substitution, for the rows k+nb .. row_end-1 of the block column
// (the envelope): each row solves x L11^T = a.  Columns go in blocks of TRC_BW: the
// block's small triangle by plain substitution (one thread per row), then a rank-TRC_BW
// update of the row's remaining columns spread over all threads, so the FP64 pipe sees
// independent FMAs instead of one long dependent chain.  Same operations as the
// unblocked solve up to summation order, hence its backward stability.  TRC_ROWS rows per
// block keep about one block per SM on the envelopes of interest; 256 threads spread the
// rank-4 updates thin enough that the 4-column triangles set the pace (128 threads
// measured 14% slower, 384 and 512 no faster).
//
// With split outputs (tensor-core back end) the block also writes the finished rows as
// the SYRK's operands, so no separate split launch follows: each row's largest biased
// exponent (the 8 threads of a row reduce it) into eA and eB, and its 7 digit planes into
// tA (128-row tiles) and tB (32-row tiles), the layout k_split writes for K = nb.
constexpr int TRC_ROWS = 16, TRC_THREADS = 256, TRC_BW = 4;
constexpr int TRC_SPLIT = TRC_ROWS * NB / 8;  // threads of the split: one per 8 entries of the rows
__global__ void __launch_bounds__(TRC_THREADS) k_trsm_chol_rows(double* __restrict__ S, int ld, int k, int nb,
                                                                int row_end, void* tA, void* tB, int* eA,
                                                                int* eB) {
  __shared__ double L[NB][NB + 1];
  __shared__ double X[TRC_ROWS][NB + 1];
  __shared__ double rd[NB];
  const int t = threadIdx.x;
  const int r0 = k + nb + blockIdx.x * TRC_ROWS;
  for (int e = t; e < NB * NB; e += TRC_THREADS) {
    const int i = e % NB, j = e / NB;
    L[i][j] = (i < nb && j < nb && i >= j) ? S[(k + i) + (size_t)(k + j) * ld] : (i == j ? 1.0 : 0.0);
  }
  for (int e = t; e < TRC_ROWS * NB; e += TRC_THREADS) {
    const int r = e % TRC_ROWS, j = e / TRC_ROWS;
    X[r][j] = (r0 + r < row_end && j < nb) ? S[(r0 + r) + (size_t)(k + j) * ld] : 0.0;
  }
  __syncthreads();
  if (t < NB) rd[t] = 1.0 / L[t][t];
  __syncthreads();
  for (int b = 0; b < nb; b += TRC_BW) {
    if (t < TRC_ROWS) {
      double x[TRC_BW];
#pragma unroll
      for (int q = 0; q < TRC_BW; ++q) {
        double v = X[t][b + q];
#pragma unroll
        for (int l = 0; l < q; ++l) v = fma(-x[l], L[b + q][b + l], v);
        x[q] = v * rd[b + q];
        X[t][b + q] = x[q];
      }
    }
    __syncthreads();
    const int c0 = b + TRC_BW, pairs = TRC_ROWS * (nb - c0);
    for (int e = t; e < pairs; e += TRC_THREADS) {
      const int r = e % TRC_ROWS, c = c0 + e / TRC_ROWS;
      double v = X[r][c];
#pragma unroll
      for (int l = 0; l < TRC_BW; ++l) v = fma(-X[r][b + l], L[c][b + l], v);
      X[r][c] = v;
    }
    __syncthreads();
  }
  for (int e = t; e < TRC_ROWS * NB; e += TRC_THREADS) {
    const int r = e % TRC_ROWS, j = e / TRC_ROWS;
    if (r0 + r < row_end && j < nb) S[(r0 + r) + (size_t)(k + j) * ld] = X[r][j];
  }
  if (tA && t < TRC_SPLIT) {  // 128 threads = 16 rows x 8 groups of 8 k (whole warps)
    static_assert(TRC_SPLIT <= TRC_THREADS && TRC_SPLIT % 32 == 0, "one thread per 8 entries of the block's rows");
    const int r = t >> 3, g8 = t & 7, kc = g8 >> 2, kg = g8 & 3;
    const int gr = blockIdx.x * TRC_ROWS + r;  // row of L21
    const bool valid = r0 + r < row_end;
    double x[8];
    unsigned em = 0u;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      x[j] = X[r][8 * g8 + j];  // zero beyond nb and on rows past the envelope
      em = max(em, biased_exp(x[j]));
    }
    em = max(em, __shfl_xor_sync(0xffffffffu, em, 1));
    em = max(em, __shfl_xor_sync(0xffffffffu, em, 2));
    em = max(em, __shfl_xor_sync(0xffffffffu, em, 4));
    const int nkc = (nb + OZ_KC - 1) / OZ_KC;
    if (valid && kc < nkc) {
      uint32_t w[OZ_S][4];
      split8(x, em, w);
      __nv_bfloat16* oa = static_cast<__nv_bfloat16*>(tA) + (size_t)((gr >> 7) * nkc + kc) * OZ_S * 128 * OZ_KC;
      __nv_bfloat16* ob = static_cast<__nv_bfloat16*>(tB) + (size_t)((gr >> 5) * nkc + kc) * OZ_S * 32 * OZ_KC;
      const int offa = tile_off32(gr & 127, kg * 8), offb = tile_off32(gr & 31, kg * 8);
#pragma unroll
      for (int p = 0; p < OZ_S; ++p) {
        const uint4 v = make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
        *reinterpret_cast<uint4*>(oa + (size_t)p * 128 * OZ_KC + offa) = v;
        *reinterpret_cast<uint4*>(ob + (size_t)p * 32 * OZ_KC + offb) = v;
      }
      if (g8 == 0) {
        eA[gr] = (int)em;
        eB[gr] = (int)em;
      }
    }
  }
}

// Forward substitution step for block k: y_k = L_kk^{-1} r_k with the stored inverse of
// the diagonal block (a 64 x 64 matrix-vector product, no division chain), then
// r_i -= L_ik y_k for the rows k+nb <= i < row_end that can hold nonzeros of the block
// column (the envelope).  Every block forms y_k itself, so one launch covers the step;
// when Linv is NULL the small triangle is solved by substitution instead.
__global__ void __launch_bounds__(256) k_chol_fwd(const double* __restrict__ L, int ld, int n, int k,
                                                  int nb, int row_end, const double* __restrict__ Linv,
                                                  double* __restrict__ r, double* __restrict__ y) {
  __shared__ double Ls[NB][NB + 1];
  __shared__ double rs[NB], ys[NB];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* rr = r + (size_t)blockIdx.y * n;
  double* yy = y + (size_t)blockIdx.y * n;
  const double* src = Linv ? Linv : L;
  const int lds = Linv ? NB : ld;
  const int off = Linv ? 0 : k;
  for (int e = tid; e < nb * nb; e += 256) {
    const int i = e % nb, j = e / nb;
    Ls[i][j] = (i >= j) ? src[(off + i) + (size_t)(off + j) * lds] : 0.0;
  }
  if (tid < nb) rs[tid] = rr[k + tid];
  __syncthreads();
  if (Linv) {
    for (int i = warp; i < nb; i += 8) {
      double p = 0.0;
      for (int l = lane; l <= i; l += 32) p = fma(Ls[i][l], rs[l], p);
      p = warp_sum(p);
      if (lane == 0) ys[i] = p;
    }
  } else if (warp == 0) {
    for (int i = 0; i < nb; ++i) {
      double p = 0.0;
      for (int l = lane; l < i; l += 32) p = fma(Ls[i][l], ys[l], p);
      p = warp_sum(p);
      const double yi = (rs[i] - p) / Ls[i][i];
      __syncwarp();
      if (lane == 0) ys[i] = yi;
      __syncwarp();
    }
  }
  __syncthreads();
  if (blockIdx.x == 0 && tid < nb) yy[k + tid] = ys[tid];
  const int i = k + nb + blockIdx.x * 256 + tid;
  if (i < row_end) {
    double t = rr[i];
    for (int l = 0; l < nb; ++l) t = fma(-L[i + (size_t)(k + l) * ld], ys[l], t);
    rr[i] = t;
  }
}

// Backward substitution step for block k: u_k = L_kk^{-T} y_k (with the stored inverse
// when given), y_j -= L_k,j^T u_k for j_begin <= j < k (L_k,j is zero left of the
// envelope's first column j_begin).
__global__ void __launch_bounds__(256) k_chol_bwd(const double* __restrict__ L, int ld, int n, int k,
                                                  int nb, int j_begin, const double* __restrict__ Linv,
                                                  double* __restrict__ y, double* __restrict__ u) {
  __shared__ double Ls[NB][NB + 1];
  __shared__ double ysh[NB], us[NB];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* yy = y + (size_t)blockIdx.y * n;
  double* uu = u + (size_t)blockIdx.y * n;
  const double* src = Linv ? Linv : L;
  const int lds = Linv ? NB : ld;
  const int off = Linv ? 0 : k;
  for (int e = tid; e < nb * nb; e += 256) {
    const int i = e % nb, j = e / nb;
    Ls[i][j] = (i >= j) ? src[(off + i) + (size_t)(off + j) * lds] : 0.0;
  }
  if (tid < nb) ysh[tid] = yy[k + tid];
  __syncthreads();
  if (Linv) {
    // u = Linv^T y: u_i = sum_{l >= i} Linv[l][i] y_l
    for (int i = warp; i < nb; i += 8) {
      double p = 0.0;
      for (int l = i + lane; l < nb; l += 32) p = fma(Ls[l][i], ysh[l], p);
      p = warp_sum(p);
      if (lane == 0) us[i] = p;
    }
  } else if (warp == 0) {
    for (int i = nb - 1; i >= 0; --i) {
      double p = 0.0;
      for (int l = i + 1 + lane; l < nb; l += 32) p = fma(Ls[l][i], us[l], p);
      p = warp_sum(p);
      const double ui = (ysh[i] - p) / Ls[i][i];
      __syncwarp();
      if (lane == 0) us[i] = ui;
      __syncwarp();
    }
  }
  __syncthreads();
  if (blockIdx.x == 0 && tid < nb) uu[k + tid] = us[tid];
  for (int j = j_begin + blockIdx.x * 8 + warp; j < k; j += gridDim.x * 8) {
    double p = 0.0;
    for (int l = lane; l < nb; l += 32) p = fma(L[(k + l) + (size_t)j * ld], us[l], p);
    p = warp_sum(p);
    if (lane == 0) yy[j] -= p;
  }
}


// ---------------------------------------------------------------------------------------
// Whole triangular solves in one cooperative launch each: the 64-row block steps of
// k_chol_fwd / k_chol_bwd separated by a grid barrier instead of a kernel boundary (a
// launch and its tail cost more than a step's work).  Every block forms the step's
// 64-entry diagonal solve itself from the stored inverse, so one barrier per step
// suffices; the vectors that other blocks update are read through L2 (ld.global.cg),
// since L1 is not coherent between SMs.  The barrier's wait is bounded (2 s of
// %globaltimer by default, set per handle): on timeout the kernel flags ST_TIMEOUT and
// every block returns.  `hold` makes every barrier wait for one arrival more than the
// grid has, i.e. for a release that never comes: the failure-detection tests use it to
// make the wait run out on purpose (no asynchronous copy is in flight in these kernels,
// so giving up and returning leaves nothing behind).
__device__ __forceinline__ unsigned long long chol_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// bar[0]: arrivals, bar[1]: generation.  Returns false (for the whole block) on timeout.
__device__ bool grid_barrier(unsigned* bar, unsigned* status, unsigned long long limit_ns, int hold) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    const unsigned g = *(volatile unsigned*)(bar + 1);
    if (atomicAdd(bar, 1u) == gridDim.x - 1 + (unsigned)hold) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = chol_ns();
      while (*(volatile unsigned*)(bar + 1) == g) {
        if (chol_ns() - t0 >= limit_ns) {
          atomicOr(status, ST_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// Four threads share each row (forward) or column (backward) of a step, a quarter of
// the 64 terms each: a single warp's FP64 instructions go through one SM sub-partition's
// quarter of the FP64 pipe, so neither a 64-term chain per thread nor a warp-wide
// shuffle reduction per row (five FP64 additions) is cheap here.
constexpr int CS_ROWS = 64;  // rows / columns per block and pass

// L y = b over all block steps; r holds b on entry and is consumed.
__global__ void __launch_bounds__(256) k_chol_fwd_all(const double* __restrict__ L, int ld, int n,
                                                      const double* __restrict__ Linv,
                                                      const int* __restrict__ rend, int nsteps,
                                                      double* r, double* y, int nrhs,
                                                      unsigned* bar, unsigned* status,
                                                      unsigned long long limit_ns, int hold) {
  __shared__ double Ls[NB][NB + 1];
  __shared__ double rs[NB], ys[NB], part[4][CS_ROWS];
  const int tid = threadIdx.x, il = tid % CS_ROWS, q = tid / CS_ROWS;
  // this thread's 16 entries of a step's diagonal-block inverse: fetched before the
  // previous step's barrier, stored after it
  double pre[NB * NB / 256];
  auto fetch = [&](int st) {
    const int nb = min(NB, n - st * NB);
    const double* Li = Linv + (size_t)st * NB * NB;
#pragma unroll
    for (int m = 0; m < NB * NB / 256; ++m) {
      const int e = tid + 256 * m, i = e % NB, j = e / NB;
      pre[m] = (i < nb && j < nb && i >= j) ? Li[i + (size_t)j * NB] : 0.0;
    }
  };
  if (nsteps > 0) fetch(0);
  for (int st = 0; st < nsteps; ++st) {
    const int k = st * NB, nb = min(NB, n - k), row_end = rend[st];
#pragma unroll
    for (int m = 0; m < NB * NB / 256; ++m) {
      const int e = tid + 256 * m;
      Ls[e % NB][e / NB] = pre[m];
    }
    for (int c = 0; c < nrhs; ++c) {
      double* rr = r + (size_t)c * n;
      __syncthreads();
      if (tid < NB) rs[tid] = tid < nb ? __ldcg(rr + k + tid) : 0.0;
      __syncthreads();
      {  // y_k = Linv r_k, row il, terms 16 q .. 16 q + 15
        double p = 0.0;
#pragma unroll
        for (int t = 0; t < 16; ++t) p = fma(Ls[il][16 * q + t], rs[16 * q + t], p);
        part[q][il] = p;
      }
      __syncthreads();
      if (tid < NB) ys[tid] = (part[0][tid] + part[1][tid]) + (part[2][tid] + part[3][tid]);
      __syncthreads();
      if (blockIdx.x == 0 && tid < nb) y[(size_t)c * n + k + tid] = ys[tid];
      for (int base = k + nb + blockIdx.x * CS_ROWS; base < row_end; base += gridDim.x * CS_ROWS) {
        const int i = base + il;
        double p = 0.0;
        if (i < row_end) {
          const double* Lr = L + i + (size_t)(k + 16 * q) * ld;
#pragma unroll
          for (int t = 0; t < 16; ++t)
            if (16 * q + t < nb) p = fma(Lr[(size_t)t * ld], ys[16 * q + t], p);
        }
        __syncthreads();
        part[q][il] = p;
        __syncthreads();
        if (q == 0 && i < row_end)
          __stcg(rr + i, __ldcg(rr + i) - ((part[0][il] + part[1][il]) + (part[2][il] + part[3][il])));
      }
    }
    if (st + 1 < nsteps) fetch(st + 1);
    if (!grid_barrier(bar, status, limit_ns, hold)) return;
  }
}

// L^T u = y over all block steps (last to first); y is consumed.
__global__ void __launch_bounds__(256) k_chol_bwd_all(const double* __restrict__ L, int ld, int n,
                                                      const double* __restrict__ Linv,
                                                      const int* __restrict__ jbeg, int nsteps,
                                                      double* y, double* u, int nrhs,
                                                      unsigned* bar, unsigned* status,
                                                      unsigned long long limit_ns, int hold) {
  __shared__ double Ls[NB][NB + 1];
  __shared__ double ysh[NB], us[NB], part[4][CS_ROWS];
  const int tid = threadIdx.x, il = tid % CS_ROWS, q = tid / CS_ROWS;
  const int jl = tid >> 2, qq = tid & 3;  // column pass: 4 lanes per column
  double pre[NB * NB / 256];
  auto fetch = [&](int st) {
    const int nb = min(NB, n - st * NB);
    const double* Li = Linv + (size_t)st * NB * NB;
#pragma unroll
    for (int m = 0; m < NB * NB / 256; ++m) {
      const int e = tid + 256 * m, i = e % NB, j = e / NB;
      pre[m] = (i < nb && j < nb && i >= j) ? Li[i + (size_t)j * NB] : 0.0;
    }
  };
  if (nsteps > 0) fetch(nsteps - 1);
  for (int st = nsteps - 1; st >= 0; --st) {
    const int k = st * NB, nb = min(NB, n - k), j_begin = jbeg[st];
#pragma unroll
    for (int m = 0; m < NB * NB / 256; ++m) {
      const int e = tid + 256 * m;
      Ls[e % NB][e / NB] = pre[m];
    }
    for (int c = 0; c < nrhs; ++c) {
      double* yy = y + (size_t)c * n;
      __syncthreads();
      if (tid < NB) ysh[tid] = tid < nb ? __ldcg(yy + k + tid) : 0.0;
      __syncthreads();
      {  // u_k = Linv^T y_k: u_i = sum_l Linv[l][i] y_l, terms 16 q .. 16 q + 15
        double p = 0.0;
#pragma unroll
        for (int t = 0; t < 16; ++t) p = fma(Ls[16 * q + t][il], ysh[16 * q + t], p);
        part[q][il] = p;
      }
      __syncthreads();
      if (tid < NB) us[tid] = (part[0][tid] + part[1][tid]) + (part[2][tid] + part[3][tid]);
      __syncthreads();
      if (blockIdx.x == 0 && tid < nb) u[(size_t)c * n + k + tid] = us[tid];
      // y_j -= L_{k,j}^T u_k for j_begin <= j < k: column j's 64 rows are contiguous
      for (int base = j_begin + blockIdx.x * CS_ROWS; base < k; base += gridDim.x * CS_ROWS) {
        const int j = base + jl;
        double p = 0.0;
        if (j < k) {
          const double* Lc = L + (k + 16 * qq) + (size_t)j * ld;
#pragma unroll
          for (int t = 0; t < 16; ++t)
            if (16 * qq + t < nb) p = fma(Lc[t], us[16 * qq + t], p);
        }
        p += __shfl_xor_sync(0xffffffffu, p, 1);
        p += __shfl_xor_sync(0xffffffffu, p, 2);
        if (qq == 0 && j < k) __stcg(yy + j, __ldcg(yy + j) - p);
      }
    }
    if (st > 0) fetch(st - 1);
    if (!grid_barrier(bar, status, limit_ns, hold)) return;
  }
}

// y = rcp_newton(x) element by element (the self-test of the pivot reciprocal).
__global__ void k_rcp_newton(const double* __restrict__ x, double* __restrict__ y, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = rcp_newton(x[i]);
}

}  // namespace

cudaError_t launch_potrf_diag(double* S, int ld, int k, int nb, unsigned* status, cudaStream_t st) {
  k_potrf_diag<<<1, POTRF_THREADS, 0, st>>>(S, ld, k, nb, status); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_tri_inv(const double* S, int ld, int n, double* inv, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int smem = 2 * NB * (NB + 1) * (int)sizeof(double);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_tri_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_tri_inv<<<(n + NB - 1) / NB, NB, smem, st>>>(S, ld, n, inv); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_rcp_newton(const double* x, double* y, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_rcp_newton<<<(n + 255) / 256, 256, 0, st>>>(x, y, n); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_trsm_chol_rows(double* S, int ld, int k, int nb, int row_end, cudaStream_t st,
                                  void* tA, void* tB, int* eA, int* eB) {
  const int rows = row_end - k - nb;
  if (rows <= 0) return cudaSuccess;
  k_trsm_chol_rows<<<(rows + TRC_ROWS - 1) / TRC_ROWS, TRC_THREADS, 0, st>>>(S, ld, k, nb, row_end, tA, tB,
                                                                            eA, eB); count_launch();
  return cudaGetLastError();
}

cudaError_t launch_chol_fwd(const double* L, int ld, int n, int k, int nb, double* r,
                            double* y, int nrhs, cudaStream_t st, int row_end, const double* Linv) {
  if (row_end < 0 || row_end > n) row_end = n;
  const int rows = row_end - k - nb;
  const int gx = rows > 0 ? (rows + 255) / 256 : 1;
  k_chol_fwd<<<dim3(gx, nrhs), 256, 0, st>>>(L, ld, n, k, nb, row_end, Linv, r, y); count_launch();
  return cudaGetLastError();
}

int chol_solve_grid(bool forward, int work_max) {
  int g = (work_max + CS_ROWS - 1) / CS_ROWS;  // rows (forward) or columns (backward) per block
  if (g < 1) g = 1;
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, forward ? (const void*)k_chol_fwd_all
                                                              : (const void*)k_chol_bwd_all, 256, 0);
  const int cap = sms * (occ > 0 ? occ : 0);
  if (g > sms) g = sms;
  return g <= cap ? g : 0;  // 0: no co-resident grid (use the step kernels)
}

cudaError_t launch_chol_fwd_all(const double* L, int ld, int n, const double* Linv, const int* rend,
                                int nsteps, double* r, double* y, int nrhs, int grid, unsigned* bar,
                                unsigned* status, cudaStream_t st, unsigned long long limit_ns, int hold) {
  cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&L, (void*)&ld, (void*)&n, (void*)&Linv, (void*)&rend, (void*)&nsteps,
                  (void*)&r, (void*)&y, (void*)&nrhs, (void*)&bar, (void*)&status, (void*)&limit_ns,
                  (void*)&hold};
  e = cudaLaunchCooperativeKernel((const void*)k_chol_fwd_all, dim3(grid), dim3(256), args, 0, st);
  count_launch();
  return e;
}

cudaError_t launch_chol_bwd_all(const double* L, int ld, int n, const double* Linv, const int* jbeg,
                                int nsteps, double* y, double* u, int nrhs, int grid, unsigned* bar,
                                unsigned* status, cudaStream_t st, unsigned long long limit_ns, int hold) {
  cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&L, (void*)&ld, (void*)&n, (void*)&Linv, (void*)&jbeg, (void*)&nsteps,
                  (void*)&y, (void*)&u, (void*)&nrhs, (void*)&bar, (void*)&status, (void*)&limit_ns,
                  (void*)&hold};
  e = cudaLaunchCooperativeKernel((const void*)k_chol_bwd_all, dim3(grid), dim3(256), args, 0, st);
  count_launch();
  return e;
}

cudaError_t launch_chol_bwd(const double* L, int ld, int n, int k, int nb, double* y,
                            double* u, int nrhs, cudaStream_t st, int j_begin, const double* Linv) {
  if (j_begin < 0 || j_begin > k) j_begin = 0;
  int gx = (k - j_begin + 7) / 8;
  if (gx < 1) gx = 1;
  if (gx > 1024) gx = 1024;
  k_chol_bwd<<<dim3(gx, nrhs), 256, 0, st>>>(L, ld, n, k, nb, j_begin, Linv, y, u); count_launch();
  return cudaGetLastError();
}

}  // namespace elmddm
