// Batched FP64 GEMM on the FP64 pipe, and batched block additions.
//
// Every dense update of the solver goes through launch_gemm: the trailing updates of
// the blocked Householder QR (step (b)), D_s = I - Q_G Q_G^T and M_s = -Y_s Q_G^T,
// the M^T M blocks of the Schur matrix (Eq. (3.5)) and the SYRK updates of its
// Cholesky factorisation.  On GB300 the FP64 rate is ~1/60 of FP32, so a 64x64 tile
// with 4x4 register blocking per thread keeps the DFMA pipe busy; shared-memory and
// L2 traffic are far below what the pipe can consume.
#include "common.cuh"

namespace elmddm {

namespace {

constexpr int TM = 64, TN = 64, TK = 16;

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm(const GemmDesc* __restrict__ descs, double alpha,
                                              double beta, int flags) {
  const GemmDesc d = descs[blockIdx.y];
  const int tiles_m = (d.m + TM - 1) / TM, tiles_n = (d.n + TN - 1) / TN;
  if ((int)blockIdx.x >= tiles_m * tiles_n) return;
  const int bi = blockIdx.x % tiles_m, bj = blockIdx.x / tiles_m;
  if ((flags & GEMM_LOWER) && bj > bi) return;
  const int i0 = bi * TM, j0 = bj * TN;

  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

  for (int kk0 = 0; kk0 < d.k; kk0 += TK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = t + 256 * q;
      int i, kk;
      if (TA) { kk = e & 15; i = e >> 4; } else { i = e & 63; kk = e >> 6; }
      const int gi = i0 + i, gk = kk0 + kk;
      double v = 0.0;
      if (gi < d.m && gk < d.k)
        v = TA ? d.A[gk + (size_t)gi * d.lda] : d.A[gi + (size_t)gk * d.lda];
      As[kk][i] = v;
      int j, kb;
      if (TB) { j = e & 63; kb = e >> 6; } else { kb = e & 15; j = e >> 4; }
      const int gj = j0 + j, gk2 = kk0 + kb;
      double w = 0.0;
      if (gj < d.n && gk2 < d.k)
        w = TB ? d.B[gj + (size_t)gk2 * d.ldb] : d.B[gk2 + (size_t)gj * d.ldb];
      Bs[kb][j] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[kk][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int gj = j0 + ty + 16 * b;
    if (gj >= d.n) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int gi = i0 + tx + 16 * a;
      if (gi >= d.m) continue;
      double* cp = d.C + gi + (size_t)gj * d.ldc;
      double v = alpha * acc[a][b];
      if (beta != 0.0) v = fma(beta, *cp, v);
      if ((flags & GEMM_ADD_IDENTITY) && gi == gj) v += 1.0;
      *cp = v;
    }
  }
}

__global__ void __launch_bounds__(256) k_add_blocks(const AddDesc* __restrict__ descs) {
  const AddDesc d = descs[blockIdx.y];
  const int total = d.rows * d.cols;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int i = e % d.rows, j = e / d.rows;
    d.dst[i + (size_t)j * d.ldd] += d.src[i + (size_t)j * d.lds];
  }
}

}  // namespace

cudaError_t launch_gemm(bool ta, bool tb, const GemmDesc* d, int count, int max_tiles,
                        double alpha, double beta, int flags, cudaStream_t st) {
  if (count <= 0 || max_tiles <= 0) return cudaSuccess;
  for (int off = 0; off < count; off += 65535) {
    const int c = count - off < 65535 ? count - off : 65535;
    dim3 grid(max_tiles, c);
    if (ta && tb) k_gemm<true, true><<<grid, 256, 0, st>>>(d + off, alpha, beta, flags);
    else if (ta) k_gemm<true, false><<<grid, 256, 0, st>>>(d + off, alpha, beta, flags);
    else if (tb) k_gemm<false, true><<<grid, 256, 0, st>>>(d + off, alpha, beta, flags);
    else k_gemm<false, false><<<grid, 256, 0, st>>>(d + off, alpha, beta, flags);
  }
  return cudaGetLastError();
}

cudaError_t launch_add_blocks(const AddDesc* d, int count, int max_elems, cudaStream_t st) {
  if (count <= 0 || max_elems <= 0) return cudaSuccess;
  int bx = (max_elems + 255) / 256;
  if (bx > 64) bx = 64;
  for (int off = 0; off < count; off += 65535) {
    const int c = count - off < 65535 ? count - off : 65535;
    k_add_blocks<<<dim3(bx, c), 256, 0, st>>>(d + off);
  }
  return cudaGetLastError();
}

}  // namespace elmddm
