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

constexpr int TK = 16;

// Tile TM x TN per block of 256 threads; every thread owns a 4 x 4 register block
// (rows tx + TX*a, columns ty + TY*b), so TM * TN = 4096.  64 x 64 is the general tile;
// 32 x 128 serves the skinny products of the QR panels (m = panel width 32), which a
// 64-row tile would half waste.
template <bool TA, bool TB, int TM, int TN>
__global__ void __launch_bounds__(256) k_gemm(const GemmDesc* __restrict__ descs, double alpha,
                                              double beta, int flags) {
  static_assert(TM * TN == 4096, "tile must hold 256 x 16 outputs");
  constexpr int TX = TM / 4, TY = TN / 4;
  constexpr int A_PER = TK * TM / 256, B_PER = TK * TN / 256;
  const GemmDesc d = descs[blockIdx.y];
  const int tiles_m = (d.m + TM - 1) / TM, tiles_n = (d.n + TN - 1) / TN;
  if ((int)blockIdx.x >= tiles_m * tiles_n) return;
  const int bi = blockIdx.x % tiles_m, bj = blockIdx.x / tiles_m;
  if ((flags & GEMM_LOWER) && bj * TN > bi * TM + TM - 1) return;
  const int i0 = bi * TM, j0 = bj * TN;

  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  const int t = threadIdx.x, tx = t % TX, ty = t / TX;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;

  for (int kk0 = 0; kk0 < d.k; kk0 += TK) {
#pragma unroll
    for (int q = 0; q < A_PER; ++q) {
      const int e = t + 256 * q;
      int i, kk;
      if (TA) { kk = e % TK; i = e / TK; } else { i = e % TM; kk = e / TM; }
      const int gi = i0 + i, gk = kk0 + kk;
      double v = 0.0;
      if (gi < d.m && gk < d.k)
        v = TA ? d.A[gk + (size_t)gi * d.lda] : d.A[gi + (size_t)gk * d.lda];
      As[kk][i] = v;
    }
#pragma unroll
    for (int q = 0; q < B_PER; ++q) {
      const int e = t + 256 * q;
      int j, kb;
      if (TB) { j = e % TN; kb = e / TN; } else { kb = e % TK; j = e / TK; }
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
      for (int a = 0; a < 4; ++a) av[a] = As[kk][tx + TX * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][ty + TY * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int gj = j0 + ty + TY * b;
    if (gj >= d.n) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int gi = i0 + tx + TX * a;
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

template <int TM, int TN>
void gemm_dispatch(bool ta, bool tb, dim3 grid, cudaStream_t st, const GemmDesc* d, double alpha,
                   double beta, int flags) {
  if (ta && tb) k_gemm<true, true, TM, TN><<<grid, 256, 0, st>>>(d, alpha, beta, flags);
  else if (ta) k_gemm<true, false, TM, TN><<<grid, 256, 0, st>>>(d, alpha, beta, flags);
  else if (tb) k_gemm<false, true, TM, TN><<<grid, 256, 0, st>>>(d, alpha, beta, flags);
  else k_gemm<false, false, TM, TN><<<grid, 256, 0, st>>>(d, alpha, beta, flags);
  count_launch();
}

cudaError_t launch_gemm(bool ta, bool tb, const GemmDesc* d, int count, int max_tiles,
                        double alpha, double beta, int flags, cudaStream_t st) {
  if (count <= 0 || max_tiles <= 0) return cudaSuccess;
  const bool skinny = (flags & GEMM_SKINNY) != 0;
  for (int off = 0; off < count; off += 65535) {
    const int c = count - off < 65535 ? count - off : 65535;
    dim3 grid(max_tiles, c);
    if (skinny) gemm_dispatch<32, 128>(ta, tb, grid, st, d + off, alpha, beta, flags);
    else gemm_dispatch<64, 64>(ta, tb, grid, st, d + off, alpha, beta, flags);
  }
  return cudaGetLastError();
}

cudaError_t launch_add_blocks(const AddDesc* d, int count, int max_elems, cudaStream_t st) {
  if (count <= 0 || max_elems <= 0) return cudaSuccess;
  int bx = (max_elems + 255) / 256;
  if (bx > 64) bx = 64;
  for (int off = 0; off < count; off += 65535) {
    const int c = count - off < 65535 ? count - off : 65535;
    k_add_blocks<<<dim3(bx, c), 256, 0, st>>>(d + off); count_launch();
  }
  return cudaGetLastError();
}

}  // namespace elmddm
