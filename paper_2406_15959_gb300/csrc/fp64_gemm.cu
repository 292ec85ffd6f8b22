// elm_ddm_fp64_gemm: the solver's FP64-accurate digit-split product (k_ozaki.cu) as a
// stand-alone entry point, C = alpha A B^T + beta C with general strides.  It runs the
// same split and product kernels as the QR trailing updates, the D_s / M_s products and
// the Schur Cholesky, on caller-provided workspace (it allocates nothing).
#include "elm_ddm.h"
#include "common.cuh"
#include "digits.cuh"

#include <algorithm>
#include <vector>

using namespace elmddm;

namespace {

size_t al256(size_t b) { return (b + 255) / 256 * 256; }

// Workspace layout: status word | split descriptors | product descriptor | tile table |
// row exponents of A and B | digit planes of A and B.
struct Layout {
  size_t status, sd, od, ut, ea, eb, ta, tb, hl, total;
  int brow, tiles, ksplit;
};

bool layout(int kernel, int M, int N, int K, Layout* L) {
  if (M < 1 || N < 1 || K < 1) return false;
  int brow = 32;
  switch (kernel) {
    case ELM_DDM_GEMM_TILE32: if (K > 512 * 128) return false; break;
    case ELM_DDM_GEMM_TILE64: if (K > 128) return false; brow = 64; break;
    case ELM_DDM_GEMM_PERSISTENT: if (K > 128) return false; break;
    case ELM_DDM_GEMM_PERSISTENT_WIDE: if (K > 128) return false; brow = 64; break;
    case ELM_DDM_GEMM_FUSED_SPLIT: if (N > 32 || K > 512 * 128) return false; break;
    case ELM_DDM_GEMM_FUSED_SPLIT_B: if (M > 128 || K > 512 * 128) return false; break;
    default: return false;
  }
  L->brow = brow;
  // the fused A-split product of a single 128-row tile splits K over up to 4 CTAs (exact
  // int64 accumulation, the same bits as one CTA)
  L->ksplit = (kernel == ELM_DDM_GEMM_FUSED_SPLIT && M <= 128) ? std::min(4, (K + 511) / 512) : 1;
  L->tiles = kernel == ELM_DDM_GEMM_PERSISTENT        ? ((M + 127) / 128) * ((N + 31) / 32)
             : kernel == ELM_DDM_GEMM_PERSISTENT_WIDE ? ((M + 127) / 128) * ((N + 63) / 64)
                                                      : 0;
  size_t o = 0;
  L->status = o; o += 256;
  L->sd = o; o += al256(2 * sizeof(SplitDesc));
  L->od = o; o += al256(sizeof(OzDesc));
  L->ut = o; o += al256((size_t)L->tiles * sizeof(int4));
  L->ea = o; o += al256((size_t)M * 4);
  L->eb = o; o += al256((size_t)N * 4);
  L->ta = o; o += kernel == ELM_DDM_GEMM_FUSED_SPLIT ? 0 : al256(oz_split_elems(M, K, 128) * 2);
  L->tb = o; o += kernel == ELM_DDM_GEMM_FUSED_SPLIT_B ? 0 : al256(oz_split_elems(N, K, brow) * 2);
  L->hl = o; o += L->ksplit > 1 ? al256((size_t)OZ_HL_TILE * sizeof(long long)) : 0;
  L->total = o;
  return true;
}

}  // namespace

extern "C" size_t elm_ddm_fp64_gemm_workspace(int kernel, int M, int N, int K) {
  Layout L;
  return layout(kernel, M, N, K, &L) ? L.total : 0;
}

extern "C" int elm_ddm_fp64_gemm(int kernel, int M, int N, int K, double alpha, const double* A,
                                 long long a_rs, long long a_ks, const double* B, long long b_rs,
                                 long long b_ks, double beta, double* C, long long c_rs, long long c_cs,
                                 void* workspace, size_t workspace_bytes, void* stream) {
  Layout L;
  if (!layout(kernel, M, N, K, &L)) return ELM_DDM_ERR_ARG;
  if (!A || !B || !C || !workspace || workspace_bytes < L.total) return ELM_DDM_ERR_ARG;
  if (((uintptr_t)workspace & 255) != 0) return ELM_DDM_ERR_ARG;
  if (kernel == ELM_DDM_GEMM_FUSED_SPLIT && (a_ks != 1 || alpha != 1.0 || beta != 0.0))
    return ELM_DDM_ERR_ARG;
  if (kernel == ELM_DDM_GEMM_FUSED_SPLIT_B && (b_ks != 1 || alpha != 1.0 || beta != 0.0))
    return ELM_DDM_ERR_ARG;
  if (kernel == ELM_DDM_GEMM_PERSISTENT_WIDE && ((alpha != 1.0 && alpha != -1.0) || beta != 1.0))
    return ELM_DDM_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  unsigned* status = reinterpret_cast<unsigned*>(ws + L.status);
  int* ea = reinterpret_cast<int*>(ws + L.ea);
  int* eb = reinterpret_cast<int*>(ws + L.eb);
  const bool fused = kernel == ELM_DDM_GEMM_FUSED_SPLIT, fused_b = kernel == ELM_DDM_GEMM_FUSED_SPLIT_B;
  SplitDesc sd[2] = {{A, a_rs, a_ks, M, K, ea, fused ? nullptr : ws + L.ta, 128},
                     {B, b_rs, b_ks, N, K, eb, fused_b ? nullptr : ws + L.tb, L.brow}};
  OzDesc od{fused ? (const void*)A : (const void*)(ws + L.ta), ea,
            fused_b ? (const void*)B : (const void*)(ws + L.tb), eb, C, c_rs, c_cs, M, N, K,
            0, fused ? a_rs : (fused_b ? b_rs : 0)};
  if (L.ksplit > 1) od.hl = reinterpret_cast<long long*>(ws + L.hl);
  std::vector<int4> tiles;
  if (kernel == ELM_DDM_GEMM_PERSISTENT || kernel == ELM_DDM_GEMM_PERSISTENT_WIDE) {
    tiles.resize(L.tiles);
    oz_upd_tile_table(&od, 1, 0, tiles.data(), kernel == ELM_DDM_GEMM_PERSISTENT ? 32 : UPW_TILE_N);
  }
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(unsigned), st);
  if (e == cudaSuccess && L.ksplit > 1) e = cudaMemsetAsync(ws + L.hl, 0, OZ_HL_TILE * sizeof(long long), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ws + L.sd, sd, sizeof sd, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ws + L.od, &od, sizeof od, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !tiles.empty())
    e = cudaMemcpyAsync(ws + L.ut, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice, st);
  const SplitDesc* dsd = reinterpret_cast<const SplitDesc*>(ws + L.sd);
  const OzDesc* dod = reinterpret_cast<const OzDesc*>(ws + L.od);
  const int rx_blocks = std::max(oz_rowexp_blocks(sd[0]), oz_rowexp_blocks(sd[1]));
  const int ta_tiles = (M + 127) / 128, tb_tiles = (N + L.brow - 1) / L.brow;
  const int blocks = (ta_tiles > tb_tiles ? ta_tiles : tb_tiles) * ((K + OZ_KC - 1) / OZ_KC);
  if (e == cudaSuccess) e = launch_split(dsd, 2, rx_blocks, blocks, st);
  if (e == cudaSuccess) {
    switch (kernel) {
      case ELM_DDM_GEMM_TILE32: e = launch_ozaki(32, dod, 1, oz_tiles(M, N, 32), alpha, beta, 0, status, st); break;
      case ELM_DDM_GEMM_TILE64: e = launch_ozaki(64, dod, 1, oz_tiles(M, N, 64), alpha, beta, 0, status, st); break;
      case ELM_DDM_GEMM_PERSISTENT:
        e = launch_ozaki_upd(dod, 1, reinterpret_cast<const int4*>(ws + L.ut), L.tiles, alpha, beta, 0, status,
                             st);
        break;
      case ELM_DDM_GEMM_PERSISTENT_WIDE:
        e = launch_ozaki_updw(dod, 1, reinterpret_cast<const int4*>(ws + L.ut), L.tiles, alpha, status, st);
        break;
      case ELM_DDM_GEMM_FUSED_SPLIT_B: {
        const int nbc = N >= 64 ? 64 : 32;  // as the solver's outer W1 products
        e = launch_ozaki_fb(dod, 1, (N + nbc - 1) / nbc, status, st, 8, nbc);
        break;
      }
      default: e = launch_ozaki_fa(dod, 1, (M + 127) / 128, status, st, 8, L.ksplit); break;
    }
  }
  unsigned bits = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, status, sizeof bits, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host staging above must outlive its copies
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ELM_DDM_ERR_CUDA;
  }
  if (bits & ST_TIMEOUT) return ELM_DDM_ERR_TIMEOUT;
  if (bits) return ELM_DDM_ERR_CUDA;
  return ELM_DDM_OK;
}

extern "C" int elm_ddm_selftest(int which, const double* x, double* y, int n, void* stream) {
  if (which != ELM_DDM_SELFTEST_PIVOT_RCP || !x || !y || n < 0) return ELM_DDM_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = launch_rcp_newton(x, y, n, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ELM_DDM_ERR_CUDA;
  }
  return ELM_DDM_OK;
}
