// Digit split of FP64 operands for the tensor-core products (k_ozaki.cu) and for the
// kernels that write split operands directly (the Cholesky panel solve, k_chol.cu).
// A row r of an operand is x = 2^(E_r - 1022) sum_{p=1..7} d_p 2^(1 - 8 p) with balanced
// integer digits |d_p| <= 128, E_r the largest biased exponent in the row; the digits are
// stored as 7 BF16 planes, tile by tile (row_tile rows x OZ_KC k per tile, tiles ordered
// [row tile][k chunk]) in the tcgen05 K-major no-swizzle canonical layout.
#pragma once
#include "common.cuh"

namespace elmddm {

constexpr int OZ_S = 7;    // digit planes per operand
constexpr int OZ_KC = 32;  // K per tile (two 16-wide MMA k-steps)

// Element offset of (r, k) inside an R x 32 tile in the canonical K-major layout
// [r/8][k/8][r%8][k%8].
__device__ __forceinline__ int tile_off32(int r, int k) {
  return (((r >> 3) * 4 + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}

__device__ __forceinline__ unsigned biased_exp(double x) {
  return (unsigned)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// Fixed-point image of x relative to the row bound 2^(emax-1022): the signed integer
// F = trunc(x * 2^(1077 - emax)), |F| < 2^55 (zero for x = 0, for subnormal x and for an
// all-zero row).  Branch-free: the 55-bit mantissa M << 2 is shifted right by
// emax - e in two 32-bit halves, and the sign is applied as (F ^ s) - s.
__device__ __forceinline__ long long fixed55(double x, unsigned emax) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const uint32_t e = (hi >> 20) & 0x7FFu;
  const uint32_t mh = e ? ((((hi & 0xFFFFFu) | 0x100000u) << 2) | (lo >> 30)) : 0u;
  const uint32_t ml = e ? (lo << 2) : 0u;
  const uint32_t s = min(emax - e, 63u);  // a shift of 55 or more leaves 0
  const uint32_t fl = s < 32 ? __funnelshift_r(ml, mh, s) : (mh >> (s & 31));
  const uint32_t fh = s < 32 ? (mh >> s) : 0u;
  const unsigned long long F = ((unsigned long long)fh << 32) | fl;
  const unsigned long long sg = (unsigned long long)((long long)(int)hi >> 31);
  return (long long)((F ^ sg) - sg);
}

// Balanced base-256 digits of F = sum_p d_p 256^(7-p), p = 1..7, all |d_p| <= 128,
// without a carry chain: adding 128 to each of the seven byte positions makes every low
// byte of F + C equal to d_p + 128 (p >= 2) and the bits from 48 up equal to d_1 + 128.
// Each digit becomes a BF16 through a float magic-number add (1.5 * 2^23 + b holds the
// integer b in its low mantissa bits; subtracting 1.5 * 2^23 + 128 is exact), and two
// BF16 values are packed by a byte permute of the floats' upper halves.  Returns the 7
// planes' words for 8 consecutive k (w[p][j] holds k = 2j, 2j+1).
//
// With |d| <= 128 on both operands a digit product is at most 2^14 and a group
// g = p + q has at most 7 pairs, so any 128 consecutive k sum to less than
// 7 * 2^14 * 128 < 2^24: exact in the FP32 accumulators of the tensor core.
__device__ __forceinline__ void split8(const double (&x)[8], unsigned emax, uint32_t (&w)[OZ_S][4]) {
  constexpr unsigned long long kBias = 0x0080808080808080ull;
  float f[OZ_S][8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const unsigned long long Fp = (unsigned long long)fixed55(x[j], emax) + kBias;
    const uint32_t lo = (uint32_t)Fp, hi = (uint32_t)(Fp >> 32);
    f[0][j] = __uint_as_float(0x4B400000u + (hi >> 16)) - 12583040.0f;  // bits 48.. (0..256)
#pragma unroll
    for (int p = 2; p <= OZ_S; ++p) {  // digit p sits in byte 7 - p
      const int byte = 7 - p;
      const uint32_t src = byte >= 4 ? hi : lo;
      const uint32_t b = __byte_perm(src, 0x4B400000u, 0x7650 | (byte & 3));
      f[p - 1][j] = __uint_as_float(b) - 12583040.0f;
    }
  }
#pragma unroll
  for (int p = 0; p < OZ_S; ++p)
#pragma unroll
    for (int j = 0; j < 4; ++j)
      w[p][j] = __byte_perm(__float_as_uint(f[p][2 * j]), __float_as_uint(f[p][2 * j + 1]), 0x7632);
}

}  // namespace elmddm
