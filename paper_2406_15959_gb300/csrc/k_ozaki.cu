// FP64-accurate GEMM on the BF16 tensor cores (tcgen05), by exact digit splitting.
//
// GB300 runs FP64 at ~1/60 of FP32 and has no fast FP64 tensor path, while every large
// dense update of the solver (QR trailing updates, the Schur Cholesky's SYRK, the D_s and
// M_s products) needs FP64 accuracy.  Each FP64 operand row r is written as
// x = 2^(E_r - 1022) * sum_p d_p 2^(1 - 8p), p = 1..7, with balanced integer digits
// |d_p| <= 128, exactly representable in BF16 (E_r: largest biased exponent of the row;
// truncation error < 2^(E_r - 1077), i.e. 2^-55 relative to the row's bound).  Then
//     (A B^T)_ij = 2^(E_i + F_j - 2044) * sum_g 2^(-8g + 2) * sum_{p+q=g} sum_k dA_p dB_q,
// and for g = 2..8 (28 digit pairs) the inner integer sums over 128 consecutive k are
// exact in the FP32 accumulators of the tensor core (|sum| <= 7 * 2^14 * 128 < 2^24);
// the groups g > 8 are not formed (each term loses at most 6 * 2^-54 of the product of
// its row and column maxima to them).  Each 128-wide chunk is drained from TMEM into two
// exact int64 words, and the FP64 result is built from them with integer exponent
// arithmetic and one rounding add: two FP64 operations per element instead of 2K, with
// an error bound normwise per row and column (|C_ij - exact| <= 2^-53 |C_ij| +
// 2^-54 (max|a_i| sum|b_j| + max|b_j| sum|a_i|) + 6 K 2^-54 max|a_i| max|b_j|) where an
// FP64 GEMM's is componentwise.
//
// Splitting uses only integer and FP32 operations on the FP64 bit pattern.
// Kernels:
//   k_rowexp    exponent bound (max biased exponent) of each operand row
//   k_split     7 BF16 digit planes per (row tile, 32-wide K step), written directly in
//               the tcgen05 K-major no-swizzle canonical layout (8x8 core matrices)
//   k_ozaki     one CTA per 128 x NT output tile: warp 0 streams the digit tiles with
//               cp.async.bulk, warp 1 issues the 28 digit-pair MMAs per 16-wide k-step
//               into 7 TMEM accumulators (one per g), warps 2..5 drain TMEM and write C
//   k_ozaki_fa  wide-K product whose FP64 A operand is split inside the kernel
//   k_ozaki_fb  wide-K product whose FP64 B operand is split inside the kernel
//   k_ozaki_upd persistent product for K <= 128 over a table of output tiles
#include "common.cuh"
#include "digits.cuh"

#include <cuda_bf16.h>

namespace elmddm {

namespace {

constexpr int OZ_G = 7;        // groups g = p + q = 2..8
constexpr int OZ_M = 128;      // MMA M = rows of an A tile
constexpr int OZ_THREADS = 192;
// Wide-K products accumulate each 128-wide chunk's group sums into two int64 words H, L
// (|H| < 2^45.1, |L| < 2^47.1 per chunk): exact integers converted exactly to FP64 up to 62
// chunks (K <= 7936), beyond that converted with one rounding each (at most two more FP64
// roundings of the result), up to 512 chunks (K <= 65536), where the int64 words still
// cannot overflow.
constexpr int OZ_MAX_CHUNKS = 512;
constexpr unsigned long long kWaitNs = 2000000000ull;  // every wait gives up after 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t a, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes));
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a));
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase with the given parity; false if it has not completed within 2 s
// of wall time (each try_wait may itself suspend, so the bound is on the clock).
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity) {
  const unsigned long long t0 = global_ns();
  for (unsigned it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(a), "r"(parity));
    if (ok) return true;
    if ((it & 63) == 63 && global_ns() - t0 > kWaitNs) return false;
  }
}
// Warp-uniform wait: lane 0 waits, the outcome is broadcast to the whole warp (the
// tcgen05.ld that follow are warp-collective and must be executed by all 32 lanes).
__device__ __forceinline__ bool mbar_wait_warp(uint32_t a, uint32_t parity) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(a, parity) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}
// Shared-memory matrix descriptor, K-major, no swizzle: LBO = byte step between core
// matrices along K, SBO = byte step between core matrices along M/N.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      mbar));
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                 "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&v)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
               : "r"(taddr));
}

// Asynchronous 8-byte global -> shared copies (completion tracked per thread by groups).
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// E[r] = largest biased exponent in row r (0 for an all-zero row).  A warp per row,
// lanes over k; but short rows of a column-major operand (rs == 1, K <= 256): a thread per
// row looping over k, so that a warp reads 32 consecutive rows of one column at a time
// (the grid, sized for 8 rows per block, has blocks to spare).  Both loops issue RX_UNROLL
// loads before the first maximum, so that a long row (a panel's V^T, K up to the local
// row count) waits for one memory latency per RX_UNROLL elements, not per element.
constexpr int RX_UNROLL = 8;
__host__ __device__ inline bool rowexp_by_thread(long long rs, long long ks, int K) {
  return rs == 1 && ks != 1 && K <= 256;
}
__global__ void __launch_bounds__(256) k_rowexp(const SplitDesc* __restrict__ descs) {
  const SplitDesc d = descs[blockIdx.y];
  if (rowexp_by_thread(d.rs, d.ks, d.K)) {
    const int r = blockIdx.x * 256 + threadIdx.x;
    if (r >= d.R) return;
    unsigned mx = 0;
    const double* x = d.X + r;
    int k = 0;
    for (; k + RX_UNROLL <= d.K; k += RX_UNROLL) {
      double v[RX_UNROLL];
#pragma unroll
      for (int u = 0; u < RX_UNROLL; ++u) v[u] = x[(long long)(k + u) * d.ks];
#pragma unroll
      for (int u = 0; u < RX_UNROLL; ++u) mx = max(mx, biased_exp(v[u]));
    }
    for (; k < d.K; ++k) mx = max(mx, biased_exp(x[(long long)k * d.ks]));
    d.E[r] = (int)mx;
    return;
  }
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (r >= d.R) return;
  unsigned mx = 0;
  const double* x = d.X + (long long)r * d.rs;
  int k = lane;
  for (; k + 32 * (RX_UNROLL - 1) < d.K; k += 32 * RX_UNROLL) {
    double v[RX_UNROLL];
#pragma unroll
    for (int u = 0; u < RX_UNROLL; ++u) v[u] = x[(long long)(k + 32 * u) * d.ks];
#pragma unroll
    for (int u = 0; u < RX_UNROLL; ++u) mx = max(mx, biased_exp(v[u]));
  }
  for (; k < d.K; k += 32) mx = max(mx, biased_exp(x[(long long)k * d.ks]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) d.E[r] = (int)mx;
}

// One block per (row tile, 32-wide K chunk): the 7 digit planes of that tile.  A
// descriptor without tiles asks for the row exponents only (k_rowexp).
__global__ void __launch_bounds__(256) k_split(const SplitDesc* __restrict__ descs) {
  const SplitDesc d = descs[blockIdx.y];
  if (!d.tiles) return;
  const int TR = d.row_tile;
  const int nkc = (d.K + OZ_KC - 1) / OZ_KC;
  const int ntr = (d.R + TR - 1) / TR;
  if ((int)blockIdx.x >= ntr * nkc) return;
  const int rt = blockIdx.x / nkc, kc = blockIdx.x % nkc;
  __nv_bfloat16* out =
      static_cast<__nv_bfloat16*>(d.tiles) + (size_t)(rt * nkc + kc) * OZ_S * TR * OZ_KC;
  for (int it = threadIdx.x; it < 4 * TR; it += blockDim.x) {
    int r, kg;
    if (d.ks == 1) { r = it >> 2; kg = it & 3; } else { r = it % TR; kg = it / TR; }
    const int gr = rt * TR + r;
    const unsigned emax = gr < d.R ? (unsigned)d.E[gr] : 0u;
    double x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = kc * OZ_KC + kg * 8 + j;
      x[j] = (gr < d.R && k < d.K) ? d.X[(long long)gr * d.rs + (long long)k * d.ks] : 0.0;
    }
    uint32_t w[OZ_S][4];
    split8(x, emax, w);
    const int off = tile_off32(r, kg * 8);
#pragma unroll
    for (int p = 0; p < OZ_S; ++p)
      *reinterpret_cast<uint4*>(out + (size_t)p * TR * OZ_KC + off) =
          make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
  }
}

// 2^k as a double for any integer k (0 below the subnormal range).
__device__ __forceinline__ double pow2i(int k) {
  if (k >= -1022 && k <= 1023) return __longlong_as_double((long long)(k + 1023) << 52);
  if (k > 1023) return __longlong_as_double(0x7FF0000000000000ll);
  if (k >= -1074) return __longlong_as_double(1ll << (k + 1074));
  return 0.0;
}

// x * 2^k (x an integer with |x| < 2^53, sign flipped when neg) built from its bit
// pattern with integer operations only; exact whenever the result is a normal double.
__device__ __noinline__ double i64_to_double_pow2_slow(long long x, int k, bool neg) {
  return (neg ? -1.0 : 1.0) * (double)x * pow2i(k);
}
__device__ __forceinline__ double i64_to_double_pow2(long long x, int k, bool neg) {
  if (x == 0) return 0.0;
  unsigned long long sgn = (x < 0) != neg ? (1ull << 63) : 0ull;
  const unsigned long long a = x < 0 ? (unsigned long long)(-x) : (unsigned long long)x;
  const int msb = 63 - __clzll((long long)a);
  const long long e = (long long)msb + k + 1023;
  if (e <= 0 || e >= 2047) return i64_to_double_pow2_slow(x, k, neg);  // outside the normal range
  if (msb > 52) return i64_to_double_pow2_slow(x, k, neg);               // |x| >= 2^53: rounded once
  const unsigned long long mant = (a << (52 - msb)) & 0xFFFFFFFFFFFFFull;
  return __longlong_as_double((long long)(sgn | ((unsigned long long)e << 52) | mant));
}

// One output element of a single-chunk product (K <= 128) from its seven group sums:
// V = sum_g a_g 2^(8 (6 - g)), integers with |a_g| < 2^24, times 2^k, negated when neg,
// rounded once to the nearest double (ties to even) without an FP64 addition.
// V = P 2^32 + Q with |P| < 2^40 and |Q| < 2^48 spans up to 73 bits, so it is shifted
// right by t in {0, 7, 13} (chosen from |P|) into one 63-bit integer X: for t = 0 exactly;
// otherwise X keeps at least 55 significant bits and the dropped bits are folded in by
// rounding to odd (a sticky least significant bit).  Rounding X to 53 bits then gives the
// correctly rounded V (round-to-odd at two extra bits, then round-to-nearest, is a single
// correct rounding: Boldo and Melquiond, IEEE Trans. Computers 57(4), 2008), the same
// result as two exact conversions of P 2^32 and Q and one FP64 addition.  The FP64 pipe
// (2 operations per clock per SM) is the scarce unit of this epilogue, and the remaining
// FP64 addition is the one with C.  Outside the normal range the slow path rounds twice.
// The integer part: the 63-bit X (sticky bit folded in) and its shift t in {0, 7, 13}.
__device__ __forceinline__ long long groups_to_x(const int (&a)[OZ_G], int& t) {
  const long long P = (long long)a[0] * 65536 + (long long)a[1] * 256 + a[2];
  const long long Q = (long long)a[3] * 16777216 + (long long)a[4] * 65536 + (long long)a[5] * 256 + a[6];
  const unsigned long long ap = P < 0 ? 0ull - (unsigned long long)P : (unsigned long long)P;
  t = ap < (1ull << 30) ? 0 : (ap < (1ull << 36) ? 7 : 13);
  long long X = (long long)((unsigned long long)P << (32 - t)) + (Q >> t);
  if (Q & ((1ll << t) - 1)) X |= 1;
  return X;
}
// The floating-point part: X 2^(k + t) with its sign flipped when neg.
__device__ __forceinline__ double x_to_double(long long X, int kt, bool neg) {
  if (X == 0) return 0.0;
  long long b = __double_as_longlong(__ll2double_rn(X));
  const int e = (int)((b >> 52) & 0x7FF) + kt;
  if (e <= 0 || e >= 2047) return i64_to_double_pow2_slow(X, kt, neg);
  b += (long long)kt * (1ll << 52);
  if (neg) b ^= (long long)(1ull << 63);
  return __longlong_as_double(b);
}
__device__ __forceinline__ double groups_to_double(const int (&a)[OZ_G], int k, bool neg) {
  int t;
  const long long X = groups_to_x(a, t);
  if (X == 0) return 0.0;
  // X -> double rounds to nearest (the second rounding); 2^(k + t) and the sign go into
  // the bit pattern
  long long b = __double_as_longlong(__ll2double_rn(X));
  const int e = (int)((b >> 52) & 0x7FF) + k + t;
  if (e <= 0 || e >= 2047) return i64_to_double_pow2_slow(X, k + t, neg);
  b += (long long)(k + t) * (1ll << 52);
  if (neg) b ^= (long long)(1ull << 63);
  return __longlong_as_double(b);
}

template <int NT>
struct OzSmem {
  static constexpr int A_BYTES = OZ_S * OZ_M * OZ_KC * 2;  // one stage of A digit tiles
  static constexpr int B_BYTES = OZ_S * NT * OZ_KC * 2;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int NSTAGE = 2;
  static constexpr int BAR_OFF = NSTAGE * STAGE;             // 6 mbarriers
  static constexpr int EXP_OFF = BAR_OFF + 64;               // NT column exponents
  static constexpr int SLOT_OFF = EXP_OFF + NT * 4;          // TMEM address
  static constexpr int FLAG_OFF = SLOT_OFF + 16;             // abort flag
  static constexpr int TOTAL = FLAG_OFF + 16 + 1024;         // + alignment slack
  static constexpr int TMEM_COLS = (OZ_G * NT <= 256) ? 256 : 512;
};

template <int NT>
__global__ void __launch_bounds__(OZ_THREADS, 1) k_ozaki(const OzDesc* __restrict__ descs, double alpha,
                                                        double beta, int flags, unsigned* status, int gmax) {
  using L = OzSmem<NT>;
  const OzDesc d = descs[blockIdx.y];
  const int tiles_m = (d.M + OZ_M - 1) / OZ_M, tiles_n = (d.N + NT - 1) / NT;
  if ((int)blockIdx.x >= tiles_m * tiles_n) return;
  const int bi = blockIdx.x % tiles_m, bj = blockIdx.x / tiles_m;
  if ((flags & GEMM_LOWER) && bj * NT > bi * OZ_M + OZ_M - 1) return;

  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar = sbase + L::BAR_OFF;  // full0 full1 empty0 empty1 tfull tempty
  int* sexp = reinterpret_cast<int*>(smem + L::EXP_OFF);
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + L::SLOT_OFF);
  volatile int* abort_flag = reinterpret_cast<int*>(smem + L::FLAG_OFF);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nkc = (d.K + OZ_KC - 1) / OZ_KC;
  const int nchunk = (nkc + 3) / 4;  // exact-accumulation chunks of 128
  // the wide tile keeps no accumulators across chunks; H and L stay below 2^53 (converted
  // exactly) up to 62 chunks, and below 2^57 (one more rounding each) up to 512
  if ((NT > 32 && nchunk > 1) || nchunk > OZ_MAX_CHUNKS) {
    if (tid == 0) atomicOr(status, ST_INTERNAL);
    return;
  }

  if (tid == 0) {
    mbar_init(bar + 0, 1); mbar_init(bar + 8, 1);
    mbar_init(bar + 16, 1); mbar_init(bar + 24, 1);
    mbar_init(bar + 32, 1); mbar_init(bar + 40, 128);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  for (int j = tid; j < NT; j += OZ_THREADS) {
    const int col = bj * NT + j;
    sexp[j] = col < d.N ? d.Be[col] : 0;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(slot)),
                 "r"(L::TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *slot;

  if (warp == 0) {
    // ---------------- producer: digit tiles of A (128 rows) and B (NT rows) per stage
    if (lane == 0) {
      int issued = 0;
      for (int kc = 0; kc < nkc && !*abort_flag; ++kc) {
        const int s = kc & 1, use = kc >> 1;
        if (!mbar_wait(bar + 16 + 8 * s, (use & 1) ^ 1)) { *abort_flag = 1; break; }
        const uint32_t fb = bar + 8 * s;
        mbar_expect_tx(fb, L::STAGE);
        const __nv_bfloat16* srcA =
            static_cast<const __nv_bfloat16*>(d.At) + (size_t)(bi * nkc + kc) * OZ_S * OZ_M * OZ_KC;
        const __nv_bfloat16* srcB =
            static_cast<const __nv_bfloat16*>(d.Bt) + (size_t)(bj * nkc + kc) * OZ_S * NT * OZ_KC;
        const uint32_t dst = sbase + s * L::STAGE;
#pragma unroll 1
        for (int p = 0; p < OZ_S; ++p) {
          bulk_g2s(dst + p * (OZ_M * OZ_KC * 2), srcA + (size_t)p * OZ_M * OZ_KC, OZ_M * OZ_KC * 2, fb);
          bulk_g2s(dst + L::A_BYTES + p * (NT * OZ_KC * 2), srcB + (size_t)p * NT * OZ_KC, NT * OZ_KC * 2,
                   fb);
        }
        issued = kc + 1;
      }
      // never leave copies in flight: wait (bounded) for the last issued stages to land
      for (int kc = (issued > 2 ? issued - 2 : 0); kc < issued; ++kc)
        mbar_wait(bar + 8 * (kc & 1), (kc >> 1) & 1);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(OZ_M, NT);
      for (int kc = 0; kc < nkc && !*abort_flag; ++kc) {
        const int s = kc & 1, use = kc >> 1, chunk = kc >> 2;
        const bool chunk_start = (kc & 3) == 0;
        if (chunk_start && !mbar_wait(bar + 40, (chunk & 1) ^ 1)) { *abort_flag = 1; break; }
        if (!mbar_wait(bar + 8 * s, use & 1)) { *abort_flag = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a0 = sbase + s * L::STAGE, b0 = a0 + L::A_BYTES;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
#pragma unroll
          for (int g = 2; g <= OZ_S + 1; ++g) {
            if (g > gmax) continue;  // digit groups beyond gmax are not formed
#pragma unroll
            for (int p = 1; p <= OZ_S; ++p) {
              const int q = g - p;
              if (q < 1 || q > OZ_S) continue;
              const uint32_t first = (chunk_start && t == 0 && p == (g - 1 < OZ_S ? 1 : g - OZ_S));
              const uint64_t ad = sdesc(a0 + (p - 1) * (OZ_M * OZ_KC * 2) + t * 256, 128, 512);
              const uint64_t bd = sdesc(b0 + (q - 1) * (NT * OZ_KC * 2) + t * 256, 128, 512);
              mma_bf16(tmem + (g - 2) * NT, ad, bd, idesc, first ? 0u : 1u);
            }
          }
        }
        mma_commit(bar + 16 + 8 * s);                         // stage s may be refilled
        if ((kc & 3) == 3 || kc == nkc - 1) mma_commit(bar + 32);  // 128-chunk complete
      }
    }
  } else {
    // ---------------- epilogue: warps 2..5 own TMEM lanes 32*(warp%4) ..
    // The 7 group sums of a 128-chunk are exact integers (|a_g| < 7 * 2^21); with
    //   H = a2 2^24 + a3 2^16 + a4 2^8,   L = a5 2^24 + a6 2^16 + a7 2^8 + a8
    // (a_g the sum of group g) the chunk's value is (H 2^24 + L) 2^-48 in units of
    // 2^(E_i + F_j - 14).  |H| < 2^45.1 and |L| < 2^47.1 per chunk, so their sums stay
    // below 2^53 for up to 62 chunks (converted exactly, beyond that rounded once each) and
    // are accumulated exactly in int64 and rounded once, by one FMA, at the end.
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    const int gi = bi * OZ_M + row;
    const int ei = gi < d.M ? d.Ae[gi] : 0;
    const bool unit_alpha = alpha == 1.0 || alpha == -1.0;
    const bool neg_alpha = alpha < 0.0;
    // alpha * 2^(E_i + F_j - 62) * (H 2^24 + L), with the scaling folded into the exponent
    // fields: two exact integer-to-double conversions and one rounding add.
    auto product = [&](long long H, long long Lw, int fj) -> double {
      if (ei == 0 || fj == 0) return 0.0;
      const int k = ei + fj - 2044 - 62;
      double v = i64_to_double_pow2(H, k + 24, neg_alpha) + i64_to_double_pow2(Lw, k, neg_alpha);
      return unit_alpha ? v : v * (neg_alpha ? -alpha : alpha);
    };
    auto finish = [&](long long H, long long Lw, int j) {
      const int gj = bj * NT + j;
      if (gi >= d.M || gj >= d.N) return;
      double v = product(H, Lw, sexp[j]);
      if ((flags & GEMM_ADD_IDENTITY) && gi == gj) v += 1.0;
      double* cp = d.C + (size_t)gi * d.c_rs + (size_t)gj * d.c_cs;
      if (beta == 0.0) *cp = v;
      else if (beta == 1.0) *cp = *cp + v;
      else *cp = fma(beta, *cp, v);
    };
    auto group_words = [&](const uint32_t (&v)[OZ_G][8], int j, long long& H, long long& Lw) {
      int a[OZ_G];
#pragma unroll
      for (int g = 0; g < OZ_G; ++g) a[g] = __float2int_rn(__uint_as_float(v[g][j]));
      H = ((long long)a[0] << 24) + ((long long)a[1] << 16) + ((long long)a[2] << 8);
      Lw = ((long long)a[3] << 24) + ((long long)a[4] << 16) + ((long long)a[5] << 8) + a[6];
    };
    bool ok = true;
    if (nchunk <= 1 || NT > 32) {
      // single 128-chunk (K <= 128): no persistent accumulators.  The C values this thread
      // updates are fetched before waiting for the MMAs, so their latency overlaps them.
      double cv[NT];
      const bool need_c = beta != 0.0 && gi < d.M;
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const int gj = bj * NT + j;
        cv[j] = (need_c && gj < d.N) ? d.C[(size_t)gi * d.c_rs + (size_t)gj * d.c_cs] : 0.0;
      }
      if (nchunk == 1) {
        if (!mbar_wait_warp(bar + 32, 0)) { ok = false; *abort_flag = 1; }
        asm volatile("tcgen05.fence::after_thread_sync;");
      }
      if (ok) {  // warp-uniform: every lane takes part in the tcgen05.ld below
#pragma unroll
        for (int cb = 0; cb < NT / 8; ++cb) {
          uint32_t v[OZ_G][8];
          if (nchunk == 1) {
#pragma unroll
            for (int g = 0; g < OZ_G; ++g) {
              if (g + 2 <= gmax) tmem_ld8(lane_base + g * NT + cb * 8, v[g]);
              else for (int j = 0; j < 8; ++j) v[g][j] = 0u;
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;");
          } else {
#pragma unroll
            for (int g = 0; g < OZ_G; ++g)
#pragma unroll
              for (int j = 0; j < 8; ++j) v[g][j] = 0u;
          }
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int jj = cb * 8 + j, gj = bj * NT + jj;
            if (gi < d.M && gj < d.N) {
              long long H, Lw;
              group_words(v, j, H, Lw);
              double pv = product(H, Lw, sexp[jj]);
              if ((flags & GEMM_ADD_IDENTITY) && gi == gj) pv += 1.0;
              d.C[(size_t)gi * d.c_rs + (size_t)gj * d.c_cs] =
                  beta == 0.0 ? pv : (beta == 1.0 ? cv[jj] + pv : fma(beta, cv[jj], pv));
            }
          }
        }
      }
    } else {
      long long H[NT], Lw[NT];
#pragma unroll
      for (int j = 0; j < NT; ++j) { H[j] = 0; Lw[j] = 0; }
      for (int c = 0; c < nchunk; ++c) {
        if (!mbar_wait_warp(bar + 32, c & 1)) { ok = false; *abort_flag = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
        for (int cb = 0; cb < NT / 8; ++cb) {
          uint32_t v[OZ_G][8];
#pragma unroll
          for (int g = 0; g < OZ_G; ++g) {
              if (g + 2 <= gmax) tmem_ld8(lane_base + g * NT + cb * 8, v[g]);
              else for (int j = 0; j < 8; ++j) v[g][j] = 0u;
            }
          asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            long long h, l;
            group_words(v, j, h, l);
            H[cb * 8 + j] += h;
            Lw[cb * 8 + j] += l;
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        mbar_arrive(bar + 40);
      }
      if (ok) {
#pragma unroll
        for (int j = 0; j < NT; ++j) finish(H[j], Lw[j], j);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0 && *abort_flag) atomicOr(status, ST_TIMEOUT);
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(L::TMEM_COLS));
  }
}



// ---------------------------------------------------------------------------------------
// FP32 GEMM on the tensor cores at FP32 accuracy (the warm-start network's layers):
// C = op(A) op(B) as three TF32 products of a hi/lo split of both operands, x = hi + lo with
// hi the TF32 value nearest x (sign, exponent, 10 mantissa bits) and lo = x - hi (exact in
// FP32, |lo| <= 2^-11 |hi|):  A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi.  The dropped A_lo B_lo
// and the TF32 reading of lo leave a relative error of about 2^-21 per product term, against
// 2^-24 for an FP32 FMA chain.  k_tf32_split writes both planes of an operand in the tcgen05
// K-major no-swizzle canonical layout (the digit planes' byte geometry: 16 floats of K per
// 64-byte row segment, tiles [row tile][k chunk]); k_tf32x3 computes one 128 x 64 tile of C
// per CTA: warp 0 streams the stages of both operands (4-deep ring) with cp.async.bulk, one
// thread of warp 1 issues the 6 MMAs (kind::tf32, 128 x 64 x 8) of each 16-wide K chunk into
// one TMEM accumulator, and warps 2..5 read it back (a row per thread) and apply the
// layer's epilogue: C = AB; Z = AB + bias, C = gelu(Z); C = AB + bias; C = AB gelu'(Z).
constexpr int TF_KC = 16;                       // floats of K per stage
constexpr int TF_M = 128, TF_N = 64;
constexpr int TF_PA = TF_M * TF_KC;             // floats of one plane of an A stage
constexpr int TF_PB = TF_N * TF_KC;
constexpr int TF_A = 2 * TF_PA * 4;             // bytes of the A stage (hi, lo): 16 KB
constexpr int TF_B = 2 * TF_PB * 4;             // 8 KB
constexpr int TF_STAGE = TF_A + TF_B;
constexpr int TF_NS = 4;
constexpr int TF_BAR = TF_NS * TF_STAGE;        // FULL[4] EMPTY[4] TFULL
constexpr int TF_SLOT = TF_BAR + 80;
constexpr int TF_FLAG = TF_SLOT + 16;
constexpr int TF_SMEM = TF_FLAG + 16 + 1024;
static_assert(TF_SMEM <= 227 * 1024, "TF32 product exceeds the shared memory of one CTA");

// Float offset of (r, k) in an R x 16 tile: [r/8][k/4][r%8][k%4] (8 x 16-byte core matrices).
__device__ __forceinline__ int tf_off(int r, int k) {
  return (((r >> 3) * 4 + (k >> 2)) << 5) + ((r & 7) << 2) + (k & 3);
}
// kind::tf32 instruction descriptor: FP32 accumulator, TF32 A and B, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

struct TfSplit {
  const float* X;
  long long rs, ks;  // element (r, k) at X[r * rs + k * ks]
  int R, K, TR;      // rows, K, rows per tile
  float* tiles;
};

// One block per (row tile, 16-wide K chunk) of each of the two operands (blockIdx.y).
__global__ void __launch_bounds__(256) k_tf32_split(const TfSplit a, const TfSplit b) {
  const TfSplit d = blockIdx.y == 0 ? a : b;
  const int nkc = (d.K + TF_KC - 1) / TF_KC, ntr = (d.R + d.TR - 1) / d.TR;
  if ((int)blockIdx.x >= ntr * nkc) return;
  const int rt = blockIdx.x / nkc, kc = blockIdx.x % nkc;
  float* hi = d.tiles + (size_t)(rt * nkc + kc) * 2 * d.TR * TF_KC;
  float* lo = hi + (size_t)d.TR * TF_KC;
  for (int it = threadIdx.x; it < 4 * d.TR; it += blockDim.x) {
    int r, kg;  // row, 4-wide k group; consecutive threads along the operand's contiguous index
    if (d.ks == 1) { r = it >> 2; kg = it & 3; } else { r = it % d.TR; kg = it / d.TR; }
    const int gr = rt * d.TR + r;
    float h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = kc * TF_KC + kg * 4 + j;
      const float x = (gr < d.R && k < d.K) ? d.X[(long long)gr * d.rs + (long long)k * d.ks] : 0.0f;
      h[j] = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);  // nearest TF32 (ties up)
      l[j] = x - h[j];
    }
    const int off = tf_off(r, kg * 4);
    *reinterpret_cast<float4*>(hi + off) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4*>(lo + off) = make_float4(l[0], l[1], l[2], l[3]);
  }
}

struct TfGemm {
  const float *At, *Bt;  // split planes of op(A) (M x K, 128-row tiles) and op(B)^T (N x K, 64-row tiles)
  float* C;
  int ldc, M, N, K;
  const float* bias;
  float* Z;
  int ldz;
};

__device__ __forceinline__ float tf_gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float tf_gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

template <int EPI>
__global__ void __launch_bounds__(192, 1) k_tf32x3(const TfGemm g, unsigned* status) {
  const int tiles_m = (g.M + TF_M - 1) / TF_M;
  const int bi = blockIdx.x % tiles_m, bj = blockIdx.x / tiles_m;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t sbase = smem_u32(smem);
  const uint32_t FULL = sbase + TF_BAR, EMPTY = FULL + 8 * TF_NS, TFULL = EMPTY + 8 * TF_NS;
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + TF_SLOT);
  volatile int* abort_flag = reinterpret_cast<int*>(smem + TF_FLAG);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nkc = (g.K + TF_KC - 1) / TF_KC;
  if (tid == 0) {
    for (int i = 0; i < TF_NS; ++i) {
      mbar_init(FULL + 8 * i, 1);
      mbar_init(EMPTY + 8 * i, 1);
    }
    mbar_init(TFULL, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(TF_N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *slot;

  if (warp == 0) {
    // ---------------- producer: one stage (both planes of both operands) per K chunk
    if (lane == 0) {
      int issued = 0;
      for (int kc = 0; kc < nkc && !*abort_flag; ++kc) {
        const int s = kc % TF_NS, use = kc / TF_NS;
        if (!mbar_wait(EMPTY + 8 * s, (use & 1) ^ 1)) { *abort_flag = 1; break; }
        mbar_expect_tx(FULL + 8 * s, TF_STAGE);
        const uint32_t dst = sbase + s * TF_STAGE;
        bulk_g2s(dst, g.At + (size_t)(bi * nkc + kc) * 2 * TF_PA, TF_A, FULL + 8 * s);
        bulk_g2s(dst + TF_A, g.Bt + (size_t)(bj * nkc + kc) * 2 * TF_PB, TF_B, FULL + 8 * s);
        issued = kc + 1;
      }
      // never leave copies in flight: wait (bounded) for the last issued stages to land
      for (int kc = (issued > TF_NS ? issued - TF_NS : 0); kc < issued; ++kc)
        mbar_wait(FULL + 8 * (kc % TF_NS), (kc / TF_NS) & 1);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(TF_M, TF_N);
      for (int kc = 0; kc < nkc && !*abort_flag; ++kc) {
        const int s = kc % TF_NS, use = kc / TF_NS;
        if (!mbar_wait(FULL + 8 * s, use & 1)) { *abort_flag = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t ahi = sbase + s * TF_STAGE, alo = ahi + TF_PA * 4;
        const uint32_t bhi = ahi + TF_A, blo = bhi + TF_PB * 4;
#pragma unroll
        for (int t = 0; t < 2; ++t) {  // two 8-wide k-steps: 2 core matrices (32 bytes) each
          const uint64_t ah = sdesc(ahi + t * 256, 128, 512), al = sdesc(alo + t * 256, 128, 512);
          const uint64_t bh = sdesc(bhi + t * 256, 128, 512), bl = sdesc(blo + t * 256, 128, 512);
          mma_tf32(tmem, ah, bh, idesc, (kc > 0 || t > 0) ? 1u : 0u);
          mma_tf32(tmem, ah, bl, idesc, 1u);
          mma_tf32(tmem, al, bh, idesc, 1u);
        }
        mma_commit(EMPTY + 8 * s);  // stage s may be refilled
      }
      mma_commit(TFULL);
    }
  } else {
    // ---------------- epilogue: warps 2..5 own TMEM lanes 32*(warp%4) .. (rows of the tile)
    const int quarter = warp & 3, row = quarter * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quarter * 32) << 16);
    const int gi = bi * TF_M + row;
    if (!mbar_wait_warp(TFULL, 0)) {
      *abort_flag = 1;
    } else if (!*abort_flag) {  // warp-uniform (the flag is read after the barrier completed)
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll 1
      for (int cb = 0; cb < TF_N / 8; ++cb) {
        uint32_t v[8];
        tmem_ld8(lane_base + cb * 8, v);
        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int gj = bj * TF_N + cb * 8 + j;
          if (gi >= g.M || gj >= g.N) continue;
          float x = __uint_as_float(v[j]);
          if (EPI == 1) {
            x += g.bias[gj];
            g.Z[(size_t)gi * g.ldz + gj] = x;
            x = tf_gelu(x);
          } else if (EPI == 2) {
            x += g.bias[gj];
          } else if (EPI == 3) {
            x *= tf_gelu_grad(g.Z[(size_t)gi * g.ldz + gj]);
          }
          g.C[(size_t)gi * g.ldc + gj] = x;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0 && *abort_flag) atomicOr(status, ST_TIMEOUT);
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TF_N));
  }
}

// ---------------------------------------------------------------------------------------
// Wide-K product with the digit split of the FP64 A operand fused in: C = A B^T with A
// (M x K, element (i, k) at A[i * a_rs + k], K contiguous) read from HBM once, and B
// (N <= 32) already split.  One CTA per 128-row tile of A.  Sixteen worker warps load the
// FP64 tile of each 32-wide K step (one 64-byte row segment per thread, the next step's
// segment prefetched), write its 7 BF16 digit planes into a 3-stage shared-memory ring in
// the MMA's canonical layout, and drain the TMEM group sums of each 128-wide chunk into
// exact int64 words; warp 0 streams the B planes with cp.async.bulk, one thread of warp 1
// issues the 28 digit-pair MMAs per 16-wide k-step into one of two TMEM accumulator sets,
// so the MMAs of chunk c+1 run while chunk c is drained.  Digit planes never touch HBM:
// 8 bytes per element of A instead of 8 (split read) + 14 (planes written) + 14 (planes
// read).
constexpr int FA_WORKERS = 16;
constexpr int FA_THREADS = 32 * (2 + FA_WORKERS);
constexpr int FA_NS = 3;
constexpr int FA_A = OZ_S * OZ_M * OZ_KC * 2;     // 57344 B of A planes per stage
constexpr int FA_B = OZ_S * 32 * OZ_KC * 2;       // 14336 B of B planes per stage
constexpr int FA_STAGE = FA_A + FA_B;
constexpr int FA_BAR = FA_NS * FA_STAGE;          // FULL[3] EMPTY[3] TFULL[2] TEMPTY[2] DONE
constexpr int FA_SLOT = FA_BAR + 128;
constexpr int FA_FLAG = FA_SLOT + 16;
constexpr int FA_SMEM = FA_FLAG + 16 + 1024;
static_assert(FA_SMEM <= 227 * 1024, "fused product exceeds the shared memory of one CTA");
static_assert(FA_WORKERS * 32 == 4 * OZ_M, "one worker thread per (row, 8-wide k group)");

// Split K: every CTA of a tile counts itself once it has added its part (or had no K range);
// the last one builds C from the accumulator (the two exact int64 words of every element,
// summed by integer atomics, so in any order the same) with the epilogue's arithmetic, and
// clears the accumulator and the count for the next product.  All threads of the CTA call it.
__device__ __forceinline__ void fa_splitk_finish(const OzDesc& d, int tid) {
  __shared__ int is_last;
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(d.hl) + OZ_HL_WORDS;
  if (tid == 0) is_last = atomicAdd(cnt, 1ull) == (unsigned long long)(gridDim.z - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  long long* hl = d.hl;
  for (int e = tid; e < d.M * 32; e += FA_THREADS) {
    const int row = e >> 5, col = e & 31;
    if (col >= d.N) continue;
    long long* hp = hl + 2 * (size_t)e;
    const long long H = __ldcg(hp), Lw = __ldcg(hp + 1);
    hp[0] = 0;
    hp[1] = 0;
    const int ed = (row < d.lead ? d.Ae2 : d.Ae)[row];
    const int fj = d.Be[col];
    double v = 0.0;
    if (ed != 0 && fj != 0) {
      const int k = ed + fj - 2044 - 62;
      v = i64_to_double_pow2(H, k + 24, false) + i64_to_double_pow2(Lw, k, false);
    }
    d.C[(size_t)row * d.c_rs + (size_t)col * d.c_cs] = v;
  }
  if (tid == 0) *cnt = 0ull;
}

__global__ void __launch_bounds__(FA_THREADS, 1) k_ozaki_fa(const OzDesc* __restrict__ descs,
                                                           unsigned* status, int gmax) {
  const OzDesc d = descs[blockIdx.y];
  const int tiles_m = (d.M + OZ_M - 1) / OZ_M;
  if ((int)blockIdx.x >= tiles_m) return;
  if (d.N > 32) {
    if (threadIdx.x == 0) atomicOr(status, ST_INTERNAL);
    return;
  }
  const int bi = blockIdx.x;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar = sbase + FA_BAR;
  // FULL: the workers' A planes are in; BFULL: the B planes landed (tracked on their own so
  // the producer can always wait for its copies); EMPTY: the MMAs of a stage completed.
  const uint32_t FULL = bar, BFULL = bar + 24, EMPTY = bar + 48, TFULL = bar + 72, TEMPTY = bar + 88,
                 DONE = bar + 104;
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + FA_SLOT);
  volatile int* abort_flag = reinterpret_cast<int*>(smem + FA_FLAG);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nkc_all = (d.K + OZ_KC - 1) / OZ_KC;
  const int nch_all = (nkc_all + 3) / 4;  // 128-wide chunks; H, L exact below 2^53 up to 62 of them
  if (nch_all > OZ_MAX_CHUNKS || (d.hl && tiles_m > 1)) {
    if (threadIdx.x == 0) atomicOr(status, ST_INTERNAL);
    return;
  }
  // split K (gridDim.z > 1, with the int64 accumulator d.hl): this CTA takes the chunks
  // [c0, c1); below, kc and the chunk counts are local to that range, kb its first step
  const int per = (nch_all + gridDim.z - 1) / gridDim.z;
  const int c0 = (int)blockIdx.z * per, c1 = min(nch_all, c0 + per);
  if (c0 >= c1) {  // no K range here: only counted
    if (d.hl && gridDim.z > 1) fa_splitk_finish(d, threadIdx.x);
    return;
  }
  const int kb = c0 * 4;
  const int nkc = min(nkc_all, c1 * 4) - kb;
  const int nch = (nkc + 3) / 4;

  if (tid == 0) {
    for (int i = 0; i < FA_NS; ++i) {
      mbar_init(FULL + 8 * i, 32 * FA_WORKERS);
      mbar_init(BFULL + 8 * i, 1);
      mbar_init(EMPTY + 8 * i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(TFULL + 8 * i, 1);
      mbar_init(TEMPTY + 8 * i, 32 * FA_WORKERS);
    }
    mbar_init(DONE, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *slot;

  if (warp == 0) {
    // ---------------- B planes (N <= 32 rows: a single column tile)
    if (lane == 0) {
      int issued = 0;
      for (int kc = 0; kc < nkc && !*abort_flag; ++kc) {
        const int s = kc % FA_NS, use = kc / FA_NS;
        if (!mbar_wait(EMPTY + 8 * s, (use & 1) ^ 1)) { *abort_flag = 1; break; }
        mbar_expect_tx(BFULL + 8 * s, FA_B);
        const __nv_bfloat16* src = static_cast<const __nv_bfloat16*>(d.Bt) + (size_t)(kb + kc) * OZ_S * 32 * OZ_KC;
        bulk_g2s(sbase + s * FA_STAGE + FA_A, src, FA_B, BFULL + 8 * s);
        issued = kc + 1;
      }
      for (int kc = (issued > FA_NS ? issued - FA_NS : 0); kc < issued; ++kc)
        mbar_wait(BFULL + 8 * (kc % FA_NS), (kc / FA_NS) & 1);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(OZ_M, 32);
      for (int kc = 0; kc < nkc && !*abort_flag; ++kc) {
        const int s = kc % FA_NS, use = kc / FA_NS, c = kc >> 2, buf = c & 1;
        const bool chunk_start = (kc & 3) == 0;
        if (chunk_start && !mbar_wait(TEMPTY + 8 * buf, ((c >> 1) & 1) ^ 1)) { *abort_flag = 1; break; }
        if (!mbar_wait(BFULL + 8 * s, use & 1) || !mbar_wait(FULL + 8 * s, use & 1)) {
          *abort_flag = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a0 = sbase + s * FA_STAGE, b0 = a0 + FA_A;
        const uint32_t dbase = tmem + buf * (OZ_G * 32);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
#pragma unroll
          for (int g = 2; g <= OZ_S + 1; ++g) {
            if (g > gmax) continue;  // digit groups beyond gmax are not formed
#pragma unroll
            for (int p = 1; p <= OZ_S; ++p) {
              const int q = g - p;
              if (q < 1 || q > OZ_S) continue;
              const uint32_t first = (chunk_start && t == 0 && p == (g - 1 < OZ_S ? 1 : g - OZ_S));
              const uint64_t ad = sdesc(a0 + (p - 1) * (OZ_M * OZ_KC * 2) + t * 256, 128, 512);
              const uint64_t bd = sdesc(b0 + (q - 1) * (32 * OZ_KC * 2) + t * 256, 128, 512);
              mma_bf16(dbase + (g - 2) * 32, ad, bd, idesc, first ? 0u : 1u);
            }
          }
        }
        mma_commit(EMPTY + 8 * s);
        if ((kc & 3) == 3 || kc == nkc - 1) mma_commit(TFULL + 8 * buf);
      }
      // every MMA issued so far completes before the accumulators are released
      mma_commit(DONE);
      mbar_wait(DONE, 0);
    }
  } else {
    // ---------------- workers: split A, drain TMEM
    // split item: tile row r, 8-wide k group kg.  A warp covers 8 rows x 4 groups with the
    // 8 lanes of each quarter-warp on 8 rows of one group, so their 16-byte digit stores
    // fill 128 contiguous bytes (no bank conflict).
    const int ew = warp - 2;
    const int r = ew * 8 + (lane & 7), kg = lane >> 3;
    const int gi = bi * OZ_M + r;
    const bool row_ok = gi < d.M;
    const unsigned emax = row_ok ? (unsigned)(gi < d.lead ? d.Ae2 : d.Ae)[gi] : 0u;
    const double* rowp = static_cast<const double*>(gi < d.lead ? d.At2 : d.At) + (row_ok ? (size_t)gi * d.a_rs : 0);
    const bool vec = ((reinterpret_cast<uintptr_t>(rowp) | (uintptr_t)d.a_rs * 8) & 15) == 0;
    const int quarter = warp & 3, col0 = (ew >> 2) * 8;  // drain: TMEM lane quarter, 8 columns
    const int drow = bi * OZ_M + quarter * 32 + lane;
    auto load = [&](int kc, double (&x)[8]) {
      const int k0 = (kb + kc) * OZ_KC + kg * 8;
      if (row_ok && vec && k0 + 8 <= d.K) {
        const double2* p2 = reinterpret_cast<const double2*>(rowp + k0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const double2 v = p2[j];
          x[2 * j] = v.x;
          x[2 * j + 1] = v.y;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = (row_ok && k0 + j < d.K) ? rowp[k0 + j] : 0.0;
      }
    };
    long long H[8], Lw[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) { H[j] = 0; Lw[j] = 0; }
    bool alive = true;
    auto drain = [&](int c) {
      const int buf = c & 1;
      if (!mbar_wait_warp(TFULL + 8 * buf, (c >> 1) & 1)) { alive = false; *abort_flag = 1; return; }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t lb = tmem + ((uint32_t)(quarter * 32) << 16) + buf * (OZ_G * 32) + col0;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        uint32_t v[OZ_G][4];
#pragma unroll
        for (int g = 0; g < OZ_G; ++g) {
          if (g + 2 <= gmax) tmem_ld4(lb + g * 32 + half * 4, v[g]);
          else for (int j = 0; j < 4; ++j) v[g][j] = 0u;
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (half == 1) {
          asm volatile("tcgen05.fence::before_thread_sync;");
          mbar_arrive(TEMPTY + 8 * buf);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          int a[OZ_G];
#pragma unroll
          for (int g = 0; g < OZ_G; ++g) a[g] = __float2int_rn(__uint_as_float(v[g][j]));
          H[half * 4 + j] += ((long long)a[0] << 24) + ((long long)a[1] << 16) + ((long long)a[2] << 8);
          Lw[half * 4 + j] +=
              ((long long)a[3] << 24) + ((long long)a[4] << 16) + ((long long)a[5] << 8) + a[6];
        }
      }
    };
    double xn[8];
    load(0, xn);
    for (int kc = 0; kc < nkc && alive; ++kc) {
      const int s = kc % FA_NS, use = kc / FA_NS;
      uint32_t w[OZ_S][4];
      split8(xn, emax, w);
      if (kc + 1 < nkc) load(kc + 1, xn);  // in flight while this step is stored
      if (!mbar_wait_warp(EMPTY + 8 * s, (use & 1) ^ 1)) { alive = false; *abort_flag = 1; break; }
      unsigned char* stA = smem + s * FA_STAGE;
      const int off = tile_off32(r, kg * 8);
#pragma unroll
      for (int p = 0; p < OZ_S; ++p)
        *reinterpret_cast<uint4*>(stA + 2 * ((size_t)p * OZ_M * OZ_KC + off)) =
            make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(FULL + 8 * s);
      if (((kc & 3) == 3 || kc == nkc - 1) && (kc >> 2) >= 1) drain((kc >> 2) - 1);
    }
    if (alive && nch >= 1) drain(nch - 1);
    if (alive && drow < d.M && d.hl) {
      // split K: the exact integer words go to the accumulator (one 128 x 32 tile), added in
      // any order with the same result; the tile's last CTA builds C from them (below)
      unsigned long long* hp = reinterpret_cast<unsigned long long*>(d.hl) + ((size_t)drow * 32 + col0) * 2;
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (col0 + j < d.N) {
          atomicAdd(hp + 2 * j, (unsigned long long)H[j]);
          atomicAdd(hp + 2 * j + 1, (unsigned long long)Lw[j]);
        }
      __threadfence();  // the additions are visible before this CTA is counted
    } else if (alive && drow < d.M) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int gj = col0 + j;
        if (gj < d.N) {
          const int fj = d.Be[gj];
          double v = 0.0;
          const int ed = (drow < d.lead ? d.Ae2 : d.Ae)[drow];
          if (ed != 0 && fj != 0) {
            const int k = ed + fj - 2044 - 62;
            v = i64_to_double_pow2(H[j], k + 24, false) + i64_to_double_pow2(Lw[j], k, false);
          }
          d.C[(size_t)drow * d.c_rs + (size_t)gj * d.c_cs] = v;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0 && *abort_flag) atomicOr(status, ST_TIMEOUT);
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
  if (d.hl && gridDim.z > 1) fa_splitk_finish(d, tid);
}

// ---------------------------------------------------------------------------------------
// Wide-K product with the digit split of the FP64 B operand fused in: C = A B^T (or its
// negation, optionally plus the identity: descriptor flags in tile0) with A (M <= 128
// rows, one row tile) already split, and B (N rows, element (j, k) at B[j * a_rs + k], K
// contiguous; rows j < lead from At2 with exponent bounds Ae2) read from HBM once and split
// in the kernel.  One CTA per 32-row tile of B.  This is the
// orientation of the outer-block W1 product of the two-level QR: A = V_o^T (all the
// block's reflectors, M = the block width) and B = the trailing columns, so every trailing
// column is split once per outer block, where the A-operand form would split it once per
// 32-column slice of V_o.  Warp 0 streams the A planes of each 32-wide K step with
// cp.async.bulk into a 3-stage ring; the 16 worker warps form 4 groups, group g splitting
// the B tile of the K steps kc = g mod 4 into its own buffer (one 8-wide k group of one
// row per thread, the group's next step prefetched); one thread of warp 1 issues the 28
// digit-pair MMAs per 16-wide k-step into one of two TMEM accumulator sets; and all 16
// worker warps drain each 128-wide chunk into exact int64 words while the MMAs of the
// next one run.  Every mbarrier is waited on one phase at a time by each waiter (the A
// ring in step order by the producer and the MMA thread, each B buffer by its own group
// and the MMA thread), so the parity waits cannot alias a phase two steps away.
constexpr int FB_NS = 3;                           // A stages
constexpr int FB_A = OZ_S * OZ_M * OZ_KC * 2;     // 57344 B of A planes per stage
// NBC columns of C (rows of B) per CTA:
//   32: 16 worker warps in 4 splitting groups (group g splits the K steps g mod 4 into its
//       own B buffer), two TMEM accumulator sets (the drain of one chunk overlaps the MMAs
//       of the next), 8 columns per drain thread;
//   64: 8 worker warps splitting every step into a ring of 2 B buffers, one accumulator set
//       (the 7 group accumulators of a 128 x 64 tile take 448 of the 512 TMEM columns), 32
//       columns per drain thread (registers allow it with 10 warps per CTA); its N = 64 MMAs
//       read each A plane once for twice the columns.
template <int NBC>
struct FbCfg {
  static constexpr int WORKERS = NBC == 32 ? 16 : 8;
  static constexpr int THREADS = 32 * (2 + WORKERS);
  static constexpr int NGRP = NBC == 32 ? 4 : 1;          // splitting groups
  static constexpr int GW = WORKERS / NGRP;               // warps per group
  static constexpr int NBB = NGRP == 1 ? 2 : NGRP;        // B buffers
  static constexpr int NBUF = NBC == 32 ? 2 : 1;          // TMEM accumulator sets
  static constexpr int B = OZ_S * NBC * OZ_KC * 2;        // B planes per buffer
  static constexpr int BOFF = FB_NS * FB_A;
  static constexpr int BAR = BOFF + NBB * B;              // AFULL[3] AEMPTY[3] BFULL[4] BEMPTY[4] TFULL[2] TEMPTY[2] DONE
  static constexpr int SLOT = BAR + 160;
  static constexpr int FLAG = SLOT + 16;
  static constexpr int SMEM = FLAG + 16 + 1024;
  static constexpr int DCOLS = NBC / (WORKERS / 4);       // columns each drain thread owns
  static_assert(SMEM <= 227 * 1024, "B-split product exceeds the shared memory of one CTA");
  static_assert(GW * 32 == NBC * 4, "one splitting thread per (row, 8-wide k group)");
  static_assert(NBB <= 4, "four B barrier pairs");
};

template <int NBC>
__global__ void __launch_bounds__(FbCfg<NBC>::THREADS, 1) k_ozaki_fb(const OzDesc* __restrict__ descs,
                                                           unsigned* status, int gmax) {
  using C = FbCfg<NBC>;
  const OzDesc d = descs[blockIdx.y];
  const int tiles_n = (d.N + NBC - 1) / NBC;
  if ((int)blockIdx.x >= tiles_n) return;
  if (d.M > OZ_M) {
    if (threadIdx.x == 0) atomicOr(status, ST_INTERNAL);
    return;
  }
  const int bj = blockIdx.x;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar = sbase + C::BAR;
  const uint32_t AFULL = bar, AEMPTY = bar + 24, BFULL = bar + 48, BEMPTY = bar + 80, TFULL = bar + 112,
                 TEMPTY = bar + 128, DONE = bar + 144;
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + C::SLOT);
  volatile int* abort_flag = reinterpret_cast<int*>(smem + C::FLAG);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nkc = (d.K + OZ_KC - 1) / OZ_KC;
  const int nch = (nkc + 3) / 4;
  if (nch > OZ_MAX_CHUNKS) {
    if (threadIdx.x == 0) atomicOr(status, ST_INTERNAL);
    return;
  }

  if (tid == 0) {
    for (int i = 0; i < FB_NS; ++i) {
      mbar_init(AFULL + 8 * i, 1);
      mbar_init(AEMPTY + 8 * i, 1);
    }
    for (int i = 0; i < C::NBB; ++i) {
      mbar_init(BFULL + 8 * i, 32 * C::GW);   // the warps of the group that fills buffer i
      mbar_init(BEMPTY + 8 * i, 1);
    }
    for (int i = 0; i < C::NBUF; ++i) {
      mbar_init(TFULL + 8 * i, 1);
      mbar_init(TEMPTY + 8 * i, 32 * C::WORKERS);
    }
    mbar_init(DONE, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *slot;

  if (warp == 0) {
    // ---------------- A planes (the single 128-row tile), in step order
    if (lane == 0) {
      int issued = 0;
      for (int kc = 0; kc < nkc && !*abort_flag; ++kc) {
        const int s = kc % FB_NS, use = kc / FB_NS;
        if (!mbar_wait(AEMPTY + 8 * s, (use & 1) ^ 1)) { *abort_flag = 1; break; }
        mbar_expect_tx(AFULL + 8 * s, FB_A);
        const __nv_bfloat16* src = static_cast<const __nv_bfloat16*>(d.At) + (size_t)kc * OZ_S * OZ_M * OZ_KC;
        bulk_g2s(sbase + s * FB_A, src, FB_A, AFULL + 8 * s);
        issued = kc + 1;
      }
      for (int kc = (issued > FB_NS ? issued - FB_NS : 0); kc < issued; ++kc)
        mbar_wait(AFULL + 8 * (kc % FB_NS), (kc / FB_NS) & 1);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(OZ_M, NBC);
      for (int kc = 0; kc < nkc && !*abort_flag; ++kc) {
        const int s = kc % FB_NS, use = kc / FB_NS, c = kc >> 2, gb = kc % C::NBB;
        const int buf = C::NBUF == 2 ? (c & 1) : 0, tuse = C::NBUF == 2 ? (c >> 1) : c;
        const bool chunk_start = (kc & 3) == 0;
        if (chunk_start && !mbar_wait(TEMPTY + 8 * buf, (tuse & 1) ^ 1)) { *abort_flag = 1; break; }
        if (!mbar_wait(AFULL + 8 * s, use & 1) || !mbar_wait(BFULL + 8 * gb, (kc / C::NBB) & 1)) {
          *abort_flag = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a0 = sbase + s * FB_A, b0 = sbase + C::BOFF + gb * C::B;
        const uint32_t dbase = tmem + buf * (OZ_G * NBC);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
#pragma unroll
          for (int g = 2; g <= OZ_S + 1; ++g) {
            if (g > gmax) continue;  // digit groups beyond gmax are not formed
#pragma unroll
            for (int p = 1; p <= OZ_S; ++p) {
              const int q = g - p;
              if (q < 1 || q > OZ_S) continue;
              const uint32_t first = (chunk_start && t == 0 && p == (g - 1 < OZ_S ? 1 : g - OZ_S));
              const uint64_t ad = sdesc(a0 + (p - 1) * (OZ_M * OZ_KC * 2) + t * 256, 128, 512);
              const uint64_t bd = sdesc(b0 + (q - 1) * (NBC * OZ_KC * 2) + t * 256, 128, 512);
              mma_bf16(dbase + (g - 2) * NBC, ad, bd, idesc, first ? 0u : 1u);
            }
          }
        }
        mma_commit(AEMPTY + 8 * s);
        mma_commit(BEMPTY + 8 * gb);
        if ((kc & 3) == 3 || kc == nkc - 1) mma_commit(TFULL + 8 * buf);
      }
      mma_commit(DONE);
      mbar_wait(DONE, 0);
    }
  } else {
    // ---------------- workers: split B (group grp takes the K steps kc = grp mod NGRP, into
    // buffer kc mod NBB, in step order), drain TMEM
    const int ew = warp - 2, grp = ew / C::GW;
    // split item: tile row r, 8-wide k group kg; the 8 lanes of each quarter-warp cover 8
    // rows of one k group, so their 16-byte digit stores fill 128 contiguous bytes
    const int r = (ew % C::GW) * 8 + (lane & 7), kg = lane >> 3;
    const int gj = bj * NBC + r;
    const bool row_ok = gj < d.N;
    const bool lead_row = gj < d.lead;
    const unsigned emax = row_ok ? (unsigned)(lead_row ? d.Ae2 : d.Be)[gj] : 0u;
    const double* rowp = static_cast<const double*>(lead_row ? d.At2 : d.Bt) + (row_ok ? (size_t)gj * d.a_rs : 0);
    const bool vec = ((reinterpret_cast<uintptr_t>(rowp) | (uintptr_t)d.a_rs * 8) & 15) == 0;
    const int quarter = warp & 3, col0 = (ew >> 2) * C::DCOLS;  // drain: TMEM lane quarter, DCOLS columns
    const int drow = quarter * 32 + lane;                       // row of A (and of C)
    auto load = [&](int kc, double (&x)[8]) {
      const int k0 = kc * OZ_KC + kg * 8;
      if (row_ok && vec && k0 + 8 <= d.K) {
        const double2* p2 = reinterpret_cast<const double2*>(rowp + k0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const double2 v = p2[j];
          x[2 * j] = v.x;
          x[2 * j + 1] = v.y;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = (row_ok && k0 + j < d.K) ? rowp[k0 + j] : 0.0;
      }
    };
    // the exact sum of element j is H[j] 2^24 + Lw[j]; after every chunk the part of Lw at
    // and above 2^24 moves into H, so Lw stays in [0, 2^24) and fits 32 bits
    long long H[C::DCOLS];
    int Lw[C::DCOLS];
#pragma unroll
    for (int j = 0; j < C::DCOLS; ++j) { H[j] = 0; Lw[j] = 0; }
    bool alive = true;
    auto drain = [&](int c) {
      const int buf = C::NBUF == 2 ? (c & 1) : 0, tuse = C::NBUF == 2 ? (c >> 1) : c;
      if (!mbar_wait_warp(TFULL + 8 * buf, tuse & 1)) { alive = false; *abort_flag = 1; return; }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t lb = tmem + ((uint32_t)(quarter * 32) << 16) + buf * (OZ_G * NBC) + col0;
      // columns in groups of CW = 4 (the TMEM copies of one group take 28 registers)
      constexpr int CW = 4;
#pragma unroll
      for (int cb = 0; cb < C::DCOLS / CW; ++cb) {
        uint32_t v[OZ_G][CW];
#pragma unroll
        for (int g = 0; g < OZ_G; ++g) {
          if (g + 2 <= gmax) {
            tmem_ld4(lb + g * NBC + cb * CW, v[g]);
          } else {
            for (int j = 0; j < CW; ++j) v[g][j] = 0u;
          }
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (cb == C::DCOLS / CW - 1) {
          asm volatile("tcgen05.fence::before_thread_sync;");
          mbar_arrive(TEMPTY + 8 * buf);
        }
#pragma unroll
        for (int j = 0; j < CW; ++j) {
          int a[OZ_G];
#pragma unroll
          for (int g = 0; g < OZ_G; ++g) a[g] = __float2int_rn(__uint_as_float(v[g][j]));
          const long long l = (long long)Lw[cb * CW + j] + ((long long)a[3] << 24) + ((long long)a[4] << 16) +
                              ((long long)a[5] << 8) + a[6];
          const long long carry = l >> 24;  // floor
          H[cb * CW + j] += ((long long)a[0] << 24) + ((long long)a[1] << 16) + ((long long)a[2] << 8) + carry;
          Lw[cb * CW + j] = (int)(l - (carry << 24));
        }
      }
    };
    double xn[8];
    if (grp < nkc) load(grp, xn);
    for (int kc = 0; kc < nkc && alive; ++kc) {
      if (kc % C::NGRP == grp) {
        const int bb = kc % C::NBB;
        unsigned char* stB = smem + C::BOFF + bb * C::B;
        uint32_t w[OZ_S][4];
        split8(xn, emax, w);
        if (kc + C::NGRP < nkc) load(kc + C::NGRP, xn);  // this group's next step, in flight meanwhile
        // the buffer's previous contents (step kc - NBB) have been consumed by the MMAs
        if (!mbar_wait_warp(BEMPTY + 8 * bb, ((kc / C::NBB) & 1) ^ 1)) { alive = false; *abort_flag = 1; break; }
        const int off = tile_off32(r, kg * 8);
#pragma unroll
        for (int p = 0; p < OZ_S; ++p)
          *reinterpret_cast<uint4*>(stB + 2 * ((size_t)p * NBC * OZ_KC + off)) =
              make_uint4(w[p][0], w[p][1], w[p][2], w[p][3]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(BFULL + 8 * bb);
      }
      if ((kc & 3) == 3 || kc == nkc - 1) {
        // two accumulator sets: drain the previous chunk while this one's MMAs run; one set:
        // drain this chunk now, the next chunk's MMAs wait for its TMEM to be read
        if (C::NBUF == 2) {
          if ((kc >> 2) >= 1) drain((kc >> 2) - 1);
        } else {
          drain(kc >> 2);
        }
      }
    }
    if (C::NBUF == 2 && alive && nch >= 1) drain(nch - 1);
    if (alive && drow < d.M) {
      const int ed = d.Ae[drow];
      // tile0 flags: bit 0 negates the product, bit 1 adds the identity (C row drow +
      // lower_off is the diagonal's row)
      const bool neg = (d.tile0 & 1) != 0, ident = (d.tile0 & 2) != 0;
#pragma unroll
      for (int j = 0; j < C::DCOLS; ++j) {
        const int gc = bj * NBC + col0 + j;
        if (gc < d.N) {
          const int fj = (gc < d.lead ? d.Ae2 : d.Be)[gc];
          double v = 0.0;
          if (ed != 0 && fj != 0) {
            const int k = ed + fj - 2044 - 62;
            v = i64_to_double_pow2(H[j], k + 24, neg) + i64_to_double_pow2((long long)Lw[j], k, neg);
          }
          if (ident && drow + d.lower_off == gc) v += 1.0;
          d.C[(size_t)drow * d.c_rs + (size_t)gc * d.c_cs] = v;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0 && *abort_flag) atomicOr(status, ST_TIMEOUT);
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// ---------------------------------------------------------------------------------------
// Persistent update kernel for short products (K <= 128: the rank-32 QR update and the
// Cholesky SYRK).  One CTA per SM walks the 128 x 32 tiles of the whole batch; two
// shared-memory stages and two TMEM accumulator sets (7 x 32 columns each) let the loads
// and MMAs of the next tile run while eight epilogue warps finish the current one.
// Warp roles: 0 producer, 1 MMA (and TMEM owner), 2..17 epilogue (warp w drains TMEM lane
// quarter w % 4, columns 8 * ((w - 2) / 4) .. +7); four epilogue warps per SM sub-partition
// hide the latency of the per-element integer work and of the C traffic.
constexpr int UPD_NT = 32;
constexpr int UPD_EPI_WARPS = 16;
constexpr int UPD_COLS = UPD_NT / (UPD_EPI_WARPS / 4);   // columns per epilogue thread
constexpr int UPD_THREADS = 32 * (2 + UPD_EPI_WARPS);
constexpr int UPD_A = OZ_S * OZ_M * OZ_KC * 2;       // 57344 B
constexpr int UPD_B = OZ_S * UPD_NT * OZ_KC * 2;     // 14336 B
constexpr int UPD_STAGE = UPD_A + UPD_B;
constexpr int UPD_BAR = 2 * UPD_STAGE;               // full0 full1 empty0 empty1 tfull0 tfull1 tempty0 tempty1
constexpr int UPD_SLOT = UPD_BAR + 64;
constexpr int UPD_FLAG = UPD_SLOT + 16;
// C staging: per epilogue thread two tiles' worth (UPD_COLS values each), slot-major so
// every thread's cp.async writes and reads hit consecutive 8-byte words
constexpr int UPD_CBUF = UPD_FLAG + 16;
constexpr int UPD_SMEM = UPD_CBUF + 2 * UPD_COLS * 32 * UPD_EPI_WARPS * 8 + 1024;
static_assert(UPD_SMEM <= 227 * 1024, "persistent product exceeds the shared memory of one CTA");

// Epilogue modes, fixed at compile time so no FP64 compare or select runs per element:
// EMODE 0: C = s * AB (beta = 0);  1: C = C + s * AB (beta = 1);  2: C = beta C + alpha AB.
// s = +-1 is applied through the sign bit.  IDENT adds the identity (D = I - Q_G Q_G^T).
template <int EMODE, bool IDENT>
__global__ void __launch_bounds__(UPD_THREADS, 1) k_ozaki_upd(const OzDesc* __restrict__ descs,
                                                             const int4* __restrict__ tiles,
                                                             int total_tiles, double alpha,
                                                             double beta, unsigned* status, int gmax) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar = sbase + UPD_BAR;
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + UPD_SLOT);
  volatile int* abort_flag = reinterpret_cast<int*>(smem + UPD_FLAG);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t FULL = bar, EMPTY = bar + 16, TFULL = bar + 32, TEMPTY = bar + 48;

  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(FULL + 8 * i, 1);
      mbar_init(EMPTY + 8 * i, 1);
      mbar_init(TFULL + 8 * i, 1);
      mbar_init(TEMPTY + 8 * i, 32 * UPD_EPI_WARPS);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *slot;

  if (warp == 0) {
    if (lane == 0) {
      int sc = 0;  // stage counter
      for (int t = blockIdx.x; t < total_tiles && !*abort_flag; t += gridDim.x) {
        const int4 r = tiles[t];  // (entry, row tile, column tile)
        const OzDesc& d = descs[r.x];
        const int nkc = (d.K + OZ_KC - 1) / OZ_KC;
        for (int kc = 0; kc < nkc; ++kc, ++sc) {
          const int s = sc & 1, use = sc >> 1;
          if (!mbar_wait(EMPTY + 8 * s, (use & 1) ^ 1)) { *abort_flag = 1; break; }
          mbar_expect_tx(FULL + 8 * s, UPD_STAGE);
          const __nv_bfloat16* srcA =
              static_cast<const __nv_bfloat16*>(d.At) + (size_t)(r.y * nkc + kc) * OZ_S * OZ_M * OZ_KC;
          const __nv_bfloat16* srcB =
              static_cast<const __nv_bfloat16*>(d.Bt) + (size_t)(r.z * nkc + kc) * OZ_S * UPD_NT * OZ_KC;
          const uint32_t dst = sbase + s * UPD_STAGE;
          bulk_g2s(dst, srcA, UPD_A, FULL + 8 * s);
          bulk_g2s(dst + UPD_A, srcB, UPD_B, FULL + 8 * s);
        }
      }
      // drain: wait for the copies of the last two stages
      for (int q = (sc > 2 ? sc - 2 : 0); q < sc; ++q) mbar_wait(FULL + 8 * (q & 1), (q >> 1) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(OZ_M, UPD_NT);
      int sc = 0, tc = 0;  // stage and tile counters
      for (int t = blockIdx.x; t < total_tiles && !*abort_flag; t += gridDim.x) {
        const OzDesc& d = descs[tiles[t].x];
        const int nkc = (d.K + OZ_KC - 1) / OZ_KC;
        const int buf = tc & 1;
        if (!mbar_wait(TEMPTY + 8 * buf, ((tc >> 1) & 1) ^ 1)) { *abort_flag = 1; break; }
        const uint32_t dbase = tmem + buf * (OZ_G * UPD_NT);
        bool fail = false;
        for (int kc = 0; kc < nkc; ++kc, ++sc) {
          const int s = sc & 1, use = sc >> 1;
          if (!mbar_wait(FULL + 8 * s, use & 1)) { fail = true; break; }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t a0 = sbase + s * UPD_STAGE, b0 = a0 + UPD_A;
#pragma unroll
          for (int k = 0; k < 2; ++k) {
#pragma unroll
            for (int g = 2; g <= OZ_S + 1; ++g) {
            if (g > gmax) continue;  // digit groups beyond gmax are not formed
#pragma unroll
              for (int p = 1; p <= OZ_S; ++p) {
                const int q = g - p;
                if (q < 1 || q > OZ_S) continue;
                const uint32_t first = (kc == 0 && k == 0 && p == 1);
                const uint64_t ad = sdesc(a0 + (p - 1) * (OZ_M * OZ_KC * 2) + k * 256, 128, 512);
                const uint64_t bd = sdesc(b0 + (q - 1) * (UPD_NT * OZ_KC * 2) + k * 256, 128, 512);
                mma_bf16(dbase + (g - 2) * UPD_NT, ad, bd, idesc, first ? 0u : 1u);
              }
            }
          }
          mma_commit(EMPTY + 8 * s);
        }
        if (fail) { *abort_flag = 1; break; }
        mma_commit(TFULL + 8 * buf);
        ++tc;
      }
    }
  } else {
    const int ew = warp - 2, quarter = warp & 3, part = ew >> 2;
    const int row = quarter * 32 + lane;
    const int col0 = part * UPD_COLS;
    const int wt = ew * 32 + lane;  // epilogue thread 0..511
    const bool neg_alpha = EMODE != 2 && (__double_as_longlong(alpha) < 0);
    double* cbuf = reinterpret_cast<double*>(smem + UPD_CBUF);
    constexpr int ET = 32 * UPD_EPI_WARPS;
    // Everything a tile's epilogue reads from memory is requested one tile ahead: the
    // row / column exponents into registers, the C values by cp.async into shared memory
    // (one commit group per tile), and the tile-table entry two tiles ahead.  The MMAs run
    // ahead of the epilogue, so without this the C latency would be exposed on every tile.
    auto stage = [&](const int4& r, int buf, int& ei, int (&fj)[UPD_COLS]) {
      const OzDesc& d = descs[r.x];
      const int gi = r.y * OZ_M + row, gj0 = r.z * UPD_NT + col0;
      ei = gi < d.M ? d.Ae[gi] : 0;
#pragma unroll
      for (int j = 0; j < UPD_COLS; ++j) fj[j] = gj0 + j < d.N ? d.Be[gj0 + j] : 0;
      if (EMODE != 0 && gi < d.M) {
        const double* cp = d.C + (size_t)gi * d.c_rs + (size_t)gj0 * d.c_cs;
#pragma unroll
        for (int j = 0; j < UPD_COLS; ++j)
          if (gj0 + j < d.N) cp_async8(smem_u32(cbuf + (buf * UPD_COLS + j) * ET + wt), cp + (size_t)j * d.c_cs);
      }
      cp_async_commit();
    };
    int tc = 0;
    int t = blockIdx.x;
    int4 r = t < total_tiles ? tiles[t] : make_int4(0, 0, 0, 0);
    int4 rn = t + (int)gridDim.x < total_tiles ? tiles[t + gridDim.x] : make_int4(0, 0, 0, 0);
    int ei = 0, ein = 0, fj[UPD_COLS], fjn[UPD_COLS];
#pragma unroll
    for (int j = 0; j < UPD_COLS; ++j) { fj[j] = 0; fjn[j] = 0; }
    if (t < total_tiles) stage(r, 0, ei, fj);
    while (t < total_tiles) {
      const OzDesc& d = descs[r.x];
      const int tn = t + gridDim.x, tnn = tn + gridDim.x;
      const int4 rnn = tnn < total_tiles ? tiles[tnn] : make_int4(0, 0, 0, 0);
      if (tn < total_tiles) stage(rn, (tc + 1) & 1, ein, fjn);
      const int buf = tc & 1;
      if (!mbar_wait_warp(TFULL + 8 * buf, (tc >> 1) & 1)) { *abort_flag = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t lb = tmem + ((uint32_t)(quarter * 32) << 16) + buf * (OZ_G * UPD_NT) + col0;
      if (tn < total_tiles) cp_async_wait<1>();  // this tile's C group is complete
      else cp_async_wait<0>();
      const int gi = r.y * OZ_M + row, gj0 = r.z * UPD_NT + col0;
      double* cp = d.C + (size_t)gi * d.c_rs + (size_t)gj0 * d.c_cs;
      // two halves of 4 columns keep the TMEM copies at 28 registers
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        uint32_t v[OZ_G][4];
#pragma unroll
        for (int g = 0; g < OZ_G; ++g) {
          if (g + 2 <= gmax) tmem_ld4(lb + g * UPD_NT + half * 4, v[g]);
          else for (int j = 0; j < 4; ++j) v[g][j] = 0u;
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (half == 1) {
          asm volatile("tcgen05.fence::before_thread_sync;");
          mbar_arrive(TEMPTY + 8 * buf);  // accumulators copied: the MMA may reuse this buffer
        }
        if (gi < d.M) {
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int j = half * 4 + jj;
            if (gj0 + j < d.N) {
              int a[OZ_G];
#pragma unroll
              for (int g = 0; g < OZ_G; ++g) a[g] = __float2int_rn(__uint_as_float(v[g][jj]));
              const double pv =
                  (ei != 0 && fj[j] != 0) ? groups_to_double(a, ei + fj[j] - 2044 - 62, neg_alpha) : 0.0;
              const double cv = EMODE != 0 ? cbuf[(buf * UPD_COLS + j) * ET + wt] : 0.0;
              double out;
              if (EMODE == 0) out = pv;
              else if (EMODE == 1) out = cv + pv;
              else out = fma(beta, cv, alpha * pv);
              if (IDENT && gi == gj0 + j) out += 1.0;
              cp[(size_t)j * d.c_cs] = out;
            }
          }
        }
      }
      ++tc;
      t = tn;
      r = rn;
      rn = rnn;
      ei = ein;
#pragma unroll
      for (int j = 0; j < UPD_COLS; ++j) fj[j] = fjn[j];
    }
    cp_async_wait<0>();  // no copy may land after this thread has left
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0 && *abort_flag) atomicOr(status, ST_TIMEOUT);
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// ---------------------------------------------------------------------------------------
// Wide persistent update C += s A B^T (s = +-1, K <= 128) over 128 x 64 output tiles: the
// QR's outer-block trailing update.  An N = 64 MMA reads each A plane from shared memory
// once for 64 columns (the N = 32 kernel reads it twice), so the operand traffic per
// output halves.  The 7 group accumulators of a 128 x 64 tile take 448 of the 512 TMEM
// columns: one set, so the next tile's MMAs wait until the epilogue has read it (its C
// values are requested before that wait and arrive meanwhile).  The epilogue turns the
// accumulators into exact integers first and releases the TMEM before its FP64 work (the
// conversion and the add to C, one FP64-pipe operation each per element), which then
// overlaps the next tile's MMAs.  B is split with 64-row tiles (one bulk copy per stage).
// Warp roles as in k_ozaki_upd; 8 epilogue warps (10 warps per CTA leave registers for the
// 32 exact integers each epilogue thread holds), each thread 32 columns of one row.
constexpr int UPW_NT = 64;
constexpr int UPW_EPI_WARPS = 8;
constexpr int UPW_COLS = UPW_NT / (UPW_EPI_WARPS / 4);
constexpr int UPW_THREADS = 32 * (2 + UPW_EPI_WARPS);
constexpr int UPW_A = OZ_S * OZ_M * OZ_KC * 2;       // 57344 B
constexpr int UPW_B = OZ_S * UPW_NT * OZ_KC * 2;     // 28672 B
constexpr int UPW_STAGE = UPW_A + UPW_B;
constexpr int UPW_BAR = 2 * UPW_STAGE;               // FULL[2] EMPTY[2] TFULL TEMPTY
constexpr int UPW_SLOT = UPW_BAR + 64;
constexpr int UPW_FLAG = UPW_SLOT + 16;
constexpr int UPW_SMEM = UPW_FLAG + 16 + 1024;
static_assert(UPW_SMEM <= 227 * 1024, "wide persistent product exceeds the shared memory of one CTA");

template <bool NEG>
__global__ void __launch_bounds__(UPW_THREADS, 1) k_ozaki_updw(const OzDesc* __restrict__ descs,
                                                              const int4* __restrict__ tiles, int total_tiles,
                                                              unsigned* status, int gmax) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar = sbase + UPW_BAR;
  uint32_t* slot = reinterpret_cast<uint32_t*>(smem + UPW_SLOT);
  volatile int* abort_flag = reinterpret_cast<int*>(smem + UPW_FLAG);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t FULL = bar, EMPTY = bar + 16, TFULL = bar + 32, TEMPTY = bar + 40;

  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(FULL + 8 * i, 1);
      mbar_init(EMPTY + 8 * i, 1);
    }
    mbar_init(TFULL, 1);
    mbar_init(TEMPTY, 32 * UPW_EPI_WARPS);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *slot;

  if (warp == 0) {
    if (lane == 0) {
      int sc = 0;  // stage counter
      for (int t = blockIdx.x; t < total_tiles && !*abort_flag; t += gridDim.x) {
        const int4 r = tiles[t];  // (entry, row tile, column tile)
        const OzDesc& d = descs[r.x];
        const int nkc = (d.K + OZ_KC - 1) / OZ_KC;
        for (int kc = 0; kc < nkc; ++kc, ++sc) {
          const int s = sc & 1, use = sc >> 1;
          if (!mbar_wait(EMPTY + 8 * s, (use & 1) ^ 1)) { *abort_flag = 1; break; }
          mbar_expect_tx(FULL + 8 * s, UPW_STAGE);
          const __nv_bfloat16* srcA =
              static_cast<const __nv_bfloat16*>(d.At) + (size_t)(r.y * nkc + kc) * OZ_S * OZ_M * OZ_KC;
          const __nv_bfloat16* srcB =
              static_cast<const __nv_bfloat16*>(d.Bt) + (size_t)(r.z * nkc + kc) * OZ_S * UPW_NT * OZ_KC;
          const uint32_t dst = sbase + s * UPW_STAGE;
          bulk_g2s(dst, srcA, UPW_A, FULL + 8 * s);
          bulk_g2s(dst + UPW_A, srcB, UPW_B, FULL + 8 * s);
        }
      }
      for (int q = (sc > 2 ? sc - 2 : 0); q < sc; ++q) mbar_wait(FULL + 8 * (q & 1), (q >> 1) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(OZ_M, UPW_NT);
      int sc = 0, tc = 0;
      for (int t = blockIdx.x; t < total_tiles && !*abort_flag; t += gridDim.x) {
        const OzDesc& d = descs[tiles[t].x];
        const int nkc = (d.K + OZ_KC - 1) / OZ_KC;
        // the accumulators of the previous tile have been read by the epilogue
        if (!mbar_wait(TEMPTY, (tc & 1) ^ 1)) { *abort_flag = 1; break; }
        bool fail = false;
        for (int kc = 0; kc < nkc; ++kc, ++sc) {
          const int s = sc & 1, use = sc >> 1;
          if (!mbar_wait(FULL + 8 * s, use & 1)) { fail = true; break; }
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t a0 = sbase + s * UPW_STAGE, b0 = a0 + UPW_A;
#pragma unroll
          for (int k = 0; k < 2; ++k) {
#pragma unroll
            for (int g = 2; g <= OZ_S + 1; ++g) {
              if (g > gmax) continue;  // digit groups beyond gmax are not formed
#pragma unroll
              for (int p = 1; p <= OZ_S; ++p) {
                const int q = g - p;
                if (q < 1 || q > OZ_S) continue;
                const uint32_t first = (kc == 0 && k == 0 && p == 1);
                const uint64_t ad = sdesc(a0 + (p - 1) * (OZ_M * OZ_KC * 2) + k * 256, 128, 512);
                const uint64_t bd = sdesc(b0 + (q - 1) * (UPW_NT * OZ_KC * 2) + k * 256, 128, 512);
                mma_bf16(tmem + (g - 2) * UPW_NT, ad, bd, idesc, first ? 0u : 1u);
              }
            }
          }
          mma_commit(EMPTY + 8 * s);
        }
        if (fail) { *abort_flag = 1; break; }
        mma_commit(TFULL);
        ++tc;
      }
    }
  } else {
    const int ew = warp - 2, quarter = warp & 3, part = ew >> 2;
    const int row = quarter * 32 + lane;
    const int col0 = part * UPW_COLS;
    int tc = 0;
    for (int t = blockIdx.x; t < total_tiles; t += gridDim.x, ++tc) {
      const int4 r = tiles[t];
      const OzDesc& d = descs[r.x];
      const int gi = r.y * OZ_M + row, gj0 = r.z * UPW_NT + col0;
      const bool rok = gi < d.M;
      const int ei = rok ? d.Ae[gi] : 0;
      double* cp = d.C + (size_t)(rok ? gi : 0) * d.c_rs + (size_t)gj0 * d.c_cs;
      // C in rounds of 4 columns, each round's values requested one round ahead (the first
      // before the accumulators are waited for)
      auto load_c = [&](int cb, double (&x)[4]) {
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          const int j = cb * 4 + jj;
          x[jj] = (rok && gj0 + j < d.N) ? cp[(size_t)j * d.c_cs] : 0.0;
        }
      };
      double cvn[4];
      load_c(0, cvn);
      if (!mbar_wait_warp(TFULL, tc & 1)) { *abort_flag = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t lb = tmem + ((uint32_t)(quarter * 32) << 16) + col0;
      // 1) the accumulators to exact integers (integer work only), then the TMEM is released
      //    for the next tile's MMAs; 2) the FP64 conversions and C updates meanwhile
      long long X[UPW_COLS];
      unsigned long long tcode = 0;  // the shift t of element j in bits 2j, 2j+1 (0, 7, 13 -> 0, 1, 2)
#pragma unroll
      for (int cb = 0; cb < UPW_COLS / 4; ++cb) {
        uint32_t v[OZ_G][4];
#pragma unroll
        for (int g = 0; g < OZ_G; ++g) {
          if (g + 2 <= gmax) tmem_ld4(lb + g * UPW_NT + cb * 4, v[g]);
          else for (int j = 0; j < 4; ++j) v[g][j] = 0u;
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          int a[OZ_G];
#pragma unroll
          for (int g = 0; g < OZ_G; ++g) a[g] = __float2int_rn(__uint_as_float(v[g][jj]));
          int sh;
          X[cb * 4 + jj] = groups_to_x(a, sh);
          tcode |= (unsigned long long)(sh == 0 ? 0 : (sh == 7 ? 1 : 2)) << (2 * (cb * 4 + jj));
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      mbar_arrive(TEMPTY);  // accumulators copied: the MMAs of the next tile may start
#pragma unroll
      for (int cb = 0; cb < UPW_COLS / 4; ++cb) {
        double cv[4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) cv[jj] = cvn[jj];
        if (cb + 1 < UPW_COLS / 4) load_c(cb + 1, cvn);
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) {
          const int j = cb * 4 + jj;
          if (rok && gj0 + j < d.N) {
            const int fj = d.Be[gj0 + j];
            const int code = (int)(tcode >> (2 * j)) & 3, sh = code == 0 ? 0 : (code == 1 ? 7 : 13);
            const double pv = (ei != 0 && fj != 0) ? x_to_double(X[j], ei + fj - 2044 - 62 + sh, NEG) : 0.0;
            cp[(size_t)j * d.c_cs] = cv[jj] + pv;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid == 0 && *abort_flag) atomicOr(status, ST_TIMEOUT);
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

template <int NT>
cudaError_t launch_oz(const OzDesc* d, int count, int max_tiles, double alpha, double beta,
                      int flags, unsigned* status, cudaStream_t st, int gmax) {
  static bool attr = false;
  const int smem = OzSmem<NT>::TOTAL;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_ozaki<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  for (int off = 0; off < count; off += 65535) {
    const int c = count - off < 65535 ? count - off : 65535;
    k_ozaki<NT><<<dim3(max_tiles, c), OZ_THREADS, smem, st>>>(d + off, alpha, beta, flags, status, gmax);
    count_launch();
  }
  return cudaGetLastError();
}

}  // namespace

int oz_tiles(int m, int n, int nt) { return ((m + OZ_M - 1) / OZ_M) * ((n + nt - 1) / nt); }

size_t oz_split_elems(int R, int K, int row_tile) {
  return (size_t)((R + row_tile - 1) / row_tile) * ((K + OZ_KC - 1) / OZ_KC) * OZ_S * row_tile * OZ_KC;
}

int oz_rowexp_blocks(const SplitDesc& d) {
  if (d.R <= 0) return 0;
  return rowexp_by_thread(d.rs, d.ks, d.K) ? (d.R + 255) / 256 : (d.R + 7) / 8;
}

cudaError_t launch_split(const SplitDesc* d, int count, int rowexp_blocks, int max_split_blocks,
                         cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  for (int off = 0; off < count; off += 65535) {
    const int c = count - off < 65535 ? count - off : 65535;
    if (rowexp_blocks > 0) { k_rowexp<<<dim3(rowexp_blocks, c), 256, 0, st>>>(d + off); count_launch(); }
    k_split<<<dim3(max_split_blocks, c), 256, 0, st>>>(d + off); count_launch();
  }
  return cudaGetLastError();
}

int oz_upd_tile_table(const OzDesc* descs, int count, int flags, int4* out, int nt) {
  int n = 0;
  for (int e = 0; e < count; ++e) {
    const OzDesc& d = descs[e];
    const int tm = (d.M + OZ_M - 1) / OZ_M, tn = (d.N + nt - 1) / nt;
    for (int bj = 0; bj < tn; ++bj)
      for (int bi = 0; bi < tm; ++bi) {
        if ((flags & GEMM_LOWER) && bj * nt + d.lower_off > bi * OZ_M + OZ_M - 1) continue;  // above the diagonal
        if (out) out[n] = make_int4(e, bi, bj, 0);
        ++n;
      }
  }
  return n;
}

cudaError_t launch_ozaki_upd(const OzDesc* d, int count, const int4* tiles, int total_tiles,
                             double alpha, double beta, int flags, unsigned* status, cudaStream_t st,
                             int max_grid, int gmax) {
  if (count <= 0 || total_tiles <= 0) return cudaSuccess;
  if (gmax < 2 || gmax > OZ_S + 1) return cudaErrorInvalidValue;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaSuccess;
    auto set = [&](const void* f) {
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, UPD_SMEM);
    };
    set((const void*)k_ozaki_upd<0, false>); set((const void*)k_ozaki_upd<0, true>);
    set((const void*)k_ozaki_upd<1, false>); set((const void*)k_ozaki_upd<1, true>);
    set((const void*)k_ozaki_upd<2, false>); set((const void*)k_ozaki_upd<2, true>);
    if (e != cudaSuccess) return e;
  }
  int grid = total_tiles < sms ? total_tiles : sms;
  if (max_grid > 0 && grid > max_grid) grid = max_grid;  // SMs left to a concurrent stream
  const bool unit = alpha == 1.0 || alpha == -1.0;
  const int mode = (beta == 0.0 && unit) ? 0 : (beta == 1.0 && unit) ? 1 : 2;
  const bool ident = (flags & GEMM_ADD_IDENTITY) != 0;
#define ELM_UPD(M, I) \
  k_ozaki_upd<M, I><<<grid, UPD_THREADS, UPD_SMEM, st>>>(d, tiles, total_tiles, alpha, beta, status, gmax)
  if (mode == 0) { if (ident) ELM_UPD(0, true); else ELM_UPD(0, false); }
  else if (mode == 1) { if (ident) ELM_UPD(1, true); else ELM_UPD(1, false); }
  else { if (ident) ELM_UPD(2, true); else ELM_UPD(2, false); }
#undef ELM_UPD
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_ozaki_updw(const OzDesc* d, int count, const int4* tiles, int total_tiles, double alpha,
                              unsigned* status, cudaStream_t st, int max_grid, int gmax) {
  if (count <= 0 || total_tiles <= 0) return cudaSuccess;
  if (gmax < 2 || gmax > OZ_S + 1 || (alpha != 1.0 && alpha != -1.0)) return cudaErrorInvalidValue;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaFuncSetAttribute(k_ozaki_updw<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, UPW_SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_ozaki_updw<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, UPW_SMEM);
    if (e != cudaSuccess) return e;
  }
  int grid = total_tiles < sms ? total_tiles : sms;
  if (max_grid > 0 && grid > max_grid) grid = max_grid;
  if (alpha < 0.0)
    k_ozaki_updw<true><<<grid, UPW_THREADS, UPW_SMEM, st>>>(d, tiles, total_tiles, status, gmax);
  else
    k_ozaki_updw<false><<<grid, UPW_THREADS, UPW_SMEM, st>>>(d, tiles, total_tiles, status, gmax);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_ozaki_fa(const OzDesc* d, int count, int max_tiles, unsigned* status,
                            cudaStream_t st, int gmax, int ksplit) {
  if (count <= 0 || max_tiles <= 0) return cudaSuccess;
  if (gmax < 2 || gmax > OZ_S + 1 || ksplit < 1 || (ksplit > 1 && max_tiles > 1)) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_ozaki_fa, cudaFuncAttributeMaxDynamicSharedMemorySize, FA_SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  for (int off = 0; off < count; off += 65535) {
    const int c = count - off < 65535 ? count - off : 65535;
    k_ozaki_fa<<<dim3(max_tiles, c, ksplit), FA_THREADS, FA_SMEM, st>>>(d + off, status, gmax); count_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_ozaki_fb(const OzDesc* d, int count, int max_tiles, unsigned* status,
                            cudaStream_t st, int gmax, int nbc) {
  if (count <= 0 || max_tiles <= 0) return cudaSuccess;
  if (gmax < 2 || gmax > OZ_S + 1 || (nbc != 32 && nbc != 64)) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_ozaki_fb<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         FbCfg<32>::SMEM);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_ozaki_fb<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, FbCfg<64>::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  for (int off = 0; off < count; off += 65535) {
    const int c = count - off < 65535 ? count - off : 65535;
    if (nbc == 64)
      k_ozaki_fb<64><<<dim3(max_tiles, c), FbCfg<64>::THREADS, FbCfg<64>::SMEM, st>>>(d + off, status, gmax);
    else
      k_ozaki_fb<32><<<dim3(max_tiles, c), FbCfg<32>::THREADS, FbCfg<32>::SMEM, st>>>(d + off, status, gmax);
    count_launch();
  }
  return cudaGetLastError();
}

size_t tf32x3_work_floats(int M, int N, int K) {
  const size_t kp = (size_t)((K + TF_KC - 1) / TF_KC) * TF_KC;
  return 2 * kp * ((size_t)((M + TF_M - 1) / TF_M) * TF_M + (size_t)((N + TF_N - 1) / TF_N) * TF_N);
}

cudaError_t launch_tf32x3_gemm(int M, int N, int K, const float* A, long long a_rs, long long a_ks,
                               const float* B, long long b_ns, long long b_ks, float* C, int ldc, int epi,
                               const float* bias, float* Z, int ldz, float* work, size_t work_floats,
                               unsigned* status, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (K <= 0 || epi < 0 || epi > 3 || work_floats < tf32x3_work_floats(M, N, K)) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(work) & 15) != 0) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaSuccess;
    e = cudaFuncSetAttribute(k_tf32x3<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, TF_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tf32x3<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, TF_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tf32x3<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, TF_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tf32x3<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, TF_SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int nkc = (K + TF_KC - 1) / TF_KC, tm = (M + TF_M - 1) / TF_M, tn = (N + TF_N - 1) / TF_N;
  float* At = work;
  float* Bt = work + (size_t)2 * tm * TF_M * nkc * TF_KC;
  const TfSplit sa{A, a_rs, a_ks, M, K, TF_M, At}, sb{B, b_ns, b_ks, N, K, TF_N, Bt};
  k_tf32_split<<<dim3(std::max(tm, tn) * nkc, 2), 256, 0, st>>>(sa, sb); count_launch();
  const TfGemm g{At, Bt, C, ldc, M, N, K, bias, Z, ldz};
  const dim3 grid(tm * tn);
  if (epi == 0) k_tf32x3<0><<<grid, 192, TF_SMEM, st>>>(g, status);
  else if (epi == 1) k_tf32x3<1><<<grid, 192, TF_SMEM, st>>>(g, status);
  else if (epi == 2) k_tf32x3<2><<<grid, 192, TF_SMEM, st>>>(g, status);
  else k_tf32x3<3><<<grid, 192, TF_SMEM, st>>>(g, status);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_ozaki(int nt, const OzDesc* d, int count, int max_tiles, double alpha,
                         double beta, int flags, unsigned* status, cudaStream_t st, int gmax) {
  if (count <= 0 || max_tiles <= 0) return cudaSuccess;
  if (gmax < 2 || gmax > OZ_S + 1) return cudaErrorInvalidValue;
  if (nt == 32) return launch_oz<32>(d, count, max_tiles, alpha, beta, flags, status, st, gmax);
  return launch_oz<64>(d, count, max_tiles, alpha, beta, flags, status, st, gmax);
}

}  // namespace elmddm
