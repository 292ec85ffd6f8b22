// Internal declarations shared by the CUDA translation units of libelmddm.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

namespace elmddm {

// Kernels launched by the library in this process (every launcher counts its own).
extern std::atomic<long long> g_kernel_launches;
inline void count_launch(int k = 1) { g_kernel_launches.fetch_add(k, std::memory_order_relaxed); }

constexpr int QR_NB = 32;     // panel width of the blocked Householder QR
constexpr int CHOL_NB = 64;   // block size of the Schur-matrix Cholesky
constexpr int GRP_MAX = 4;    // most subdomains one interface unknown is shared by (a cross point)
// int64 words of one split-K accumulator tile: 128 x 32 elements x 2 words, then the count
// of the tile's CTAs that have added their part (the last one converts and clears)
constexpr int OZ_HL_WORDS = 128 * 32 * 2;
constexpr int OZ_HL_TILE = OZ_HL_WORDS + 2;
constexpr int TRSV_MAX_N = 8192;  // largest n_neurons the back-solve keeps in shared memory

// Bits of the device status word.
// ST_TIMEOUT: a bounded wait inside a kernel gave up (ELM_DDM_ERR_TIMEOUT); ST_INTERNAL: a
// launch violated a kernel's documented limits (ELM_DDM_ERR_CUDA).
enum : unsigned { ST_RANK = 1u, ST_NOT_SPD = 2u, ST_NONFINITE = 4u, ST_TIMEOUT = 8u, ST_INTERNAL = 16u };

// C(m x n) = alpha * op(A) op(B) + beta * C, column-major; op = transpose or not.
struct GemmDesc {
  const double* A;
  const double* B;
  double* C;
  int m, n, k, lda, ldb, ldc;
};
// GEMM_SKINNY selects the 32 x 128 tile (every m <= 32); tile counts then use that shape.
enum : int { GEMM_LOWER = 1, GEMM_ADD_IDENTITY = 2, GEMM_SKINNY = 4 };
inline int gemm_tiles(int m, int n, int flags) {
  return (flags & GEMM_SKINNY) ? ((m + 31) / 32) * ((n + 127) / 128)
                               : ((m + 63) / 64) * ((n + 63) / 64);
}

// dst(rows x cols) += src, column-major.
struct AddDesc {
  const double* src;
  double* dst;
  int rows, cols, lds, ldd;
};

// Digit split of one FP64 operand (k_ozaki.cu): the logical R x K matrix with element
// (r, k) at X[r * rs + k * ks] becomes 7 BF16 digit planes in row tiles of row_tile rows
// (128 for the A side, the GEMM's NT for the B side); E receives per-row exponent bounds.
// tiles == nullptr: row exponents only (the operand is split inside the product kernel).
struct SplitDesc {
  const double* X;
  long long rs, ks;
  int R, K;
  int* E;
  void* tiles;
  int row_tile;
};
// C[i * c_rs + j * c_cs] = alpha * sum_k A[i, k] B[j, k] + beta * C (A, B split as above).
struct OzDesc {
  const void* At;
  const int* Ae;
  const void* Bt;
  const int* Be;
  double* C;
  long long c_rs, c_cs;
  int M, N, K;
  int tile0;  // B-split product (k_ozaki_fb): bit 0 negates, bit 1 adds the identity; else zero
  long long a_rs;  // fused-split launches: At is the FP64 A, element (i, k) at At[i * a_rs + k]
  // persistent product with GEMM_LOWER: column j of this C is column j + lower_off of the
  // symmetric matrix, so a tile is kept when its first column is on or below the diagonal;
  // B-split product with the identity flag: row i of this C is row i + lower_off
  int lower_off = 0;
  // fused-split launches: rows i < lead of A are read from At2 (same row stride a_rs) and
  // take their exponent bounds from Ae2, instead of At and Ae, so one product can stack
  // two FP64 operands with equal leading dimension (for the B-split launch these three
  // describe the leading rows of B)
  const void* At2 = nullptr;
  const int* Ae2 = nullptr;
  int lead = 0;
  // split-K A-split launches (one 128-row tile): [128][32][2] int64 accumulator of the
  // exact digit sums, zero before the launch (the conversion clears it again)
  long long* hl = nullptr;
};

// Per right-hand side state of the CG solve of the Schur system (k_cg.cu).
struct CgState {
  double rr, rz, bb;  // r^T r of the current residual, r^T M^{-1} r, b^T b
  int iters;          // CG steps taken
  int done;           // 0 running, 1 converged, 2 breakdown (p^T S p <= 0 or not finite)
};

// ---- launchers (return cudaGetLastError after the launch) ----
int oz_tiles(int m, int n, int nt);
size_t oz_split_elems(int R, int K, int row_tile);
// blocks of k_rowexp that descriptor d needs (a warp per row, or a thread per row for
// short rows of a column-major operand); a split launch takes the largest over its batch
int oz_rowexp_blocks(const SplitDesc& d);
cudaError_t launch_split(const SplitDesc* d, int count, int rowexp_blocks, int max_split_blocks,
                         cudaStream_t st);
// gmax (2..8): the digit pairs formed are those with p + q <= gmax; 8 (all 28 pairs of
// weight >= 2^-62) is the FP64-accurate product, smaller values a lower-precision one
// (5: the 10 leading pairs, an error below about 2^-28 of the row and column maxima).
cudaError_t launch_ozaki(int nt, const OzDesc* d, int count, int max_tiles, double alpha,
                         double beta, int flags, unsigned* status, cudaStream_t st, int gmax = 8);
// Persistent variant for K <= 64: one CTA per SM walks a tile table of (entry, row tile,
// column tile) over all 128 x 32 output tiles of the batch.  oz_upd_tile_table (host)
// writes that table (out may be null to count) and skips the tiles above the diagonal of
// a GEMM_LOWER product; it returns the number of tiles.
int oz_upd_tile_table(const OzDesc* descs, int count, int flags, int4* out, int nt = 32);
// C += alpha A B^T, alpha = +-1, K <= 128, over 128 x 64 output tiles (tile table with
// nt = UPW_TILE_N; B split with row_tile 64): the wide persistent update.
constexpr int UPW_TILE_N = 64;
cudaError_t launch_ozaki_updw(const OzDesc* d, int count, const int4* tiles, int total_tiles, double alpha,
                              unsigned* status, cudaStream_t st, int max_grid = 0, int gmax = 8);
// max_grid > 0 caps the persistent grid (SMs left to work on another stream).
cudaError_t launch_ozaki_upd(const OzDesc* d, int count, const int4* tiles, int total_tiles,
                             double alpha, double beta, int flags, unsigned* status,
                             cudaStream_t st, int max_grid = 0, int gmax = 8);
// C = A B^T with the FP64 A split inside the kernel (At = FP64 A, a_rs its row stride, K
// contiguous; Ae its row exponents), B split as usual with row_tile 32, N <= 32, beta = 0.
cudaError_t launch_ozaki_fa(const OzDesc* d, int count, int max_tiles, unsigned* status,
                            cudaStream_t st, int gmax = 8, int ksplit = 1);
// C = A B^T with A already split (M <= 128: one row tile) and the FP64 B operand split
// inside the kernel: B row j at Bt + j * a_rs with exponent bound Be[j], or, for j < lead,
// at At2 + j * a_rs with Ae2[j].  One CTA per nbc (32 or 64) rows of B (max_tiles = the
// most tiles).
// FP32 C (M x N, row-major, ldc) = op(A) op(B) on the tensor cores at FP32 accuracy (three
// TF32 products of a hi/lo split, k_ozaki.cu), with the warm-start network's epilogues:
// epi 0: C = AB; 1: Z = AB + bias, C = gelu(Z); 2: C = AB + bias; 3: C = AB * gelu'(Z).
// op(A): element (i, k) at A[i a_rs + k a_ks]; op(B): element (k, j) at B[j b_ns + k b_ks].
// work: 16-byte aligned device scratch of tf32x3_work_floats(M, N, K) floats (the split planes).
size_t tf32x3_work_floats(int M, int N, int K);
cudaError_t launch_tf32x3_gemm(int M, int N, int K, const float* A, long long a_rs, long long a_ks,
                               const float* B, long long b_ns, long long b_ks, float* C, int ldc, int epi,
                               const float* bias, float* Z, int ldz, float* work, size_t work_floats,
                               unsigned* status, cudaStream_t st);
cudaError_t launch_ozaki_fb(const OzDesc* d, int count, int max_tiles, unsigned* status,
                            cudaStream_t st, int gmax = 8, int nbc = 32);
cudaError_t launch_gemm(bool ta, bool tb, const GemmDesc* d, int count, int max_tiles,
                        double alpha, double beta, int flags, cudaStream_t st);
cudaError_t launch_add_blocks(const AddDesc* d, int count, int max_elems, cudaStream_t st);

// Per-subdomain coordinate tables of the factored activation (k_assemble.cu): distinct
// x (xs [N][nxmax]) and y (ys [N][nymax]) values, their counts (nxy [N][2]), a centre
// (ctr [N][2]), each row's coordinate indices (rix [N][m_max], ix | iy << 16), and the
// factor tables Tx [N][n][nxmax], Ty [N][n][nymax] filled by the assembly launch.
struct AsmTables {
  const double* xs = nullptr;
  const double* ys = nullptr;
  const int* nxy = nullptr;
  const double* ctr = nullptr;
  const int* rix = nullptr;
  double* Tx = nullptr;
  double* Ty = nullptr;
  int nxmax = 0, nymax = 0;
};
// coef: NULL for -Laplacian, else [N][m_max][3] (rho, grad rho) for -div(rho grad).
// tb: NULL (tanh per entry) or the coordinate tables (factored activation).
// nsub: NULL (n neurons everywhere) or [N] neurons per subdomain; columns n_s .. n-1 of
// K^s are then identity columns on the pad rows after the interface rows.
cudaError_t launch_assemble(double* K, long long kstride, int ld, int ncap, double* Amat,
                            long long astride, int mgld, const double* xy, const double* nrm,
                            int m_max, const int* cnt, const double* W, const double* b, int N,
                            int n, const double* coef, const AsmTables* tb, unsigned* status,
                            cudaStream_t st, const int* nsub = nullptr);
// Tikhonov rows (ELM_DDM_FLAG_RIDGE): K[ms + (n - n_s) + j][j] = alpha * max column norm, j < n_s
cudaError_t launch_ridge_rows(double* K, long long kstride, int ld, const int* cnt, const int* nsub, int N, int n,
                              double alpha, cudaStream_t st);
// theta of the pad neurons (j >= nsub[s]) set to zero, so that they evaluate to zero
cudaError_t launch_zero_pad_theta(double* W, double* b, const int* nsub, int N, int n, cudaStream_t st);
// Rows of one kind (0 interior, 1 boundary, 2 interface, 3 interface normals) of every
// subdomain into out [N][kmax][2] (zero past each subdomain's count).
cudaError_t launch_get_points(const double* xy, const double* nrm, int m_max, const int* cnt, int N,
                              int kind, int kmax, double* out, cudaStream_t st);
// Exponent bound of every column of the assembled [K^s | J] (colexp [N][ncap]): the
// biased exponent of 1.0001 |column|_2, so that 2^(E - 1022) exceeds every entry the
// column can hold under orthogonal updates of its rows (0 for a zero column).
cudaError_t launch_colexp(const double* K, long long kstride, int ld, int ncap, const int* ms, int N,
                          int* colexp, cudaStream_t st);
cudaError_t launch_eval(const double* W, const double* b, int N, int n, int npts,
                        const double* xy, const int* owner, const double* c, double* u,
                        double* grad, cudaStream_t st);

// Householder panel [k0, k0+nbe) of every subdomain: R and the reflectors in place, tau,
// the explicit reflectors in Vp (column j at Vp + s*vstride + j*ld, rows k0 .. m_s - 1, and
// rows vrow0 .. k0 - 1 zeroed).  T is formed afterwards by launch_form_t.
cudaError_t launch_panel_qr(double* K, long long kstride, int ld, const int* ms, int N, int k0,
                            int nbe, double* tau, int n, double* Vp, long long vstride, unsigned* status,
                            cudaStream_t st, bool fp32, int pcl_pref, int vrow0);
// Compact-WY T of panel [k0, k0+nbe) of every subdomain from G (v_l^T v_j at G[l*32 + j],
// l < j, per subdomain at stride gstride) and tau; T [32 x 32] column-major at T + s*tstride.
cudaError_t launch_form_t(const double* G, long long gstride, const double* tau, int n, int k0, int nbe,
                          int N, double* T, long long tstride, cudaStream_t st);
// Compact-WY T of a block of w <= 128 columns [k0, k0+w) (several panels) from its Gram
// matrix G (v_l^T v_j at G[j*gld + l], l < j, per subdomain at stride gstride): T [w x w]
// column-major with leading dimension tld at Tw + s*twstride; its diagonal 32-block
// starting at column dcol (the block's last panel) is also written to Td + s*tdstride
// (column-major, 32 x 32).
cudaError_t launch_form_t_wide(const double* G, long long gstride, int gld, const double* tau, int n,
                               int k0, int w, int N, double* Tw, long long twstride, int tld,
                               double* Td, long long tdstride, int dcol, cudaStream_t st);
cudaError_t launch_trsm_y(double* Y, long long ystride, int mgld, const double* K,
                          long long kstride, int ld, const int* mg, int mgmax, int N, int n,
                          cudaStream_t st);
// Diagonal step c0 of the blocked solve Y R = A (64 columns; the blocks to the left are
// already applied): Y[:, c0:c0+64] <- Y[:, c0:c0+64] R[c0:c0+64, c0:c0+64]^{-1}.
cudaError_t launch_trsm_y_diag(double* Y, long long ystride, int mgld, const double* K,
                               long long kstride, int ld, const int* mg, int mgmax, int N, int n,
                               int c0, cudaStream_t st);
cudaError_t launch_load_rhs(double* X, const double* rhs, int N, int m_max, int ld,
                            const int* cnt, int nrhs, unsigned* status, cudaStream_t st);
cudaError_t launch_apply_qt(double* X, const double* K, long long kstride, int ld,
                            const int* ms, int N, int n, const double* T, long long tstride,
                            int nrhs, cudaStream_t st);
// gq_s = Q_G q_s (m_Gamma rows, stride mgld) and hq_s = Y_s q_s (rows of A^s, stride mfld).
cudaError_t launch_iface_vecs(const double* X, const double* K, long long kstride, int ld,
                              const double* Y, long long ystride, int mgld, const int* mg, int mfld,
                              const int* mf, int N, int n, int nrhs, double* gq, double* hq,
                              cudaStream_t st);
// out[i] (+)= sum of a[s][l] over the (s, l) pairs of entry i: map [n][2 kmax], a list
// shorter than kmax ends at s = -1 (its first two pairs are always present).
cudaError_t launch_gather2(const int* map, int kmax, int n, int ldv, int N, const double* a,
                           double* out, int accumulate, int nrhs, cudaStream_t st);
// z_s = M_s^T (P_s h): M_s has mf[s] rows (ld mfld) and mg[s] columns; row k of M_s reads
// h[ffd[s][k]] (h of length n_flux); z has stride mgld.
cudaError_t launch_mt_h(const double* M, long long mstride, int mfld, const int* mf, const int* mg,
                        const int* ffd, const double* h, int n_flux, int N, int mgld, int nrhs,
                        double* z, cudaStream_t st);
// A-rows at explicit (collocation row, normal) pairs: A[s][f][c] = (w_c . n_f)(1 - t^2),
// t = tanh(w_c . x + b_c) at x = xy[s][frow[s][f]] (the corner rule of the remark in
// Section 3); columns of pad neurons (c >= nsub[s]) stay zero.
cudaError_t launch_flux_rows(double* A, long long astride, int mfld, const int* mf, int mfmax,
                             const int* frow, const double* fnrm, const double* xy, int m_max,
                             const double* W, const double* b, int N, int n, const int* nsub,
                             unsigned* status, cudaStream_t st);
cudaError_t launch_backsolve(const double* X, const double* K, long long kstride, int ld,
                             const int* mg, const int* ifc_dof, int mgld, const double* u,
                             int n_gamma, int N, int n, int nrhs, double* c, cudaStream_t st);

// Cholesky factor of the nb x nb diagonal block at (k, k) of S, in place (lower).
cudaError_t launch_potrf_diag(double* S, int ld, int k, int nb, unsigned* status, cudaStream_t st);
// Whole triangular solves with the factor in S (envelope per 64-row step: rend / jbeg,
// device arrays of nsteps; Linv the stored diagonal-block inverses), one cooperative
// launch each on `grid` blocks (chol_solve_grid: 0 when no co-resident grid fits).
// bar: 2 device words of barrier state.  Each grid barrier gives up after limit_ns of
// %globaltimer (flagging ST_TIMEOUT); hold = 1 withholds its release (test hook).
int chol_solve_grid(bool forward, int work_max);
constexpr unsigned long long kDefaultWaitNs = 2000000000ull;
cudaError_t launch_chol_fwd_all(const double* L, int ld, int n, const double* Linv, const int* rend,
                                int nsteps, double* r, double* y, int nrhs, int grid, unsigned* bar,
                                unsigned* status, cudaStream_t st,
                                unsigned long long limit_ns = kDefaultWaitNs, int hold = 0);
cudaError_t launch_chol_bwd_all(const double* L, int ld, int n, const double* Linv, const int* jbeg,
                                int nsteps, double* y, double* u, int nrhs, int grid, unsigned* bar,
                                unsigned* status, cudaStream_t st,
                                unsigned long long limit_ns = kDefaultWaitNs, int hold = 0);
// Inverses of every CHOL_NB diagonal block of the factor L (in S), column-major, ld CHOL_NB.
cudaError_t launch_tri_inv(const double* S, int ld, int n, double* inv, cudaStream_t st);
// L21 = A21 L11^{-T} by substitution for rows k+nb .. row_end-1 (16 rows per block).  With
// tA non-NULL it also writes L21's digit split for the SYRK: planes tA (128-row tiles) and
// tB (32-row tiles), row exponents eA and eB (K = nb).
cudaError_t launch_trsm_chol_rows(double* S, int ld, int k, int nb, int row_end, cudaStream_t st,
                                  void* tA = nullptr, void* tB = nullptr, int* eA = nullptr,
                                  int* eB = nullptr);
// row_end < 0 means n; j_begin 0 means all rows above the block; Linv (nullable) is the
// inverse of the diagonal block (CHOL_NB x CHOL_NB, column-major) when it is stored.
cudaError_t launch_chol_fwd(const double* L, int ld, int n, int k, int nb, double* r,
                            double* y, int nrhs, cudaStream_t st, int row_end = -1,
                            const double* Linv = nullptr);
cudaError_t launch_chol_bwd(const double* L, int ld, int n, int k, int nb, double* y,
                            double* u, int nrhs, cudaStream_t st, int j_begin = 0,
                            const double* Linv = nullptr);
cudaError_t launch_gather_perm(const int* idx, int n, const double* src, double* dst, int nrhs,
                               cudaStream_t st);
// q = S p without forming S (zl, wl: [nrhs][N][mgld] scratch, wg: [nrhs][ng] scratch).
cudaError_t launch_schur_apply(const double* D, const double* M, long long mstride, int mgld,
                               const int* mg, int mgmax, const int* ifc_dof, const int* dofmap,
                               const double* p, double* q, double* zl, double* wl, double* wg,
                               int ng, int N, int nrhs, cudaStream_t st);
// (Preconditioned) CG on the Schur system: dinv = 1 / diag(S) (Jacobi) or NULL.
cudaError_t launch_pcg_init(const double* b, const double* q, double* r, double* p, const double* dinv,
                            CgState* state, int ng, int nrhs, int has_x0, double tol2, cudaStream_t st);
cudaError_t launch_pcg_update(double* x, double* r, double* p, const double* q, const double* dinv,
                              CgState* state, int ng, int nrhs, double tol2, cudaStream_t st);
// Block-Jacobi preconditioner of the CG solves: the inverse of each interface edge's
// diagonal block of S (edge e: internal unknowns off[e] .. off[e] + len[e] - 1, len <= 128,
// inverse row-major at inv + ioff[e]), and its application z = B^{-1} r.
cudaError_t launch_block_inv(const double* S, int ng, const int* off, const int* len, const long long* ioff,
                             int nedges, int maxlen, double* inv, unsigned* status, cudaStream_t st);
cudaError_t launch_bj_apply(const double* inv, const int* off, const int* len, const long long* ioff, int nedges,
                            const double* r, double* z, int ng, int nrhs, cudaStream_t st);
// A CG step split around a preconditioner launched in between: step_a (alpha, x, r, r^T r),
// then z = M^{-1} r, then step_b (r^T z, beta, p; first = 1 at the start: p = z).
cudaError_t launch_pcg_step_a(double* x, double* r, const double* p, const double* q, CgState* state, int ng,
                              int nrhs, cudaStream_t st);
cudaError_t launch_pcg_step_b(const double* r, const double* z, double* p, CgState* state, int ng, int nrhs,
                              double tol2, int first, cudaStream_t st);
cudaError_t launch_scatter_perm(const int* idx, int n, const double* src, double* dst, int nrhs,
                                cudaStream_t st);
cudaError_t launch_diag_inv(const double* S, int n, double* dinv, cudaStream_t st);

// Mixed-precision refinement (k_refine.cu): FP64 residuals of the (c, w, u) system and
// the pieces of its correction.  Layouts: e, kw, F [nrhs][N][ld]; c, w, r1, t [nrhs][N][n];
// z, interface products [nrhs][N][mgld]; u, g [nrhs][ng] (internal interface order).
cudaError_t launch_resid_rows(const double* K, long long kstride, int ld, int n, const int* ms, const int* cnt,
                              const int* ifc_dof, int mgld, const double* F, const double* c, const double* w,
                              const double* u, int ng, int N, int mmax, int nrhs, double* e, double* kw,
                              double* z, cudaStream_t st);
cudaError_t launch_resid_cols(const double* K, long long kstride, int ld, int n, const int* ms, const double* e,
                              const double* kw, int N, int nrhs, double* r1, double* t, cudaStream_t st);
cudaError_t launch_amul(const double* A, long long astride, int mgld, const int* mg, int mgmax, int n,
                        const double* x, int N, int nrhs, double* out, cudaStream_t st);
// out = A^T (E g) + sg * t; with r1 non-NULL also d = r1 - out
cudaError_t launch_atmul(const double* A, long long astride, int mgld, const int* mg, const int* ifc_dof, int n,
                         const double* g, int ng, const double* t, double sg, const double* r1, int N, int nrhs,
                         double* out, double* d, cudaStream_t st);
// p = R^{-T} v for nvec vectors per subdomain (v at v + (vec N + s) vs, p at p + (vec N + s) ps)
cudaError_t launch_rt_solve(const double* K, long long kstride, int ld, int n, const double* v, long long vs,
                            double* p, long long ps, int N, int nvec, cudaStream_t st);
cudaError_t launch_refine_update(double* c, const double* dc, double* w, const double* dw, long long nc, double* u,
                                 const double* du, int ng, int nrhs, unsigned long long* nrm, cudaStream_t st);

// ---- device helpers ----
#ifdef __CUDACC__
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block (blockDim.x a multiple of 32, <= 1024); result in every thread.
// `red` must hold at least 33 doubles.  Contains __syncthreads.
__device__ __forceinline__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < nw ? red[lane] : 0.0;
    t = warp_sum(t);
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// 32 partial sums per lane -> lane L returns the warp-wide sum of entry L.
// Recursive halving: 31 shuffles instead of 32 x 5.
__device__ __forceinline__ double warp_transpose_sum32(double (&a)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < off; ++i) {
      const double send = up ? a[i] : a[i + off];
      const double keep = up ? a[i + off] : a[i];
      a[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  return a[0];
}
#endif

// Reciprocal of a positive normal double from an FP32 seed: d = m 2^(e - 1023) with m in
// [1, 2) truncated to 24 bits, r0 = 2^(1023 - e) / m (FP32 reciprocal, relative error below
// 2^-22 against 1/d), then one step of the third-order iteration for 1/d: with
// eps = 1 - d r0, 1/d = r0 / (1 - eps) = r0 (1 + eps + eps^2 + ...), so r0 (1 + eps + eps^2)
// has relative error about eps^3 < 2^-66, below the final rounding (Newton's second-order
// step r <- r + r (1 - d r) would need two steps).  Three dependent FP64 FMAs on the pivot
// chain instead of a division; d outside [2^-1020, 2^1020] takes the division.
__device__ __forceinline__ double rcp_newton(double d) {
  const long long b = __double_as_longlong(d);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e < 3 || e > 2043) return 1.0 / d;
  const float rf = __frcp_rn(__int_as_float(0x3F800000 | (int)((b >> 29) & 0x7FFFFF)));  // in (0.5, 1]
  const int fb = __float_as_int(rf);
  const long long rb = ((long long)(((fb >> 23) & 0xFF) - 127 + 2046 - e) << 52) | ((long long)(fb & 0x7FFFFF) << 29);
  const double r = __longlong_as_double(rb);
  const double eps = fma(-d, r, 1.0);
  return fma(r, fma(eps, eps, eps), r);
}

// y[i] = rcp_newton(x[i]) (self-test of the Cholesky pivots' reciprocal).
cudaError_t launch_rcp_newton(const double* x, double* y, int n, cudaStream_t st);

}  // namespace elmddm
