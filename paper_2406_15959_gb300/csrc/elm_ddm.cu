// Host side of the C ABI (include/elm_ddm.h): handle lifecycle, validation of the
// decomposition, the interface-edge structure of the Schur matrix, and the launch
// plans of Algorithm 1.  All launch descriptors are built once at setup, so the
// compute entry points only enqueue kernels.
#include "elm_ddm.h"
#include "common.cuh"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

namespace elmddm {
std::atomic<long long> g_kernel_launches{0};
}  // namespace elmddm

using namespace elmddm;

namespace {

struct LaunchRec {
  int kind;  // 0 = FP64 gemm, 1 = add_blocks, 2 = digit split, 3 = tensor-core digit GEMM,
             // 4 = persistent tensor-core digit GEMM for K <= 64 (max_tiles = total tiles),
             // 5 = tensor-core digit GEMM with the FP64 A operand split in the kernel,
             // 6 = diagonal step of the blocked Y = A R^{-1} (off = first column, nt = width),
             // 7 = compact-WY T of QR panel `off` from the Gram rows of its W1 product,
             // 8 = compact-WY T of the outer QR block of nt columns from column toff, whose
             //     last panel is `off`,
             // 9 = tensor-core digit GEMM with the FP64 B operand split in the kernel,
             // 10 = wide persistent tensor-core digit update (128 x 64 tiles, K <= 128)
  int off, count, max_tiles;  // split: max_tiles = blocks of k_split, nt = blocks of k_rowexp
  bool ta, tb;
  double alpha, beta;
  int flags;
  double flops;  // algorithmic flops of the launch (2mnk per GEMM; m(m+1)k for a lower SYRK)
  int nt;        // tensor-core GEMM: tile width (32 or 64); split: k_rowexp blocks
  double bytes = 0.0;          // algorithmic HBM bytes (FP64 operands read, C read/written)
  const char* name = nullptr;  // kernel class for profiling (nullptr: the caller's name)
  int toff = 0;                // persistent launches: offset of the tile table
  int side = 0;                // 1: runs on the handle's second stream, one SM left free
};

// One profiled launch: events around it, its class and algorithmic flops.
struct ProfRec {
  cudaEvent_t a, b;
  const char* name;
  double flops, bytes;
};

// An interface group ("edge"): a maximal run of consecutive interface unknowns held by
// the same k subdomains s[q], at local interface rows i[q] .. i[q] + len - 1 (k = 2 inside
// an edge, up to GRP_MAX at a cross point of the corner rule in Section 3).
struct Edge {
  int g0, len, k = 2;
  int s[GRP_MAX], i[GRP_MAX];  // owning subdomains and local interface-row offsets
};

// A flux group: a maximal run of consecutive flux conditions (rows of the global A) carried
// by the same two subdomains s[q], at rows i[q] .. i[q] + len - 1 of A^{s[q]}.  Without
// explicit flux rows the flux groups are the edges.
struct FGroup {
  int f0, len;
  int s[2], i[2];
};

inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Digit groups g = p + q of the low-precision local products (the 10 leading digit pairs:
// an error below about 2^-28 of the row and column maxima, against the FP32 panels' 2^-24).
constexpr int LO_GMAX = 5;

// Two-level blocking of the tensor-core QR: 32-column Householder panels inside outer
// blocks of QR_NBO columns.  Each panel updates only the rest of its outer block; the
// columns beyond it are updated once per outer block, with the block's aggregated
// compact-WY factor (K = QR_NBO in the update product instead of 32), so the trailing
// matrix is read and written n / QR_NBO times instead of n / 32.
#ifndef ELM_QR_NBO
#define ELM_QR_NBO 128
#endif
constexpr int QR_NBO = ELM_QR_NBO;
static_assert(QR_NBO % QR_NB == 0 && QR_NBO >= QR_NB && QR_NBO <= 128,
              "outer QR block: a multiple of the panel width, at most 128 (one product chunk)");

std::string g_setup_error;

// Reverse Cuthill-McKee ordering of a graph given by adjacency lists (self loops
// ignored): breadth-first from a pseudo-peripheral vertex of each component, neighbours
// in order of increasing degree, then reversed.  Keeps the Schur matrix's nonzero
// blocks close to the diagonal, so Cholesky fill stays inside a narrow envelope.
std::vector<int> rcm_order(const std::vector<std::vector<int>>& adj) {
  const int n = (int)adj.size();
  std::vector<int> deg(n);
  for (int i = 0; i < n; ++i) deg[i] = (int)adj[i].size();
  std::vector<char> done(n, 0);
  std::vector<int> order;
  order.reserve(n);
  auto farthest = [&](int start) {
    std::vector<int> dist(n, -1), q{start};
    dist[start] = 0;
    int best = start;
    for (size_t h = 0; h < q.size(); ++h) {
      const int v = q[h];
      if (dist[v] > dist[best] || (dist[v] == dist[best] && deg[v] < deg[best])) best = v;
      for (int w : adj[v])
        if (w != v && !done[w] && dist[w] < 0) { dist[w] = dist[v] + 1; q.push_back(w); }
    }
    return best;
  };
  while ((int)order.size() < n) {
    int start = -1;
    for (int i = 0; i < n; ++i)
      if (!done[i] && (start < 0 || deg[i] < deg[start])) start = i;
    start = farthest(farthest(start));
    std::vector<int> q{start};
    done[start] = 1;
    for (size_t h = 0; h < q.size(); ++h) {
      const int v = q[h];
      order.push_back(v);
      std::vector<int> nb;
      for (int w : adj[v])
        if (w != v && !done[w]) { done[w] = 1; nb.push_back(w); }
      std::sort(nb.begin(), nb.end(), [&](int a, int b) { return deg[a] != deg[b] ? deg[a] < deg[b] : a < b; });
      q.insert(q.end(), nb.begin(), nb.end());
    }
  }
  std::reverse(order.begin(), order.end());
  return order;
}

}  // namespace

struct elm_ddm_handle {
  elm_ddm_desc desc{};
  cudaStream_t st = nullptr;
  // Cholesky look-ahead (tensor-core back end): the SYRK of block step k beyond the next
  // block column runs on st2 while st factors that column; evS / evB order the two
  int sms = 0;
  char* creg = nullptr;       // the two parity buffers of L21's digit planes and exponents
  size_t creg_c1 = 0, creg_c2 = 0, creg_ce = 0;
  cudaStream_t st2 = nullptr;
  cudaEvent_t evS = nullptr, evB = nullptr;
  int N = 0, n = 0, m_max = 0, ld = 0, ncap = 0, mgmax = 0, mgld = 0, ng = 0, nblk = 0;
  int max_rhs = 1;
  long long kstride = 0, astride = 0, mstride = 0, tstride = 0, vstride = 0, wstride = 0;
  std::vector<int> cnt_h, ms_h, mg_h;
  // ELM_DDM_FLAG_NEURONS_PER_SUB: neurons of each subdomain (n_s <= n); the n - n_s pad
  // columns of K^s are identity columns on as many pad rows after the interface rows, so
  // ms_h = m_i + m_b + m_Gamma + (n - n_s) and mr_h = m_i + m_b + m_Gamma (rows with points)
  std::vector<int> ns_h, mr_h;
  int* nsub = nullptr;          // device copy of ns_h (NULL when every subdomain has n)
  // ELM_DDM_FLAG_RIDGE: n_s rows lambda_s I after the pad rows (Tikhonov regularisation of
  // the local least-squares problems), lambda_s = ridge_alpha * largest column norm of K^s
  bool ridge = false;
  double ridge_alpha = 1e-14;
  std::vector<Edge> edges;
  std::vector<FGroup> fgroups;
  // rows of A^s (flux rows): one per interface row, or the explicit rows of
  // elm_ddm_setup_flux; n_flux global flux conditions (internal order: the unknowns' without
  // explicit rows, the caller's with them)
  std::vector<int> mf_h;
  int mfmax = 0, mfld = 0, n_flux = 0;
  bool explicit_flux = false;
  int* mf = nullptr;            // device copy of mf_h
  int* fluxmap = nullptr;       // [n_flux][4]: (subdomain, row of A^s) of both rows of a condition
  int* ffd = nullptr;           // [N][mfld]: flux condition of every row of A^s
  int* frow = nullptr;          // [N][mfld]: collocation row of every explicit row of A^s
  double* fnrm = nullptr;       // [N][mfld][2]: its normal
  std::vector<int> newoff;      // internal offset of each edge's first unknown
  std::vector<int> perm_h;      // caller interface unknown -> internal index
  std::vector<int> chol_rend;   // per Cholesky block step: end of the envelope rows
  std::vector<int> chol_jbeg;   // per Cholesky block step: first column the block rows touch
  int* d_rend = nullptr;        // device copies of chol_rend / chol_jbeg
  int* d_jbeg = nullptr;
  unsigned* cbar = nullptr;     // grid-barrier state of the persistent triangular solves
  unsigned long long wait_ns = kDefaultWaitNs;  // limit of their bounded grid-barrier waits
  int wait_hold = 0;            // 1: withhold every barrier's release (failure-detection test)
  // tile choices (elm_ddm_set_tuning): CTAs per subdomain of the FP64 Householder panel
  // (0: the smallest cluster whose shared memory holds the panel), and the grid cap of the
  // persistent products (0: one CTA per SM)
  int tune_panel = 0, tune_upd_grid = 0;
  int fwd_grid = 0, bwd_grid = 0;  // their grids (0: one launch per block step instead)
  // device buffers
  double *K = nullptr, *Am = nullptr, *tau = nullptr, *T = nullptr, *Vp = nullptr;
  // two-level QR (tensor-core path): compact-WY T of each outer block of QR_NBO columns,
  // [N][QR_NBO][QR_NBO] column-major, and where each panel writes its explicit reflectors
  double* Tab = nullptr;
  long long* hlbuf = nullptr;   // [N][OZ_HL_TILE] split-K accumulators of the inner W1 products
  std::vector<int> panel_vcol, panel_vrow0;  // per panel: column of Vp, first zeroed row
  double *W1 = nullptr, *W2 = nullptr, *D = nullptr, *M = nullptr, *S = nullptr;
  double *Mdiag = nullptr, *thW = nullptr, *thb = nullptr, *xy = nullptr, *nrm = nullptr;
  double* cinv = nullptr;             // inverses of the Cholesky diagonal blocks, one per step
  // factored activation (k_assemble.cu): distinct coordinates per subdomain and tables
  AsmTables tabs;
  bool use_tabs = false;
  double *tab_xs = nullptr, *tab_ys = nullptr, *tab_ctr = nullptr, *tab_Tx = nullptr, *tab_Ty = nullptr;
  int *tab_nxy = nullptr, *tab_rix = nullptr;
  std::vector<LaunchRec> ty_recs;     // blocked Y = A R^{-1} (tensor-core path)
  double *X = nullptr, *gq = nullptr, *hq = nullptr, *zv = nullptr;
  double *rv = nullptr, *hv = nullptr, *yv = nullptr, *uv = nullptr;
  int *cnt = nullptr, *ms = nullptr, *mg = nullptr, *dofmap = nullptr, *ifc_dof = nullptr;
  int* perm = nullptr;
  int* colexp = nullptr;        // [N][ncap] exponent bounds of the columns of [K^s | J] (tensor-core QR)
  unsigned* status = nullptr;
  GemmDesc* gd = nullptr;
  AddDesc* ad = nullptr;
  SplitDesc* sd = nullptr;
  OzDesc* od = nullptr;
  int4* ut = nullptr;  // tile tables of the persistent launches
  bool emulated = true;          // FP64 products on the tensor cores (digit split)
  // mixed-precision mode (ELM_DDM_FLAG_MIXED): the local factorisation in low precision
  // (FP32 Householder panels, digit-split products with LO_GMAX groups), the Schur matrix
  // assembled and factored in FP64, and the solve refined on FP64 residuals
  bool mixed = false;
  bool lowfac = false;           // the current factorisation is the low-precision one
  int refine_maxit = 16;
  double refine_tol = 1e-12;     // relative size of the last u_Gamma correction
  int last_iters = 0, last_fallback = 0;
  double last_eta = 0.0;
  double *K64 = nullptr, *A64 = nullptr, *F64 = nullptr;  // FP64 K^s (n columns), A^s, F^s
  double *cit = nullptr, *wit = nullptr, *uit = nullptr;  // iterates c, w, u (internal order)
  double *dcv = nullptr, *dwv = nullptr, *ebuf = nullptr, *kwbuf = nullptr, *zb = nullptr;
  double *r1b = nullptr, *r3b = nullptr, *r13b = nullptr, *tb = nullptr, *Pb = nullptr;
  double *Acl = nullptr, *Acg = nullptr, *zero_ng = nullptr, *gq2 = nullptr, *hq2 = nullptr;
  unsigned long long* nrmb = nullptr;
  bool cg_only = false;          // S is neither formed nor factored (elm_ddm_solve_cg only)
  int op = ELM_DDM_OP_POISSON;
  double* coef = nullptr;        // [N][m_max][3] rho, grad rho (ELM_DDM_OP_VARCOEF)
  bool coef_set = false;
  double *cg_p = nullptr, *cg_q = nullptr;  // CG search direction and S p, [max_rhs][ng]
  CgState* cg_st = nullptr;                 // [max_rhs]
  double* sdinv = nullptr;                  // 1 / diag(S), internal order (Jacobi), set by schur
  // ELM_DDM_FLAG_BLOCK_JACOBI: inverses of S's diagonal block of every edge (set by schur)
  bool bj = false, has_bj = false;
  int bj_maxlen = 0;
  int *bj_off = nullptr, *bj_len = nullptr;
  long long* bj_ioff = nullptr;
  double *bj_inv = nullptr, *cg_z = nullptr;
  bool has_sdinv = false;
  void* sp_buf = nullptr;        // digit tiles and row exponents of the split operands
  std::vector<int> qr_first;     // first record of each panel in qr_recs
  // algorithmic flops of each Householder panel launch: per subdomain the m' x nb panel's
  // Householder work, 2 m' nb^2 - 2 nb^3 / 3 (the compact-WY factor T, m' nb^2 more, is
  // blocking overhead and not counted)
  std::vector<double> panel_flops, panel_bytes;  // per QR panel, summed over subdomains
  double asm_bytes = 0.0;        // algorithmic HBM bytes of one assembly: [K^s | J] and A^s written
  std::vector<int> syrk_first;   // first record of each Cholesky step in syrk_recs
  size_t mdiag_elems = 0;
  // plans
  std::vector<LaunchRec> qr_recs;    // per panel: the trailing-update launches
  std::vector<LaunchRec> dm_recs;    // D and M
  std::vector<LaunchRec> s_recs;     // Mdiag adds, D adds, M^T M gemms
  std::vector<LaunchRec> syrk_recs;  // one per Cholesky block step
  int state = 0;
  bool profiling = false;
  std::string prof_only;  // non-empty: profile launches of this class only
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<ProfRec> prof;
  int prof_dropped = 0;
  long long launches = 0;
  size_t bytes = 0;
  std::string err;
  std::vector<void*> allocs;
};

namespace {

int fail(elm_ddm_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  else g_setup_error = msg;
  return code;
}

int cuda_fail(elm_ddm_handle* h, cudaError_t e, const char* where) {
  return fail(h, ELM_DDM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

template <class T>
bool dev_alloc(elm_ddm_handle* h, T** p, size_t count) {
  if (count == 0) count = 1;
  void* q = nullptr;
  if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  h->allocs.push_back(q);
  h->bytes += count * sizeof(T);
  *p = static_cast<T*>(q);
  return true;
}

void free_all(elm_ddm_handle* h) {
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
  if (h->st2) { cudaStreamSynchronize(h->st2); cudaStreamDestroy(h->st2); h->st2 = nullptr; }
  if (h->evS) { cudaEventDestroy(h->evS); h->evS = nullptr; }
  if (h->evB) { cudaEventDestroy(h->evB); h->evB = nullptr; }
}

cudaEvent_t next_event(elm_ddm_handle* h) {
  if (h->ev_used < h->ev_pool.size()) return h->ev_pool[h->ev_used++];
  if (h->ev_pool.size() >= 65536) return nullptr;
  cudaEvent_t e;
  if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  h->ev_pool.push_back(e);
  h->ev_used++;
  return e;
}

// Records an event pair around one launch when profiling is enabled.
struct ProfScope {
  elm_ddm_handle* h;
  cudaEvent_t a = nullptr;
  const char* name;
  double flops, bytes;
  cudaStream_t st;
  ProfScope(elm_ddm_handle* h_, const char* n, double f, double by = 0.0, cudaStream_t s = nullptr)
      : h(h_), name(n), flops(f), bytes(by), st(s ? s : h_->st) {
    if (h->profiling && (h->prof_only.empty() || h->prof_only == name)) {
      a = next_event(h);
      if (a) cudaEventRecord(a, st);
      else h->prof_dropped++;
    }
  }
  ~ProfScope() {
    if (!a) return;
    cudaEvent_t b = next_event(h);
    if (!b) { h->prof_dropped++; return; }
    cudaEventRecord(b, st);
    h->prof.push_back({a, b, name, flops, bytes});
  }
};

#define ELM_LAUNCH_FB(h, expr, where, flops, bytes)          \
  do {                                                       \
    cudaError_t e_;                                          \
    {                                                        \
      ProfScope ps_((h), (where), (flops), (bytes));         \
      e_ = (expr);                                           \
    }                                                        \
    (h)->launches++;                                         \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, where); \
  } while (0)
#define ELM_LAUNCH_F(h, expr, where, flops)                  \
  do {                                                       \
    cudaError_t e_;                                          \
    {                                                        \
      ProfScope ps_((h), (where), (flops));                  \
      e_ = (expr);                                           \
    }                                                        \
    (h)->launches++;                                         \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, where); \
  } while (0)
#define ELM_LAUNCH(h, expr, where) ELM_LAUNCH_F(h, expr, where, 0.0)

int run_recs(elm_ddm_handle* h, const std::vector<LaunchRec>& recs, size_t first, size_t cnt,
             const char* gemm_name, int gmax = 8) {
  for (size_t r = first; r < first + cnt && r < recs.size(); ++r) {
    const LaunchRec& L = recs[r];
    if (L.count <= 0) continue;
    const char* nm = L.name ? L.name : gemm_name;
    if (L.kind == 0)
      ELM_LAUNCH_FB(h, launch_gemm(L.ta, L.tb, h->gd + L.off, L.count, L.max_tiles, L.alpha, L.beta,
                                   L.flags, h->st), nm, L.flops, L.bytes);
    else if (L.kind == 1)
      ELM_LAUNCH(h, launch_add_blocks(h->ad + L.off, L.count, L.max_tiles, h->st), "add_blocks");
    else if (L.kind == 2)
      ELM_LAUNCH_FB(h, launch_split(h->sd + L.off, L.count, L.nt, L.max_tiles, h->st), nm, 0.0,
                    L.bytes);
    else if (L.kind == 3)
      ELM_LAUNCH_FB(h, launch_ozaki(L.nt, h->od + L.off, L.count, L.max_tiles, L.alpha, L.beta,
                                    L.flags, h->status, h->st, gmax), nm, L.flops, L.bytes);
    else if (L.kind == 7)
      ELM_LAUNCH(h, launch_form_t(h->W1, h->wstride, h->tau, h->n, L.off * QR_NB, L.nt, h->N,
                                  h->T + (size_t)L.off * QR_NB * QR_NB, h->tstride, h->st), nm);
    else if (L.kind == 8)
      ELM_LAUNCH(h, launch_form_t_wide(h->W1, h->wstride, QR_NBO, h->tau, h->n, L.toff, L.nt, h->N, h->Tab,
                                       (long long)QR_NBO * QR_NBO, QR_NBO,
                                       h->T + (size_t)L.off * QR_NB * QR_NB, h->tstride,
                                       L.off * QR_NB - L.toff, h->st), nm);
    else if (L.kind == 6)
      ELM_LAUNCH_F(h, launch_trsm_y_diag(h->Am, h->astride, h->mfld, h->K, h->kstride, h->ld, h->mf,
                                         h->mfmax, h->N, h->n, L.off, h->st), nm, L.flops);
    else if (L.kind == 4 && L.side) {
      cudaError_t e_;
      {
        ProfScope ps_(h, nm, L.flops, L.bytes, h->st2);
        e_ = launch_ozaki_upd(h->od + L.off, L.count, h->ut + L.toff, L.max_tiles, L.alpha, L.beta,
                              L.flags, h->status, h->st2, h->sms - 1, gmax);
      }
      h->launches++;
      if (e_ != cudaSuccess) return cuda_fail(h, e_, nm);
    } else if (L.kind == 4)
      ELM_LAUNCH_FB(h, launch_ozaki_upd(h->od + L.off, L.count, h->ut + L.toff, L.max_tiles, L.alpha,
                                        L.beta, L.flags, h->status, h->st, h->tune_upd_grid, gmax), nm,
                    L.flops, L.bytes);
    else if (L.kind == 10)
      ELM_LAUNCH_FB(h, launch_ozaki_updw(h->od + L.off, L.count, h->ut + L.toff, L.max_tiles, L.alpha, h->status,
                                         h->st, h->tune_upd_grid, gmax), nm, L.flops, L.bytes);
    else if (L.kind == 9)
      ELM_LAUNCH_FB(h, launch_ozaki_fb(h->od + L.off, L.count, L.max_tiles, h->status, h->st, gmax, L.nt), nm,
                    L.flops, L.bytes);
    else
      ELM_LAUNCH_FB(h, launch_ozaki_fa(h->od + L.off, L.count, L.max_tiles, h->status, h->st, gmax,
                                       L.nt > 1 ? L.nt : 1), nm, L.flops, L.bytes);
  }
  return ELM_DDM_OK;
}

// Step (a) from the handle's theta: K^s, J, A^s (and, in mixed-precision mode, the FP64
// copies of K^s and A^s that the refinement's residuals use).
int assemble_launch(elm_ddm_handle* h) {
  cudaError_t e = cudaMemsetAsync(h->Am, 0, (size_t)h->N * h->astride * sizeof(double), h->st);
  if (e != cudaSuccess) return cuda_fail(h, e, "assemble: clear A");
  if (h->nsub && (h->desc.flags & ELM_DDM_FLAG_NEURONS_PER_SUB))
    ELM_LAUNCH(h, launch_zero_pad_theta(h->thW, h->thb, h->nsub, h->N, h->n, h->st), "assemble");
  // A^s: with the interface rows (one row per interface row, its normal), or from the
  // explicit rows
  ELM_LAUNCH_FB(h, launch_assemble(h->K, h->kstride, h->ld, h->ncap, h->explicit_flux ? nullptr : h->Am,
                                   h->astride, h->mfld, h->xy, h->nrm, h->m_max, h->cnt, h->thW, h->thb,
                                   h->N, h->n, h->op == ELM_DDM_OP_VARCOEF ? h->coef : nullptr,
                                   h->use_tabs ? &h->tabs : nullptr, h->status, h->st, h->nsub),
                "assemble", 0.0, h->asm_bytes);
  if (h->explicit_flux)
    ELM_LAUNCH(h, launch_flux_rows(h->Am, h->astride, h->mfld, h->mf, h->mfmax, h->frow, h->fnrm, h->xy,
                                   h->m_max, h->thW, h->thb, h->N, h->n, h->nsub, h->status, h->st),
               "assemble");
  if (h->ridge)
    ELM_LAUNCH(h, launch_ridge_rows(h->K, h->kstride, h->ld, h->cnt, h->nsub, h->N, h->n, h->ridge_alpha, h->st),
               "assemble");
  if (h->emulated)
    ELM_LAUNCH(h, launch_colexp(h->K, h->kstride, h->ld, h->ncap, h->ms, h->N, h->colexp, h->st), "colexp");
  if (h->mixed) {
    const size_t col = (size_t)h->ld * h->n * sizeof(double);
    e = cudaMemcpy2DAsync(h->K64, col, h->K, (size_t)h->kstride * sizeof(double), col, h->N,
                          cudaMemcpyDeviceToDevice, h->st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h->A64, h->Am, (size_t)h->N * h->astride * sizeof(double), cudaMemcpyDeviceToDevice,
                          h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "assemble: FP64 copies");
  }
  h->state = 1;
  return ELM_DDM_OK;
}

int solve_refined(elm_ddm_handle* h, const double* rhs, int nrhs, double* u_gamma, double* c);
int chol_solves(elm_ddm_handle* h, int nrhs);

}  // namespace

extern "C" {

int elm_ddm_setup(const elm_ddm_desc* desc, const int32_t* counts, const double* xy,
                  const double* nrm, const int32_t* dof, void* stream, elm_ddm_handle** out) {
  return elm_ddm_setup_flux(desc, counts, xy, nrm, dof, nullptr, stream, out);
}

int elm_ddm_setup_flux(const elm_ddm_desc* desc, const int32_t* counts, const double* xy,
                       const double* nrm, const int32_t* dof, const elm_ddm_flux_rows* flux,
                       void* stream, elm_ddm_handle** out) {
  if (!out) return fail(nullptr, ELM_DDM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!desc || !counts || !xy || !nrm || !dof)
    return fail(nullptr, ELM_DDM_ERR_ARG, "NULL descriptor or geometry array");
  const int N = desc->n_sub, n = desc->n_neurons, m_max = desc->m_max, ng = desc->n_gamma;
  if (N < 1 || n < 1 || m_max < 1 || ng < 0)
    return fail(nullptr, ELM_DDM_ERR_ARG, "n_sub, n_neurons, m_max must be >= 1 and n_gamma >= 0");
  if (desc->op != ELM_DDM_OP_POISSON && desc->op != ELM_DDM_OP_VARCOEF)
    return fail(nullptr, ELM_DDM_ERR_ARG, "unsupported operator");
  const int max_rhs = desc->max_rhs == 0 ? 1 : desc->max_rhs;
  if (max_rhs < 1 || max_rhs > 64) return fail(nullptr, ELM_DDM_ERR_ARG, "max_rhs must be in 1..64");
  if (n > TRSV_MAX_N) return fail(nullptr, ELM_DDM_ERR_ARG, "n_neurons > 8192 is not supported");
  if (desc->flags & ~(ELM_DDM_FLAG_FP64_SIMT | ELM_DDM_FLAG_SCHUR_CG | ELM_DDM_FLAG_DIRECT_ASSEMBLY |
                      ELM_DDM_FLAG_MIXED | ELM_DDM_FLAG_NEURONS_PER_SUB | ELM_DDM_FLAG_RIDGE |
                      ELM_DDM_FLAG_BLOCK_JACOBI))
    return fail(nullptr, ELM_DDM_ERR_ARG, "unknown flags");
  if ((desc->flags & ELM_DDM_FLAG_BLOCK_JACOBI) && (desc->flags & (ELM_DDM_FLAG_SCHUR_CG | ELM_DDM_FLAG_MIXED)))
    return fail(nullptr, ELM_DDM_ERR_ARG,
                "ELM_DDM_FLAG_BLOCK_JACOBI needs the assembled S of the FP64 factorisation");
  if ((desc->flags & ELM_DDM_FLAG_MIXED) && (desc->flags & (ELM_DDM_FLAG_FP64_SIMT | ELM_DDM_FLAG_SCHUR_CG)))
    return fail(nullptr, ELM_DDM_ERR_ARG,
                "ELM_DDM_FLAG_MIXED needs the tensor-core back end and the direct Schur solve");
  if ((long long)N * m_max > (1ll << 31)) return fail(nullptr, ELM_DDM_ERR_ARG, "geometry too large");
  if (flux) {
    if (desc->flags & (ELM_DDM_FLAG_SCHUR_CG | ELM_DDM_FLAG_MIXED | ELM_DDM_FLAG_BLOCK_JACOBI))
      return fail(nullptr, ELM_DDM_ERR_ARG,
                  "explicit flux rows: not with ELM_DDM_FLAG_SCHUR_CG, _MIXED or _BLOCK_JACOBI");
    if (!flux->count || !flux->row || !flux->nrm || !flux->fdof || flux->f_max < 1 || flux->n_flux < 0 ||
        (ng > 0 && flux->n_flux < 1) || (long long)N * flux->f_max > (1ll << 31))
      return fail(nullptr, ELM_DDM_ERR_ARG, "explicit flux rows: NULL array or bad n_flux / f_max");
  }

  auto h = new elm_ddm_handle();
  h->desc = *desc;
  h->st = static_cast<cudaStream_t>(stream);
  h->N = N; h->n = n; h->m_max = m_max; h->ng = ng; h->max_rhs = max_rhs;
  h->emulated = !(desc->flags & ELM_DDM_FLAG_FP64_SIMT);
  h->cg_only = (desc->flags & ELM_DDM_FLAG_SCHUR_CG) != 0;
  h->mixed = (desc->flags & ELM_DDM_FLAG_MIXED) != 0;
  h->ridge = (desc->flags & ELM_DDM_FLAG_RIDGE) != 0;
  h->bj = (desc->flags & ELM_DDM_FLAG_BLOCK_JACOBI) != 0;
  h->op = desc->op;
  const int cst = (desc->flags & ELM_DDM_FLAG_NEURONS_PER_SUB) ? 4 : 3;  // counts row stride
  h->cnt_h.resize(3 * (size_t)N);
  h->ms_h.resize(N); h->mg_h.resize(N); h->ns_h.resize(N); h->mr_h.resize(N);
  int msmax = 0, mgmax = 0;
  for (int s = 0; s < N; ++s) {
    const int mi = counts[cst * s], mb = counts[cst * s + 1], mgs = counts[cst * s + 2];
    const int ns = cst == 4 ? counts[cst * s + 3] : n;
    if (mi < 0 || mb < 0 || mgs < 0 || mi + mb + mgs > m_max) {
      delete h;
      return fail(nullptr, ELM_DDM_ERR_ARG, "counts of subdomain " + std::to_string(s) + " invalid");
    }
    if (ns < 1 || ns > n) {
      delete h;
      return fail(nullptr, ELM_DDM_ERR_ARG,
                  "neurons of subdomain " + std::to_string(s) + " not in 1..n_neurons");
    }
    if (mi + mb + mgs < ns) {
      delete h;
      return fail(nullptr, ELM_DDM_ERR_ARG,
                  "subdomain " + std::to_string(s) + " has fewer rows than neurons");
    }
    h->cnt_h[3 * s] = mi; h->cnt_h[3 * s + 1] = mb; h->cnt_h[3 * s + 2] = mgs;
    h->ns_h[s] = ns;
    h->mr_h[s] = mi + mb + mgs;
    if ((ng == 0) != (mgs == 0) && N > 1) {
      delete h;
      return fail(nullptr, ELM_DDM_ERR_ARG, "interface rows inconsistent with n_gamma");
    }
    if (N == 1 && mgs != 0) {
      delete h;
      return fail(nullptr, ELM_DDM_ERR_ARG, "a single subdomain cannot have interface rows");
    }
    h->ms_h[s] = mi + mb + mgs + (n - ns) + (h->ridge ? ns : 0);
    h->mg_h[s] = mgs;
    msmax = std::max(msmax, h->ms_h[s]);
    mgmax = std::max(mgmax, mgs);
  }
  for (size_t i = 0; i < (size_t)N * m_max * 2; ++i) {
    if (!std::isfinite(xy[i])) {
      delete h;
      return fail(nullptr, ELM_DDM_ERR_NONFINITE, "non-finite collocation point");
    }
  }

  // ---- interface unknowns: owners, edges ----
  std::vector<std::vector<std::pair<int, int>>> owners(ng);
  for (int s = 0; s < N; ++s) {
    const int r0 = h->cnt_h[3 * s] + h->cnt_h[3 * s + 1];
    for (int i = 0; i < h->mg_h[s]; ++i) {
      const int g = dof[(size_t)s * m_max + r0 + i];
      if (g < 0 || g >= ng) {
        delete h;
        return fail(nullptr, ELM_DDM_ERR_ARG, "interface unknown index out of range");
      }
      owners[g].push_back({s, i});
    }
  }
  const size_t kmax_own = flux ? GRP_MAX : 2;
  for (int g = 0; g < ng; ++g) {
    std::vector<int> ss;
    for (auto& o : owners[g]) ss.push_back(o.first);
    std::sort(ss.begin(), ss.end());
    if (owners[g].size() < 2 || owners[g].size() > kmax_own ||
        std::unique(ss.begin(), ss.end()) != ss.end()) {
      delete h;
      return fail(nullptr, ELM_DDM_ERR_ARG,
                  "interface unknown " + std::to_string(g) +
                      (flux ? " is not shared by two to four subdomains" : " is not shared by exactly two subdomains"));
    }
    std::sort(owners[g].begin(), owners[g].end());
  }
  auto same_owners = [&](int g1, int g2) {
    if (owners[g1].size() != owners[g2].size()) return false;
    for (size_t q = 0; q < owners[g1].size(); ++q)
      if (owners[g1][q].first != owners[g2][q].first) return false;
    return true;
  };
  // segments: maximal runs with consecutive unknowns and the same sharing subdomains
  std::map<int, std::vector<std::array<int, 3>>> segs;  // g0 -> list of {s, i0, len}
  for (int s = 0; s < N; ++s) {
    const int r0 = h->cnt_h[3 * s] + h->cnt_h[3 * s + 1];
    const int* d = dof + (size_t)s * m_max + r0;
    int i = 0;
    while (i < h->mg_h[s]) {
      int j = i + 1;
      while (j < h->mg_h[s] && d[j] == d[j - 1] + 1 && same_owners(d[j], d[i])) ++j;
      segs[d[i]].push_back({s, i, j - i});
      i = j;
    }
  }
  int covered = 0;
  for (auto& kv : segs) {
    const size_t k = owners[kv.first].size();
    bool okk = kv.second.size() == k;
    for (size_t q = 1; okk && q < k; ++q) okk = kv.second[q][2] == kv.second[0][2];
    if (!okk) {
      delete h;
      return fail(nullptr, ELM_DDM_ERR_ARG, "interface rows do not form matching edges");
    }
    Edge e;
    e.g0 = kv.first;
    e.len = kv.second[0][2];
    e.k = (int)k;
    std::sort(kv.second.begin(), kv.second.end());
    for (size_t q = 0; q < k; ++q) { e.s[q] = kv.second[q][0]; e.i[q] = kv.second[q][1]; }
    if (e.g0 != covered) {
      delete h;
      return fail(nullptr, ELM_DDM_ERR_ARG, "interface edges overlap or leave gaps");
    }
    covered += e.len;
    h->edges.push_back(e);
  }
  if (covered != ng) {
    delete h;
    return fail(nullptr, ELM_DDM_ERR_ARG, "interface edges do not cover all unknowns");
  }

  // ---- rows of A^s and the flux conditions they belong to ----
  // Without explicit rows: one per interface row (its point and normal), condition = its
  // unknown.  fr_h / fd_h: per subdomain the interface-row index and condition of each row.
  h->explicit_flux = flux != nullptr;
  h->n_flux = flux ? flux->n_flux : ng;
  h->mf_h.assign(N, 0);
  std::vector<std::vector<int>> fr_h(N), fd_h(N);
  std::vector<std::vector<double>> fn_h(N);
  for (int s = 0; s < N; ++s) {
    const int r0 = h->cnt_h[3 * s] + h->cnt_h[3 * s + 1];
    if (!flux) {
      h->mf_h[s] = h->mg_h[s];
      for (int i = 0; i < h->mg_h[s]; ++i) {
        fr_h[s].push_back(i);
        fd_h[s].push_back(dof[(size_t)s * m_max + r0 + i]);
      }
      continue;
    }
    const int c = flux->count[s];
    if (c < 0 || c > flux->f_max || (c > 0 && h->mg_h[s] == 0)) {
      delete h;
      return fail(nullptr, ELM_DDM_ERR_ARG, "flux rows of subdomain " + std::to_string(s) + ": bad count");
    }
    h->mf_h[s] = c;
    for (int f = 0; f < c; ++f) {
      const size_t q = (size_t)s * flux->f_max + f;
      const int r = flux->row[q], cd = flux->fdof[q];
      const double nx = flux->nrm[2 * q], ny = flux->nrm[2 * q + 1];
      if (r < 0 || r >= h->mg_h[s] || cd < 0 || cd >= flux->n_flux) {
        delete h;
        return fail(nullptr, ELM_DDM_ERR_ARG, "flux rows of subdomain " + std::to_string(s) + ": row or condition out of range");
      }
      if (!std::isfinite(nx) || !std::isfinite(ny)) {
        delete h;
        return fail(nullptr, ELM_DDM_ERR_NONFINITE, "non-finite flux-row normal");
      }
      fr_h[s].push_back(r);
      fd_h[s].push_back(cd);
      fn_h[s].push_back(nx);
      fn_h[s].push_back(ny);
    }
  }
  for (int s = 0; s < N; ++s) h->mfmax = std::max(h->mfmax, h->mf_h[s]);
  std::vector<std::vector<std::pair<int, int>>> fown(h->n_flux);
  for (int s = 0; s < N; ++s)
    for (int f = 0; f < h->mf_h[s]; ++f) fown[fd_h[s][f]].push_back({s, f});
  for (int c = 0; c < h->n_flux; ++c) {
    if (fown[c].size() != 2 || fown[c][0].first == fown[c][1].first) {
      delete h;
      return fail(nullptr, ELM_DDM_ERR_ARG,
                  "flux condition " + std::to_string(c) + " is not carried by rows of exactly two subdomains");
    }
    std::sort(fown[c].begin(), fown[c].end());
  }
  {
    auto partner = [&](int c, int s) { return fown[c][0].first == s ? fown[c][1].first : fown[c][0].first; };
    std::map<int, std::vector<std::array<int, 3>>> fsegs;  // f0 -> {s, first row, len}
    for (int s = 0; s < N; ++s) {
      const std::vector<int>& d = fd_h[s];
      int i = 0;
      while (i < h->mf_h[s]) {
        int j = i + 1;
        while (j < h->mf_h[s] && d[j] == d[j - 1] + 1 && partner(d[j], s) == partner(d[i], s)) ++j;
        fsegs[d[i]].push_back({s, i, j - i});
        i = j;
      }
    }
    int fcov = 0;
    for (auto& kv : fsegs) {
      if (kv.second.size() != 2 || kv.second[0][2] != kv.second[1][2] || kv.first != fcov) {
        delete h;
        return fail(nullptr, ELM_DDM_ERR_ARG, "flux rows do not form matching groups");
      }
      std::sort(kv.second.begin(), kv.second.end());
      FGroup F;
      F.f0 = kv.first;
      F.len = kv.second[0][2];
      for (int q = 0; q < 2; ++q) { F.s[q] = kv.second[q][0]; F.i[q] = kv.second[q][1]; }
      fcov += F.len;
      h->fgroups.push_back(F);
    }
    if (fcov != h->n_flux) {
      delete h;
      return fail(nullptr, ELM_DDM_ERR_ARG, "flux rows do not cover all conditions");
    }
  }

  // ---- Schur-matrix block pattern, interface ordering and Cholesky envelope ----
  // Edges e1, e2 couple in S when they share a subdomain (the D term) or some flux group
  // shares a subdomain with both (the M^T M term).  nbr[e]: edges sharing a subdomain with
  // e; fnbr[f]: edges sharing a subdomain with flux group f; efl[e]: flux groups sharing a
  // subdomain with edge e.
  const int ne = (int)h->edges.size(), nfg = (int)h->fgroups.size();
  std::vector<std::vector<int>> sub_edges(N), sub_fg(N), nbr(ne), spat(ne), fnbr(nfg), efl(ne);
  auto uniq = [](std::vector<int>& v) {
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
  };
  for (int e = 0; e < ne; ++e) for (int q = 0; q < h->edges[e].k; ++q) sub_edges[h->edges[e].s[q]].push_back(e);
  for (int f = 0; f < nfg; ++f) for (int q = 0; q < 2; ++q) sub_fg[h->fgroups[f].s[q]].push_back(f);
  for (int e = 0; e < ne; ++e) {
    for (int q = 0; q < h->edges[e].k; ++q) {
      for (int e2 : sub_edges[h->edges[e].s[q]]) nbr[e].push_back(e2);
      for (int f : sub_fg[h->edges[e].s[q]]) efl[e].push_back(f);
    }
    uniq(nbr[e]);
    uniq(efl[e]);
  }
  for (int f = 0; f < nfg; ++f) {
    for (int q = 0; q < 2; ++q) for (int e2 : sub_edges[h->fgroups[f].s[q]]) fnbr[f].push_back(e2);
    uniq(fnbr[f]);
  }
  for (int e1 = 0; e1 < ne; ++e1) {
    spat[e1] = nbr[e1];
    for (int f : efl[e1]) for (int e2 : fnbr[f]) spat[e1].push_back(e2);
    uniq(spat[e1]);
  }
  {
    const std::vector<int> order = rcm_order(spat);
    h->newoff.assign(ne, 0);
    int off = 0;
    for (int pos = 0; pos < ne; ++pos) { h->newoff[order[pos]] = off; off += h->edges[order[pos]].len; }
    if (h->bj) {
      for (const Edge& ed : h->edges) h->bj_maxlen = std::max(h->bj_maxlen, ed.len);
      if (h->bj_maxlen > 128) {
        delete h;
        return fail(nullptr, ELM_DDM_ERR_ARG, "ELM_DDM_FLAG_BLOCK_JACOBI: an interface edge has more than 128 unknowns");
      }
    }
    h->perm_h.assign(ng, 0);
    for (int e = 0; e < ne; ++e)
      for (int k = 0; k < h->edges[e].len; ++k) h->perm_h[h->edges[e].g0 + k] = h->newoff[e] + k;
    // first nonzero column of every internal row (fill stays right of it)
    std::vector<int> first_col(ng, 0);
    for (int e1 = 0; e1 < ne; ++e1) {
      int f = h->newoff[e1];
      for (int e2 : spat[e1]) f = std::min(f, h->newoff[e2]);
      for (int k = 0; k < h->edges[e1].len; ++k) first_col[h->newoff[e1] + k] = f;
    }
    for (int k = 0; k < ng; k += CHOL_NB) {
      const int nb = std::min(CHOL_NB, ng - k);
      int rend = k + nb, jb = k;
      for (int i = k; i < ng; ++i) if (first_col[i] < k + nb) rend = i + 1;
      for (int i = k; i < k + nb; ++i) jb = std::min(jb, first_col[i]);
      h->chol_rend.push_back(rend);
      h->chol_jbeg.push_back(jb);
    }
  }

  // ---- sizes ----
  h->ld = round_up(std::max(msmax, 1), 32);
  if (h->mixed && (size_t)((h->ld + 7) / 8) * 33 * sizeof(float) > 180 * 1024) {
    delete h;
    return fail(nullptr, ELM_DDM_ERR_ARG, "ELM_DDM_FLAG_MIXED: too many rows per subdomain for the FP32 panels");
  }
  h->mgmax = mgmax;
  h->mgld = round_up(std::max(mgmax, 1), 32);
  h->ncap = n + mgmax;
  h->nblk = (n + QR_NB - 1) / QR_NB;
  h->kstride = (long long)h->ld * h->ncap;
  h->mfld = round_up(std::max(h->mfmax, 1), 32);
  h->astride = (long long)h->mfld * n;
  h->mstride = (long long)std::max(h->mfld, h->mgld) * h->mgld;
  h->tstride = (long long)h->nblk * QR_NB * QR_NB;
  h->vstride = (long long)h->ld * QR_NBO;
  h->wstride = (long long)QR_NBO * h->ncap;
  // M blocks that two subdomains contribute to (a flux group and an edge both subdomains
  // of the group hold): summed once into Mdiag before the M^T M products
  std::map<std::pair<int, int>, size_t> msum_off;
  for (int f = 0; f < nfg; ++f)
    for (int e : fnbr[f]) {
      const FGroup& F = h->fgroups[f];
      const Edge& E = h->edges[e];
      int common = 0;
      for (int q = 0; q < 2; ++q)
        for (int p = 0; p < E.k; ++p) common += E.s[p] == F.s[q];
      if (common == 2) {
        msum_off[{f, e}] = h->mdiag_elems;
        h->mdiag_elems += (size_t)F.len * E.len;
      }
    }
  for (int s = 0; s < N; ++s)
    h->asm_bytes += 8.0 * ((double)h->ms_h[s] * (n + h->mg_h[s]) + (double)h->mf_h[s] * n);

  // ---- distinct coordinates of each subdomain's rows (factored activation) ----
  std::vector<double> txs, tys, tctr(2 * (size_t)N);
  std::vector<int> tnxy(2 * (size_t)N), trix;
  {
    std::vector<std::vector<double>> ux(N), uy(N);
    size_t total = 0, rows = 0;
    int nxmax = 0, nymax = 0;
    for (int s = 0; s < N; ++s) {
      for (int r = 0; r < h->mr_h[s]; ++r) {
        ux[s].push_back(xy[((size_t)s * m_max + r) * 2]);
        uy[s].push_back(xy[((size_t)s * m_max + r) * 2 + 1]);
      }
      for (auto* u : {&ux[s], &uy[s]}) {
        std::sort(u->begin(), u->end());
        u->erase(std::unique(u->begin(), u->end()), u->end());
      }
      nxmax = std::max(nxmax, (int)ux[s].size());
      nymax = std::max(nymax, (int)uy[s].size());
      total += ux[s].size() + uy[s].size();
      rows += h->mr_h[s];
    }
    // a table entry costs one exp, about what an entry's tanh costs, so the tables pay
    // when they hold fewer activations than K^s (the grids: about a tenth)
    h->use_tabs = !(desc->flags & ELM_DDM_FLAG_DIRECT_ASSEMBLY) && rows > 0 && total <= rows &&
                  nxmax < 65536 && nymax < 65536;
    if (h->use_tabs) {
      h->tabs.nxmax = nxmax;
      h->tabs.nymax = nymax;
      txs.assign((size_t)N * nxmax, 0.0);
      tys.assign((size_t)N * nymax, 0.0);
      trix.assign((size_t)N * m_max, 0);
      for (int s = 0; s < N; ++s) {
        tnxy[2 * s] = (int)ux[s].size();
        tnxy[2 * s + 1] = (int)uy[s].size();
        std::copy(ux[s].begin(), ux[s].end(), txs.begin() + (size_t)s * nxmax);
        std::copy(uy[s].begin(), uy[s].end(), tys.begin() + (size_t)s * nymax);
        tctr[2 * s] = ux[s].empty() ? 0.0 : 0.5 * (ux[s].front() + ux[s].back());
        tctr[2 * s + 1] = uy[s].empty() ? 0.0 : 0.5 * (uy[s].front() + uy[s].back());
        for (int r = 0; r < h->mr_h[s]; ++r) {
          const double x = xy[((size_t)s * m_max + r) * 2], y = xy[((size_t)s * m_max + r) * 2 + 1];
          const int ix = (int)(std::lower_bound(ux[s].begin(), ux[s].end(), x) - ux[s].begin());
          const int iy = (int)(std::lower_bound(uy[s].begin(), uy[s].end(), y) - uy[s].begin());
          trix[(size_t)s * m_max + r] = ix | (iy << 16);
        }
      }
    }
  }

  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaStreamCreateWithFlags(&h->st2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->evS, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->evB, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (h->st2) cudaStreamDestroy(h->st2);
      if (h->evS) cudaEventDestroy(h->evS);
      if (h->evB) cudaEventDestroy(h->evB);
      delete h;
      return fail(nullptr, ELM_DDM_ERR_CUDA, "setup: second stream");
    }
  }

  // ---- allocation ----
  bool ok = dev_alloc(h, &h->K, (size_t)N * h->kstride) &&
            dev_alloc(h, &h->Am, (size_t)N * h->astride) &&
            dev_alloc(h, &h->tau, (size_t)N * n) && dev_alloc(h, &h->T, (size_t)N * h->tstride) &&
            dev_alloc(h, &h->Vp, (size_t)N * h->vstride) &&
            dev_alloc(h, &h->Tab, (size_t)N * QR_NBO * QR_NBO) &&
            dev_alloc(h, &h->hlbuf, h->emulated ? (size_t)N * OZ_HL_TILE : (size_t)1) &&
            dev_alloc(h, &h->W1, (size_t)N * h->wstride) &&
            dev_alloc(h, &h->W2, (size_t)N * h->wstride) &&
            dev_alloc(h, &h->D, (size_t)N * h->mstride) &&
            dev_alloc(h, &h->M, (size_t)N * h->mstride) &&
            dev_alloc(h, &h->S, h->cg_only ? (size_t)1 : (size_t)ng * ng) &&
            dev_alloc(h, &h->Mdiag, h->mdiag_elems) &&
            dev_alloc(h, &h->cg_p, (size_t)max_rhs * std::max(ng, 1)) &&
            dev_alloc(h, &h->cg_q, (size_t)max_rhs * std::max(ng, 1)) &&
            dev_alloc(h, &h->cg_st, (size_t)max_rhs) &&
            dev_alloc(h, &h->sdinv, (size_t)std::max(ng, 1)) &&
            dev_alloc(h, &h->coef, h->op == ELM_DDM_OP_VARCOEF ? (size_t)N * m_max * 3 : (size_t)1) &&
            dev_alloc(h, &h->thW, (size_t)N * n * 2) && dev_alloc(h, &h->thb, (size_t)N * n) &&
            dev_alloc(h, &h->xy, (size_t)N * m_max * 2) &&
            dev_alloc(h, &h->nrm, (size_t)N * m_max * 2) &&
            dev_alloc(h, &h->X, (size_t)max_rhs * N * h->ld) &&
            dev_alloc(h, &h->gq, (size_t)max_rhs * N * h->mgld) &&
            dev_alloc(h, &h->hq, (size_t)max_rhs * N * h->mfld) &&
            dev_alloc(h, &h->zv, (size_t)max_rhs * N * h->mgld) &&
            dev_alloc(h, &h->rv, (size_t)max_rhs * ng) && dev_alloc(h, &h->hv, (size_t)max_rhs * h->n_flux) &&
            dev_alloc(h, &h->yv, (size_t)max_rhs * ng) && dev_alloc(h, &h->uv, (size_t)max_rhs * ng) &&
            dev_alloc(h, &h->cnt, (size_t)N * 3) && dev_alloc(h, &h->ms, (size_t)N) &&
            dev_alloc(h, &h->mg, (size_t)N) && dev_alloc(h, &h->dofmap, (size_t)ng * 2 * GRP_MAX) &&
            dev_alloc(h, &h->mf, (size_t)N) && dev_alloc(h, &h->fluxmap, (size_t)h->n_flux * 4) &&
            dev_alloc(h, &h->ffd, (size_t)N * h->mfld) &&
            (!h->explicit_flux || (dev_alloc(h, &h->frow, (size_t)N * h->mfld) &&
                                   dev_alloc(h, &h->fnrm, (size_t)N * h->mfld * 2))) &&
            dev_alloc(h, &h->ifc_dof, (size_t)N * h->mgld) && dev_alloc(h, &h->perm, (size_t)ng) &&
            dev_alloc(h, &h->cinv, (size_t)((ng + CHOL_NB - 1) / CHOL_NB + 1) * CHOL_NB * CHOL_NB) &&
            dev_alloc(h, &h->d_rend, h->chol_rend.size()) && dev_alloc(h, &h->d_jbeg, h->chol_jbeg.size()) &&
            dev_alloc(h, &h->cbar, (size_t)2) &&
            ((cst == 3 && !h->ridge) || dev_alloc(h, &h->nsub, (size_t)N)) &&
            dev_alloc(h, &h->colexp, h->emulated ? (size_t)N * h->ncap : (size_t)1) &&
            dev_alloc(h, &h->status, 1);
  std::vector<int> bj_len_h;
  std::vector<long long> bj_ioff_h;
  if (ok && h->bj) {
    long long tot = 0;
    for (const Edge& ed : h->edges) {
      bj_len_h.push_back(ed.len);
      bj_ioff_h.push_back(tot);
      tot += (long long)ed.len * ed.len;
    }
    const size_t ne = h->edges.size();
    ok = dev_alloc(h, &h->bj_off, std::max<size_t>(ne, 1)) && dev_alloc(h, &h->bj_len, std::max<size_t>(ne, 1)) &&
         dev_alloc(h, &h->bj_ioff, std::max<size_t>(ne, 1)) && dev_alloc(h, &h->bj_inv, (size_t)std::max(tot, 1ll)) &&
         dev_alloc(h, &h->cg_z, (size_t)max_rhs * std::max(ng, 1));
  }
  if (ok && h->mixed) {
    const size_t R = (size_t)max_rhs, ngs = (size_t)std::max(ng, 1);
    const size_t xn = R * N * h->ld, cn = R * N * n, gn = R * N * h->mgld;
    ok = dev_alloc(h, &h->K64, (size_t)N * h->ld * n) && dev_alloc(h, &h->A64, (size_t)N * h->astride) &&
         dev_alloc(h, &h->F64, xn) && dev_alloc(h, &h->cit, cn) && dev_alloc(h, &h->wit, cn) &&
         dev_alloc(h, &h->uit, R * ngs) && dev_alloc(h, &h->dcv, cn) && dev_alloc(h, &h->dwv, cn) &&
         dev_alloc(h, &h->ebuf, xn) && dev_alloc(h, &h->kwbuf, xn) && dev_alloc(h, &h->zb, gn) &&
         dev_alloc(h, &h->r1b, cn) && dev_alloc(h, &h->r3b, cn) && dev_alloc(h, &h->r13b, cn) &&
         dev_alloc(h, &h->tb, cn) && dev_alloc(h, &h->Pb, 2 * xn) && dev_alloc(h, &h->Acl, gn) &&
         dev_alloc(h, &h->Acg, R * ngs) && dev_alloc(h, &h->zero_ng, R * ngs) &&
         dev_alloc(h, &h->gq2, 2 * gn) && dev_alloc(h, &h->hq2, 2 * gn) && dev_alloc(h, &h->nrmb, 4 * R);
    if (ok) ok = cudaMemset(h->zero_ng, 0, R * ngs * sizeof(double)) == cudaSuccess;
  }
  if (ok && h->use_tabs) {
    const AsmTables& t = h->tabs;
    ok = dev_alloc(h, &h->tab_xs, (size_t)N * t.nxmax) && dev_alloc(h, &h->tab_ys, (size_t)N * t.nymax) &&
         dev_alloc(h, &h->tab_ctr, (size_t)N * 2) && dev_alloc(h, &h->tab_nxy, (size_t)N * 2) &&
         dev_alloc(h, &h->tab_rix, (size_t)N * m_max) &&
         dev_alloc(h, &h->tab_Tx, (size_t)N * n * t.nxmax) && dev_alloc(h, &h->tab_Ty, (size_t)N * n * t.nymax);
    h->tabs.xs = h->tab_xs; h->tabs.ys = h->tab_ys; h->tabs.ctr = h->tab_ctr; h->tabs.nxy = h->tab_nxy;
    h->tabs.rix = h->tab_rix; h->tabs.Tx = h->tab_Tx; h->tabs.Ty = h->tab_Ty;
  }
  if (!ok) {
    free_all(h);
    delete h;
    return fail(nullptr, ELM_DDM_ERR_OOM, "device allocation failed");
  }
  // Split workspace (tensor-core FP64 products): per subdomain the digit tiles of the
  // trailing block A2^T, of V^T, of V and of W2^T, then for the Cholesky the panel L21 as
  // both operands.  Each region is 256-byte aligned.
  const int n2max = h->ncap - std::min(QR_NB, n), mpmax = msmax;
  int restmax = 0;
  for (int k = 0, st = 0; k < ng; k += CHOL_NB, ++st)
    restmax = std::max(restmax, h->chol_rend[st] - k - std::min(CHOL_NB, ng - k));
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  // (A2^T is split inside the fused product kernel: only its row exponents are stored)
  const size_t s1 = 0, e1 = 0;  // (unused region)
  // (QR operands for an outer block of up to min(QR_NBO, n) reflectors)
  const int nbo = std::min(QR_NBO, round_up(n, QR_NB));
  const size_t s2 = al(oz_split_elems(nbo, mpmax, 128) * 2), e2 = al((size_t)nbo * 4);
  const size_t s3 = al(oz_split_elems(mpmax, nbo, 128) * 2), e3 = al((size_t)mpmax * 4);
  const size_t s4 = al(oz_split_elems(n2max, nbo, 64) * 2), e4 = al((size_t)n2max * 4);  // (64-row tiles)
  // D_s / M_s products: Q_G as both operands, Y as the left operand (K = n_N)
  const int mgm = std::max(mgmax, 1);
  const size_t s5 = al(oz_split_elems(mgm, n, 128) * 2), e5 = al((size_t)mgm * 4);
  const size_t s6 = al(oz_split_elems(mgm, n, 32) * 2), e6 = al((size_t)mgm * 4);
  const int mfm = std::max(h->mfmax, 1);  // Y_s rows (rows of A^s)
  const size_t s7 = al(oz_split_elems(mfm, n, 128) * 2), e7 = al((size_t)mfm * 4);
  // Y = A R^{-1} updates: the 64-row block of R to the right of the diagonal (Y_b reuses s7)
  const size_t s8 = al(oz_split_elems(n, 64, 32) * 2), e8 = al((size_t)n * 4);
  // W2^T = W1^T T per QR panel: W1^T (rows = trailing columns) and T^T
  const size_t s9 = al(oz_split_elems(n2max, nbo, 128) * 2), e9 = al((size_t)n2max * 4);
  const size_t s10 = al(oz_split_elems(nbo, nbo, 32) * 2), e10 = al((size_t)nbo * 4);
  const size_t per_sub = s1 + e1 + s2 + e2 + s3 + e3 + s4 + e4 + s5 + e5 + s6 + e6 + s7 + e7 + s8 + e8 +
                         s9 + e9 + s10 + e10;
  const size_t c1 = al(oz_split_elems(std::max(restmax, 1), CHOL_NB, 128) * 2);
  const size_t c2 = al(oz_split_elems(std::max(restmax, 1), CHOL_NB, 32) * 2);
  const size_t ce = al((size_t)std::max(restmax, 1) * 4);
  if (h->emulated) {
    char* base = nullptr;
    if (!dev_alloc(h, &base, per_sub * N + 2 * (c1 + c2 + 2 * ce))) {
      free_all(h);
      delete h;
      return fail(nullptr, ELM_DDM_ERR_OOM, "device allocation failed (split workspace)");
    }
    h->sp_buf = base;
  }
  auto sub_region = [&](int s, int which) -> char* {
    const size_t sz[20] = {s1, e1, s2, e2, s3, e3, s4, e4, s5, e5, s6, e6, s7, e7, s8, e8, s9, e9, s10, e10};
    size_t off = 0;
    for (int i = 0; i < which; ++i) off += sz[i];
    return (char*)h->sp_buf + (size_t)s * per_sub + off;
  };
  char* chol_region = (char*)h->sp_buf + per_sub * N;
  h->creg = chol_region;
  h->creg_c1 = c1;
  h->creg_c2 = c2;
  h->creg_ce = ce;

  // ---- geometry tables ----
  // dofmap: the (subdomain, interface row) pairs of every unknown in internal order
  // (subdomain -1 ends a list shorter than GRP_MAX); fluxmap: the two (subdomain, A-row)
  // pairs of every flux condition in internal order (the unknowns' order without explicit
  // flux rows, so that h lines up with u_Gamma there)
  std::vector<int> dofmap((size_t)ng * 2 * GRP_MAX, -1), ifc((size_t)N * h->mgld, -1);
  for (int g = 0; g < ng; ++g) {
    const size_t gi = (size_t)h->perm_h[g];
    for (size_t q = 0; q < owners[g].size(); ++q) {
      dofmap[2 * GRP_MAX * gi + 2 * q] = owners[g][q].first;
      dofmap[2 * GRP_MAX * gi + 2 * q + 1] = owners[g][q].second;
    }
  }
  for (int s = 0; s < N; ++s) {
    const int r0 = h->cnt_h[3 * s] + h->cnt_h[3 * s + 1];
    for (int i = 0; i < h->mg_h[s]; ++i)
      ifc[(size_t)s * h->mgld + i] = h->perm_h[dof[(size_t)s * m_max + r0 + i]];
  }
  auto fint = [&](int c) { return h->explicit_flux ? c : h->perm_h[c]; };
  std::vector<int> fluxmap((size_t)h->n_flux * 4), ffd((size_t)N * h->mfld, 0), frow_d;
  std::vector<double> fnrm_d;
  for (int c = 0; c < h->n_flux; ++c)
    for (int q = 0; q < 2; ++q) {
      fluxmap[4 * (size_t)fint(c) + 2 * q] = fown[c][q].first;
      fluxmap[4 * (size_t)fint(c) + 2 * q + 1] = fown[c][q].second;
    }
  for (int s = 0; s < N; ++s)
    for (int f = 0; f < h->mf_h[s]; ++f) ffd[(size_t)s * h->mfld + f] = fint(fd_h[s][f]);
  if (h->explicit_flux) {
    frow_d.assign((size_t)N * h->mfld, 0);
    fnrm_d.assign((size_t)N * h->mfld * 2, 0.0);
    for (int s = 0; s < N; ++s) {
      const int r0 = h->cnt_h[3 * s] + h->cnt_h[3 * s + 1];
      for (int f = 0; f < h->mf_h[s]; ++f) {
        frow_d[(size_t)s * h->mfld + f] = r0 + fr_h[s][f];
        fnrm_d[2 * ((size_t)s * h->mfld + f)] = fn_h[s][2 * f];
        fnrm_d[2 * ((size_t)s * h->mfld + f) + 1] = fn_h[s][2 * f + 1];
      }
    }
  }

  // ---- launch plans ----
  std::vector<GemmDesc> gds;
  std::vector<AddDesc> ads;
  auto add_gemm_rec = [&](std::vector<LaunchRec>& recs, const std::vector<GemmDesc>& batch, bool ta,
                          bool tb, double alpha, double beta, int flags) {
    bool skinny = !(flags & GEMM_LOWER);
    for (const GemmDesc& d : batch) skinny = skinny && d.m <= 32;
    if (skinny) flags |= GEMM_SKINNY;
    LaunchRec L{0, (int)gds.size(), 0, 0, ta, tb, alpha, beta, flags, 0.0, 0};
    for (const GemmDesc& d : batch) {
      if (d.m <= 0 || d.n <= 0) continue;
      gds.push_back(d);
      L.count++;
      L.max_tiles = std::max(L.max_tiles, gemm_tiles(d.m, d.n, flags));
      L.flops += (flags & GEMM_LOWER) ? (double)d.m * (d.m + 1) * d.k : 2.0 * d.m * d.n * d.k;
    }
    recs.push_back(L);
  };
  auto add_add_rec = [&](std::vector<LaunchRec>& recs, const std::vector<AddDesc>& batch) {
    LaunchRec L{1, (int)ads.size(), 0, 0, false, false, 0, 0, 0, 0.0, 0};
    for (const AddDesc& d : batch) {
      if (d.rows <= 0 || d.cols <= 0) continue;
      ads.push_back(d);
      L.count++;
      L.max_tiles = std::max(L.max_tiles, d.rows * d.cols);
    }
    recs.push_back(L);
  };
  const int ld = h->ld;
  // QR trailing updates, panel b: W1 = V^T A2, W2 = T^T W1, A2 -= V W2.  With the
  // tensor-core path, W1^T = A2^T V and A2 -= V W2 are digit-split products and only the
  // small T^T W1 stays on the FP64 pipe.
  std::vector<SplitDesc> sds;
  std::vector<OzDesc> ods;
  std::vector<int4> uts;
  auto add_split_rec = [&](std::vector<LaunchRec>& recs, const std::vector<SplitDesc>& batch,
                           const char* name) {
    LaunchRec L{2, (int)sds.size(), 0, 0, false, false, 0, 0, 0, 0.0, 0};
    L.name = name;
    for (const SplitDesc& d : batch) {
      if (d.R <= 0 || d.K <= 0) continue;
      sds.push_back(d);
      L.count++;
      L.nt = std::max(L.nt, oz_rowexp_blocks(d));
      if (!d.tiles) {  // row exponents only
        L.bytes += 8.0 * d.R * d.K;
        continue;
      }
      L.bytes += (8.0 + 2.0 * 7) * d.R * d.K;  // FP64 read once, 7 BF16 digit planes written
      L.max_tiles = std::max(L.max_tiles, (d.R + d.row_tile - 1) / d.row_tile * ((d.K + 31) / 32));
    }
    recs.push_back(L);
  };
  auto add_oz_rec = [&](std::vector<LaunchRec>& recs, const std::vector<OzDesc>& batch, int nt,
                        double alpha, double beta, int flags, const char* name) {
    // nt == 0: persistent K <= 64 kernel over a table of 128 x 32 tiles (max_tiles = its size)
    LaunchRec L{nt == 0 ? 4 : 3, (int)ods.size(), 0, 0, false, false, alpha, beta, flags, 0.0, nt};
    L.name = name;
    for (const OzDesc& d : batch) {
      if (d.M <= 0 || d.N <= 0) continue;
      if (nt != 0) L.max_tiles = std::max(L.max_tiles, oz_tiles(d.M, d.N, nt));
      ods.push_back(d);
      L.count++;
      const bool low = (flags & GEMM_LOWER) != 0;
      L.flops += low ? (double)d.M * (d.M + 1) * d.K : 2.0 * d.M * d.N * d.K;
      // FP64 operands read once, C written (and read when beta != 0)
      const double cbytes = (beta != 0.0 ? 16.0 : 8.0) * (low ? 0.5 * d.M * (d.M + 1.0) : (double)d.M * d.N);
      L.bytes += 8.0 * ((double)d.M * d.K + (low ? 0.0 : (double)d.N * d.K)) + cbytes;
    }
    if (nt == 0 && L.count > 0) {
      L.toff = (int)uts.size();
      L.max_tiles = oz_upd_tile_table(ods.data() + L.off, L.count, flags, nullptr);
      uts.resize(uts.size() + L.max_tiles);
      oz_upd_tile_table(ods.data() + L.off, L.count, flags, uts.data() + L.toff);
    }
    recs.push_back(L);
  };
  // C += alpha A B^T (alpha = +-1) over 128 x 64 tiles: the wide persistent update
  auto add_updw_rec = [&](std::vector<LaunchRec>& recs, const std::vector<OzDesc>& batch, double alpha,
                          const char* name) {
    LaunchRec L{10, (int)ods.size(), 0, 0, false, false, alpha, 1.0, 0, 0.0, 64};
    L.name = name;
    for (const OzDesc& d : batch) {
      if (d.M <= 0 || d.N <= 0) continue;
      ods.push_back(d);
      L.count++;
      L.flops += 2.0 * d.M * d.N * d.K;
      L.bytes += 8.0 * ((double)d.M * d.K + (double)d.N * d.K) + 16.0 * d.M * d.N;
    }
    if (L.count > 0) {
      L.toff = (int)uts.size();
      L.max_tiles = oz_upd_tile_table(ods.data() + L.off, L.count, 0, nullptr, UPW_TILE_N);
      uts.resize(uts.size() + L.max_tiles);
      oz_upd_tile_table(ods.data() + L.off, L.count, 0, uts.data() + L.toff, UPW_TILE_N);
    }
    recs.push_back(L);
  };
  // C = A B^T with A = FP64 operand split inside the kernel (N <= 32, beta = 0); ksplit > 1:
  // K split over that many CTAs per tile (one 128-row tile, the descriptors' hl set)
  auto add_fa_rec = [&](std::vector<LaunchRec>& recs, const std::vector<OzDesc>& batch, const char* name,
                        int ksplit = 1) {
    LaunchRec L{5, (int)ods.size(), 0, 0, false, false, 1.0, 0.0, 0, 0.0, ksplit};
    L.name = name;
    for (const OzDesc& d : batch) {
      if (d.M <= 0 || d.N <= 0) continue;
      ods.push_back(d);
      L.count++;
      L.max_tiles = std::max(L.max_tiles, (d.M + 127) / 128);
      L.flops += 2.0 * d.M * d.N * d.K;
      L.bytes += 8.0 * ((double)d.M * d.K + (double)d.N * d.K + (double)d.M * d.N);
    }
    recs.push_back(L);
  };
  // C = A B^T with B = FP64 operand split inside the kernel (M <= 128, beta = 0)
  // (64 rows of B per CTA when some descriptor has that many: N = 64 MMAs)
  auto add_fb_rec = [&](std::vector<LaunchRec>& recs, const std::vector<OzDesc>& batch, const char* name) {
    int nbc = 32;
    for (const OzDesc& d : batch) if (d.N >= 64) nbc = 64;
    LaunchRec L{9, (int)ods.size(), 0, 0, false, false, 1.0, 0.0, 0, 0.0, nbc};
    L.name = name;
    for (const OzDesc& d : batch) {
      if (d.M <= 0 || d.N <= 0) continue;
      ods.push_back(d);
      L.count++;
      L.max_tiles = std::max(L.max_tiles, (d.N + nbc - 1) / nbc);
      L.flops += 2.0 * d.M * d.N * d.K;
      L.bytes += 8.0 * ((double)d.M * d.K + (double)d.N * d.K + (double)d.M * d.N);
    }
    recs.push_back(L);
  };
  // the inner steps' W1 products are one 128-row tile per subdomain: split their K over
  // the CTAs the GPU has beyond one per subdomain (at most 4)
  const int inner_ksplit = h->emulated ? std::max(1, std::min(4, h->sms / std::max(N, 1))) : 1;
  for (int b = 0; b < h->nblk; ++b) {
    const int k0 = b * QR_NB, nbe = std::min(QR_NB, n - k0);
    double pf = 0.0, pb = 0.0;
    for (int s = 0; s < N; ++s) {
      const double mp = std::max(0, h->ms_h[s] - k0);
      pf += 2.0 * mp * nbe * nbe - 2.0 * nbe * (double)nbe * nbe / 3.0;
      pb += 2.0 * 8.0 * mp * nbe;  // the panel read and written once
    }
    h->panel_flops.push_back(pf);
    h->panel_bytes.push_back(pb);
    h->qr_first.push_back((int)h->qr_recs.size());
    LaunchRec FT{7, b, 1, 0, false, false, 0.0, 0.0, 0, 0.0, nbe};
    FT.name = "form_t";
    if (!h->emulated) {
      // FP64 back end, one level: W1 = V^T [P | A2] (P the panel's stored columns, whose
      // rows give v_l^T v_j for l < j exactly: what T needs, launch_form_t), then
      // W2 = T^T W1 and A2 -= V W2 on the trailing columns
      h->panel_vcol.push_back(0);
      h->panel_vrow0.push_back(k0);
      std::vector<GemmDesc> g1, g2, g3;
      for (int s = 0; s < N; ++s) {
        const int n2 = n + h->mg_h[s] - (k0 + nbe), mp = h->ms_h[s] - k0;
        if (mp <= 0) continue;
        double* Ks = h->K + (size_t)s * h->kstride;
        const double* V = h->Vp + (size_t)s * h->vstride + k0;
        double* PA2 = Ks + k0 + (size_t)k0 * ld;
        double* w1 = h->W1 + (size_t)s * h->wstride;
        double* w2 = h->W2 + (size_t)s * h->wstride;
        const double* Tb = h->T + (size_t)s * h->tstride + (size_t)b * QR_NB * QR_NB;
        g1.push_back({V, PA2, w1, nbe, n2 + nbe, mp, ld, ld, QR_NB});
        if (n2 > 0) {
          g2.push_back({Tb, w1 + (size_t)nbe * QR_NB, w2, nbe, n2, nbe, QR_NB, QR_NB, QR_NB});
          g3.push_back({V, w2, PA2 + (size_t)nbe * ld, mp, n2, nbe, ld, QR_NB, ld});
        }
      }
      add_gemm_rec(h->qr_recs, g1, true, false, 1.0, 0.0, 0);
      h->qr_recs.push_back(FT);
      add_gemm_rec(h->qr_recs, g2, true, false, 1.0, 0.0, 0);
      add_gemm_rec(h->qr_recs, g3, false, false, -1.0, 1.0, 0);
      continue;
    }
    // Tensor-core back end, two levels.  Panel b is panel j of the outer block of wo columns
    // from k0o; its explicit reflectors go to column j * 32 of Vp, with rows k0o .. k0 - 1
    // zeroed, so that columns 0 .. wo - 1 of Vp from row k0o are the block's V.
    const int k0o = k0 / QR_NBO * QR_NBO, wo = std::min(QR_NBO, n - k0o);
    const int np = (wo + QR_NB - 1) / QR_NB, j = (k0 - k0o) / QR_NB;
    h->panel_vcol.push_back(j * QR_NB);
    h->panel_vrow0.push_back(k0o);
    std::vector<SplitDesc> sp1, sp3, spt;
    std::vector<OzDesc> o1, o3, ot;
    if (j < np - 1) {
      // Inner step: the rest of the outer block (n2i columns) takes this panel's reflectors.
      // W1^T = [V | A2]^T V (A split inside the product: the first nbe rows are the Gram
      // rows v_l^T v_j that T needs, from the explicit reflectors (|v| <= 1 with a unit
      // diagonal, so the digit split keeps them to FP64 accuracy, where the stored panel
      // columns would be truncated relative to R's entries); the rows of A2^T take the
      // exponent bounds of their columns' original norms, which no orthogonal update of
      // the column can exceed), T from the Gram rows, W2^T = W1^T T, A2 -= V W2 (K = 32).
      const int n2i = k0o + wo - (k0 + nbe);
      for (int s = 0; s < N; ++s) {
        const int mp = h->ms_h[s] - k0;
        if (mp <= 0) continue;
        double* Ks = h->K + (size_t)s * h->kstride;
        const double* V = h->Vp + (size_t)s * h->vstride + (size_t)j * QR_NB * ld + k0;
        double* PA2 = Ks + k0 + (size_t)k0 * ld;           // [P | A2], n2i + nbe columns
        double* A2 = PA2 + (size_t)nbe * ld;
        double* w1 = h->W1 + (size_t)s * h->wstride;       // W1^T, row stride 32
        double* w1t = w1 + (size_t)nbe * QR_NB;
        double* w2 = h->W2 + (size_t)s * h->wstride;
        const double* Tb = h->T + (size_t)s * h->tstride + (size_t)b * QR_NB * QR_NB;
        void* t2 = sub_region(s, 2); int* x2 = (int*)sub_region(s, 3);
        void* t3 = sub_region(s, 4); int* x3 = (int*)sub_region(s, 5);
        void* t4 = sub_region(s, 6); int* x4 = (int*)sub_region(s, 7);
        void* t9 = sub_region(s, 16); int* x9 = (int*)sub_region(s, 17);
        void* t10 = sub_region(s, 18); int* x10 = (int*)sub_region(s, 19);
        sp1.push_back({V, ld, 1, nbe, mp, x2, t2, 32});              // V^T: rows = panel columns
        // V itself (the update's left operand) is ready once the panel is: split in the
        // same launch as V^T rather than after the W1 product
        sp1.push_back({V, 1, ld, mp, nbe, x3, t3, 128});             // V: rows = matrix rows
        OzDesc ow{PA2, h->colexp + (size_t)s * h->ncap + k0, t2, x2, w1, QR_NB, 1, n2i + nbe, nbe, mp, 0, ld};
        ow.At2 = V;   // rows i < nbe at V + i * ld, rows i >= nbe at PA2 + i * ld = A2
        ow.Ae2 = x2;
        ow.lead = nbe;
        if (inner_ksplit > 1) ow.hl = h->hlbuf + (size_t)s * OZ_HL_TILE;
        o1.push_back(ow);
        // W2^T = W1^T T: A = W1^T (row r = column r of A2, 32 contiguous values), B = T^T
        // (row i = column i of the column-major T)
        spt.push_back({w1t, QR_NB, 1, n2i, nbe, x9, t9, 128});
        spt.push_back({Tb, QR_NB, 1, nbe, nbe, x10, t10, 32});
        ot.push_back({t9, x9, t10, x10, w2, QR_NB, 1, n2i, nbe, nbe, 0});
        sp3.push_back({w2, QR_NB, 1, n2i, nbe, x4, t4, 32});  // W2^T: rows = columns of A2
        o3.push_back({t3, x3, t4, x4, A2, 1, ld, mp, n2i, nbe, 0});
      }
      FT.name = "form_t_in";
      add_split_rec(h->qr_recs, sp1, "split_qr_in");
      add_fa_rec(h->qr_recs, o1, "oz_qr_w_in", inner_ksplit);
      h->qr_recs.push_back(FT);
      add_split_rec(h->qr_recs, spt, "split_qr_in");
      add_oz_rec(h->qr_recs, ot, 0, 1.0, 0.0, 0, "oz_qr_t_in");
      add_split_rec(h->qr_recs, sp3, "split_qr_in");
      add_oz_rec(h->qr_recs, o3, 0, -1.0, 1.0, 0, "oz_qr_update_in");
      continue;
    }
    // Outer step, after the block's last panel: W1 = V_o^T [V_o | A2] over the trailing
    // columns, as one product whose A operand is V_o^T (all wo reflectors, split once) and
    // whose B operand, the block's explicit reflectors then the trailing columns, is split
    // inside the kernel (each trailing column once per outer block); its first wo columns
    // are the block's Gram matrix.  Then T_o of the whole block (its last diagonal 32-block
    // is this panel's T), W2^T = W1^T T_o and A2 -= V_o W2 (K = wo).
    for (int s = 0; s < N; ++s) {
      const int mpo = h->ms_h[s] - k0o, n2o = n + h->mg_h[s] - (k0o + wo);
      if (mpo <= 0) continue;
      double* Ks = h->K + (size_t)s * h->kstride;
      const double* Vo = h->Vp + (size_t)s * h->vstride + k0o;  // wo columns from row k0o
      double* Ao = Ks + k0o + (size_t)k0o * ld;                  // [P_o | A2], wo + n2o columns
      double* A2 = Ao + (size_t)wo * ld;
      double* w1 = h->W1 + (size_t)s * h->wstride;               // W1^T, row stride QR_NBO
      double* w1t = w1 + (size_t)wo * QR_NBO;
      double* w2 = h->W2 + (size_t)s * h->wstride;
      const double* To = h->Tab + (size_t)s * QR_NBO * QR_NBO;
      void* t2 = sub_region(s, 2); int* x2 = (int*)sub_region(s, 3);
      void* t3 = sub_region(s, 4); int* x3 = (int*)sub_region(s, 5);
      void* t4 = sub_region(s, 6); int* x4 = (int*)sub_region(s, 7);
      void* t9 = sub_region(s, 16); int* x9 = (int*)sub_region(s, 17);
      void* t10 = sub_region(s, 18); int* x10 = (int*)sub_region(s, 19);
      sp1.push_back({Vo, ld, 1, wo, mpo, x2, t2, 128});            // V_o^T: rows = block columns
      if (n2o > 0) sp1.push_back({Vo, 1, ld, mpo, wo, x3, t3, 128});  // V_o: rows = matrix rows
      // C[i, j] = W1^T[j][i] at w1 + j * QR_NBO + i
      OzDesc ob{t2, x2, Ao, h->colexp + (size_t)s * h->ncap + k0o, w1, 1, QR_NBO, wo, wo + n2o, mpo, 0, ld};
      ob.At2 = Vo;  // B rows j < wo at Vo + j * ld (explicit reflectors), j >= wo at Ao + j * ld = A2
      ob.Ae2 = x2;
      ob.lead = wo;
      o1.push_back(ob);
      if (n2o <= 0) continue;
      spt.push_back({w1t, QR_NBO, 1, n2o, wo, x9, t9, 128});
      spt.push_back({To, QR_NBO, 1, wo, wo, x10, t10, 32});
      ot.push_back({t9, x9, t10, x10, w2, QR_NBO, 1, n2o, wo, wo, 0});
      sp3.push_back({w2, QR_NBO, 1, n2o, wo, x4, t4, 64});  // 64-row tiles for the wide update
      o3.push_back({t3, x3, t4, x4, A2, 1, ld, mpo, n2o, wo, 0});
    }
    LaunchRec FW{8, b, 1, 0, false, false, 0.0, 0.0, 0, 0.0, wo};
    FW.toff = k0o;
    FW.name = "form_t";
    add_split_rec(h->qr_recs, sp1, "split_qr_w");
    add_fb_rec(h->qr_recs, o1, "oz_qr_w");
    h->qr_recs.push_back(FW);
    add_split_rec(h->qr_recs, spt, "split_qr_t");
    add_oz_rec(h->qr_recs, ot, 0, 1.0, 0.0, 0, "oz_qr_t");
    add_split_rec(h->qr_recs, sp3, "split_qr_update");
    add_updw_rec(h->qr_recs, o3, -1.0, "oz_qr_update");
  }
  h->qr_first.push_back((int)h->qr_recs.size());
  // Y = A R^{-1}, blocked by 64 columns: substitution on the diagonal block of R, then the
  // columns to its right take Y_b R[b, >b] off as a digit-split product (K = 64).
  if (h->emulated && h->mfmax > 0) {
    for (int c0 = 0; c0 < n; c0 += 64) {
      const int nbe = std::min(64, n - c0), nrest = n - c0 - nbe;
      LaunchRec D{6, c0, 1, 0, false, false, 0.0, 0.0, 0, 0.0, nbe};
      for (int s = 0; s < N; ++s) D.flops += (double)h->mf_h[s] * nbe * nbe;
      D.name = "trsm_y";
      h->ty_recs.push_back(D);
      if (nrest <= 0) continue;
      std::vector<SplitDesc> sp;
      std::vector<OzDesc> od;
      for (int s = 0; s < N; ++s) {
        const int mfs = h->mf_h[s];
        if (mfs == 0) continue;
        double* Ys = h->Am + (size_t)s * h->astride;
        const double* Rb = h->K + (size_t)s * h->kstride + c0 + (size_t)(c0 + nbe) * ld;
        void* ty = sub_region(s, 12); int* xy = (int*)sub_region(s, 13);
        void* tr = sub_region(s, 14); int* xr = (int*)sub_region(s, 15);
        sp.push_back({Ys + (size_t)c0 * h->mfld, 1, h->mfld, mfs, nbe, xy, ty, 128});
        sp.push_back({Rb, ld, 1, nrest, nbe, xr, tr, 32});
        od.push_back({ty, xy, tr, xr, Ys + (size_t)(c0 + nbe) * h->mfld, 1, h->mfld, mfs, nrest, nbe, 0});
      }
      add_split_rec(h->ty_recs, sp, "split_trsm_y");
      add_oz_rec(h->ty_recs, od, 0, -1.0, 1.0, 0, "oz_trsm_y");
    }
  }
  // D_s = I - (Q_G^T)^T Q_G^T and M_s = -Y_s Q_G^T (K = n_N): tensor-core products whose
  // left operands (Q_G, Y_s) are split in 128-row tiles and whose right operand, the columns
  // of Q_G^T, is split inside the B-split kernel (64 columns per CTA, one descriptor per left
  // row tile), or FP64 GEMMs.
  {
    std::vector<GemmDesc> gD, gM;
    std::vector<SplitDesc> sp;
    std::vector<OzDesc> oD, oM;
    for (int s = 0; s < N; ++s) {
      const int mgs = h->mg_h[s];
      if (mgs == 0) continue;
      const int mfs = h->mf_h[s];
      const double* QGt = h->K + (size_t)s * h->kstride + (size_t)n * ld;
      double* Ds = h->D + (size_t)s * h->mstride;
      double* Ms = h->M + (size_t)s * h->mstride;
      const double* Ys = h->Am + (size_t)s * h->astride;
      gD.push_back({QGt, QGt, Ds, mgs, mgs, n, ld, ld, h->mgld});
      if (mfs > 0) gM.push_back({Ys, QGt, Ms, mfs, mgs, n, h->mfld, ld, h->mfld});
      if (h->emulated) {
        void* t5 = sub_region(s, 8); int* x5 = (int*)sub_region(s, 9);
        int* x6 = (int*)sub_region(s, 11);
        void* t7 = sub_region(s, 12); int* x7 = (int*)sub_region(s, 13);
        sp.push_back({QGt, ld, 1, mgs, n, x5, t5, 128});        // Q_G, left operand
        sp.push_back({QGt, ld, 1, mgs, n, x6, nullptr, 128});   // Q_G^T columns: exponent bounds only
        if (mfs > 0) sp.push_back({Ys, 1, h->mfld, mfs, n, x7, t7, 128});  // Y_s, left operand
        const size_t tile = oz_split_elems(128, n, 128) * 2;    // bytes of one 128-row tile's planes
        for (int r0 = 0; r0 < mgs; r0 += 128) {
          OzDesc od{(char*)t5 + (size_t)(r0 / 128) * tile, x5 + r0, QGt, x6, Ds + r0, 1, h->mgld,
                    std::min(128, mgs - r0), mgs, n, 3, ld};  // -(Q_G Q_G^T) + I
          od.lower_off = r0;
          oD.push_back(od);
        }
        for (int r0 = 0; r0 < mfs; r0 += 128)
          oM.push_back({(char*)t7 + (size_t)(r0 / 128) * tile, x7 + r0, QGt, x6, Ms + r0, 1, h->mfld,
                        std::min(128, mfs - r0), mgs, n, 1, ld});  // -(Y_s Q_G^T)
      }
    }
    if (h->emulated) {
      add_split_rec(h->dm_recs, sp, "split_dm");
      std::vector<OzDesc> odm(oD);
      odm.insert(odm.end(), oM.begin(), oM.end());
      add_fb_rec(h->dm_recs, odm, "oz_dm");
    } else {
      add_gemm_rec(h->dm_recs, gD, true, false, -1.0, 0.0, GEMM_ADD_IDENTITY);
      add_gemm_rec(h->dm_recs, gM, false, false, -1.0, 0.0, 0);
    }
  }
  // Schur matrix (lower edge blocks, internal order): S[e1,e2] = sum of D blocks +
  // sum_f Mblk(f,e1)^T Mblk(f,e2) over the flux groups f, each output block written once per
  // round.  Not formed at all when the interface problem is solved by CG.
  if (ng > 0 && !h->cg_only) {
    auto local = [&](int e, int s) -> int {  // first interface row of edge e in subdomain s, or -1
      const Edge& E = h->edges[e];
      for (int q = 0; q < E.k; ++q)
        if (E.s[q] == s) return E.i[q];
      return -1;
    };
    // Mdiag[(f, e)] = M_{s0}[f, e] + M_{s1}[f, e] where both subdomains of flux group f hold
    // edge e (without explicit flux rows: f = e)
    for (int q = 0; q < 2; ++q) {
      std::vector<AddDesc> batch;
      for (const auto& kv : msum_off) {
        const FGroup& F = h->fgroups[kv.first.first];
        const int e = kv.first.second, s = F.s[q];
        const double* src = h->M + (size_t)s * h->mstride + F.i[q] + (size_t)local(e, s) * h->mfld;
        batch.push_back({src, h->Mdiag + kv.second, F.len, h->edges[e].len, h->mfld, F.len});
      }
      add_add_rec(h->s_recs, batch);
    }
    // the block of M in flux group f's rows and edge e's columns
    auto mblk = [&](int f, int e, const double** p, int* ldp) {
      const auto it = msum_off.find({f, e});
      if (it != msum_off.end()) { *p = h->Mdiag + it->second; *ldp = h->fgroups[f].len; return; }
      const FGroup& F = h->fgroups[f];
      for (int q = 0; q < 2; ++q) {
        const int s = F.s[q], l2 = local(e, s);
        if (l2 >= 0) {
          *p = h->M + (size_t)s * h->mstride + F.i[q] + (size_t)l2 * h->mfld;
          *ldp = h->mfld;
          return;
        }
      }
      *p = nullptr;
    };
    std::vector<std::vector<AddDesc>> drounds;
    std::vector<std::vector<GemmDesc>> mrounds;
    for (int e1 = 0; e1 < ne; ++e1) {
      const Edge& E1 = h->edges[e1];
      for (int e2 : spat[e1]) {
        if (h->newoff[e2] > h->newoff[e1]) continue;
        const Edge& E2 = h->edges[e2];
        double* dst = h->S + h->newoff[e1] + (size_t)h->newoff[e2] * ng;
        int r = 0;
        for (int q = 0; q < E1.k; ++q) {
          const int s = E1.s[q], l2 = local(e2, s);
          if (l2 < 0) continue;
          if ((int)drounds.size() <= r) drounds.emplace_back();
          drounds[r++].push_back({h->D + (size_t)s * h->mstride + E1.i[q] + (size_t)l2 * h->mgld, dst,
                                  E1.len, E2.len, h->mgld, ng});
        }
        r = 0;
        for (int f : efl[e1]) {
          if (!std::binary_search(fnbr[f].begin(), fnbr[f].end(), e2)) continue;
          const double *pa, *pb;
          int la, lb;
          mblk(f, e1, &pa, &la);
          mblk(f, e2, &pb, &lb);
          if (!pa || !pb) continue;
          if ((int)mrounds.size() <= r) mrounds.emplace_back();
          mrounds[r++].push_back({pa, pb, dst, E1.len, E2.len, h->fgroups[f].len, la, lb, ng});
        }
      }
    }
    for (auto& b : drounds) add_add_rec(h->s_recs, b);
    // M^T M blocks: with the tensor-core path every distinct M block is split once (as a
    // 128-row A operand and a 64-row B operand; rows = the block's columns, K = its rows)
    // and each round is one launch of the wide persistent product (128 x 64 tiles,
    // K = flux-group length <= 128).
    int maxlen = 0;  // K of the M^T M products: the flux groups' rows
    for (const FGroup& F : h->fgroups) maxlen = std::max(maxlen, F.len);
    if (h->emulated && maxlen <= 128) {
      struct MB { const double* p; int ld, rows, K; size_t ta, tb, ea, eb; };
      std::vector<MB> blocks;
      std::map<const double*, int> idx;
      size_t bytes = 0;
      for (auto& b : mrounds)
        for (const GemmDesc& g : b)
          for (int side = 0; side < 2; ++side) {
            const double* ptr = side ? g.B : g.A;
            if (idx.count(ptr)) continue;
            MB m{ptr, side ? g.ldb : g.lda, side ? g.n : g.m, g.k, 0, 0, 0, 0};
            m.ta = bytes; bytes += al(oz_split_elems(m.rows, m.K, 128) * 2);
            m.tb = bytes; bytes += al(oz_split_elems(m.rows, m.K, 64) * 2);
            m.ea = bytes; bytes += al((size_t)m.rows * 4);
            m.eb = bytes; bytes += al((size_t)m.rows * 4);
            idx[ptr] = (int)blocks.size();
            blocks.push_back(m);
          }
      char* mbase = nullptr;
      if (!blocks.empty() && !dev_alloc(h, &mbase, bytes)) {
        free_all(h);
        delete h;
        return fail(nullptr, ELM_DDM_ERR_OOM, "device allocation failed (Schur split workspace)");
      }
      std::vector<SplitDesc> sp;
      for (const MB& m : blocks) {
        sp.push_back({m.p, m.ld, 1, m.rows, m.K, (int*)(mbase + m.ea), mbase + m.ta, 128});
        sp.push_back({m.p, m.ld, 1, m.rows, m.K, (int*)(mbase + m.eb), mbase + m.tb, 64});
      }
      add_split_rec(h->s_recs, sp, "split_schur");
      for (auto& b : mrounds) {
        std::vector<OzDesc> od;
        for (const GemmDesc& g : b) {
          const MB& A = blocks[idx[g.A]];
          const MB& B = blocks[idx[g.B]];
          od.push_back({mbase + A.ta, (int*)(mbase + A.ea), mbase + B.tb, (int*)(mbase + B.eb), g.C, 1,
                        g.ldc, g.m, g.n, g.k, 0});
        }
        add_updw_rec(h->s_recs, od, 1.0, "oz_schur");
      }
    } else {
      for (auto& b : mrounds) add_gemm_rec(h->s_recs, b, true, false, 1.0, 1.0, 0);
    }
    // Cholesky trailing updates, restricted to the envelope rows [k+nb, rend)
    for (int k = 0, step = 0; k < ng; k += CHOL_NB, ++step) {
      const int nb = std::min(CHOL_NB, ng - k), rest = h->chol_rend[step] - k - nb;
      h->syrk_first.push_back((int)h->syrk_recs.size());
      if (rest <= 0) continue;
      double* L21 = h->S + (k + nb) + (size_t)k * ng;
      double* S22 = h->S + (k + nb) + (size_t)(k + nb) * ng;
      if (h->emulated) {
        // digit planes of L21 in one of two buffers (by step parity: the split of step
        // k + 1 runs while part B of step k still reads those of step k)
        char* reg = chol_region + (size_t)(step & 1) * (c1 + c2 + 2 * ce);
        int* xa = (int*)(reg + c1 + c2);
        int* xb = (int*)(reg + c1 + c2 + ce);
        // the panel solve L21 = A21 L11^{-T} (launch_trsm_chol_rows) writes L21's split:
        // planes reg (128-row tiles), reg + c1 (32-row tiles), exponents xa, xb
        // SYRK A22 -= L21 L21^T in two parts: A, the next block column (what the next
        // step's factor and panel solve need), on the main stream; B, the columns beyond,
        // on the second stream (B operand rows and C columns offset by nb2)
        const int nb2 = std::min(CHOL_NB, rest);
        add_oz_rec(h->syrk_recs, {{reg, xa, reg + c1, xb, S22, 1, ng, rest, nb2, nb, 0}}, 0, -1.0, 1.0,
                   GEMM_LOWER, "oz_syrk");
        if (rest > nb2) {
          const size_t btile = oz_split_elems(32, nb, 32) * 2;  // bytes of one 32-row B tile
          OzDesc b{reg, xa, reg + c1 + (size_t)(nb2 / 32) * btile, xb + nb2, S22 + (size_t)nb2 * ng,
                   1, ng, rest, rest - nb2, nb, 0};
          b.lower_off = nb2;
          add_oz_rec(h->syrk_recs, {b}, 0, -1.0, 1.0, GEMM_LOWER, "oz_syrk_b");
          h->syrk_recs.back().side = 1;
        }
      } else {
        add_gemm_rec(h->syrk_recs, {{L21, L21, S22, rest, rest, nb, ng, ng, ng}}, false, true, -1.0,
                     1.0, GEMM_LOWER);
      }
    }
    h->syrk_first.push_back((int)h->syrk_recs.size());
  }
  ok = dev_alloc(h, &h->gd, gds.size()) && dev_alloc(h, &h->ad, ads.size()) &&
       dev_alloc(h, &h->sd, sds.size()) && dev_alloc(h, &h->od, ods.size()) &&
       dev_alloc(h, &h->ut, uts.size());
  if (!ok) {
    free_all(h);
    delete h;
    return fail(nullptr, ELM_DDM_ERR_OOM, "device allocation failed");
  }
  cudaError_t e = cudaSuccess;
  auto cp = [&](void* dst, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  };
  cp(h->gd, gds.data(), gds.size() * sizeof(GemmDesc));
  cp(h->ad, ads.data(), ads.size() * sizeof(AddDesc));
  cp(h->sd, sds.data(), sds.size() * sizeof(SplitDesc));
  cp(h->od, ods.data(), ods.size() * sizeof(OzDesc));
  cp(h->ut, uts.data(), uts.size() * sizeof(int4));
  cp(h->xy, xy, (size_t)N * m_max * 2 * sizeof(double));
  cp(h->nrm, nrm, (size_t)N * m_max * 2 * sizeof(double));
  cp(h->cnt, h->cnt_h.data(), (size_t)N * 3 * sizeof(int));
  if (h->nsub) cp(h->nsub, h->ns_h.data(), (size_t)N * sizeof(int));
  cp(h->ms, h->ms_h.data(), (size_t)N * sizeof(int));
  cp(h->mg, h->mg_h.data(), (size_t)N * sizeof(int));
  cp(h->dofmap, dofmap.data(), dofmap.size() * sizeof(int));
  cp(h->mf, h->mf_h.data(), (size_t)N * sizeof(int));
  cp(h->fluxmap, fluxmap.data(), fluxmap.size() * sizeof(int));
  cp(h->ffd, ffd.data(), ffd.size() * sizeof(int));
  if (h->explicit_flux) {
    cp(h->frow, frow_d.data(), frow_d.size() * sizeof(int));
    cp(h->fnrm, fnrm_d.data(), fnrm_d.size() * sizeof(double));
  }
  cp(h->ifc_dof, ifc.data(), ifc.size() * sizeof(int));
  cp(h->perm, h->perm_h.data(), h->perm_h.size() * sizeof(int));
  cp(h->d_rend, h->chol_rend.data(), h->chol_rend.size() * sizeof(int));
  cp(h->d_jbeg, h->chol_jbeg.data(), h->chol_jbeg.size() * sizeof(int));
  if (e == cudaSuccess && h->emulated) e = cudaMemset(h->hlbuf, 0, (size_t)N * OZ_HL_TILE * sizeof(long long));
  if (h->bj && !h->edges.empty()) {
    cp(h->bj_off, h->newoff.data(), h->newoff.size() * sizeof(int));
    cp(h->bj_len, bj_len_h.data(), bj_len_h.size() * sizeof(int));
    cp(h->bj_ioff, bj_ioff_h.data(), bj_ioff_h.size() * sizeof(long long));
  }
  {
    int rows = 0, cols = 0;
    for (size_t st = 0; st < h->chol_rend.size(); ++st) {
      const int k = (int)st * CHOL_NB, nb = std::min(CHOL_NB, ng - k);
      rows = std::max(rows, h->chol_rend[st] - k - nb);
      cols = std::max(cols, k - h->chol_jbeg[st]);
    }
    h->fwd_grid = ng > 0 ? chol_solve_grid(true, rows) : 0;
    h->bwd_grid = ng > 0 ? chol_solve_grid(false, cols) : 0;
  }
  if (h->use_tabs) {
    cp(h->tab_xs, txs.data(), txs.size() * sizeof(double));
    cp(h->tab_ys, tys.data(), tys.size() * sizeof(double));
    cp(h->tab_ctr, tctr.data(), tctr.size() * sizeof(double));
    cp(h->tab_nxy, tnxy.data(), tnxy.size() * sizeof(int));
    cp(h->tab_rix, trix.data(), trix.size() * sizeof(int));
  }
  if (e == cudaSuccess) e = cudaMemset(h->status, 0, sizeof(unsigned));
  if (e != cudaSuccess) {
    std::string msg = std::string("setup copy: ") + cudaGetErrorString(e);
    free_all(h);
    delete h;
    return fail(nullptr, ELM_DDM_ERR_CUDA, msg);
  }
  *out = h;
  return ELM_DDM_OK;
}

int elm_ddm_set_coefficient(elm_ddm_handle* h, const double* coef) {
  if (!h) return ELM_DDM_ERR_ARG;
  if (h->op != ELM_DDM_OP_VARCOEF) return fail(h, ELM_DDM_ERR_ARG, "set_coefficient: operator has none");
  if (!coef) return fail(h, ELM_DDM_ERR_ARG, "set_coefficient: NULL coef");
  cudaError_t e = cudaMemcpyAsync(h->coef, coef, (size_t)h->N * h->m_max * 3 * sizeof(double),
                                  cudaMemcpyDeviceToDevice, h->st);
  if (e != cudaSuccess) return cuda_fail(h, e, "set_coefficient");
  h->coef_set = true;
  return ELM_DDM_OK;
}

int elm_ddm_assemble(elm_ddm_handle* h, const double* W, const double* b) {
  if (!h) return ELM_DDM_ERR_ARG;
  if (!W || !b) return fail(h, ELM_DDM_ERR_ARG, "assemble: NULL theta");
  if (h->op == ELM_DDM_OP_VARCOEF && !h->coef_set)
    return fail(h, ELM_DDM_ERR_STATE, "assemble: call elm_ddm_set_coefficient first");
  const size_t nw = (size_t)h->N * h->n;
  cudaError_t e = cudaMemcpyAsync(h->thW, W, nw * 2 * sizeof(double), cudaMemcpyDeviceToDevice, h->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h->thb, b, nw * sizeof(double), cudaMemcpyDeviceToDevice, h->st);
  if (e != cudaSuccess) return cuda_fail(h, e, "assemble: copy theta");
  h->lowfac = h->mixed;  // the next factorisation is the low-precision one
  return assemble_launch(h);
}

int elm_ddm_schur(elm_ddm_handle* h) {
  if (!h) return ELM_DDM_ERR_ARG;
  if (h->state != 1) return fail(h, ELM_DDM_ERR_STATE, "schur: call elm_ddm_assemble first");
  // digit groups of the local products (QR, Y, D_s, M_s): all of them, or the leading ones of
  // the low-precision factorisation; the Schur matrix's M^T M and Cholesky stay FP64
  const int lo_gmax = h->lowfac ? LO_GMAX : 8;
  // (b) blocked Householder QR of [K^s | J]
  for (int b = 0; b < h->nblk; ++b) {
    const int k0 = b * QR_NB, nbe = std::min(QR_NB, h->n - k0);
    ELM_LAUNCH_FB(h, launch_panel_qr(h->K, h->kstride, h->ld, h->ms, h->N, k0, nbe, h->tau, h->n,
                                     h->Vp + (size_t)h->panel_vcol[b] * h->ld, h->vstride, h->status,
                                     h->st, h->lowfac, h->tune_panel, h->panel_vrow0[b]),
                  "panel_qr", h->panel_flops[b], h->panel_bytes[b]);
    int rc = run_recs(h, h->qr_recs, h->qr_first[b], h->qr_first[b + 1] - h->qr_first[b],
                      "gemm_qr", lo_gmax);
    if (rc) return rc;
  }
  h->state = 0;  // K is factored in place: assemble again before another schur
  if (h->ng > 0) {
    int rc;
    if (h->emulated) {
      rc = run_recs(h, h->ty_recs, 0, h->ty_recs.size(), "trsm_y", lo_gmax);
      if (rc) return rc;
    } else {
      ELM_LAUNCH(h, launch_trsm_y(h->Am, h->astride, h->mfld, h->K, h->kstride, h->ld, h->mf, h->mfmax,
                                  h->N, h->n, h->st), "trsm_y");
    }
    rc = run_recs(h, h->dm_recs, 0, h->dm_recs.size(), "gemm_dm", lo_gmax);
    if (rc) return rc;
    if (h->cg_only) {  // D_s and M_s are all that elm_ddm_solve_cg needs
      h->state = 2;
      return ELM_DDM_OK;
    }
    cudaError_t e = cudaMemsetAsync(h->S, 0, (size_t)h->ng * h->ng * sizeof(double), h->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->Mdiag, 0, h->mdiag_elems * sizeof(double), h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "schur: memset");
    rc = run_recs(h, h->s_recs, 0, h->s_recs.size(), "gemm_schur");
    if (rc) return rc;
    // Jacobi preconditioner of the CG solves, taken before the factorisation overwrites S
    ELM_LAUNCH(h, launch_diag_inv(h->S, h->ng, h->sdinv, h->st), "diag_inv");
    h->has_sdinv = true;
    if (h->bj) {
      ELM_LAUNCH(h, launch_block_inv(h->S, h->ng, h->bj_off, h->bj_len, h->bj_ioff, (int)h->edges.size(),
                                     h->bj_maxlen, h->bj_inv, h->status, h->st), "block_inv");
      h->has_bj = true;
    }
    // Look-ahead (tensor-core back end): part B of step k's SYRK (columns beyond the next
    // block column) runs on st2 while st factors and solves that column.  st2 starts B
    // after st's panel solve of step k, which writes the split operands (evS); st waits
    // for B(k - 1) (evB) before its part A(k), the first launch that touches B(k - 1)'s
    // columns.
    bool b_pending = false;
    for (int k = 0, step = 0; k < h->ng; k += CHOL_NB, ++step) {
      const int nb = std::min(CHOL_NB, h->ng - k);
      // the factor (nb^3/3), then the panel solve L21 = A21 L11^{-T} by substitution
      const int rend = h->chol_rend[step];
      ELM_LAUNCH_F(h, launch_potrf_diag(h->S, h->ng, k, nb, h->status, h->st), "potrf",
                   nb * nb * (double)nb / 3.0);
      if (rend - k - nb > 0) {
        void *tA = nullptr, *tB = nullptr;
        int *eA = nullptr, *eB = nullptr;
        if (h->emulated) {  // this step's parity buffer (see the look-ahead below)
          char* reg = h->creg + (size_t)(step & 1) * (h->creg_c1 + h->creg_c2 + 2 * h->creg_ce);
          tA = reg;
          tB = reg + h->creg_c1;
          eA = (int*)(reg + h->creg_c1 + h->creg_c2);
          eB = (int*)(reg + h->creg_c1 + h->creg_c2 + h->creg_ce);
        }
        ELM_LAUNCH_F(h, launch_trsm_chol_rows(h->S, h->ng, k, nb, rend, h->st, tA, tB, eA, eB),
                     "trsm_rows", (double)(rend - k - nb) * nb * nb);
      }
      if (rend - k - nb > 0) {
        const int r0 = h->syrk_first[step], nr = h->syrk_first[step + 1] - r0;
        if (!h->emulated) {
          rc = run_recs(h, h->syrk_recs, r0, nr, "gemm_syrk");
          if (rc) return rc;
        } else {
          // records: part A, part B (when there are columns beyond the next block); the
          // panel solve above wrote their split operands
          const bool has_b = nr == 2 && h->syrk_recs[r0 + 1].side;
          cudaError_t e2 = cudaSuccess;
          if (has_b) {
            e2 = cudaEventRecord(h->evS, h->st);
            if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(h->st2, h->evS, 0);
          }
          if (e2 == cudaSuccess && b_pending) e2 = cudaStreamWaitEvent(h->st, h->evB, 0);
          if (e2 != cudaSuccess) return cuda_fail(h, e2, "schur: look-ahead events");
          b_pending = false;
          rc = run_recs(h, h->syrk_recs, r0, 1, "oz_syrk");
          if (rc) return rc;
          if (has_b) {
            rc = run_recs(h, h->syrk_recs, r0 + 1, 1, "oz_syrk_b");
            if (rc) return rc;
            e2 = cudaEventRecord(h->evB, h->st2);
            if (e2 != cudaSuccess) return cuda_fail(h, e2, "schur: look-ahead events");
            b_pending = true;
          }
        }
      }
    }
    if (b_pending) {
      const cudaError_t e2 = cudaStreamWaitEvent(h->st, h->evB, 0);
      if (e2 != cudaSuccess) return cuda_fail(h, e2, "schur: look-ahead join");
    }
    // inverses of the diagonal blocks for the triangular solves of the solve phase
    ELM_LAUNCH(h, launch_tri_inv(h->S, h->ng, h->ng, h->cinv, h->st), "tri_inv");
  }
  h->state = 2;
  return ELM_DDM_OK;
}

int elm_ddm_solve(elm_ddm_handle* h, const double* rhs, int nrhs, double* u_gamma, double* c) {
  if (!h) return ELM_DDM_ERR_ARG;
  if (h->state != 2) return fail(h, ELM_DDM_ERR_STATE, "solve: call elm_ddm_schur first");
  if (h->lowfac) {
    if (!rhs || !c) return fail(h, ELM_DDM_ERR_ARG, "solve: NULL rhs or c");
    if (nrhs < 1 || nrhs > h->max_rhs) return fail(h, ELM_DDM_ERR_ARG, "solve: nrhs out of range");
    return solve_refined(h, rhs, nrhs, u_gamma, c);
  }
  if (h->cg_only)
    return fail(h, ELM_DDM_ERR_STATE, "solve: S is not factored (ELM_DDM_FLAG_SCHUR_CG); use elm_ddm_solve_cg");
  if (!rhs || !c) return fail(h, ELM_DDM_ERR_ARG, "solve: NULL rhs or c");
  if (nrhs < 1 || nrhs > h->max_rhs) return fail(h, ELM_DDM_ERR_ARG, "solve: nrhs out of range");
  const int N = h->N, n = h->n, ng = h->ng;
  ELM_LAUNCH(h, launch_load_rhs(h->X, rhs, N, h->m_max, h->ld, h->cnt, nrhs, h->status, h->st),
             "load_rhs");
  ELM_LAUNCH(h, launch_apply_qt(h->X, h->K, h->kstride, h->ld, h->ms, N, n, h->T, h->tstride, nrhs,
                                h->st), "apply_qt");
  if (ng > 0) {
    ELM_LAUNCH(h, launch_iface_vecs(h->X, h->K, h->kstride, h->ld, h->Am, h->astride, h->mgld, h->mg,
                                    h->mfld, h->mf, N, n, nrhs, h->gq, h->hq, h->st), "iface_vecs");
    ELM_LAUNCH(h, launch_gather2(h->dofmap, GRP_MAX, ng, h->mgld, N, h->gq, h->rv, 0, nrhs, h->st), "gather_r");
    ELM_LAUNCH(h, launch_gather2(h->fluxmap, 2, h->n_flux, h->mfld, N, h->hq, h->hv, 0, nrhs, h->st),
               "gather_h");
    ELM_LAUNCH(h, launch_mt_h(h->M, h->mstride, h->mfld, h->mf, h->mg, h->ffd, h->hv, h->n_flux, N, h->mgld,
                              nrhs, h->zv, h->st), "mt_h");
    ELM_LAUNCH(h, launch_gather2(h->dofmap, GRP_MAX, ng, h->mgld, N, h->zv, h->rv, 1, nrhs, h->st), "gather_z");
    const int rc = chol_solves(h, nrhs);
    if (rc) return rc;
  }
  ELM_LAUNCH(h, launch_backsolve(h->X, h->K, h->kstride, h->ld, h->mg, h->ifc_dof, h->mgld,
                                 ng > 0 ? h->uv : h->rv, ng, N, n, nrhs, c, h->st), "backsolve");
  if (u_gamma && ng > 0)
    ELM_LAUNCH(h, launch_gather_perm(h->perm, ng, h->uv, u_gamma, nrhs, h->st), "gather_u");
  return ELM_DDM_OK;
}

}  // extern "C"

namespace {

// u = S^{-1} r for nrhs vectors (rv -> yv -> uv) with the Cholesky factor in S.
int chol_solves(elm_ddm_handle* h, int nrhs) {
  const int ng = h->ng;
  {
    const int nsteps = (int)h->chol_rend.size();
    if (h->fwd_grid > 0 && h->bwd_grid > 0) {
      ELM_LAUNCH(h, launch_chol_fwd_all(h->S, ng, ng, h->cinv, h->d_rend, nsteps, h->rv, h->yv, nrhs,
                                        h->fwd_grid, h->cbar, h->status, h->st, h->wait_ns, h->wait_hold),
                 "chol_fwd");
      ELM_LAUNCH(h, launch_chol_bwd_all(h->S, ng, ng, h->cinv, h->d_jbeg, nsteps, h->yv, h->uv, nrhs,
                                        h->bwd_grid, h->cbar, h->status, h->st, h->wait_ns, h->wait_hold),
                 "chol_bwd");
    } else {
      for (int k = 0, step = 0; k < ng; k += CHOL_NB, ++step) {
        const int nb = std::min(CHOL_NB, ng - k);
        ELM_LAUNCH(h, launch_chol_fwd(h->S, ng, ng, k, nb, h->rv, h->yv, nrhs, h->st,
                                      h->chol_rend[step], h->cinv + (size_t)step * CHOL_NB * CHOL_NB),
                   "chol_fwd");
      }
      for (int k = ((ng - 1) / CHOL_NB) * CHOL_NB; k >= 0; k -= CHOL_NB) {
        const int nb = std::min(CHOL_NB, ng - k);
        ELM_LAUNCH(h, launch_chol_bwd(h->S, ng, ng, k, nb, h->yv, h->uv, nrhs, h->st,
                                      h->chol_jbeg[k / CHOL_NB],
                                      h->cinv + (size_t)(k / CHOL_NB) * CHOL_NB * CHOL_NB),
                   "chol_bwd");
      }
    }
  }
  return ELM_DDM_OK;
}

// Solve of the mixed-precision mode.  Iterates (c, w, u) of the block system in k_refine.cu
// start at zero; every step takes the FP64 residual (products with the FP64 K^s, A^s) and
// adds the correction the low-precision factors give by the elimination of Eq. (3.5):
//   p1 = R^{-T} r1,  p13 = R^{-T} (r1 - r3),
//   S du = r2 + sum_s E_s^T Q_G p13 + M^T h,  h = sum_s E_s^T Y p1,
//   dc = R^{-1} (p1 + Q_G^T E du),  dw = R^{-1} R^{-T} (r3 + A^T A dc).
// It stops when the relative u_Gamma correction eta (the c correction when there is no
// interface) is at most refine_tol, or below 1e-10 and no longer contracting (the rounding
// floor).  Otherwise -- a step from the third on that does not halve eta, a correction that
// is not finite, refine_maxit steps -- refinement has stalled: the handle falls back to the
// FP64 path (re-assembly from theta, FP64 factorisation, direct solve), which also serves
// the later solves until the next elm_ddm_assemble.
int solve_refined(elm_ddm_handle* h, const double* rhs, int nrhs, double* u_gamma, double* c) {
  const int N = h->N, n = h->n, ng = h->ng, ld = h->ld, mgld = h->mgld;
  const size_t cn = (size_t)nrhs * N * n, xn = (size_t)nrhs * N * ld;
  const long long k64 = (long long)ld * n;
  int mmax = 0;
  for (int s = 0; s < N; ++s) mmax = std::max(mmax, h->ms_h[s]);
  ELM_LAUNCH(h, launch_load_rhs(h->F64, rhs, N, h->m_max, ld, h->cnt, nrhs, h->status, h->st), "load_rhs");
  cudaError_t e = cudaMemsetAsync(h->cit, 0, cn * sizeof(double), h->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->wit, 0, cn * sizeof(double), h->st);
  if (e == cudaSuccess && ng > 0) e = cudaMemsetAsync(h->uit, 0, (size_t)nrhs * ng * sizeof(double), h->st);
  if (e != cudaSuccess) return cuda_fail(h, e, "solve: refinement start");
  const double* ug = ng > 0 ? h->uv : h->zero_ng;  // the u_Gamma correction (zero without interface)
  std::vector<unsigned long long> nb(4 * (size_t)nrhs);
  double eta = INFINITY, eta_prev = INFINITY;
  bool converged = false;
  int steps = 0;
  for (int it = 0; it < h->refine_maxit; ++it) {
    // FP64 residual: e = F - K c + [0; 0; E u], z = -(e + K w) (interface rows), r1 = K^T e,
    // r3 = A^T (A c) - K^T K w, r13 = r1 - r3
    ELM_LAUNCH(h, launch_resid_rows(h->K64, k64, ld, n, h->ms, h->cnt, h->ifc_dof, mgld, h->F64, h->cit, h->wit,
                                    h->uit, ng, N, mmax, nrhs, h->ebuf, h->kwbuf, h->zb, h->st), "refine_resid");
    ELM_LAUNCH(h, launch_resid_cols(h->K64, k64, ld, n, h->ms, h->ebuf, h->kwbuf, N, nrhs, h->r1b, h->tb, h->st),
               "refine_resid");
    if (ng > 0) {
      ELM_LAUNCH(h, launch_amul(h->A64, h->astride, mgld, h->mg, h->mgmax, n, h->cit, N, nrhs, h->Acl, h->st),
                 "refine_resid");
      ELM_LAUNCH(h, launch_gather2(h->dofmap, GRP_MAX, ng, mgld, N, h->Acl, h->Acg, 0, nrhs, h->st), "refine_resid");
    }
    ELM_LAUNCH(h, launch_atmul(h->A64, h->astride, mgld, h->mg, h->ifc_dof, n, ng > 0 ? h->Acg : h->zero_ng, ng,
                               h->tb, -1.0, h->r1b, N, nrhs, h->r3b, h->r13b, h->st), "refine_resid");
    // correction through the low-precision factors
    ELM_LAUNCH(h, launch_rt_solve(h->K, h->kstride, ld, n, h->r1b, n, h->Pb, ld, N, nrhs, h->st), "refine_rt");
    ELM_LAUNCH(h, launch_rt_solve(h->K, h->kstride, ld, n, h->r13b, n, h->Pb + xn, ld, N, nrhs, h->st),
               "refine_rt");
    if (ng > 0) {
      const size_t gslot = (size_t)nrhs * N * mgld;
      ELM_LAUNCH(h, launch_gather2(h->dofmap, GRP_MAX, ng, mgld, N, h->zb, h->rv, 0, nrhs, h->st), "gather_r");
      ELM_LAUNCH(h, launch_iface_vecs(h->Pb, h->K, h->kstride, ld, h->Am, h->astride, mgld, h->mg, mgld, h->mg, N, n, 2 * nrhs,
                                      h->gq2, h->hq2, h->st), "iface_vecs");
      ELM_LAUNCH(h, launch_gather2(h->dofmap, GRP_MAX, ng, mgld, N, h->gq2 + gslot, h->rv, 1, nrhs, h->st), "gather_r");
      ELM_LAUNCH(h, launch_gather2(h->dofmap, GRP_MAX, ng, mgld, N, h->hq2, h->hv, 0, nrhs, h->st), "gather_h");
      ELM_LAUNCH(h, launch_mt_h(h->M, h->mstride, mgld, h->mg, h->mg, h->ifc_dof, h->hv, ng, N, mgld, nrhs, h->zv, h->st),
                 "mt_h");
      ELM_LAUNCH(h, launch_gather2(h->dofmap, GRP_MAX, ng, mgld, N, h->zv, h->rv, 1, nrhs, h->st), "gather_z");
      const int rc = chol_solves(h, nrhs);
      if (rc) return rc;
    }
    ELM_LAUNCH(h, launch_backsolve(h->Pb, h->K, h->kstride, ld, h->mg, h->ifc_dof, mgld, ug, ng, N, n, nrhs,
                                   h->dcv, h->st), "backsolve");
    if (ng > 0) {
      ELM_LAUNCH(h, launch_amul(h->A64, h->astride, mgld, h->mg, h->mgmax, n, h->dcv, N, nrhs, h->Acl, h->st),
                 "refine_resid");
      ELM_LAUNCH(h, launch_gather2(h->dofmap, GRP_MAX, ng, mgld, N, h->Acl, h->Acg, 0, nrhs, h->st), "refine_resid");
    }
    ELM_LAUNCH(h, launch_atmul(h->A64, h->astride, mgld, h->mg, h->ifc_dof, n, ng > 0 ? h->Acg : h->zero_ng, ng,
                               h->r3b, 1.0, nullptr, N, nrhs, h->r13b, nullptr, h->st), "refine_resid");
    ELM_LAUNCH(h, launch_rt_solve(h->K, h->kstride, ld, n, h->r13b, n, h->Pb, ld, N, nrhs, h->st), "refine_rt");
    ELM_LAUNCH(h, launch_backsolve(h->Pb, h->K, h->kstride, ld, h->mg, h->ifc_dof, mgld, h->zero_ng, ng, N, n,
                                   nrhs, h->dwv, h->st), "backsolve");
    e = cudaMemsetAsync(h->nrmb, 0, 4 * (size_t)nrhs * sizeof(unsigned long long), h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "solve: refinement norms");
    ELM_LAUNCH(h, launch_refine_update(h->cit, h->dcv, h->wit, h->dwv, (long long)N * n, h->uit, ug, ng, nrhs,
                                       h->nrmb, h->st), "refine_update");
    e = cudaMemcpyAsync(nb.data(), h->nrmb, nb.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) return cuda_fail(h, e, "solve: refinement norms");
    steps = it + 1;
    eta = 0.0;
    for (int r = 0; r < nrhs; ++r) {
      double v[4];
      for (int q = 0; q < 4; ++q) memcpy(&v[q], &nb[4 * (size_t)r + q], sizeof(double));
      const double er = ng > 0 ? (v[1] > 0.0 ? v[0] / v[1] : (v[0] > 0.0 ? INFINITY : 0.0))
                               : (v[3] > 0.0 ? v[2] / v[3] : (v[2] > 0.0 ? INFINITY : 0.0));
      eta = std::isnan(er) || std::isnan(eta) ? NAN : std::max(eta, er);
    }
    if (!std::isfinite(eta)) break;
    if (eta <= h->refine_tol) { converged = true; break; }
    if (it >= 2 && eta > 0.5 * eta_prev) {
      converged = eta <= 1e-10;  // the rounding floor above refine_tol
      break;
    }
    eta_prev = eta;
  }
  h->last_iters = steps;
  h->last_eta = eta;
  if (!converged) {
    h->last_fallback = 1;
    h->lowfac = false;
    int rc = assemble_launch(h);
    if (rc == ELM_DDM_OK) rc = elm_ddm_schur(h);
    if (rc == ELM_DDM_OK) rc = elm_ddm_solve(h, rhs, nrhs, u_gamma, c);
    return rc;
  }
  h->last_fallback = 0;
  e = cudaMemcpyAsync(c, h->cit, cn * sizeof(double), cudaMemcpyDeviceToDevice, h->st);
  if (e != cudaSuccess) return cuda_fail(h, e, "solve: refined c");
  if (u_gamma && ng > 0)
    ELM_LAUNCH(h, launch_gather_perm(h->perm, ng, h->uit, u_gamma, nrhs, h->st), "gather_u");
  return ELM_DDM_OK;
}

}  // namespace

static int solve_cg_impl(elm_ddm_handle* h, const double* rhs, int nrhs, const double* x0, int jacobi,
                         double tol, int maxit, double* u_gamma, double* c, int* iters) {
  if (!h) return ELM_DDM_ERR_ARG;
  if (iters) *iters = 0;
  if (h->state != 2) return fail(h, ELM_DDM_ERR_STATE, "solve_cg: call elm_ddm_schur first");
  if (h->lowfac)
    return fail(h, ELM_DDM_ERR_STATE, "solve_cg: the factorisation is the low-precision one (ELM_DDM_FLAG_MIXED)");
  if (h->explicit_flux)
    return fail(h, ELM_DDM_ERR_STATE, "solve_cg: not with explicit flux rows (elm_ddm_setup_flux)");
  if (!rhs || !c) return fail(h, ELM_DDM_ERR_ARG, "solve_cg: NULL rhs or c");
  if (nrhs < 1 || nrhs > h->max_rhs) return fail(h, ELM_DDM_ERR_ARG, "solve_cg: nrhs out of range");
  if (!(tol > 0.0) || !std::isfinite(tol)) return fail(h, ELM_DDM_ERR_ARG, "solve_cg: tol must be > 0");
  if (maxit < 1) return fail(h, ELM_DDM_ERR_ARG, "solve_cg: maxit must be >= 1");
  if (jacobi < 0 || jacobi > 2) return fail(h, ELM_DDM_ERR_ARG, "solve_cg: preconditioner must be 0, 1 or 2");
  if (jacobi == 1 && !h->has_sdinv)
    return fail(h, ELM_DDM_ERR_STATE, "solve_cg: Jacobi needs the assembled S (not ELM_DDM_FLAG_SCHUR_CG)");
  if (jacobi == 2 && !h->has_bj)
    return fail(h, ELM_DDM_ERR_STATE, "solve_cg: block-Jacobi needs ELM_DDM_FLAG_BLOCK_JACOBI and elm_ddm_schur");
  const int N = h->N, n = h->n, ng = h->ng;
  ELM_LAUNCH(h, launch_load_rhs(h->X, rhs, N, h->m_max, h->ld, h->cnt, nrhs, h->status, h->st),
             "load_rhs");
  ELM_LAUNCH(h, launch_apply_qt(h->X, h->K, h->kstride, h->ld, h->ms, N, n, h->T, h->tstride, nrhs,
                                h->st), "apply_qt");
  bool converged = true;
  int taken = 0;
  if (ng > 0) {
    // right-hand side of Eq. (3.5), as in elm_ddm_solve
    ELM_LAUNCH(h, launch_iface_vecs(h->X, h->K, h->kstride, h->ld, h->Am, h->astride, h->mgld, h->mg,
                                    h->mfld, h->mf, N, n, nrhs, h->gq, h->hq, h->st), "iface_vecs");
    ELM_LAUNCH(h, launch_gather2(h->dofmap, GRP_MAX, ng, h->mgld, N, h->gq, h->rv, 0, nrhs, h->st), "gather_r");
    ELM_LAUNCH(h, launch_gather2(h->fluxmap, 2, h->n_flux, h->mfld, N, h->hq, h->hv, 0, nrhs, h->st),
               "gather_h");
    ELM_LAUNCH(h, launch_mt_h(h->M, h->mstride, h->mfld, h->mf, h->mg, h->ffd, h->hv, h->n_flux, N, h->mgld,
                              nrhs, h->zv, h->st), "mt_h");
    ELM_LAUNCH(h, launch_gather2(h->dofmap, GRP_MAX, ng, h->mgld, N, h->zv, h->rv, 1, nrhs, h->st), "gather_z");
    // CG: x in uv, r in yv; gq / hq / hv are free now and serve as the operator's scratch
    const double tol2 = tol * tol;
    const double* dinv = jacobi == 1 ? h->sdinv : nullptr;
    const bool block = jacobi == 2;
    const int nedges = (int)h->edges.size();
    if (x0) {  // start from the caller's guess: x = x0 (internal order), q = S x
      ELM_LAUNCH(h, launch_scatter_perm(h->perm, ng, x0, h->uv, nrhs, h->st), "cg_x0");
      ELM_LAUNCH(h, launch_schur_apply(h->D, h->M, h->mstride, h->mgld, h->mg, h->mgmax, h->ifc_dof,
                                       h->dofmap, h->uv, h->cg_q, h->gq, h->hq, h->hv, ng, N, nrhs,
                                       h->st), "cg_apply");
    } else {
      cudaError_t e = cudaMemsetAsync(h->uv, 0, (size_t)nrhs * ng * sizeof(double), h->st);
      if (e != cudaSuccess) return cuda_fail(h, e, "solve_cg: x0");
    }
    ELM_LAUNCH(h, launch_pcg_init(h->rv, h->cg_q, h->yv, h->cg_p, dinv, h->cg_st, ng, nrhs, x0 ? 1 : 0,
                                  tol2, h->st), "cg_init");
    if (block) {  // z = B^{-1} r, p = z, rz = r^T z
      ELM_LAUNCH(h, launch_bj_apply(h->bj_inv, h->bj_off, h->bj_len, h->bj_ioff, nedges, h->yv, h->cg_z, ng,
                                    nrhs, h->st), "cg_prec");
      ELM_LAUNCH(h, launch_pcg_step_b(h->yv, h->cg_z, h->cg_p, h->cg_st, ng, nrhs, tol2, 1, h->st), "cg_update");
    }
    std::vector<CgState> hs(nrhs);
    {
      cudaError_t e = cudaMemcpyAsync(hs.data(), h->cg_st, nrhs * sizeof(CgState), cudaMemcpyDeviceToHost,
                                      h->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
      if (e != cudaSuccess) return cuda_fail(h, e, "solve_cg: state");
    }
    bool start_done = true;
    for (const CgState& q : hs) start_done = start_done && q.done != 0;
    for (int it = 0; it < maxit && !start_done;) {
      const int chunk = std::min(16, maxit - it);
      for (int k = 0; k < chunk; ++k) {
        ELM_LAUNCH(h, launch_schur_apply(h->D, h->M, h->mstride, h->mgld, h->mg, h->mgmax, h->ifc_dof,
                                         h->dofmap, h->cg_p, h->cg_q, h->gq, h->hq, h->hv, ng, N, nrhs,
                                         h->st), "cg_apply");
        if (block) {
          ELM_LAUNCH(h, launch_pcg_step_a(h->uv, h->yv, h->cg_p, h->cg_q, h->cg_st, ng, nrhs, h->st),
                     "cg_update");
          ELM_LAUNCH(h, launch_bj_apply(h->bj_inv, h->bj_off, h->bj_len, h->bj_ioff, nedges, h->yv, h->cg_z, ng,
                                        nrhs, h->st), "cg_prec");
          ELM_LAUNCH(h, launch_pcg_step_b(h->yv, h->cg_z, h->cg_p, h->cg_st, ng, nrhs, tol2, 0, h->st),
                     "cg_update");
        } else {
          ELM_LAUNCH(h, launch_pcg_update(h->uv, h->yv, h->cg_p, h->cg_q, dinv, h->cg_st, ng, nrhs, tol2,
                                          h->st), "cg_update");
        }
      }
      it += chunk;
      cudaError_t e = cudaMemcpyAsync(hs.data(), h->cg_st, nrhs * sizeof(CgState), cudaMemcpyDeviceToHost,
                                      h->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
      if (e != cudaSuccess) return cuda_fail(h, e, "solve_cg: state");
      bool all = true;
      for (const CgState& q : hs) all = all && q.done != 0;
      if (all) break;
    }
    for (const CgState& q : hs) {
      taken = std::max(taken, q.iters);
      converged = converged && q.done == 1;
    }
  }
  ELM_LAUNCH(h, launch_backsolve(h->X, h->K, h->kstride, h->ld, h->mg, h->ifc_dof, h->mgld,
                                 ng > 0 ? h->uv : h->rv, ng, N, n, nrhs, c, h->st), "backsolve");
  if (u_gamma && ng > 0)
    ELM_LAUNCH(h, launch_gather_perm(h->perm, ng, h->uv, u_gamma, nrhs, h->st), "gather_u");
  if (iters) *iters = taken;
  if (!converged) return fail(h, ELM_DDM_ERR_NOCONV, "solve_cg: relative residual above tol");
  return ELM_DDM_OK;
}

extern "C" {

int elm_ddm_solve_cg(elm_ddm_handle* h, const double* rhs, int nrhs, double tol, int maxit,
                     double* u_gamma, double* c, int* iters) {
  return solve_cg_impl(h, rhs, nrhs, nullptr, 0, tol, maxit, u_gamma, c, iters);
}

int elm_ddm_solve_pcg(elm_ddm_handle* h, const double* rhs, int nrhs, const double* x0, int jacobi,
                      double tol, int maxit, double* u_gamma, double* c, int* iters) {
  return solve_cg_impl(h, rhs, nrhs, x0, jacobi, tol, maxit, u_gamma, c, iters);
}

int elm_ddm_eval(elm_ddm_handle* h, int npts, const double* xy, const int32_t* owner,
                 const double* c, double* u, double* grad) {
  if (!h) return ELM_DDM_ERR_ARG;
  if (npts < 0) return fail(h, ELM_DDM_ERR_ARG, "eval: npts < 0");
  if (npts == 0) return ELM_DDM_OK;
  if (!xy || !owner || !c || !u) return fail(h, ELM_DDM_ERR_ARG, "eval: NULL pointer");
  ELM_LAUNCH(h, launch_eval(h->thW, h->thb, h->N, h->n, npts, xy, owner, c, u, grad, h->st), "eval");
  return ELM_DDM_OK;
}

int elm_ddm_export(elm_ddm_handle* h, int what, int s, double* dst, int ld_dst) {
  if (!h) return ELM_DDM_ERR_ARG;
  if (!dst) return fail(h, ELM_DDM_ERR_ARG, "export: NULL dst");
  if (what != ELM_DDM_BUF_L && (s < 0 || s >= h->N)) return fail(h, ELM_DDM_ERR_ARG, "export: bad s");
  const double* src = nullptr;
  int rows = 0, cols = 0, lds = 0;
  switch (what) {
    case ELM_DDM_BUF_K:
      src = h->K + (size_t)s * h->kstride; rows = h->ms_h[s]; cols = h->n + h->mg_h[s]; lds = h->ld; break;
    case ELM_DDM_BUF_A:
      src = h->Am + (size_t)s * h->astride; rows = h->mf_h[s]; cols = h->n; lds = h->mfld; break;
    case ELM_DDM_BUF_D:
      src = h->D + (size_t)s * h->mstride; rows = cols = h->mg_h[s]; lds = h->mgld; break;
    case ELM_DDM_BUF_M:
      src = h->M + (size_t)s * h->mstride; rows = h->mf_h[s]; cols = h->mg_h[s]; lds = h->mfld; break;
    case ELM_DDM_BUF_L:
      if (h->cg_only) return fail(h, ELM_DDM_ERR_STATE, "export: S is not formed (ELM_DDM_FLAG_SCHUR_CG)");
      src = h->S; rows = cols = h->ng; lds = h->ng; break;
    default: return fail(h, ELM_DDM_ERR_ARG, "export: unknown buffer");
  }
  if (rows == 0 || cols == 0) return ELM_DDM_OK;
  if (ld_dst < rows) return fail(h, ELM_DDM_ERR_ARG, "export: ld_dst too small");
  cudaError_t e = cudaMemcpy2DAsync(dst, (size_t)ld_dst * sizeof(double), src, (size_t)lds * sizeof(double),
                                    (size_t)rows * sizeof(double), cols, cudaMemcpyDeviceToDevice, h->st);
  if (e != cudaSuccess) return cuda_fail(h, e, "export");
  return ELM_DDM_OK;
}

int elm_ddm_check(elm_ddm_handle* h) {
  if (!h) return ELM_DDM_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return cuda_fail(h, e, "check: stream");
  unsigned bits = 0;
  e = cudaMemcpy(&bits, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(h->status, 0, sizeof(unsigned));
  if (e != cudaSuccess) return cuda_fail(h, e, "check: status");
  if (bits & ST_NONFINITE) return fail(h, ELM_DDM_ERR_NONFINITE, "non-finite value in theta, f/g or R");
  if (bits & ST_RANK) return fail(h, ELM_DDM_ERR_RANK, "a local R has an exactly zero diagonal entry");
  if (bits & ST_NOT_SPD) return fail(h, ELM_DDM_ERR_NOT_SPD, "Schur matrix is not positive definite");
  if (bits & ST_TIMEOUT) return fail(h, ELM_DDM_ERR_TIMEOUT, "a device-side wait timed out");
  if (bits & ST_INTERNAL) return fail(h, ELM_DDM_ERR_CUDA, "a kernel was launched outside its limits");
  return ELM_DDM_OK;
}

int elm_ddm_get_points(elm_ddm_handle* h, int kind, double* xy, int32_t* counts) {
  if (!h) return ELM_DDM_ERR_ARG;
  if (kind < ELM_DDM_PTS_INTERIOR || kind > ELM_DDM_PTS_NORMALS)
    return fail(h, ELM_DDM_ERR_ARG, "get_points: unknown kind");
  const int col = kind == ELM_DDM_PTS_NORMALS ? 2 : kind;
  int kmax = 0;
  for (int s = 0; s < h->N; ++s) {
    const int c = h->cnt_h[3 * s + col];
    if (counts) counts[s] = c;
    kmax = std::max(kmax, c);
  }
  if (!xy) return ELM_DDM_OK;
  ELM_LAUNCH(h, launch_get_points(h->xy, h->nrm, h->m_max, h->cnt, h->N, kind, kmax, xy, h->st),
             "get_points");
  return ELM_DDM_OK;
}

int elm_ddm_set_wait_limit(elm_ddm_handle* h, double seconds, int hold_release) {
  if (!h) return ELM_DDM_ERR_ARG;
  if (!(seconds >= 0.0) || !(seconds <= 60.0))
    return fail(h, ELM_DDM_ERR_ARG, "set_wait_limit: seconds must be in [0, 60]");
  if (hold_release != 0 && hold_release != 1)
    return fail(h, ELM_DDM_ERR_ARG, "set_wait_limit: hold_release must be 0 or 1");
  h->wait_ns = (unsigned long long)(seconds * 1e9);
  h->wait_hold = hold_release;
  return ELM_DDM_OK;
}

int elm_ddm_set_ridge(elm_ddm_handle* h, double alpha) {
  if (!h) return ELM_DDM_ERR_ARG;
  if (!h->ridge) return fail(h, ELM_DDM_ERR_STATE, "set_ridge: the handle was set up without ELM_DDM_FLAG_RIDGE");
  if (!(alpha >= 0.0) || !(alpha < 1.0)) return fail(h, ELM_DDM_ERR_ARG, "set_ridge: alpha must be in [0, 1)");
  h->ridge_alpha = alpha;
  return ELM_DDM_OK;
}

int elm_ddm_set_tuning(elm_ddm_handle* h, int key, int value) {
  if (!h) return ELM_DDM_ERR_ARG;
  switch (key) {
    case ELM_DDM_TUNE_PANEL_CTAS:
      if (value != 0 && value != 4 && value != 8)
        return fail(h, ELM_DDM_ERR_ARG, "set_tuning: panel CTAs must be 0, 4 or 8");
      h->tune_panel = value;
      return ELM_DDM_OK;
    case ELM_DDM_TUNE_UPD_GRID:
      if (value < 0) return fail(h, ELM_DDM_ERR_ARG, "set_tuning: grid cap must be >= 0");
      h->tune_upd_grid = value;
      return ELM_DDM_OK;
    default:
      return fail(h, ELM_DDM_ERR_ARG, "set_tuning: unknown key");
  }
}

int elm_ddm_interface_order(const elm_ddm_handle* h, int32_t* order) {
  if (!h || (!order && h->ng > 0)) return ELM_DDM_ERR_ARG;
  for (int g = 0; g < h->ng; ++g) order[g] = h->perm_h[g];
  return ELM_DDM_OK;
}

int elm_ddm_profile(elm_ddm_handle* h, int enable) {
  if (!h) return ELM_DDM_ERR_ARG;
  h->profiling = enable != 0;
  return ELM_DDM_OK;
}

int elm_ddm_profile_only(elm_ddm_handle* h, const char* kernel_class) {
  if (!h) return ELM_DDM_ERR_ARG;
  h->prof_only = kernel_class ? kernel_class : "";
  return ELM_DDM_OK;
}

int elm_ddm_profile_report(elm_ddm_handle* h, char* buf, int buflen) {
  if (!h || !buf || buflen < 2) return ELM_DDM_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) return cuda_fail(h, e, "profile_report");
  struct Acc { long long n = 0; double ms = 0, flops = 0, bytes = 0; };
  std::map<std::string, Acc> acc;
  for (const ProfRec& r : h->prof) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) { cudaGetLastError(); continue; }
    Acc& a = acc[r.name];
    a.n++; a.ms += ms; a.flops += r.flops; a.bytes += r.bytes;
  }
  std::string out = "{";
  bool first = true;
  for (auto& kv : acc) {
    char tmp[256];
    snprintf(tmp, sizeof tmp,
             "%s\"%s\": {\"launches\": %lld, \"ms\": %.6f, \"flops\": %.6e, \"bytes\": %.6e}",
             first ? "" : ", ", kv.first.c_str(), kv.second.n, kv.second.ms, kv.second.flops,
             kv.second.bytes);
    out += tmp;
    first = false;
  }
  char tail[64];
  snprintf(tail, sizeof tail, "%s\"_dropped\": %d}", first ? "" : ", ", h->prof_dropped);
  out += tail;
  h->prof.clear();
  h->ev_used = 0;
  h->prof_dropped = 0;
  if ((int)out.size() + 1 > buflen) return fail(h, ELM_DDM_ERR_ARG, "profile_report: buffer too small");
  memcpy(buf, out.c_str(), out.size() + 1);
  return ELM_DDM_OK;
}

int elm_ddm_get_info(const elm_ddm_handle* h, int key, double* value) {
  if (!h || !value) return ELM_DDM_ERR_ARG;
  switch (key) {
    case 0: *value = h->ng; break;
    case 1: *value = (double)h->bytes; break;
    case 2: *value = (double)h->launches; break;
    case 3: *value = (double)h->edges.size(); break;
    case 4: *value = h->m_max; break;
    case 7: *value = (double)elmddm::g_kernel_launches.load(); break;
    case 8: *value = h->use_tabs ? 1.0 : 0.0; break;
    case 9: *value = (h->fwd_grid > 0 && h->bwd_grid > 0) ? 1.0 : 0.0; break;
    case 10: *value = h->last_iters; break;
    case 11: *value = h->last_fallback; break;
    case 12: *value = h->last_eta; break;
    case 13: *value = h->lowfac ? 1.0 : 0.0; break;
    case 5: *value = h->n; break;
    case 6: *value = h->N; break;
    default: return ELM_DDM_ERR_ARG;
  }
  return ELM_DDM_OK;
}

int elm_ddm_destroy(elm_ddm_handle* h) {
  if (!h) return ELM_DDM_ERR_ARG;
  cudaStreamSynchronize(h->st);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  free_all(h);
  delete h;
  return ELM_DDM_OK;
}

const char* elm_ddm_last_error(const elm_ddm_handle* h) {
  return h ? h->err.c_str() : g_setup_error.c_str();
}

}  // extern "C"
