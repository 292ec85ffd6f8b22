/*
 * elm_ddm.h -- C ABI of the GB300 nonoverlapping domain-decomposition ELM solver.
 *
 * The method (arxiv 2406.15959, Section 3 and Algorithm 1) solves a 2-D elliptic
 * problem L u = f in Omega, u = g on the boundary (Eq. (2.1)) with one random-feature
 * network per subdomain, u_s(x) = sum_j c^s_j tanh(w^s_j . x + b^s_j), joined by an
 * interface unknown u_Gamma.  The entry points follow Algorithm 1:
 *
 *   elm_ddm_setup     geometry of the decomposition (points, normals, interface map);
 *                     elm_ddm_setup_flux also takes explicit rows of A^s (cross points)
 *   elm_ddm_assemble  step (a): K^s, A^s of Eq. (3.1) from the hidden parameters theta^s
 *   elm_ddm_schur     step (b): local Householder QR of K^s, and the RHS-independent
 *                     part of step (c): assembly and Cholesky factorisation of the
 *                     Schur matrix of Eq. (3.5)
 *   elm_ddm_solve     the RHS part of step (c) (right-hand side of Eq. (3.5), triangular
 *                     solves for u_Gamma) and step (d): the local back-solves
 *                     c^s = K^{s+}(F^s - B^s u_Gamma) (Algorithm 1, last loop)
 *   elm_ddm_eval      u and grad u of the trained networks at arbitrary points
 *
 * Conventions
 * -----------
 * - All floating point is IEEE binary64.  Matrices are column-major.
 * - Subdomain s has rows ordered [interior | boundary | interface] (the row blocks of
 *   K^s in Section 3); counts[s] = {m_i, m_b, m_Gamma}; per-row arrays have a row
 *   stride of desc->m_max.
 * - Every interface unknown must be shared by exactly two subdomains (elm_ddm_setup), or
 *   by two to four (elm_ddm_setup_flux: a cross point, where several edges meet).
 *   Interface rows are grouped into "edges": maximal runs of a subdomain's interface rows
 *   with consecutive global unknowns and the same set of sharing subdomains.  Each edge
 *   must appear, with the same unknowns in the same order, in all those subdomains.
 * - Pointers documented "host" are read during the call only.  Pointers documented
 *   "device" are borrowed for the duration of the call (the kernels they feed are
 *   enqueued on the handle's stream; the caller keeps them alive and unmodified until
 *   that stream reaches the point of the call).  The handle owns all workspace.
 * - Compute entry points are asynchronous: they enqueue work on the stream given to
 *   elm_ddm_setup and return.  Numerical failures found by the kernels (non-SPD
 *   Schur matrix, exactly zero R diagonal, non-finite data) are recorded in a device
 *   status word and reported by elm_ddm_check, which synchronises the stream.
 * - Nothing in this library allocates or frees memory outside elm_ddm_setup and
 *   elm_ddm_destroy.
 */
#ifndef ELM_DDM_H
#define ELM_DDM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define ELM_DDM_OK            0
#define ELM_DDM_ERR_ARG       1  /* invalid argument or geometry */
#define ELM_DDM_ERR_STATE     2  /* entry points called out of order */
#define ELM_DDM_ERR_CUDA      3  /* a CUDA runtime call failed */
#define ELM_DDM_ERR_OOM       4  /* device allocation failed */
#define ELM_DDM_ERR_NONFINITE 5  /* NaN or Inf in theta, f/g or an intermediate */
#define ELM_DDM_ERR_RANK      6  /* some R^s has an exactly zero diagonal entry */
#define ELM_DDM_ERR_NOT_SPD   7  /* a Cholesky pivot of the Schur matrix was <= 0 */
#define ELM_DDM_ERR_CAPACITY  8  /* request larger than a no-allocation entry point's fixed scratch */
#define ELM_DDM_ERR_NOCONV    9  /* elm_ddm_solve_cg: tolerance not reached (outputs hold the last iterate) */
#define ELM_DDM_ERR_TIMEOUT  10  /* a bounded device-side wait gave up (see elm_ddm_set_wait_limit);
                                    the outputs of the affected call are invalid, the handle
                                    and the CUDA context stay usable */

/* elm_ddm_desc.flags */
#define ELM_DDM_FLAG_FP64_SIMT 1  /* run every dense update on the FP64 pipe (default: the
                                     large ones as FP64-accurate digit-split products on the
                                     BF16 tensor cores) */
#define ELM_DDM_FLAG_SCHUR_CG  2  /* the paper's interface solve only: elm_ddm_schur stops
                                     after D_s and M_s, the Schur matrix is neither formed
                                     nor factored (no n_gamma^2 workspace); solve with
                                     elm_ddm_solve_cg (elm_ddm_solve returns ERR_STATE) */
#define ELM_DDM_FLAG_DIRECT_ASSEMBLY 4  /* evaluate tanh for every entry of K^s and A^s.
                                     Default: where the collocation points of the
                                     subdomains share few x and y coordinates (the paper's
                                     grids), exp(2 z) is factored into per-neuron tables over
                                     those coordinates (same values to a few ulp) */

#define ELM_DDM_FLAG_MIXED 8  /* mixed precision: elm_ddm_schur factors the local matrices in
                                     low precision (FP32 Householder panels; BF16 digit-split
                                     products with FP32 accumulation keeping the 10 leading
                                     digit pairs, about 28 bits), assembles the Schur matrix and
                                     factors it in FP64; elm_ddm_solve refines the solution on
                                     FP64 residuals of the method's system (products with the
                                     FP64 K^s and A^s, kept from elm_ddm_assemble) until the
                                     relative u_Gamma correction is <= 1e-12, and falls back to
                                     the FP64 path (re-assembly, FP64 factorisation, direct
                                     solve) when refinement stalls.  elm_ddm_get_info keys
                                     10-13 report the steps, the fallback and the last
                                     correction.  Not with ELM_DDM_FLAG_FP64_SIMT or
                                     ELM_DDM_FLAG_SCHUR_CG; the CG entry points return
                                     ERR_STATE while the factorisation is the low-precision one.
                                     Needs about one more copy of K^s in device memory */

#define ELM_DDM_FLAG_NEURONS_PER_SUB 16  /* counts passed to elm_ddm_setup are [N][4] =
                                     {m_i, m_b, m_Gamma, n_s}: subdomain s has n_s <= n_neurons
                                     neurons (independent problems with different network sizes
                                     share one decomposition and one launch sequence).  Its
                                     columns n_s .. n_neurons-1 are identity columns on as many
                                     extra rows after the interface rows (no collocation point;
                                     m_max need not cover them): the least-squares solution of
                                     the other columns is unchanged, their weights come out 0,
                                     and their theta is ignored (set to 0 in the handle).
                                     Requires m_i + m_b + m_Gamma >= n_s */

#define ELM_DDM_FLAG_RIDGE 32  /* Tikhonov-regularised local least squares: every K^s gets
                                     n_s extra rows lambda_s I (after the pad rows), so each local
                                     problem becomes min |K c - F|^2 + lambda_s^2 |c|^2, with
                                     lambda_s = alpha * (largest column norm of K^s), alpha from
                                     elm_ddm_set_ridge (default 1e-14).  The paper does not name
                                     its local solver; at its Table 2 setup (rows barely more than
                                     neurons, K^s numerically rank deficient) the unregularised
                                     solution interpolates with huge weights, and this option
                                     reaches the paper's accuracy */

#define ELM_DDM_FLAG_BLOCK_JACOBI 64  /* elm_ddm_schur also inverts S's diagonal block of every
                                     interface edge (every edge at most 128 unknowns), the
                                     block-Jacobi preconditioner that elm_ddm_solve_pcg takes with
                                     jacobi = 2.  Not with ELM_DDM_FLAG_SCHUR_CG or
                                     ELM_DDM_FLAG_MIXED */

/* Differential operators. */
#define ELM_DDM_OP_POISSON 0  /* L = -Laplacian (Eq. (4.4)) */
#define ELM_DDM_OP_VARCOEF 1  /* L = -div(rho grad) (Section 4, the variable-coefficient
                                 problem); rho given by elm_ddm_set_coefficient */

typedef struct elm_ddm_handle elm_ddm_handle;

typedef struct elm_ddm_desc {
  int32_t n_sub;      /* N, number of subdomains (>= 1) */
  int32_t n_neurons;  /* n_N, hidden neurons per subdomain (>= 1) */
  int32_t m_max;      /* row stride of the per-row arrays; >= m_i + m_b + m_Gamma of every s */
  int32_t n_gamma;    /* number of global interface unknowns (0 when N == 1) */
  int32_t op;         /* ELM_DDM_OP_* */
  int32_t max_rhs;    /* largest nrhs elm_ddm_solve will be given, 1..64 (0 means 1) */
  int32_t flags;      /* ELM_DDM_FLAG_* */
} elm_ddm_desc;

/*
 * Geometry of the decomposition (Section 3: the point sets x^s_i, x^s_b, x^s_Gamma,
 * the outward normals n_s on Gamma, and the map B^s = [0; 0; -E_s] of interface rows
 * onto u_Gamma).
 *   counts  host int32  [N][3]        {m_i, m_b, m_Gamma}; each subdomain needs
 *                                     m_i + m_b + m_Gamma >= n_neurons (the premise of
 *                                     the full-rank proposition in Section 3); [N][4]
 *                                     {m_i, m_b, m_Gamma, n_s} with
 *                                     ELM_DDM_FLAG_NEURONS_PER_SUB
 *   xy      host double [N][m_max][2] collocation points
 *   nrm     host double [N][m_max][2] outward unit normal of interface rows (other rows ignored)
 *   dof     host int32  [N][m_max]    global interface unknown of interface rows, in
 *                                     [0, n_gamma) (other rows ignored)
 *   stream  cudaStream_t to enqueue all work on (NULL = legacy default stream)
 * Returns ELM_DDM_OK and a new handle in *out, or an error code (no handle is
 * created).  Allocates every device workspace the solver needs.
 */
int elm_ddm_setup(const elm_ddm_desc* desc, const int32_t* counts, const double* xy,
                  const double* nrm, const int32_t* dof, void* stream, elm_ddm_handle** out);

/*
 * Explicit rows of A^s, for decompositions with cross points (the remark in Section 3:
 * at an interface point where several edges meet, A^s gets one row per edge through the
 * point, with that edge's normal n_s).  The global flux conditions (rows of the global A)
 * are numbered 0 .. n_flux-1; each is the sum of exactly two rows, of the two subdomains
 * of its edge, and the method's pieces become M = A K^+ B = sum_s P_s^T M_s E_s and
 * h = sum_s P_s^T Y_s q_s, with P_s the map of the rows of A^s onto the conditions
 * (S and the right-hand side as in elm_ddm_schur / elm_ddm_solve).  elm_ddm_setup is the
 * case of one row per interface row, with that row's normal and its unknown's condition.
 *   n_flux  number of global flux conditions (>= 1 when n_gamma > 0)
 *   f_max   row stride of row, nrm, fdof (>= every count[s])
 *   count   host int32  [N]           rows of A^s
 *   row     host int32  [N][f_max]    interface row each A-row sits at, as an index among
 *                                     the subdomain's interface rows (0 <= row < m_Gamma)
 *   nrm     host double [N][f_max][2] its unit normal
 *   fdof    host int32  [N][f_max]    its flux condition, in [0, n_flux)
 * Rows of A^s are grouped like the interface rows: maximal runs with consecutive
 * conditions and the same other subdomain, appearing identically in both subdomains.
 */
typedef struct elm_ddm_flux_rows {
  int32_t n_flux;
  int32_t f_max;
  const int32_t* count;
  const int32_t* row;
  const double* nrm;
  const int32_t* fdof;
} elm_ddm_flux_rows;

/*
 * elm_ddm_setup with explicit rows of A^s (flux: see elm_ddm_flux_rows; NULL is
 * elm_ddm_setup itself).  With flux rows the per-row normals nrm are not read, interface
 * unknowns may be shared by up to four subdomains, ELM_DDM_BUF_A / _M export m_F x n_N /
 * m_F x m_Gamma (m_F = count[s]), and the CG interface solves are not available:
 * ELM_DDM_FLAG_SCHUR_CG, ELM_DDM_FLAG_MIXED and ELM_DDM_FLAG_BLOCK_JACOBI give ERR_ARG,
 * elm_ddm_solve_cg / elm_ddm_solve_pcg give ERR_STATE.
 */
int elm_ddm_setup_flux(const elm_ddm_desc* desc, const int32_t* counts, const double* xy,
                       const double* nrm, const int32_t* dof, const elm_ddm_flux_rows* flux,
                       void* stream, elm_ddm_handle** out);

/*
 * Step (a) of Algorithm 1 (Section 3, definitions of K^s and A^s): with
 * t = tanh(w.x + b), interior rows get L phi = 2|w|^2 t (1 - t^2), boundary and
 * interface rows get phi = t, and A^s rows get d phi/d n = (w.n)(1 - t^2).
 *   W  device double [N][n_neurons][2]  hidden weights w^s_j (global coordinates)
 *   b  device double [N][n_neurons]     hidden biases b^s_j
 * theta is copied into the handle (elm_ddm_eval uses it).
 */
int elm_ddm_assemble(elm_ddm_handle* h, const double* W, const double* b);

/*
 * Coefficient of ELM_DDM_OP_VARCOEF (Section 4: -div(rho grad u) = f).  Interior rows
 * of K^s become L phi = 2 rho |w|^2 t (1 - t^2) - (grad rho . w)(1 - t^2); rho is taken
 * continuous across the interfaces, so the flux condition rho du/dn reduces to the
 * normal-derivative rows A^s, which are unchanged.
 *   coef  device double [N][m_max][3]: (rho, d rho/dx, d rho/dy) at every row of every
 *         subdomain (only the interior rows are read); copied into the handle.
 * Required before elm_ddm_assemble for ELM_DDM_OP_VARCOEF (assemble returns ERR_STATE
 * without it); returns ERR_ARG for ELM_DDM_OP_POISSON.  Non-finite values make
 * elm_ddm_assemble flag ELM_DDM_ERR_NONFINITE (reported by elm_ddm_check).
 */
int elm_ddm_set_coefficient(elm_ddm_handle* h, const double* coef);

/*
 * Step (b) and the RHS-independent part of step (c): Householder QR K^s = Q_s R_s
 * (reflectors kept for elm_ddm_solve), Q_G = interface rows of Q_s,
 * Y_s = A^s R_s^{-1}, D_s = I - Q_G Q_G^T, M_s = -Y_s Q_G^T, the Schur matrix
 * S = sum_s E_s^T D_s E_s + M^T M of Eq. (3.5) with M = sum_s E_s^T M_s E_s, and its
 * Cholesky factor S = L L^T.  Requires elm_ddm_assemble.
 */
int elm_ddm_schur(elm_ddm_handle* h);

/*
 * RHS part of step (c) and step (d), for nrhs right-hand sides at once:
 * q_s = Q_s^T F^s, rhs = sum_s E_s^T Q_G q_s + M^T h with h = sum_s E_s^T Y_s q_s,
 * u_Gamma = S^{-1} rhs, c^s = R_s^{-1}(q_s + Q_G^T E_s u_Gamma).
 *   rhs      device double [nrhs][N][m_max]  f at interior rows, g at boundary rows;
 *                                           interface rows and padding are ignored (F^s
 *                                           is zero there, Section 3)
 *   u_gamma  device double [nrhs][n_gamma]   output (may be NULL)
 *   c        device double [nrhs][N][n_neurons] output weights c^s (must not be NULL)
 * Requires elm_ddm_schur.  1 <= nrhs <= desc->max_rhs.
 */
int elm_ddm_solve(elm_ddm_handle* h, const double* rhs, int nrhs, double* u_gamma, double* c);

/*
 * The paper's interface solve (Section 4: the Schur system of Eq. (3.5) by conjugate
 * gradients to a relative residual): as elm_ddm_solve, but u_Gamma comes from
 * unpreconditioned CG started at zero, with S applied from the stored local pieces,
 * S p = sum_s E_s^T D_s E_s p + M^T (M p), M p = sum_s E_s^T M_s E_s p (never formed).
 * Every right-hand side stops once |r| <= tol |rhs|.
 *   tol    relative residual, finite and > 0 (the paper uses 1e-9)
 *   maxit  iteration limit, >= 1
 *   iters  host int (may be NULL): the largest number of CG steps any right-hand side took
 * Synchronises with the host every 16 steps to test convergence.  Returns ELM_DDM_OK, or
 * ELM_DDM_ERR_NOCONV when some right-hand side did not reach tol within maxit steps (or
 * CG broke down: p^T S p <= 0); its outputs then hold the last iterate.  Works after
 * elm_ddm_schur with or without ELM_DDM_FLAG_SCHUR_CG.
 */
int elm_ddm_solve_cg(elm_ddm_handle* h, const double* rhs, int nrhs, double tol, int maxit,
                     double* u_gamma, double* c, int* iters);

/*
 * As elm_ddm_solve_cg, started from an initial guess and optionally preconditioned (the
 * paper names no preconditioner; a learned initial guess is the warm start of the
 * learned-interface extension):
 *   x0      device double [nrhs][n_gamma] initial u_Gamma in the caller's order, or NULL (zero)
 *   jacobi  1: preconditioner diag(S)^{-1} (needs the assembled S, i.e. not
 *           ELM_DDM_FLAG_SCHUR_CG; ERR_STATE otherwise); 2: block-Jacobi, the inverse of
 *           S's diagonal block of every interface edge (needs ELM_DDM_FLAG_BLOCK_JACOBI;
 *           ERR_STATE otherwise); 0: none.  Other values: ERR_ARG
 * The stopping rule is on the true residual of the recurrence, |r| <= tol |rhs|, checked
 * also at the start (a guess that already meets it takes 0 steps).
 */
int elm_ddm_solve_pcg(elm_ddm_handle* h, const double* rhs, int nrhs, const double* x0, int jacobi,
                      double tol, int maxit, double* u_gamma, double* c, int* iters);

/*
 * u(x) = sum_j c^s_j tanh(w^s_j . x + b^s_j) and grad u at npts points, s = owner[i].
 *   xy     device double [npts][2]
 *   owner  device int32  [npts]   subdomain index of each point, in [0, N)
 *   c      device double [N][n_neurons]
 *   u      device double [npts]   output
 *   grad   device double [npts][2] output (may be NULL)
 * Requires elm_ddm_assemble (for theta).
 */
int elm_ddm_eval(elm_ddm_handle* h, int npts, const double* xy, const int32_t* owner,
                 const double* c, double* u, double* grad);

/*
 * Synchronises the handle's stream and returns the first failure the kernels
 * recorded since the previous check (ELM_DDM_ERR_NONFINITE, _RANK, _NOT_SPD, _TIMEOUT in
 * that order of precedence), a pending CUDA error (ELM_DDM_ERR_CUDA), or ELM_DDM_OK.
 * Clears the status word.
 */
int elm_ddm_check(elm_ddm_handle* h);

/* Internal matrices that elm_ddm_export can copy out (for inspection and tests). */
#define ELM_DDM_BUF_K 0  /* m_s x (n_N + m_Gamma): [K^s | J] after assemble; after schur the
                            Householder factors: R on and above the diagonal, reflectors
                            below it, Q_G^T in rows 0..n_N-1 of the last m_Gamma columns */
#define ELM_DDM_BUF_A 1  /* m_F x n_N: A^s after assemble, Y_s = A^s R_s^{-1} after schur
                            (m_F = m_Gamma, or the explicit rows of elm_ddm_setup_flux) */
#define ELM_DDM_BUF_D 2  /* m_Gamma x m_Gamma: D_s = I - Q_G Q_G^T (after schur) */
#define ELM_DDM_BUF_M 3  /* m_F x m_Gamma: M_s = -Y_s Q_G^T (after schur) */
#define ELM_DDM_BUF_L 4  /* n_gamma x n_gamma: lower Cholesky factor of S in the internal
                            interface order (elm_ddm_interface_order), after schur; s ignored;
                            the strict upper triangle is unspecified */

/*
 * Collocation points of the decomposition as the handle holds them (Section 3: the
 * point sets x^s_i, x^s_b, x^s_Gamma, and the outward normals n_s on Gamma).  The
 * geometry enters through elm_ddm_setup as explicit point arrays, so any point layout
 * (the paper's global grid, per-subdomain grids, random points) and any batch of
 * independent problems can be described; this call returns it in per-kind form.
 *   kind    ELM_DDM_PTS_INTERIOR, _BOUNDARY, _INTERFACE (points) or _NORMALS (the outward
 *           normal of every interface point)
 *   xy      device double [N][kmax][2], kmax = the largest count of that kind over the
 *           subdomains; row i of subdomain s is its i-th point of the kind (in the order
 *           of elm_ddm_setup's rows), rows past counts[s] are zero.  May be NULL: only
 *           the counts are returned.  Written on the handle's stream.
 *   counts  host int32 [N] (may be NULL): number of points of the kind per subdomain.
 * Returns ELM_DDM_ERR_ARG for an unknown kind.
 */
#define ELM_DDM_PTS_INTERIOR  0
#define ELM_DDM_PTS_BOUNDARY  1
#define ELM_DDM_PTS_INTERFACE 2
#define ELM_DDM_PTS_NORMALS   3
int elm_ddm_get_points(elm_ddm_handle* h, int kind, double* xy, int32_t* counts);

/*
 * Limit of the bounded device-side waits of elm_ddm_solve's triangular solves (the grid
 * barriers between the block steps of the cooperative forward and backward substitution
 * kernels; the paper has no counterpart: failure detection).  A barrier that has not been
 * released within `seconds` of wall time makes every block of the kernel record the
 * timeout and return; elm_ddm_check then reports ELM_DDM_ERR_TIMEOUT and the solve's
 * outputs are invalid, while the handle stays usable.
 *   seconds       0 .. 60 (default 2)
 *   hold_release  0 normally; 1 makes every barrier wait for one arrival more than the
 *                 kernel's grid supplies, so the wait runs out for certain (a test hook
 *                 for the timeout path; no asynchronous copy is in flight at these waits)
 * Applies to later calls; host-only.  elm_ddm_get_info key 9 says whether this handle's
 * solves use the cooperative kernels (when no co-resident grid fits, one launch per block
 * step is used instead and there is no device-side wait).
 */
int elm_ddm_set_wait_limit(elm_ddm_handle* h, double seconds, int hold_release);

/*
 * Regularisation parameter of ELM_DDM_FLAG_RIDGE (see the flag): alpha in [0, 1), applied
 * from the next elm_ddm_assemble.  ERR_STATE without the flag.  The paper has no
 * counterpart (its local solver is unspecified).
 */
int elm_ddm_set_ridge(elm_ddm_handle* h, double alpha);

/*
 * Tile choices of the factorisation (the paper has no counterpart; performance only, the
 * results are the same up to rounding).  Host-only; applies to later calls.
 *   ELM_DDM_TUNE_PANEL_CTAS  CTAs per subdomain of the FP64 Householder panel: 0 (default)
 *                            the smallest cluster whose shared memory holds the panel (4 or
 *                            8), 4 or 8 to ask for one (8 gives small batches more SMs; a
 *                            size that does not fit is replaced by the default)
 *   ELM_DDM_TUNE_UPD_GRID    grid cap of the persistent tensor-core products: 0 (default)
 *                            one CTA per SM, else at most this many CTAs
 * Returns ELM_DDM_ERR_ARG for an unknown key or value.  An autotuner that times these per
 * shape class is paper_2406_15959_gb300/autotune.py.
 */
#define ELM_DDM_TUNE_PANEL_CTAS 0
#define ELM_DDM_TUNE_UPD_GRID   1
int elm_ddm_set_tuning(elm_ddm_handle* h, int key, int value);

/*
 * The Schur matrix is assembled and factored with its interface unknowns renumbered
 * (reverse Cuthill-McKee on the interface edges, so the Cholesky factor stays inside a
 * narrow envelope).  order (host int32 [n_gamma]) receives, for every caller unknown g,
 * its internal index.  elm_ddm_solve's u_gamma is always in the caller's numbering.
 */
int elm_ddm_interface_order(const elm_ddm_handle* h, int32_t* order);

/*
 * Copies internal matrix `what` (ELM_DDM_BUF_*) of subdomain s, column-major, into the
 * device buffer dst with leading dimension ld_dst (>= its row count).  Enqueued on the
 * handle's stream.
 */
int elm_ddm_export(elm_ddm_handle* h, int what, int s, double* dst, int ld_dst);

/*
 * Queries.  key: 0 = n_gamma, 1 = device workspace bytes, 2 = number of launch calls
 * (one per kernel class invocation, some launch several kernels) enqueued since setup,
 * 3 = number of Schur-matrix edges (interface blocks), 4 = m_max, 5 = n_neurons,
 * 6 = n_sub, 7 = CUDA kernels launched by the library in this process (all handles),
 * 8 = 1 if elm_ddm_assemble uses the factored activation tables, else 0,
 * 9 = 1 if elm_ddm_solve's triangular solves run as one cooperative launch each, else 0,
 * 10 = refinement steps of the last mixed-precision solve, 11 = 1 if that solve stalled and
 * fell back to the FP64 path, 12 = its last relative u_Gamma correction (the c correction
 * without interface unknowns), the solve's error estimate, 13 = 1 while the current
 * factorisation is the low-precision one.
 */
int elm_ddm_get_info(const elm_ddm_handle* h, int key, double* value);

/*
 * Per-launch device timing.  While enabled, every kernel launch of the handle is
 * bracketed by a pair of CUDA events on its stream (events are created on first use
 * and reused; no device memory is allocated).  elm_ddm_profile_report synchronises the
 * stream and writes a JSON object {"<kernel class>": {"launches": L, "ms": T,
 * "flops": F, "bytes": B}, ..., "_dropped": D} into buf (NUL-terminated), where F and B
 * are the algorithmic flops and HBM bytes of the dense-update and operand-split launches
 * (0 for other classes), then clears the records.  Returns ELM_DDM_ERR_ARG if buf is too
 * small.
 */
int elm_ddm_profile(elm_ddm_handle* h, int enable);
int elm_ddm_profile_report(elm_ddm_handle* h, char* buf, int buflen);

/*
 * Restrict per-launch profiling to one kernel class (the names elm_ddm_profile_report
 * prints; NULL or "" restores all classes), so that a timed region can measure one class's
 * launches without bracketing every other launch with events.  Host-only; the paper has
 * no counterpart (measurement support).  Returns ELM_DDM_ERR_ARG for a NULL handle.
 */
int elm_ddm_profile_only(elm_ddm_handle* h, const char* kernel_class);

/*
 * No-allocation Cholesky solve.  The paper has no counterpart: this entry point exists
 * for callers that cannot call cudaMalloc -- code running while a CUDA graph is being
 * captured in global mode (an allocation there invalidates the capture), hosts that route
 * all device memory through their own pool and forbid hidden allocations, real-time
 * loops.  It solves L L^T u = b for nrhs right-hand sides with the same blocked
 * substitution kernels as elm_ddm_solve's interface solve, needs no handle, and calls no
 * cudaMalloc, cudaFree or allocating library routine: its working vectors live in one
 * fixed device array of 2 * ELM_DDM_NOALLOC_MAX_ELEMS doubles (2 MiB) that every GPU
 * loading the library holds until the process exits.
 *   L     device double, lower Cholesky factor (n x n, column-major, leading dimension
 *         ld >= n; the strict upper triangle is not read) -- e.g. elm_ddm_export's
 *         ELM_DDM_BUF_L
 *   b     device double [nrhs][n] right-hand sides (read only; may alias u)
 *   u     device double [nrhs][n] solutions
 *   stream cudaStream_t to enqueue on (NULL = legacy default stream)
 * b and u are in the order of L's rows.  With the factor that ELM_DDM_BUF_L exports, that
 * is the handle's internal interface order: unknown g of the caller's numbering is entry
 * order[g] of b and u, with order from elm_ddm_interface_order; a vector in the caller's
 * order (as elm_ddm_solve takes and returns them) must be permuted first.
 * Returns ELM_DDM_ERR_ARG for NULL pointers, n < 1, nrhs < 1, nrhs > 65535 or ld < n;
 * ELM_DDM_ERR_CAPACITY if n * nrhs > ELM_DDM_NOALLOC_MAX_ELEMS (nothing is enqueued
 * in either case); ELM_DDM_ERR_CUDA if a launch or copy fails.  Asynchronous otherwise.
 * The first call on each device looks up the array's device address (once per device,
 * with that device current) and keeps it for the life of the process; make that first
 * call before any stream capture begins.  The kept address does not survive
 * cudaDeviceReset (or anything else that unloads the library's module from the device):
 * do not call this entry point on a device after resetting it.
 * All calls share the array and it keeps the previous call's contents (nothing in it
 * needs to start at zero: each call overwrites what it reads).  Calls whose work
 * overlaps on the GPU -- on different streams, or from different host threads without
 * ordering -- race on the array; order them on one stream.
 */
#define ELM_DDM_NOALLOC_MAX_ELEMS 131072
int elm_ddm_chol_solve_noalloc(const double* L, int n, int ld, const double* b, int nrhs,
                               double* u, void* stream);

/*
 * FP64-accurate matrix product on the BF16 tensor cores: the digit-split scheme the
 * solver runs its dense updates with (QR trailing updates, D_s and M_s of Eq. (3.5), the
 * Schur matrix's M^T M blocks and Cholesky SYRK), as a stand-alone call.  The paper has
 * no counterpart (it states these products in FP64; this is how they are computed here):
 *   C[i*c_rs + j*c_cs] = alpha * sum_k A(i,k) B(j,k) + beta * C[i*c_rs + j*c_cs],
 *   A(i,k) = A[i*a_rs + k*a_ks],  B(j,k) = B[j*b_rs + k*b_ks],  0 <= i < M, 0 <= j < N.
 * Each row of A and of B is written as 2^(E-1022) sum_{p=1..7} d_p 2^(1-8p) with integer
 * digits |d_p| <= 128 (E its largest biased exponent; truncation below 2^-54 of the
 * row's largest magnitude), the 28 digit pairs with p + q <= 8 are multiplied exactly on
 * the tensor cores (the pairs not formed weigh at most 6 * 2^-54 of the row maxima's
 * product per term), and each element is rounded once.  The error bound is therefore
 * normwise per row and column, not componentwise like an FP64 GEMM's:
 *   |C_ij - (A B^T)_ij| <= 2^-53 |(A B^T)_ij|
 *                          + 2^-54 (max_k |A(i,k)| sum_k |B(j,k)| + max_k |B(j,k)| sum_k |A(i,k)|)
 *                          + 6 K 2^-54 max_k |A(i,k)| max_k |B(j,k)|
 * (with beta != 0 or |alpha| != 1 one more rounding of the update; for K > 7936 up to two
 * more roundings of the result): entries far below the largest of their row and column
 * carry no relative accuracy of their own.
 *   kernel  ELM_DDM_GEMM_TILE32      one CTA per 128 x 32 output tile, K <= 65536
 *           ELM_DDM_GEMM_TILE64      one CTA per 128 x 64 output tile, K <= 128
 *           ELM_DDM_GEMM_PERSISTENT  one CTA per SM over a table of 128 x 32 tiles, K <= 128
 *           ELM_DDM_GEMM_FUSED_SPLIT A split inside the product kernel: a_ks = 1, N <= 32,
 *                                    K <= 65536, alpha = 1, beta = 0
 *           ELM_DDM_GEMM_FUSED_SPLIT_B  B split inside the product kernel: b_ks = 1,
 *                                    M <= 128, K <= 65536, alpha = 1, beta = 0
 *           ELM_DDM_GEMM_PERSISTENT_WIDE  one CTA per SM over 128 x 64 tiles (the QR's
 *                                    outer-block update): K <= 128, alpha = +-1, beta = 1
 *   A, B, C  device double (C must not overlap A or B)
 *   workspace  device memory, 256-byte aligned, of at least
 *              elm_ddm_fp64_gemm_workspace(kernel, M, N, K) bytes (0 for an unsupported
 *              shape); owned by the caller, free again when the call returns
 *   stream  cudaStream_t (NULL = legacy default stream)
 * Synchronises the stream before returning.  Returns ELM_DDM_ERR_ARG for an unsupported
 * kernel or shape, NULL pointers, a short or misaligned workspace;
 * ELM_DDM_ERR_TIMEOUT if a bounded wait of the product kernel gave up; ELM_DDM_ERR_CUDA.
 */
#define ELM_DDM_GEMM_TILE32      0
#define ELM_DDM_GEMM_TILE64      1
#define ELM_DDM_GEMM_PERSISTENT  2
#define ELM_DDM_GEMM_FUSED_SPLIT 3
#define ELM_DDM_GEMM_FUSED_SPLIT_B 4
#define ELM_DDM_GEMM_PERSISTENT_WIDE 5
size_t elm_ddm_fp64_gemm_workspace(int kernel, int M, int N, int K);
int elm_ddm_fp64_gemm(int kernel, int M, int N, int K, double alpha, const double* A,
                      long long a_rs, long long a_ks, const double* B, long long b_rs,
                      long long b_ks, double beta, double* C, long long c_rs, long long c_cs,
                      void* workspace, size_t workspace_bytes, void* stream);

/* Numerical self-test of a device routine the solver uses, element by element:
 * y[i] = f(x[i]) for 0 <= i < n, x and y device double arrays (caller-owned).
 *   which  ELM_DDM_SELFTEST_PIVOT_RCP: the reciprocal of the Schur Cholesky's pivots
 *          (one third-order iteration from an FP32 seed; defined for positive normal x,
 *          within two units in the last place of 1/x)
 * Synchronises the stream.  Returns ELM_DDM_ERR_ARG for an unknown `which`, NULL arrays or
 * n < 0; ELM_DDM_ERR_CUDA. */
#define ELM_DDM_SELFTEST_PIVOT_RCP 0
int elm_ddm_selftest(int which, const double* x, double* y, int n, void* stream);

/* Frees all device workspace and the handle.  Synchronises the stream first. */
int elm_ddm_destroy(elm_ddm_handle* h);

/* Message of the last failure on this handle ("" if none).  h may be NULL, in which
 * case the message of the last failed elm_ddm_setup in this process is returned. */
const char* elm_ddm_last_error(const elm_ddm_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* ELM_DDM_H */
