"""Plain FP64 CPU oracle for the nonoverlapping DDM for ELMs (arxiv 2406.15959).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call this
module: only the tests, the package's smoke check and the CPU-baseline leg of
the benchmark do.  It shares no code with the CUDA path; the only thing both
consume is the seeded input generator (``paper_2406_15959_gb300.workload``),
which holds none of the method's arithmetic.

What is computed (Section 3).  For every subdomain s the local network is
u_s(x) = sum_j c^s_j phi^s_j(x) with phi^s_j(x) = tanh(w^s_j . x + b^s_j).  The
collocation blocks K^s, A^s, B^s, F^s of Eq. (3.1) are assembled, and the
result is the least-squares solution of the *eliminated* system Eq. (3.3)
(the paper solves that system instead of the LS problem of Eq. (3.1)), i.e.
u_Gamma solves the Schur complement system Eq. (3.5) and
c^s = K^{s+} (F^s - B^s u_Gamma) (Algorithm 1, last loop).

Three routes compute that result:

* ``solve``: the DDM route of Algorithm 1, per subdomain.  K^s = Q_s R_s by
  Householder QR (LAPACK through numpy), K^{s+} = R_s^{-1} Q_s^T.  Writing
  E_s for the 0/1 map of subdomain s's interface rows onto the global
  unknowns (so B^s = [0; 0; -E_s] and the global A = sum_s E_s^T A^s), the
  pieces of Eq. (3.5) are
      B^T (I - K K^+) B          = sum_s E_s^T (I - Q_G Q_G^T) E_s
      A K^+ B            =: M    = sum_s E_s^T (-Y_s Q_G^T) E_s,  Y_s = A^s R_s^{-1}
      B^T (I - K K^+) F          = sum_s E_s^T Q_G q_s,            q_s = Q_s^T F^s
      A K^+ F            =: h    = sum_s E_s^T Y_s q_s
  where Q_G are the interface rows of Q_s, so that
      S = B^T (I + K^{+T} A^T A K^+ - K K^+) B = sum_s E_s^T D_s E_s + M^T M,
      rhs = sum_s E_s^T Q_G q_s + M^T h.
  S is solved by Cholesky (the paper says the system is SPD), and the local
  weights come from c^s = R_s^{-1} (q_s + Q_G^T E_s u_Gamma).
* ``monolithic_ls``: the dense LS problem of Eq. (3.3) itself (tiny inputs).
* ``normal_equations``: the dense system Eq. (3.4) solved by LU (tiny inputs).

Readings of the paper used here (the paper gives A^s, B^s only for N = 2):
one A-row per global interface point, carrying the outward-normal derivatives
of the two subdomains that share it; L = -Laplacian (Eq. (4.4)); all rows have
unit weight; the Schur system is solved directly instead of by CG.

Cross points (the remark in Section 3).  Where several edges meet at an
interface point, that point is one unknown shared by all its subdomains, and
A^s gets one row per edge of s through it, with that edge's normal.  The
global flux conditions are then no longer one per unknown: with P_s the 0/1
map of the rows of A^s onto the global conditions (each condition sums the
rows of the two subdomains of its edge), A = sum_s P_s^T A^s and
      M = A K^+ B = sum_s P_s^T (-Y_s Q_G^T) E_s,   h = sum_s P_s^T Y_s q_s,
with S and rhs as above.  Without cross points P_s = E_s.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


# --------------------------------------------------------------------------
# Step (a): local collocation blocks, Section 3 (definition of K^s, A^s, F^s)
# --------------------------------------------------------------------------

def hidden(W, b, xy):
    """phi_j(x) = tanh(w_j . x + b_j) for points xy [m, 2] and neurons W [n, 2], b [n].
    Returns t [m, n]."""
    z = xy @ W.T + b[None, :]
    return np.tanh(z)


def assemble_local(xy, nrm, counts, W, b, coef=None, flux=None):
    """K^s [m, n] and A^s [m_F, n] of subdomain s (Section 3).

    Rows of K^s: L phi_j at interior points, phi_j at boundary points, phi_j at
    interface points.  With t = tanh(w.x + b):
      d phi / dx_d = w_d (1 - t^2),  d^2 phi / dx_d^2 = -2 w_d^2 t (1 - t^2),
      L phi = -Laplacian phi = 2 |w|^2 t (1 - t^2),
      d phi / d n  = (w . n)(1 - t^2)   (rows of A^s, outward normal n).
    With a variable coefficient (Section 4, -div(rho grad u) = f; coef = rows of
    (rho, d rho/dx, d rho/dy) at the points):
      L phi = -rho Laplacian phi - grad rho . grad phi
            = 2 rho |w|^2 t (1 - t^2) - (grad rho . w)(1 - t^2).
    The transmission rows are unchanged: with rho continuous across Gamma the flux
    condition rho du/dn is the normal-derivative condition.
    flux: None (one A-row per interface row, with its normal nrm) or (rows, normals):
    the A-rows at interface rows ``rows`` (indices among the interface rows) with those
    normals (the corner rule of the remark in Section 3).
    """
    mi, mb, mg = (int(v) for v in counts)
    m = mi + mb + mg
    t = hidden(W, b, xy[:m])
    wsq = (W * W).sum(axis=1)
    K = t.copy()
    K[:mi] = 2.0 * wsq[None, :] * t[:mi] * (1.0 - t[:mi] ** 2)
    if coef is not None:
        rho, grho = coef[:mi, 0:1], coef[:mi, 1:3]
        K[:mi] = rho * K[:mi] - (grho @ W.T) * (1.0 - t[:mi] ** 2)
    tg = t[mi + mb:m]
    if flux is None:
        wn = nrm[mi + mb:m] @ W.T                 # [m_G, n]: w_j . n_i
        A = wn * (1.0 - tg ** 2)
    else:
        rows, fn = flux
        A = (np.asarray(fn) @ W.T) * (1.0 - tg[np.asarray(rows, np.int64)] ** 2)
    return K, A


def flux_rows(geom, s):
    """(rows, normals, conditions) of the A-rows of subdomain s: the explicit ones of
    geom.flux, else one per interface row with its normal and its unknown."""
    mi, mb, mg = (int(v) for v in geom.counts[s])
    if getattr(geom, "flux", None) is None:
        return (np.arange(mg), geom.nrm[s, mi + mb:mi + mb + mg],
                geom.dof[s, mi + mb:mi + mb + mg].astype(np.int64))
    f = geom.flux
    c = int(f.count[s])
    return f.row[s, :c].astype(np.int64), f.nrm[s, :c], f.fdof[s, :c].astype(np.int64)


def n_flux(geom):
    """Number of global flux conditions (rows of A)."""
    return geom.n_gamma if getattr(geom, "flux", None) is None else int(geom.flux.n_flux)


def rhs_local(rhs_row, counts):
    """F^s = [f(x_i); g(x_b); 0] (Section 3)."""
    mi, mb, mg = (int(v) for v in counts)
    F = np.zeros(mi + mb + mg)
    F[:mi + mb] = rhs_row[:mi + mb]
    return F


# --------------------------------------------------------------------------
# Steps (b)-(d): Algorithm 1 with the Schur system Eq. (3.5)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Local:
    """Per-subdomain factorisation pieces used by Eq. (3.5)."""
    K: np.ndarray
    A: np.ndarray
    Q: np.ndarray       # thin Q of K^s
    R: np.ndarray       # upper triangular R of K^s
    dof: np.ndarray     # global interface unknowns of the interface rows
    mi_mb: int          # first interface row
    QG: np.ndarray      # interface rows of Q
    Y: np.ndarray       # A^s R^{-1}
    D: np.ndarray       # I - Q_G Q_G^T
    M: np.ndarray       # -Y Q_G^T
    fdof: np.ndarray = None   # global flux condition of every row of A^s (P_s)


def factor_local(K, A, dof, mi_mb, fdof=None):
    """Householder QR of K^s and the local pieces of Eq. (3.5)."""
    Q, R = np.linalg.qr(K, mode="reduced")
    QG = Q[mi_mb:]
    # Y = A R^{-1}  <=>  R^T Y^T = A^T
    Y = sla.solve_triangular(R, A.T, trans="T", lower=False).T if A.size else np.zeros_like(A)
    D = np.eye(len(dof)) - QG @ QG.T
    M = -(Y @ QG.T)
    return Local(K, A, Q, R, dof, mi_mb, QG, Y, D, M, dof if fdof is None else fdof)


def schur_matrix(locs, n_gamma, n_flux=None):
    """S = sum_s E_s^T D_s E_s + M^T M with M = sum_s P_s^T M_s E_s (Eq. (3.5)); P_s = E_s
    without cross points."""
    n_flux = n_gamma if n_flux is None else n_flux
    S = np.zeros((n_gamma, n_gamma))
    rows, cols, vals = [], [], []
    for L in locs:
        if len(L.dof) == 0:
            continue
        S[np.ix_(L.dof, L.dof)] += L.D
        rr, cc = np.meshgrid(L.fdof, L.dof, indexing="ij")
        rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append(L.M.ravel())
    M = None
    if rows:
        M = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(n_flux, n_gamma)).tocsr()
        S += (M.T @ M).toarray()
    return S, M


def schur_rhs(locs, qs, M, n_gamma, n_flux=None):
    """rhs = sum_s E_s^T Q_G q_s + M^T h, h = sum_s P_s^T Y_s q_s (Eq. (3.5))."""
    r = np.zeros(n_gamma)
    h = np.zeros(n_gamma if n_flux is None else n_flux)
    for L, q in zip(locs, qs):
        if len(L.dof) == 0:
            continue
        np.add.at(r, L.dof, L.QG @ q)
        np.add.at(h, L.fdof, L.Y @ q)
    if M is not None:
        r += M.T @ h
    return r


def back_solve(L, q, u_gamma):
    """c^s = K^{s+}(F^s - B^s u_Gamma) = R^{-1}(q_s + Q_G^T E_s u_Gamma) (Algorithm 1)."""
    v = q + (L.QG.T @ u_gamma[L.dof] if len(L.dof) else 0.0)
    return sla.solve_triangular(L.R, v, lower=False)


@dataclasses.dataclass
class Result:
    u_gamma: np.ndarray       # [n_gamma]
    c: np.ndarray             # [N, n]
    S: np.ndarray             # Schur matrix
    rhs: np.ndarray           # Schur right-hand side
    rdiag_ratio: np.ndarray   # min|R_ii| / max|R_ii| per subdomain
    locs: list


def ridge_rows(K, F, first_ifc, alpha):
    """Tikhonov regularisation of a local least-squares problem (the library's
    ELM_DDM_FLAG_RIDGE; the paper does not name its local solver): min |K c - F|^2 +
    lambda^2 |c|^2 with lambda = alpha * the largest column norm of K, written as the least
    squares problem of K stacked on lambda I (F stacked on 0).  The rows go before the
    interface rows, which stay last; returns (K', F', index of the first interface row)."""
    m, n = K.shape
    lam = alpha * np.sqrt((K * K).sum(axis=0)).max()
    Ka = np.vstack([K[:first_ifc], lam * np.eye(n), K[first_ifc:]])
    Fa = np.concatenate([F[:first_ifc], np.zeros(n), F[first_ifc:]])
    return Ka, Fa, first_ifc + n


def solve(geom, W, b, rhs_rows, keep=True, coef=None, ridge=None):
    """Algorithm 1: assemble, factor, solve Eq. (3.5) by Cholesky, back-solve.
    coef: None (-Laplacian) or [N, m_max, 3] rows of (rho, grad rho).
    ridge: None, or alpha of the Tikhonov-regularised local problems (ridge_rows)."""
    N = geom.n_sub
    locs, qs = [], []
    for s in range(N):
        mi, mb, mg = (int(v) for v in geom.counts[s])
        frow, fnrm, fdof = flux_rows(geom, s)
        K, A = assemble_local(geom.xy[s], geom.nrm[s], geom.counts[s], W[s], b[s],
                              None if coef is None else coef[s], (frow, fnrm))
        dof = geom.dof[s, mi + mb:mi + mb + mg].astype(np.int64)
        F = rhs_local(rhs_rows[s], geom.counts[s])
        i0 = mi + mb
        if ridge is not None:
            K, F, i0 = ridge_rows(K, F, mi + mb, ridge)
        L = factor_local(K, A, dof, i0, fdof)
        locs.append(L)
        qs.append(L.Q.T @ F)
    S, M = schur_matrix(locs, geom.n_gamma, n_flux(geom))
    r = schur_rhs(locs, qs, M, geom.n_gamma, n_flux(geom))
    if geom.n_gamma:
        Lc = np.linalg.cholesky(S)
        y = sla.solve_triangular(Lc, r, lower=True)
        u = sla.solve_triangular(Lc.T, y, lower=False)
    else:
        u = np.zeros(0)
    c = np.stack([back_solve(L, q, u) for L, q in zip(locs, qs)])
    ratio = np.array([np.abs(np.diag(L.R)).min() / np.abs(np.diag(L.R)).max() for L in locs])
    return Result(u, c, S, r, ratio, locs if keep else [])


def cg_solve(S, rhs, tol, maxit):
    """Conjugate gradients (Hestenes and Stiefel) for the SPD interface system S u = rhs,
    the solver the paper uses for Eq. (3.5) (Section 4: stopped at a relative residual
    of 1e-9).  Unpreconditioned, started at u = 0, stopped at the first step with
    |r| <= tol |rhs|.  Returns (u, steps, converged)."""
    b = np.asarray(rhs, dtype=np.float64)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    target = tol * tol * rr
    if rr == 0.0:
        return x, 0, True
    for k in range(1, maxit + 1):
        q = S @ p
        alpha = rr / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        rr_new = float(r @ r)
        if rr_new <= target:
            return x, k, True
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x, maxit, False


def evaluate(W, b, c, xy, owner):
    """u(x) = sum_j c^s_j tanh(w^s_j . x + b^s_j) and grad u, s = owner of x."""
    u = np.zeros(len(xy))
    g = np.zeros((len(xy), 2))
    for s in np.unique(owner):
        idx = np.nonzero(owner == s)[0]
        t = hidden(W[s], b[s], xy[idx])
        u[idx] = t @ c[s]
        d = (1.0 - t * t) * c[s][None, :]
        g[idx] = d @ W[s]
    return u, g


def rel_errors(u, g, u_ex, g_ex):
    """Discrete relative L2 and H1 errors on the test points."""
    l2 = np.linalg.norm(u - u_ex) / np.linalg.norm(u_ex)
    num = np.sum((u - u_ex) ** 2) + np.sum((g - g_ex) ** 2)
    den = np.sum(u_ex ** 2) + np.sum(g_ex ** 2)
    return l2, float(np.sqrt(num / den))


# --------------------------------------------------------------------------
# Global dense operators of Eqs. (3.1)-(3.4), for brute-force checks (tiny inputs)
# --------------------------------------------------------------------------

def global_blocks(geom, W, b, rhs_rows, coef=None):
    """Dense K = diag(K^s), B = [B^s], A = [P_s^T A^s] (one row per flux condition: per
    interface unknown without cross points), F = [F^s] of Eq. (3.2)."""
    Ks, As, Fs, Bs = [], [], [], []
    n = W.shape[1]
    N = geom.n_sub
    for s in range(N):
        mi, mb, mg = (int(v) for v in geom.counts[s])
        frow, fnrm, fdof = flux_rows(geom, s)
        K, A = assemble_local(geom.xy[s], geom.nrm[s], geom.counts[s], W[s], b[s],
                              None if coef is None else coef[s], (frow, fnrm))
        Ks.append(K)
        Fs.append(rhs_local(rhs_rows[s], geom.counts[s]))
        Bs_ = np.zeros((mi + mb + mg, geom.n_gamma))
        Ag = np.zeros((n_flux(geom), n))
        for r in range(mg):
            Bs_[mi + mb + r, int(geom.dof[s, mi + mb + r])] = -1.0
        for r in range(len(fdof)):
            Ag[int(fdof[r])] += A[r]
        Bs.append(Bs_)
        As.append(Ag)
    K = sla.block_diag(*Ks)
    B = np.vstack(Bs)
    A = np.hstack(As)
    F = np.concatenate(Fs)
    return K, A, B, F


def monolithic_ls(geom, W, b, rhs_rows, coef=None):
    """LS solution of Eq. (3.3): [[K, B], [0, -A K^+ B]] [c; u] = [F; -A K^+ F],
    K^+ = (K^T K)^{-1} K^T.  Returns (c [N, n], u_gamma)."""
    K, A, B, F = global_blocks(geom, W, b, rhs_rows, coef)
    Kp = np.linalg.solve(K.T @ K, K.T)
    top = np.hstack([K, B])
    bot = np.hstack([np.zeros((A.shape[0], K.shape[1])), -A @ Kp @ B])
    Z = np.vstack([top, bot])
    rhs = np.concatenate([F, -A @ Kp @ F])
    x = np.linalg.lstsq(Z, rhs, rcond=None)[0]
    nc = K.shape[1]
    return x[:nc].reshape(geom.n_sub, -1), x[nc:]


def normal_equations(geom, W, b, rhs_rows, coef=None):
    """Dense Eq. (3.4) solved by LU.  Returns (c [N, n], u_gamma)."""
    K, A, B, F = global_blocks(geom, W, b, rhs_rows, coef)
    Kp = np.linalg.solve(K.T @ K, K.T)
    T = np.eye(K.shape[0]) + Kp.T @ A.T @ A @ Kp
    top = np.hstack([K.T @ K, K.T @ B])
    bot = np.hstack([B.T @ K, B.T @ T @ B])
    rhs = np.concatenate([K.T @ F, B.T @ T @ F])
    x = np.linalg.solve(np.vstack([top, bot]), rhs)
    nc = K.shape[1]
    return x[:nc].reshape(geom.n_sub, -1), x[nc:]


def classical_elm(xy, counts, W, b, rhs_row, nrm=None):
    """Plain ELM on one domain: c = K^+ F (least squares, SVD-based)."""
    K, _ = assemble_local(xy, np.zeros_like(xy) if nrm is None else nrm, counts, W, b)
    F = rhs_local(rhs_row, counts)
    return np.linalg.lstsq(K, F, rcond=None)[0]


# --------------------------------------------------------------------------
# Timing helper for the CPU baseline
# --------------------------------------------------------------------------

def timed_solve(geom, W, b, rhs_rows, test_xy, owner):
    """One full solve (Algorithm 1) plus evaluation; returns (seconds, u, grad, result)."""
    t0 = time.perf_counter()
    res = solve(geom, W, b, rhs_rows, keep=False)
    u, g = evaluate(W, b, res.c, test_xy, owner)
    return time.perf_counter() - t0, u, g, res
