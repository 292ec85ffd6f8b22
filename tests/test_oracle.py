"""Pins for the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Each test is chosen so that a plausible mistake in the oracle (a dropped term,
a wrong sign, a wrong index map, a transposed operand) fails at least one of
them.  None of them compares the oracle with itself.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import elm_oracle as O
from paper_2406_15959_gb300 import workload as wl


def tiny(gx=2, gy=2, n=12, mi=6, p=5, seed=3, theta="paper", source="sinsin", c=0.5):
    return wl.build(gx, gy, n, mi, mi, p, p, theta=theta, theta_seed=seed,
                    source=source, source_seed=seed, c=c, n_test_side=20)


# ----------------------------------------------------------------- assembly

def test_features_match_symbolic_derivatives():
    """K^s / A^s rows (Section 3) against sympy's own derivatives of tanh(w.x+b):
    -Laplacian at interior rows, value at boundary/interface rows, outward normal
    derivative for A^s.  Pins the sign of L, the factor 2 and the normal."""
    sympy = pytest.importorskip("sympy")
    x, y, w1, w2, b = sympy.symbols("x y w1 w2 b", real=True)
    phi = sympy.tanh(w1 * x + w2 * y + b)
    lap = sympy.lambdify((x, y, w1, w2, b), -(sympy.diff(phi, x, 2) + sympy.diff(phi, y, 2)))
    dx = sympy.lambdify((x, y, w1, w2, b), sympy.diff(phi, x))
    dy = sympy.lambdify((x, y, w1, w2, b), sympy.diff(phi, y))
    val = sympy.lambdify((x, y, w1, w2, b), phi)
    w = tiny(gx=2, gy=1, n=5, mi=3, p=2, seed=11)
    g = w.geom
    for s in range(g.n_sub):
        K, A = O.assemble_local(g.xy[s], g.nrm[s], g.counts[s], w.W[s], w.b[s])
        ri, rb, rg = g.rows(s)
        for j in range(w.n_neurons):
            pj = (w.W[s, j, 0], w.W[s, j, 1], w.b[s, j])
            for r in range(ri.start, ri.stop):
                assert K[r, j] == pytest.approx(float(lap(*g.xy[s, r], *pj)), rel=1e-12, abs=1e-12)
            for r in range(rb.start, rg.stop):
                assert K[r, j] == pytest.approx(float(val(*g.xy[s, r], *pj)), rel=1e-13, abs=1e-14)
            for k, r in enumerate(range(rg.start, rg.stop)):
                nx, ny = g.nrm[s, r]
                ref = nx * dx(*g.xy[s, r], *pj) + ny * dy(*g.xy[s, r], *pj)
                assert A[k, j] == pytest.approx(float(ref), rel=1e-12, abs=1e-14)


def test_features_match_finite_differences():
    """Second, library-free pin of the same rows: central differences of tanh."""
    w = tiny(gx=2, gy=2, n=7, mi=4, p=3, seed=5)
    g = w.geom
    h = 1e-4
    for s in range(g.n_sub):
        K, A = O.assemble_local(g.xy[s], g.nrm[s], g.counts[s], w.W[s], w.b[s])
        ri, _, rg = g.rows(s)
        W, b = w.W[s], w.b[s]

        def phi(p):
            return np.tanh(p @ W.T + b)
        for r in range(ri.start, ri.stop):
            p0 = g.xy[s, r]
            ex, ey = np.array([h, 0.0]), np.array([0.0, h])
            lap = (phi(p0 + ex) + phi(p0 - ex) + phi(p0 + ey) + phi(p0 - ey) - 4 * phi(p0)) / h ** 2
            np.testing.assert_allclose(K[r], -lap, rtol=2e-5, atol=1e-4)
        for k, r in enumerate(range(rg.start, rg.stop)):
            p0, n = g.xy[s, r], g.nrm[s, r]
            dn = (phi(p0 + h * n) - phi(p0 - h * n)) / (2 * h)
            np.testing.assert_allclose(A[k], dn, rtol=1e-6, atol=1e-8)


def test_geometry_invariants():
    """Every interface unknown is shared by exactly two subdomains at the same
    point with opposite outward normals (the transmission conditions of Eq. (2.2))."""
    for gx, gy in [(2, 2), (3, 2), (4, 4)]:
        g = wl.make_geometry(gx, gy, 3, 4, 5, 6)
        seen = {}
        for s in range(g.n_sub):
            _, _, rg = g.rows(s)
            for r in range(rg.start, rg.stop):
                seen.setdefault(int(g.dof[s, r]), []).append((s, g.xy[s, r], g.nrm[s, r]))
        assert sorted(seen) == list(range(g.n_gamma))
        for d, lst in seen.items():
            assert len(lst) == 2
            (s0, x0, n0), (s1, x1, n1) = lst
            assert s0 != s1
            assert np.array_equal(x0, x1)
            assert np.array_equal(n0, -n1)


# ----------------------------------------------------------------- the three routes

@pytest.mark.parametrize("gx,gy,seed", [(2, 2, 3), (3, 2, 4), (2, 3, 6)])
def test_ddm_route_matches_monolithic_and_normal_equations(gx, gy, seed):
    """Route 1 (Schur system Eq. (3.5) + back-solve) equals the dense LS solution of
    the eliminated system Eq. (3.3) and the dense normal equations Eq. (3.4)."""
    w = tiny(gx=gx, gy=gy, seed=seed)
    res = O.solve(w.geom, w.W, w.b, w.rhs)
    assert res.rdiag_ratio.min() > 1e-3           # well-conditioned, so c itself is pinned
    c2, u2 = O.monolithic_ls(w.geom, w.W, w.b, w.rhs)
    c3, u3 = O.normal_equations(w.geom, w.W, w.b, w.rhs)
    for c, u in [(c2, u2), (c3, u3)]:
        assert np.linalg.norm(res.u_gamma - u) <= 1e-10 * np.linalg.norm(u)
        assert np.linalg.norm(res.c - c) <= 1e-9 * np.linalg.norm(c)


def test_eliminated_ls_differs_from_original_ls():
    """The paper solves the LS problem of Eq. (3.3), not of Eq. (3.1); for an
    inconsistent system the two minimisers differ, and the oracle follows Eq. (3.3)."""
    w = tiny(gx=2, gy=2, seed=9)
    K, A, B, F = O.global_blocks(w.geom, w.W, w.b, w.rhs)
    Z = np.block([[K, B], [A, np.zeros((A.shape[0], B.shape[1]))]])
    x = np.linalg.lstsq(Z, np.concatenate([F, np.zeros(A.shape[0])]), rcond=None)[0]
    res = O.solve(w.geom, w.W, w.b, w.rhs)
    u_orig = x[K.shape[1]:]
    assert np.linalg.norm(res.u_gamma - u_orig) > 1e-8 * np.linalg.norm(u_orig)


def test_single_subdomain_is_classical_elm():
    """N = 1: no interface, Algorithm 1 reduces to the classical ELM c = K^+ F."""
    w = tiny(gx=1, gy=1, n=15, mi=7, p=6, seed=2)
    assert w.geom.n_gamma == 0
    res = O.solve(w.geom, w.W, w.b, w.rhs)
    g = w.geom
    c_ref = O.classical_elm(g.xy[0], g.counts[0], w.W[0], w.b[0], w.rhs[0])
    np.testing.assert_allclose(res.c[0], c_ref, rtol=1e-9, atol=1e-9 * np.abs(c_ref).max())


@pytest.mark.parametrize("gx,gy", [(2, 2), (3, 2)])
def test_consistent_system_is_recovered_exactly(gx, gy):
    """If the local networks c* are continuous across Gamma (values and normal
    fluxes) and F^s = K^s c*^s away from Gamma, then (c*, u* = traces of the
    networks on Gamma) solves Eq. (3.1) exactly and so minimises Eq. (3.3) with
    zero residual: the oracle must return it."""
    w = tiny(gx=gx, gy=gy, n=14, mi=6, p=3, seed=17)
    g = w.geom
    N, n = g.n_sub, w.n_neurons
    Ks, As = [], []
    for s in range(N):
        K, A = O.assemble_local(g.xy[s], g.nrm[s], g.counts[s], w.W[s], w.b[s])
        Ks.append(K); As.append(A)
    # Constraints on the stacked c: value jump and flux sum at every interface point.
    C = np.zeros((2 * g.n_gamma, N * n))
    sign = {}
    for s in range(N):
        _, _, rg = g.rows(s)
        for k, r in enumerate(range(rg.start, rg.stop)):
            d = int(g.dof[s, r])
            sg = sign.setdefault(d, 1.0)
            sign[d] = -1.0
            C[d, s * n:(s + 1) * n] += sg * Ks[s][r]
            C[g.n_gamma + d, s * n:(s + 1) * n] += As[s][k]
    Nul = sla.null_space(C)
    assert Nul.shape[1] > 0
    cstar = (Nul @ np.random.default_rng(0).standard_normal(Nul.shape[1])).reshape(N, n)
    rhs = np.zeros_like(w.rhs)
    ustar = np.zeros(g.n_gamma)
    for s in range(N):
        ri, rb, rg = g.rows(s)
        v = Ks[s] @ cstar[s]
        rhs[s, :rb.stop] = v[:rb.stop]
        ustar[g.dof[s, rg]] = v[rg]
    res = O.solve(g, w.W, w.b, rhs)
    assert np.linalg.norm(res.u_gamma - ustar) <= 1e-9 * np.linalg.norm(ustar)
    assert np.linalg.norm(res.c - cstar) <= 1e-7 * np.linalg.norm(cstar)


# ----------------------------------------------------------------- invariants

def test_schur_matrix_is_spd_and_backsolve_is_optimal():
    """S is symmetric positive definite (Section 3, before Algorithm 1), and each
    c^s satisfies the local normal equations K^T K c = K^T (F - B u) (Algorithm 1)."""
    w = wl.build(3, 3, 40, 9, 8, 11, 10, theta="paper", theta_seed=4, source="fourier",
                 source_seed=4, n_test_side=10)
    res = O.solve(w.geom, w.W, w.b, w.rhs)
    S = res.S
    assert np.abs(S - S.T).max() <= 1e-14 * np.abs(S).max()
    assert np.linalg.eigvalsh(S).min() > 0
    g = w.geom
    for s in range(g.n_sub):
        K, _ = O.assemble_local(g.xy[s], g.nrm[s], g.counts[s], w.W[s], w.b[s])
        F = O.rhs_local(w.rhs[s], g.counts[s])
        _, _, rg = g.rows(s)
        r = K @ res.c[s] - F
        r[rg] -= res.u_gamma[g.dof[s, rg]]           # K c + B u - F with B = [0; 0; -E]
        assert np.linalg.norm(K.T @ r) <= 1e-9 * np.linalg.norm(K.T @ F)


def test_schur_pieces_project_onto_range():
    """[K K^+]_GG = Q_G Q_G^T is a block of an orthogonal projector:
    eigenvalues of D_s = I - Q_G Q_G^T lie in [0, 1]."""
    w = tiny(gx=3, gy=3, n=20, mi=7, p=4, seed=8)
    res = O.solve(w.geom, w.W, w.b, w.rhs)
    for L in res.locs:
        ev = np.linalg.eigvalsh(L.D)
        assert ev.min() > -1e-12 and ev.max() < 1 + 1e-12
        np.testing.assert_allclose(L.Q.T @ L.Q, np.eye(L.Q.shape[1]), atol=1e-12)


def test_evaluation_matches_collocation_rows():
    """u(x) at boundary/interface collocation points equals the corresponding rows of K c."""
    w = tiny(gx=2, gy=2, n=10, mi=5, p=4, seed=12)
    res = O.solve(w.geom, w.W, w.b, w.rhs)
    g = w.geom
    for s in range(g.n_sub):
        _, rb, rg = g.rows(s)
        K, _ = O.assemble_local(g.xy[s], g.nrm[s], g.counts[s], w.W[s], w.b[s])
        pts = g.xy[s, rb.start:rg.stop]
        u, _ = O.evaluate(w.W, w.b, res.c, pts, np.full(len(pts), s))
        np.testing.assert_allclose(u, K[rb.start:rg.stop] @ res.c[s], rtol=1e-12, atol=1e-12)


def test_evaluated_gradient_matches_central_differences_of_u():
    """grad u of the oracle's evaluation against central differences of its own u (the
    u half is pinned by the collocation rows above), at random points of every
    subdomain, each point kept with its owner.  A wrong sign, a missing (1 - t^2) or the
    weights applied per component in the wrong order fails this."""
    w = tiny(gx=2, gy=2, n=9, mi=5, p=4, seed=21)
    res = O.solve(w.geom, w.W, w.b, w.rhs)
    g = w.geom
    rng = np.random.default_rng(4)
    h = 1e-5
    for s in range(g.n_sub):
        x0, x1, y0, y1 = g.box(s)
        pts = np.stack([rng.uniform(x0, x1, 12), rng.uniform(y0, y1, 12)], axis=1)
        own = np.full(len(pts), s)
        _, gr = O.evaluate(w.W, w.b, res.c, pts, own)
        for d in range(2):
            e = np.zeros(2)
            e[d] = h
            up, _ = O.evaluate(w.W, w.b, res.c, pts + e, own)
            um, _ = O.evaluate(w.W, w.b, res.c, pts - e, own)
            fd = (up - um) / (2 * h)
            np.testing.assert_allclose(gr[:, d], fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())


def test_evaluated_gradient_of_one_neuron_is_the_sech_squared_closed_form():
    """u = c tanh(w.x + b) has grad u = c w sech^2(w.x + b): one neuron per subdomain,
    values written out by hand (sech through cosh, not through 1 - tanh^2)."""
    import math
    W = np.array([[[1.5, -0.5]], [[-2.0, 0.25]]])
    b = np.array([[0.3], [-0.1]])
    c = np.array([[2.0], [-0.75]])
    pts = np.array([[0.2, 0.7], [0.9, 0.1], [0.5, 0.5]])
    for s in range(2):
        u, gr = O.evaluate(W, b, c, pts, np.full(3, s))
        for i, (x, y) in enumerate(pts):
            z = W[s, 0, 0] * x + W[s, 0, 1] * y + b[s, 0]
            sech2 = 1.0 / math.cosh(z) ** 2
            assert u[i] == pytest.approx(c[s, 0] * math.tanh(z), rel=1e-14)
            assert gr[i, 0] == pytest.approx(c[s, 0] * W[s, 0, 0] * sech2, rel=1e-13)
            assert gr[i, 1] == pytest.approx(c[s, 0] * W[s, 0, 1] * sech2, rel=1e-13)


def test_relative_h1_error_has_its_closed_form_on_the_test_grid():
    """Discrete relative L2 / H1 errors (the metric of Table 2) on the cell-centred test
    grid, where sum_i sin^2(pi x_i) = sum_i cos^2(pi x_i) = n/2 exactly: for
    u_ex = sin(pi x) sin(pi y), sum u_ex^2 = n^2/4 and sum |grad u_ex|^2 = 2 pi^2 n^2/4.
    A shift u = u_ex + eps and a gradient error (delta, 0) at every point then give
    L2 = 2 eps and H1 = 2 sqrt(eps^2 + delta^2) / sqrt(1 + 2 pi^2)."""
    import math
    g = wl.make_geometry(2, 2, 3, 3, 3, 3)
    n = 40
    xy, _ = wl.test_points(g, n)
    src = wl.make_source("sinsin")
    u_ex, g_ex = src.u(xy), src.grad_u(xy)
    eps, delta = 1e-3, 3e-3
    l2, h1 = O.rel_errors(u_ex + eps, g_ex + np.array([delta, 0.0]), u_ex, g_ex)
    assert l2 == pytest.approx(2 * eps, rel=1e-10)
    assert h1 == pytest.approx(2 * math.sqrt(eps ** 2 + delta ** 2) / math.sqrt(1 + 2 * math.pi ** 2),
                               rel=1e-10)
    # exact values and gradients: both errors vanish
    assert O.rel_errors(u_ex, g_ex, u_ex, g_ex) == (0.0, 0.0)


def test_error_falls_with_neurons_and_points():
    """Manufactured solution sin(pi x) sin(pi y): the relative L2 error at the test
    points falls as the networks and the point sets grow (Theorem 2.1, Table 2)."""
    errs = []
    for n, mi, p in [(10, 5, 5), (40, 10, 10), (120, 18, 18)]:
        w = wl.build(2, 2, n, mi, mi, p, p, theta="paper", theta_seed=1, source="sinsin",
                     n_test_side=40)
        res = O.solve(w.geom, w.W, w.b, w.rhs)
        u, gr = O.evaluate(w.W, w.b, res.c, w.test_xy, w.test_owner)
        errs.append(O.rel_errors(u, gr, w.src.u(w.test_xy), w.src.grad_u(w.test_xy))[0])
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-5


def test_fourier_source_has_the_stated_exact_solution():
    """The sine-mode source and its closed-form u satisfy -Laplacian u = f (checked by FD)."""
    src = wl.make_source("fourier", seed=5, modes=4)
    rng = np.random.default_rng(1)
    p = rng.uniform(0.1, 0.9, size=(50, 2))
    h = 1e-4
    ex, ey = np.array([h, 0.0]), np.array([0.0, h])
    lap = (src.u(p + ex) + src.u(p - ex) + src.u(p + ey) + src.u(p - ey) - 4 * src.u(p)) / h ** 2
    np.testing.assert_allclose(-lap, src.f(p), rtol=1e-5, atol=1e-6)


# --- CG for the interface system (Section 4), pinned to properties of the algorithm ---

def test_cg_terminates_in_distinct_eigenvalue_count():
    """In exact arithmetic CG ends after as many steps as S has distinct eigenvalues;
    with 4 well-separated ones it must meet a tight tolerance within 4 (+1) steps."""
    rng = np.random.default_rng(7)
    Qm, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    lam = np.repeat([1.0, 3.0, 7.0, 20.0], 10)
    S = (Qm * lam) @ Qm.T
    b = rng.standard_normal(40)
    x, k, ok = O.cg_solve(S, b, 1e-12, 200)
    assert ok and k <= 5
    assert np.linalg.norm(x - np.linalg.solve(S, b)) <= 1e-10 * np.linalg.norm(x)


def test_cg_matches_direct_solve_within_condition_bound():
    rng = np.random.default_rng(8)
    B = rng.standard_normal((60, 60))
    S = B @ B.T + 60 * np.eye(60)
    b = rng.standard_normal(60)
    tol = 1e-10
    x, k, ok = O.cg_solve(S, b, tol, 1000)
    xd = np.linalg.solve(S, b)
    assert ok
    assert np.linalg.norm(S @ x - b) <= tol * np.linalg.norm(b) * (1 + 1e-6)
    assert np.linalg.norm(x - xd) <= np.linalg.cond(S) * tol * np.linalg.norm(xd) * 2


def test_cg_reports_non_convergence_at_maxit():
    rng = np.random.default_rng(9)
    B = rng.standard_normal((50, 50))
    S = B @ B.T + 1e-3 * np.eye(50)
    x, k, ok = O.cg_solve(S, rng.standard_normal(50), 1e-14, 5)
    assert not ok and k == 5


def test_cg_on_schur_system_reaches_cholesky_solution():
    """On the 2x2 tiny problem the CG interface solution agrees with the Cholesky one
    to the accuracy the residual bound allows."""
    g = wl.make_geometry(2, 2, 6, 6, 6, 6)
    n = 12
    W, b = wl.draw_theta(g, n, mode="paper", c=0.5, seed=3)
    rows = wl.rhs_rows(g, wl.make_source("sinsin"))
    res = O.solve(g, W, b, rows)
    tol = 1e-11
    u, k, ok = O.cg_solve(res.S, res.rhs, tol, 10 * len(res.rhs))
    assert ok
    kappa = np.linalg.cond(res.S)
    assert np.linalg.norm(u - res.u_gamma) <= 2 * kappa * tol * np.linalg.norm(res.u_gamma)


# --- variable coefficient -div(rho grad u) = f (Section 4) ---

def test_varcoef_rows_match_conservative_finite_differences():
    """Interior rows against a flux-form difference of -div(rho grad phi) with the
    coefficient evaluated at half points (independent of the closed form)."""
    w = tiny(gx=2, gy=2, n=7, mi=4, p=3, seed=5)
    g = w.geom
    cf = wl.make_coefficient("sine", seed=3)
    crow = wl.coef_rows(g, cf)
    h = 1e-4
    for s in range(g.n_sub):
        K, _ = O.assemble_local(g.xy[s], g.nrm[s], g.counts[s], w.W[s], w.b[s], crow[s])
        ri, _, _ = g.rows(s)
        W, b = w.W[s], w.b[s]

        def phi(p):
            return np.tanh(p @ W.T + b)
        for r in range(ri.start, ri.stop):
            p0 = g.xy[s, r]
            div = 0.0
            for e in (np.array([h, 0.0]), np.array([0.0, h])):
                rp, rm = cf.rho(p0 + e / 2), cf.rho(p0 - e / 2)
                div = div + (rp * (phi(p0 + e) - phi(p0)) - rm * (phi(p0) - phi(p0 - e))) / h ** 2
            np.testing.assert_allclose(K[r], -div, rtol=1e-5, atol=1e-3)


def test_unit_coefficient_reduces_to_poisson_rows():
    w = tiny(gx=2, gy=2, n=9, mi=5, p=4, seed=6)
    g = w.geom
    crow = wl.coef_rows(g, wl.make_coefficient("const", value=1.0))
    for s in range(g.n_sub):
        K0, A0 = O.assemble_local(g.xy[s], g.nrm[s], g.counts[s], w.W[s], w.b[s])
        K1, A1 = O.assemble_local(g.xy[s], g.nrm[s], g.counts[s], w.W[s], w.b[s], crow[s])
        assert np.array_equal(K0, K1) and np.array_equal(A0, A1)


def test_varcoef_manufactured_source_and_routes():
    """f of the manufactured problem is -div(rho grad u) (checked by differences of u),
    and the DDM route equals the monolithic LS of Eq. (3.3) with the coefficient."""
    w = wl.build(2, 2, 12, 6, 6, 6, 6, theta="paper", theta_seed=3, c=0.5, source="sinsin",
                 coef="sine", coef_seed=2, n_test_side=8)
    cf, src, h = w.coef, w.src, 1e-4
    p0 = np.array([[0.31, 0.67], [0.52, 0.18]])
    div = 0.0
    for e in (np.array([h, 0.0]), np.array([0.0, h])):
        div = div + (cf.rho(p0 + e / 2) * (src.u(p0 + e) - src.u(p0))
                     - cf.rho(p0 - e / 2) * (src.u(p0) - src.u(p0 - e))) / h ** 2
    np.testing.assert_allclose(src.f(p0), -div, rtol=1e-6)
    res = O.solve(w.geom, w.W, w.b, w.rhs, coef=w.coef_rows)
    c_m, u_m = O.monolithic_ls(w.geom, w.W, w.b, w.rhs, coef=w.coef_rows)
    assert np.linalg.norm(res.u_gamma - u_m) <= 1e-10 * np.linalg.norm(u_m)


def test_varcoef_error_falls_with_neurons():
    errs = []
    for n, m in ((30, 8), (120, 16)):
        w = wl.build(2, 2, n, m, m, m, m, theta="local_unit", theta_seed=1, source="sinsin",
                     coef="sine", coef_seed=2, n_test_side=20)
        res = O.solve(w.geom, w.W, w.b, w.rhs, coef=w.coef_rows)
        u, g = O.evaluate(w.W, w.b, res.c, w.test_xy, w.test_owner)
        errs.append(np.linalg.norm(u - w.src.u(w.test_xy)) / np.linalg.norm(w.src.u(w.test_xy)))
    assert errs[1] < 0.1 * errs[0] and errs[1] < 1e-4, errs


# --- the learned warm start's network (oracle/mlp_oracle.py) ---

def test_mlp_gradient_matches_central_differences():
    from oracle import mlp_oracle as MO
    rng = np.random.default_rng(21)
    d_in, d_h, d_out, B = 5, 7, 4, 6
    n = d_in * d_h + d_h + d_h * d_h + d_h + d_h * d_out + d_out
    p = rng.standard_normal(n) * 0.5
    X, T = rng.standard_normal((B, d_in)), rng.standard_normal((B, d_out))
    _, g = MO.loss_and_grad(p, X, T, d_in, d_h, d_out)
    h = 1e-6
    for i in rng.choice(n, size=40, replace=False):
        e = np.zeros(n)
        e[i] = h
        lp, _ = MO.loss_and_grad(p + e, X, T, d_in, d_h, d_out)
        lm, _ = MO.loss_and_grad(p - e, X, T, d_in, d_h, d_out)
        assert abs((lp - lm) / (2 * h) - g[i]) <= 1e-7 * max(1.0, abs(g[i]))


def test_gelu_matches_its_definition_and_derivative():
    from oracle import mlp_oracle as MO
    import math
    for z in (-3.0, -0.7, 0.0, 0.4, 2.5):
        phi = 0.5 * (1 + math.erf(z / math.sqrt(2)))
        assert abs(MO.gelu(np.array(z)) - z * phi) <= 1e-15
        h = 1e-6
        fd = (MO.gelu(np.array(z + h)) - MO.gelu(np.array(z - h))) / (2 * h)
        assert abs(MO.gelu_grad(np.array(z)) - fd) <= 1e-8


def test_adam_first_step_is_signed_learning_rate():
    """With zero moments the bias-corrected first step (Kingma and Ba, Section 2 form
    with the step size folded: alpha_t = alpha sqrt(1 - b2^t) / (1 - b1^t)) is
    -lr g / (|g| + eps / sqrt(1 - b2)): the signed learning rate for |g| >> eps."""
    from oracle import mlp_oracle as MO
    g = np.array([0.3, -2.0, 1e-3])
    p1, _, _ = MO.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 0.01)
    np.testing.assert_allclose(p1, -0.01 * g / (np.abs(g) + 1e-8 / np.sqrt(1 - 0.999)), rtol=1e-12)


def test_adam_steps_with_constant_gradient_follow_the_bias_corrected_closed_form():
    """With a constant gradient g and zero initial moments, m_t = (1 - b1^t) g and
    v_t = (1 - b2^t) g^2 after t steps, so step t moves a parameter by exactly
    -lr g / (|g| + eps / sqrt(1 - b2^t)).  The sum over t = 1..5 pins the powers t of
    the bias correction (a factor b1 * t instead of b1^t flips the second step)."""
    from oracle import mlp_oracle as MO
    g = np.array([0.3, -2.0, 1e-3, 5.0])
    lr, b1, b2, eps = 0.01, 0.9, 0.999, 1e-8
    p = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    expect = np.zeros(4)
    for t in range(1, 6):
        p, m, v = MO.adam_step(p, g, m, v, t, lr, b1, b2, eps)
        expect -= lr * g / (np.abs(g) + eps / np.sqrt(1.0 - b2 ** t))
        np.testing.assert_allclose(m, (1 - b1 ** t) * g, rtol=1e-13)
        np.testing.assert_allclose(v, (1 - b2 ** t) * g * g, rtol=1e-12)
        np.testing.assert_allclose(p, expect, rtol=1e-12)


def test_radial_weights_have_density_proportional_to_norm():
    """Remark 4.2's radial initialisation: w on [-l, l]^2 with density proportional to |w|.
    Under that density E|w| = E_u|w|^2 / E_u|w| with E_u the uniform square:
    l (2/3) / ((sqrt 2 + asinh 1) / 3) = 0.8712 l."""
    import math
    g = wl.make_geometry(1, 1, 4, 4, 3, 3)
    W, _ = wl.draw_theta(g, 40000, "radial", seed=3, c=0.125)
    lim = 0.125 * math.sqrt(40000)
    r = np.hypot(W[0, :, 0], W[0, :, 1]) / lim
    expect = (2.0 / 3.0) / ((math.sqrt(2.0) + math.asinh(1.0)) / 3.0)
    assert abs(r.mean() - expect) < 0.01
    assert np.abs(W).max() <= lim


def _fp32_qr_refinement(w, s=0, iters=12):
    """Least squares K c = F from an FP32 Householder QR refined in FP64 by the corrected
    seminormal equations (Bjorck): c <- c + R^{-1} R^{-T} K^T (F - K c) with the FP32 R.
    Returns (kappa(K), relative error of K c against the FP64 least-squares fit)."""
    import scipy.linalg as sla
    g = w.geom
    K, _ = O.assemble_local(g.xy[s], g.nrm[s], g.counts[s], w.W[s], w.b[s])
    F = O.rhs_local(w.rhs[s], g.counts[s])
    ref = K @ np.linalg.lstsq(K, F, rcond=None)[0]
    Q32, R32 = np.linalg.qr(K.astype(np.float32))
    R = R32.astype(np.float64)
    c = sla.solve_triangular(R, Q32.T.astype(np.float64) @ F)
    for _ in range(iters):
        c = c + sla.solve_triangular(R, sla.solve_triangular(R.T, K.T @ (F - K @ c), lower=True))
    sv = np.linalg.svd(K, compute_uv=False)
    with np.errstate(all="ignore"):
        err = np.linalg.norm(K @ c - ref) / np.linalg.norm(ref)
    return sv[0] / sv[-1], err


def test_mixed_precision_refinement_needs_kappa_below_inverse_unit_roundoff():
    """The precision axis: refinement from an FP32-level factorisation converges only when
    kappa(K) u_32 < 1 (u_32 = 2^-24).  It does on a well-conditioned local matrix and fails
    on the paper's initialisation, whose K^s have kappa ~ 1e14: why every product of the
    path keeps FP64 accuracy (digit-split on the BF16 tensor cores) instead."""
    good = wl.build(2, 2, 40, 10, 10, 10, 10, theta="local_unit", theta_seed=1, source="sinsin",
                    n_test_side=10)
    paper = wl.build(2, 2, 200, 20, 20, 40, 40, theta="paper", theta_seed=2, source="sinsin",
                     n_test_side=10)
    k1, e1 = _fp32_qr_refinement(good)
    k2, e2 = _fp32_qr_refinement(paper)
    assert k1 * 2.0 ** -24 < 1 and e1 < 1e-12
    assert k2 * 2.0 ** -24 > 1e6 and not (e2 < 1e-6)


def _refined_solve(w, iters=12):
    """The mixed-precision path's algorithm on the CPU: low-precision (float32) local QR,
    FP64 Schur Cholesky of the low-precision Schur matrix, and refinement of (c, w, u) on
    FP64 residuals of K^T K c + K^T B u = K^T F, K^T K w - A^T A c = 0,
    B^T K c - B^T K w + B^T B u = B^T F (Eq. (3.4) with K^{+T} A^T A c written as K w),
    corrected by the elimination of Eq. (3.5) with the low-precision factors.  Returns the
    relative u corrections per step and the final (c, u)."""
    g = w.geom
    N, ng = g.n_sub, g.n_gamma
    Ks, As, Fs, dofs, L = [], [], [], [], []
    for s in range(N):
        mi, mb, mg = (int(v) for v in g.counts[s])
        K, A = O.assemble_local(g.xy[s], g.nrm[s], g.counts[s], w.W[s], w.b[s])
        Q, R = np.linalg.qr(K.astype(np.float32))
        Q, R = Q.astype(np.float64), R.astype(np.float64)
        QG = Q[mi + mb:]
        Y = sla.solve_triangular(R, A.T, trans="T").T
        Ks.append(K); As.append(A); Fs.append(O.rhs_local(w.rhs[s], g.counts[s]))
        dofs.append(g.dof[s, mi + mb:mi + mb + mg].astype(int))
        L.append((R, QG, Y, mi + mb))
    S = np.zeros((ng, ng)); Mg = np.zeros((ng, ng))
    for s in range(N):
        R, QG, Y, _ = L[s]
        S[np.ix_(dofs[s], dofs[s])] += np.eye(len(dofs[s])) - QG @ QG.T
        Mg[np.ix_(dofs[s], dofs[s])] += -(Y @ QG.T)
    Lc = np.linalg.cholesky(S + Mg.T @ Mg)

    def gsum(v):
        out = np.zeros(ng)
        for s in range(N):
            np.add.at(out, dofs[s], v[s])
        return out
    n = w.n_neurons
    c, wv, u = np.zeros((N, n)), np.zeros((N, n)), np.zeros(ng)
    etas = []
    for _ in range(iters):
        Ac = gsum([As[s] @ c[s] for s in range(N)])
        r1, r3, z = [], [], []
        for s in range(N):
            ifc = L[s][3]
            e = Fs[s] - Ks[s] @ c[s]
            e[ifc:] += u[dofs[s]]
            kw = Ks[s] @ wv[s]
            r1.append(Ks[s].T @ e)
            r3.append(As[s].T @ Ac[dofs[s]] - Ks[s].T @ kw)
            z.append(-(e[ifc:] + kw[ifc:]))
        p1 = [sla.solve_triangular(L[s][0], r1[s], trans="T") for s in range(N)]
        p13 = [sla.solve_triangular(L[s][0], r1[s] - r3[s], trans="T") for s in range(N)]
        rhs = gsum(z) + gsum([L[s][1] @ p13[s] for s in range(N)]) + Mg.T @ gsum([L[s][2] @ p1[s] for s in range(N)])
        du = sla.solve_triangular(Lc.T, sla.solve_triangular(Lc, rhs, lower=True), lower=False)
        dc = np.array([sla.solve_triangular(L[s][0], p1[s] + L[s][1].T @ du[dofs[s]]) for s in range(N)])
        Adc = gsum([As[s] @ dc[s] for s in range(N)])
        dw = np.array([sla.solve_triangular(L[s][0], sla.solve_triangular(
            L[s][0], r3[s] + As[s].T @ Adc[dofs[s]], trans="T")) for s in range(N)])
        c, wv, u = c + dc, wv + dw, u + du
        with np.errstate(all="ignore"):
            etas.append(np.abs(du).max() / np.abs(u).max())
    return etas, c, u


def test_mixed_precision_refinement_system_converges_to_the_method_result():
    """The (c, w, u) system the mixed-precision path refines has the method's result as its
    solution: refinement from a float32 factorisation reaches the oracle (Eq. (3.5) solved
    in FP64) to rounding level on a well-conditioned case, with the relative correction
    contracting by orders of magnitude per step, and does not converge at the paper's
    initialisation (kappa(K^s) ~ 1e14 > 1 / u_32), where the path falls back to FP64."""
    good = wl.build(3, 3, 60, 12, 12, 12, 12, theta="local_unit", theta_seed=3, source="fourier",
                    source_seed=3, n_test_side=10)
    etas, c, u = _refined_solve(good)
    res = O.solve(good.geom, good.W, good.b, good.rhs)
    assert np.linalg.norm(u - res.u_gamma) <= 1e-12 * np.linalg.norm(res.u_gamma)
    assert np.abs(c - res.c).max() <= 1e-9 * np.abs(res.c).max()
    assert etas[3] < 1e-4 and min(etas) < 1e-12
    paper = wl.build(2, 2, 200, 20, 20, 40, 40, theta="paper", theta_seed=2, source="sinsin",
                     n_test_side=10)
    etas_p, _, _ = _refined_solve(paper, iters=6)
    assert not (min(etas_p[2:]) < 0.5)                       # no contraction: a stall


def test_ridge_zero_is_the_exact_least_squares_solution():
    """ridge_rows with alpha = 0 adds zero rows: the oracle's result is unchanged."""
    w = tiny(gx=2, gy=2, seed=3)
    a = O.solve(w.geom, w.W, w.b, w.rhs)
    z = O.solve(w.geom, w.W, w.b, w.rhs, ridge=0.0)
    assert np.linalg.norm(z.u_gamma - a.u_gamma) <= 1e-12 * np.linalg.norm(a.u_gamma)
    np.testing.assert_allclose(z.c, a.c, rtol=1e-10, atol=1e-12 * np.abs(a.c).max())


def test_ridge_single_subdomain_is_ridge_regression():
    """N = 1 with the Tikhonov rows: c = (K^T K + lambda^2 I)^{-1} K^T F with
    lambda = alpha * max_j |K_j| (the normal equations of ridge regression, solved by LU:
    a route independent of the augmented QR)."""
    w = tiny(gx=1, gy=1, n=15, mi=7, p=6, seed=2)
    g = w.geom
    K, _ = O.assemble_local(g.xy[0], g.nrm[0], g.counts[0], w.W[0], w.b[0])
    F = O.rhs_local(w.rhs[0], g.counts[0])
    alpha = 1e-3
    lam = alpha * np.sqrt((K * K).sum(axis=0)).max()
    c_ref = np.linalg.solve(K.T @ K + lam ** 2 * np.eye(K.shape[1]), K.T @ F)
    res = O.solve(g, w.W, w.b, w.rhs, ridge=alpha)
    np.testing.assert_allclose(res.c[0], c_ref, rtol=1e-9, atol=1e-10 * np.abs(c_ref).max())


# ----------------------------------------------------------------- cross points (corner rule)

def cross(G, n_grid, n, seed=5, source="sin2pi_exp"):
    """The paper's grid with its cross points (the corner rule of the remark in Section 3)."""
    return wl.paper_grid_workload(G, n_total=n * G * G, theta="local_unit", seed=seed, source=source,
                                  n_grid=n_grid, n_test_side=10, cross_points=True)


@pytest.mark.parametrize("G,n_grid", [(2, 9), (3, 13), (4, 17)])
def test_cross_point_geometry_follows_the_corner_rule(G, n_grid):
    """Every interface unknown sits at one point shared by 2 subdomains (inside an edge) or
    by the 4 around a cross point; every flux condition sums the rows of the two subdomains
    across one edge, at the same point, with opposite normals pointing from each to the
    other; and a subdomain has one row per edge through each of its cross points: 2 rows
    there, 4 conditions per cross point.  Read off the coordinates only."""
    g = wl.make_paper_grid_geometry(G, n_grid, cross_points=True)
    f = g.flux
    owners = {}
    for s in range(g.n_sub):
        _, _, rg = g.rows(s)
        for r in range(rg.start, rg.stop):
            owners.setdefault(int(g.dof[s, r]), []).append((s, tuple(g.xy[s, r])))
    assert sorted(owners) == list(range(g.n_gamma))
    ncross = 0
    for d, lst in owners.items():
        assert len({p for _, p in lst}) == 1 and len({s for s, _ in lst}) == len(lst)
        x, y = lst[0][1]
        on_x = any(abs(x - i / G) < 1e-12 for i in range(1, G))
        on_y = any(abs(y - i / G) < 1e-12 for i in range(1, G))
        assert len(lst) == (4 if on_x and on_y else 2)
        ncross += on_x and on_y
    assert ncross == (G - 1) ** 2
    cond = {}
    for s in range(g.n_sub):
        mi, mb, _ = g.counts[s]
        for k in range(int(f.count[s])):
            p = tuple(g.xy[s, mi + mb + f.row[s, k]])
            cond.setdefault(int(f.fdof[s, k]), []).append((s, p, tuple(f.nrm[s, k])))
    assert sorted(cond) == list(range(f.n_flux))
    per_point = {}
    for c, lst in cond.items():
        assert len(lst) == 2
        (s0, p0, n0), (s1, p1, n1) = lst
        assert p0 == p1 and np.array_equal(np.array(n0), -np.array(n1))
        # the normal of s0 points at s1: the neighbour across that edge
        ix, iy = s0 % G, s0 // G
        assert s1 == (iy + int(n0[1])) * G + (ix + int(n0[0]))
        per_point.setdefault(p0, []).append(lst)
    for p, conds in per_point.items():
        x, y = p
        if any(abs(x - i / G) < 1e-12 for i in range(1, G)) and any(abs(y - i / G) < 1e-12 for i in range(1, G)):
            assert len(conds) == 4
            rows = [(s, n) for lst in conds for s, _, n in lst]
            for s in {s for s, _ in rows}:
                assert len([n for t, n in rows if t == s]) == 2
        else:
            assert len(conds) == 1
    assert f.n_flux == g.n_gamma + 3 * (G - 1) ** 2


def test_corner_rows_are_normal_derivatives():
    """Every A-row of a cross-point geometry, the extra corner rows included, is the
    derivative of the features along its row's normal at its row's point (central
    differences), so A^s c is the normal flux of u_s there."""
    w = cross(2, 9, 6, seed=4)
    g = w.geom
    h = 1e-4
    for s in range(g.n_sub):
        frow, fnrm, _ = O.flux_rows(g, s)
        _, A = O.assemble_local(g.xy[s], g.nrm[s], g.counts[s], w.W[s], w.b[s], flux=(frow, fnrm))
        mi, mb, _ = g.counts[s]
        assert A.shape == (len(frow), w.n_neurons)
        for k in range(len(frow)):
            p0, n = g.xy[s, mi + mb + frow[k]], fnrm[k]
            dn = (np.tanh((p0 + h * n) @ w.W[s].T + w.b[s]) - np.tanh((p0 - h * n) @ w.W[s].T + w.b[s])) / (2 * h)
            np.testing.assert_allclose(A[k], dn, rtol=1e-6, atol=1e-8)


@pytest.mark.parametrize("G,n_grid,n", [(2, 17, 30), (3, 19, 24)])
def test_ddm_route_with_cross_points_matches_monolithic_and_normal_equations(G, n_grid, n):
    """With cross points the Schur route (P_s != E_s in M and h) still equals the dense LS
    solution of Eq. (3.3) and the dense normal equations Eq. (3.4), whose global A is
    assembled row by row from the flux conditions."""
    w = cross(G, n_grid, n)
    g = w.geom
    res = O.solve(g, w.W, w.b, w.rhs)
    assert res.rdiag_ratio.min() > 1e-6
    c2, u2 = O.monolithic_ls(g, w.W, w.b, w.rhs)
    c3, u3 = O.normal_equations(g, w.W, w.b, w.rhs)
    for c, u in [(c2, u2), (c3, u3)]:
        assert np.linalg.norm(res.u_gamma - u) <= 1e-9 * np.linalg.norm(u)
        assert np.linalg.norm(res.c - c) <= 1e-7 * np.linalg.norm(c)
    # the corner rows change the answer (they are not redundant)
    g0 = wl.make_paper_grid_geometry(G, n_grid, cross_points=True)
    g0.flux = None
    keep = {}
    for s in range(g0.n_sub):
        _, _, rg = g0.rows(s)
        for r in range(rg.start, rg.stop):
            keep.setdefault(int(g0.dof[s, r]), []).append(s)
    assert any(len(v) == 4 for v in keep.values())


@pytest.mark.parametrize("G,n_grid", [(2, 9), (3, 13)])
def test_consistent_system_with_cross_points_is_recovered_exactly(G, n_grid):
    """Networks c* continuous across Gamma (every unknown's value equal in all its
    subdomains, cross points included) whose normal fluxes cancel in every flux condition
    (the corner rows included), with F^s = K^s c*^s away from Gamma, solve Eq. (3.1)
    exactly: the oracle must return them.  A flux condition that paired the wrong rows, or
    M and h indexed by unknowns instead of flux conditions, leaves a residual."""
    w = cross(G, n_grid, 16, seed=17)
    g = w.geom
    N, n = g.n_sub, w.n_neurons
    Ks, As, maps = [], [], []
    for s in range(N):
        frow, fnrm, fdof = O.flux_rows(g, s)
        K, A = O.assemble_local(g.xy[s], g.nrm[s], g.counts[s], w.W[s], w.b[s], flux=(frow, fnrm))
        Ks.append(K); As.append(A); maps.append(fdof)
    rows = []
    first = {}
    for s in range(N):
        _, _, rg = g.rows(s)
        for r in range(rg.start, rg.stop):
            d = int(g.dof[s, r])
            if d in first:                      # value of s equals value of the first owner
                s0, r0 = first[d]
                row = np.zeros(N * n)
                row[s * n:(s + 1) * n] += Ks[s][r]
                row[s0 * n:(s0 + 1) * n] -= Ks[s0][r0]
                rows.append(row)
            else:
                first[d] = (s, r)
    F = np.zeros((g.flux.n_flux, N * n))
    for s in range(N):
        for k, c in enumerate(maps[s]):
            F[c, s * n:(s + 1) * n] += As[s][k]
    C = np.vstack([np.array(rows), F])
    Nul = sla.null_space(C)
    assert Nul.shape[1] > 0
    cstar = (Nul @ np.random.default_rng(1).standard_normal(Nul.shape[1])).reshape(N, n)
    rhs = np.zeros_like(w.rhs)
    ustar = np.zeros(g.n_gamma)
    for s in range(N):
        ri, rb, rg = g.rows(s)
        v = Ks[s] @ cstar[s]
        rhs[s, :rb.stop] = v[:rb.stop]
        ustar[g.dof[s, rg]] = v[rg]
    res = O.solve(g, w.W, w.b, rhs)
    assert res.rdiag_ratio.min() > 1e-6
    assert np.linalg.norm(res.u_gamma - ustar) <= 1e-8 * np.linalg.norm(ustar)
    assert np.linalg.norm(res.c - cstar) <= 1e-6 * np.linalg.norm(cstar)
