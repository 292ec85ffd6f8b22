"""GPU parity of the corner rule (the remark in Section 3): the paper's grid with its cross
points, where one interface unknown is shared by four subdomains and A^s has one row per
edge through the point, with that edge's normal (elm_ddm_setup_flux).  CUDA path through the
C ABI against the FP64 CPU oracle, with the tolerances of test_gpu_parity: assembly rtol
1e-13, u and u_Gamma relative L2 <= 1e-8, factor pieces on well-conditioned cases."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import elm_oracle as O
from paper_2406_15959_gb300 import elm_ddm as E
from paper_2406_15959_gb300 import workload as wl

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

DEV = torch.device("cuda:0")

CASES = {
    # one cross point; 31 interface rows per subdomain (two edges of 15 and the corner)
    "2x2_k16": dict(G=2, n_grid=33, n=120, theta="local_unit"),
    # four cross points, interior subdomain with all four corners (48 interface rows)
    "3x3_k12": dict(G=3, n_grid=37, n=100, theta="paper"),
    # nine cross points, ragged edge groups (15 points + 1 or 2 corner rows), K^s of
    # 289 .. 324 rows over two 128-column outer QR blocks
    "4x4_k16": dict(G=4, n_grid=65, n=200, theta="paper"),
    # well-conditioned local problems, for the factor pieces
    "3x3_wellcond": dict(G=3, n_grid=31, n=30, theta="local_unit"),
}

_cache = {}


def get(name):
    if name not in _cache:
        c = CASES[name]
        w = wl.paper_grid_workload(c["G"], n_total=c["n"] * c["G"] ** 2, theta=c["theta"], seed=11,
                                   source="sin2pi_exp", n_grid=c["n_grid"], n_test_side=40,
                                   cross_points=True)
        res = O.solve(w.geom, w.W, w.b, w.rhs)
        u, g = O.evaluate(w.W, w.b, res.c, w.test_xy, w.test_owner)
        _cache[name] = (w, res, u, g)
    return _cache[name]


def t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV, dtype=dtype)


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def run(w, fp64_simt=False, ridge=None):
    s = E.Solver(w.geom, w.n_neurons, fp64_simt=fp64_simt, ridge=ridge)
    s.assemble(t(w.W), t(w.b))
    s.schur()
    ug, c = s.solve(t(w.rhs))
    u, g = s.eval(t(w.test_xy), t(w.test_owner, torch.int32), c)
    s.check()
    return s, ug, c, u, g


@pytest.mark.parametrize("name", list(CASES))
def test_corner_rows_assemble_like_the_oracle(name):
    """A^s rows at explicit (point, normal) pairs, the two rows per cross point included."""
    w, _, _, _ = get(name)
    g = w.geom
    s = E.Solver(g, w.n_neurons)
    s.assemble(t(w.W), t(w.b))
    for sd in range(g.n_sub):
        frow, fnrm, _ = O.flux_rows(g, sd)
        _, A = O.assemble_local(g.xy[sd], g.nrm[sd], g.counts[sd], w.W[sd], w.b[sd], flux=(frow, fnrm))
        Ag = s.export(E.BUF_A, sd).cpu().numpy()
        assert Ag.shape == A.shape == (int(g.flux.count[sd]), w.n_neurons)
        np.testing.assert_allclose(Ag, A, rtol=1e-13, atol=1e-14 * np.abs(A).max())
    s.check()
    s.close()


@pytest.mark.parametrize("fp64_simt", [False, True], ids=["tensor-core", "fp64-pipe"])
@pytest.mark.parametrize("name", list(CASES))
def test_corner_rule_solution_matches_oracle(name, fp64_simt):
    w, res, u_or, g_or = get(name)
    s, ug, c, u, g = run(w, fp64_simt)
    assert rel(ug.cpu().numpy(), res.u_gamma) <= 1e-8, rel(ug.cpu().numpy(), res.u_gamma)
    assert rel(u.cpu().numpy(), u_or) <= 1e-8
    assert rel(g.cpu().numpy(), g_or) <= 1e-7
    if res.rdiag_ratio.min() > 1e-6:
        assert rel(c.cpu().numpy(), res.c) <= 1e-8
    s.close()


@pytest.mark.parametrize("fp64_simt", [False, True], ids=["tensor-core", "fp64-pipe"])
def test_corner_rule_factor_pieces_match_oracle(fp64_simt):
    """M_s has one row per A-row (m_F x m_Gamma); S = sum E^T D E + M^T M with M's rows the
    flux conditions: L L^T against the oracle's S entrywise."""
    w, res, _, _ = get("3x3_wellcond")
    assert res.rdiag_ratio.min() > 1e-6
    s, *_ = run(w, fp64_simt)
    for sd, L in enumerate(res.locs):
        D = s.export(E.BUF_D, sd).cpu().numpy()
        M = s.export(E.BUF_M, sd).cpu().numpy()
        assert M.shape == L.M.shape
        assert np.abs(D - L.D).max() <= 1e-11
        assert np.abs(M - L.M).max() <= 1e-10 * max(1.0, np.abs(L.M).max())
    Lg = np.tril(s.export(E.BUF_L).cpu().numpy())
    inv = np.argsort(s.interface_order())
    S_or = res.S[np.ix_(inv, inv)]
    assert np.abs(Lg @ Lg.T - S_or).max() <= 1e-11 * np.abs(res.S).max()
    s.close()


def test_corner_rule_has_no_cg_interface_solve():
    w, _, _, _ = get("2x2_k16")
    s, *_ = run(w)
    with pytest.raises(E.ElmDdmError) as ei:
        s.solve_cg(t(w.rhs))
    assert ei.value.code == E.ERR_STATE
    s.close()


def test_corner_rule_at_the_papers_size_matches_oracle():
    """Table 2's 8 x 8 setup with the cross points kept (n = 65,536 neurons, the global
    257 x 257 grid: 49 cross points, each an unknown of four subdomains with four flux
    conditions), Tikhonov-regularised local least squares (alpha = 1e-14) as in the
    cross-point-free Table 2 test: GPU against the oracle's ridge solve, and the error
    against the exact solution at Table 2's accuracy."""
    w = wl.paper_grid_workload(8, seed=7, cross_points=True)
    assert w.geom.n_gamma == 2 * 8 * 7 * 31 + 49
    ue = w.src.u(w.test_xy)
    res = O.solve(w.geom, w.W, w.b, w.rhs, keep=False, ridge=1e-14)
    u_or, _ = O.evaluate(w.W, w.b, res.c, w.test_xy, w.test_owner)
    s, ug, c, u, _ = run(w, ridge=1e-14)
    u = u.cpu().numpy()
    assert rel(u, u_or) <= 1e-8, rel(u, u_or)
    assert rel(ug.cpu().numpy(), res.u_gamma) <= 1e-8
    assert rel(u, ue) < 1e-8, rel(u, ue)
    s.close()
