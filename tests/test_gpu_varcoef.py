"""GPU parity for the variable-coefficient operator -div(rho grad u) = f (Section 4)
against the oracle: assembly elementwise, the solution at the test points and u_Gamma
to 1e-8 (both back ends), the manufactured-solution error, and the call-order checks.

The paper's own case (rho = tanh(grf) + 1.1 with alpha = 16) is nearly a step function
with |grad rho| up to ~3e3; at 4x4 x 800 neurons its local least-squares problems are
unresolved and so ill-conditioned that two backward-stable solvers return different fits
(parity unpinned there, like c on rank-deficient K^s).  The same coefficient with a
smooth field (alpha = 4) is pinned here; the alpha = 16 workload is only run.
"""
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
    "3x3_sine": lambda: wl.build(3, 3, 120, 14, 12, 16, 15, theta="paper", theta_seed=11,
                                 source="sinsin", coef="sine", coef_seed=11, n_test_side=50),
    "varcoef_4x4_n800": wl.varcoef_4x4_n800,
    # the paper's coefficient rho = tanh(grf) + 1.1 with a smooth field and a manufactured
    # solution (f = 1 leaves a large least-squares residual, whose solution sensitivity
    # grows with kappa^2 times the residual: 8e-5 between two solvers on this case)
    "3x3_grf_alpha4": lambda: wl.build(3, 3, 150, 16, 16, 20, 20, theta="paper", theta_seed=12,
                                       source="sinsin", coef="grf", coef_seed=12, coef_alpha=4.0,
                                       n_test_side=50),
}

_cache = {}


def get(name):
    if name not in _cache:
        w = CASES[name]()
        res = O.solve(w.geom, w.W, w.b, w.rhs, keep=False, coef=w.coef_rows)
        u, g = O.evaluate(w.W, w.b, res.c, w.test_xy, w.test_owner)
        _cache[name] = (w, res, u)
    return _cache[name]


def t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV, dtype=dtype)


def solver(w, fp64_simt=False):
    s = E.Solver(w.geom, w.n_neurons, fp64_simt=fp64_simt, op=E.OP_VARCOEF)
    s.set_coefficient(t(w.coef_rows))
    s.assemble(t(w.W), t(w.b))
    return s


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def test_varcoef_assembly_matches_oracle():
    w, _, _ = get("3x3_sine")
    s = solver(w)
    g = w.geom
    for sd in range(g.n_sub):
        K, A = O.assemble_local(g.xy[sd], g.nrm[sd], g.counts[sd], w.W[sd], w.b[sd], w.coef_rows[sd])
        Kg = s.export(E.BUF_K, sd).cpu().numpy()[:, :w.n_neurons]
        np.testing.assert_allclose(Kg, K, rtol=1e-13, atol=1e-14 * np.abs(K).max())
        if int(g.counts[sd][2]):
            Ag = s.export(E.BUF_A, sd).cpu().numpy()
            np.testing.assert_allclose(Ag, A, rtol=1e-13, atol=1e-14 * np.abs(A).max())
    s.check()


@pytest.mark.parametrize("fp64_simt", [False, True], ids=["tensor-core", "fp64-pipe"])
@pytest.mark.parametrize("name", list(CASES))
def test_varcoef_solution_matches_oracle(name, fp64_simt):
    w, res, u_or = get(name)
    s = solver(w, fp64_simt)
    s.schur()
    ug, c = s.solve(t(w.rhs))
    u, gr = s.eval(t(w.test_xy), t(w.test_owner, torch.int32), c)
    s.check()
    assert rel(u.cpu().numpy(), u_or) <= 1e-8
    assert rel(ug.cpu().numpy(), res.u_gamma) <= 1e-8
    if w.src.has_exact:
        l2, _ = O.rel_errors(u.cpu().numpy(), gr.cpu().numpy(), w.src.u(w.test_xy),
                             w.src.grad_u(w.test_xy))
        assert l2 < 1e-6, l2


def test_varcoef_call_order_and_arguments():
    w, _, _ = get("3x3_sine")
    s = E.Solver(w.geom, w.n_neurons, op=E.OP_VARCOEF)
    with pytest.raises(E.ElmDdmError) as ei:      # no coefficient yet
        s.assemble(t(w.W), t(w.b))
    assert ei.value.code == E.ERR_STATE
    p = E.Solver(w.geom, w.n_neurons)              # the Poisson operator takes none
    with pytest.raises(E.ElmDdmError) as ei:
        p.set_coefficient(t(w.coef_rows))
    assert ei.value.code == E.ERR_ARG
    bad = w.coef_rows.copy()
    bad[0, 0, 0] = np.nan
    s.set_coefficient(t(bad))
    s.assemble(t(w.W), t(w.b))
    with pytest.raises(E.ElmDdmError) as ei:
        s.check()
    assert ei.value.code == E.ERR_NONFINITE


def test_paper_grf_coefficient_runs():
    """The paper's variable-coefficient problem at alpha = 16: the solve completes with
    finite output and no status bit (its fit is not identifiable at this resolution)."""
    w = wl.varcoef_grf_4x4_n800()
    s = solver(w)
    s.schur()
    ug, c = s.solve(t(w.rhs))
    u, _ = s.eval(t(w.test_xy), t(w.test_owner, torch.int32), c)
    s.check()
    assert torch.isfinite(u).all() and torch.isfinite(ug).all()
