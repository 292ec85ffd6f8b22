"""The two assembly routes of step (a) against the FP64 oracle, entry by entry.

Where the collocation points share few x and y coordinates (the paper's grids) the
library factors exp(2 z) into per-neuron tables over those coordinates instead of one
tanh per entry; ELM_DDM_FLAG_DIRECT_ASSEMBLY forces one tanh per entry.  Both must agree
with the oracle to the rounding of the activation's argument z = w . x + b: an entry
t = tanh(z) moves by (1 - t^2) dz with |dz| a few ulp of |w_x x| + |w_y y| + |b|, an
interior entry 2 |w|^2 t (1 - t^2) by 2 |w|^2 times that, an interface-derivative entry
(w . n)(1 - t^2) by |w| times that.  The bound below is 64 ulp of that scale; with
the paper's weights (|w| up to c sqrt(N n_N)) it is still far below what a wrong
formula, a wrong index into the tables or a dropped term would give (order 1 of the
entry).  Off-grid points must take the direct route and still match the oracle's
solution.
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

EPS = np.finfo(np.float64).eps

CASES = {
    "2x2_n200": wl.poisson_2x2_n200,
    "3x3_ragged": lambda: wl.build(3, 3, 150, 17, 13, 23, 21, theta="paper", theta_seed=5,
                                   source="fourier", source_seed=5, n_test_side=40),
    "3x3_radial": lambda: wl.build(3, 3, 110, 13, 12, 18, 16, theta="radial", theta_seed=13,
                                   source="sin2pi_exp", n_test_side=40),
    "4x4_n1000": wl.poisson_4x4_n1000,
}


def t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda", dtype=dtype)


def bounds(xy, counts, W, b):
    """Per-entry tolerance of K^s and A^s (see the module docstring)."""
    mi, mb, mg = (int(v) for v in counts)
    m = mi + mb + mg
    zs = np.abs(xy[:m, 0:1]) * np.abs(W[None, :, 0]) + np.abs(xy[:m, 1:2]) * np.abs(W[None, :, 1]) \
        + np.abs(b)[None, :] + 1.0
    wsq = (W * W).sum(axis=1)
    tk = 64 * EPS * zs
    tk[:mi] *= np.maximum(2.0 * wsq, 1.0)[None, :]
    ta = 64 * EPS * zs[mi + mb:] * np.maximum(np.sqrt(wsq), 1.0)[None, :]
    return tk, ta


def check_against_oracle(s, w):
    g = w.geom
    n = w.n_neurons
    worst = 0.0
    for sd in range(g.n_sub):
        K, A = O.assemble_local(g.xy[sd], g.nrm[sd], g.counts[sd], w.W[sd], w.b[sd])
        tk, ta = bounds(g.xy[sd], g.counts[sd], w.W[sd], w.b[sd])
        Kg = s.export(E.BUF_K, sd).cpu().numpy()[:, :n]
        worst = max(worst, float((np.abs(Kg - K) / tk).max()))
        assert np.all(np.abs(Kg - K) <= tk), (sd, float((np.abs(Kg - K) / tk).max()))
        if int(g.counts[sd][2]):
            Ag = s.export(E.BUF_A, sd).cpu().numpy()
            assert np.all(np.abs(Ag - A) <= ta), (sd, float((np.abs(Ag - A) / ta).max()))
    return worst


@pytest.mark.parametrize("name", list(CASES))
def test_factored_and_direct_assembly_match_oracle(name):
    w = CASES[name]()
    st = E.Solver(w.geom, w.n_neurons)
    sd = E.Solver(w.geom, w.n_neurons, direct_assembly=True)
    assert st.info(8) == 1.0 and sd.info(8) == 0.0
    for s in (st, sd):
        s.assemble(t(w.W), t(w.b))
        check_against_oracle(s, w)
        s.check()


def test_factored_assembly_variable_coefficient():
    w = wl.build(3, 3, 120, 14, 12, 20, 18, theta="paper", theta_seed=21, coef="grf",
                 coef_seed=3, coef_alpha=4.0, n_test_side=30)
    s = E.Solver(w.geom, w.n_neurons, op=E.OP_VARCOEF)
    assert s.info(8) == 1.0
    s.set_coefficient(t(w.coef_rows))
    s.assemble(t(w.W), t(w.b))
    g = w.geom
    n = w.n_neurons
    for k in range(g.n_sub):
        K, _ = O.assemble_local(g.xy[k], g.nrm[k], g.counts[k], w.W[k], w.b[k], coef=w.coef_rows[k])
        tk, _ = bounds(g.xy[k], g.counts[k], w.W[k], w.b[k])
        mi = int(g.counts[k][0])
        # the coefficient rows add (grad rho . w)(1 - t^2): scale by |rho| + |grad rho| |w|
        c = w.coef_rows[k][:mi]
        tk[:mi] *= (np.abs(c[:, 0:1]) + np.abs(c[:, 1:2]) + np.abs(c[:, 2:3]) + 1.0)
        Kg = s.export(E.BUF_K, k).cpu().numpy()[:, :n]
        assert np.all(np.abs(Kg - K) <= tk), (k, float((np.abs(Kg - K) / tk).max()))
    s.check()


def test_off_grid_points_take_the_direct_route():
    """Interior points jittered off the grid: every row has its own coordinates, the
    tables would not save work, and the direct route must give the oracle's solution."""
    w = wl.build(3, 3, 120, 14, 12, 20, 18, theta="paper", theta_seed=11, source="fourier",
                 source_seed=11, n_test_side=40)
    g = w.geom
    rng = np.random.default_rng(5)
    for k in range(g.n_sub):
        mi = int(g.counts[k][0])
        g.xy[k][:mi] += rng.uniform(-1e-3, 1e-3, size=(mi, 2)) / 3.0
    w.rhs = wl.rhs_rows(g, w.src)  # the data at the moved points
    s = E.Solver(g, w.n_neurons)
    assert s.info(8) == 0.0
    s.assemble(t(w.W), t(w.b))
    check_against_oracle(s, w)
    s.schur()
    ug, c = s.solve(t(w.rhs))
    res = O.solve(g, w.W, w.b, w.rhs)
    u_or, _ = O.evaluate(w.W, w.b, res.c, w.test_xy, w.test_owner)
    u, _ = s.eval(t(w.test_xy), t(w.test_owner, torch.int32), c)
    u = u.cpu().numpy()
    assert np.linalg.norm(u - u_or) <= 1e-8 * np.linalg.norm(u_or)
    s.check()
