"""Mixed precision on the GPU (ELM_DDM_FLAG_MIXED): low-precision local factorisation
(FP32 Householder panels, digit-split products with the 10 leading BF16 digit pairs and
FP32 accumulation), FP64 Schur factorisation, refinement on FP64 residuals, and the
fallback to the FP64 path when refinement stalls.

Every result is compared with the FP64 oracle at the same bar as the FP64 path (relative
L2 <= 1e-8 of u at the test points and of u_Gamma); the library's own error estimate
(the last relative u_Gamma correction) is checked against the measured error.
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


def t(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV, dtype=dtype)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - b) / max(np.linalg.norm(b), 1e-300)


def run(w, mixed=True, max_rhs=1, rhs=None):
    s = E.Solver(w.geom, w.n_neurons, mixed=mixed, max_rhs=max_rhs)
    s.assemble(t(w.W), t(w.b))
    s.schur()
    ug, c = s.solve(t(w.rhs if rhs is None else rhs))
    u, g = s.eval(t(w.test_xy), t(w.test_owner, torch.int32), c)
    s.check()
    return s, ug, c, u, g


WELL = {
    # local U(-1, 1) weights with few neurons: kappa(K^s) 1e5 .. 2e7 (the largest per case in
    # the comments, from numpy's SVD), so kappa * 2^-24 < 1 or close to it and refinement from
    # FP32-level factors converges
    "3x3_local": lambda: wl.build(3, 3, 60, 12, 12, 12, 12, theta="local_unit", theta_seed=3,
                                  source="fourier", source_seed=3, n_test_side=40),     # 1.7e7
    "2x2_n40_local": lambda: wl.build(2, 2, 40, 10, 10, 10, 10, theta="local_unit", theta_seed=1,
                                      source="sinsin", n_test_side=40),                # 2.1e5
    "4x4_n40_local": lambda: wl.build(4, 4, 40, 12, 12, 12, 12, theta="local_unit", theta_seed=5,
                                      source="fourier", source_seed=5, n_test_side=40),  # 1.3e6
    # 3120 rows: the FP32 panels run on 4-CTA clusters
    "4x4_n50_tall_local": lambda: wl.build(4, 4, 50, 60, 50, 30, 30, theta="local_unit", theta_seed=6,
                                           source="sinsin", n_test_side=40),           # 2.0e6
    "8x8_n40_local": lambda: wl.build(8, 8, 40, 12, 10, 10, 10, theta="local_unit", theta_seed=9,
                                      source="fourier", source_seed=9, n_test_side=40),  # 3.3e6
    "1x1_local": lambda: wl.build(1, 1, 50, 12, 11, 15, 1, theta="local_unit", theta_seed=7,
                                  source="sinsin", n_test_side=30),
}


@pytest.mark.parametrize("name", list(WELL))
def test_refinement_converges_to_the_oracle(name):
    w = WELL[name]()
    res = O.solve(w.geom, w.W, w.b, w.rhs)
    u_or, _ = O.evaluate(w.W, w.b, res.c, w.test_xy, w.test_owner)
    s, ug, c, u, g = run(w)
    info = s.refinement
    assert not info["fell_back"] and info["low_precision_factor"], info
    assert 2 <= info["steps"] <= 16 and info["eta"] <= 1e-10, info
    err_u = rel(u.cpu().numpy(), u_or)
    assert err_u <= 1e-8, (err_u, info)
    if w.geom.n_gamma:
        err_g = rel(ug.cpu().numpy(), res.u_gamma)
        assert err_g <= 1e-8, (err_g, info)
        # the library's estimate: the last correction bounds the remaining error's order
        assert err_g <= max(1e3 * info["eta"], 1e-13), (err_g, info)
    if res.rdiag_ratio.min() > 1e-6:
        assert rel(c.cpu().numpy(), res.c) <= 1e-8
    s.close()


@pytest.mark.parametrize("name", ["paper_2x2_n200", "local_2x2_n200"])
def test_refinement_stalls_and_falls_back_when_ill_conditioned(name):
    """Eq. (4.3) weights make kappa(K^s) ~ 1e14, and 200 local U(-1, 1) neurons on a 2 x 2
    decomposition 3.7e13: far beyond what an FP32-level factorisation can be refined from.
    The stall is detected, the handle re-assembles and factors in FP64, and the result
    matches the oracle like the FP64 path's."""
    w = (wl.build(2, 2, 200, 20, 20, 40, 40, theta="paper", theta_seed=2, source="sinsin", n_test_side=40)
         if name.startswith("paper") else wl.poisson_2x2_n200())
    res = O.solve(w.geom, w.W, w.b, w.rhs)
    u_or, _ = O.evaluate(w.W, w.b, res.c, w.test_xy, w.test_owner)
    s, ug, c, u, g = run(w)
    info = s.refinement
    assert info["fell_back"] and not info["low_precision_factor"], info
    assert rel(u.cpu().numpy(), u_or) <= 1e-8
    assert rel(ug.cpu().numpy(), res.u_gamma) <= 1e-8
    # later solves use the FP64 factorisation directly
    ug2, c2 = s.solve(t(w.rhs))
    s.check()
    assert torch.equal(ug2, ug) and torch.equal(c2, c)
    # the next assembly tries the low-precision factorisation again
    s.assemble(t(w.W), t(w.b))
    s.schur()
    assert s.refinement["low_precision_factor"]
    s.close()


def test_mixed_multiple_rhs_and_repeat():
    w = WELL["3x3_local"]()
    srcs = [wl.make_source("fourier", seed=k, modes=3) for k in range(3)]
    rhs = np.stack([wl.rhs_rows(w.geom, sr) for sr in srcs])
    s = E.Solver(w.geom, w.n_neurons, mixed=True, max_rhs=3)
    s.assemble(t(w.W), t(w.b))
    s.schur()
    ug3, c3 = s.solve(t(rhs))
    s.check()
    assert not s.refinement["fell_back"]
    for k in range(3):
        res = O.solve(w.geom, w.W, w.b, rhs[k], keep=False)
        assert rel(ug3[k].cpu().numpy(), res.u_gamma) <= 1e-8
    ug3b, c3b = s.solve(t(rhs))          # same factors, same iterates: bitwise repeatable
    s.check()
    assert torch.equal(ug3, ug3b) and torch.equal(c3, c3b)
    s.close()


def test_mixed_mode_refuses_cg_and_bad_flags():
    w = WELL["3x3_local"]()
    s = E.Solver(w.geom, w.n_neurons, mixed=True)
    s.assemble(t(w.W), t(w.b))
    s.schur()
    with pytest.raises(E.ElmDdmError) as ei:
        s.solve_cg(t(w.rhs))
    assert ei.value.code == E.ERR_STATE
    s.close()
    for kw in (dict(fp64_simt=True), dict(schur_cg=True)):
        with pytest.raises(E.ElmDdmError) as ei:
            E.Solver(w.geom, w.n_neurons, mixed=True, **kw)
        assert ei.value.code == E.ERR_ARG
