"""Failure detection and the geometry query of the C ABI, on the GPU.

The bounded waits of the interface solve are made to run out on purpose through the
library's test hook (every grid barrier waits for one arrival more than the grid has,
i.e. for a release that nothing sends): the kernels must give up within the limit,
elm_ddm_check must report ELM_DDM_ERR_TIMEOUT, and the same handle must then solve
correctly with the default limit.  No GPU fault, trap or hang is involved: the waits
are bounded and have no asynchronous copy in flight.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2406_15959_gb300 import elm_ddm as E
from paper_2406_15959_gb300 import workload as wl

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

DEV = torch.device("cuda:0")


def _solver(w):
    s = E.Solver(w.geom, w.n_neurons)
    s.assemble(torch.as_tensor(w.W, device=DEV), torch.as_tensor(w.b, device=DEV))
    s.schur()
    return s


def test_interface_solve_wait_runs_out_then_recovers():
    w = wl.build(4, 4, 120, 12, 12, 24, 24, theta="paper", theta_seed=7, source="fourier",
                 source_seed=7, n_test_side=20)
    s = _solver(w)
    assert s.cooperative_solves, "this case must use the cooperative triangular solves"
    rhs = torch.as_tensor(w.rhs, device=DEV)
    ug_ref, c_ref = s.solve(rhs)
    s.check()
    ug_ref, c_ref = ug_ref.clone(), c_ref.clone()
    # every barrier withholds its release; a 5 ms limit ends each wait
    s.set_wait_limit(0.005, hold_release=True)
    s.solve(rhs)
    with pytest.raises(E.ElmDdmError) as ei:
        s.check()
    assert ei.value.code == E.ERR_TIMEOUT
    # the status word was cleared by the check; the context and the handle still work
    s.set_wait_limit(2.0, hold_release=False)
    ug, c = s.solve(rhs)
    s.check()
    assert torch.equal(ug, ug_ref) and torch.equal(c, c_ref)


def test_set_wait_limit_rejects_bad_arguments():
    w = wl.build(2, 2, 20, 6, 6, 6, 6, theta="paper", theta_seed=1, n_test_side=10)
    s = E.Solver(w.geom, w.n_neurons)
    for sec, hold in [(-1.0, 0), (61.0, 0), (float("nan"), 0), (1.0, 2)]:
        with pytest.raises(E.ElmDdmError) as ei:
            s.set_wait_limit(sec, hold)
        assert ei.value.code == E.ERR_ARG
    s.close()


def test_get_points_returns_the_setup_geometry():
    w = wl.build(3, 2, 30, 7, 5, 6, 8, theta="paper", theta_seed=2, n_test_side=10)
    g = w.geom
    s = E.Solver(g, w.n_neurons)
    for kind, col in [(E.PTS_INTERIOR, 0), (E.PTS_BOUNDARY, 1), (E.PTS_INTERFACE, 2), (E.PTS_NORMALS, 2)]:
        pts, counts = s.get_points(kind)
        pts = pts.cpu().numpy()
        np.testing.assert_array_equal(counts, g.counts[:, col])
        for sd in range(g.n_sub):
            sl = g.rows(sd)[col]
            src = g.nrm if kind == E.PTS_NORMALS else g.xy
            np.testing.assert_array_equal(pts[sd, :counts[sd]], src[sd, sl])
            assert not pts[sd, counts[sd]:].any()
    with pytest.raises(E.ElmDdmError):
        s.get_points(4)
    s.close()
