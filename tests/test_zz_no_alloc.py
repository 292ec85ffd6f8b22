"""The no-allocation Cholesky solve, elm_ddm_chol_solve_noalloc, called through the C ABI.

It serves callers that cannot call cudaMalloc (a CUDA graph being captured in global
mode, a host that owns all device memory through its own pool, a real-time loop).
The test checks its output against the interface solution u_Gamma that elm_ddm_solve
computes with the same Cholesky factor, on two calls in a row (the fixed scratch array
keeps the first call's contents when the second one runs), that the second call
changes the device's free memory by nothing, and that three right-hand sides in one
call give what the three give one at a time.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2406_15959_gb300 import elm_ddm as E
from paper_2406_15959_gb300 import workload as wl

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

MAX_ELEMS = 131072  # ELM_DDM_NOALLOC_MAX_ELEMS in include/elm_ddm.h


def _fn():
    lib = E.load()
    f = lib.elm_ddm_chol_solve_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def test_noalloc_solve_matches_elm_ddm_solve_on_two_calls():
    dev = torch.device("cuda:0")
    w = wl.build(3, 3, 150, 17, 13, 23, 21, theta="paper", theta_seed=5, source="fourier",
                 source_seed=5, n_test_side=20)
    srcs = [w.rhs, wl.rhs_rows(w.geom, wl.make_source("fourier", seed=11, modes=3))]
    s = E.Solver(w.geom, w.n_neurons)
    s.assemble(torch.as_tensor(w.W, device=dev), torch.as_tensor(w.b, device=dev))
    s.schur()
    ref = []
    for r in srcs:
        ug, _ = s.solve(torch.as_tensor(r, device=dev))
        ref.append(ug.clone())
    s.check()
    n = w.geom.n_gamma
    L = s.export(E.BUF_L)                        # the factor, indexed L[i, j]
    inv = torch.as_tensor(np.argsort(s.interface_order()), device=dev)  # internal -> caller
    Lcm = L.t().contiguous()                     # its column-major buffer
    Ltri = torch.tril(L)
    stream = torch.cuda.current_stream(dev)
    f = _fn()
    free = []
    for k, u_user in enumerate(ref):
        u_ref = u_user[inv].contiguous()           # u_Gamma in the factor's internal order
        b = (Ltri @ (Ltri.t() @ u_ref)).contiguous()   # S u_Gamma with S = L L^T
        u = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
        torch.cuda.synchronize(dev)
        free.append(torch.cuda.mem_get_info(dev)[0])
        rc = f(Lcm.data_ptr(), n, n, b.data_ptr(), 1, u.data_ptr(), stream.cuda_stream)
        assert rc == E.OK
        torch.cuda.synchronize(dev)
        err = (torch.linalg.norm(u - u_ref) / torch.linalg.norm(u_ref)).item()
        assert err <= 1e-8, (k, err)
    free.append(torch.cuda.mem_get_info(dev)[0])
    assert free[1] == free[2]                    # the second call allocated nothing
    # three right-hand sides in one call ([nrhs][n] layout, each its own grid row) against
    # the same three solved one at a time
    us = [ref[0][inv], ref[1][inv], (ref[0] - 2.0 * ref[1])[inv]]
    B = torch.stack([(Ltri @ (Ltri.t() @ v)) for v in us]).contiguous()
    U = torch.full((3, n), float("nan"), dtype=torch.float64, device=dev)
    assert f(Lcm.data_ptr(), n, n, B.data_ptr(), 3, U.data_ptr(), stream.cuda_stream) == E.OK
    one = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
    for k in range(3):
        bk = B[k].contiguous()
        assert f(Lcm.data_ptr(), n, n, bk.data_ptr(), 1, one.data_ptr(), stream.cuda_stream) == E.OK
        torch.cuda.synchronize(dev)
        assert (torch.linalg.norm(U[k] - one) / torch.linalg.norm(one)).item() <= 1e-12, k
        assert (torch.linalg.norm(U[k] - us[k]) / torch.linalg.norm(us[k])).item() <= 1e-8, k
    s.close()


def test_noalloc_solve_rejects_sizes_beyond_its_scratch():
    f = _fn()
    dev = torch.device("cuda:0")
    x = torch.zeros(4, dtype=torch.float64, device=dev)
    # n * nrhs one past the capacity: refused before anything is enqueued
    assert f(x.data_ptr(), MAX_ELEMS // 2 + 1, MAX_ELEMS // 2 + 1, x.data_ptr(), 2,
             x.data_ptr(), None) == E.ERR_CAPACITY
    assert f(x.data_ptr(), 4, 3, x.data_ptr(), 1, x.data_ptr(), None) == E.ERR_ARG
    # within the capacity but more right-hand sides than a grid's y dimension holds
    assert f(x.data_ptr(), 1, 1, x.data_ptr(), 65536, x.data_ptr(), None) == E.ERR_ARG
    assert f(None, 4, 4, x.data_ptr(), 1, x.data_ptr(), None) == E.ERR_ARG
