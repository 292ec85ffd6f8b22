"""The learned interface warm start on the GPU: the network's forward pass, loss gradient
and Adam step against the FP64 oracle (oracle/mlp_oracle.py, itself pinned by finite
differences), and the gain of the trained network as the initial guess of the CG
interface solve, with the direct solve as the reference for the error.

Tolerances: the library computes in FP32, its layer products on the tensor cores as three
TF32 products of a hi/lo split (about 2^-21 relative per product term instead of an FP32
FMA's 2^-24).  A forward value or gradient entry is a sum of at most a few hundred such
products (relative error <= K * 2^-21 ~ 2.4e-4 for K = 512 in the worst case, about
sqrt(K) * 2^-21 ~ 1e-5 for terms of random sign), so forward values are compared at 1e-5
and gradients at 1e-4 relative to each block's norm; one Adam step moves every parameter
by about lr, so parameters after a step are compared at 1e-3 lr absolute (the gradient's
relative error enters the step only through m / sqrt(v)).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp_oracle as MO
from paper_2406_15959_gb300 import elm_ddm as E
from paper_2406_15959_gb300 import mlp as M
from paper_2406_15959_gb300 import warmstart as WS
from paper_2406_15959_gb300 import workload as wl

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

D_IN, D_H, D_OUT, B = 9, 70, 130, 37   # ragged against the 64 x 64 tiles


def blocks(v):
    sizes = [D_IN * D_H, D_H, D_H * D_H, D_H, D_H * D_OUT, D_OUT]
    return np.split(np.asarray(v, dtype=np.float64), np.cumsum(sizes)[:-1])


def make(seed=3):
    rng = np.random.default_rng(seed)
    net = M.MLP(D_IN, D_H, D_OUT, 64, seed=seed)
    X = torch.as_tensor(rng.standard_normal((B, D_IN)), dtype=torch.float32, device="cuda")
    T = torch.as_tensor(rng.standard_normal((B, D_OUT)), dtype=torch.float32, device="cuda")
    return net, X, T


def test_mlp_forward_and_gradient_match_oracle():
    net, X, T = make()
    p = net.params().cpu().numpy().astype(np.float64)
    Xn, Tn = X.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64)
    y_or, _ = MO.forward(p, Xn, D_IN, D_H, D_OUT)
    y = net.forward(X).cpu().numpy()
    assert np.linalg.norm(y - y_or) <= 1e-5 * np.linalg.norm(y_or)
    loss, g = net.gradient(X, T)
    l_or, g_or = MO.loss_and_grad(p, Xn, Tn, D_IN, D_H, D_OUT)
    assert abs(float(loss) - l_or) <= 1e-5 * l_or
    for gb, ob in zip(blocks(g.cpu().numpy()), blocks(g_or)):
        assert np.linalg.norm(gb - ob) <= 1e-4 * np.linalg.norm(ob)


@pytest.mark.parametrize("dims", [(64, 300, 700, 200), (33, 129, 257, 129)])
def test_mlp_spanning_several_tiles_matches_oracle(dims):
    """Layer products over several 128 x 64 output tiles and 16-wide K chunks, ragged in
    every dimension, against the FP64 oracle."""
    d_in, d_h, d_out, b = dims
    rng = np.random.default_rng(11)
    net = M.MLP(d_in, d_h, d_out, b, seed=4)
    X = torch.as_tensor(rng.standard_normal((b, d_in)), dtype=torch.float32, device="cuda")
    T = torch.as_tensor(rng.standard_normal((b, d_out)), dtype=torch.float32, device="cuda")
    p = net.params().cpu().numpy().astype(np.float64)
    Xn, Tn = X.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64)
    y_or, _ = MO.forward(p, Xn, d_in, d_h, d_out)
    y = net.forward(X).cpu().numpy()
    assert np.linalg.norm(y - y_or) <= 1e-5 * np.linalg.norm(y_or)
    _, g = net.gradient(X, T)
    _, g_or = MO.loss_and_grad(p, Xn, Tn, d_in, d_h, d_out)
    sizes = [d_in * d_h, d_h, d_h * d_h, d_h, d_h * d_out, d_out]
    for gb, ob in zip(np.split(g.cpu().numpy().astype(np.float64), np.cumsum(sizes)[:-1]),
                      np.split(g_or, np.cumsum(sizes)[:-1])):
        assert np.linalg.norm(gb - ob) <= 1e-4 * np.linalg.norm(ob)
    net.check()
    net.close()


def test_adam_step_matches_oracle():
    net, X, T = make(5)
    p0 = net.params().cpu().numpy().astype(np.float64)
    lr = 1e-2
    net.train_step(X, T, lr)
    p1 = net.params().cpu().numpy().astype(np.float64)
    _, g = MO.loss_and_grad(p0, X.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64),
                            D_IN, D_H, D_OUT)
    p1_or, _, _ = MO.adam_step(p0, g, np.zeros_like(p0), np.zeros_like(p0), 1, lr)
    assert np.abs(p1 - p1_or).max() <= 1e-3 * lr


def test_training_reduces_the_loss():
    net, X, T = make(7)
    l0 = float(net.gradient(X, T)[0])
    for _ in range(200):
        net.train_step(X, T, 3e-3)
    l1 = float(net.gradient(X, T)[0])
    assert l1 < 0.05 * l0


def test_mlp_rejects_bad_arguments():
    net, X, T = make()
    with pytest.raises(E.ElmDdmError):
        net.train_step(X, T, 0.0)
    with pytest.raises(E.ElmDdmError):
        net.forward(torch.zeros((65, D_IN), dtype=torch.float32, device="cuda"))  # > max_batch


def test_warm_start_saves_cg_steps():
    """4x4 subdomains (n_Gamma = 2400), sources with 4 x 4 sine modes: 2048 method-generated
    solves train the network; on held-out sources the preconditioned CG (diagonal and
    per-edge block-Jacobi) started at its prediction needs clearly fewer steps than from
    zero, and ends within the tolerance's reach of the direct solution.  The direct
    RHS-only solve of the same handle is timed beside it: it is the bar a warm-started
    iterative solve has to beat, and the test records (does not assert) how far off it is."""
    w = wl.poisson_4x4_n1000()
    s = E.Solver(w.geom, w.n_neurons, max_rhs=64, block_jacobi=True)
    s.assemble(torch.as_tensor(w.W, device="cuda"), torch.as_tensor(w.b, device="cuda"))
    s.schur()
    basis = wl.fourier_basis_rows(w.geom, 4)
    A, U = WS.generate(s, basis, 2048, seed=1)
    ws = WS.WarmStart(16, w.geom.n_gamma, max_batch=256, seed=2)
    losses = ws.fit(A, U, epochs=60, batch=128, lr=2e-3)
    assert losses[-1] < 0.05 * losses[0]
    At = np.random.default_rng(42).standard_normal((4, 16))
    precs = ["jacobi", "block"]
    rows = WS.evaluate(s, ws, basis, At, tol=1e-9, precs=precs)
    summ = WS.summarise(rows, precs)
    print("warm start:", summ)
    for name in precs:
        cold, warm = summ[name]["cold_steps"], summ[name]["warm_steps"]
        # the step counts move with the rounding of D_s and M_s (S is determined by the data
        # only to a few percent at this initialisation), so the bar is a 10% saving, not a
        # ratio tuned to one build
        assert warm < 0.9 * cold, (name, warm, cold)
        # CG error bound kappa_M * tol with kappa_M <= kappa(S) = 2.9e5 at this size
        assert summ[name]["warm_rel_err_vs_direct_max"] < 1e-3, (name, summ[name])
    assert summ["block"]["cold_steps"] <= summ["jacobi"]["cold_steps"], summ
    assert max(r["prediction_rel_err"] for r in rows) < 0.1
    s.check()
