"""Learned interface warm start: an MLP maps the coefficients a of a source
f = sum a_kl sin(k pi x) sin(l pi y) to the interface variable u_Gamma of Eq. (3.5), and
its prediction starts the preconditioned CG interface solve (diagonal or per-edge
block-Jacobi); the direct solve of the same handle is the fallback and the reference for
the error, and its RHS-only time the bar the warm start is measured against.

The training set is generated by the method itself: one factorisation, then batches of
right-hand sides through the direct solve.  Network, loss and Adam run in the library's
kernels (include/elm_mlp.h); torch only holds the tensors (and shuffles and normalises the
data).  Note that u_Gamma is linear in a (the method is linear in F), so a perfect model
exists; the network has to learn it from samples like any other map.

    python -m paper_2406_15959_gb300.warmstart [--workload poisson_8x8_n1000] [--samples 20000]
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import elm_ddm as E
from . import mlp as M
from . import workload as wl


def generate(solver, basis: np.ndarray, n: int, seed: int, batch: int = 64):
    """n samples (a ~ N(0, I), u_Gamma(a) by the direct solve).  Returns (a [n, modes^2]
    float64 numpy, u [n, n_gamma] float64 CUDA tensor)."""
    import torch
    rng = np.random.default_rng(seed)
    nb = basis.shape[0]
    flat = basis.reshape(nb, -1)
    A = rng.standard_normal((n, nb))
    U = torch.empty((n, solver.n_gamma), dtype=torch.float64, device="cuda")
    for i in range(0, n, batch):
        a = A[i:i + batch]
        rhs = torch.as_tensor((a @ flat).reshape(len(a), solver.N, solver.m_max), device="cuda")
        ug, _ = solver.solve(rhs)
        U[i:i + len(a)] = ug
    solver.check()
    return A, U


class WarmStart:
    """Normalised targets (per-unknown mean and standard deviation of the training set)."""

    def __init__(self, n_in: int, n_gamma: int, hidden: int = 512, max_batch: int = 256, seed: int = 0):
        self.net = M.MLP(n_in, hidden, n_gamma, max_batch, seed=seed)
        self.max_batch = max_batch
        self.mu = self.sd = None

    def fit(self, A: np.ndarray, U, epochs: int, batch: int = 256, lr: float = 1e-3, seed: int = 0,
            lr_decay: float = 0.97):
        import torch
        self.mu = U.mean(0)
        self.sd = U.std(0).clamp_min(1e-30)
        X = torch.as_tensor(A, dtype=torch.float32, device="cuda")
        T = ((U - self.mu) / self.sd).float()
        g = torch.Generator(device="cuda").manual_seed(seed)
        losses = []
        n = X.shape[0]
        for ep in range(epochs):
            order = torch.randperm(n, device="cuda", generator=g)
            tot = torch.zeros(1, dtype=torch.float32, device="cuda")
            nb = 0
            for i in range(0, n - batch + 1, batch):
                idx = order[i:i + batch]
                tot += self.net.train_step(X[idx].contiguous(), T[idx].contiguous(), lr)
                nb += 1
            losses.append(float(tot / max(nb, 1)))
            lr *= lr_decay
        self.net.check()
        return losses

    def predict(self, A: np.ndarray):
        import torch
        X = torch.as_tensor(A, dtype=torch.float32, device="cuda")
        out = []
        for i in range(0, X.shape[0], self.max_batch):
            out.append(self.net.forward(X[i:i + self.max_batch].contiguous()).double())
        return torch.cat(out) * self.sd + self.mu


PRECONDITIONERS = {"none": False, "jacobi": True, "block": "block"}


def evaluate(solver, ws: WarmStart, basis: np.ndarray, A: np.ndarray, tol: float = 1e-9,
             maxit: int = 100000, jacobi=True, precs=None):
    """Per held-out sample: the direct RHS-only solve (time, the reference), and for every
    preconditioner in `precs` (names of PRECONDITIONERS; default: the one `jacobi` selects)
    the CG steps and wall time from zero and from the prediction, and the warm result's
    distance to the direct solve; plus the prediction's relative error.  Times are wall
    clock around each call (the CG entry points poll their convergence from the host)."""
    import torch
    if precs is None:
        precs = ["block" if jacobi == "block" else ("jacobi" if jacobi else "none")]
    flat = basis.reshape(basis.shape[0], -1)
    pred = ws.predict(A)

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, 1e3 * (time.perf_counter() - t0)

    rows = []
    for i in range(A.shape[0]):
        rhs = torch.as_tensor((A[i] @ flat).reshape(1, solver.N, solver.m_max), device="cuda")
        (ud, _), t_direct = timed(lambda: solver.solve(rhs))
        nd = float(torch.linalg.norm(ud))
        row = {"direct_ms": t_direct, "prediction_rel_err": float(torch.linalg.norm(pred[i] - ud[0])) / nd}
        for name in precs:
            pj = PRECONDITIONERS[name]
            (_, _, it0), t0 = timed(lambda: solver.solve_cg(rhs, tol=tol, maxit=maxit, jacobi=pj))
            (ug1, _, it1), t1 = timed(lambda: solver.solve_cg(rhs, tol=tol, maxit=maxit, jacobi=pj,
                                                              x0=pred[i:i + 1]))
            row[name] = {"cold_steps": it0, "cold_ms": t0, "warm_steps": it1, "warm_ms": t1,
                         "warm_rel_err_vs_direct": float(torch.linalg.norm(ug1 - ud)) / nd}
        if len(precs) == 1:  # flat keys for a single preconditioner
            row.update(row[precs[0]])
        rows.append(row)
    return rows


def summarise(rows, precs):
    out = {"direct_ms_mean": float(np.mean([r["direct_ms"] for r in rows])),
           "prediction_rel_err_mean": float(np.mean([r["prediction_rel_err"] for r in rows]))}
    for name in precs:
        out[name] = {k: float(np.mean([r[name][k] for r in rows]))
                     for k in ("cold_steps", "cold_ms", "warm_steps", "warm_ms")}
        out[name]["warm_rel_err_vs_direct_max"] = float(np.max([r[name]["warm_rel_err_vs_direct"] for r in rows]))
    return out


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="poisson_8x8_n1000")
    ap.add_argument("--samples", type=int, default=20000)
    ap.add_argument("--modes", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--test", type=int, default=16)
    args = ap.parse_args(argv)
    w = wl.WORKLOADS[args.workload]()
    s = E.Solver(w.geom, w.n_neurons, max_rhs=64, block_jacobi=True)
    s.assemble(torch.as_tensor(w.W, device="cuda"), torch.as_tensor(w.b, device="cuda"))
    s.schur()
    basis = wl.fourier_basis_rows(w.geom, args.modes)
    t0 = time.perf_counter()
    A, U = generate(s, basis, args.samples, seed=5)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    ws = WarmStart(args.modes * args.modes, w.geom.n_gamma)
    t0 = time.perf_counter()
    losses = ws.fit(A, U, args.epochs)
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t0
    At = np.random.default_rng(99).standard_normal((args.test, args.modes * args.modes))
    precs = list(PRECONDITIONERS)
    rows = evaluate(s, ws, basis, At, precs=precs)
    print(json.dumps({
        "workload": args.workload, "n_gamma": w.geom.n_gamma, "samples": args.samples,
        "generate_s": t_gen, "train_s": t_fit, "epochs": args.epochs,
        "final_train_loss": losses[-1], "test_samples": args.test,
        **summarise(rows, precs),
    }))


if __name__ == "__main__":
    main()
