"""Batched serving on the GPU: the stacked instances solved in one launch sequence agree
with the oracle's per-instance solutions (relative L2 <= 1e-8 at each instance's test
points, the parity bound of the single-instance path)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import elm_oracle as O
from paper_2406_15959_gb300 import batch as B

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from tests.test_batch import instances  # noqa: E402


def test_batched_solve_matches_per_instance_oracle():
    ws = instances()
    bt = B.combine(ws)
    bs = B.BatchSolver(bt)
    ug, c, u = bs.run()
    bs.solver.check()
    ug, c, u = ug.cpu().numpy(), c.cpu().numpy(), u.cpu().numpy()
    for w, (ug_b, _, u_b) in zip(ws, B.split(bt, ug, c, u)):
        res = O.solve(w.geom, w.W, w.b, w.rhs, coef=w.coef_rows)
        u1, _ = O.evaluate(w.W, w.b, res.c, w.test_xy, w.test_owner)
        assert np.linalg.norm(u_b - u1) <= 1e-8 * np.linalg.norm(u1)
        assert np.linalg.norm(ug_b - res.u_gamma) <= 1e-8 * np.linalg.norm(res.u_gamma)


def test_serving_plan_runs_every_batch():
    ws = B.serving_instances(6, (40,), seed=3)
    groups = B.plan(ws, max_gamma=1200)
    for g in groups:
        bt = B.combine([ws[i] for i in g])
        bs = B.BatchSolver(bt)
        _, _, u = bs.run()
        bs.solver.check()
        assert torch.isfinite(u).all()


def test_graph_replay_equals_eager_and_oracle():
    """Serving captures a batch's whole solve (assembly, factorisation, Schur solve,
    back-solves, evaluation) as one CUDA graph and replays it: the replay must give the
    eager run's bits, and both must match the per-instance oracle."""
    ws = instances()
    bt = B.combine(ws)
    eager = B.BatchSolver(bt)
    out = eager.run()
    eager.solver.check()                  # synchronises the batch's stream
    ug_e, c_e, u_e = (x.clone() for x in out)
    torch.cuda.synchronize()
    bs = B.BatchSolver(bt)
    bs.capture()
    for _ in range(2):
        ug_g, c_g, u_g = bs.replay()
        torch.cuda.synchronize()
        bs.solver.check()
        assert torch.equal(ug_g, ug_e) and torch.equal(c_g, c_e) and torch.equal(u_g, u_e)
    ug, c, u = ug_g.cpu().numpy(), c_g.cpu().numpy(), u_g.cpu().numpy()
    for w, (ug_b, _, u_b) in zip(ws, B.split(bt, ug, c, u)):
        res = O.solve(w.geom, w.W, w.b, w.rhs, coef=w.coef_rows)
        u1, _ = O.evaluate(w.W, w.b, res.c, w.test_xy, w.test_owner)
        assert np.linalg.norm(u_b - u1) <= 1e-8 * np.linalg.norm(u1)


def test_uneven_neuron_counts_in_one_launch_sequence():
    """Instances with different networks (20 .. 30 neurons per subdomain, variable
    coefficient, mixed grids) in one batch: the per-subdomain neuron counts pad the smaller
    networks, and every instance still matches its own oracle solution."""
    ws = B.serving_instances(5, (20, 24, 30), seed=12)
    assert len({w.n_neurons for w in ws}) > 1
    bt = B.combine(ws)
    bs = B.BatchSolver(bt)
    ug, c, u = bs.run()
    bs.solver.check()
    ug, c, u = ug.cpu().numpy(), c.cpu().numpy(), u.cpu().numpy()
    for w, (ug_b, c_b, u_b) in zip(ws, B.split(bt, ug, c, u)):
        res = O.solve(w.geom, w.W, w.b, w.rhs, coef=w.coef_rows)
        u1, _ = O.evaluate(w.W, w.b, res.c, w.test_xy, w.test_owner)
        assert np.linalg.norm(u_b - u1) <= 1e-8 * np.linalg.norm(u1)
        assert np.linalg.norm(ug_b - res.u_gamma) <= 1e-8 * np.linalg.norm(res.u_gamma)
        assert c_b.shape[1] == w.n_neurons
    # the pad neurons' weights are zero
    for i, w in enumerate(ws):
        s0, s1 = bt.sub_off[i], bt.sub_off[i + 1]
        assert np.abs(c[s0:s1, w.n_neurons:]).max(initial=0.0) <= 1e-12 * max(np.abs(c[s0:s1]).max(), 1.0)


def test_serving_waves_with_autotuner_match_the_oracle(tmp_path):
    """The serving driver on a scaled-down mix (neurons 24 .. 40 per subdomain, grids
    2x2 / 4x4 / 8x8, variable coefficient): batches padded within 25%, two memory-bounded
    waves each captured as one CUDA graph, tile choices from the autotuner (cached in a
    file); every instance's u at its test points matches its own oracle solution."""
    from paper_2406_15959_gb300 import autotune as AT
    ws = B.serving_instances(10, range(24, 41), seed=21)
    tuner = AT.Autotuner(str(tmp_path / "tuning.json"))
    groups = B.plan(ws, max_gamma=4096, max_pad=0.25)
    assert len(groups) >= 2
    budget = 1.01 * max(B._workspace_estimate([ws[i] for i in g]) for g in groups) / 1e9  # one batch a wave
    rep, res = B.serve_in_waves(ws, max_gamma=4096, max_pad=0.25, budget_gb=budget, steps=2, warmup=1,
                                tuner=tuner)
    assert len(rep["waves"]) >= 2 and rep["instances_per_s"] > 0
    assert (tmp_path / "tuning.json").exists() and rep["tuning"]["choices"]
    for w, u in zip(ws, res):
        r = O.solve(w.geom, w.W, w.b, w.rhs, keep=False, coef=w.coef_rows)
        u1, _ = O.evaluate(w.W, w.b, r.c, w.test_xy, w.test_owner)
        assert np.linalg.norm(u - u1) <= 1e-8 * np.linalg.norm(u1)
    # a second tuner on the same cache reuses the choices without timing
    t2 = AT.Autotuner(str(tmp_path / "tuning.json"))
    assert t2.table == tuner.table
