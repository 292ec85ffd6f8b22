"""Batched serving (paper_2406_15959_gb300/batch.py): independent instances stacked
into one decomposition.

CPU pins of the stacking itself: the oracle's solution of the stacked decomposition
equals the oracle's per-instance solutions (the Schur matrix of Eq. (3.5) is block
diagonal across instances, so the interface values and the fitted functions must agree
to rounding), every interface unknown of the batch keeps exactly two owning
subdomains, and the batch plan respects the neuron-count grouping and the interface cap.
"""
import numpy as np
import pytest

from oracle import elm_oracle as O
from paper_2406_15959_gb300 import batch as B
from paper_2406_15959_gb300 import workload as wl


def instances():
    return [
        wl.build(2, 2, 30, 7, 6, 8, 8, theta="paper", theta_seed=31, source="fourier",
                 source_seed=31, n_test_side=12),
        wl.build(3, 2, 30, 6, 6, 7, 6, theta="paper", theta_seed=32, source="sinsin", coef="sine",
                 coef_seed=32, n_test_side=12),
        wl.build(2, 2, 30, 6, 7, 9, 7, theta="paper", theta_seed=33, source="sin2pi_exp",
                 n_test_side=12),
    ]


def solve_oracle(geom, W, b, rhs, coef, txy, town):
    res = O.solve(geom, W, b, rhs, coef=coef)
    u, _ = O.evaluate(W, b, res.c, txy, town)
    return res, u


def test_stacked_oracle_equals_per_instance_oracle():
    ws = instances()
    bt = B.combine(ws)
    assert bt.coef_rows is not None  # one instance has a coefficient: the batch uses the flux form
    res, u = solve_oracle(bt.geom, bt.W, bt.b, bt.rhs, bt.coef_rows, bt.test_xy, bt.test_owner)
    for w, (ug_b, c_b, u_b) in zip(ws, B.split(bt, res.u_gamma, res.c, u)):
        r1, u1 = solve_oracle(w.geom, w.W, w.b, w.rhs, w.coef_rows, w.test_xy, w.test_owner)
        assert np.linalg.norm(ug_b - r1.u_gamma) <= 1e-10 * np.linalg.norm(r1.u_gamma)
        assert np.linalg.norm(u_b - u1) <= 1e-10 * np.linalg.norm(u1)


def test_stacked_interface_map_has_two_owners_per_unknown():
    bt = B.combine(instances())
    g = bt.geom
    owners = [set() for _ in range(g.n_gamma)]
    for s in range(g.n_sub):
        mi, mb, mg = (int(v) for v in g.counts[s])
        for d in g.dof[s, mi + mb:mi + mb + mg]:
            owners[int(d)].add(s)
        assert np.all(g.dof[s, :mi + mb] == -1)
    assert all(len(o) == 2 for o in owners)
    # the unknowns of instance i are owned by instance i's subdomains only
    for i in range(bt.n_instances):
        s0, s1 = bt.sub_off[i], bt.sub_off[i + 1]
        for d in range(bt.gamma_off[i], bt.gamma_off[i + 1]):
            assert all(s0 <= s < s1 for s in owners[d])


def test_plan_groups_by_neurons_and_caps_the_interface():
    ws = B.serving_instances(12, (20, 24, 30), seed=7)
    groups = B.plan(ws, max_gamma=700, max_pad=0.0)
    assert sorted(i for g in groups for i in g) == list(range(12))
    for g in groups:
        assert len({ws[i].n_neurons for i in g}) == 1
        ng = sum(ws[i].geom.n_gamma for i in g)
        assert ng <= 700 or len(g) == 1
    # with padding allowed, neuron counts within the factor share batches
    groups = B.plan(ws, max_gamma=10 ** 6, max_pad=0.25)
    for g in groups:
        ns = [ws[i].n_neurons for i in g]
        assert max(ns) <= 1.25 * min(ns)
    assert any(len({ws[i].n_neurons for i in g}) > 1 for g in groups)


def test_padded_neurons_leave_the_solution_unchanged():
    """The library's per-subdomain neuron counts (identity columns on extra pad rows,
    Section 3's K^s otherwise unchanged): the oracle's factorisation of the padded K^s
    gives the unpadded interface solution, the same weights for the real neurons and zero
    weights for the pad ones.  (The oracle takes the interface rows last, so the pad rows
    go before them here; a least-squares solution does not depend on the row order.)"""
    w = wl.build(2, 2, 14, 6, 6, 5, 5, theta="paper", theta_seed=3, source="sinsin", c=0.5, n_test_side=10)
    g = w.geom
    pad = 5
    ref = O.solve(g, w.W, w.b, w.rhs)
    locs, qs = [], []
    for s in range(g.n_sub):
        mi, mb, mg = (int(v) for v in g.counts[s])
        K, A = O.assemble_local(g.xy[s], g.nrm[s], g.counts[s], w.W[s], w.b[s])
        m, n = K.shape
        i0 = mi + mb
        Kp = np.zeros((m + pad, n + pad))
        Kp[:i0, :n] = K[:i0]
        Kp[i0:i0 + pad, n:] = np.eye(pad)     # pad rows (no collocation point)
        Kp[i0 + pad:, :n] = K[i0:]            # interface rows last
        Ap = np.zeros((A.shape[0], n + pad))
        Ap[:, :n] = A
        L = O.factor_local(Kp, Ap, g.dof[s, mi + mb:mi + mb + mg].astype(np.int64), i0 + pad)
        F = np.zeros(m + pad)
        F[:i0] = O.rhs_local(w.rhs[s], g.counts[s])[:i0]
        locs.append(L)
        qs.append(L.Q.T @ F)
    S, M = O.schur_matrix(locs, g.n_gamma)
    r = O.schur_rhs(locs, qs, M, g.n_gamma)
    u = np.linalg.solve(S, r)
    c = np.stack([O.back_solve(L, q, u) for L, q in zip(locs, qs)])
    assert np.linalg.norm(u - ref.u_gamma) <= 1e-10 * np.linalg.norm(ref.u_gamma)
    np.testing.assert_allclose(c[:, :w.n_neurons], ref.c, rtol=1e-8, atol=1e-8 * np.abs(ref.c).max())
    assert np.abs(c[:, w.n_neurons:]).max() <= 1e-12 * np.abs(ref.c).max()


def test_combine_pads_smaller_networks():
    ws = B.serving_instances(4, (20, 30), seed=11)
    bt = B.combine(ws)
    assert bt.n_neurons == max(w.n_neurons for w in ws)
    for i, w in enumerate(ws):
        s0, s1 = bt.sub_off[i], bt.sub_off[i + 1]
        assert np.all(bt.neurons[s0:s1] == w.n_neurons)
        assert np.array_equal(bt.W[s0:s1, :w.n_neurons], w.W)
        assert not bt.W[s0:s1, w.n_neurons:].any() and not bt.b[s0:s1, w.n_neurons:].any()


def test_autotuner_shape_classes_and_candidates():
    from paper_2406_15959_gb300 import autotune as AT
    assert AT.shape_key(64, 1000, 2400, 400) == "N64_n1024_m4096_g512"
    assert AT.shape_key(16, 1000, 2400, 400) != AT.shape_key(64, 1000, 2400, 400)
    assert AT.shape_key(60, 990, 2300, 390) == AT.shape_key(64, 1000, 2400, 400)
    c = AT.candidates(152)
    assert (0, 0) in c and all(p in (0, 4, 8) and g >= 0 for p, g in c)


def test_combine_rejects_cross_point_geometries():
    """Batching stacks one A-row per interface row; geometries with explicit flux rows (the
    corner rule) are refused instead of losing their corner rows."""
    w = wl.paper_grid_workload(2, n_total=4 * 30, theta="local_unit", n_grid=17, n_test_side=10,
                               cross_points=True)
    with pytest.raises(ValueError):
        B.combine([w])
