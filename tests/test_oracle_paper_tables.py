"""The oracle at the paper's own Poisson experiments, against the errors the paper prints.

Section 4.2.1, Table 2 (relative L2 / H1 errors for u = sin(2 pi x) e^y with n = 65,536
neurons on the global 257 x 257 grid) and Section 4.1, Table 1 (RMSE of u_Gamma for three
weight ranges) are stored with their citations under tests/golden/.  The paper's seeds
are not published, so a printed error is a bound that the method reaches at that setup,
not a digit-for-digit target: a dropped term, a wrong sign or index anywhere in the
oracle's assembly, elimination, back-solve, evaluation or error metric leaves errors
orders of magnitude above it (the exact local least squares, for one, stays at ~1e-3).
The setup is the paper's grid with its cross points under the corner rule and the
Tikhonov-regularised local solves (alpha = 1e-14; the paper does not name its local
solver).  Each oracle solve takes about half a minute on a few cores.
"""
from __future__ import annotations

from pathlib import Path

import numpy as np
import pytest

from oracle import elm_oracle as O
from paper_2406_15959_gb300 import workload as wl

GOLDEN = Path(__file__).parent / "golden"
RIDGE = 1e-14
SEED = 7


def read_table(name: str) -> dict:
    """Rows of a golden table: first column (an int or a name) -> the remaining floats."""
    out = {}
    for line in (GOLDEN / name).read_text().splitlines():
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        out[int(key) if key.isdigit() else key] = [float(v) for v in vals]
    return out


TABLE2 = read_table("table2_poisson_sin2pix_ey.txt")
TABLE1 = read_table("table1_init_rmse_u_gamma.txt")


def oracle_run(G: int, theta: str = "paper"):
    """One oracle solve of the paper's setup on G x G subdomains: (rel L2, rel H1, RMSE of
    u_Gamma) against the exact solution, with the metric of Table 2 (100 x 100 test
    points) and Table 1 (the interface unknowns)."""
    w = wl.paper_grid_workload(G, theta=theta, seed=SEED, cross_points=True)
    res = O.solve(w.geom, w.W, w.b, w.rhs, keep=False, ridge=RIDGE)
    u, g = O.evaluate(w.W, w.b, res.c, w.test_xy, w.test_owner)
    l2, h1 = O.rel_errors(u, g, w.src.u(w.test_xy), w.src.grad_u(w.test_xy))
    geo = w.geom
    uex = np.zeros(geo.n_gamma)
    for s in range(geo.n_sub):
        _, _, rg = geo.rows(s)
        uex[geo.dof[s, rg]] = w.src.u(geo.xy[s, rg])
    rmse = float(np.sqrt(np.mean((res.u_gamma - uex) ** 2)))
    return l2, h1, rmse


@pytest.fixture(scope="module")
def run_8x8():
    return oracle_run(8)


def test_golden_tables_are_the_ones_the_reproduction_prints():
    """The paper's values that `paper_2406_15959_gb300.tables` prints beside its GPU runs
    are the stored ones."""
    from paper_2406_15959_gb300 import tables as T
    for G, row in T.PAPER_TABLE2.items():
        assert list(row) == TABLE2[G]
    cols = {2: 0, 4: 1, 8: 2}
    for G, (sug, man, he) in T.PAPER_TABLE1.items():
        assert (sug, man, he) == (TABLE1["suggested"][cols[G]], TABLE1["manual"][cols[G]],
                                  TABLE1["he"][cols[G]])


def test_oracle_reaches_table2_accuracy_8x8(run_8x8):
    """8 x 8 subdomains, 1024 neurons and 1089 rows each: at or below the paper's 2.6e-8
    (L2) and 8.2e-8 (H1)."""
    l2, h1, _ = run_8x8
    assert l2 <= TABLE2[8][0] and h1 <= TABLE2[8][1], (l2, h1)


def test_oracle_reaches_table2_accuracy_16x16():
    """16 x 16 subdomains, 256 neurons and 289 rows each: at or below the paper's 1.0e-7
    (L2) and 1.5e-7 (H1)."""
    l2, h1, _ = oracle_run(16)
    assert l2 <= TABLE2[16][0] and h1 <= TABLE2[16][1], (l2, h1)


def test_oracle_table1_initialisations_8x8(run_8x8):
    """Table 1 at 8 x 8: the paper's initialisation reaches its printed RMSE of u_Gamma,
    and He's (small weights, zero biases: near-identical basis functions) is worse by
    orders of magnitude, the paper's finding."""
    _, _, rmse_suggested = run_8x8
    assert rmse_suggested <= TABLE1["suggested"][2], rmse_suggested
    _, _, rmse_he = oracle_run(8, theta="he")
    assert rmse_he > 100 * rmse_suggested and rmse_he > TABLE1["suggested"][2], (rmse_he, rmse_suggested)
