"""Static parts of bench.py (no GPU): the workload config both arms report, and the
DRAM-traffic ratios agreeing with the ncu summaries they cite under profiles/."""
import argparse
import os
import re

import bench
from paper_2406_15959_gb300 import workload as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_workload_config_describes_the_workload():
    a = argparse.Namespace(workload="poisson_2x2_n200", schur_solver="direct")
    w = wl.poisson_2x2_n200()
    c = bench.workload_config(a, w, 1)
    assert c["workload"] == "poisson_2x2_n200" and c["subdomains"] == "2x2"
    assert c["neurons_per_subdomain"] == w.n_neurons and c["n_gamma"] == w.geom.n_gamma
    assert c["test_points"] == len(w.test_xy) and c["parallelism"] == "replicas1"
    assert "direct" in c["schur_solver"]
    a.schur_solver = "cg"
    assert "cg" in bench.workload_config(a, w, 2)["schur_solver"]


def _dram_bytes(md):
    """dram__bytes_read.sum + dram__bytes_write.sum from a profile summary table."""
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    total = 0.0
    for name in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
        m = re.search(r"\| " + re.escape(name) + r" \| (\w+) \| ([0-9.]+) \|", md)
        assert m, name
        total += float(m.group(2)) * scale[m.group(1)]
    return total


def test_traffic_ratios_match_the_cited_profiles():
    for cls, (dram, algo, path) in bench.TRAFFIC_PER_ALGO_BYTE.items():
        md = open(os.path.join(ROOT, path)).read()
        measured = _dram_bytes(md)
        assert abs(dram - measured) <= 1e-6 * measured, (cls, dram, measured)
        assert 0.0 < dram / algo <= 1.2, (cls, dram / algo)  # no re-reads beyond the algorithmic bytes
