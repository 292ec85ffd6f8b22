"""Tile autotuner of the factorisation for batched serving.

The library exposes two tile choices through elm_ddm_set_tuning: the number of CTAs per
subdomain of the FP64 Householder panel (a 4- or 8-CTA cluster: 8 puts twice the SMs on a
small batch's panels, 4 runs more subdomains at once) and the grid cap of the persistent
tensor-core products.  Which is faster depends on the batch's shape (subdomain count,
neurons, rows), so for each shape class the tuner times the factorisation (assemble +
schur, the part these choices affect) under every candidate on the batch itself, keeps
the fastest, and caches the choice in a JSON file keyed by the class.  Host-side timing
logic only: every measured launch is the library's.
"""
from __future__ import annotations

import json
import os

from . import elm_ddm as E


def candidates(sms: int):
    """(panel CTAs, persistent grid cap) pairs tried per shape class."""
    return [(0, 0), (8, 0), (0, max(1, sms - 8)), (8, max(1, sms - 8))]


def shape_key(n_sub: int, n_neurons: int, rows: int, iface_rows: int) -> str:
    """Shape class: subdomains and rows rounded up to powers of two, neurons to 64."""
    p2 = lambda v: 1 << max(0, int(v - 1).bit_length())
    return f"N{p2(n_sub)}_n{-(-n_neurons // 64) * 64}_m{p2(rows)}_g{p2(max(iface_rows, 1))}"


class Autotuner:
    def __init__(self, cache_path: str | None = None, repeats: int = 2):
        self.path = cache_path
        self.repeats = repeats
        self.table = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.table = json.load(f)
        self.measured = {}  # key -> {candidate: ms} for the classes tuned in this process

    def _save(self):
        if self.path:
            os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
            with open(self.path, "w") as f:
                json.dump(self.table, f, indent=1, sort_keys=True)

    def key_of(self, solver: E.Solver) -> str:
        counts = solver._keep.counts
        return shape_key(solver.N, solver.n, int(counts.sum(1).max()), int(counts[:, 2].max()))

    def tune(self, solver: E.Solver, W, b, stream) -> tuple:
        """Choose and set the tile choices for this solver's shape class (timing its own
        assemble + schur under each candidate when the class is not cached yet)."""
        import torch
        key = self.key_of(solver)
        if key not in self.table:
            sms = torch.cuda.get_device_properties(stream.device).multi_processor_count
            times = {}
            for cand in candidates(sms):
                solver.set_tuning(*cand)
                with torch.cuda.stream(stream):
                    solver.assemble(W, b)
                    solver.schur()          # warm-up of this candidate
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    for _ in range(self.repeats):
                        solver.assemble(W, b)
                        solver.schur()
                    e1.record(stream)
                solver.check()
                times[cand] = e0.elapsed_time(e1) / self.repeats
            best = min(times, key=times.get)
            self.table[key] = list(best)
            self.measured[key] = {f"{c[0]},{c[1]}": round(t, 3) for c, t in times.items()}
            self._save()
        choice = tuple(self.table[key])
        solver.set_tuning(*choice)
        return choice
