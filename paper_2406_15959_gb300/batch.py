"""Batched serving of independent problem instances as one decomposition.

Instances are solved together by stacking their subdomains into one batch and numbering
their interface unknowns one instance after another.  No interface unknown couples two instances, so the Schur
matrix of Eq. (3.5) is block diagonal (one block per instance) and the library's
reverse Cuthill-McKee envelope keeps every Cholesky step inside its instance's block:
the batch costs what its instances cost together, but every launch of assemble / schur /
solve / eval covers all instances at once (one launch sequence instead of one per
instance).  Instances may mix subdomain grids; the operator is the variable-coefficient
one whenever any instance has a coefficient (the others get rho = 1, grad rho = 0).

Instances with different neuron counts share a batch through the library's per-subdomain
neuron counts (ELM_DDM_FLAG_NEURONS_PER_SUB: a smaller network's missing columns are
identity columns on pad rows, which leave its least-squares solution unchanged and
cost their share of the batch's work), so `plan` groups instances whose neuron counts are
within `max_pad` of each other (the padded work stays below that fraction); a batch whose
interface would outgrow `max_gamma` unknowns is split too: the library stores the Schur
matrix densely (n_Gamma^2 doubles, though only each block's envelope is computed).  This
module is host-side marshalling only: every step of the solve runs in the library's
kernels through elm_ddm.Solver.
"""
from __future__ import annotations

import dataclasses
import json
import time

import numpy as np

from . import elm_ddm as E
from . import workload as wl


@dataclasses.dataclass
class BatchGeometry:
    """The stacked decomposition (the attributes elm_ddm.Solver reads; the same layout as
    workload.Geometry)."""
    counts: np.ndarray    # int32 [N, 3]
    xy: np.ndarray        # float64 [N, m_max, 2]
    nrm: np.ndarray       # float64 [N, m_max, 2]
    dof: np.ndarray       # int32 [N, m_max], interface unknown of the batch or -1
    n_gamma: int

    @property
    def n_sub(self) -> int:
        return int(self.counts.shape[0])

    @property
    def m_max(self) -> int:
        return int(self.xy.shape[1])


@dataclasses.dataclass
class Batch:
    geom: BatchGeometry
    n_neurons: int                # the largest neuron count of the batch
    W: np.ndarray                 # [N, n, 2]
    b: np.ndarray                 # [N, n]
    rhs: np.ndarray               # [N, m_max]
    coef_rows: np.ndarray | None  # [N, m_max, 3] or None
    test_xy: np.ndarray           # [T, 2]
    test_owner: np.ndarray        # [T], subdomain of the batch
    sub_off: np.ndarray           # [I + 1]: subdomains of instance i are sub_off[i]:sub_off[i+1]
    gamma_off: np.ndarray         # [I + 1]: its interface unknowns
    test_off: np.ndarray          # [I + 1]: its test points
    neurons: np.ndarray = None    # [N] neurons of every subdomain (<= n_neurons)

    @property
    def n_instances(self) -> int:
        return len(self.sub_off) - 1


def combine(workloads) -> Batch:
    """Stack workload.Workload instances into one Batch (neuron counts may differ: the
    smaller networks are padded to the largest with zero parameters, which the library's
    per-subdomain neuron counts turn into identity columns)."""
    ws = list(workloads)
    if not ws:
        raise ValueError("no instances")
    if any(getattr(w.geom, "flux", None) is not None for w in ws):
        raise ValueError("instances with explicit flux rows (cross points) are not batched")
    n = max(w.n_neurons for w in ws)
    m_max = max(w.geom.m_max for w in ws)
    N = sum(w.geom.n_sub for w in ws)
    counts = np.zeros((N, 3), np.int32)
    neurons = np.zeros(N, np.int32)
    xy = np.zeros((N, m_max, 2))
    nrm = np.zeros((N, m_max, 2))
    dof = np.full((N, m_max), -1, np.int32)
    rhs = np.zeros((N, m_max))
    W = np.zeros((N, n, 2))
    b = np.zeros((N, n))
    any_coef = any(w.coef_rows is not None for w in ws)
    coef = np.zeros((N, m_max, 3)) if any_coef else None
    sub_off, gamma_off, test_off = [0], [0], [0]
    txy, town = [], []
    for w in ws:
        g = w.geom
        s0, s1 = sub_off[-1], sub_off[-1] + g.n_sub
        mm = g.m_max
        counts[s0:s1] = g.counts
        neurons[s0:s1] = w.n_neurons
        xy[s0:s1, :mm] = g.xy
        nrm[s0:s1, :mm] = g.nrm
        d = np.asarray(g.dof, np.int64)
        dof[s0:s1, :mm] = np.where(d >= 0, d + gamma_off[-1], -1)
        rhs[s0:s1, :mm] = w.rhs
        W[s0:s1, :w.n_neurons] = w.W
        b[s0:s1, :w.n_neurons] = w.b
        if any_coef:
            if w.coef_rows is not None:
                coef[s0:s1, :mm] = w.coef_rows
            else:
                coef[s0:s1, :, 0] = 1.0
        txy.append(w.test_xy)
        town.append(np.asarray(w.test_owner, np.int64) + s0)
        sub_off.append(s1)
        gamma_off.append(gamma_off[-1] + g.n_gamma)
        test_off.append(test_off[-1] + len(w.test_xy))
    geom = BatchGeometry(counts, xy, nrm, dof, int(gamma_off[-1]))
    return Batch(geom, n, W, b, rhs, coef, np.concatenate(txy), np.concatenate(town).astype(np.int32),
                 np.array(sub_off), np.array(gamma_off), np.array(test_off), neurons)


def plan(workloads, max_gamma: int = 32768, max_pad: float = 0.25):
    """Indices of the instances, grouped into batches: neuron counts within a factor
    1 + max_pad of the batch's smallest (so padding adds at most that fraction of columns),
    and at most max_gamma interface unknowns per batch (an instance larger than that
    alone).  max_pad = 0 groups equal neuron counts only."""
    order = sorted(range(len(workloads)), key=lambda i: (workloads[i].n_neurons, i))
    batches, cur, ng, n0 = [], [], 0, None
    for i in order:
        w = workloads[i]
        g = w.geom.n_gamma
        if cur and (ng + g > max_gamma or w.n_neurons > (1.0 + max_pad) * n0):
            batches.append(cur)
            cur, ng = [], 0
        if not cur:
            n0 = w.n_neurons
        cur.append(i)
        ng += g
    if cur:
        batches.append(cur)
    return batches


def split(batch: Batch, u_gamma=None, c=None, u=None):
    """Per-instance pieces of batch results: lists of (u_gamma, c, u at its test points)."""
    out = []
    for i in range(batch.n_instances):
        s0, s1 = batch.sub_off[i], batch.sub_off[i + 1]
        g0, g1 = batch.gamma_off[i], batch.gamma_off[i + 1]
        t0, t1 = batch.test_off[i], batch.test_off[i + 1]
        nn = batch.n_neurons if batch.neurons is None else int(batch.neurons[s0])
        out.append((None if u_gamma is None else u_gamma[g0:g1],
                    None if c is None else c[s0:s1, :nn],
                    None if u is None else u[t0:t1]))
    return out


class BatchSolver:
    """One elm_ddm.Solver over a Batch: assemble + schur + solve + eval for all instances,
    on its own CUDA stream (a new one unless given), so that several batches submitted one
    after another run concurrently on the GPU."""

    def __init__(self, batch: Batch, stream=None, tuner=None):
        """tuner: an autotune.Autotuner that picks (and caches) the tile choices for this
        batch's shape class."""
        import torch
        self.batch = batch
        self.stream = stream if stream is not None else torch.cuda.Stream()
        op = E.OP_VARCOEF if batch.coef_rows is not None else E.OP_POISSON
        uneven = batch.neurons is not None and int(batch.neurons.min()) < batch.n_neurons
        self.solver = E.Solver(E.GeometryArrays.from_geometry(batch.geom), batch.n_neurons,
                               stream=self.stream, op=op, neurons=batch.neurons if uneven else None)
        dev = torch.device("cuda")
        t = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), device=dev, dtype=dt)
        # inputs resident on the device from here on
        self.W, self.b, self.rhs = t(batch.W), t(batch.b), t(batch.rhs)
        self.coef = t(batch.coef_rows) if batch.coef_rows is not None else None
        self.test_xy, self.test_owner = t(batch.test_xy), t(batch.test_owner, torch.int32)
        self.tuning = None
        if tuner is not None:
            if self.coef is not None:
                self.solver.set_coefficient(self.coef)
            self.tuning = tuner.tune(self.solver, self.W, self.b, self.stream)

    def run(self):
        """One full solve of every instance, enqueued on this batch's stream; returns
        device (u_gamma, c, u at test points), valid once that stream has run."""
        import torch
        s = self.solver
        with torch.cuda.stream(self.stream):  # outputs are allocated for this stream
            if self.coef is not None:
                s.set_coefficient(self.coef)
            s.assemble(self.W, self.b)
            s.schur()
            ug, c = s.solve(self.rhs)
            u, _ = s.eval(self.test_xy, self.test_owner, c)
        return ug, c, u

    def capture(self):
        """Record run() once as a CUDA graph (every entry point is stream-ordered, with no
        allocation and no host synchronisation after setup); replay() then submits the
        whole solve as one graph launch.  Returns the graph's output tensors."""
        import torch
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            self.graph_out = self.run()
        return self.graph_out

    def replay(self):
        import torch
        with torch.cuda.stream(self.stream):
            self.graph.replay()
        return self.graph_out


def serving_instances(count: int, neurons=(200,), seed: int = 0):
    """Seeded instances of the serving workload: -div(a grad u) = f with
    a = 1 + 0.5 sin(2 pi k . x), k in {1..4}^2, sine-mode f, subdomain grids drawn from
    {2x2, 4x4, 8x8}, neurons per subdomain drawn from `neurons`, 2 n_N interior points per
    subdomain and 64 points per edge."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        G = int(rng.choice([2, 4, 8]))
        n = int(rng.choice(list(neurons)))
        mi_x = int(np.ceil(np.sqrt(2 * n)))
        mi_y = int(np.ceil(2 * n / mi_x))
        s = int(rng.integers(0, 2 ** 31 - 1))
        out.append(wl.build(G, G, n, mi_x, mi_y, 64, 64, theta="paper", theta_seed=s,
                            source="fourier", source_seed=s, coef="sine", coef_seed=s,
                            n_test_side=20, name=f"instance{i}"))
    return out


def serve_in_waves(instances, max_gamma: int = 32768, max_pad: float = 0.25, budget_gb: float = 150.0,
                   steps: int = 3, warmup: int = 1, tuner=None, graphs: bool = True):
    """Full solves of every instance, batched by `plan` and run in waves whose handles fit
    `budget_gb` of device memory (all instances at once need more than the GPU holds at the
    serving configuration's sizes).  Each wave's batches share one stream; with `graphs`
    the whole wave is captured as one CUDA graph after `warmup` eager rounds and replayed
    `steps` times.  Returns per-wave timings (device time of the replays, CUDA events) and
    the per-instance results of the last replay as host arrays (u at the test points)."""
    import torch
    groups = plan(instances, max_gamma, max_pad)
    waves, cur, cur_bytes = [], [], 0
    results = [None] * len(instances)
    report = {"batches": len(groups), "waves": [], "tuning": {}}

    def run_wave(batches):
        st = torch.cuda.Stream()
        solvers = [BatchSolver(combine([instances[i] for i in g]), stream=st, tuner=tuner) for g in batches]
        for _ in range(warmup):
            for bs in solvers:
                bs.run()
        st.synchronize()
        graph = None
        if graphs:
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=st):
                outs = [bs.run() for bs in solvers]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            e0.record(st)
            for _ in range(steps):
                if graph is not None:
                    graph.replay()
                else:
                    outs = [bs.run() for bs in solvers]
            e1.record(st)
        st.synchronize()
        for bs in solvers:
            bs.solver.check()
        ms = e0.elapsed_time(e1) / steps
        n_inst = sum(len(g) for g in batches)
        for g, bs, (ug, c, u) in zip(batches, solvers, outs):
            for i, (_, _, u_i) in zip(g, split(bs.batch, None, None, u.cpu().numpy())):
                results[i] = u_i
        mem = sum(bs.solver.workspace_bytes for bs in solvers)
        report["waves"].append({"batches": len(batches), "instances": n_inst, "ms_per_round": ms,
                                "workspace_gb": mem / 1e9})
        del solvers, graph
        torch.cuda.synchronize()
        torch.cuda.empty_cache()

    for g in groups:
        need = _workspace_estimate([instances[i] for i in g])
        if cur and cur_bytes + need > budget_gb * 1e9:
            waves.append(cur)
            cur, cur_bytes = [], 0
        cur.append(g)
        cur_bytes += need
    if cur:
        waves.append(cur)
    for w in waves:
        run_wave(w)
    if tuner is not None:
        report["tuning"] = {"choices": tuner.table, "measured_ms": tuner.measured}
    report["ms_per_round"] = sum(wv["ms_per_round"] for wv in report["waves"])
    report["instances_per_s"] = len(instances) / (report["ms_per_round"] * 1e-3)
    return report, results


def _workspace_estimate(ws) -> int:
    """Device bytes a batch of these instances needs (dominant terms: [K | J], the Schur
    matrix, the split planes ~ 2.2 x K with 32-column QR operands, plus what the outer QR
    blocks of up to 128 columns add: the explicit reflectors, W1, W2 and their digit
    planes, nbo (36 ld + 44 (n + m_Gamma)) bytes per subdomain for nbo = 128 - 32)."""
    n = max(w.n_neurons for w in ws)
    rows = max(int(w.geom.counts.sum(1).max()) + n - w.n_neurons for w in ws)
    mg = max(int(w.geom.counts[:, 2].max()) for w in ws)
    subs = sum(w.geom.n_sub for w in ws)
    ng = sum(w.geom.n_gamma for w in ws)
    ld = -(-rows // 32) * 32
    nbo = max(0, min(128, -(-n // 32) * 32) - 32)
    return int(subs * (3.2 * ld * (n + mg) * 8 + nbo * (36 * ld + 44 * (n + mg))) + 8 * ng * ng)


def _main(argv=None):
    """Serving measurement.  Default: `--instances` seeded instances of 200 neurons per
    subdomain, all resident, every batch on its own stream (wall clock around synchronised
    rounds).  `--waves`: the serving configuration (neurons drawn from 200..1500), batched
    with padding, run in memory-bounded waves, each captured as one CUDA graph (device
    time of the replays), optionally with the tile autotuner."""
    import argparse
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--instances", type=int, default=64)
    ap.add_argument("--neurons", type=int, nargs="+", default=[200])
    ap.add_argument("--neuron-range", type=int, nargs=2, default=None,
                    help="draw neurons uniformly from this closed range instead of --neurons")
    ap.add_argument("--max-gamma", type=int, default=32768)
    ap.add_argument("--max-pad", type=float, default=0.25)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--graphs", action="store_true", help="replay CUDA graphs")
    ap.add_argument("--waves", action="store_true", help="memory-bounded waves, one CUDA graph each")
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--autotune", default=None, metavar="CACHE.json",
                    help="tile autotuner with its cache file")
    a = ap.parse_args(argv)
    t0 = time.perf_counter()
    neurons = range(a.neuron_range[0], a.neuron_range[1] + 1) if a.neuron_range else a.neurons
    inst = serving_instances(a.instances, neurons, a.seed)
    host_s = time.perf_counter() - t0
    if a.waves:
        tuner = None
        if a.autotune:
            from .autotune import Autotuner
            tuner = Autotuner(a.autotune)
        t1 = time.perf_counter()
        rep, res = serve_in_waves(inst, a.max_gamma, a.max_pad, a.budget_gb, a.steps, a.warmup, tuner, True)
        rep["wall_s_incl_setup_and_capture"] = time.perf_counter() - t1
        neur = [w.n_neurons for w in inst]
        print(json.dumps({"metric": "batched serving, memory-bounded waves, one CUDA graph per wave",
                          "instances": a.instances, "neurons_min_max": [min(neur), max(neur)],
                          "grids": sorted({f"{w.geom.gx}x{w.geom.gy}" for w in inst}),
                          "host_instance_generation_s": host_s, **rep}))
        return
    groups = plan(inst, a.max_gamma, a.max_pad)
    solvers = [BatchSolver(combine([inst[i] for i in g])) for g in groups]
    host_s = time.perf_counter() - t0
    for _ in range(a.warmup):
        for bs in solvers:
            bs.run()
    torch.cuda.synchronize()
    same = None
    if a.graphs:
        eager = [bs.run()[2].clone() for bs in solvers]
        torch.cuda.synchronize()
        for bs in solvers:
            bs.capture()
        for bs in solvers:
            bs.replay()
        torch.cuda.synchronize()
        same = all(torch.equal(e, bs.graph_out[2]) for e, bs in zip(eager, solvers))
    step = (lambda bs: bs.replay()) if a.graphs else (lambda bs: bs.run())
    t1 = time.perf_counter()
    for _ in range(a.steps):
        for bs in solvers:
            step(bs)
        torch.cuda.synchronize()
    ms = 1e3 * (time.perf_counter() - t1) / a.steps
    for bs in solvers:
        bs.solver.check()
    print(json.dumps({"metric": "batched serving (full solves, inputs resident, wall clock)",
                      "instances": a.instances, "neurons": list(a.neurons), "batches": len(solvers),
                      "subdomains": int(sum(bs.batch.geom.n_sub for bs in solvers)),
                      "n_gamma": int(sum(bs.batch.geom.n_gamma for bs in solvers)),
                      "ms_per_round": ms, "instances_per_s": a.instances / (ms * 1e-3),
                      "cuda_graphs": a.graphs, "graph_equals_eager": same,
                      "host_setup_s": host_s}))


if __name__ == "__main__":
    _main()
