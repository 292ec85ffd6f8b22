"""Benchmark of the GB300 DDM-ELM solver (one JSON line on rank 0).

A step is one full solve of the method (Algorithm 1) on the 8x8-subdomain Poisson
workload: assembly of K^s/A^s from theta, blocked Householder QR of all 64 local
matrices, Schur-matrix assembly and Cholesky, right-hand side, triangular solves,
back-solves, and evaluation at 10,000 test points.  Inputs are synthetic and seeded
(workload.poisson_8x8_n1000).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores: every step (warm-up steps
included) is one complete oracle solve of the same workload.
With N > 1 (torchrun) every rank solves its own independent instance ("replicas only":
the method has no exchange between independent problems), no collective touches the
data path; value = all ranks' solves / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ELM-DDM solves/sec & ms/solve at stated rel-L2 vs FP64 oracle; % of roofline"
CG_TOL = 1e-9  # the paper's stopping rule for the Schur system
WORKLOAD = "poisson_8x8_n1000"
# FP64 FMA pipe of GB300: 152 SMs x 2 FP64 FMA/clk (4 flop/clk) x 2.07 GHz.
FP64_PEAK_GFLOPS = 152 * 4 * 2.07
# classes whose kernel runs as one CTA (their roofline is one SM's FP64 pipe)
SINGLE_CTA_CLASSES = ("potrf",)
KERNEL_OF_CLASS = {
    "panel_qr": "k_panel_qr_cl (Householder panel of 32 columns, 4-CTA cluster per subdomain, FP64 pipe)",
    "oz_qr_update_in": "k_ozaki_upd (persistent tensor-core FP64 product: the inner QR steps' updates of the rest of an outer block)",
    "potrf": "k_potrf_diag (64x64 diagonal Cholesky, one CTA, FP64 pipe)",
    "trsm_rows": "k_trsm_chol_rows (Cholesky panel solve by substitution in 4-column blocks, 16 rows per CTA, FP64 pipe)",
    "oz_qr_update": "k_ozaki_updw (wide persistent tensor-core FP64 product, 128 x 64 tiles: A2 -= V_o W2, one K = 128 update per outer QR block)",
    "oz_qr_w": "k_ozaki_fb<64> (tensor-core FP64 product, B split in the kernel, 64-column tiles: W1 = V_o^T [V_o | A2] per outer QR block)",
    "oz_qr_w_in": "k_ozaki_fa (tensor-core FP64 product, A split in the kernel: W1 of the inner panel steps)",
    "oz_syrk": "k_ozaki_upd (persistent tensor-core FP64 product: Schur Cholesky SYRK)",
    "split_qr_w": "k_rowexp + k_split (digit split of the outer block's V_o^T)",
    "assemble": "k_exp_tables + k_assemble (K^s, J and A^s from theta: factored activation)",
    "split_qr_update": "k_rowexp + k_split (digit split of V and W2^T)",
    "gemm_qr": "k_gemm (FP64 pipe: QR trailing updates)",
    "gemm_syrk": "k_gemm (FP64 pipe: Schur Cholesky SYRK)",
    "gemm_dm": "k_gemm (FP64 pipe: D_s, M_s)",
}


# DRAM traffic per algorithmic byte of the top kernels, from one ncu capture each on the
# 4x4 workload (poisson_4x4_n1000, 16 subdomains; the bench's 8x8 workload is too large
# to capture under the size rule), dram__bytes_read.sum + dram__bytes_write.sum over the
# launch's algorithmic bytes; traffic scales with the units a launch processes, so the
# bench's per-launch traffic is this ratio times its per-launch algorithmic bytes.
TRAFFIC_PER_ALGO_BYTE = {
    # class: (DRAM bytes of the captured launch, its algorithmic bytes, summary)
    # first QR panel: 9.859 MB read + 5.6 KB written (the panel's writes stay in L2) for
    # 16 x 2400 x 32 x 8 B read and written once
    "panel_qr": (9.864704e6, 19.6608e6, "profiles/k_panel_qr_cl_poisson_4x4_n1000.md"),
    # first outer-block trailing update A2 -= V_o W2 (K = 128, 128 x 64 tiles): C read +
    # written, V_o and W2 once
    "oz_qr_update": (769.099008e6, 778.600448e6, "profiles/k_ozaki_updw_poisson_4x4_n1000.md"),
    # first outer-block W1 = V_o^T [V_o | A2] (64-column tiles): V_o^T, [V_o | A2] and W1 once
    "oz_qr_w": (489.178368e6, 459.980800e6, "profiles/k_ozaki_fb_poisson_4x4_n1000.md"),
}

# Digit pairs a tensor-core FP64 product forms (the p + q <= 8 pairs of the 7 BF16 digit
# planes of each operand): the BF16 work per FP64-equivalent multiply-add.
DIGIT_PAIRS = 28


def measured_bf16_peak(sustained=True):
    """Dense BF16 tensor throughput measured on this machine, TFLOP/s (the sustained figure for
    kernels timed inside a long step), else the recipe fallback."""
    key = "bf16_tflops_sustained" if sustained else "bf16_tflops"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key]), f"MEASURED_PEAKS.json {key} (of measured)"
    except (OSError, KeyError, ValueError):
        return (1700.0 if sustained else 1900.0), "recipe fallback (of fallback)"


def measured_hbm_peak():
    """HBM copy bandwidth measured on this machine (MEASURED_PEAKS.json), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "recipe fallback 6.8 TB/s (of fallback)"


# --------------------------------------------------------------------------- helpers

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- CPU oracle

def oracle_local(w, s):
    """The oracle's local phase of Algorithm 1 for subdomain s (assembly, Householder
    QR, the Schur pieces of Eq. (3.5), q_s = Q_s^T F^s)."""
    from oracle import elm_oracle as O
    g = w.geom
    mi, mb, mg = (int(v) for v in g.counts[s])
    K, A = O.assemble_local(g.xy[s], g.nrm[s], g.counts[s], w.W[s], w.b[s])
    L = O.factor_local(K, A, g.dof[s, mi + mb:mi + mb + mg].astype(np.int64), mi + mb)
    return L, L.Q.T @ O.rhs_local(w.rhs[s], g.counts[s])


def oracle_global(w, locs, qs):
    """The oracle's global phase: Schur matrix and right-hand side, Cholesky solve,
    back-solves, evaluation at the test points."""
    from oracle import elm_oracle as O
    import scipy.linalg as sla
    g = w.geom
    S, M = O.schur_matrix(locs, g.n_gamma)
    r = O.schur_rhs(locs, qs, M, g.n_gamma)
    Lc = np.linalg.cholesky(S)
    u = sla.solve_triangular(Lc.T, sla.solve_triangular(Lc, r, lower=True), lower=False)
    c = np.stack([O.back_solve(L, q, u) for L, q in zip(locs, qs)])
    return O.evaluate(w.W, w.b, c, w.test_xy, w.test_owner)


def oracle_full_solve(w):
    """One complete oracle solve of the workload (Algorithm 1 and the evaluation at the
    test points).  Returns (seconds, u at the test points)."""
    t0 = time.perf_counter()
    pieces = [oracle_local(w, sd) for sd in range(w.geom.n_sub)]
    u, _ = oracle_global(w, [p[0] for p in pieces], [p[1] for p in pieces])
    return time.perf_counter() - t0, u


def cpu_cores():
    try:
        from threadpoolctl import threadpool_info
        n = max((i.get("num_threads", 0) for i in threadpool_info()), default=0)
        if n:
            return n
    except Exception:
        pass
    return os.cpu_count()


def workload_config(args, w, ws):
    """The `config` object of both arms' JSON lines for workload w."""
    n = w.n_neurons
    mg = int(w.geom.counts[:, 2].max())
    k_gb = w.geom.n_sub * int(w.geom.counts[0].sum()) * (n + mg) * 8 / 1e9
    return {"workload": args.workload, "subdomains": f"{w.geom.gx}x{w.geom.gy}",
            "neurons_per_subdomain": n, "rows_per_subdomain": int(w.geom.counts[0].sum()),
            "n_gamma": w.geom.n_gamma, "test_points": len(w.test_xy), "parallelism": f"replicas{ws}",
            "l2_flush": f"inputs larger than L2 (K alone is {k_gb:.1f} GB per step)",
            "schur_solver": ("cg (unpreconditioned, relative residual 1e-9, matrix-free S)"
                             if args.schur_solver == "cg" else "direct (envelope Cholesky)"),
            "precision": getattr(args, "precision", "fp64")}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2406_15959_gb300 import workload as wl
    w = wl.WORKLOADS[args.workload]()
    for _ in range(args.warmup):
        oracle_full_solve(w)
    times = [oracle_full_solve(w)[0] for _ in range(args.steps)]
    sec = statistics.mean(times)
    sample = (f"every step one complete oracle solve of the workload ({w.geom.n_sub} local "
              f"Householder QRs, Schur matrix n_Gamma={w.geom.n_gamma}, Cholesky, solves, "
              "back-solves, evaluation at the test points); no extrapolation")
    line = {"impl": "reference", "metric": METRIC, "value": 1.0 / sec, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sec, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, w, ws),
            "cpu_baseline": {"value": 1.0 / sec, "unit": "solves/s", "cores": cpu_cores(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": 1.0 / sec, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU arm

def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_2406_15959_gb300 import elm_ddm as E
    from paper_2406_15959_gb300 import workload as wl

    w = wl.WORKLOADS[args.workload]()
    stream = torch.cuda.current_stream(dev)
    cg = args.schur_solver == "cg"
    mixed = args.precision == "mixed"
    s = E.Solver(w.geom, w.n_neurons, stream=stream, schur_cg=cg, mixed=mixed)
    host = {
        "W": torch.as_tensor(w.W).pin_memory(), "b": torch.as_tensor(w.b).pin_memory(),
        "rhs": torch.as_tensor(w.rhs).pin_memory(),
    }
    d = {k: v.to(dev) for k, v in host.items()}
    txy = torch.as_tensor(w.test_xy, device=dev)
    own = torch.as_tensor(w.test_owner, device=dev, dtype=torch.int32)
    N, n = w.geom.n_sub, w.n_neurons
    c_dev = torch.empty((1, N, n), dtype=torch.float64, device=dev)
    ug_dev = torch.empty((1, w.geom.n_gamma), dtype=torch.float64, device=dev)
    u_dev = torch.empty(len(w.test_xy), dtype=torch.float64, device=dev)
    g_dev = torch.empty((len(w.test_xy), 2), dtype=torch.float64, device=dev)
    out_c = torch.empty((N, n), dtype=torch.float64).pin_memory()
    out_u = torch.empty(len(w.test_xy), dtype=torch.float64).pin_memory()

    cg_steps = []

    def step(Wt, bt, rt):
        s.assemble(Wt, bt)
        s.schur()
        if cg:  # the paper's interface solve: CG to a relative residual of 1e-9
            _, _, it = s.solve_cg(rt.unsqueeze(0), tol=CG_TOL, maxit=100000, u_gamma=ug_dev, c=c_dev)
            cg_steps.append(it)
        else:
            s.solve(rt.unsqueeze(0), ug_dev, c_dev)
        s.eval(txy, own, c_dev[0], u_dev, g_dev)

    from paper_2406_15959_gb300 import replicas as R

    def barrier():
        R.barrier(ws)

    def max_over_ranks(x):
        return R.max_over_ranks(x, ws, device=dev)

    for _ in range(args.warmup):
        step(d["W"], d["b"], d["rhs"])
    s.check()

    # ---- one profiled step (not timed): per-class device times and the dominant class
    hbm_peak, hbm_src = measured_hbm_peak()
    s.profile(True)
    s.profile_report()
    step(d["W"], d["b"], d["rhs"])
    prof1 = s.profile_report()
    s.profile(False)
    classes = {k: v for k, v in prof1.items() if not k.startswith("_")}

    bf16_peak, bf16_src = measured_bf16_peak(sustained=True)

    def roof(k, v, ms):
        if k.startswith("oz_") and v["flops"] > 0:
            # tensor-core FP64 product: the 2MNK of the FP64 product times the digit pairs
            # formed is the BF16 work the tensor cores must do for it
            # (the low-precision local factorisation forms the 10 leading pairs)
            pairs = 10 if mixed and k not in ("oz_syrk", "oz_syrk_b", "oz_schur") else DIGIT_PAIRS
            ach = v["flops"] * pairs / (ms * 1e-3) / 1e12
            return {"bound": "tensor", "achieved": ach, "peak": bf16_peak, "unit": "TFLOP/s",
                    "frac": ach / bf16_peak, "digit_pairs": pairs,
                    "fp64_equiv_tflops": v["flops"] / (ms * 1e-3) / 1e12,
                    "hbm_frac": v["bytes"] / (ms * 1e-3) / 1e9 / hbm_peak}
        if k.startswith("oz_") or k.startswith("split") or k == "assemble":
            ach = v["bytes"] / (ms * 1e-3) / 1e9
            return {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                    "frac": ach / hbm_peak}
        if v["flops"] > 0:
            ach = v["flops"] / (ms * 1e-3) / 1e9
            peak = FP64_PEAK_GFLOPS / 152 if k in SINGLE_CTA_CLASSES else FP64_PEAK_GFLOPS
            return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "GFLOP/s",
                    "frac": ach / peak}
        return None

    roof_all = {k: r for k, v in classes.items() if v["ms"] > 0 for r in [roof(k, v, v["ms"])] if r}
    dom = max(roof_all, key=lambda k: classes[k]["ms"]) if roof_all else None

    # ---- device-resident timed region: CUDA events around the whole steps, and around
    # the dominant class's launches only (its live average launch time gives `achieved`)
    s.profile(True, only=dom)
    s.profile_report()
    clocks = ClockSampler(torch.cuda.current_device() if ws == 1 else local)
    clocks.start()
    time.sleep(0.3)
    l0 = s.kernels_launched
    barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(d["W"], d["b"], d["rhs"])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    launches = (s.kernels_launched - l0) // args.steps
    clk = clocks.stop()
    prof = s.profile_report()
    s.profile(False)
    s.check()
    ms = max_over_ranks(e0.elapsed_time(e1)) / args.steps

    # ---- end to end through the API with host buffers (pinned H2D / D2H every step)
    barrier()
    torch.cuda.synchronize(dev)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        Wt = host["W"].to(dev, non_blocking=True)
        bt = host["b"].to(dev, non_blocking=True)
        rt = host["rhs"].to(dev, non_blocking=True)
        step(Wt, bt, rt)
        out_c.copy_(c_dev[0], non_blocking=True)
        out_u.copy_(u_dev, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    ms_e2e = max_over_ranks(f0.elapsed_time(f1)) / args.steps
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = out_c.numel() * 8 + out_u.numel() * 8

    # ---- accuracy of this step's result
    u_gpu = out_u.numpy().copy()
    l2_exact = None
    if w.src.has_exact:
        ue = w.src.u(w.test_xy)
        l2_exact = float(np.linalg.norm(u_gpu - ue) / np.linalg.norm(ue))

    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel class (by device time), measured live in the
    # timed region; every class from the profiled step in roofline_by_class
    roofline = None
    if dom and dom in prof:
        v = prof[dom]
        roofline = roof(dom, v, v["ms"])
        per_launch_bytes = v["bytes"] / max(v["launches"], 1)
        cap = TRAFFIC_PER_ALGO_BYTE.get(dom)
        roofline.update({
            "traffic": (cap[0] / cap[1] * per_launch_bytes if cap and per_launch_bytes > 0 else None),
            "traffic_source": (f"ncu DRAM bytes of the 4x4 workload ({cap[2]}) scaled by this "
                               f"launch's algorithmic bytes" if cap else None),
            "kernel_class": dom,
            "kernel": KERNEL_OF_CLASS.get(dom, dom),
            "launches_per_step": v["launches"] // args.steps,
            "avg_launch_us": 1e3 * v["ms"] / max(v["launches"], 1),
            "per_launch": {"flops": v["flops"] / max(v["launches"], 1),
                           "bytes": v["bytes"] / max(v["launches"], 1)},
            "peak_source": (hbm_src if roofline["bound"] == "hbm" else bf16_src if roofline["bound"] == "tensor"
                            else "derived: 152 SM x 4 FP64 flop/clk x 2.07 GHz (recipe units/clock)")})
    step_ms_breakdown = {k: round(v["ms"], 3) for k, v in sorted(classes.items())}

    # ---- CPU oracle: parity of this result and the timed baseline
    cpu = None
    l2_oracle = None
    if not args.no_cpu_baseline:
        t_full, u_or = oracle_full_solve(w)
        l2_oracle = float(np.linalg.norm(u_gpu - u_or) / np.linalg.norm(u_or))
        cpu = {"value": 1.0 / t_full, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": "one full oracle solve of the same workload (Algorithm 1 + evaluation)",
               "seconds": t_full}

    line = {
        "metric": METRIC, "value": R.job_throughput(ms, ws), "unit": "solves/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if not mixed else "f32/bf16 factors + f64 refinement",
        "data": "synthetic",
        "config": workload_config(args, w, ws),
        "rel_l2_vs_oracle": l2_oracle, "rel_l2_vs_exact": l2_exact,
        "e2e": {"value": R.job_throughput(ms_e2e, ws), "unit": "solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clk,
        "roofline": roofline,
        "roofline_by_class": roof_all,
        "step_ms_by_kernel_class": step_ms_breakdown,
        "breakdown_note": ("step_ms_by_kernel_class and roofline_by_class come from one extra "
                           "profiled step (every launch bracketed by events), not the timed region"),
        "cpu_baseline": cpu,
    }
    if cg:
        line["cg_steps"] = max(cg_steps) if cg_steps else None
    if mixed:
        line["precision"] = "mixed"
        line["refinement"] = s.refinement
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--schur-solver", choices=["direct", "cg"], default="direct",
                    help="interface solve: direct Cholesky (default) or the paper's CG")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64",
                    help="fp64 (default) or the mixed-precision path (low-precision local factors, "
                         "FP64 Schur factorisation, FP64-residual refinement, FP64 fallback)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
