"""Benchmark of the Laplace expected-information-gain hot path on GB300.

One step = one EIG evaluation of the batched workload (401x201 grid, h = 5 m,
2000 leap-frog steps, 256 Monte Carlo nodes x 15 central-FD solves = 3840
solves, 20 surface receivers): source setup, all time steps (FP32 stencil),
FP64 Jacobian / Hessian, FP64 scaled log-determinants and the quadrature sum.
Inputs are resident in HBM when the timed region starts; the 5.1 GB of
wavefields per step exceed the 129 MB L2, so no flush is needed.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "EIG evals/s & stencil Gcell-upd/s (% HBM roofline) at rel err<=1e-3; p50/p99"
BYTES_PER_CELL_UPDATE = {"f32": 24, "f64": 48}   # read u^m, u^{m-1}; write u^{m+1}; 2 comps
# FP32 operations of one interior node update as the kernels evaluate it (both
# components, stencil_cell.cuh, a multiply-add counted as 2): per component the
# second difference 2.5 (three neighbour differences shared by a column pair), the
# vertical and cross differences 1 + 1 (each shared with the next row), the operator
# term 1 multiply + 4 multiply-adds = 9, the leap-frog increment form 3
FLOPS_PER_CELL_UPDATE = 33
# FP32 lane operations behind those flops (the FP32 pipe's own roofline: 25 per node; a
# packed two-wide instruction counts as two, one per lane it occupies)
FP32_INSTR_PER_CELL_UPDATE = 25
# FP32 peak derived from the unit counts and clocks: 152 SMs x 128 FP32 lanes x 2 (FMA)
# x 2.07 GHz maximum SM clock
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def kernel_label(t):
    """Human-readable stencil kernel for a (cluster, rows, warps) tuning triple."""
    if t[0] > 0:
        return "cluster-resident, %d CTAs per solve" % t[0]
    if t[0] < 0:
        return "TMA streaming (persistent, 4-stage mbarrier ring)"
    return "streaming, %d rows/thread, %d warps/block" % (t[1], t[2])


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched",
                    choices=["batched", "plain_small", "layered", "design_sweep", "paper_scenarios",
                             "paper_study"])
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample-nodes", type=int, default=2)
    ap.add_argument("--nodes", type=int, default=0, help="override the node count (profiling runs)")
    ap.add_argument("--sigma", type=float, default=0.0, help="use this noise std instead of 1%% of peak")
    ap.add_argument("--tuning", default="auto",
                    help="stencil kernel: auto, or C,rows,warps (C>0 cluster-resident)")
    ap.add_argument("--jacobian", default="pairs", choices=["pairs", "difference"])
    ap.add_argument("--no-difference", action="store_true",
                    help="skip the extra measurement of the difference-form Jacobian")
    ap.add_argument("--study-levels", type=int, default=20,
                    help="paper_study: sparse grids 5 .. 5 + n - 1 (20: the paper's 351 .. 271857 nodes)")
    ap.add_argument("--study-realisations", type=int, default=10)
    ap.add_argument("--dlmc-sizes", type=lambda v: [int(x) for x in v.split(",")],
                    default=[256, 1024, 4096, 16384, 65536])
    ap.add_argument("--serving", action="store_true",
                    help="serving benchmark: Poisson arrivals of mixed EIG requests")
    ap.add_argument("--requests", type=int, default=32)
    ap.add_argument("--rate", type=float, default=8.0, help="mean arrivals per second")
    return ap.parse_args()


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of a rank's node batch: every rank evaluates its own independent batch."""
    return base_seed + 7919 * rank


def max_over_ranks(x: float, dist, device) -> float:
    """The slowest rank's value (all ranks get it); identity without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(world: int, steps: int, max_ms: float) -> float:
    """Whole-job EIG evaluations per second: all ranks' evaluations over the slowest time."""
    return world * steps / (max_ms * 1e-3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCES = {"k_resident": ("resident.cu", "stencil_cell.cuh", "oed_internal.cuh"),
                  "k_step": ("stencil.cu", "stencil_cell.cuh", "oed_internal.cuh"),
                  "k_step_tma": ("stream_tma.cu", "stencil_cell.cuh", "oed_internal.cuh")}


def _code_only(text: str) -> str:
    """C/C++ source without comments and with whitespace collapsed (string literals in
    these kernels hold no comment markers)."""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_sources_hash(kernel: str) -> str:
    """Hash of a stencil kernel's code (comments and layout ignored): a committed ncu
    traffic figure is used only while the code it was taken on is unchanged."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1502_07873_gb300", "csrc", f)) as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def ncu_entry(kernel: str):
    """The committed ncu figures of a stencil kernel, or None when the summary is missing
    or the kernel's code changed since they were taken."""
    p = os.path.join(ROOT, "profiles", "stencil_dram_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        e = json.load(f).get(kernel)
    if not e or e.get("sources_sha") != kernel_sources_hash(kernel):
        return None
    return e


def ncu_traffic(kernel: str):
    """DRAM bytes per cell-update of a stencil kernel from the committed ncu summary,
    or None when the summary is missing or the kernel's code changed since."""
    e = ncu_entry(kernel)
    return float(e["dram_bytes_per_cell_update"]) if e else None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[3 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def workload(name):
    return W.batched() if name == "batched" else W.plain_small()


def noise_sigma_gpu(P, torch, w, precision):
    """sigma = 1% of the peak |u| over all surface nodes at the prior-mean source
    (computed once per grid / medium / duration, outside the timed region)."""
    prob = P.problem_from_workload(w, precision, rec_ix=list(range(w.nx)))
    ctx = P.Context(prob, max_solves=15)
    mean = (np.array(w.prior_lo) + np.array(w.prior_hi)) / 2
    g = torch.empty((1, w.nlevels, w.nx, 2), dtype=torch.float64, device="cuda")
    P.oed_forward(ctx, torch.tensor(mean[None], device="cuda"), g)
    torch.cuda.synchronize()
    ctx.close()
    return w.sigma_frac * float(g.abs().max().item())


def cpu_baseline(w, sigma, nodes: int):
    """The FP64 oracle on a bounded sample: `nodes` nodes of the same workload, each
    node's 14 perturbed solves spread over the host cores."""
    from oracle import oracle as O
    O.build()
    G = O.Grid.from_workload(w)
    th, wt = O.mc_nodes(w.uniforms(), w.prior_lo, w.prior_hi)
    lp = O.log_uniform_density(w.prior_lo, w.prior_hi)
    t0 = time.perf_counter()
    for i in range(nodes):
        H, _ = O.node_hessian(G, th[i], w.prior_lo, w.prior_hi, w.rel_step, sigma)
        ld, _, ok = O.scaled_logdet(H)
        O.dkl(ld, 7, lp)
    dt = time.perf_counter() - t0
    threads = min(14, os.cpu_count() or 1)
    per_eval = dt / nodes * w.n_nodes
    return {"value": 1.0 / per_eval, "unit": "EIG evals/s", "cores": int(threads), "kind": "oracle",
            "sample": f"{nodes} of {w.n_nodes} nodes ({nodes * 14} FP64 solves of "
                      f"{w.nx}x{w.nz}x{w.nsteps} steps), {dt:.1f} s wall, scaled to one EIG "
                      f"evaluation"}, dt


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = workload(args.workload)
    from oracle import oracle as O
    O.build()
    sigma_w = W.batched().sigma_frac
    mean = (np.array(w.prior_lo) + np.array(w.prior_hi)) / 2
    Gs = O.Grid(w.nx, w.nz, w.h, w.dt, w.nsteps, w.layers, list(range(w.nx)))
    sigma = O.noise_sigma(Gs, mean, sigma_w)
    times = []
    nodes = max(1, min(args.cpu_sample_nodes, w.n_nodes))
    for k in range(args.warmup + args.steps):
        cb, dt = cpu_baseline(w, sigma, nodes)
        if k >= args.warmup:
            times.append(dt / nodes * w.n_nodes)
    per = statistics.mean(times)
    out = {"impl": "reference", "metric": METRIC, "value": 1.0 / per, "unit": "EIG evals/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": per * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": w.name, "grid": f"{w.nx}x{w.nz}", "time_steps": w.nsteps,
                      "nodes": w.n_nodes, "solves": 15 * w.n_nodes, "receivers": w.nrec},
           "cpu_baseline": {**cb, "value": 1.0 / per},
           "e2e": {"value": 1.0 / per, "unit": "EIG evals/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_ours(args, rank, world, local):
    import torch
    import paper_1502_07873_gb300 as P
    from paper_1502_07873_gb300 import build as B

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    w = workload(args.workload)
    if args.nodes:
        w.n_nodes = args.nodes
    prec = P.OED_FP32 if args.precision == "f32" else P.OED_FP64
    sigma = args.sigma if args.sigma > 0 else noise_sigma_gpu(P, torch, w, prec)
    dev = torch.device("cuda", local)
    nsolve = 15 * w.n_nodes
    ctx = P.Context(P.problem_from_workload(w, prec), max_solves=nsolve)
    # each rank evaluates its own independent batch of nodes (weak scaling)
    u = w.uniforms(seed=rank_seed(w.seed, rank))
    lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)
    theta = torch.tensor(lo + (hi - lo) * u, dtype=torch.float64, device=dev)
    wt = torch.full((w.n_nodes,), 1.0 / w.n_nodes, dtype=torch.float64, device=dev)
    H = torch.empty((w.n_nodes, 7, 7), dtype=torch.float64, device=dev)
    eig = torch.empty(1, dtype=torch.float64, device=dev)
    nbad = torch.empty(1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    if args.jacobian == "difference":
        ctx.jacobian = P.OED_JAC_DIFFERENCE
        nsolve = 7 * w.n_nodes
    if args.tuning == "auto":
        tuning = ctx.autotune(nsolve, stream=stream)   # launch shape of the stencil, set once
    else:
        ctx.set_tuning(*[int(x) for x in args.tuning.split(",")])
        tuning = ctx.tuning

    def step():
        P.oed_hessian(ctx, theta, w.prior_lo, w.prior_hi, w.rel_step, sigma, H, stream=stream)
        P.oed_eig(ctx, H, wt, w.prior_lo, w.prior_hi, eig, n_bad=nbad, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    step_ms, stencil_ms = [], []
    with ClockSampler(local) as clk:
        ev[0].record(stream)
        for k in range(args.steps):
            step()
            ev[k + 1].record(stream)
            ev[k + 1].synchronize()
            ms, launches = ctx.last_step_time()
            stencil_ms.append(ms / launches)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
    for k in range(args.steps):
        step_ms.append(ev[k].elapsed_time(ev[k + 1]))
    total_ms = max_over_ranks(ev[0].elapsed_time(ev[args.steps]), dist, dev)
    eig_val = float(eig.item())

    # end to end through the host-buffer entry point (pinned inputs, H2D + D2H inside)
    e2e = None
    if not args.no_e2e:
        th_h = theta.cpu().pin_memory()
        w_h = wt.cpu().pin_memory()
        P.oed_eig_host(ctx, th_h, w_h, w.prior_lo, w.prior_hi, w.rel_step, sigma)
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e_h, _, _ = P.oed_eig_host(ctx, th_h, w_h, w.prior_lo, w.prior_hi, w.rel_step, sigma)
        el = max_over_ranks(time.perf_counter() - t0, dist, dev)
        e2e = {"value": weak_scaling_value(world, args.steps, el * 1e3), "unit": "EIG evals/s",
               "h2d_bytes_per_step": int(th_h.numel() * 8 + w_h.numel() * 8),
               "d2h_bytes_per_step": 8 + 4}

    # the same evaluation with the difference-form Jacobian (7 solves per node)
    diff = None
    if args.jacobian == "pairs" and not args.no_difference:
        ctx.jacobian = P.OED_JAC_DIFFERENCE
        dtun = ctx.autotune(7 * w.n_nodes, stream=stream) if args.tuning == "auto" else ctx.tuning
        step()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        dms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
        eig_d = float(eig.item())
        diff = {"value": weak_scaling_value(world, args.steps, dms), "unit": "EIG evals/s",
                "ms_per_step": dms / args.steps, "solves_per_gpu": 7 * w.n_nodes, "eig": eig_d,
                "rel_diff_vs_pairs": abs(eig_d - eig_val) / abs(eig_val),
                "stencil_kernel": kernel_label(dtun)}
        ctx.jacobian = P.OED_JAC_PAIRS

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    cells = w.cells * w.nsteps * nsolve
    per_launch_cells = w.cells * nsolve
    bpc = BYTES_PER_CELL_UPDATE[args.precision]
    st_ms = statistics.median(stencil_ms)          # per time step of all solves
    peak, peak_kind = measured_peaks()
    hbm_equiv = per_launch_cells * bpc / (st_ms * 1e-3) / 1e9
    if tuning[0] > 0:
        # cluster-resident kernel: one launch integrates every step; the wavefield never
        # leaves the chip, so the bound is FP32 issue, not HBM
        launch_ms = st_ms * w.nsteps
        flops = FLOPS_PER_CELL_UPDATE * cells
        achieved = flops / (launch_ms * 1e-3) / 1e12
        tb = ncu_traffic("k_resident")
        roofline = {"bound": "alu", "kernel": "k_resident (cluster-resident leap-frog, all steps)",
                    "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                    "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                    "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                    "algorithmic_flops_per_cell_update": FLOPS_PER_CELL_UPDATE,
                    "fp32_pipe_frac": FP32_INSTR_PER_CELL_UPDATE * cells / (launch_ms * 1e-3)
                    / (FP32_PEAK_TFLOPS * 1e12 / 2),
                    "traffic": (tb * cells if tb is not None else None), "launch_ms": launch_ms,
                    "hbm_equivalent": {"gbs": hbm_equiv, "frac_of_measured_hbm": hbm_equiv / peak,
                                       "note": "24 B per cell-update a streaming kernel would move"}}
        onchip = ncu_entry("k_resident")
        if onchip and "l1tex_throughput_frac_active" in onchip:
            # the unit that binds the resident kernel: L1 / shared memory (ncu, committed)
            roofline["on_chip"] = {"l1tex_throughput_frac_active": onchip["l1tex_throughput_frac_active"],
                                   "shared_wavefronts_frac_elapsed": onchip["shared_wavefronts_frac_elapsed"],
                                   "source": "ncu --set full of the same code, 60 solves (profiles/)"}
        launches_per_step = 5
    else:
        kname = "k_step_tma" if tuning[0] < 0 else "k_step"
        tb = ncu_traffic(kname)
        roofline = {"bound": "hbm", "kernel": kname + " (streaming leap-frog, one step)",
                    "achieved": hbm_equiv, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                    "frac": hbm_equiv / peak, "algorithmic_bytes_per_cell_update": bpc,
                    "traffic": (tb * per_launch_cells if tb is not None else None),
                    "launch_ms": st_ms}
        launches_per_step = w.nsteps + 5
    value = weak_scaling_value(world, args.steps, total_ms)
    cb = None
    if not args.no_cpu_baseline and world == 1:
        cb, _ = cpu_baseline(w, sigma, max(1, args.cpu_sample_nodes))
    lat = sorted(step_ms)

    def pct(q):
        return lat[min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1)]

    out = {
        "metric": METRIC, "value": value, "unit": "EIG evals/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.precision, "data": "synthetic",
        "config": {"workload": w.name, "grid": f"{w.nx}x{w.nz}", "h_m": w.h, "time_steps": w.nsteps,
                   "nodes_per_gpu": w.n_nodes, "solves_per_gpu": nsolve, "receivers": w.nrec,
                   "precision": f"{args.precision} stencil; f64 jacobian, hessian, log-det, sum",
                   "jacobian": (f"{args.jacobian}: " + ("15 solves per node, FP64 subtraction of the "
                                "+/- seismograms" if args.jacobian == "pairs" else
                                "7 solves per node driven by FP64 forcing differences")),
                   "parallelism": f"replicas x{world} (independent node batches)",
                   "stencil_kernel": kernel_label(tuning),
                   "l2": "no flush: 5.1 GB of wavefields per step exceed the 129 MB L2"},
        "gcell_upd_per_s": world * cells * args.steps / (total_ms * 1e-3) / 1e9,
        "stencil_gcell_upd_per_s": per_launch_cells / (st_ms * 1e-3) / 1e9,
        "latency_ms": {"p50": pct(0.5), "p99": pct(0.99)},
        "eig": eig_val,
        "sigma": sigma,
        "roofline": roofline,
        "clocks": clk.summary(),
        "gpu_launches": args.steps * launches_per_step,
        "e2e": e2e,
        "jacobian_difference_form": diff,
    }
    if cb:
        out["cpu_baseline"] = cb
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def run_other_workload(args, rank, world, local):
    """One EIG evaluation of the layered Smolyak workload (801x401, 3 layers, 4000 steps,
    589 nodes) or one design sweep (401x201, 2400 steps, 1024 nodes, 40 candidates,
    3 windows x 5120 designs), FP32 stencil with the difference-form Jacobian."""
    import torch
    import paper_1502_07873_gb300 as P
    from paper_1502_07873_gb300 import build as B
    torch.cuda.set_device(local)
    B.build()
    dev = torch.device("cuda", local)
    w = W.layered() if args.workload == "layered" else W.design_sweep()
    sigma = args.sigma if args.sigma > 0 else noise_sigma_gpu(P, torch, w, P.OED_FP32)
    if args.workload == "layered":
        x, wt = P.oed_nodes_smolyak(7, w.smolyak_level, w.prior_lo, w.prior_hi)
        chunk = 7 * 96
    else:
        lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)
        x = lo + (hi - lo) * w.uniforms(seed=rank_seed(w.seed, rank))
        wt = np.full(w.n_nodes, 1.0 / w.n_nodes)
        chunk = 7 * w.n_nodes
    n = x.shape[0]
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=chunk)
    ctx.jacobian = P.OED_JAC_DIFFERENCE
    stream = torch.cuda.current_stream(dev)
    tuning = ctx.autotune(chunk, stream=stream) if args.tuning == "auto" else \
        (ctx.set_tuning(*[int(v) for v in args.tuning.split(",")]) or ctx.tuning)
    theta = torch.tensor(x, device=dev)
    w_t = torch.tensor(wt, device=dev)
    H = torch.empty((n, 7, 7), dtype=torch.float64, device=dev)
    eig = torch.empty(1, dtype=torch.float64, device=dev)
    if args.workload == "design_sweep":
        wl = w.win_levels()
        Hr = torch.empty((n, w.nrec, len(wl), 28), dtype=torch.float64, device=dev)
        masks = torch.tensor(W.design_subsets(w.nrec, 10, 512, seed=w.seed), device=dev)
        deig = torch.empty((len(wl), masks.shape[0]), dtype=torch.float64, device=dev)

    def step():
        if args.workload == "layered":
            P.oed_hessian(ctx, theta, w.prior_lo, w.prior_hi, w.rel_step, sigma, H, stream=stream)
            P.oed_eig(ctx, H, w_t, w.prior_lo, w.prior_hi, eig, stream=stream)
        else:
            P.oed_hessian(ctx, theta, w.prior_lo, w.prior_hi, w.rel_step, sigma, H, win_levels=wl,
                          H_rec=Hr, stream=stream)
            for k in range(len(wl)):
                P.oed_eig_designs(ctx, Hr, k, masks, w_t, w.prior_lo, w.prior_hi, deig[k], stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    solves = 7 * n
    cells = w.cells * w.nsteps * solves
    evals = 1 if args.workload == "layered" else int(deig.numel())
    out = {"metric": METRIC, "workload": w.name, "value": evals / (ms * 1e-3), "unit": "EIG evals/s",
           "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup, "nodes": n, "solves": solves,
           "gcell_upd_per_s": cells / (ms * 1e-3) / 1e9, "jacobian": "difference",
           "stencil_kernel": kernel_label(tuning),
           "clocks": clk.summary()}
    if args.workload == "layered":
        out["eig"] = float(eig.item())
    else:
        e = deig.cpu().numpy()
        out["designs_per_window"] = int(masks.shape[0])
        out["best_design_eig_per_window"] = [float(np.nanmax(r)) for r in e]
    if rank == 0:
        print(json.dumps(out))


def run_paper_scenarios(args, rank, world, local):
    """The paper's model problem (Sec. 4.1: two layers, h = 200 m, dt = 0.025 s, T = 8 s,
    C_eps = 1e-4 I) and its Scenarios I-III (Sec. 4.5): per-receiver partial Hessians over
    the 91 candidate surface nodes from sensitivity solves (Alg. 1 steps 1-5), then the EIG
    of all 36 designs, for the sparse grid of 8583 nodes and M = 10^4 MC nodes."""
    import torch
    import paper_1502_07873_gb300 as P
    from paper_1502_07873_gb300 import build as B
    torch.cuda.set_device(local)
    B.build()
    dev = torch.device("cuda", local)
    w = W.paper_model()
    sigma = 0.01
    scen = W.paper_scenarios()
    masks = torch.tensor(np.stack([m for _, _, m in scen]), device=dev)
    chunk = 2048
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=7 * chunk)
    ctx.jacobian = P.OED_JAC_SENSITIVITY
    stream = torch.cuda.current_stream(dev)
    tuning = ctx.autotune(7 * chunk, stream=stream)
    rules = {}
    x, wt = P.oed_nodes_smolyak(7, 5, w.prior_lo, w.prior_hi)
    rules["sparse_grid_8583"] = (x, wt)
    lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)
    u = np.random.default_rng(6).random((10000, 7))
    rules["monte_carlo_10000"] = (lo + (hi - lo) * u, np.full(10000, 1e-4))
    out = {"metric": "paper model problem, Scenarios I-III (Sec. 4.5)", "workload": w.name,
           "jacobian": "sensitivity (Alg. 1 steps 1-5)", "sigma": sigma,
           "stencil_kernel": kernel_label(tuning), "rules": {}}
    for name, (x, wt) in rules.items():
        n = x.shape[0]
        th = torch.tensor(x, device=dev)
        w_t = torch.tensor(wt, device=dev)
        H = torch.empty((n, 7, 7), dtype=torch.float64, device=dev)
        Hr = torch.empty((n, w.nrec, 1, 28), dtype=torch.float64, device=dev)
        eig = torch.empty(len(scen), dtype=torch.float64, device=dev)
        nb = torch.empty(len(scen), dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        P.oed_hessian(ctx, th, w.prior_lo, w.prior_hi, w.rel_step, sigma, H, win_levels=[w.nlevels],
                      H_rec=Hr, stream=stream)
        P.oed_eig_designs(ctx, Hr, 0, masks, w_t, w.prior_lo, w.prior_hi, eig, n_bad=nb, stream=stream)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        e = eig.cpu().numpy()
        b = nb.cpu().numpy()
        res = {"nodes": n, "solves": 7 * n, "seconds": el, "designs": len(scen),
               "cell_updates": w.cells * w.nsteps * 7 * n}
        for sc in ("I", "II", "III"):
            res[f"scenario_{sc}"] = [[v, float(e[k]), int(b[k])] for k, (s_, v, _) in enumerate(scen) if s_ == sc]
        out["rules"][name] = res
    # conditioning at the prior mean (Sec. 4.2 prints 3.88e30 unscaled and 12.16 scaled)
    th = torch.tensor(np.array([W.PAPER_PRIOR_MEAN]), device=dev)
    H = torch.empty((1, 7, 7), dtype=torch.float64, device=dev)
    P.oed_hessian(ctx, th, w.prior_lo, w.prior_hi, w.rel_step, sigma, H, stream=stream)
    Hm = H[0].cpu().numpy()
    S = np.sqrt(np.diag(Hm))
    out["prior_mean_cond"] = {"unscaled": float(np.linalg.cond(Hm)),
                              "scaled": float(np.linalg.cond(Hm / np.outer(S, S))),
                              "receivers": "all 91 candidates"}
    if rank == 0:
        print(json.dumps(out))


def _fit_rate(n, err):
    """Convergence rate r of err ~ n^-r by least squares in log-log."""
    n, err = np.asarray(n, float), np.asarray(err, float)
    ok = err > 0
    if ok.sum() < 2:
        return None
    return float(-np.polyfit(np.log(n[ok]), np.log(err[ok]), 1)[0])


def run_paper_study(args, rank, world, local):
    """Sec. 4.3-4.4 on the model problem: three unknowns (theta_2 depth, theta_4 omega,
    theta_5 m_xx), the other four known; observed for T = 1.25 s at x_1 = -9000 m and
    1000 m; C_eps = 1e-4 I.
    (a) Laplace EIG (Thm 4 on the unknowns, sensitivity solves, FP32 stencil) on the
        twenty sparse grids of Sec. 4.3 (351 ... 271857 nodes) and on Monte Carlo samples
        M = 1e2 ... 1e5 (ten realisations each); relative errors and fitted rates (the paper:
        0.40 sparse, 0.49 MC).
    (b) Double-loop Monte Carlo estimate of the definition (FP64 seismograms, N = M outer /
        inner samples, independent and reused) against the finest Laplace value (the paper:
        within 4%)."""
    import torch
    import paper_1502_07873_gb300 as P
    from paper_1502_07873_gb300 import build as B
    torch.cuda.set_device(local)
    B.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    w = W.paper_study_model()
    sigma = 0.01
    unknown = list(W.PAPER_STUDY_UNKNOWN)
    lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)
    chunk = 4096
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=7 * chunk)
    ctx.jacobian = P.OED_JAC_SENSITIVITY
    tuning = ctx.autotune(7 * chunk, stream=stream)

    def laplace(theta, wts):
        n = theta.shape[0]
        th = torch.tensor(theta, device=dev)
        H = torch.empty((n, 7, 7), dtype=torch.float64, device=dev)
        eig = torch.empty(1, dtype=torch.float64, device=dev)
        nb = torch.empty(1, dtype=torch.int32, device=dev)
        P.oed_hessian(ctx, th, w.prior_lo, w.prior_hi, w.rel_step, sigma, H, stream=stream)
        P.oed_eig_subset(ctx, H, torch.tensor(wts, device=dev), w.prior_lo, w.prior_hi, unknown, eig,
                         n_bad=nb, stream=stream)
        return float(eig.item()), int(nb.item())

    t0 = time.perf_counter()
    sparse = []
    for L in range(5, 5 + args.study_levels):
        x, wt = P.oed_nodes_smolyak(3, L, lo[unknown], hi[unknown])
        th = np.tile(np.array(W.PAPER_STUDY_KNOWN), (x.shape[0], 1))
        th[:, unknown] = x
        e, nb = laplace(th, wt)
        sparse.append([int(x.shape[0]), e, nb])
    t_sparse = time.perf_counter() - t0
    ref = sparse[-1][1]
    sp_err = [[sparse[i][0], abs(sparse[i + 1][1] - sparse[i][1]) / abs(sparse[i + 1][1])]
              for i in range(len(sparse) - 1)]
    t0 = time.perf_counter()
    mc = []
    rng = np.random.default_rng(43)
    for M in (100, 1000, 10000, 50000, 100000):
        vals = [laplace(W.paper_study_thetas(rng.random((M, 3))), np.full(M, 1.0 / M))[0]
                for _ in range(args.study_realisations)]
        # relative error of one estimate: the spread of the realisations over their mean
        mc.append([M, float(np.mean(vals)), float(np.std(vals)), float(np.std(vals) / abs(np.mean(vals)))])
    t_mc = time.perf_counter() - t0
    ref = mc[-1][1]   # the most accurate Laplace value: 10 realisations of M = 1e5
    # (b) double-loop Monte Carlo, FP64 seismograms
    ctx64 = P.Context(P.problem_from_workload(w, P.OED_FP64), max_solves=chunk)
    D = w.nlevels * w.nrec * 2
    gen = torch.Generator(device=dev)
    gen.manual_seed(44)
    dl = []
    for N in args.dlmc_sizes:
        r = np.random.default_rng(1000 + N)
        th_o = torch.tensor(W.paper_study_thetas(r.random((N, 3))), device=dev)
        th_i = torch.tensor(W.paper_study_thetas(r.random((N, 3))), device=dev)
        g_o = torch.empty((N, D), dtype=torch.float64, device=dev)
        g_i = torch.empty((N, D), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for a in range(0, N, chunk):
            b = min(N, a + chunk)
            P.oed_forward(ctx64, th_o[a:b], g_o[a:b], stream=stream)
            P.oed_forward(ctx64, th_i[a:b], g_i[a:b], stream=stream)
        eps = sigma * torch.randn((N, D), dtype=torch.float64, device=dev, generator=gen)
        le = torch.empty(N, dtype=torch.float64, device=dev)
        e_ind = torch.empty(1, dtype=torch.float64, device=dev)
        e_re = torch.empty(1, dtype=torch.float64, device=dev)
        P.oed_dlmc(g_o, eps, g_i, sigma, le, e_ind, stream=stream)
        P.oed_dlmc(g_o, eps, g_o, sigma, le, e_re, stream=stream)
        torch.cuda.synchronize()
        dl.append([N, float(e_ind.item()), float(e_re.item()), time.perf_counter() - t1])
    # (c) Thm 3 (H_1 + H_II at the Newton estimate on noisy data) against Thm 4 on M = 1000
    #     Monte Carlo nodes, FP64 stencil, one noise realisation per node
    M3 = 1000
    ctx3 = P.Context(P.problem_from_workload(w, P.OED_FP64), max_solves=7 * 1024)
    ctx3.jacobian = P.OED_JAC_SENSITIVITY
    th3 = torch.tensor(W.paper_study_thetas(np.random.default_rng(45).random((M3, 3))), device=dev)
    g3 = torch.empty((M3, w.nlevels, w.nrec, 2), dtype=torch.float64, device=dev)
    P.oed_forward(ctx3, th3, g3, stream=stream)
    y3 = g3 + sigma * torch.randn(g3.shape, dtype=torch.float64, device=dev, generator=gen)
    w3 = torch.full((M3,), 1.0 / M3, dtype=torch.float64, device=dev)
    H3 = torch.empty((M3, 7, 7), dtype=torch.float64, device=dev)
    gr3 = torch.empty((M3, 7), dtype=torch.float64, device=dev)
    e4 = torch.empty(1, dtype=torch.float64, device=dev)
    e3 = torch.empty(1, dtype=torch.float64, device=dev)
    nb3 = torch.empty(1, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    P.oed_hessian(ctx3, th3, w.prior_lo, w.prior_hi, w.rel_step, sigma, H3, stream=stream)
    P.oed_eig_subset(ctx3, H3, w3, w.prior_lo, w.prior_hi, unknown, e4, stream=stream)
    torch.cuda.synchronize()
    t_thm4 = time.perf_counter() - t1
    H3.zero_()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    P.oed_hessian_ii(ctx3, th3, y3, sigma, H3, grad=gr3, stream=stream)   # one primal + one dual per node
    torch.cuda.synchronize()
    t_hii = time.perf_counter() - t1
    theta_hat = th3.clone()
    t1 = time.perf_counter()
    P.oed_hessian_map(ctx3, theta_hat, y3, w.prior_lo, w.prior_hi, w.rel_step, sigma, 4, H3, gr3, free=unknown,
                      stream=stream)
    P.oed_eig_subset(ctx3, H3, w3, w.prior_lo, w.prior_hi, unknown, e3, n_bad=nb3, stream=stream)
    torch.cuda.synchronize()
    t_thm3 = time.perf_counter() - t1
    thm3 = {"nodes": M3, "thm4_eig": float(e4.item()), "thm3_eig": float(e3.item()),
            "thm3_not_pd": int(nb3.item()), "newton_iterations": 4, "seconds_thm4": t_thm4,
            "seconds_thm3": t_thm3, "seconds_h_ii": t_hii,
            "h_ii_gcell_upd_per_s": 2 * w.cells * w.nsteps * M3 / t_hii / 1e9,
            "note": "H_II: one primal and one dual solve per node (FP64), Gcell-updates of both"}
    out = {"metric": "Sec. 4.3-4.4: Laplace EIG convergence and Laplace vs double-loop MC",
           "workload": w.name, "unknown": ["theta_2 (depth)", "theta_4 (omega)", "theta_5 (m_xx)"],
           "sigma": sigma, "stencil_kernel": kernel_label(tuning),
           "laplace_sparse": sparse, "sparse_rel_err": sp_err,
           "sparse_rate": _fit_rate([e[0] for e in sp_err], [e[1] for e in sp_err]),
           "laplace_mc": mc, "mc_rate": _fit_rate([m[0] for m in mc], [m[3] for m in mc]),
           "laplace_reference": ref, "laplace_reference_from": "mean of the M = 1e5 realisations",
           "seconds_sparse": t_sparse, "seconds_mc": t_mc,
           "dlmc_columns": ["N = M", "independent inner samples", "inner = outer samples (reused)",
                            "seconds"],
           "dlmc": dl, "dlmc_reused_rel_to_laplace": [(d[2] - ref) / abs(ref) for d in dl],
           "thm3_vs_thm4": thm3}
    if rank == 0:
        print(json.dumps(out))


SERVING_GRIDS = ((201, 101, 10.0), (401, 201, 5.0))


def run_serving(args, rank, world, local):
    """Seeded Poisson arrivals of EIG requests mixing two grids, homogeneous and 3-layer
    media, 16-128 nodes and 5-40 receivers (T = 0.25 s), served with continuous batching
    (FP32 stencil, difference-form Jacobian, autotuned kernels) and by the plain form (FP64,
    pairs Jacobian, one request and one node at a time).  Reports p50 / p99 latency and
    EIG evals/s for both and the largest relative EIG difference between them."""
    import torch
    import paper_1502_07873_gb300 as P
    from paper_1502_07873_gb300 import build as B
    torch.cuda.set_device(local)
    B.build()
    reqs = W.serving_requests(args.requests, rate_hz=args.rate, seed=5 + rank, t_end=0.25,
                              grids=SERVING_GRIDS, m_range=(16, 128))
    sig = {}

    def sigma_of(w, prec):
        key = (w.nx, w.nz, w.layers, w.nsteps, prec)
        if key not in sig:
            sig[key] = noise_sigma_gpu(P, torch, w, prec)
        return sig[key]

    def build_requests(prec, jac):
        out = []
        for t, w in reqs:
            lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)
            th = lo + (hi - lo) * w.uniforms()
            out.append((t, P.make_request(P.problem_from_workload(w, prec), th,
                                          np.full(w.n_nodes, 1.0 / w.n_nodes), w.prior_lo,
                                          w.prior_hi, w.rel_step, sigma_of(w, prec), jac)))
        return out

    def serve(items, **kw):
        srv = P.Server(int(kw.pop("budget", 200 << 30)), **kw)
        # warm the per-shape tuning cache outside the timed stream
        seen = set()
        for t, r in items:
            key = (r.problem.nx, r.problem.nz)
            if key not in seen:
                seen.add(key)
                srv.wait(srv.submit(r))
        t0 = time.perf_counter()
        ids = []
        for t, r in items:
            d = t0 + t - time.perf_counter()
            if d > 0:
                time.sleep(d)
            ids.append(srv.submit(r))
        res = [srv.wait(i, 3600.0) for i in ids]
        srv.close()
        ok = [r for r in res if r.status == P.OED_OK]
        lat = sorted((r.t_done - r.t_submit) * 1e3 for r in ok)
        span = max(r.t_done for r in ok) - min(r.t_submit for r in ok)

        def pct(q):
            return lat[min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1)]
        failed = [(k, r.status, items[k][1].problem.nx, items[k][1].n) for k, r in enumerate(res)
                  if r.status != P.OED_OK]
        return {"requests": len(items), "completed": len(ok), "failed": failed, "p50_ms": pct(0.5),
                "p99_ms": pct(0.99), "eig_evals_per_s": len(ok) / span,
                "eig": [r.eig if r.status == P.OED_OK else None for r in res]}

    served_items = build_requests(P.OED_FP32, P.OED_JAC_DIFFERENCE)
    served = serve(served_items, max_active=4, chunk_nodes=64)
    # capacity: every request submitted at once; then arrivals at fractions of it (the same
    # seeded Poisson sequence, times scaled)
    burst = serve([(0.0, r) for _, r in served_items], max_active=4, chunk_nodes=64)
    capacity = burst["eig_evals_per_s"]
    sweep = []
    for frac in (0.5, 0.8):
        rate = frac * capacity
        items = [(t * args.rate / rate, r) for t, r in served_items]
        res = serve(items, max_active=4, chunk_nodes=64)
        sweep.append({"arrivals_per_s": rate, "fraction_of_capacity": frac, "p50_ms": res["p50_ms"],
                      "p99_ms": res["p99_ms"], "eig_evals_per_s": res["eig_evals_per_s"],
                      "completed": res["completed"]})
    burst.pop("eig")
    plain = serve(build_requests(P.OED_FP64, P.OED_JAC_PAIRS), max_active=1, chunk_nodes=1,
                  autotune=False)
    diffs = [(abs(a - b) / abs(b), k) for k, (a, b) in enumerate(zip(served.pop("eig"), plain.pop("eig")))
             if a is not None and b is not None]
    rel = max(diffs)[0]
    worst = [{"request": k, "rel_diff": d, "grid": f"{reqs[k][1].nx}x{reqs[k][1].nz}",
              "nodes": reqs[k][1].n_nodes, "receivers": reqs[k][1].nrec,
              "layers": len(reqs[k][1].layers)} for d, k in sorted(diffs, reverse=True)[:4]]
    if rank == 0:
        print(json.dumps({"metric": "serving: p50/p99 latency and EIG evals/s", "impl": "ours",
                          "arrivals_per_s": args.rate, "grids": [f"{a}x{b}" for a, b, _ in SERVING_GRIDS],
                          "served_fp32_batched": served, "plain_fp64_one_at_a_time": plain,
                          "served_capacity_all_at_once": burst, "served_rate_sweep": sweep,
                          "max_rel_eig_diff_served_vs_plain": rel,
                          "median_rel_eig_diff": sorted(d for d, _ in diffs)[len(diffs) // 2],
                          "largest_diffs": worst}))


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.serving:
        run_serving(args, rank, world, local)
        return
    if args.workload == "paper_scenarios" and args.impl == "ours":
        run_paper_scenarios(args, rank, world, local)
        return
    if args.workload == "paper_study" and args.impl == "ours":
        run_paper_study(args, rank, world, local)
        return
    if args.workload in ("layered", "design_sweep") and args.impl == "ours":
        run_other_workload(args, rank, world, local)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
