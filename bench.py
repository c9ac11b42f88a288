"""Benchmark of the Laplace expected-information-gain hot path on GB300.

One step = one EIG evaluation of the batched workload (401x201 grid, h = 5 m,
2000 leap-frog steps, 256 Monte Carlo nodes x 15 central-FD solves = 3840
solves, 20 surface receivers): source setup, all time steps (FP32 stencil),
FP64 Jacobian / Hessian, FP64 scaled log-determinants and the quadrature sum.
Inputs are resident in HBM when the timed region starts; the 5.1 GB of
wavefields per step exceed the 129 MB L2, so no flush is needed.  The line
carries the timed run's own per-node gains on ten nodes spread over the prior
box against the FP64 oracle (``parity``), and, at N = 1, three sub-objects
timed after it: ``layered`` (801x401, 3 layers, 4000 steps, 589 Smolyak nodes),
``design_sweep`` (1024 nodes, 40 candidates, 3 windows x 5120 designs) and
``serving`` (a bounded seeded draw from the serving mix of four grid sizes,
served against the plain FP64 one-at-a-time form).

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
# FP32 lanes per SM on sm_103a (4 sub-partitions x 32), each retiring one FMA (2 flops)
# per cycle; the peak is this x the device's SM count x the SM clock
FP32_LANES_PER_SM = 128


def fp32_peak_tflops(sm_count: int, sm_mhz: float) -> float:
    """FP32 peak derived from the unit counts and the clock (FMA counted as 2 flops)."""
    return sm_count * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def sm_max_mhz_default() -> float:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            v = json.load(f).get("sm_max_mhz")
        if v:
            return float(v)
    return 2070.0


def kernel_label(t):
    """Human-readable stencil kernel for a (cluster, rows, warps) tuning triple."""
    if t[0] > 0:
        return "cluster-resident, %d CTAs per solve" % t[0]
    if t[0] == -2:
        return "two-step TMA streaming (two leap-frog steps per pass, persistent, 4-stage mbarrier ring)"
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
    ap.add_argument("--cpu-sample-nodes", type=int, default=2,
                    help="--impl reference: nodes of the oracle's timed sample per step")
    ap.add_argument("--parity-nodes", type=int, default=10,
                    help="nodes of the timed run checked against the oracle (spread over the prior box)")
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
    ap.add_argument("--study-unknown", default="1,3,4",
                    help="paper_study: indices of the unknown parameters (the paper's: 1,3,4 = depth, omega, "
                         "m_xx); any other set runs the convergence rates only")
    ap.add_argument("--dlmc-sizes", type=lambda v: [int(x) for x in v.split(",")],
                    default=[256, 1024, 4096, 16384, 65536])
    ap.add_argument("--serving", action="store_true",
                    help="serving benchmark: Poisson arrivals of mixed EIG requests")
    ap.add_argument("--requests", type=int, default=24,
                    help="serving: requests taken from the head of the seeded config-5 stream")
    ap.add_argument("--serving-work", type=float, default=1.2e13,
                    help="serving: bound on the draw's total cell-updates")
    ap.add_argument("--serving-workers", type=int, default=4,
                    help="serving: requests the server runs at once (max_active)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the layered, design-sweep and serving sub-objects of the default line")
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


KERNEL_SOURCES = {"k_resident": ("resident.cu", "pair_math.cuh", "stencil_cell.cuh", "oed_internal.cuh"),
                  "k_step": ("stencil.cu", "stencil_cell.cuh", "oed_internal.cuh"),
                  "k_step_tma": ("stream_tma.cu", "tma_sync.cuh", "stencil_cell.cuh", "oed_internal.cuh"),
                  "k_step2_tma": ("stream_tma2.cu", "pair_math.cuh", "tma_sync.cuh", "stencil_cell.cuh",
                                  "oed_internal.cuh")}


def streaming_kernel_name(tuning) -> str:
    return {-2: "k_step2_tma", -1: "k_step_tma"}.get(tuning[0], "k_step")


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


def oracle_dkl(w, sigma, theta, idx):
    """The FP64 oracle's D_KL-hat (Thm 4) of the nodes theta[idx] with the same prior box,
    FD step and noise level, each node's 14 perturbed solves spread over the host cores.
    Returns (values, wall seconds)."""
    from oracle import oracle as O
    O.build()
    G = O.Grid.from_workload(w)
    lp = O.log_uniform_density(w.prior_lo, w.prior_hi)
    out = []
    t0 = time.perf_counter()
    for i in idx:
        H, _ = O.node_hessian(G, theta[i], w.prior_lo, w.prior_hi, w.rel_step, sigma)
        ld, _, ok = O.scaled_logdet(H)
        out.append(O.dkl(ld, 7, lp) if ok else float("nan"))
    return out, time.perf_counter() - t0


def cpu_baseline_from(w, nodes: int, dt: float):
    """The oracle's throughput from a timed sample of `nodes` nodes, scaled to one EIG
    evaluation of the whole workload."""
    threads = min(14, os.cpu_count() or 1)
    per_eval = dt / nodes * w.n_nodes
    return {"value": 1.0 / per_eval, "unit": "EIG evals/s", "cores": int(threads), "kind": "oracle",
            "sample": f"{nodes} of {w.n_nodes} nodes ({nodes * 14} FP64 solves of "
                      f"{w.nx}x{w.nz}x{w.nsteps} steps), {dt:.1f} s wall, scaled to one EIG "
                      f"evaluation"}


def cpu_baseline(w, sigma, nodes: int):
    """The FP64 oracle on a bounded sample: the first `nodes` nodes of the same workload."""
    from oracle import oracle as O
    th, _ = O.mc_nodes(w.uniforms(), w.prior_lo, w.prior_hi)
    _, dt = oracle_dkl(w, sigma, th, list(range(nodes)))
    return cpu_baseline_from(w, nodes, dt), dt


def parity_summary(dkl_gpu, dkl_ref, idx, weights):
    """Per-node D_KL-hat of the timed run against the oracle on the sampled nodes: the
    largest relative error, and the relative error of the sampled part of the EIG sum."""
    rel = [abs(dkl_gpu[i] - r) / abs(r) for i, r in zip(idx, dkl_ref)]
    e_gpu = sum(weights[i] * dkl_gpu[i] for i in idx)
    e_ref = sum(weights[i] * r for i, r in zip(idx, dkl_ref))
    return {"nodes": [int(i) for i in idx], "max_rel_dkl": max(rel), "median_rel_dkl": float(np.median(rel)),
            "sampled_eig_rel": abs(e_gpu - e_ref) / abs(e_ref), "bar": 1e-3,
            "within_bar": bool(max(rel) <= 1e-3),
            "dkl_gpu": [float(dkl_gpu[i]) for i in idx], "dkl_oracle": [float(r) for r in dkl_ref]}


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
    dkl = torch.empty(w.n_nodes, dtype=torch.float64, device=dev)
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
        P.oed_eig(ctx, H, wt, w.prior_lo, w.prior_hi, eig, dkl=dkl, n_bad=nbad, stream=stream)

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
    dkl_timed = dkl.cpu().numpy()          # the last timed step's per-node gains
    n_bad_timed = int(nbad.item())

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
    clocks = clk.summary()
    if tuning[0] > 0:
        # cluster-resident kernel: one launch integrates every step; the wavefield never
        # leaves the chip, so the bound is FP32 issue, not HBM
        launch_ms = st_ms * w.nsteps
        flops = FLOPS_PER_CELL_UPDATE * cells
        achieved = flops / (launch_ms * 1e-3) / 1e12
        tb = ncu_traffic("k_resident")
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz_max = clocks.get("sm_max_mhz") or sm_max_mhz_default()
        mhz = clocks.get("sm_mhz") or mhz_max
        peak_fp32 = fp32_peak_tflops(n_sm, mhz)
        roofline = {"bound": "alu", "kernel": "k_resident (cluster-resident leap-frog, all steps)",
                    "achieved": achieved, "peak": peak_fp32,
                    "peak_kind": f"derived: {n_sm} SMs (device attribute) x {FP32_LANES_PER_SM} FP32 lanes "
                                 f"x 2 x {mhz:.0f} MHz (median SM clock sampled in the timed region)",
                    "unit": "TFLOP/s", "frac": achieved / peak_fp32,
                    "frac_at_max_clock": achieved / fp32_peak_tflops(n_sm, mhz_max),
                    "algorithmic_flops_per_cell_update": FLOPS_PER_CELL_UPDATE,
                    "fp32_pipe_frac": FP32_INSTR_PER_CELL_UPDATE * cells / (launch_ms * 1e-3)
                    / (peak_fp32 * 1e12 / 2),
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
        kname = streaming_kernel_name(tuning)
        tb = ncu_traffic(kname)
        roofline = {"bound": "hbm", "kernel": kname + " (streaming leap-frog, one step)",
                    "achieved": hbm_equiv, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                    "frac": hbm_equiv / peak, "algorithmic_bytes_per_cell_update": bpc,
                    "traffic": (tb * per_launch_cells if tb is not None else None),
                    "launch_ms": st_ms}
        launches_per_step = w.nsteps + 5
    value = weak_scaling_value(world, args.steps, total_ms)
    # accuracy of the timed run itself: its per-node gains on nodes spread over the prior
    # box against the FP64 oracle (the same nodes' solves time the CPU baseline)
    cb, parity = None, None
    if not args.no_cpu_baseline:
        th_np = theta.cpu().numpy()
        idx = W.spread_sample(th_np, w.prior_lo, w.prior_hi)[:max(2, args.parity_nodes)]
        ref, dt = oracle_dkl(w, sigma, th_np, idx)
        parity = parity_summary(dkl_timed, ref, idx, wt.cpu().numpy())
        parity["oracle"] = "FP64 C oracle: literal +/- solves, FD Jacobian, H_1, scaled Cholesky, D_KL-hat"
        if world == 1:
            cb = cpu_baseline_from(w, len(idx), dt)
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
        "n_bad": n_bad_timed,
        "parity": parity,
        "sigma": sigma,
        "roofline": roofline,
        "clocks": clocks,
        "gpu_launches": args.steps * launches_per_step,
        "e2e": e2e,
        "jacobian_difference_form": diff,
    }
    if cb:
        out["cpu_baseline"] = cb
    if world == 1 and not args.no_extra:
        # the other configurations, each timed on its own after the headline: the layered
        # Smolyak workload (config 3), the design sweep (config 4) and the serving mix
        # (config 5, a bounded draw)
        ctx.close()
        del H, dkl, theta
        torch.cuda.empty_cache()
        extra_oracle = 0 if args.no_cpu_baseline else 2
        out["layered"] = measure_layered(P, torch, dev, args, rank, oracle_nodes=extra_oracle)
        torch.cuda.empty_cache()
        out["design_sweep"] = measure_design_sweep(P, torch, dev, args, rank, oracle_nodes=extra_oracle)
        torch.cuda.empty_cache()
        out["serving"] = measure_serving(P, torch, dev, args, rank, n_first=args.requests,
                                         work_bound=args.serving_work)
    print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def streaming_roofline(kname, ms_per_launch, cells_per_launch, bpc=24):
    """HBM roofline of a streaming stencil kernel (one time step of a batch per launch)."""
    peak, peak_kind = measured_peaks()
    gbs = cells_per_launch * bpc / (ms_per_launch * 1e-3) / 1e9
    tb = ncu_traffic(kname)
    return {"bound": "hbm", "kernel": kname, "achieved": gbs, "peak": peak, "peak_kind": peak_kind,
            "unit": "GB/s", "frac": gbs / peak, "algorithmic_bytes_per_cell_update": bpc,
            "traffic": (tb * cells_per_launch if tb is not None else None),
            "traffic_note": "committed ncu DRAM bytes per cell-update of the same code (one-pass capture "
                            "named in profiles/stencil_dram_traffic.json) x the cell-updates of one launch",
            "launch_ms": ms_per_launch}


def resident_roofline(launch_ms, cells, n_sm, mhz):
    """FP32 roofline of the cluster-resident kernel (all steps of a batch per launch)."""
    peak = fp32_peak_tflops(n_sm, mhz)
    achieved = FLOPS_PER_CELL_UPDATE * cells / (launch_ms * 1e-3) / 1e12
    tb = ncu_traffic("k_resident")
    return {"bound": "alu", "kernel": "k_resident", "achieved": achieved, "peak": peak,
            "peak_kind": f"derived: {n_sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {mhz:.0f} MHz",
            "unit": "TFLOP/s", "frac": achieved / peak, "algorithmic_flops_per_cell_update": FLOPS_PER_CELL_UPDATE,
            "traffic": (tb * cells if tb is not None else None), "launch_ms": launch_ms}


def measure_layered(P, torch, dev, args, rank, oracle_nodes=2):
    """One EIG evaluation of the layered Smolyak workload (801x401, 3 layers, 4000 steps,
    level-3 sparse grid of 589 nodes, 40 receivers; FP32 stencil, difference-form Jacobian):
    warm-up on one chunk, then the whole evaluation timed once; sampled nodes' D_KL-hat
    against the FP64 oracle."""
    w = W.layered()
    sigma = args.sigma if args.sigma > 0 else noise_sigma_gpu(P, torch, w, P.OED_FP32)
    x, wt = P.oed_nodes_smolyak(7, w.smolyak_level, w.prior_lo, w.prior_hi)
    if args.nodes:   # profiling runs: the first nodes of the rule only
        x, wt = x[:args.nodes], wt[:args.nodes]
    chunk_nodes = 96
    n = x.shape[0]
    # the rule lists its nodes grouped by the coordinates they vary (in some runs of 96
    # nodes every source sits at one position); taking every k-th node per chunk spreads
    # each chunk's sources over the grid, which the two-step kernel runs faster (the sum
    # does not depend on the order)
    nchunk = (n + chunk_nodes - 1) // chunk_nodes
    perm = np.concatenate([np.arange(c, n, nchunk) for c in range(nchunk)])
    x, wt = x[perm], wt[perm]
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=7 * chunk_nodes)
    ctx.jacobian = P.OED_JAC_DIFFERENCE
    stream = torch.cuda.current_stream(dev)
    tuning = ctx.autotune(7 * chunk_nodes, stream=stream) if args.tuning == "auto" else \
        (ctx.set_tuning(*[int(v) for v in args.tuning.split(",")]) or ctx.tuning)
    theta = torch.tensor(x, device=dev)
    w_t = torch.tensor(wt, device=dev)
    H = torch.empty((n, 7, 7), dtype=torch.float64, device=dev)
    eig = torch.empty(1, dtype=torch.float64, device=dev)
    dkl = torch.empty(n, dtype=torch.float64, device=dev)
    nb = torch.empty(1, dtype=torch.int32, device=dev)
    # warm-up: one full chunk and the last, partial one (their captured time loops)
    tail = n - (n // chunk_nodes) * chunk_nodes
    warm = list(range(min(chunk_nodes, n))) + (list(range(n - tail, n)) if tail and n > chunk_nodes else [])
    P.oed_hessian(ctx, theta[warm], w.prior_lo, w.prior_hi, w.rel_step, sigma, H[:len(warm)], stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st_ms, st_launches, st_cells = 0.0, 0, 0   # the stencil launches of every chunk
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record(stream)
        for a in range(0, n, chunk_nodes):   # one chunk per call, so each chunk's time loop is read
            b = min(n, a + chunk_nodes)
            P.oed_hessian(ctx, theta[a:b], w.prior_lo, w.prior_hi, w.rel_step, sigma, H[a:b], stream=stream)
            stream.synchronize()
            ms_k, l_k = ctx.last_step_time()
            st_ms += ms_k
            st_launches += l_k
            st_cells += w.cells * 7 * (b - a) * w.nsteps
        P.oed_eig(ctx, H, w_t, w.prior_lo, w.prior_hi, eig, dkl=dkl, n_bad=nb, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    solves = 7 * n
    cells = w.cells * w.nsteps * solves
    if tuning[0] > 0:
        roof = resident_roofline(st_ms, st_cells, torch.cuda.get_device_properties(dev).multi_processor_count,
                                 clk.summary().get("sm_mhz") or sm_max_mhz_default())
    else:
        kname = streaming_kernel_name(tuning)
        roof = streaming_roofline(kname, st_ms / max(1, st_launches), st_cells / max(1, st_launches))
    out_stencil_share = st_ms / ms
    out = {"workload": w.name, "value": 1.0 / (ms * 1e-3), "unit": "EIG evals/s", "ms_per_eval": ms,
           "nodes": n, "solves": solves, "time_steps": w.nsteps, "grid": f"{w.nx}x{w.nz}",
           "receivers": w.nrec, "layers": len(w.layers), "jacobian": "difference (7 solves per node, FP64 "
           "forcing differences)", "chunk_nodes": chunk_nodes,
           "gcell_upd_per_s": cells / (ms * 1e-3) / 1e9, "stencil_kernel": kernel_label(tuning),
           "eig": float(eig.item()), "n_bad": int(nb.item()), "sigma": sigma, "roofline": roof,
           "clocks": clk.summary(), "stencil_share_of_time": out_stencil_share,
           "timed": "one evaluation after a warm-up of two chunks",
           "chunks": "nodes interleaved across chunks (every k-th node of the rule per chunk)"}
    if oracle_nodes > 0 and rank == 0:
        d = dkl.cpu().numpy()
        idx = W.spread_sample(x, w.prior_lo, w.prior_hi, first=(0, n // 2))[:oracle_nodes]
        ref, dt = oracle_dkl(w, sigma, x, idx)
        out["parity"] = parity_summary(d, ref, idx, wt)
        out["parity"]["oracle_seconds"] = dt
    ctx.close()
    return out


def measure_design_sweep(P, torch, dev, args, rank, oracle_nodes=2):
    """The design sweep (401x201, 2400 steps, 1024 MC nodes, 40 candidate receivers,
    windows T = 0.5 / 1 / 2 s, EIG of 512 seeded subsets for every k = 1..10 in every
    window; FP32 stencil, difference form): per-receiver, per-window partial Hessians in
    one pass, then 3 x 5120 design EIGs; one warm-up sweep and two timed; sampled nodes'
    full-design D_KL-hat against the FP64 oracle."""
    w = W.design_sweep()
    sigma = args.sigma if args.sigma > 0 else noise_sigma_gpu(P, torch, w, P.OED_FP32)
    lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)
    x = lo + (hi - lo) * w.uniforms(seed=rank_seed(w.seed, rank))
    wt = np.full(w.n_nodes, 1.0 / w.n_nodes)
    n = x.shape[0]
    ctx = P.Context(P.problem_from_workload(w, P.OED_FP32), max_solves=7 * n)
    ctx.jacobian = P.OED_JAC_DIFFERENCE
    stream = torch.cuda.current_stream(dev)
    tuning = ctx.autotune(7 * n, stream=stream) if args.tuning == "auto" else \
        (ctx.set_tuning(*[int(v) for v in args.tuning.split(",")]) or ctx.tuning)
    theta = torch.tensor(x, device=dev)
    w_t = torch.tensor(wt, device=dev)
    H = torch.empty((n, 7, 7), dtype=torch.float64, device=dev)
    wl = w.win_levels()
    Hr = torch.empty((n, w.nrec, len(wl), 28), dtype=torch.float64, device=dev)
    masks = torch.tensor(W.design_subsets(w.nrec, 10, 512, seed=w.seed), device=dev)
    deig = torch.empty((len(wl), masks.shape[0]), dtype=torch.float64, device=dev)

    def sweep():
        P.oed_hessian(ctx, theta, w.prior_lo, w.prior_hi, w.rel_step, sigma, H, win_levels=wl, H_rec=Hr,
                      stream=stream)
        for k in range(len(wl)):
            P.oed_eig_designs(ctx, Hr, k, masks, w_t, w.prior_lo, w.prior_hi, deig[k], stream=stream)

    sweep()
    torch.cuda.synchronize()
    reps = 2
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st = []
    with ClockSampler(torch.cuda.current_device()) as clk:
        e0.record(stream)
        for _ in range(reps):
            sweep()
            torch.cuda.synchronize()
            st.append(ctx.last_step_time()[0])
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    solves = 7 * n
    cells = w.cells * w.nsteps * solves
    evals = int(deig.numel())
    clocks = clk.summary()
    if tuning[0] > 0:
        roof = resident_roofline(statistics.median(st), cells,
                                 torch.cuda.get_device_properties(dev).multi_processor_count,
                                 clocks.get("sm_mhz") or sm_max_mhz_default())
    else:
        kname = streaming_kernel_name(tuning)
        roof = streaming_roofline(kname, statistics.median(st) / w.nsteps, w.cells * solves)
    e = deig.cpu().numpy()
    out = {"workload": w.name, "value": evals / (ms * 1e-3), "unit": "design EIG evals/s", "ms_per_sweep": ms,
           "designs_per_window": int(masks.shape[0]), "windows_s": list(w.win_seconds), "nodes": n,
           "solves": solves, "receivers": w.nrec, "time_steps": w.nsteps,
           "gcell_upd_per_s": cells / (ms * 1e-3) / 1e9, "stencil_kernel": kernel_label(tuning),
           "best_design_eig_per_window": [float(np.nanmax(r)) for r in e], "sigma": sigma, "roofline": roof,
           "clocks": clocks, "timed": f"{reps} sweeps after one warm-up sweep"}
    if oracle_nodes > 0 and rank == 0:
        dkl = torch.empty(n, dtype=torch.float64, device=dev)
        eig = torch.empty(1, dtype=torch.float64, device=dev)
        P.oed_eig(ctx, H, w_t, w.prior_lo, w.prior_hi, eig, dkl=dkl, stream=stream)
        idx = W.spread_sample(x, w.prior_lo, w.prior_hi)[:oracle_nodes]
        ref, dt = oracle_dkl(w, sigma, x, idx)
        out["parity"] = parity_summary(dkl.cpu().numpy(), ref, idx, wt)
        out["parity"]["what"] = "D_KL-hat of the full design (all 40 receivers, T = 2 s) at sampled nodes"
        out["parity"]["oracle_seconds"] = dt
    ctx.close()
    return out


def run_other_workload(args, rank, world, local):
    """--workload layered / design_sweep: the sub-object alone, as one JSON line."""
    import torch
    import paper_1502_07873_gb300 as P
    from paper_1502_07873_gb300 import build as B
    torch.cuda.set_device(local)
    B.build()
    dev = torch.device("cuda", local)
    fn = measure_layered if args.workload == "layered" else measure_design_sweep
    out = fn(P, torch, dev, args, rank, oracle_nodes=0 if args.no_cpu_baseline else 2)
    out["metric"] = METRIC
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
    unknown = [int(v) for v in args.study_unknown.split(",")]
    rates_only = tuple(unknown) != tuple(W.PAPER_STUDY_UNKNOWN)
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
        x, wt = P.oed_nodes_smolyak(len(unknown), L, lo[unknown], hi[unknown])
        th = np.tile(np.array(W.PAPER_STUDY_KNOWN), (x.shape[0], 1))
        th[:, unknown] = x
        e, nb = laplace(th, wt)
        sparse.append([int(x.shape[0]), e, nb])
    t_sparse = time.perf_counter() - t0
    # consecutive differences of the sparse-grid values (the measure an earlier reading used)
    sp_diff = [[sparse[i][0], abs(sparse[i + 1][1] - sparse[i][1]) / abs(sparse[i + 1][1])]
               for i in range(len(sparse) - 1)]
    t0 = time.perf_counter()
    mc = []
    rng = np.random.default_rng(43)
    for M in (100, 1000, 10000, 50000, 100000):
        vals = [laplace(W.paper_study_thetas(rng.random((M, len(unknown))), unknown), np.full(M, 1.0 / M))[0]
                for _ in range(args.study_realisations)]
        # relative error of one estimate: the spread of the realisations over their mean
        mc.append([M, float(np.mean(vals)), float(np.std(vals)), float(np.std(vals) / abs(np.mean(vals)))])
    t_mc = time.perf_counter() - t0
    ref = mc[-1][1]   # the most accurate Laplace value: 10 realisations of M = 1e5
    ref_se = mc[-1][2] / math.sqrt(args.study_realisations)   # its standard error
    # the sparse grids' relative error against that converged reference (Sec. 4.3 measures
    # the error of each rule against a reference value); errors below a few standard
    # errors of the reference are not resolved and are left out of the rate fit
    sp_err = [[n_, abs(e_ - ref) / abs(ref)] for n_, e_, _ in sparse]
    resolved = [x for x in sp_err if x[1] * abs(ref) > 3 * ref_se]
    if rates_only:
        if rank == 0:
            print(json.dumps({"metric": "Sec. 4.3: Laplace EIG convergence, other unknowns", "workload": w.name,
                              "unknown": unknown, "sigma": sigma, "laplace_sparse": sparse,
                              "sparse_rel_err_vs_mc_reference": sp_err,
                              "sparse_rate": _fit_rate([e[0] for e in resolved], [e[1] for e in resolved]),
                              "sparse_rate_points": len(resolved), "sparse_rel_consecutive_diff": sp_diff,
                              "laplace_mc": mc, "mc_rate": _fit_rate([m[0] for m in mc], [m[3] for m in mc]),
                              "laplace_reference": ref, "laplace_reference_standard_error": ref_se}))
        return
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
           "laplace_sparse": sparse, "sparse_rel_err_vs_mc_reference": sp_err,
           "sparse_rate": _fit_rate([e[0] for e in resolved], [e[1] for e in resolved]),
           "sparse_rate_points": len(resolved),
           "sparse_rel_consecutive_diff": sp_diff,
           "sparse_rate_consecutive_diff": _fit_rate([e[0] for e in sp_diff], [e[1] for e in sp_diff]),
           "laplace_reference_standard_error": ref_se,
           "laplace_mc": mc, "mc_rate": _fit_rate([m[0] for m in mc], [m[3] for m in mc]),
           "laplace_reference": ref, "laplace_reference_from": "mean of the M = 1e5 realisations",
           "seconds_sparse": t_sparse, "seconds_mc": t_mc,
           "dlmc_columns": ["N = M", "independent inner samples", "inner = outer samples (reused)",
                            "seconds"],
           "dlmc": dl, "dlmc_reused_rel_to_laplace": [(d[2] - ref) / abs(ref) for d in dl],
           "thm3_vs_thm4": thm3}
    if rank == 0:
        print(json.dumps(out))


def serving_draw(n_first: int, work_bound: float, seed: int = 5):
    """The first n_first requests of the seeded config-5 stream (Poisson arrivals at 50/s;
    grids 201x101, 401x201, 801x401, 1601x801; 64-2048 nodes, log-uniform; 5-40
    receivers; homogeneous or 3-layer; T = 0.5 s), skipping any request that would take
    the total work (cell-updates of the difference-form solves) past work_bound."""
    keep, skipped, total = [], [], 0.0
    for t, w in W.serving_requests(n_first, rate_hz=50.0, seed=seed, t_end=0.5):
        cu = float(w.cells) * w.nsteps * 7 * w.n_nodes
        if total + cu <= work_bound:
            keep.append((t, w))
            total += cu
        else:
            skipped.append({"grid": f"{w.nx}x{w.nz}", "nodes": w.n_nodes, "cell_updates": cu})
    return keep, skipped, total


def _pct(vals, q):
    v = sorted(vals)
    return v[min(len(v) - 1, max(0, int(math.ceil(q * len(v))) - 1))]


def measure_serving(P, torch, dev, args, rank, n_first=24, work_bound=1.2e13, plain_nodes=1):
    """Config 5 served with continuous batching (FP32 stencil, difference-form Jacobian,
    autotuned kernels, pooled workspaces) against the plain form (FP64, central-FD pairs,
    one request and one node at a time).  The served stream is run twice: with the draw's
    own Poisson arrivals (50/s: far beyond capacity, so latency is queueing) and with the
    same arrivals slowed to 80% of the capacity measured in the first run.  The plain form
    is too slow to run whole: its per-node time is measured on `plain_nodes` nodes of every
    request (plus the request's setup) and its one-at-a-time queue is computed from those
    service times and the same arrival times.  Accuracy: the served per-node D_KL-hat (from
    the server's per-node checkpoint) against the plain FP64 D_KL-hat at the same nodes."""
    stream = torch.cuda.current_stream(dev)
    draw, skipped, total_cu = serving_draw(n_first, work_bound)
    sig = {}

    def sigma_of(w, prec):
        key = (w.nx, w.nz, w.layers, w.nsteps, prec)
        if key not in sig:
            sig[key] = noise_sigma_gpu(P, torch, w, prec)
        return sig[key]

    thetas = []
    for t, w in draw:
        lo, hi = np.array(w.prior_lo), np.array(w.prior_hi)
        thetas.append(lo + (hi - lo) * w.uniforms())
    chunk = 256

    def served_items():
        return [(t, P.make_request(P.problem_from_workload(w, P.OED_FP32), th, np.full(w.n_nodes, 1.0 / w.n_nodes),
                                   w.prior_lo, w.prior_hi, w.rel_step, sigma_of(w, P.OED_FP32), P.OED_JAC_DIFFERENCE,
                                   tag=k))
                for k, ((t, w), th) in enumerate(zip(draw, thetas))]

    items = served_items()
    srv = P.Server(200 << 30, max_active=args.serving_workers, chunk_nodes=chunk)
    # warm the per-shape tuning cache outside the timed streams: for each grid shape a
    # request of a full chunk of nodes and a few steps (the launch shape depends on the
    # grid and the batch, not on the step count)
    seen = set()
    for (t, w), th in zip(draw, thetas):
        if (w.nx, w.nz) in seen:
            continue
        seen.add((w.nx, w.nz))
        short = P.make_problem(w.nx, w.nz, w.h, w.dt, 16, w.layers, w.rec_ix, P.OED_FP32)
        r = P.make_request(short, np.resize(th, (chunk, 7)), np.full(chunk, 1.0 / chunk), w.prior_lo,
                           w.prior_hi, w.rel_step, sigma_of(w, P.OED_FP32), P.OED_JAC_DIFFERENCE)
        srv.wait(srv.submit(r), 3600.0)

    def run(arrivals):
        t0 = time.perf_counter()
        ids = []
        for (_, r), ta in zip(items, arrivals):
            d = t0 + ta - time.perf_counter()
            if d > 0:
                time.sleep(d)
            ids.append(srv.submit(r))
        res = [srv.wait(i, 7200.0) for i in ids]
        ok = [r for r in res if r.status == P.OED_OK]
        lat = [(r.t_done - r.t_submit) * 1e3 for r in ok]
        span = max(r.t_done for r in ok) - min(r.t_submit for r in ok)
        return ids, res, {"requests": len(res), "completed": len(ok), "p50_ms": _pct(lat, 0.5),
                          "p99_ms": _pct(lat, 0.99), "eig_evals_per_s": len(ok) / span, "span_s": span,
                          "reused_workspaces": int(sum(r.workspace_reused for r in res))}

    arr = [t for t, _ in draw]
    with ClockSampler(torch.cuda.current_device()) as clk:
        ids, res, at50 = run(arr)
    cap = at50["eig_evals_per_s"]
    # per-request metrics lines of the first run, summarised per grid
    per_grid = {}
    for i in ids:
        m = srv.metrics(i)
        g = per_grid.setdefault(m["grid"], {"requests": 0, "gcell_upd_per_s": []})
        g["requests"] += 1
        g["gcell_upd_per_s"].append(m["gcell_upd_per_s"])
    for g in per_grid.values():
        g["gcell_upd_per_s"] = float(np.median(g["gcell_upd_per_s"]))
    # served per-node Hessians of the nodes the plain form is timed on
    served_H = {k: srv.checkpoint(i)[:plain_nodes] for k, i in enumerate(ids)}
    rate80 = 0.8 * cap
    scale = (len(arr) / rate80) / max(arr[-1], 1e-9)   # same arrival pattern, mean rate 0.8 x capacity
    _, _, at80 = run([t * scale for t in arr])
    at80["arrivals_per_s"] = rate80
    srv.close()

    # the plain form: FP64, pairs, one node at a time, one request at a time
    service, dkl_rel = [], []
    for k, ((t, w), th) in enumerate(zip(draw, thetas)):
        t1 = time.perf_counter()
        ctx = P.Context(P.problem_from_workload(w, P.OED_FP64), max_solves=15)
        sg = sigma_of(w, P.OED_FP32)
        Hp = torch.empty((plain_nodes, 7, 7), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        t_setup = time.perf_counter() - t1
        t2 = time.perf_counter()
        for j in range(plain_nodes):
            P.oed_hessian(ctx, torch.tensor(th[j:j + 1], device=dev), w.prior_lo, w.prior_hi, w.rel_step, sg,
                          Hp[j:j + 1], stream=stream)
        torch.cuda.synchronize()
        t_node = (time.perf_counter() - t2) / plain_nodes
        ctx.close()
        service.append(t_setup + w.n_nodes * t_node)
        # D_KL-hat of the same nodes from the served FP32 Hessians and the plain FP64 ones
        Hs = torch.tensor(served_H[k], device=dev)
        ones = torch.ones(plain_nodes, dtype=torch.float64, device=dev)
        e = torch.empty(1, dtype=torch.float64, device=dev)
        ds = torch.empty(plain_nodes, dtype=torch.float64, device=dev)
        dp = torch.empty(plain_nodes, dtype=torch.float64, device=dev)
        P.oed_eig(None, Hs, ones, w.prior_lo, w.prior_hi, e, dkl=ds, stream=stream)
        P.oed_eig(None, Hp, ones, w.prior_lo, w.prior_hi, e, dkl=dp, stream=stream)
        for a_, b_ in zip(ds.cpu().numpy(), dp.cpu().numpy()):
            dkl_rel.append(abs(a_ - b_) / abs(b_))
    done, lat = 0.0, []
    for ta, sv in zip(arr, service):
        done = max(done, ta) + sv
        lat.append((done - ta) * 1e3)
    plain = {"p50_ms": _pct(lat, 0.5), "p99_ms": _pct(lat, 0.99), "eig_evals_per_s": len(arr) / (done - arr[0]),
             "how": f"service time = setup + nodes x the measured time of {plain_nodes} node(s) per request "
                    "(15 FP64 solves each); queue computed from those and the same arrival times"}
    grids = {}
    for t, w in draw:
        grids[f"{w.nx}x{w.nz}"] = grids.get(f"{w.nx}x{w.nz}", 0) + 1
    return {"workload": "config 5 serving mix, bounded draw", "requests": len(draw),
            "draw": f"first {n_first} requests of the seeded stream (seed 5, Poisson 50/s, T = 0.5 s), "
                    f"skipping those that would take the total past {work_bound:.2g} cell-updates",
            "skipped": skipped, "grids": grids, "cell_updates": total_cu,
            "nodes_range": [min(w.n_nodes for _, w in draw), max(w.n_nodes for _, w in draw)],
            "served_fp32_batched_at_50_per_s": at50, "served_capacity_eig_evals_per_s": cap,
            "served_at_80pct_capacity": at80, "served_per_grid": per_grid,
            "plain_fp64_one_at_a_time": plain,
            "served_vs_plain_max_rel_dkl": max(dkl_rel), "served_vs_plain_median_rel_dkl": float(np.median(dkl_rel)),
            "accuracy_nodes": len(dkl_rel), "clocks": clk.summary(),
            "server": f"max_active {args.serving_workers}, chunk 256 nodes, budget 200 GiB, pooled workspaces, admission past a "
                      "blocked head within 10 s"}


def run_serving(args, rank, world, local):
    """--serving: the config-5 serving measurement alone, as one JSON line."""
    import torch
    import paper_1502_07873_gb300 as P
    from paper_1502_07873_gb300 import build as B
    torch.cuda.set_device(local)
    B.build()
    dev = torch.device("cuda", local)
    out = measure_serving(P, torch, dev, args, rank, n_first=args.requests, work_bound=args.serving_work)
    out["metric"] = "serving: p50/p99 latency and EIG evals/s"
    if rank == 0:
        print(json.dumps(out))


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
