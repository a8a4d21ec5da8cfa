"""Benchmark of the batched AC power flow on the 118-bus / 4096-scenario workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {gb300,reference}]

One step = one pf_solve over the whole batch (every Newton iteration of every
scenario, inputs already resident on the device).  Prints one JSON line:
converged solves/s of the mixed-precision form (FP32 factor + FP64 mismatch and
refinement) as the headline, the all-FP64 form and the implicit layer's
forward+backward rate beside it, the end-to-end rate through host buffers, the
ALU/HBM roofline of the solve kernel and the CPU oracle's rate.

``--impl reference`` times the CPU oracle (the plain FP64 Newton-Raphson the
tests compare against) on the host cores instead; there is no other reference
implementation of this method to run.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import platform
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "c1"
WORKLOAD_DESC = ("synthetic 118-bus meshed grid (186 branches, 9 transformers, 1 slack, 53 PV, "
                 "64 PQ), 4096 load scenarios x U(0.7, 1.3), flat start, tol 1e-8 pu, max 20 iterations")
# Plan schedules the headline's tuner compares: the default plan, and top regions of
# levels of at most 2, 3 or 5 rows whatever the network's size (and of at most 8 rows on
# the ordering with degree slack 2).
HEADLINE_SCHEDULES = ({}, {"top_rows": 2, "top_min_pivots": 0}, {"top_rows": 3, "top_min_pivots": 0},
                      {"top_rows": 5, "top_min_pivots": 0},
                      {"order_slack": 2, "top_rows": 8, "top_min_pivots": 0})
METRIC = "PF solves/s at <=1e-8 pu mismatch (mixed precision form)"

UNIT = "solves/s"
L2_FLUSH_BYTES = 256 << 20
# Peaks for the roofline.  HBM: the measured copy bandwidth of this GPU family
# (MEASURED_PEAKS.json).  ALU: FP64 and FP32 FMA throughput measured by this run on its
# own GPU (pf_measure_fma_peak, inside the clock-sampled region); the nominal figures
# (unit counts x 2.07 GHz) are reported beside them.
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_NOMINAL_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
HBM_FALLBACK_GBS = 6800.0


# the device code of the solve kernels (a committed capture is valid while these are unchanged)
KERNEL_SOURCES = ("pf_body.cuh", "pf_kernels.cu", "pf_device.cuh", "pf_si.cu")


def headline_kernel(shape):
    """The solve kernel a tuned launch shape runs, and the name of its committed ncu summary."""
    if shape and shape.get("placement") == 5:
        cl = "true" if shape.get("cluster", 1) > 1 else "false"
        return (f"nr_solve_si_kernel<float, {shape['pack']}, {cl}>",
                "nr_solve_si_c1_mixed.json")
    return "nr_solve_kernel<float>", "nr_solve_c1_mixed.json"


def profiled_traffic(kernel_json="nr_solve_c1_mixed.json"):
    """DRAM bytes per launch from the committed ncu capture, if the kernel source is
    unchanged since the capture (else None)."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", kernel_json)) as fh:
            prof = json.load(fh)
        src = b""
        for f in KERNEL_SOURCES:
            with open(os.path.join(ROOT, "paper_2606_07099_gb300", "csrc", f), "rb") as fh:
                src += fh.read()
        if hashlib.sha256(src).hexdigest()[:16] != prof["source_sha256_16"]:
            return None
        return prof["dram_bytes_read_per_launch"] + prof["dram_bytes_write_per_launch"]
    except Exception:
        return None


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


# ---------------------------------------------------------------- oracle leg (CPU)
def _oracle_chunk(args):
    name, lo, hi = args
    sys.path.insert(0, ROOT)
    import oracle.pf_oracle as O
    from synthgrid import configs
    g = configs.grid(name)
    sc = configs.scenarios(name, g=g)
    Y = O.build_ybus(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap)
    conv = 0
    for s in range(lo, hi):
        r = O.nr_solve(Y, g.bus_type, sc.Pd[s], sc.Qd[s], sc.Pg[s], sc.Vset[s], 1e-8, 20)
        conv += r["status"] == 0
    return conv


def _oracle_results(args):
    """The oracle's full results on the listed scenarios of a workload (for the parity
    block of the bench line)."""
    name, idx = args
    sys.path.insert(0, ROOT)
    import oracle.pf_oracle as O
    from synthgrid import configs
    g = configs.grid(name)
    sc = configs.scenarios(name, max(idx) + 1, g)
    Y = O.build_ybus(g.n_bus, g.f, g.t, g.r, g.x, g.b, g.tap)
    out = {k: [] for k in ("Vm", "Va", "Pg", "Qg", "iters", "status")}
    for s in idx:
        r = O.nr_solve(Y, g.bus_type, sc.Pd[s], sc.Qd[s], sc.Pg[s], sc.Vset[s], 1e-8, 20)
        for k in out:
            out[k].append(r[k])
    return {k: np.asarray(v) for k, v in out.items()}


def sig(x, d=3):
    """x rounded to d significant digits (the bench line keeps its tail short)."""
    if x is None or not np.isfinite(x) or x == 0:
        return x
    return float(f"{x:.{d}g}")


def parity_stats(gpu: dict, orc: dict) -> dict:
    """Per-result error of a GPU form against the FP64 oracle on the same scenarios:
    n scenarios, flags equal, both converged, the iteration-count difference (GPU -
    oracle) as a histogram, and the largest |dVm| (dV, pu), |dtheta| (dth, rad) and
    max(|dPg|, |dQg|) (dPQ, pu) over the scenarios both sides solved."""
    st_g, st_o = np.asarray(gpu["status"]), np.asarray(orc["status"])
    both = (st_g == 0) & (st_o == 0)
    d_it = (np.asarray(gpu["iters"]) - np.asarray(orc["iters"]))[both]
    hist = {str(int(k)): int((d_it == k).sum()) for k in np.unique(d_it)}

    def mx(*keys):
        if not both.any():
            return None
        return sig(max(float(np.max(np.abs(np.asarray(gpu[k])[both] - np.asarray(orc[k])[both])))
                       for k in keys), 2)
    return {"n": int(st_g.shape[0]), "flags": int((st_g == st_o).sum()), "conv": int(both.sum()),
            "it": hist, "dV": mx("Vm"), "dth": mx("Va"), "dPQ": mx("Pg", "Qg")}


class OraclePool:
    """A spawn-started process pool (one BLAS thread per worker) running the oracle."""

    def __init__(self, n_sample_hint: int):
        cores = os.cpu_count() or 1
        self.procs = max(1, min(cores, n_sample_hint))
        for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[var] = "1"
        self.pool = mp.get_context("spawn").Pool(self.procs)
        self.pool.map(_oracle_chunk, [(WORKLOAD, 0, 1)] * self.procs)  # warm: imports, grid

    def rate(self, n_sample: int):
        """Converged solves/s on the first n_sample scenarios of the workload."""
        bounds = np.linspace(0, n_sample, self.procs + 1).astype(int)
        chunks = [(WORKLOAD, int(bounds[i]), int(bounds[i + 1])) for i in range(self.procs)]
        t0 = time.perf_counter()
        conv = sum(self.pool.map(_oracle_chunk, chunks))
        dt = time.perf_counter() - t0
        return conv / dt, dt, conv

    def results(self, name: str, idx):
        """The oracle's results on the scenarios idx of a workload, in idx order."""
        idx = [int(i) for i in idx]
        parts = [p.tolist() for p in np.array_split(np.asarray(idx), min(self.procs, len(idx)))
                 if len(p)]
        outs = self.pool.map(_oracle_results, [(name, p) for p in parts])
        return {k: np.concatenate([o[k] for o in outs]) for k in outs[0]}

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"pf_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        try:
            rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
        except Exception:
            rows = []
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = []
        for k, nm in enumerate(names):
            if any(r[5 + k].strip().lower().startswith("active") for r in rows if len(r) > 5 + k):
                reasons.append(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------- GPU leg
# FP64 refinement residuals evaluated per Newton step in the bench's mixed form (at most
# ir_steps = 2; the gate at ||F1|| <= 1e-2 and the forcing term leave about one): with
# this value the FP64 count below, 2.51e8 flop per launch on the 118-bus batch, matches
# ncu's executed DADD + DMUL + 2 DFMA count of one launch, 2.48e8 (the ncu summary of the
# headline kernel records both).
RESID_PER_STEP = 1.0


def alg_counts(info: dict, n_bus: int, iters: np.ndarray, ir_steps: int, precision: str,
               resid_per_step: float = RESID_PER_STEP):
    """Algorithmic FP64 / FP32 flops and HBM bytes of one pf_solve launch.

    Per Newton iteration of one scenario: the FP64 mismatch (complex SpMV, 8
    flop per Ybus entry, plus ~20 flop per bus for V, S and F), the Jacobian
    fill (~12 flop per 2x2 block; FP32 in the mixed form), the block LU (16 flop per Schur block
    update, ~24 per L-column scaling), the triangular solves (8 flop per stored
    block per sweep pair member), and per refinement residual a matrix-free FP64
    residual (another complex SpMV + ~30 flop per bus); `resid_per_step` of them per
    Newton step (the measured average), each followed at most by one more solve.  One
    final mismatch evaluation per scenario follows the last update.
    """
    nnzY, nnzb, nb = info["nnz_ybus"], info["nnzb_lu"], info["n_block"]
    schur, la = info["schur_block_ops"], nnzb - nb  # L entries scaled once each (half of off-diag)
    it = float(iters.sum())
    n_sc = iters.shape[0]
    mism = 8 * nnzY + 20 * n_bus
    fill = 12 * nnzb
    lu = 16 * schur + 24 * (la // 2) + 10 * nb
    solve = 8 * nnzb
    resid = 8 * nnzY + 30 * n_bus
    mixed = precision == "mixed"
    # the mixed form fills the Jacobian in FP32 (it feeds the FP32 factor)
    f64 = (it + n_sc) * mism + (it * min(ir_steps, resid_per_step) * resid if mixed else it * fill)
    fsolve = it * (lu + solve * (1 + (min(ir_steps, resid_per_step) if mixed else 0)))
    f32 = fsolve + it * fill if mixed else 0.0
    if not mixed:
        f64 += fsolve
    hbm = n_sc * (8 * 4 * n_bus + 8 * 4 * n_bus + 16 + 16 * n_bus + 16)
    return f64, f32, hbm


def rank_scenarios(workload, g, rank, world, batch=0):
    """This rank's scenarios.  One GPU solves the workload's batch (or its first `batch`
    scenarios); with N ranks, rank r solves the r-th of N equal batches drawn from one
    seeded stream, so every rank does the same amount of distinct work (weak scaling, no
    collective on the data path)."""
    from synthgrid import Scenarios, configs
    if world == 1:
        return configs.scenarios(workload, batch or None, g=g)
    n = batch or configs.CONFIGS[workload]["n_scen"]
    sc = configs.scenarios(workload, n * world, g)
    part = slice(rank * n, (rank + 1) * n)
    return Scenarios(Pd=sc.Pd[part].copy(), Qd=sc.Qd[part].copy(), Pg=sc.Pg[part].copy(),
                     Vset=sc.Vset[part].copy())


def over_ranks(world, dev, total_ms, count):
    """(the slowest rank's timed total in ms, the sum of a count over the ranks): the
    job's time is the max over ranks, its work the units every rank processed."""
    if world == 1:
        return total_ms, count
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([float(count)], dtype=torch.float64, device=dev)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(c.item()))


def gpu_leg(args, rank, world):
    import torch
    import torch.distributed as dist

    from paper_2606_07099_gb300.powerflow import PowerFlow, SolveResult
    from synthgrid import configs

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    g = configs.grid(args.workload)
    sc = rank_scenarios(args.workload, g, rank, world, args.batch)
    N, nb = sc.n, g.n_bus
    pf = PowerFlow.from_grid(g)
    info = pf.info()
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (sc.Pd, sc.Qd, sc.Pg, sc.Vset)]
    Pd, Qd, Pg, Vset = [h.to(dev) for h in host]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed(fn, steps, warmup, name):
        for _ in range(warmup):
            fn()
        barrier()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        torch.cuda.nvtx.range_push(f"timed_{name}")  # lets a profiler select the timed steps
        for e0, e1 in evs:
            flush.fill_(1)  # evict the previous step's data from L2 (outside the timed events)
            e0.record(stream)
            fn()
            e1.record(stream)
        torch.cuda.nvtx.range_pop()
        barrier()
        return [e0.elapsed_time(e1) for e0, e1 in evs]

    opts = dict(precision="mixed", ir_steps=args.ir_steps, ir_rtol=args.ir_rtol, ir_gate=args.ir_gate)
    secs = set(args.sections.split(","))
    tuned = {}
    from paper_2606_07099_gb300.powerflow import autotune_schedule
    # the largest workspace any section needs, allocated once (captured graphs keep its address)
    pf.workspace(N, pf.make_opts("fp64", keep_factors=True, placement=3))
    pfh = pf  # the headline solve's network plan (the default one unless tuned)
    if args.plan:  # an explicit plan schedule for the headline solve (no schedule tuning)
        plan = {k: int(v) for k, v in (kv.split("=") for kv in args.plan.split(","))}
        pfh = PowerFlow.from_grid(g, plan)
    hopts = dict(opts)  # the headline solve's options
    if args.shape:  # an explicit launch shape for the headline solve (no tuning for it)
        pl, th, pk, cl = (int(v) for v in args.shape.split(","))
        hopts.update(placement=pl, group_threads=th, pack=pk, cluster=cl)
        tuned["mixed"] = {"group_threads": th, "placement": pl, "instances_per_cta": 1,
                          "pack": pk, "cluster": cl, "fixed": True, "schedule": pfh.plan}
        if args.autotune and "fp64" in secs:
            tuned["fp64"] = pf.autotune(Pd, Qd, Pg, Vset, precision="fp64")
    elif args.autotune and args.plan:  # the launch shape of the given plan
        tuned["mixed"] = {**pfh.autotune(Pd, Qd, Pg, Vset, **opts), "schedule": pfh.plan}
        tuned["mixed_default_plan"] = pf.autotune(Pd, Qd, Pg, Vset, **opts)
        if "fp64" in secs:
            tuned["fp64"] = pf.autotune(Pd, Qd, Pg, Vset, precision="fp64")
    elif args.autotune:  # plan schedule and launch shape, picked on these inputs (setup)
        # the headline's mixed solve: the default plan against top regions on this network
        # (a small network gets none by default); the other sections keep the default plan
        pfh, rep = autotune_schedule(g, Pd, Qd, Pg, Vset, schedules=HEADLINE_SCHEDULES, **opts)
        tuned["mixed"] = {**rep["shape"], "schedule": rep["schedule"], "trials": rep["trials"]}
        if pfh is not pf:
            pfh.workspace(N, pfh.make_opts("mixed", keep_factors=False, placement=3))
        # the default plan's own shapes (the per-scenario ones serve kept factors, reactive
        # limits and the host-buffer solve)
        tuned["mixed_default_plan"] = pf.autotune(Pd, Qd, Pg, Vset, **opts)
        if "fp64" in secs:
            tuned["fp64"] = pf.autotune(Pd, Qd, Pg, Vset, precision="fp64")
    info = pfh.info()

    def graphed(fn):
        """Record one step into a CUDA graph (the whole Newton loop is one kernel)."""
        fn()
        torch.cuda.synchronize(dev)
        if not args.graph:
            return fn
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr):
            fn()
        return gr.replay

    res = pfh.solve(Pd, Qd, Pg, Vset, **hopts)
    mixed_fn = graphed(lambda: pfh.solve(Pd, Qd, Pg, Vset, out=res, **hopts))
    if "fp64" in secs:
        res64 = pf.solve(Pd, Qd, Pg, Vset, precision="fp64")
        fp64_fn = graphed(lambda: pf.solve(Pd, Qd, Pg, Vset, precision="fp64", out=res64))

    # forward + backward of the implicit layer with the config-2 style loss cotangents
    slack = torch.as_tensor(g.bus_type == 2, device=dev)

    def make_fwd_bwd(pfx, inputs, slack_mask, resx):
        def step():
            r = pfx.solve(*inputs, keep_factors=True, out=resx, **opts)
            Vm = r.Vm
            dVm = 2 * torch.relu(Vm - 1.06) - 2 * torch.relu(0.94 - Vm)
            dPg = 2 * r.Pg * slack_mask
            pfx.adjoint(dVm, torch.zeros_like(Vm), dPg, None)
        return step

    if "fwdbwd" in secs:
        resk = pf.solve(Pd, Qd, Pg, Vset, keep_factors=True, **opts)
        fwd_bwd = graphed(make_fwd_bwd(pf, (Pd, Qd, Pg, Vset), slack, resk))
    if "layer_c2" in secs:  # the implicit layer on the 1354-bus workload, batch 1024
        g2 = configs.grid("c2")
        sc2 = configs.scenarios("c2", g=g2)
        pf2 = PowerFlow.from_grid(g2)
        in2 = [torch.as_tensor(np.ascontiguousarray(a), device=dev) for a in (sc2.Pd, sc2.Qd, sc2.Pg, sc2.Vset)]
        pf2.workspace(sc2.n, pf2.make_opts("fp64", keep_factors=True, placement=3))
        if args.autotune:
            tuned["layer_c2"] = pf2.autotune(*in2, keep_factors=True, **opts)
        res2 = pf2.solve(*in2, keep_factors=True, **opts)
        fb2 = graphed(make_fwd_bwd(pf2, in2, torch.as_tensor(g2.bus_type == 2, device=dev), res2))

    if "multi_c4" in secs:  # uneven batch: 30/300/2000-bus networks in one persistent launch
        from paper_2606_07099_gb300.powerflow import solve_multi
        grids4, inputs4, slacks4 = [], [], []
        for name in ("c4a", "c4b", "c4c"):
            g4 = configs.grid(name)
            sc4 = configs.scenarios(name, g=g4)
            grids4.append(g4)
            inputs4.append([torch.as_tensor(np.ascontiguousarray(a), device=dev)
                            for a in (sc4.Pd, sc4.Qd, sc4.Pg, sc4.Vset)])
            slacks4.append(torch.as_tensor(g4.bus_type == 2, device=dev))
        # each network's plan schedule and the single launch's shape (pf_autotune_multi:
        # threads per CTA x per-network forms or all-global placement), on these inputs
        # (setup, not timed)
        from paper_2606_07099_gb300.powerflow import (autotune_multi_schedule,
                                                      multi_workspace_bytes)
        if args.autotune:
            pfs4, rep4 = autotune_multi_schedule(grids4, inputs4, keep_factors=True, **opts)
            tuned["multi_c4"] = {**rep4["shape"], "schedules": rep4["schedules"]}
        else:
            pfs4 = [PowerFlow.from_grid(g4) for g4 in grids4]
            tuned["multi_c4"] = {"group_threads": 256, "placement": 0}
        items4 = [(p4, *in4) for p4, in4 in zip(pfs4, inputs4)]
        n4 = sum(it[1].shape[0] for it in items4)
        shape4 = dict(group_threads=tuned["multi_c4"]["group_threads"],
                      placement=tuned["multi_c4"]["placement"])
        # preallocated results, gradients and workspace: the captured steps allocate nothing
        ws4 = torch.empty(multi_workspace_bytes(items4, PowerFlow.make_opts(
            keep_factors=True, **shape4, **opts))[0], dtype=torch.uint8, device=dev)
        res4 = solve_multi(items4, keep_factors=True, workspace=ws4, **shape4, **opts)
        cts4 = []
        for (pfx, *_), r, sl in zip(items4, res4, slacks4):
            dVm = 2 * torch.relu(r.Vm - 1.06) - 2 * torch.relu(0.94 - r.Vm)
            cts4.append((dVm, torch.zeros_like(r.Vm), 2 * r.Pg * sl))
        grads4 = [pfx.adjoint(*ct, None) for (pfx, *_), ct in zip(items4, cts4)]

        def multi_fwd_step():
            solve_multi(items4, workspace=ws4, out=res4, **shape4, **opts)

        def multi_fwd_bwd_step():
            rs = solve_multi(items4, keep_factors=True, workspace=ws4, out=res4, **shape4, **opts)
            for (pfx, *_), r, sl, (dVm, dVa, dPg), gr in zip(items4, rs, slacks4, cts4, grads4):
                torch.sub(2 * torch.relu(r.Vm - 1.06), 2 * torch.relu(0.94 - r.Vm), out=dVm)
                torch.mul(2 * r.Pg, sl, out=dPg)
                pfx.adjoint(dVm, dVa, dPg, None, out=gr)
        multi_fwd = graphed(multi_fwd_step)
        multi_fwd_bwd = graphed(multi_fwd_bwd_step)
    large = {}  # the grids whose factors stream through memory: 9241 and 25,000 buses
    for lname in ("c3", "c5"):
        if lname not in secs:
            continue
        gl = configs.grid(lname)
        scl = configs.scenarios(lname, g=gl)
        inl = [torch.as_tensor(np.ascontiguousarray(a), device=dev) for a in (scl.Pd, scl.Qd, scl.Pg, scl.Vset)]
        if args.autotune:  # plan schedule and launch shape, picked on these inputs
            pfl, rep = autotune_schedule(gl, *inl, **opts)
            tuned[lname] = {**rep["shape"], "schedule": rep["schedule"]}
        else:
            pfl = PowerFlow.from_grid(gl)
        # sized for the FP64 form too (the parity block solves it once, after the timing;
        # captured graphs keep this buffer's address)
        pfl.workspace(scl.n, pfl.make_opts("fp64", placement=3))
        resl = pfl.solve(*inl, **opts)
        # the tuple keeps the inputs alive: a captured graph holds only their addresses
        large[lname] = (gl, scl, pfl, resl,
                        graphed(lambda pfl=pfl, inl=inl, resl=resl: pfl.solve(*inl, out=resl, **opts)),
                        inl)

    if "qlim" in secs:  # reactive limits at a third of the PV buses (PV -> PQ switching)
        Qg0 = res.Qg[0].clone()
        pv = np.flatnonzero(g.bus_type == 1)
        pick = torch.as_tensor(np.random.default_rng(1).choice(pv, len(pv) // 3, replace=False),
                               device=dev)
        qmax_row = torch.full((nb,), 1e30, dtype=torch.float64, device=dev)
        qmin_row = torch.full((nb,), -1e30, dtype=torch.float64, device=dev)
        qmax_row[pick] = Qg0[pick] - 0.02
        qmin_row[pick] = Qg0[pick] - 1.0
        Qmax_b = qmax_row.expand(N, nb).contiguous()
        Qmin_b = qmin_row.expand(N, nb).contiguous()
        resq = [pf.solve_qlim(Pd, Qd, Pg, Vset, Qmin_b, Qmax_b, **opts)]
        qlim_fn = lambda: resq.__setitem__(0, pf.solve_qlim(Pd, Qd, Pg, Vset, Qmin_b, Qmax_b, **opts))

    if "jacobian" in secs:  # block-diagonal export of J1 (Alg. 1 values into the BDE template)
        jac_cases = []
        for jname, jn in (("c2", 64), ("c2", 1024), ("c3", 64)):
            gj = configs.grid(jname)
            pfj = PowerFlow.from_grid(gj)
            scj = configs.scenarios(jname, jn, gj)
            rj = pfj.solve(*[torch.as_tensor(np.ascontiguousarray(a), device=dev)
                             for a in (scj.Pd, scj.Qd, scj.Pg, scj.Vset)], precision="fp64")
            outj = pfj.export_jacobian(rj.Vm, rj.Va)
            jac_cases.append((jname, jn, gj, pfj, rj, outj))

    bde_cases = []
    if "bde" in secs:  # the same FP64 solve run as one block-diagonal matrix, phase by phase
        for bname in ("c1", "c2", "c3"):
            if bname == "c1":
                gb_, pfb_, inb_ = g, pf, [Pd, Qd, Pg, Vset]
            else:
                gb_ = configs.grid(bname)
                scb_ = configs.scenarios(bname, g=gb_)
                pfb_ = large[bname][2] if bname in large else PowerFlow.from_grid(gb_)
                inb_ = [torch.as_tensor(np.ascontiguousarray(a), device=dev)
                        for a in (scb_.Pd, scb_.Qd, scb_.Pg, scb_.Vset)]
            bde_cases.append((bname, gb_, pfb_, inb_))

    sweep_cases = []
    if "sweep" in secs:  # solve time vs batch size on the large grids (the shape of Table II)
        for sname, sizes in (("c1", (256, 1024, 2048, 4096)), ("c2", (4, 16, 64, 256, 1024)),
                             ("c3", (4, 16, 64, 256)), ("c5", (4, 16, 64, 256))):
            if sname == "c1":  # the headline network, on a handle of its own (the sweep
                # retunes the launch shape at every batch size)
                gs_, scs_, pfs_ = g, sc, PowerFlow.from_grid(g)
            elif sname in large:
                gs_, scs_, pfs_ = large[sname][0], large[sname][1], large[sname][2]
            else:
                gs_ = configs.grid(sname)
                scs_ = configs.scenarios(sname, max(sizes), gs_)
                pfs_ = PowerFlow.from_grid(gs_)
            ins_ = [torch.as_tensor(np.ascontiguousarray(a[:max(sizes)]), device=dev)
                    for a in (scs_.Pd, scs_.Qd, scs_.Pg, scs_.Vset)]
            if sname not in large and sname != "c1":  # (captured graphs hold the others')
                pfs_.workspace(max(sizes), pfs_.make_opts("fp64", placement=3))
            if args.autotune and sname not in large and sname != "c1":
                tuned[sname] = pfs_.autotune(*ins_, **opts)
            sweep_cases.append((sname, gs_, pfs_, ins_, sizes))

    if "train" in secs:  # the layer inside a DC3-style training loop (network -> PF -> loss)
        from paper_2606_07099_gb300 import embedded as em
        from synthgrid import make_opf_limits
        train_sets = []
        for tname, batches in (("c1", (256, 1024, 4096)), ("c2", (64, 256, 1024))):
            gt = configs.grid(tname)
            sct = configs.scenarios(tname, 2 * max(batches), gt)
            pft = PowerFlow.from_grid(gt)
            ldt = [torch.as_tensor(np.ascontiguousarray(a), device=dev) for a in (sct.Pd, sct.Qd)]
            pft.workspace(max(batches), pft.make_opts("fp64", keep_factors=True, placement=3))
            if args.autotune:  # launch shape of the layer's solve (setup, not timed)
                tuned[f"train_{tname}"] = pft.autotune(
                    ldt[0][:max(batches)], ldt[1][:max(batches)],
                    torch.as_tensor(sct.Pg[:max(batches)], device=dev),
                    torch.as_tensor(sct.Vset[:max(batches)], device=dev), keep_factors=True, **opts)
            train_sets.append((tname, gt, pft, ldt, batches, make_opf_limits(gt, 11)))

    def train_run(gt, pft, ldt, B, lim, steps, warmup, graph):
        torch.manual_seed(0)
        base_mem = torch.cuda.memory_allocated(dev)
        torch.cuda.reset_peak_memory_stats(dev)
        model = em.EmbeddedPF(pft, gt.bus_type, gt.Pd0, gt.Qd0, lim, hidden=256,
                              ir_steps=args.ir_steps, ir_rtol=args.ir_rtol,
                              ir_gate=args.ir_gate).to(dev)
        optim = torch.optim.Adam(model.net.parameters(), lr=1e-3, capturable=graph)
        nbt = ldt[0].shape[0] // B
        Pdb = ldt[0][:nbt * B].view(nbt, B, -1)
        Qdb = ldt[1][:nbt * B].view(nbt, B, -1)
        stats = []
        it = [0]
        if graph:
            trainer = em.GraphedTrainer(model, optim, Pdb[0], Qdb[0])
            one = trainer.step
        else:
            one = lambda Pd_, Qd_: em.train_step(model, optim, Pd_, Qd_)

        def step():
            k = it[0] % nbt
            it[0] += 1
            L_, n_ = one(Pdb[k], Qdb[k])
            stats.append((L_.clone(), n_.clone()))
        t_host = time.perf_counter()
        ts = timed(step, steps, warmup, f"train_{gt.name}_{B}{'_graph' if graph else ''}")
        t_host = (time.perf_counter() - t_host) / (steps + warmup)
        loss = torch.stack([x[0] for x in stats]).cpu().numpy()
        n_ok = torch.stack([x[1] for x in stats]).cpu().numpy()
        peak = torch.cuda.max_memory_allocated(dev) - base_mem
        return {"batch": B, "graph": graph, "samples_per_s": world * B * steps / (agg(ts) / 1e3),
                "ms_per_step": agg(ts) / steps, "host_ms_per_step": 1e3 * t_host,
                "converged_frac": float(n_ok.sum() / (B * len(n_ok))),
                "loss_first": float(loss[0]), "loss_last": float(loss[-1]),
                "peak_train_mem_mb": peak / 2**20, "train_mem_mb_per_sample": peak / 2**20 / B}

    def agg(ts):
        tot = sum(ts)
        if world > 1:
            t = torch.tensor([tot], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            tot = float(t.item())
        return tot

    # end to end through the C ABI with host buffers (pf_solve_host): every step the solve
    # kernel reads the step's four input arrays from page-locked host memory and writes
    # Vm, Va and the status flags back there, in place (over NVLink-C2C on GB300); the
    # step ends when the stream has finished, with the results in host memory
    host_in = torch.stack(host).pin_memory()
    host_views = [host_in[k] for k in range(4)]
    out_host = torch.empty(2, N, nb, dtype=torch.float64).pin_memory()
    st_host = torch.empty(N, dtype=torch.int32).pin_memory()
    rese = SolveResult(Vm=out_host[0], Va=out_host[1], Pg=None, Qg=None, iters=None,
                       status=st_host, final_mismatch=None)

    # two ways through the public API, the faster kept (setup, not timed): the default
    # plan's per-scenario kernels (what pf_solve_host picks by itself), and the headline's
    # plan and interleaved shape given explicitly
    e2e_ways = {"per_scenario": (pf, dict(opts))}
    tm = tuned.get("mixed", {})
    if tm.get("placement") == 5:
        e2e_ways["interleaved"] = (pfh, dict(opts, placement=5, pack=tm["pack"],
                                             cluster=tm["cluster"],
                                             group_threads=tm["group_threads"]))
    e2e_ms = {}
    for wname, (pfx, kw) in e2e_ways.items():
        pfx.solve_host(*host_views, out=rese, **kw)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(3):
            pfx.solve_host(*host_views, out=rese, **kw)
        torch.cuda.synchronize(dev)
        e2e_ms[wname] = (time.perf_counter() - t0) / 3 * 1e3
    e2e_way = min(e2e_ms, key=e2e_ms.get)
    e2e_pf, e2e_kw = e2e_ways[e2e_way]

    def e2e():
        e2e_pf.solve_host(*host_views, out=rese, **e2e_kw)

    none = [float("nan")]
    with ClockSampler(dev.index) as clk:
        t_mixed = timed(mixed_fn, args.steps, args.warmup, "mixed")
        t_fp64 = timed(fp64_fn, args.steps, args.warmup, "fp64") if "fp64" in secs else none
        t_fb = timed(fwd_bwd, args.steps, args.warmup, "fwdbwd") if "fwdbwd" in secs else none
        t_fb2 = timed(fb2, args.steps, args.warmup, "layer_c2") if "layer_c2" in secs else none
        t_e2e = timed(e2e, args.steps, args.warmup, "e2e") if "e2e" in secs else none
        t_m4 = timed(multi_fwd, args.steps, args.warmup, "multi_c4") if "multi_c4" in secs else none
        t_m4b = (timed(multi_fwd_bwd, args.steps, args.warmup, "multi_c4_fb")
                 if "multi_c4" in secs else none)
        t_large = {k: timed(v[4], args.steps, args.warmup, k) for k, v in large.items()}
        t_qlim = timed(qlim_fn, args.steps, args.warmup, "qlim") if "qlim" in secs else none
        t_jac = [timed(lambda c=c: c[3].export_jacobian(c[4].Vm, c[4].Va, out=c[5]), args.steps,
                       args.warmup, f"jacobian_{c[0]}_{c[1]}")
                 for c in (jac_cases if "jacobian" in secs else [])]
        bde_out = {}
        for bname, gb_, pfb_, inb_ in bde_cases:
            rb_ = pfb_.solve_bde(*inb_)
            tb_ = timed(lambda: pfb_.solve_bde(*inb_, out=rb_), 5, 3, f"bde_{bname}")
            rf_ = pfb_.solve(*inb_, precision="fp64")
            tf_ = timed(lambda: pfb_.solve(*inb_, precision="fp64", out=rf_), 5, 3, f"bde_fused_{bname}")
            bde_out[bname] = {
                "n_bus": gb_.n_bus, "batch": int(inb_[0].shape[0]),
                "one_big_matrix_ms": statistics.median(tb_), "fused_fp64_ms": statistics.median(tf_),
                "fused_speedup": statistics.median(tb_) / statistics.median(tf_),
                "converged": [int((rb_.status == 0).sum().item()), int((rf_.status == 0).sum().item())],
                "iters_max": [int(rb_.iters.max().item()), int(rf_.iters.max().item())]}
        sweep_out = {}
        for sname, gs_, pfs_, ins_, sizes in sweep_cases:
            rows_ = []
            for n_ in sizes:
                sub = [t[:n_] for t in ins_]
                for prec_ in (("mixed", "fp64") if n_ == 64 else ("mixed",)):
                    o_ = dict(opts, precision=prec_)
                    # launch shape for this batch size (a few scenarios of a large grid
                    # want more threads each than a full batch does); setup, not timed
                    shape_ = pfs_.autotune(*sub, **o_) if args.autotune else None
                    r_ = pfs_.solve(*sub, **o_)
                    tn = timed(lambda: pfs_.solve(*sub, out=r_, **o_), 5, 3, f"sweep_{sname}_{n_}_{prec_}")
                    ms_ = statistics.median(tn)
                    rows_.append({"batch": n_, "precision": prec_, "ms": ms_, "shape": shape_,
                                  "solves_per_s": n_ / (ms_ / 1e3),
                                  "iters": [int(r_.iters.min().item()), int(r_.iters.max().item())],
                                  "converged": int((r_.status == 0).sum().item()),
                                  "max_final_mismatch": float(r_.final_mismatch.max().item())})
            sweep_out[sname] = {"n_bus": gs_.n_bus, "rows": rows_}
        train_out = {}
        if "train" in secs:
            ksteps = max(5, min(args.steps, 20))
            for tname, gt, pft, ldt, batches, lim in train_sets:
                train_out[tname] = [train_run(gt, pft, ldt, B, lim, ksteps, max(3, args.warmup), gr)
                                    for B in batches for gr in (True, False)]
        # the ALU roofline's denominators, measured on this GPU at these clocks (best of 3)
        from paper_2606_07099_gb300 import _lib as pflib
        peak64 = max(pflib.measure_fma_peak(True, 1 << 14, stream.cuda_stream) for _ in range(3))
        peak32 = max(pflib.measure_fma_peak(False, 1 << 19, stream.cuda_stream) for _ in range(3))
    clocks = clk.summary()
    torch.cuda.synchronize(dev)
    st = res.status.cpu().numpy()
    its = res.iters.cpu().numpy()
    conv = int((st == 0).sum())
    conv64 = int((res64.status.cpu().numpy() == 0).sum()) if "fp64" in secs else 0
    conve = int((rese.status.cpu().numpy() == 0).sum()) if "e2e" in secs else 0
    fmax = float(res.final_mismatch.max().item())

    T_mixed, T_fp64, T_fb, T_fb2, T_e2e, T_m4, T_m4b = (
        agg(t) for t in (t_mixed, t_fp64, t_fb, t_fb2, t_e2e, t_m4, t_m4b))
    K = args.steps
    extra = {}
    if "multi_c4" in secs:
        conv4 = sum(int((r.status == 0).sum().item()) for r in res4)
        extra["multi_c4"] = {
            "workload": "2048 x 30-bus + 512 x 300-bus + 64 x 2000-bus scenarios, loads x U(0.6, 1.4), "
                        "one persistent launch (pf_solve_multi; fwd+bwd adds the three adjoints), "
                        "CUDA-graph replay on preallocated buffers", "scenarios": n4, "converged": conv4,
            "solves_per_s": world * conv4 * K / (T_m4 / 1e3), "ms_per_step": T_m4 / K,
            "fwd_bwd_per_s": world * n4 * K / (T_m4b / 1e3), "fwd_bwd_ms_per_step": T_m4b / K}
    for lname, (gl, scl, pfl, resl, _, _) in large.items():
        Tl = agg(t_large[lname])
        convl = int((resl.status == 0).sum().item())
        # factor traffic per Newton iteration and scenario: written by the fill, read and
        # written once by the LU (every block is a Schur target or an L/U operand at least
        # once), read by each triangular solve pair
        fac_b = 16 * pfl.info()["nnzb_lu"]
        itl = float(resl.iters.sum().item())
        bytesl = itl * fac_b * (1 + 2 + 2) + scl.n * (8 * 8 * gl.n_bus)
        extra[lname] = {"workload": f"{gl.n_bus}-bus grid, {scl.n} scenarios, mixed",
                        "converged": convl, "mean_iters": itl / scl.n,
                        "solves_per_s": world * convl * K / (Tl / 1e3), "ms_per_step": Tl / K,
                        "hbm_algorithmic_gbs": bytesl / (Tl / K / 1e3) / 1e9,
                        "hbm_frac": bytesl / (Tl / K / 1e3) / 1e9 / hbm_peak()[0],
                        "traffic_per_launch": profiled_traffic(f"nr_solve_{lname}_mixed.json")}
    if "qlim" in secs:
        Tq = agg(t_qlim)
        rq = resq[0]
        convq = int((rq.status == 0).sum().item())
        extra["qlim"] = {
            "workload": "the headline batch with reactive limits just below the unlimited "
                        "output at a third of the PV buses (PV -> PQ switching, pf_solve_qlim)",
            "converged": convq, "solves_per_s": world * convq * K / (Tq / 1e3),
            "ms_per_step": Tq / K, "mean_rounds": float(rq.rounds.double().mean().item()),
            "mean_iters": float(rq.iters.double().mean().item()),
            "switched_buses_per_scenario": float(((rq.bus_type == 0).sum(1).double()
                                                  - int((g.bus_type == 0).sum())).mean().item())}
    if "jacobian" in secs:
        rows = []
        for (jname, jn, gj, pfj, rj, outj), tj in zip(jac_cases, t_jac):
            ms = agg(tj) / K
            info_j = pfj.info()
            byts = jn * (8 * info_j["nnz_j1"] + 16 * gj.n_bus)  # values written, V read
            rows.append({"workload": f"{gj.n_bus}-bus grid, {jn} scenarios", "ms": ms,
                         "values_per_s": jn * info_j["nnz_j1"] / (ms / 1e3),
                         "hbm_gbs": byts / (ms / 1e3) / 1e9,
                         "hbm_frac": byts / (ms / 1e3) / 1e9 / hbm_peak()[0]})
        extra["jacobian_export"] = {
            "what": "pf_export_jacobian: J1 values of every scenario at its solution, written "
                    "in FP64 into the fixed block-diagonal (BDE) template",
            "cases": rows}
    if "bde" in secs and "c1" in bde_out and "fp64" in secs:
        # the mixed form against the faster of the two FP64 executions of the same solve
        best64 = min(T_fp64 / K, bde_out["c1"]["one_big_matrix_ms"])
        extra_fp64 = {"best_fp64_ms": best64, "mixed_speedup_vs_best_fp64": best64 / (T_mixed / K)}
    else:
        extra_fp64 = {}
    if "bde" in secs:
        extra["one_big_matrix"] = {
            "what": "FP64 solve as one block-diagonal matrix (pf_solve_bde: batch-wide kernels "
                    "per phase and elimination level, host convergence check per iteration) "
                    "against the fused one-launch FP64 solve on the same plan; median of 5",
            **bde_out}
    if "sweep" in secs:
        extra["batch_sweep"] = {
            "what": "one pf_solve per batch size (launch shape autotuned at that size, except "
                    "the headline network, tuned on its full batch), median of 5 CUDA-event "
                    "runs, L2 flushed before each; iters = [min, max]",
            **sweep_out}
    if "memory" in secs:  # device bytes: the shared plan plus a fixed slot per scenario
        mem = {}
        for mname in ("c0", "c1", "c2", "c3", "c5"):
            gm = configs.grid(mname)
            pfm_ = PowerFlow.from_grid(gm)
            per = {}
            for prec in ("mixed", "fp64"):
                for keep in (False, True):
                    o_ = pfm_.make_opts(prec, keep_factors=keep, placement=3)
                    b1, b2 = pfm_.workspace_bytes(1, o_), pfm_.workspace_bytes(1024, o_)
                    assert b2 == 1024 * b1  # linear in the batch, no per-batch term
                    per[f"{prec}{'_keep' if keep else ''}"] = b1
            mem[mname] = {"n_bus": gm.n_bus, "plan_bytes": pfm_.info()["plan_bytes"],
                          "workspace_bytes_per_scenario": per}
            pfm_.close()
        extra["memory"] = {"note": "workspace = batch x slot (global placement), plan shared by "
                                   "all scenarios; keep = factors kept for the adjoint",
                           "grids": mem}
    if "train" in secs:
        extra["train"] = {
            "workload": ("DC3-style learning loop: MLP (2 x 256, ReLU, FP32) from loads to "
                         "[pg_G; Vm_B\\D], PF layer (mixed, fwd + implicit bwd), loss = cost + "
                         "100 x squared limit violations, Adam 1e-3; batches cycle through "
                         "2 x max-batch synthetic load scenarios; graph: the whole step "
                         "(forward, implicit backward, optimiser) replayed from one CUDA graph, "
                         "else eager PyTorch around the libpf calls"),
            "unit": "samples/s", **train_out}
    # GPU results for the parity block (per-result error against the oracle, computed on
    # the host after the timing): the headline batch in both forms, and samples of the
    # other workloads (their FP64 forms solved once here, untimed)
    def arrays(r, idx=None):
        sel = slice(None) if idx is None else torch.as_tensor(idx, device=dev)
        return {k: getattr(r, k)[sel].cpu().numpy()
                for k in ("Vm", "Va", "Pg", "Qg", "iters", "status")}
    par_in = {}
    if world == 1:
        par_in[args.workload] = {"idx": list(range(N)), "mixed": arrays(res)}
        if "fp64" in secs:
            par_in[args.workload]["fp64"] = arrays(res64)
        samples = {"c2": 32, "c3": 16, "c5": 8}
        for pname, (pfx, inx, rx) in (
                [("c2", (pf2, in2, res2))] if "layer_c2" in secs else []) + [
                (k, (v[2], v[5], v[3])) for k, v in large.items()]:
            idx = np.linspace(0, inx[0].shape[0] - 1, samples[pname]).astype(int).tolist()
            r64 = pfx.solve(*inx, precision="fp64")
            par_in[pname] = {"idx": idx, "mixed": arrays(rx, idx), "fp64": arrays(r64, idx)}
        if "multi_c4" in secs:
            for (pfx, *inx), rx, name4 in zip(items4, res4, ("c4a", "c4b", "c4c")):
                idx = np.linspace(0, inx[0].shape[0] - 1, 16).astype(int).tolist()
                par_in[name4] = {"idx": idx, "mixed": arrays(rx, idx)}
        torch.cuda.synchronize(dev)

    T_job, conv_job = over_ranks(world, dev, sum(t_mixed), conv)
    value = conv_job * K / (T_job / 1e3)
    ms_launch = statistics.mean(t_mixed)
    f64, f32, hbm_bytes = alg_counts(info, nb, its, args.ir_steps, "mixed")
    hbm_peak_gbs, hbm_src = hbm_peak()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": T_mixed / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC if args.workload == WORKLOAD
                   else f"synthgrid workload {args.workload}", "n_bus": nb, "batch_per_gpu": N,
                   "global_batch": N * world, "precision": "mixed (FP32 LU + FP64 mismatch/refinement)",
                   "ir_steps": args.ir_steps, "ir_rtol": args.ir_rtol, "ir_gate": args.ir_gate,
                   "launch": "CUDA-graph replay of one pf_solve" if args.graph else "direct",
                   "tuned": tuned,
                   "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MB write)",
                   "parallelism": f"replicas x{world} (scenarios sharded, no collective)"},
        "converged": conv, "max_final_mismatch": fmax, "mean_iters": float(its.mean()),
        "fp64_form": {"value": world * conv64 * K / (T_fp64 / 1e3), "unit": UNIT,
                      "ms_per_step": T_fp64 / K, "mixed_speedup": T_fp64 / T_mixed, **extra_fp64},
        "fwd_bwd": {"value": world * N * K / (T_fb / 1e3), "unit": "fwd+bwd/s",
                    "ms_per_step": T_fb / K},
        "fwd_bwd_c2": {"value": world * 1024 * K / (T_fb2 / 1e3), "unit": "fwd+bwd/s",
                       "ms_per_step": T_fb2 / K,
                       "workload": "1354-bus grid, 1024 scenarios, config-2 loss cotangents"},
        "e2e": {"value": over_ranks(world, dev, 0.0, conve)[1] * K / (T_e2e / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": 4 * N * nb * 8, "d2h_bytes_per_step": 2 * N * nb * 8 + 4 * N,
                "api": "pf_solve_host: the solve kernel reads the inputs from and writes Vm, Va "
                       "and status to page-locked host memory in place",
                "kernel": e2e_way, "setup_ms": e2e_ms},
        "gpu_launches": K,
        "roofline": {"bound": "alu", "achieved": f64 / (ms_launch / 1e3) / 1e12, "peak": peak64,
                     "unit": "TFLOP/s", "frac": f64 / (ms_launch / 1e3) / 1e12 / peak64,
                     "traffic": (profiled_traffic(headline_kernel(tuned.get("mixed"))[1])
                                 if args.workload == WORKLOAD else None),
                     "kernel": headline_kernel(tuned.get("mixed"))[0],
                     "note": ("FP64 pipe: achieved = algorithmic FP64 flops per launch / mean "
                              "launch time; peak = FP64 FMA rate measured in this run "
                              "(pf_measure_fma_peak, of measured); the FP32 work's share of its "
                              "own measured peak is f32_frac"),
                     "flops_f64": f64, "flops_f32": f32,
                     "f32_frac": f32 / (ms_launch / 1e3) / 1e12 / peak32,
                     "peak_fp32": peak32,
                     "nominal": {"fp64": FP64_NOMINAL_TFLOPS, "fp32": FP32_NOMINAL_TFLOPS}},
        "hbm": {"achieved_gbs": hbm_bytes / (ms_launch / 1e3) / 1e9, "peak_gbs": hbm_peak_gbs,
                "peak_source": hbm_src, "frac": hbm_bytes / (ms_launch / 1e3) / 1e9 / hbm_peak_gbs,
                "bytes_per_launch": hbm_bytes},
        "clocks": clocks,
        **extra,
    }
    # the compact summary the tail of the line carries (3 significant digits)
    summ = {"mixed_ms": sig(T_mixed / K)}
    if "fp64" in secs:
        summ.update(fp64_ms=sig(T_fp64 / K), mixed_speedup=sig(T_fp64 / T_mixed))
    if "fwdbwd" in secs:
        summ["fwd_bwd_per_s"] = sig(line["fwd_bwd"]["value"])
    if "layer_c2" in secs:
        summ["c2_fwd_bwd_per_s"] = sig(line["fwd_bwd_c2"]["value"])
    for key in ("multi_c4", "c3", "c5", "qlim"):
        if key in extra:
            e = extra[key]
            summ[key] = {k: sig(e[k]) for k in ("ms_per_step", "solves_per_s", "fwd_bwd_per_s",
                                                 "fwd_bwd_ms_per_step", "hbm_frac") if k in e}
    line["results"] = summ
    return line, par_in


# keys printed last: the driver's record keeps only the tail of the line, so the
# compact results, the parity block, the roofline and the baselines go there
TAIL_KEYS = ("results", "parity", "roofline", "e2e", "gpu_launches", "clocks", "cpu_baseline")


def ordered(line: dict) -> dict:
    """The bench line with the bulky sections first and the compact summary last."""
    head = {k: v for k, v in line.items() if k not in TAIL_KEYS}
    head.update({k: line[k] for k in TAIL_KEYS if k in line})
    return head


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--ir-steps", type=int, default=2)
    ap.add_argument("--ir-rtol", type=float, default=1e-3,
                    help="refine while the FP64 residual exceeds this fraction of ||F1||")
    ap.add_argument("--ir-gate", type=float, default=1e-2,
                    help="check/refine Newton steps only once ||F1||_inf <= this (0 = all)")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--shape", default="",
                    help="placement,threads,pack,cluster of the headline solve instead of the "
                         "autotuned one (e.g. 3,32,0,0: per-scenario, 32 threads, global)")
    ap.add_argument("--plan", default="",
                    help="key=value,... plan schedule of the headline solve instead of the "
                         "tuned one (e.g. order_slack=1,top_rows=5,top_min_pivots=0)")
    ap.add_argument("--no-graph", dest="graph", action="store_false")
    ap.add_argument("--cpu-sample", type=int, default=4096,
                    help="scenarios the CPU oracle solves for cpu_baseline (0 = skip)")
    ap.add_argument("--sections", default="mixed,fp64,fwdbwd,layer_c2,e2e,multi_c4,c3,c5,qlim,jacobian,memory,bde,sweep,train",
                    help="timed sections to run (the first one, mixed, always runs)")
    ap.add_argument("--workload", default="c1", help="synthgrid workload (c1 is the bench line)")
    ap.add_argument("--batch", type=int, default=0,
                    help="scenarios per GPU for the headline section (0 = the workload's batch)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        # the CPU oracle on a bounded sample of the workload, per step
        per_step = max(64, args.cpu_sample // 4)
        pool = OraclePool(per_step)
        procs = pool.procs
        for _ in range(args.warmup):
            pool.rate(per_step)
        rates = [pool.rate(per_step)[0] for _ in range(args.steps)]
        pool.close()
        v = statistics.median(rates)
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "ms_per_step": 1e3 * per_step / v, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "n_bus": 118, "batch_per_step": per_step},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": f"first {per_step} of the 4096 scenarios per step",
                             "cpu": cpu_model()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }), flush=True)
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    line, par_in = gpu_leg(args, rank, world)
    if rank == 0:
        if args.cpu_sample > 0:
            # the oracle on the host cores: the first cpu_sample scenarios of the headline
            # batch (timed: cpu_baseline), whose results also give the per-result error of
            # both GPU forms; then samples of the other workloads for the same comparison
            n_c = min(args.cpu_sample, line["config"]["batch_per_gpu"])
            pool = OraclePool(n_c)
            try:
                t0 = time.perf_counter()
                orc = pool.results(args.workload, range(n_c))
                dt = time.perf_counter() - t0
                conv = int((orc["status"] == 0).sum())
                parity = {}
                for pname, d in par_in.items():
                    o = orc if pname == args.workload else pool.results(pname, d["idx"])
                    n_p = len(o["status"])
                    parity[pname] = {form: parity_stats({k: v[:n_p] for k, v in d[form].items()}, o)
                                     for form in ("mixed", "fp64") if form in d}
            finally:
                pool.close()
            one = mp.get_context("spawn").Pool(1)
            try:  # one core: the same oracle on a smaller sample
                n1 = min(256, n_c)
                one.map(_oracle_chunk, [(args.workload, 0, 1)])
                t1 = time.perf_counter()
                conv1 = one.map(_oracle_chunk, [(args.workload, 0, n1)])[0]
                dt1 = time.perf_counter() - t1
            finally:
                one.close()
                one.join()
            if par_in:
                line["parity"] = parity
            line["cpu_baseline"] = {"value": conv / dt, "unit": UNIT, "cores": pool.procs,
                                    "kind": "oracle", "single_core_value": conv1 / dt1,
                                    "sample": f"first {n_c} of the {line['config']['batch_per_gpu']} "
                                              f"scenarios ({dt:.1f} s "
                                              f"wall); single core: first {n1}",
                                    "cpu": cpu_model()}
        print(json.dumps(ordered(line)), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
