#!/usr/bin/env python
"""Benchmark of the DiffPower hot path on GB300.

One step = the whole hot path once on the roofline-scale synthetic netlist
(2,000,000 cells, 147,456 startpoints, depth 80, fanout cap 32):
forward SP/TR + model power, 4,096-vector Markov simulation with PopCount
toggles, hybrid beta + hybrid power, and the full adjoint (paper's beta rule),
with gradients w.r.t. input SP/TR, pin caps and net loads written out.

value = cells x ranks / (max over ranks of the device time per step) in
cell-evals/s; e2e = the same through the C-ABI with host (pinned) buffers,
host<->device copies included.  Multi-GPU runs are independent replicas.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd cell-evals/s vs HBM roofline; served p50/p99 latency vs plain loop"
UNIT = "cell-evals/s"
L2_FLUSH_BYTES = 256 << 20   # > 2x the 126 MB L2


def peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def fanin_bytes(nc: int, ne: int) -> int:
    """Compact fanin CSR: row pointers, fanin net ids, one opcode byte per cell."""
    return 4 * (nc + 1) + 4 * ne + nc


def fanout_bytes(nn: int, ne: int) -> int:
    """Compact fanout CSR: row pointers and edge ids."""
    return 4 * (nn + 1) + 4 * ne


def fwd_bwd_bytes(nn: int, ns: int, nc: int, ne: int) -> dict:
    """Compulsory bytes of one forward + reverse pass with the model gradient, every structure or
    value array read or written once (int32 indices, binary32 values; repeated gathers and the edge
    adjoints not counted).  Forward: fanin CSR, startpoint SP and TR in, C_load in, SP and TR of
    every net out.  Reverse: fanin CSR, SP and C_load in, fanout CSR, the adjoint of every net
    written, the pin-cap gradient of every cell and the SP and TR gradients of every startpoint out."""
    fwd = fanin_bytes(nc, ne) + 8 * ns + 4 * nn + 8 * nn
    bwd = fanin_bytes(nc, ne) + 4 * nn + 4 * nn + fanout_bytes(nn, ne) + 4 * nn + 4 * nc + 8 * ns
    return {"forward": fwd, "backward": bwd, "total": fwd + bwd}


def algorithmic_bytes(nn: int, ns: int, nc: int, ne: int, T: int) -> dict:
    """Compulsory bytes per phase of the step (same counting as fwd_bwd_bytes)."""
    fb = fwd_bwd_bytes(nn, ns, nc, ne)
    return {
        "forward": fb["forward"],
        # generator: startpoint SP and TR in, their words out; cells: fanin CSR, every fanin word
        # read once, every cell's words written once; toggles + ones of every net written
        "simulation": 8 * ns + 8 * T * ns + fanin_bytes(nc, ne) + 8 * T * nn + 8 * T * nc + 8 * nn,
        # TR_model and toggles read, beta and hybrid TR written, C_load read for the power
        "hybrid": 4 * nn * 5,
        # the reverse pass with the paper's beta rule (beta read) and the gradient outputs of the step:
        # the pass's compulsory bytes, beta, and the C_load gradient (hybrid TR in, gradient out)
        "backward": fb["backward"] + 4 * nn + 8 * nn,
        # outputs: the four gradient arrays copied into the caller's buffers (read + write)
        "outputs": 8 * (2 * ns + nc + nn),
    }


def sim_bytes(nn: int, ns: int, nc: int, ne: int, T: int) -> int:
    """The simulation pass alone: every net's words written once and read once (T uint64 per
    net), the fanin CSR, and toggles + ones of every net written."""
    return 2 * 8 * T * nn + fanin_bytes(nc, ne) + 8 * nn


def batched_algorithmic_bytes(nn: int, ns: int, nc: int, ne: int, S: int) -> int:
    """Forward + power + reverse pass of S scenarios: structures once per pass (fanin in both,
    fanout in the reverse, C_load in both), and per scenario the inputs (SP, TR), one SP per
    net written by the forward and read by the reverse pass, and the input gradients out."""
    fanin = 4 * (nc + 1) + 4 * ne + nc
    fanout = 4 * (nn + 1) + 4 * ne
    return 2 * fanin + fanout + 8 * nn + S * (8 * ns + 4 * nn + 4 * nn + 8 * ns)


# DRAM traffic per launch of the dominant kernels, from `ncu --metrics
# dram__bytes_read.sum,dram__bytes_write.sum` on the 2,000,000-cell step (the
# captures and commands are summarised under profiles/).  A figure is reported
# only for the workload it was taken on, and while the kernel's source files
# still hash to the value it was taken with; otherwise the traffic is unknown
# (null).
TRAFFIC = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,lts__t_bytes.sum,... (one launch),
    # 2M-cell step, 4th step (profiles/roofline_step_k_sim_wide_traffic.md)
    "k_sim_wide": {"bytes": 224_526_080 + 162_210_304, "l2_bytes": 7_799_694_112, "workload": "roofline",
                   "files": ["kern_persist.cu", "kern_common.cuh"],
                   "sha": "d68f35c894eb261c"},
}


# L2 <-> SM throughput ceiling for the L2 fraction of the dominant kernel: ncu's peak of
# lts__t_bytes on this part (summarised with the capture under profiles/); None until measured.
L2_PEAK_GBS = 36_130.0
L2_PEAK_SOURCE = ("ncu on k_sim_wide, 2M-cell step: lts__t_bytes.sum.per_second 11,471 GB/s at "
                  "lts__t_bytes.sum.pct_of_peak_sustained_elapsed 31.75 %")


def kernel_l2_bytes(kernel: str, workload: str) -> int | None:
    """lts__t_bytes of one launch, under the same conditions as kernel_traffic."""
    t = TRAFFIC.get(kernel)
    if not t or "l2_bytes" not in t or L2_PEAK_GBS is None or kernel_traffic(kernel, workload) is None:
        return None
    return int(t["l2_bytes"])


def kernel_traffic(kernel: str, workload: str) -> int | None:
    import hashlib
    t = TRAFFIC.get(kernel)
    if not t or t["workload"] != workload:
        return None
    m = hashlib.sha256()
    for name in t["files"]:
        with open(os.path.join(ROOT, "paper_2608_03778_gb300", "csrc", name), "rb") as f:
            m.update(f.read())
    return int(t["bytes"]) if m.hexdigest()[:16] == t["sha"] else None


class Clocks:
    """Samples nvidia-smi during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "50", "-i", str(gpu)], stdout=self.f, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.p = None

    def stop(self) -> dict | None:
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as g:
            for line in g:
                c = [x.strip() for x in line.split(",")]
                if len(c) >= 9:
                    rows.append(c)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(world: int):
    import torch
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return dist if world > 1 else None


def max_over_ranks(x: float, world: int) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def workload(name: str):
    from paper_2608_03778_gb300 import netgen
    spec = netgen.WORKLOADS[name]
    lib = netgen.library_text()
    text = netgen.netlist_text(spec)
    sp, tr = netgen.scenario_inputs(spec.n_start, 1000)
    return spec, lib, text, np.ascontiguousarray(sp[:, 0]), np.ascontiguousarray(tr[:, 0])


def host_cpu() -> dict:
    """Host cores and CPU model of this machine (nproc; the model from lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip().lower() == "model name" and ":" in line:
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    k = line.split(":")[0].strip().lower()
                    if k in ("model name", "cpu model", "hardware") and ":" in line:
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    return {"nproc": os.cpu_count(), "cpu_model": model}


def bench_config(name: str, spec, world: int) -> dict:
    """The `config` object of both arms: the workload and what one step does."""
    return {
        "workload": f"{name}: {spec.n_cells} cells, {spec.n_start} startpoints ({spec.n_pi} PI + {spec.n_dff} "
                    f"DFF), depth {spec.depth}, fanout cap {spec.fanout_cap}, seed {spec.seed}",
        "step": "forward SP/TR + power, 4,096-vector simulation, hybrid beta + power, adjoint "
                "(grad_mode 1) with all gradient outputs",
        "global_batch": 1, "parallelism": f"replicas x{world}",
        "l2": "256 MB buffer written before every timed step (outside the step's events)",
    }


def oracle_step_times(o, sp, tr, T: int, reps: int, parallel: bool) -> list[float]:
    """Seconds of `reps` full steps of the FP64 oracle (forward, power, simulation, hybrid, adjoint
    with the paper's beta rule and every gradient output), timed outright."""
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        o.step(sp, tr, seed=42, T=T, grad_mode=1, parallel=parallel)
        ts.append(time.perf_counter() - t0)
    return ts


def cpu_baseline(text: str, lib: str, sp, tr, n_cells: int, T: int, reps: int = 5) -> dict:
    """The FP64 oracle, as it stands, on full steps of the same workload: single-threaded (the
    paper's CPU comparator), median of `reps`; beside it the oracle's level-parallel variant on all
    host cores (OpenMP), median of `reps`."""
    from oracle.oracle import Oracle, threads
    o = Oracle(text, lib)
    t1 = oracle_step_times(o, sp, tr, T, reps, parallel=False)
    tp = oracle_step_times(o, sp, tr, T, reps, parallel=True)
    m1, mp = statistics.median(t1), statistics.median(tp)
    host = host_cpu()
    return {"value": n_cells / m1, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"full steps (forward, power, {64 * T}-vector simulation, hybrid, adjoint) of the same "
                      f"netlist, median of {reps}: {m1:.2f} s, single thread",
            "step_s": t1, **host,
            "all_cores": {"value": n_cells / mp, "unit": UNIT, "cores": threads(), "kind": "oracle, level-parallel",
                          "sample": f"the same full steps with the oracle's level-parallel variant (OpenMP), "
                                    f"median of {reps}: {mp:.2f} s", "step_s": tp}}


REFERENCE_BUDGET_S = 120.0   # the whole --impl reference run, warm-up included


def run_reference(args, rank: int, world: int) -> None:
    """Reference arm: the FP64 CPU oracle as it stands, single-threaded, rank 0 only.

    Each step is one full step of the oracle (forward, power, 4,096-vector simulation, hybrid,
    adjoint with every gradient output), timed outright, on a bounded sample of the workload: the
    same generator recipe (startpoint shares, depth, fanout cap, seed) at a cell count chosen so
    that the warm-up and timed steps together take about REFERENCE_BUDGET_S on this host (the
    oracle's rate on a 20,000-cell draw sets it; the full netlist when it fits)."""
    if rank != 0:
        return
    from dataclasses import replace

    from oracle.oracle import Oracle
    from paper_2608_03778_gb300 import netgen
    full = netgen.WORKLOADS[args.workload]
    lib = netgen.library_text()
    T = 64

    def draw(n_cells: int):
        if n_cells >= full.n_cells:
            spec = full
        else:
            f = n_cells / full.n_cells
            spec = replace(full, n_cells=n_cells, n_pi=max(8, round(full.n_pi * f)),
                           n_dff=max(8, round(full.n_dff * f)), depth=max(2, min(full.depth, n_cells // 16)))
        text = netgen.netlist_text(spec)
        sp, tr = netgen.scenario_inputs(spec.n_start, 1000)
        return spec, Oracle(text, lib), np.ascontiguousarray(sp[:, 0]), np.ascontiguousarray(tr[:, 0])

    probe_spec, o, sp, tr = draw(min(20_000, full.n_cells))
    rate = probe_spec.n_cells / min(oracle_step_times(o, sp, tr, T, 2, parallel=False))
    per_step = REFERENCE_BUDGET_S / max(1, args.steps + args.warmup)
    n = int(min(full.n_cells, max(probe_spec.n_cells, 0.9 * rate * per_step)))
    spec, o, sp, tr = (probe_spec, o, sp, tr) if n == probe_spec.n_cells else draw(n)

    oracle_step_times(o, sp, tr, T, args.warmup, parallel=False)
    ts = oracle_step_times(o, sp, tr, T, args.steps, parallel=False)
    ms = 1e3 * sum(ts) / len(ts)
    val = spec.n_cells / (ms / 1e3)
    sample = "the full netlist" if spec is full else (
        f"a {spec.n_cells}-cell draw of the same recipe ({spec.n_start} startpoints, depth {spec.depth})")
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(args.workload, full, world),
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"per step: one full step of the FP64 oracle (forward, power, {64 * T}-vector "
                                   f"simulation, hybrid, adjoint with every gradient output) on {sample}, timed "
                                   f"outright; sized for about {REFERENCE_BUDGET_S:.0f} s in all; single thread",
                         "step_ms_median": 1e3 * statistics.median(ts), **host_cpu()},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def pct(ts, q: float) -> float:
    return float(np.percentile(np.asarray(ts, np.float64), q))


def timed_reps(fn, stream, flush, reps: int) -> list[float]:
    """CUDA-event milliseconds of `reps` calls of fn on `stream`; with a flush buffer, L2 is flushed
    by writing it before each call, outside the events."""
    import torch
    out = []
    for i in range(reps):
        if flush is not None:
            flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        out.append(e0.elapsed_time(e1))
    return out


def rep_stats(ts) -> dict:
    return {"median_ms": statistics.median(ts), "p10_ms": pct(ts, 10), "p90_ms": pct(ts, 90), "reps": len(ts)}


def fwd_bwd_record(dp, ctx, d, stream, flush, reps: int, pk: dict) -> dict:
    """dp_propagate + dp_backward with the model gradient and the compulsory outputs (SP and TR
    gradients of the startpoints, pin-cap gradients), L2 flushed and warm, median of `reps`."""
    import torch
    info = dp.dp_design_info(d)
    nn, ns, nc, ne = info.n_nets, info.n_start, info.n_cells, info.n_edges
    dev = torch.device("cuda", torch.cuda.current_device())
    gsp, gtr, gpin = (torch.zeros(n, device=dev) for n in (ns, ns, nc))
    cfg0 = dp.config(grad_mode=0)

    def fn():
        dp.dp_propagate(ctx, d, cfg0)
        dp.dp_backward(ctx, d, cfg0, gsp, gtr, gpin, None, 1)

    for _ in range(5):
        fn()
    torch.cuda.synchronize()
    cold, ph = [], []
    for _ in range(reps):
        cold += timed_reps(fn, stream, flush, 1)
        ph.append(dp.dp_phase_times(ctx, d))   # library events around the forward and the reverse pass
    ph = np.median(np.stack(ph), axis=0)
    warm = timed_reps(fn, stream, None, reps)
    fb = fwd_bwd_bytes(nn, ns, nc, ne)
    ms, wms = statistics.median(cold), statistics.median(warm)
    return {"ms": ms, **{k: v for k, v in rep_stats(cold).items() if k != "median_ms"},
            "cell_evals_per_s": nc / (ms * 1e-3),
            "algorithmic_bytes": fb["total"], "achieved_gbs": fb["total"] / (ms * 1e-3) / 1e9,
            "frac": fb["total"] / (ms * 1e-3) / 1e9 / pk["hbm_gbs"],
            "warm_l2": {**rep_stats(warm), "cell_evals_per_s": nc / (wms * 1e-3),
                        "frac": fb["total"] / (wms * 1e-3) / 1e9 / pk["hbm_gbs"]},
            "levels": 2 * int(info.n_levels),
            "forward_ms": float(ph[0]), "backward_ms": float(ph[3]),
            "what": "dp_propagate + dp_backward (grad_mode 0; startpoint SP/TR and pin-cap gradients out); "
                    "L2 flushed before each repetition (warm_l2: not flushed); median"}


def bench_config_passes(dp, torch, dev, name: str, reps: int, pk: dict, with_sim: bool) -> dict:
    """One single-scenario workload: forward + reverse pass (fwd_bwd_record), and with `with_sim`
    the 4,096-vector simulation alone (generator + bitwise levels, then beta + hybrid power) with
    its own roofline; L2 flushed and warm."""
    spec, lib, text, sp, tr = workload(name)
    stream = torch.cuda.current_stream()
    ctx = dp.dp_create(dev.index or 0, stream.cuda_stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    try:
        d = dp.dp_design_load(ctx, text, lib)
        try:
            info = dp.dp_design_info(d)
            nn, ns, nc, ne = info.n_nets, info.n_start, info.n_cells, info.n_edges
            dp.dp_set_inputs(ctx, d, sp, tr)
            out = {"workload": f"{name}: {nc} cells, {ns} startpoints ({spec.n_pi} PI + {spec.n_dff} DFF), depth "
                               f"{info.n_levels}, seed {spec.seed}",
                   "fwd_bwd": fwd_bwd_record(dp, ctx, d, stream, flush, reps, pk)}
            out["fwd_bwd"]["us"] = 1e3 * out["fwd_bwd"]["ms"]
            if with_sim:
                cfg = dp.config()
                dp.dp_propagate(ctx, d, cfg)
                sim = lambda: dp.dp_simulate(ctx, d, cfg)  # noqa: E731
                for _ in range(5):
                    sim()
                torch.cuda.synchronize()
                res = {}
                for key, fl in (("cold", flush), ("warm_l2", None)):
                    ts, ph = [], []
                    for i in range(reps):
                        ts += timed_reps(sim, stream, fl, 1)
                        ph.append(dp.dp_phase_times(ctx, d))
                    ph = np.median(np.stack(ph), axis=0)
                    b = sim_bytes(nn, ns, nc, ne, cfg.sim_words)
                    res[key] = {**rep_stats(ts), "levels_ms": float(ph[1]), "hybrid_ms": float(ph[2]),
                                "achieved_gbs": b / (float(ph[1]) * 1e-3) / 1e9,
                                "frac": b / (float(ph[1]) * 1e-3) / 1e9 / pk["hbm_gbs"]}
                out["simulation"] = {"vectors": 64 * cfg.sim_words, "algorithmic_bytes": b,
                                     "roofline": "hbm, on the generator + bitwise levels time (levels_ms)",
                                     **res["cold"], "warm_l2": res["warm_l2"],
                                     "what": "dp_simulate: Philox Markov startpoints + bitwise levels with PopCount "
                                             "(levels_ms), then beta + hybrid power (hybrid_ms)"}
        finally:
            dp.dp_design_free(d)
    finally:
        dp.dp_destroy(ctx)
    return out


# The paper's kernel times (Table II: forward "Alg.", bitwise simulation, backward; 1x A100,
# its three proprietary designs), beside which the same passes are timed on synthetic
# netlists of the same cell count and depth.  Context only: other hardware, other designs.
PAPER_TABLE_II_MS = {
    "paper_small": {"cells": 13_000, "levels": 70, "forward": 13.5, "bitwise": 12.4, "backward": 13.2},
    "paper_medium": {"cells": 117_000, "levels": 84, "forward": 16.1, "bitwise": 16.0, "backward": 16.5},
    "paper_large": {"cells": 652_000, "levels": 104, "forward": 28.9, "bitwise": 26.9, "backward": 24.2},
}


def bench_paper_shaped(dp, torch, dev, reps: int, pk: dict) -> dict:
    """Forward, 4,096-vector simulation and backward on synthetic netlists with the cell count
    and depth of the paper's three designs, L2 flushed, beside the paper's Table II times."""
    out = {}
    for name, paper in PAPER_TABLE_II_MS.items():
        r = bench_config_passes(dp, torch, dev, name, reps, pk, True)
        fb, sim = r["fwd_bwd"], r["simulation"]
        out[name] = {"workload": r["workload"],
                     "forward_ms": fb["forward_ms"], "backward_ms": fb["backward_ms"],
                     "fwd_bwd_ms": fb["ms"], "simulation_levels_ms": sim["levels_ms"],
                     "simulation_ms": sim["median_ms"],
                     "paper_a100_ms": {k: paper[k] for k in ("forward", "bitwise", "backward")},
                     "paper_over_this": {"forward": paper["forward"] / fb["forward_ms"],
                                         "bitwise": paper["bitwise"] / sim["levels_ms"],
                                         "backward": paper["backward"] / fb["backward_ms"]}}
    out["note"] = ("context only: the paper's times are its A100 on its proprietary designs; these are "
                   "synthetic netlists of the same cell count and depth (the generator's fanin mix, "
                   "about 3.2 pins per cell against the paper's 4), 4,096 simulated vectors")
    return out


def bench_batched(args, dp, torch, dev, pk: dict) -> dict:
    """The 120,000-cell netlist x 512 input-activity scenarios (scenario-innermost SoA, one
    launch per level for all scenarios, launch shapes from the library's autotuner):
    forward + power + reverse pass timed with CUDA events, L2 flushed before each
    repetition; then 200 projected ascent steps for all 512 starts (Algorithm 4) through
    the autograd Function, captured in a CUDA graph, and P_virus (Eq. 3) of the result."""
    from paper_2608_03778_gb300 import netgen, torch_api as ta
    # ascent rate in SP per fF of proxy gradient: the median gradient is about 4 fF and the
    # 90th percentile about 40 fF on this netlist, so a step moves most inputs by < 0.1
    ETA = 2e-3
    spec = netgen.WORKLOADS["mid"]
    lib, text = netgen.library_text(), netgen.netlist_text(spec)
    S = 512
    sp, tr = netgen.scenario_inputs(spec.n_start, 1000, S)
    des = ta.Design(text, lib, dev.index or 0)
    try:
        info = dp.dp_design_info(des.d)
        nn, ns, nc, ne, L = info.n_nets, info.n_start, info.n_cells, info.n_edges, info.n_levels
        sp_d, tr_d = torch.from_numpy(sp).to(dev), torch.from_numpy(tr).to(dev)
        cfg = dp.config(grad_mode=0, tr_mode=0)
        power = torch.empty(S, dtype=torch.float64, device=dev)
        gsp = torch.empty_like(sp_d)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

        def fwd_bwd():
            des.follow_stream()
            dp.dp_set_inputs_batch(des.ctx, des.d, sp_d, tr_d, S, 1)
            dp.dp_propagate(des.ctx, des.d, cfg)
            dp.dp_get_power(des.ctx, des.d, power, 0, 1)
            dp.dp_backward_weighted(des.ctx, des.d, cfg, None, 0, gsp, None, None, None, 1)

        for _ in range(args.warmup):
            fwd_bwd()
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        ts = timed_reps(fwd_bwd, stream, flush, max(args.steps, 20))
        warm = timed_reps(fwd_bwd, stream, None, max(args.steps, 20))
        ms = statistics.median(ts)
        fwd_shape, bwd_shape, tune_ms = dp.dp_batch_tuning(des.d)
        ab = batched_algorithmic_bytes(nn, ns, nc, ne, S)
        ach = ab / (ms * 1e-3) / 1e9
        # kernels per forward + reverse pass: start + L levels, 2 power, seed, L levels + start
        launches = (1 if ns else 0) + L + 2 + 1 + L + (1 if ns else 0)

        # Algorithm 4: 200 steps for all 512 starts, the proxy of Eq. 9 (tr_mode 1)
        steps = 200
        p0 = torch.empty(S, dtype=torch.float64, device=dev)
        dp.dp_virus_eval(des.ctx, des.d, sp_d, S, p0, None, 1)
        res = ta.power_virus(des, sp_d, tr_d, steps, ETA, tr_mode=1, graph=True)
        pv0, pv1 = p0.cpu().numpy(), res.p_virus.cpu().numpy()
        out = {
            "workload": f"mid: {nc} cells, {ns} startpoints, depth {L}, seed {spec.seed}; {S} scenarios "
                        f"(SP ~ U[0.1, 0.9], TR ~ U[0, 2 min(SP, 1-SP)], seeds 1000..{1000 + S - 1})",
            "fwd_bwd_ms": ms, "fwd_bwd_ms_p10_p90": [pct(ts, 10), pct(ts, 90)],
            "cell_evals_per_s": nc * S / (ms * 1e-3),
            "warm_l2": {**rep_stats(warm), "cell_evals_per_s": nc * S / (statistics.median(warm) * 1e-3),
                        "frac": ab / (statistics.median(warm) * 1e-3) / 1e9 / pk["hbm_gbs"]},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": ach / pk["hbm_gbs"], "algorithmic_bytes": ab, "traffic": None,
                         "kernels": "k_fwdb_level / k_bwdb_level per level, k_powerb_*"},
            "shapes": {"forward": list(fwd_shape), "backward": list(bwd_shape), "tuner_ms": list(tune_ms)},
            "gpu_launches_per_fwd_bwd": launches,
            "ascent": {"steps": steps, "starts": S, "eta": ETA, "proxy": "Eq. 9 (tr_mode 1)",
                       "graph": res.graph, "ms_total": res.ms_ascent, "ms_per_step": res.ms_ascent / steps,
                       "gpu_launches_per_step": launches + 1,
                       "proxy_fF_mean": [float(res.proxy_start.mean()), float(res.proxy_end.mean())],
                       "p_virus_fF_mean": [float(pv0.mean()), float(pv1.mean())],
                       "p_virus_fF_best": [float(pv0.max()), float(pv1.max())]},
            "l2": "256 MB buffer written before every timed repetition; working set > 1 GB",
            "device_bytes": int(dp.dp_design_info(des.d).device_bytes),
        }
    finally:
        des.close()
    return out


def bench_serving(args, dp, torch, dev) -> dict:
    """Served requests on 8 resident netlists (5K, 20K, 50K, 120K, 300K, 600K, 1M and 2M cells,
    generator seeds 1-8): 2,000 requests, each naming a design uniformly and carrying either new
    input SP/TR or a sizing delta (1 % of the design's X1 cells moved to X2 or X4), half of them
    asking for gradients.  Three kinds of runs of the same requests: Poisson arrivals at 5,000
    requests/s through the continuous-batching server (latency from submission to completion,
    p50/p99; one untimed run of the same stream first, then three timed ones, their medians
    reported with every run); all 2,000 submitted back to back (saturated throughput; one untimed
    run, then three, the median one reported with every run); and the plain loop - one request
    at a time,
    synchronous, the same kernels with one scenario per launch.  The server runs two batch slots per
    design (one batch's copies beside the next one's kernels).  The served results must equal the
    plain loop's bit for bit."""
    from paper_2608_03778_gb300 import netgen
    names = [f"serve_{n}" for n in (5000, 20000, 50000, 120000, 300000, 600000, 1000000, 2000000)]
    lib = netgen.library_text()
    n_req, rate, max_batch, slots = 2000, 5000.0, 64, 2
    rng = np.random.default_rng(2026)
    texts = [netgen.netlist_text(netgen.WORKLOADS[n]) for n in names]
    x1 = []
    for t in texts:
        c = dp.dp_compile(t, lib)
        v = dp.dp_compiled_view_get(c)
        dp.dp_compiled_free(c)
        x1.append(np.flatnonzero(v["pincap"][v["cell_of_user"]] == np.float32(0.8)).astype(np.int32))
    pin = lambda n, dt: torch.empty(n, dtype=dt, pin_memory=True).numpy()  # noqa: E731
    srv = dp.dp_server_create(dp.server_config(device=dev.index or 0, max_batch=max_batch, slots_per_design=slots))
    plain = dp.dp_server_create(dp.server_config(device=dev.index or 0, plain=1))
    try:
        infos = []
        for i, t in enumerate(texts):
            ns = netgen.WORKLOADS[names[i]].n_start
            sp, tr = netgen.scenario_inputs(ns, 500 + i, 1)
            ref = (np.ascontiguousarray(sp[:, 0]), np.ascontiguousarray(tr[:, 0]))
            a = dp.dp_server_add_design(srv, t, lib, *ref)
            b = dp.dp_server_add_design(plain, t, lib, *ref)
            assert a == b == i
            infos.append(dp.dp_server_design_info(srv, i))
        jobs = []
        for j in range(n_req):
            k = int(rng.integers(len(names)))
            ns, nc = infos[k].n_start, infos[k].n_cells
            job = {"design": k, "grad": int(rng.integers(2)), "power": pin(1, torch.float64)}
            if rng.integers(2):
                sp, tr = netgen.scenario_inputs(ns, 10_000 + j, 1)
                job["sp"], job["tr"] = pin(ns, torch.float32), pin(ns, torch.float32)
                job["sp"][:], job["tr"][:] = sp[:, 0], tr[:, 0]
                job["kind"] = "inputs"
            else:
                m = max(1, nc // 100)
                cells = rng.choice(x1[k], min(m, len(x1[k])), replace=False).astype(np.int32)
                job["cells"], job["caps"] = pin(len(cells), torch.int32), pin(len(cells), torch.float32)
                job["cells"][:] = cells
                job["caps"][:] = rng.choice(np.array([1.6, 3.2], np.float32), len(cells))
                job["kind"] = "sizing"
            if job["grad"]:
                job["gsp"], job["gtr"], job["gpin"] = pin(ns, torch.float32), pin(ns, torch.float32), pin(
                    nc, torch.float32)
            job["req"] = dp.request(k, job["power"], job.get("sp"), job.get("tr"), job.get("cells"),
                                    job.get("caps"), job["grad"], job.get("gsp"), job.get("gtr"), job.get("gpin"))
            jobs.append(job)

        def results():
            return [[j["power"].copy()] + ([j["gsp"].copy(), j["gtr"].copy(), j["gpin"].copy()] if j["grad"] else [])
                    for j in jobs]

        # warm-up: every design once through each server
        for k in range(len(names)):
            w = [j for j in jobs if j["design"] == k][:2]
            for j in w:
                dp.dp_server_wait(srv, dp.dp_server_submit(srv, j["req"]), 120.0)
                dp.dp_server_wait(plain, dp.dp_server_submit(plain, j["req"]), 120.0)

        # Poisson arrivals: one untimed run (batches of every size the stream forms meet their
        # first launch there), then three timed runs in a row on the same (long-running) server
        gaps = rng.exponential(1.0 / rate, n_req)
        arrive = np.cumsum(gaps) - gaps[0]
        runs = []
        for rep in range(4):
            st0 = dp.dp_server_get_stats(srv)
            tickets = []
            t0 = time.perf_counter()
            for j, ta in zip(jobs, arrive):
                while time.perf_counter() - t0 < ta:
                    pass
                tickets.append(dp.dp_server_submit(srv, j["req"]))
            lat = np.array([dp.dp_server_wait(srv, t, 600.0) for t in tickets])
            t_poisson = time.perf_counter() - t0
            st1 = dp.dp_server_get_stats(srv)
            nb = st1.batches - st0.batches
            if rep == 0:
                continue
            runs.append({"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                         "throughput_rps": n_req / t_poisson, "batches": int(nb),
                         "mean_batch": (st1.requests - st0.requests) / max(nb, 1),
                         "host_launch_us_per_batch": 1e6 * (st1.host_launch_s - st0.host_launch_s) / max(nb, 1)})
        # (results are read once the runs are over: host work between runs left the GPU idle, and
        # a run that starts on an idle GPU is slower)
        served = results()
        # saturated: all requests at once; one untimed run (the GPU idled while the host read the
        # results), then three back to back, the median one reported with all three
        sat_runs = []
        for rep in range(4):
            st1 = dp.dp_server_get_stats(srv)
            t0 = time.perf_counter()
            tickets = [dp.dp_server_submit(srv, j["req"]) for j in jobs]   # back to back
            lat_sat = np.array([dp.dp_server_wait(srv, t, 600.0) for t in tickets])
            t_sat = time.perf_counter() - t0
            st2 = dp.dp_server_get_stats(srv)
            if rep == 0:
                continue
            sat_runs.append({"throughput_rps": n_req / t_sat, "seconds": t_sat,
                             "p50_ms": float(np.percentile(lat_sat, 50)), "p99_ms": float(np.percentile(lat_sat, 99)),
                             "mean_batch": (st2.requests - st1.requests) / max(st2.batches - st1.batches, 1)})
        saturated = results()
        sat_med = sorted(sat_runs, key=lambda r: r["seconds"])[1]
        # plain loop (a few untimed requests first, as the GPU idled while the host read the results)
        for j in jobs[:50]:
            dp.dp_server_wait(plain, dp.dp_server_submit(plain, j["req"]), 600.0)
        t0 = time.perf_counter()
        lat_plain = np.array([dp.dp_server_wait(plain, dp.dp_server_submit(plain, j["req"]), 600.0) for j in jobs])
        t_plain = time.perf_counter() - t0
        base = results()
        same = all(all(np.array_equal(x, y) for x, y in zip(a, b)) for a, b in zip(served, base)) and all(
            all(np.array_equal(x, y) for x, y in zip(a, b)) for a, b in zip(saturated, base))
        return {
            "workload": "8 resident netlists serve_5000 ... serve_2000000 (seeds 1-8); 2,000 requests, half new "
                        "input SP/TR, half sizing deltas (1 % of X1 cells to X2/X4); gradients on half",
            "max_batch": max_batch,
            "slots_per_design": slots,
            "cuda_device_max_connections": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS", "8 (default)"),
            "poisson": {"rate_per_s": rate,
                        "p50_ms": float(np.median([r["p50_ms"] for r in runs])),
                        "p99_ms": float(np.median([r["p99_ms"] for r in runs])),
                        "throughput_rps": float(np.median([r["throughput_rps"] for r in runs])),
                        "reported": "median over the three runs", "runs": runs},
            "saturated": {**sat_med, "reported": "the median of three runs", "runs": sat_runs},
            "plain_loop": {"throughput_rps": n_req / t_plain, "p50_ms": float(np.percentile(lat_plain, 50)),
                           "p99_ms": float(np.percentile(lat_plain, 99))},
            "speedup_saturated_vs_plain": t_plain / sat_med["seconds"],
            "identical_to_plain_loop": bool(same),
            "device_bytes": int(dp.dp_server_get_stats(srv).device_bytes),
        }
    finally:
        dp.dp_server_destroy(srv)
        dp.dp_server_destroy(plain)


def serving_in_child(device: int) -> dict:
    """The serving measurement in a fresh interpreter on the same GPU: its own CUDA
    context, streams, threads and host allocations, so that nothing the earlier
    measurements leave in this process enters its latencies (servers created one after
    another in one process serve Poisson arrivals a little more slowly each time).  The
    child gets 32 hardware work queues (CUDA_DEVICE_MAX_CONNECTIONS, unless the caller set
    it): the server's 16 slot streams and the plain loop's 8 then share none."""
    drop = {"RANK", "WORLD_SIZE", "LOCAL_RANK", "LOCAL_WORLD_SIZE", "GROUP_RANK", "ROLE_RANK",
            "MASTER_ADDR", "MASTER_PORT", "TORCHELASTIC_RUN_ID"}
    env = {k: v for k, v in os.environ.items() if k not in drop}
    env.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--serving-only", "--device", str(device)],
                       env=env, capture_output=True, text=True, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(f"serving measurement failed ({r.returncode}): {r.stderr[-2000:]}")
    for line in r.stdout.splitlines():
        if line.startswith("{"):
            return json.loads(line)
    raise RuntimeError("serving measurement printed no result")


def bench_adjoint_vs_fd(dp, torch, dev) -> dict:
    """Gradient of the model power with respect to every startpoint SP of the 120,000-cell
    netlist: the GPU adjoint (compile + upload + forward + reverse pass, wall clock, as the
    paper counts graph creation; and the device time of the two passes) against one-sided
    finite differences on the CPU (one perturbation per startpoint, eps = 1e-4, as in the paper's
    sweep) with the FP64 oracle, extrapolated from timed forward passes.  Agreement on a stratified
    sample of startpoints: Pearson r and top-k overlap."""
    from oracle.oracle import Oracle
    from paper_2608_03778_gb300 import netgen
    spec = netgen.WORKLOADS["mid"]
    lib, text = netgen.library_text(), netgen.netlist_text(spec)
    sp, tr = netgen.scenario_inputs(spec.n_start, 1000)
    sp, tr = np.ascontiguousarray(sp[:, 0]), np.ascontiguousarray(tr[:, 0])
    cfg = dp.config(grad_mode=0)
    ctx = dp.dp_create(dev.index or 0, torch.cuda.current_stream().cuda_stream)
    try:
        g = np.zeros(spec.n_start, np.float32)
        t0 = time.perf_counter()
        d = dp.dp_design_load(ctx, text, lib)
        dp.dp_set_inputs(ctx, d, sp, tr)
        dp.dp_propagate(ctx, d, cfg)
        dp.dp_backward(ctx, d, cfg, g)
        wall = time.perf_counter() - t0
        for _ in range(3):
            dp.dp_propagate(ctx, d, cfg)
            dp.dp_backward(ctx, d, cfg, g)
        ph = dp.dp_phase_times(ctx, d)
        dev_ms = float(ph[0] + ph[3])
        dp.dp_design_free(d)
    finally:
        dp.dp_destroy(ctx)
    o = Oracle(text, lib)
    sp64, tr64 = sp.astype(np.float64), tr.astype(np.float64)
    cl = o.cload()
    K = 0.5 * 0.8 * 0.8 * 1e9 * 1e-15

    def power(x):
        return K * float(np.sum(o.forward(x, tr64, 0)[1] * cl))

    t0 = time.perf_counter()
    p0 = power(sp64)
    n_timed = 3
    for _ in range(n_timed - 1):
        power(sp64)
    t_fwd = (time.perf_counter() - t0) / n_timed
    rng = np.random.default_rng(7)
    order = np.argsort(-np.abs(g))
    idx = np.concatenate([order[:16], rng.choice(order[16:], 32, replace=False)])
    fd = []
    for k in idx:
        x = sp64.copy()
        x[k] += 1e-4
        fd.append((power(x) - p0) / 1e-4)
    fd = np.array(fd)
    r = float(np.corrcoef(fd, g[idx].astype(np.float64))[0, 1])
    top = len(set(np.argsort(-np.abs(fd))[:10]) & set(np.argsort(-np.abs(g[idx]))[:10]))
    fd_all = (spec.n_start + 1) * t_fwd
    return {"netlist": f"mid: {spec.n_cells} cells, {spec.n_start} startpoints, depth {spec.depth}",
            "gpu_wall_s": wall, "gpu_device_ms": dev_ms,
            "cpu_fd_s": fd_all, "cpu_fd": f"({spec.n_start} + 1) oracle forward passes of {t_fwd:.3f} s "
                                         f"(mean of {n_timed}), single thread, extrapolated",
            "speedup_vs_gpu_wall": fd_all / wall, "speedup_vs_gpu_device": fd_all / (dev_ms * 1e-3),
            "sample": {"startpoints": int(len(idx)), "pearson_r": r, "top10_overlap": top}}


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="roofline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 512-scenario measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the request-server measurement")
    ap.add_argument("--no-fd", action="store_true", help="skip the adjoint-vs-finite-difference timing")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 2K- and 120K-cell single-scenario timings and the paper-shaped netlists")
    ap.add_argument("--no-probe", action="store_true", help="skip the level-latency probe")
    ap.add_argument("--serving-only", action="store_true", help=argparse.SUPPRESS)   # the child of serving_in_child
    ap.add_argument("--device", type=int, default=0, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.serving_only:
        import torch
        torch.cuda.set_device(args.device)
        from paper_2608_03778_gb300 import dp
        print(json.dumps(bench_serving(args, dp, torch, torch.device("cuda", args.device))), flush=True)
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    args.warmup = max(3, args.warmup)
    # the request server first, in its own process, while this one holds no CUDA context yet:
    # measured after the other sections, with this process's context (idle) on the same GPU,
    # its saturated runs varied two-fold between otherwise identical runs
    serving = serving_in_child(local) if rank == 0 and not args.no_serving else None

    import torch
    torch.cuda.set_device(local)
    dist_setup(world)
    from paper_2608_03778_gb300 import dp

    spec, lib, text, sp, tr = workload(args.workload)
    stream = torch.cuda.current_stream()
    ctx = dp.dp_create(local, stream.cuda_stream)
    d = dp.dp_design_load(ctx, text, lib)
    info = dp.dp_design_info(d)
    nn, ns, nc, ne = info.n_nets, info.n_start, info.n_cells, info.n_edges
    cfg = dp.config()   # grad_mode 1 (paper's beta rule), 64 words, tr_mode 0
    dev = torch.device("cuda", local)
    sp_d, tr_d = torch.from_numpy(sp).to(dev), torch.from_numpy(tr).to(dev)
    g = {k: torch.zeros(n, device=dev) for k, n in [("sp", ns), ("tr", ns), ("pin", nc), ("cl", nn)]}
    watts = np.zeros(2)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        dp.dp_set_inputs(ctx, d, sp_d, tr_d, 1, 1)
        dp.dp_step(ctx, d, cfg, g["sp"], g["tr"], g["pin"], g["cl"], None, 1)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- device-timed steps, L2 flushed before each (outside the events)
    clk = Clocks(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    phases = []
    barrier(world)
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        phases.append(dp.dp_phase_times(ctx, d))   # library events around each phase of this step
    torch.cuda.synchronize()
    barrier(world)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = max_over_ranks(sum(step_ms) / len(step_ms), world)
    ph = np.median(np.stack(phases), axis=0)
    kernels = dp.dp_step_kernels(d)
    # the same steps with L2 warm (no flush between them): what a re-propagation loop sees
    warm_ms = timed_reps(step, stream, None, max(args.steps, 5))
    dp.dp_step(ctx, d, cfg, g["sp"], g["tr"], g["pin"], g["cl"], watts, 1)

    # ---- end to end through the C-ABI with pinned host buffers
    pin = lambda n, dt: torch.empty(n, dtype=dt, pin_memory=True).numpy()  # noqa: E731
    sp_h, tr_h = pin(ns, torch.float32), pin(ns, torch.float32)
    sp_h[:], tr_h[:] = sp, tr
    hg = {k: pin(n, torch.float32) for k, n in [("sp", ns), ("tr", ns), ("pin", nc), ("cl", nn)]}
    w_h = pin(2, torch.float64)
    for _ in range(2):
        dp.dp_set_inputs(ctx, d, sp_h, tr_h, 1, 0)
        dp.dp_step(ctx, d, cfg, hg["sp"], hg["tr"], hg["pin"], hg["cl"], w_h, 0)
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        dp.dp_set_inputs(ctx, d, sp_h, tr_h, 1, 0)
        dp.dp_step(ctx, d, cfg, hg["sp"], hg["tr"], hg["pin"], hg["cl"], w_h, 0)
    e2e_ms = max_over_ranks(1e3 * (time.perf_counter() - t0) / args.steps, world)
    barrier(world)
    h2d = 8 * ns
    d2h = 4 * (2 * ns + nc + nn) + 16

    # ---- roofline of the dominant kernel (each phase below is one kernel of the step, plus
    # the small power reduction in the forward phase)
    pk = peaks()
    ab = algorithmic_bytes(nn, ns, nc, ne, cfg.sim_words)
    names = ["forward", "simulation", "hybrid", "backward", "outputs"]
    kernel_of = {"forward": "k_fwd_persist", "simulation": "k_sim_wide", "backward": "k_bwd_persist"}
    per_phase = {}
    for i, n in enumerate(names):
        t = float(ph[i]) * 1e-3
        ach = ab[n] / t / 1e9 if t > 0 else 0.0
        per_phase[n] = {"ms": float(ph[i]), "algorithmic_bytes": ab[n], "achieved_gbs": ach,
                        "frac": ach / pk["hbm_gbs"]}
    dom = max(["forward", "simulation", "backward"], key=lambda n: per_phase[n]["ms"])
    roof = {"bound": "hbm", "kernel": f"{kernel_of[dom]} ({dom}, one cooperative launch per step)",
            "achieved": per_phase[dom]["achieved_gbs"], "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": per_phase[dom]["frac"], "traffic": kernel_traffic(kernel_of[dom], args.workload),
            "algorithmic_bytes": ab[dom], "peak_source": pk["source"]}
    l2b = kernel_l2_bytes(kernel_of[dom], args.workload)
    if l2b is not None:
        # L2 <-> SM bytes of the same launch against the L2 bandwidth measured on this part
        roof["l2"] = {"bytes": l2b, "achieved_gbs": l2b / (per_phase[dom]["ms"] * 1e-3) / 1e9,
                      "peak_gbs": L2_PEAK_GBS, "frac": l2b / (per_phase[dom]["ms"] * 1e-3) / 1e9 / L2_PEAK_GBS,
                      "peak_source": L2_PEAK_SOURCE}
    line = {
        "metric": METRIC,
        "value": nc * world / (ms / 1e3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": bench_config(args.workload, spec, world),
        "roofline": roof,
        "phases": per_phase,
        "warm_l2_step": {**rep_stats(warm_ms), "cell_evals_per_s": nc / (statistics.median(warm_ms) * 1e-3)},
        "power_w": {"model": float(watts[0]), "hybrid": float(watts[1])},
        "e2e": {"value": nc * world / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(kernels) * args.steps,   # kernel nodes of the step graph x timed steps
        "gpu_launches_per_step": int(kernels),
        "device_bytes": int(info.device_bytes),
    }
    # ---- forward + reverse alone (model gradient, no simulation): N_c / (t_fwd + t_bwd)
    fbm = fwd_bwd_record(dp, ctx, d, stream, flush, max(args.steps, 50), pk)
    line["fwd_bwd_model"] = fbm
    # clocks sampled from the first timed step to here (step, warm-L2 steps, forward + reverse)
    line["clocks"] = clk.stop()
    # ---- the latency floor of the level-synchronous passes, measured with the library's barrier
    if not args.no_probe:
        lat = dp.dp_probe_latency(ctx, 1000)
        L = int(info.n_levels)
        floor_ms = L * (lat["level_us_256"] + lat["level_us_512"]) * 1e-3
        line["latency_floor"] = {
            **lat, "levels_forward": L, "levels_reverse": L, "floor_ms": floor_ms,
            "fwd_bwd_frac_of_floor": floor_ms / fbm["ms"],
            "forward_us_per_level": 1e3 * fbm["forward_ms"] / L, "reverse_us_per_level": 1e3 * fbm["backward_ms"] / L,
            "what": "dp_probe_latency: per level, a grid barrier plus three loads through L2 of values other "
                    "blocks stored in the level before and one store, on the forward (256-thread) and reverse "
                    "(512-thread) grids; floor = L x both; fwd_bwd_model's time against it"}

    # ---- Eq. 8 sizing scores and the top 1,000 cells from the step's adjoint (re-ranking cost)
    dp.dp_step(ctx, d, cfg, g["sp"], g["tr"], g["pin"], g["cl"], None, 1)
    top = np.zeros(1000, np.int32)
    dp.dp_sizing_scores(ctx, d, cfg, 0, None, 1000, top)
    t0 = time.perf_counter()
    for _ in range(5):
        dp.dp_sizing_scores(ctx, d, cfg, 0, None, 1000, top)
    line["sizing"] = {"cells": int(nc), "k": 1000, "ms_scores_and_top_k": 1e3 * (time.perf_counter() - t0) / 5,
                      "score": "Eq. 8, mode 0 (SP adjoint of the output net x hybrid P_sw)"}
    dp.dp_design_free(d)
    dp.dp_destroy(ctx)
    del flush
    if not args.no_configs:
        line["configs"] = {"small": bench_config_passes(dp, torch, dev, "small", max(args.steps, 50), pk, False),
                           "mid": bench_config_passes(dp, torch, dev, "mid", max(args.steps, 50), pk, True)}
        line["paper_shaped"] = bench_paper_shaped(dp, torch, dev, max(args.steps, 20), pk)
    if not args.no_batched:
        line["batched"] = bench_batched(args, dp, torch, dev, pk)
    if serving is not None:
        line["serving"] = serving
    if rank == 0 and world == 1 and not args.no_fd:
        line["adjoint_vs_fd"] = bench_adjoint_vs_fd(dp, torch, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(text, lib, sp, tr, nc, cfg.sim_words)
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
