#!/usr/bin/env python3
"""Throughput of the GB300 cell-based FMM gravity solve (Octo-Tiger, arXiv 1908.03121).

One step = the whole hot path on one synthetic workload: upward pass, same-level
(M2L) pass, downward pass, forces and conservation sums, replayed from one
captured CUDA graph.  The metric is same-level cell-interactions per second
(evaluated directed target<-source cell pairs, all four kinds) over the whole
step time.  Default workload: the level-7 contact binary (cfg5), mixed
precision.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun): every rank solves its own replica (the solve has no
exchange step); the time is the maximum over ranks and the value sums all
ranks' interactions.  ``--impl reference`` times the FP64 CPU oracle instead,
on a bounded sample of target cells per step, on the host's cores.
"""

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "M2L cell-interactions/s on 1 GB300, FP32-mixed vs FP64 at rel. force err ≤1e-6"
UNIT = "cell-interactions/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
PROFILES = os.path.join(ROOT, "profiles")
# FP32 FMA peak of a GB300 from its unit counts: 152 SMs x 128 lanes x 2 flop
# x 2.07 GHz maximum clock (the measured figure, from an FMA loop timed on
# the GPU in use, is what the roofline uses)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# FP64 rate of a GB300 (Blackwell Ultra): 1.25 TFLOP/s nominal
FP64_PEAK_TFLOPS = 1.25
# the paper's operation counts per interaction (Sec. 4.3): multipole targets
# 455, monopole<-monopole 12, with its 1074-point stencil at theta = 0.35
PAPER_FLOPS_MULTIPOLE = 455
PAPER_FLOPS_MONOPOLE = 12
# the paper's Table 2 FMM rates (FP64, whole same-level pass), context only
PAPER_TABLE2_GFLOPS = {"P100 (Piz Daint node)": 973, "V100 PCIe": 2271}
L2_FLUSH_BYTES = 256 << 20

WORKLOAD_TEXT = {
    "cfg1": "root + 8 leaf sub-grids (4096 cells), two Gaussians",
    "cfg2": "uniform level-3 octree, 64 leaf sub-grids (32768 cells), polytrope binary q=0.3",
    "cfg3": "adaptive octree to level 5 around a polytrope binary (q=0.3)",
    "cfg4": "16 independent adaptive octrees (levels 4-7, q=0.1..1.0) batched in one solve",
    "cfg5": "contact binary of two n=1.5 polytropes (q=0.3), adaptive octree to level 7",
    "cfg5_small": "cfg5's binary refined to level 6 (profiler captures)",
}


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    # 300 steps time about 0.9 s of solve: enough for several clock samples
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="cfg5")
    p.add_argument("--precision", choices=["mixed", "fp64", "dfloat"], default="mixed")
    p.add_argument("--fp64-steps", type=int, default=3)
    p.add_argument("--dfloat-steps", type=int, default=5)
    p.add_argument("--theta035-steps", type=int, default=5)
    # the other full-size workloads reported beside the headline one
    p.add_argument("--extra-workloads", default="cfg3,cfg4", help="comma-separated, or none")
    p.add_argument("--extra-steps", type=int, default=20)
    # the full FP64 oracle solve of the adaptive level-5 binary (cfg3), for
    # each precision's error against the oracle itself (about 20-40 s of CPU)
    p.add_argument("--no-oracle-accuracy", action="store_true")
    # leave out the dataflow, time-derivative and SCF timings
    p.add_argument("--no-extras", action="store_true")
    # a fixed launch tuning (JSON object of fmm_tuning fields) instead of the
    # autotuner's pick, e.g. so that a profiler's run has the plain run's shapes
    p.add_argument("--tuning", default=None)
    p.add_argument("--cpu-seconds", type=float, default=10.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    # other modes (no bench line): a minimal run of one pass for profiler
    # captures, and an opening-angle sweep
    p.add_argument("--profile-pass", choices=["upward", "m2l", "downward", "forces", "step"],
                   default=None, help="run one pass --reps times (for ncu) and exit")
    p.add_argument("--reps", type=int, default=1)
    p.add_argument("--mono-subgrids", type=int, default=2)
    p.add_argument("--theta-sweep", default=None,
                   help="comma-separated opening angles: time the step at each and exit")
    return p.parse_args()


# ------------------------------------------------------------- helpers
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, pci=None):
        self.proc = None
        self.path = None
        self.pci = pci

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
               "-lms", "100"]
        if self.pci:
            cmd += ["-i", self.pci]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)                   # the sample in flight at the end
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def rank_max(torch, dist, v, device):
    """The maximum of v over the ranks of the process group (v itself without
    one): replicas are timed by the slowest rank."""
    if dist is None:
        return v
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(interactions_per_step, world, ms_max):
    """Whole-job throughput of `world` independent replicas: every rank's
    interactions over the slowest rank's step time."""
    return interactions_per_step * world / (ms_max / 1000.0)


def measured_peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except (OSError, ValueError):
        return {}


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("fmm_m2l.cu", "fmm_tensor.cuh", "fmm_dfloat.cuh", "fmm_convert.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1908_03121_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, workload):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    path = os.path.join(PROFILES, f"{kernel}_{workload}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    src = re.search(r"source_hash:\s*([0-9a-f]+)", text)
    val = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not src or not val or src.group(1) != kernel_source_hash():
        return None
    return float(val.group(1))


# the same-level kernels and the interactions each evaluates (fmm_get_stats'
# kernel_interactions order)
M2L_KERNELS = (("multipole", "mp<-mp and mp<-mono (multipole kernel)"),
               ("monopole", "mono<-mono (monopole kernel)"),
               ("mono_multi", "mono<-mp (monopole<-multipole kernel)"),
               ("root", "root level, every kind (root kernel)"))


def m2l_rates_by_kernel(per_kernel, kernel_interactions):
    """Interactions/s of each same-level kernel: the interactions it evaluates
    per step over its measured ms per step (kernels that did not run are left
    out)."""
    rates = {}
    for (key, label), n in zip(M2L_KERNELS, kernel_interactions):
        ms = per_kernel.get(key, {}).get("ms_per_step", 0.0)
        if ms > 0 and n > 0:
            rates[label] = n / (ms / 1000.0)
    return rates


def per_cell_force_errors(g, g_ref, floor=1e-3):
    """Median and 99th percentile (nearest rank) of the per-cell relative
    force error |g - g_ref| / |g_ref|, vector norms over the three
    components, over the cells whose |g_ref| exceeds `floor` times the
    largest (g vanishes at the stars' centres).  g, g_ref: tensors
    [n_leaf][3][512] on any device."""
    d = (g - g_ref).double().norm(dim=1).flatten()
    r = g_ref.double().norm(dim=1).flatten()
    keep = r > floor * r.max()
    e = (d[keep] / r[keep]).sort().values
    n = int(e.numel())
    return {"median": float(e[(n - 1) // 2]), "p99": float(e[int(0.99 * (n - 1))]),
            "cells": n}


def workload_config(name, c, stats, sizes, precision):
    cells = int(sizes["n_leaf"]) * 512
    return {
        "workload": f"{name}: {WORKLOAD_TEXT.get(name, name)}; {sizes['n_nodes']} sub-grids, "
                    f"{sizes['n_leaf']} leaves ({cells} leaf cells), theta={c['theta']}, "
                    f"order 3, {precision}",
        "n_trees": int(sizes["n_trees"]),
        "n_nodes": int(sizes["n_nodes"]),
        "leaf_cells": cells,
        "theta": c["theta"],
        "interactions_per_step": int(sum(stats["interactions"])),
        "interactions_by_kind": {"mp<-mp": stats["interactions"][0],
                                 "mp<-mono": stats["interactions"][1],
                                 "mono<-mono": stats["interactions"][2],
                                 "mono<-mp": stats["interactions"][3]},
        "l2": "flushed (256 MiB write) before every timed step; working set > L2",
    }


# ------------------------------------------------------------ CPU oracle
def oracle_rate(c, seconds, batch=4096, seed=0, n_threads=None):
    """The FP64 oracle's same-level pass on random target cells of the workload,
    batch after batch until ``seconds`` elapse.  Returns (rate, info)."""
    from oracle import oracle as O
    tree = O.Tree.from_config(c)
    M, com = O.upward(tree, c["rho"])
    rng = np.random.default_rng(seed)
    n_threads = n_threads or os.cpu_count() or 1
    total_cells = tree.n * 512
    done = 0
    inter = 0
    t0 = time.perf_counter()
    while True:
        targets = np.sort(rng.choice(total_cells, size=batch, replace=False))
        _, _, counts = O.m2l(tree, M, com, targets=targets, n_threads=n_threads,
                            compact=True)
        done += batch
        inter += int(counts.sum())
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return inter / el, dict(cells=done, interactions=inter, seconds=el, cores=n_threads)


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from workloads import make_config
    c = make_config(args.workload)
    from oracle import oracle as O
    tree = O.Tree.from_config(c)
    M, com = O.upward(tree, c["rho"])
    n_threads = os.cpu_count() or 1
    rng = np.random.default_rng(1)
    batch = 2048
    total_cells = tree.n * 512

    def one_step():
        targets = np.sort(rng.choice(total_cells, size=batch, replace=False))
        t0 = time.perf_counter()
        _, _, counts = O.m2l(tree, M, com, targets=targets, n_threads=n_threads, compact=True)
        return time.perf_counter() - t0, int(counts.sum())

    for _ in range(args.warmup):
        one_step()
    times, inters = [], []
    for _ in range(args.steps):
        t, n = one_step()
        times.append(t)
        inters.append(n)
    value = sum(inters) / sum(times)
    ms = 1000.0 * sum(times) / len(times)
    sample = (f"FP64 oracle same-level pass over {batch} random target cells per step "
              f"(all levels) of {args.workload}, upward pass untimed")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": f"{args.workload}: {WORKLOAD_TEXT.get(args.workload)}",
                      "sample_cells_per_step": batch, "theta": c["theta"]},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": n_threads, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


# -------------------------------------------------------- measured peaks
def measure_peaks(torch, F, pci=None):
    """FP32 and FP64 fused multiply-add rates of this GPU: the library's
    fmm_peak_rate loop (every SM, 8 CTAs of 256 threads, 8 independent chains
    per thread), timed by CUDA events on the launch stream, best of several
    launches, with the SM clock sampled meanwhile.  Changes no GPU setting."""
    stream = torch.cuda.current_stream()
    sink = torch.zeros(1, dtype=torch.float32, device="cuda")
    out = {}
    clocks = ClockSampler(pci)
    clocks.start()
    for kind, iters, reps in (("fp32", 40000, 12), ("fp32x2", 20000, 6), ("fp64", 600, 6)):
        F.fmm_peak_rate(kind, iters, 8, sink)              # warm-up
        best = 0.0
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fl = F.fmm_peak_rate(kind, iters, 8, sink)
            b.record(stream)
            b.synchronize()
            best = max(best, fl / (a.elapsed_time(b) / 1000.0) / 1e12)
        out[kind + "_tflops"] = best
    torch.cuda.synchronize()
    out["clocks"] = clocks.stop()
    out["how"] = ("fmm_peak_rate: fused multiply-add loop on every SM (8 CTAs x 256 threads, "
                  "8 independent chains per thread), CUDA events, best launch")
    return out


# ------------------------------------------------------------ next rows
def _graph_ms(torch, solver, steps, flush, stream):
    solver.capture()
    _, per, _ = time_graph(torch, solver, steps, 2, flush, stream, label="extras")
    return float(np.median(per))


def _direct_field(pos, m, G=1.0):
    """O(N^2) point-mass field at the points (self term excluded), numpy."""
    g = np.zeros_like(pos)
    for s0 in range(0, len(pos), 256):
        d = pos[s0:s0 + 256, None, :] - pos[None, :, :]
        r2 = (d * d).sum(-1)
        idx = np.arange(s0, min(s0 + 256, len(pos)))
        r2[idx - s0, idx] = np.inf
        g[s0:s0 + 256] = -G * ((m[None, :] / r2 ** 1.5)[:, :, None] * d).sum(1)
    return g


def order_sweep(torch, F, autotune, c, flush, stream, steps=10):
    """Expansion orders 2 and 3: the headline workload's mixed-precision step
    (median ms, interactions/s; the field of order 2 against order 3), and
    each order's FP64 field against the O(N^2) direct sum on the 4096-cell
    two-Gaussian workload (cfg1)."""
    from workloads import make_config, leaf_cell_centres
    out = {}
    g = {}
    for order in (2, 3):
        s = F.Solver(c["desc"], c["theta"], precision="mixed", order=order)
        s.rho.copy_(torch.from_numpy(c["rho"]).cuda())
        s.step()
        autotune.tune(s, flush=flush)
        ms = _graph_ms(torch, s, steps, flush, stream)
        inter = int(sum(s.tree.stats["interactions"]))
        fl = s.tree.stats["flops_per_interaction"]
        g[order] = s.g.clone()
        out[f"order_{order}"] = {"ms_per_step": ms, "value": inter / (ms / 1000.0), "unit": UNIT,
                                 "flops_per_interaction": fl}
        s.close()
    out["field_difference_order2_vs_order3"] = float((g[2] - g[3]).abs().max() / g[3].abs().max())
    c1 = make_config("cfg1")
    pos = leaf_cell_centres(c1["desc"]).reshape(-1, 3)
    h = 1.0 / 16.0
    gd = _direct_field(pos, (c1["rho"] * h ** 3).reshape(-1))
    for order in (2, 3):
        s = F.Solver(c1["desc"], c1["theta"], precision="fp64", order=order)
        s.rho.copy_(torch.from_numpy(c1["rho"]).cuda())
        s.step()
        gg = s.g.cpu().numpy().transpose(0, 2, 1).reshape(-1, 3)
        out[f"order_{order}"]["cfg1_field_err_vs_direct_sum"] = float(
            np.abs(gg - gd).max() / np.abs(gd).max())
        s.close()
    return out


def dataflow_ab(torch, F, solver, best, flush, stream, steps=30):
    """The headline step with the dataflow downward pass on and off (all
    else at the tuned values), median ms of each."""
    out = {}
    for df in (0, 1):
        F.fmm_set_tuning(solver.tree, **dict(best, dataflow=df))
        out[f"ms_per_step_dataflow_{df}"] = _graph_ms(torch, solver, steps, flush, stream)
    F.fmm_set_tuning(solver.tree, **best)
    solver.graph = None
    return out


def time_derivative_timing(torch, F, autotune, c, flush, reps=3):
    """fmm_field_time_derivative on the headline workload (four solves) in
    FP64 and double-float, device ms per call, with rho_dot = rho sin(7 x)."""
    out = {}
    x = np.linspace(0.0, 1.0, c["rho"].size).reshape(c["rho"].shape)
    rd = torch.from_numpy(c["rho"] * np.sin(7.0 * x)).cuda()
    for prec in ("fp64", "dfloat"):
        s = F.Solver(c["desc"], c["theta"], precision=prec)
        s.rho.copy_(torch.from_numpy(c["rho"]).cuda())
        s.step()
        autotune.tune(s, flush=flush)
        pd, gd, work = torch.empty_like(s.phi), torch.empty_like(s.g), torch.empty_like(s.rho)
        s.time_derivative(rd, 1e-3, pd, gd, rho_work=work)
        ms = []
        for _ in range(reps):
            flush()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            s.time_derivative(rd, 1e-3, pd, gd, rho_work=work)
            b.record()
            b.synchronize()
            ms.append(a.elapsed_time(b))
        out[prec] = {"ms_per_call": float(np.median(ms)), "solves_per_call": 4}
        s.close()
    return out


def scf_timing(torch, F):
    """Self-consistent-field binary on a uniform level-4 tree (64^3 cells),
    FP64 and mixed solves: iterations to settle (Omega^2 and C to 1e-6) and
    wall ms per iteration (solve, the update's two host reads, the density
    kernels)."""
    from paper_1908_03121_gb300 import scf as D
    from workloads import uniform_tree
    from workloads.density import polytrope
    desc = uniform_tree(4)
    leaves = desc[desc[:, 5] < 0]
    h = 1.0 / 64.0
    cc = np.arange(512)
    loc = np.stack([cc & 7, (cc >> 3) & 7, cc >> 6], axis=1)
    pos = (8.0 * leaves[:, None, 1:4] + loc[None] + 0.5) * h
    c1, c2 = np.array([0.3, 0.5, 0.5]), np.array([0.72, 0.5, 0.5])
    rho0 = polytrope(pos, c1, 0.15, 1.0) + polytrope(pos, c2, 0.13, 0.5) + 1e-10
    p = D.binary_params(c1, 0.15, c2, 0.13, (1.0, 0.5), h)
    out = {"workload": "binary of two n=1.5 polytropes on a uniform level-4 tree (262144 cells)"}
    for prec in ("fp64", "mixed"):
        s = F.Solver(desc, 0.5, precision=prec)
        s.rho.copy_(torch.from_numpy(rho0).cuda())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res, k = D.solve(s, p, iters=80, tol=1e-6)
        torch.cuda.synchronize()
        out[prec] = {"iterations": k, "ms_per_iteration": 1000.0 * (time.perf_counter() - t0) / k,
                     "omega2": res["omega2"]}
        s.close()
    return out


# ----------------------------------------------------- other workloads
def net_sums(tot):
    """Largest net force and net torque over the trees, each relative to its
    normaliser (sum |f|, sum |x cross f|)."""
    return (float(np.max(np.linalg.norm(tot[:, 0:3], axis=1) / tot[:, 6])),
            float(np.max(np.linalg.norm(tot[:, 3:6], axis=1) / tot[:, 7])))


def other_workload(torch, F, autotune, name, args, flush, stream, keep):
    """One full-size workload in every precision: interactions/s of the
    captured, autotuned step (median of --extra-steps; FP64 of --fp64-steps),
    force error against the FP64 GPU path, net force and torque.  The fields
    are left in ``keep[name]`` (host arrays) for the oracle comparison."""
    from workloads import make_config
    cw = make_config(name)
    rho = torch.from_numpy(cw["rho"]).cuda()
    out = {"workload": f"{name}: {WORKLOAD_TEXT.get(name, name)}"}
    got = {}
    for prec in ("mixed", "dfloat", "fp64"):
        sw = F.Solver(cw["desc"], cw["theta"], precision=prec)
        st, sz = sw.tree.stats, sw.tree.sizes
        sw.rho.copy_(rho)
        sw.step()
        tuning = autotune.tune(sw, flush=flush)[0]
        sw.capture()
        steps = max(1, args.fp64_steps) if prec == "fp64" else args.extra_steps
        ms, _, _ = time_graph(torch, sw, steps, 2, flush, stream, label=f"{name}_{prec}")
        inter = int(sum(st["interactions"]))
        nf, nt = net_sums(sw.totals.double().cpu().numpy())
        got[prec] = sw.g.clone()
        out[prec] = {"value": inter / (ms / 1000.0), "unit": UNIT, "ms_per_step": ms,
                     "net_force": nf, "net_torque": nt, "tuning": tuning}
        out["n_trees"], out["n_nodes"], out["leaf_cells"] = (int(sz["n_trees"]), int(sz["n_nodes"]),
                                                             int(sz["n_leaf"]) * 512)
        out["interactions_per_step"] = inter
        sw.close()
    g64 = got["fp64"]
    for prec in ("mixed", "dfloat"):
        out[prec]["force_err_vs_fp64_path"] = float((got[prec] - g64).abs().max() / g64.abs().max())
        out[prec]["force_err_per_cell_p99"] = per_cell_force_errors(got[prec], g64)["p99"]
        out[prec]["speedup_over_fp64"] = out["fp64"]["ms_per_step"] / out[prec]["ms_per_step"]
    keep[name] = {k: v.cpu().numpy() for k, v in got.items()}
    return out


def oracle_accuracy(name, fields):
    """Each precision's field against the complete FP64 oracle solve of the
    workload: max |g - g_oracle| / max |g_oracle| over every leaf cell, and the
    per-cell 99th percentile."""
    import torch
    from oracle import oracle as O
    from workloads import make_config
    c = make_config(name)
    t0 = time.perf_counter()
    ref = O.solve(O.Tree.from_config(c), c["rho"])
    gref = ref["g"]
    out = {"workload": name, "oracle_seconds": time.perf_counter() - t0,
           "oracle_cores": os.cpu_count()}
    for prec, g in fields.items():
        out[prec] = {"force_err": float(np.abs(g - gref).max() / np.abs(gref).max()),
                     "force_err_per_cell_p99": per_cell_force_errors(
                         torch.from_numpy(g), torch.from_numpy(gref))["p99"]}
    return out


# ------------------------------------------------------------------- ours
def time_graph(torch, solver, steps, warmup, flush, stream, clocks=None, label="timed_steps"):
    """Per-step device ms of graph replays; the L2 flush runs between steps,
    outside the events."""
    for _ in range(warmup):
        flush()
        solver.replay()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if clocks:
        clocks.start()
    # the NVTX range lets a profiler's launch list keep the timed steps only
    # (ncu --nvtx --nvtx-include "<label>/")
    torch.cuda.nvtx.range_push(label)
    for k in range(steps):
        flush()
        starts[k].record(stream)
        solver.replay()
        ends[k].record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop() if clocks else None
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    return float(np.median(ms)), ms, clk


def run_ours(args):
    import torch
    import paper_1908_03121_gb300 as F
    from workloads import make_config

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(v):
        return rank_max(torch, dist, v, "cuda")

    c = make_config(args.workload)
    rho_host = torch.from_numpy(c["rho"]).pin_memory()
    flush_buf = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    flush_val = [0]

    def flush():
        flush_val[0] = (flush_val[0] + 1) & 0xFF
        flush_buf.fill_(flush_val[0])

    stream = torch.cuda.current_stream()
    solver = F.Solver(c["desc"], c["theta"], precision=args.precision)
    stats, sizes = solver.tree.stats, solver.tree.sizes
    interactions = int(sum(stats["interactions"]))
    solver.rho.copy_(rho_host.cuda())
    from paper_1908_03121_gb300 import autotune
    solver.step()
    if args.tuning:
        best = json.loads(args.tuning)
        F.fmm_set_tuning(solver.tree, **best)
    else:
        best, tune_results = autotune.tune(solver, reps=7, flush=flush)
    solver.capture()
    pci = None
    try:
        pci = torch.cuda.get_device_properties(local).pci_bus_id
    except Exception:
        pass
    barrier()
    torch.cuda.synchronize()
    ms, per_step, clk = time_graph(torch, solver, args.steps, args.warmup, flush, stream,
                                   ClockSampler(pci) if rank == 0 else None)
    torch.cuda.synchronize()
    barrier()
    ms_max = max_over_ranks(ms)
    value = replica_value(interactions, world, ms_max)

    # end to end through the public API, every step: the density from pinned
    # host memory, the totals back to pinned host memory.  Three ways:
    # - one step at a time with a synchronisation on both sides, the density
    #   copied to the device first;
    # - the same, with the step's P2M kernel reading the pinned density itself
    #   (over the host link; the step reads the density nowhere else);
    # - a stream of steps (Solver.run_stream): step k + 1's density copied on
    #   a copy stream while step k computes, every step's totals read back on
    #   the host one step later, the L2 flush enqueued before every step
    #   inside the timed region.  The inputs alternate between two densities.
    # The line reports the fastest.
    tot_host = torch.empty_like(solver.totals, device="cpu").pin_memory()

    def e2e_run(copy_in):
        out = []
        for k in range(args.warmup + args.steps):
            flush()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if copy_in:
                solver.rho.copy_(rho_host, non_blocking=True)
            solver.replay()
            tot_host.copy_(solver.totals, non_blocking=True)
            torch.cuda.synchronize()
            if k >= args.warmup:
                out.append(1000.0 * (time.perf_counter() - t0))
        return max_over_ranks(float(np.mean(out)))

    rho_host2 = (rho_host * 1.001).pin_memory()
    seen = []

    def consume(k, totals):
        seen.append(bool(torch.isfinite(totals).all()))

    def e2e_stream():
        solver.run_stream([rho_host, rho_host2] * 2, consume, flush)     # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        solver.run_stream([rho_host2, rho_host] * (args.steps // 2) + [rho_host] * (args.steps % 2),
                          consume, flush)
        torch.cuda.synchronize()
        ms_step = 1000.0 * (time.perf_counter() - t0) / args.steps
        if not all(seen):
            raise RuntimeError("non-finite totals in the streamed steps")
        return max_over_ranks(ms_step)

    e2e_copy_ms = e2e_run(True)
    solver.capture(rho=rho_host)          # the graph now reads the pinned density
    e2e_direct_ms = e2e_run(False)
    solver.capture()                      # back to the device copy for what follows
    e2e_stream_ms = e2e_stream()
    solver.rho.copy_(rho_host)            # the density the later checks expect
    solver.capture()
    paths = {"separate host-to-device copy": e2e_copy_ms,
             "P2M reads the pinned host density": e2e_direct_ms,
             "stream of steps, next density copied during this step": e2e_stream_ms}
    e2e_path = min(paths, key=paths.get)
    e2e_ms_max = paths[e2e_path]
    e2e = {"value": replica_value(interactions, world, e2e_ms_max), "unit": UNIT,
           "h2d_bytes_per_step": int(rho_host.numel() * 8),
           "d2h_bytes_per_step": int(tot_host.numel() * 8),
           "ms_per_step": e2e_ms_max,
           "input_path": e2e_path,
           "ms_per_step_separate_copy": e2e_copy_ms,
           "ms_per_step_direct_read": e2e_direct_ms,
           "ms_per_step_streamed": e2e_stream_ms}

    # accuracy and conservation of this run, against the FP64 GPU path
    g_mixed = solver.g.clone()
    tot = solver.totals.double().cpu().numpy()
    net_torque = float(np.max(np.linalg.norm(tot[:, 3:6], axis=1) / tot[:, 7]))
    net_force = float(np.max(np.linalg.norm(tot[:, 0:3], axis=1) / tot[:, 6]))
    solver.graph = None

    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
              "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
              "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
              "config": dict(workload_config(args.workload, c, stats, sizes, args.precision),
                             parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                             tuning=best)}
    result["e2e"] = e2e
    # (counted under the tuning the timed steps ran with)
    result["gpu_launches"] = int(F.fmm_get_stats(solver.tree)["launches_fused"]) * args.steps
    result["clocks"] = clk

    if rank == 0:
        # per-kernel device times, measured live with events on the launch stream
        def kernel_times(precision, tuning, nrep):
            tsolver = F.Solver(c["desc"], c["theta"], precision=precision, timing=True)
            F.fmm_set_tuning(tsolver.tree, **tuning)
            tsolver.rho.copy_(solver.rho)
            for _ in range(2):
                flush()
                tsolver.step()
            tsolver.kernel_times()          # discard warm-up timings
            for _ in range(nrep):
                flush()
                tsolver.step()
            kt = tsolver.kernel_times()
            tsolver.close()
            out = {k: {"ms_per_launch": (v[0] / v[1]) if v[1] else 0.0,
                       "ms_per_step": v[0] / nrep, "launches_per_step": v[1] / nrep}
                   for k, v in kt.items() if v[1]}
            total = sum(v["ms_per_step"] for v in out.values())
            for v in out.values():
                v["share"] = v["ms_per_step"] / total if total else 0.0
            return out

        peaks = measure_peaks(torch, F, pci)
        result["peaks"] = peaks
        per_kernel = kernel_times(args.precision, best, max(3, min(args.steps, 20)))
        result["kernels"] = per_kernel
        inter = stats["interactions"]
        kin = stats["kernel_interactions"]
        fl = stats["flops_per_interaction"]
        # the multipole kernel evaluates every multipole-target pair except the
        # root level's (all multipole<-multipole), which the root kernel takes
        work = {"multipole": (kin[0] - inter[1]) * fl[0] + inter[1] * fl[1],
                "monopole": kin[1] * fl[2],
                "mono_multi": kin[2] * fl[3]}
        dom = max(work, key=lambda k: per_kernel.get(k, {}).get("ms_per_step", 0.0))
        dom_ms = per_kernel[dom]["ms_per_launch"]
        achieved = work[dom] / (dom_ms / 1000.0) / 1e12
        # the same-level kernels of the mixed and double-float precisions run
        # on the FP32 pipe, the FP64 precision's on the FP64 pipe: the peak is
        # that pipe's fused multiply-add rate measured above on this GPU
        if args.precision in ("mixed", "dfloat"):
            peak = peaks["fp32_tflops"]
            which = (f"measured FP32 FMA loop ({peak:.1f} TFLOP/s; derived from unit counts "
                     f"and the 2.07 GHz clock: {FP32_PEAK_TFLOPS:.1f})")
        else:
            peak = peaks["fp64_tflops"]
            which = f"measured FP64 FMA loop ({peak:.2f} TFLOP/s; nominal {FP64_PEAK_TFLOPS})"
        result["roofline"] = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak,
                              "unit": "TFLOP/s", "frac": achieved / peak,
                              "traffic": profiled_traffic(dom, args.workload),
                              "peak_source": which,
                              "flops_per_launch": work[dom],
                              "flops_per_interaction": fl}
        result["m2l_interactions_per_s"] = interactions / (
            sum(per_kernel.get(k, {}).get("ms_per_step", 0.0)
                for k in ("pack", "root", "multipole", "monopole", "mono_multi")) / 1000.0)
        result["m2l_interactions_per_s_by_kernel"] = m2l_rates_by_kernel(per_kernel, kin)

        # FP64 GPU path on the same workload: rate and the mixed path's error
        if args.precision == "mixed" and args.fp64_steps > 0:
            s64 = F.Solver(c["desc"], c["theta"], precision="fp64")
            s64.rho.copy_(solver.rho)
            s64.step()
            autotune.tune(s64, flush=flush)
            s64.capture()
            ms64, _, _ = time_graph(torch, s64, args.fp64_steps, 1, flush, stream,
                                   label="fp64_steps")
            g64 = s64.g
            err = float((g_mixed - g64).abs().max() / g64.abs().max())
            tot64 = s64.totals.cpu().numpy()
            result["fp64_path"] = {
                "value": interactions / (ms64 / 1000.0), "ms_per_step": ms64,
                "speedup_mixed_over_fp64": ms64 / ms,
                "net_torque": float(np.max(np.linalg.norm(tot64[:, 3:6], axis=1) / tot64[:, 7]))}
            pc = per_cell_force_errors(g_mixed, g64)
            result["mixed_accuracy"] = {"force_err_vs_fp64_path": err,
                                        "force_err_per_cell_median": pc["median"],
                                        "force_err_per_cell_p99": pc["p99"],
                                        "net_torque": net_torque, "net_force": net_force}
            # the conserving (double-float) precision on the same workload
            if args.dfloat_steps > 0:
                sdf = F.Solver(c["desc"], c["theta"], precision="dfloat")
                sdf.rho.copy_(solver.rho)
                sdf.step()
                best_df = autotune.tune(sdf, flush=flush)[0]
                sdf.capture()
                msdf, _, _ = time_graph(torch, sdf, args.dfloat_steps, 1, flush, stream,
                                        label="dfloat_steps")
                totdf = sdf.totals.cpu().numpy()
                result["conserving_path"] = {
                    "precision": "dfloat (float pairs on the FP32 pipe)",
                    "value": interactions / (msdf / 1000.0), "unit": UNIT, "ms_per_step": msdf,
                    "speedup_over_fp64": ms64 / msdf,
                    "force_err_vs_fp64_path": float((sdf.g - g64).abs().max() / g64.abs().max()),
                    "force_err_per_cell_p99": per_cell_force_errors(sdf.g, g64)["p99"],
                    "net_force": float(np.max(np.linalg.norm(totdf[:, 0:3], axis=1) / totdf[:, 6])),
                    "net_torque": float(np.max(np.linalg.norm(totdf[:, 3:6], axis=1) / totdf[:, 7]))}
                sdf.close()
                result["conserving_path"]["kernels"] = {
                    k: round(v["ms_per_step"], 4) for k, v in kernel_times("dfloat", best_df, 3).items()}
            s64.close()

        # the paper's production opening angle (theta = 0.35, the 1074-point
        # stencil of Sec. 4.3) on the same tree and density, mixed precision
        if args.precision == "mixed" and args.theta035_steps > 0:
            s35 = F.Solver(c["desc"], 0.35, precision="mixed")
            s35.rho.copy_(solver.rho)
            s35.step()
            autotune.tune(s35, flush=flush)
            s35.capture()
            ms35, _, _ = time_graph(torch, s35, args.theta035_steps, 1, flush, stream,
                                    label="theta035_steps")
            st35 = s35.tree.stats
            inter35 = int(sum(st35["interactions"]))
            target_cells = int(s35.tree.sizes["n_nodes"]) * 512
            sz35 = s35.tree.sizes
            union = int(st35["stencil_union"])
            # the paper's accounting (Sec. 4.3, Sec. 6.1): every sub-grid's
            # kernel evaluates the whole superimposed stencil for its 512
            # cells, at 455 operations per point for a multipole target and
            # 12 for a monopole target, over the step time
            paper_ops = 512 * union * (int(sz35["n_refined"]) * PAPER_FLOPS_MULTIPOLE +
                                       int(sz35["n_leaf"]) * PAPER_FLOPS_MONOPOLE)
            result["theta_0.35"] = {
                "value": inter35 / (ms35 / 1000.0), "unit": UNIT, "ms_per_step": ms35,
                "interactions_per_step": inter35,
                "stencil_union": union,
                "paper_equivalent_stencil_evaluations_per_s": union * target_cells / (ms35 / 1000.0),
                "paper_gflops": paper_ops / (ms35 / 1000.0) / 1e9,
                "paper_table2_gflops_fp64_context": PAPER_TABLE2_GFLOPS,
                "note": "paper-equivalent = 1074-point stencil x all target cells / step time; "
                        "paper_gflops = the same points x 455 (multipole targets) or 12 "
                        "(monopole targets) / step time, the paper's own accounting"}
            s35.close()

        # the next rows on the headline workload: the dataflow downward pass
        # against the level launches (N3), the field's time derivative (N2),
        # and self-consistent-field iterations (N4)
        if not args.no_extras:
            result["order_sweep"] = order_sweep(torch, F, autotune, c, flush, stream)
            result["dataflow"] = dataflow_ab(torch, F, solver, best, flush, stream)
            result["time_derivative"] = time_derivative_timing(torch, F, autotune, c, flush)
            result["scf"] = scf_timing(torch, F)

        # the other full-size workloads: each precision through the captured,
        # autotuned step (median of --extra-steps), with its error against
        # the FP64 GPU path and its net force and torque
        extra = [w for w in args.extra_workloads.split(",") if w not in ("", "none", args.workload)]
        accuracy_ref = {}
        for wname in extra:
            result[wname] = other_workload(torch, F, autotune, wname, args, flush, stream,
                                           accuracy_ref)
        if world == 1 and not args.no_cpu_baseline:
            # the CPU-oracle leg: the oracle's rate on the host cores, and its
            # complete solve of cfg3 for every precision's error against it
            if not args.no_oracle_accuracy and "cfg3" in accuracy_ref:
                result["accuracy_vs_oracle"] = oracle_accuracy("cfg3", accuracy_ref["cfg3"])
            rate, info = oracle_rate(c, args.cpu_seconds)
            rate1, info1 = oracle_rate(c, max(2.0, args.cpu_seconds / 2), batch=256, n_threads=1)
            result["cpu_baseline"] = {
                "value": rate, "unit": UNIT, "cores": info["cores"], "kind": "oracle",
                "sample": f"FP64 oracle same-level pass over {info['cells']} random target "
                          f"cells of {args.workload} ({info['interactions']} interactions, "
                          f"{info['seconds']:.1f} s), upward pass untimed",
                "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                                  "sample": f"{info1['cells']} random target cells "
                                            f"({info1['interactions']} interactions, "
                                            f"{info1['seconds']:.1f} s)"}}
        print(json.dumps(result), flush=True)
    solver.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------ profiling driver
def run_profile_pass(args):
    """The smallest program around one pass, for profiler captures: the
    chosen workload's buffers, one upward pass, then the pass --reps times.
    No graph, no timing tree, no oracle."""
    import torch
    import paper_1908_03121_gb300 as F
    from workloads import make_config

    c = make_config(args.workload)
    s = F.Solver(c["desc"], c["theta"], precision=args.precision)
    if args.tuning:
        F.fmm_set_tuning(s.tree, **json.loads(args.tuning))
    else:
        F.fmm_set_tuning(s.tree, mono_subgrids=args.mono_subgrids)
    s.rho.copy_(torch.from_numpy(c["rho"]).cuda())
    s.upward()
    if args.profile_pass in ("downward", "forces"):
        s.m2l()
    if args.profile_pass == "forces":
        s.downward()
    run = {"upward": s.upward, "m2l": s.m2l, "downward": s.downward, "forces": s.forces,
           "step": s.step}[args.profile_pass]
    for _ in range(args.reps):
        run()
    torch.cuda.synchronize()
    print(f"{args.workload} {args.precision} {args.profile_pass} x{args.reps}: ok", flush=True)
    s.close()
    return 0


# ---------------------------------------------------- opening-angle sweep
def run_theta_sweep(args):
    """The whole step at each opening angle: the tree planned anew (reach,
    far/near offsets per parity, their union: 1074 at theta = 0.35), the
    autotuned step captured and replayed with an L2 flush before each timed
    replay, median of --steps; the FP64 path beside it for the speedup and the
    field error, and the net force and torque.  One JSON object per angle,
    then a markdown table."""
    import torch
    import paper_1908_03121_gb300 as F
    from paper_1908_03121_gb300 import autotune
    from workloads import make_config

    stream = torch.cuda.current_stream()
    flush_buf = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def flush():
        flush_buf.fill_(1)

    def net(tot):
        return (float(np.max(np.linalg.norm(tot[:, 0:3], axis=1) / tot[:, 6])),
                float(np.max(np.linalg.norm(tot[:, 3:6], axis=1) / tot[:, 7])))

    rows = []
    for theta in [float(t) for t in args.theta_sweep.split(",")]:
        c = make_config(args.workload, theta=theta)
        rho = torch.from_numpy(c["rho"]).cuda()
        s = F.Solver(c["desc"], c["theta"], precision=args.precision)
        st = s.tree.stats
        inter = int(sum(st["interactions"]))
        s.rho.copy_(rho)
        s.step()
        autotune.tune(s, flush=flush)
        s.capture()
        _, per, _ = time_graph(torch, s, args.steps, 2, flush, stream, label="theta_sweep")
        ms = float(np.median(per))
        g_ours = s.g.clone()
        nf, nt = net(s.totals.cpu().numpy())
        cells = int(s.tree.sizes["n_nodes"]) * 512          # every target cell
        s.close()
        s64 = F.Solver(c["desc"], c["theta"], precision="fp64")
        s64.rho.copy_(rho)
        s64.step()
        s64.capture()
        _, per64, _ = time_graph(torch, s64, max(1, args.fp64_steps), 1, flush, stream,
                                 label="theta_sweep_fp64")
        ms64 = float(np.median(per64))
        err = float((g_ours - s64.g).abs().max() / s64.g.abs().max())
        s64.close()
        row = {"theta": theta, "precision": args.precision, "reach": int(st["reach"]),
               "stencil_far": int(st["stencil_far"]), "stencil_near": int(st["stencil_near"]),
               "stencil_union": int(st["stencil_union"]), "interactions_per_step": inter,
               "ms_per_step": ms, "interactions_per_s": inter / (ms / 1000.0),
               "paper_equivalent_evals_per_s": st["stencil_union"] * cells / (ms / 1000.0),
               "fp64_ms_per_step": ms64, "speedup_over_fp64": ms64 / ms,
               "force_err_vs_fp64": err, "net_force": nf, "net_torque": nt}
        rows.append(row)
        print(json.dumps(row), flush=True)
    print()
    print("| theta | reach | far + near per parity | union | interactions / step | ms | "
          "interactions/s | paper-equivalent evals/s | FP64 ms | speedup | force err | net torque |")
    print("|---:|---:|---:|---:|---:|---:|---:|---:|---:|---:|---:|---:|")
    for r in rows:
        print(f"| {r['theta']} | {r['reach']} | {r['stencil_far']} + {r['stencil_near']} | "
              f"{r['stencil_union']} | {r['interactions_per_step']:,} | {r['ms_per_step']:.2f} | "
              f"{r['interactions_per_s']:.3g} | {r['paper_equivalent_evals_per_s']:.3g} | "
              f"{r['fp64_ms_per_step']:.1f} | {r['speedup_over_fp64']:.1f}x | "
              f"{r['force_err_vs_fp64']:.1e} | {r['net_torque']:.1e} |")
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_pass:
        return run_profile_pass(args)
    if args.theta_sweep:
        return run_theta_sweep(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
