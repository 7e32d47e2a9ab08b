"""Opening-angle sweep of the whole solve step on one workload.

For each theta, the tree is planned anew. That gives the stencil reach, the
per-parity far/near offsets and their union, which is 1074 points at the
paper's theta = 0.35. The step is then timed as `bench.py` times it: the
autotuned `fmm_step` is captured into a CUDA graph and replayed, with a
256 MiB L2 flush before every timed replay and CUDA events on the launch
stream. The mixed precision is timed, the FP64 path beside it, and the mixed
field's error and net force / torque are reported against the FP64 path.

Usage (GB300):
    python -m paper_1908_03121_gb300.theta_sweep --workload cfg5 --thetas 0.3,0.35,0.4,0.5,0.55

Prints one JSON object per theta, then a markdown table.
"""

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _time(torch, solver, steps, flush, stream):
    for _ in range(2):
        flush()
        solver.replay()
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        solver.replay()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return float(np.median(ms))


def _net(tot):
    return (float(np.max(np.linalg.norm(tot[:, 0:3], axis=1) / tot[:, 6])),
            float(np.max(np.linalg.norm(tot[:, 3:6], axis=1) / tot[:, 7])))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cfg5")
    ap.add_argument("--thetas", default="0.3,0.35,0.4,0.5,0.55")
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--fp64-steps", type=int, default=2)
    args = ap.parse_args()

    import torch
    import paper_1908_03121_gb300 as F
    from paper_1908_03121_gb300 import autotune
    from workloads import make_config

    stream = torch.cuda.current_stream()
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    val = [0]

    def flush():
        val[0] = (val[0] + 1) & 0xFF
        flush_buf.fill_(val[0])

    rows = []
    for theta in [float(t) for t in args.thetas.split(",")]:
        c = make_config(args.workload, theta=theta)
        rho = torch.from_numpy(c["rho"]).cuda()
        s = F.Solver(c["desc"], c["theta"], precision="mixed")
        st = s.tree.stats
        inter = int(sum(st["interactions"]))
        s.rho.copy_(rho)
        s.step()
        autotune.tune(s)
        s.capture()
        ms = _time(torch, s, args.steps, flush, stream)
        g_mixed = s.g.clone()
        nf, nt = _net(s.totals.cpu().numpy())
        cells = int(s.tree.sizes["n_nodes"]) * 512          # every target cell
        s.close()
        s64 = F.Solver(c["desc"], c["theta"], precision="fp64")
        s64.rho.copy_(rho)
        s64.step()
        s64.capture()
        ms64 = _time(torch, s64, args.fp64_steps, flush, stream)
        err = float((g_mixed - s64.g).abs().max() / s64.g.abs().max())
        s64.close()
        row = {"theta": theta, "reach": int(st["reach"]),
               "stencil_far": int(st["stencil_far"]), "stencil_near": int(st["stencil_near"]),
               "stencil_union": int(st["stencil_union"]), "interactions_per_step": inter,
               "ms_per_step": ms, "interactions_per_s": inter / (ms / 1000.0),
               "paper_equivalent_evals_per_s": st["stencil_union"] * cells / (ms / 1000.0),
               "fp64_ms_per_step": ms64, "speedup_over_fp64": ms64 / ms,
               "force_err_vs_fp64": err, "net_force": nf, "net_torque": nt}
        rows.append(row)
        print(json.dumps(row), flush=True)
    print()
    print("| theta | reach | far + near per parity | union | interactions / step | mixed ms | "
          "interactions/s | paper-equivalent evals/s | FP64 ms | speedup | force err | net torque |")
    print("|---:|---:|---:|---:|---:|---:|---:|---:|---:|---:|---:|---:|")
    for r in rows:
        print(f"| {r['theta']} | {r['reach']} | {r['stencil_far']} + {r['stencil_near']} | "
              f"{r['stencil_union']} | {r['interactions_per_step']:,} | {r['ms_per_step']:.2f} | "
              f"{r['interactions_per_s']:.3g} | {r['paper_equivalent_evals_per_s']:.3g} | "
              f"{r['fp64_ms_per_step']:.1f} | {r['speedup_over_fp64']:.1f}x | "
              f"{r['force_err_vs_fp64']:.1e} | {r['net_torque']:.1e} |")


if __name__ == "__main__":
    main()
