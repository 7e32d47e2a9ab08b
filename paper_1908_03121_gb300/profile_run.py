"""Minimal driver for ncu captures of one pass of the solve.

Allocates only what the chosen pass needs, runs the upward pass once, then the
chosen pass ``--reps`` times; no graph, no timing trees, no oracle:

  python -m paper_1908_03121_gb300.profile_run --workload cfg5 --pass m2l --reps 2
"""

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cfg5")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "dfloat", "fp64"])
    ap.add_argument("--pass", dest="which", default="m2l",
                    choices=["upward", "m2l", "downward", "forces", "step"])
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--mono-subgrids", type=int, default=2)
    args = ap.parse_args()

    import torch
    import paper_1908_03121_gb300 as F
    from workloads import make_config

    c = make_config(args.workload)
    s = F.Solver(c["desc"], c["theta"], precision=args.precision)
    F.fmm_set_tuning(s.tree, mono_subgrids=args.mono_subgrids)
    s.rho.copy_(torch.from_numpy(c["rho"]).cuda())
    s.upward()
    if args.which in ("downward", "forces"):
        s.m2l()
    if args.which == "forces":
        s.downward()
    for _ in range(args.reps):
        if args.which == "upward":
            s.upward()
        elif args.which == "m2l":
            s.m2l()
        elif args.which == "downward":
            s.downward()
        elif args.which == "forces":
            s.forces()
        else:
            s.step()
    torch.cuda.synchronize()
    print(f"{args.workload} {args.precision} {args.which} x{args.reps}: ok")
    s.close()


if __name__ == "__main__":
    main()
