"""Profiling driver: the 8-sphere workload of the benchmark (same geometry
recipe and solver settings) on a 2^n grid for a fixed number of iterations,
all load cases side by side, with a workspace sized for the grid. Meant to
run under ncu (kernel launch lists, single-kernel captures) where the full
benchmark's workspace and launch count are too large.

    python -m paper_2412_11566_gb300.profile_case --n 8 --iters 2 --loads 6
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=6)
    ap.add_argument("--iters", type=int, default=2)
    ap.add_argument("--loads", type=int, default=6)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--workspace-gb", type=float, default=0.0,
                    help="0 = sized from the grid")
    args = ap.parse_args()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import __graft_entry__ as ge
    ge.build()
    from paper_2412_11566_gb300 import qtt as Q, synth

    w = synth.spheres256(n=args.n)
    cells = 1 << (3 * args.n)
    ws = args.workspace_gb or max(2.0, 36 * 16 * cells * 3.3 / 2 ** 30 + 2.0 * args.loads)
    prec = Q.QTT_FP32 if args.precision == "fp32" else Q.QTT_FP64
    ctx = Q.Context(0, prec, int(ws * 2 ** 30), seed=2412)
    ctx.set_concurrency(args.loads)
    t = time.perf_counter()
    dC = Q.qtt_from_phase_field(ctx, w.phase, w.n, w.E, w.nu, None, w.eps_tt, w.rmax)
    params = Q.solve_params(1e-300, args.iters, w.eps_tt, w.rmax, 0, 16)
    C, infos, rc = Q.ls_solve_ceff(ctx, dC, params, loads=list(range(args.loads)))
    ctx.torch.cuda.synchronize()
    print(f"n={args.n} loads={args.loads} iters={args.iters} workspace={ws:.1f} GiB "
          f"wall={time.perf_counter() - t:.2f}s launches={ctx.launches()} "
          f"peak={ctx.bytes_peak() / 2 ** 30:.2f} GiB", flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
