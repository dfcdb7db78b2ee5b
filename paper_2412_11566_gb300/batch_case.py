"""Batched C_eff throughput: aligned-fibre microstructures (the batched
training-data workload: fibres along x3, volume fraction U(0.3, 0.5),
contrast U(5, 50), seeds 2413 + i, grid sizes 2^n with n in {6, 7, 8, 9})
solved with ls_solve_batched in FP32 mode, all six loads per item.

    python -m paper_2412_11566_gb300.batch_case --items 12 --max-n 8 --lanes 24 --iters 60

Prints one JSON line: items, grid sizes, solves/s, iterations and residuals."""
from __future__ import annotations

import argparse
import json
import os
import sys
import time


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--items", type=int, default=12)
    ap.add_argument("--max-n", type=int, default=8)
    ap.add_argument("--lanes", type=int, default=24)
    ap.add_argument("--iters", type=int, default=60)
    ap.add_argument("--workspace-gb", type=float, default=120.0)
    args = ap.parse_args()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import __graft_entry__ as ge
    ge.build()
    import torch
    from paper_2412_11566_gb300 import qtt as Q, synth

    pool = [w for w in synth.fibre_batch(4 * args.items) if w.n <= args.max_n]
    items = pool[: args.items]
    ctx = Q.Context(0, Q.QTT_FP32, int(args.workspace_gb * 2 ** 30), seed=2412)
    t = time.perf_counter()
    dCs = [Q.qtt_from_phase_field(ctx, w.phase, w.n, w.E, w.nu, None, w.eps_tt, w.rmax)
           for w in items]
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t
    p = Q.solve_params(items[0].tol, args.iters, items[0].eps_tt, items[0].rmax)
    ctx.set_concurrency(args.lanes)
    Q.ls_solve_batched(ctx, dCs[:1], p)   # operators of the first grid and medium built here
    t = time.perf_counter()
    C, infos, rc = Q.ls_solve_batched(ctx, dCs, p)
    dt = time.perf_counter() - t
    solves = 6 * len(items)
    print(json.dumps({
        "items": len(items), "n": [w.n for w in items], "lanes": args.lanes,
        "max_iter": args.iters, "solves": solves, "seconds": round(dt, 2),
        "solves_per_s": solves / dt, "stiffness_builds_s": round(t_build, 2),
        "iters": [[f["iters"] for f in row] for row in infos],
        "max_residual": max(f["residual"] for row in infos for f in row),
        "rank_cap_hit": any(f["rank_cap_hit"] for row in infos for f in row),
        "note": "time includes the Green/SFFT builds of grids and media not seen before"}),
        flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
