"""Writes tests/golden/<workload>_ceff_tol<tol>.json: the C_eff columns of a
named benchmark workload by the dense FFT basic scheme (oracle A, Alg. 1,
fp64) at the workload's stop tolerance. Calls only oracle/ and the seeded
geometry generator. Run from the repo root:

    python tests/golden/make_ceff_golden.py --workload lamfib256 [--tol 1e-4] [--loads 0,1,2,3,4,5]
    python tests/golden/make_ceff_golden.py --family lamfib256 --items 64

With --family the items of synth.lamfib_family (n = 8) are written to
tests/golden/<family>_family_ceff_tol<tol>.json under "items" (item index ->
its columns).

A phase field with a broadcast axis (extent 1) is solved on its reduced grid,
which is the same discrete problem as the full grid (its Fourier content lies
at frequency 0 along that axis; pinned by
tests/test_oracle_dense.py::test_broadcast_grid_equals_full_grid).
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import dense  # noqa: E402
from paper_2412_11566_gb300 import synth  # noqa: E402


def solve_columns(w, loads, tol, dst):
    """Adds the missing load columns of workload w to the dict dst."""
    lam0, mu0 = dense.reference_lame(w.E, w.nu)
    green = None
    for k in loads:
        if str(k) in dst:
            continue
        if green is None:
            green = dense.green_field(w.phase.shape, lam0, mu0)
        t = time.time()
        r = dense.basic_scheme(w.phase, w.E, w.nu, np.eye(6)[k], tol=tol, max_iter=5000,
                               green=green)
        dst[str(k)] = {"sigma_bar_re": r["sigma_bar"].real.tolist(),
                       "sigma_bar_im": r["sigma_bar"].imag.tolist(),
                       "iters": r["iters"], "history": r["history"],
                       "seconds": time.time() - t}
        print(f"{w.name} load {k}: {r['iters']} iterations, {time.time() - t:.0f} s", flush=True)
        yield


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="spheres256")
    ap.add_argument("--family", default=None)
    ap.add_argument("--items", type=int, default=64)
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--loads", default="0,1,2,3,4,5")
    args = ap.parse_args()
    loads = [int(v) for v in args.loads.split(",")]
    if args.family:
        assert args.family == "lamfib256"
        ws = synth.lamfib_family(8, args.items)
        out_path = os.path.join(os.path.dirname(__file__),
                                f"{args.family}_family_ceff_tol{args.tol:g}.json")
        res = json.load(open(out_path)) if os.path.exists(out_path) else {
            "_about": f"C_eff columns of the items of synth.lamfib_family(8) by oracle A (dense "
                      f"FFT basic scheme, Alg. 1, fp64), written by "
                      f"tests/golden/make_ceff_golden.py",
            "n": 8, "tol": args.tol, "items": {}}
        for i, w in enumerate(ws):
            item = res["items"].setdefault(str(i), {"name": w.name, "E": list(w.E),
                                                    "nu": list(w.nu), "columns": {}})
            for _ in solve_columns(w, loads, args.tol, item["columns"]):
                json.dump(res, open(out_path, "w"), indent=0)
        return
    w = synth.by_name(args.workload)
    out_path = os.path.join(os.path.dirname(__file__), f"{args.workload}_ceff_tol{args.tol:g}.json")
    res = json.load(open(out_path)) if os.path.exists(out_path) else {
        "_about": f"C_eff columns of the {args.workload} workload by oracle A (dense FFT basic "
                  f"scheme, Alg. 1, fp64), written by tests/golden/make_ceff_golden.py",
        "n": w.n, "tol": args.tol, "E": list(w.E), "nu": list(w.nu),
        "grid": list(w.phase.shape), "columns": {}}
    for _ in solve_columns(w, loads, args.tol, res["columns"]):
        json.dump(res, open(out_path, "w"), indent=1)


if __name__ == "__main__":
    main()
