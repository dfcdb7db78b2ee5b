"""Writes tests/golden/spheres256_ceff.json: C_eff of the 256^3 8-sphere
workload (seed 2412) by the dense FFT basic scheme (oracle A, Alg. 1) at the
workload's stop tolerance 1e-4 and, for the convergence reference, 1e-6.
Calls only oracle/ and the seeded geometry generator. Run from the repo root:
    python tests/golden/make_spheres256_ceff.py [--tol 1e-4] [--loads 0,1,2,3,4,5]
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--loads", default="0,1,2,3,4,5")
    ap.add_argument("--n", type=int, default=8)
    args = ap.parse_args()
    w = synth.spheres256(n=args.n)
    loads = [int(v) for v in args.loads.split(",")]
    out_path = os.path.join(os.path.dirname(__file__), f"spheres{1 << args.n}_ceff_tol{args.tol:g}.json")
    res = json.load(open(out_path)) if os.path.exists(out_path) else {
        "_about": "C_eff columns of the 8-sphere workload (seed 2412) by oracle A (dense FFT "
                  "basic scheme, Alg. 1, fp64), written by tests/golden/make_spheres256_ceff.py",
        "n": args.n, "tol": args.tol, "E": list(w.E), "nu": list(w.nu), "columns": {}}
    for k in loads:
        if str(k) in res["columns"]:
            continue
        t = time.time()
        r = dense.basic_scheme(w.phase, w.E, w.nu, np.eye(6)[k], tol=args.tol, max_iter=5000)
        res["columns"][str(k)] = {"sigma_bar_re": r["sigma_bar"].real.tolist(),
                                  "sigma_bar_im": r["sigma_bar"].imag.tolist(),
                                  "iters": r["iters"], "history": r["history"],
                                  "seconds": time.time() - t}
        json.dump(res, open(out_path, "w"), indent=1)
        print(f"load {k}: {r['iters']} iterations, {time.time() - t:.0f} s", flush=True)


if __name__ == "__main__":
    main()
