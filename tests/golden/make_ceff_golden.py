"""Writes tests/golden/<workload>_ceff_tol<tol>.json: the C_eff columns of a
named benchmark workload by the dense FFT basic scheme (oracle A, Alg. 1,
fp64) at the workload's stop tolerance. Calls only oracle/ and the seeded
geometry generator. Run from the repo root:

    python tests/golden/make_ceff_golden.py --workload lamfib256 [--tol 1e-4] [--loads 0,1,2,3,4,5]
    python tests/golden/make_ceff_golden.py --family lamfib256 --items 64
    python tests/golden/make_ceff_golden.py --plane2d square256

With --plane2d the 2D plane-strain C_eff (Voigt 11, 22, 12) of the paper's
Square section (synth.square2d, side L/2, the paper's materials) on a 256^2
grid is written by the 2D oracle (oracle/dense2d.py) to
tests/golden/square256_plane_strain_ceff_tol<tol>.json, columns of 3 entries.

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

from oracle import dense, dense2d  # noqa: E402
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


def plane2d_square(tol):
    """The paper's 2D Square section at 256^2 with its materials, plane strain."""
    n = 8
    sec = synth.square2d(n)
    E, nu = synth.paper_materials()
    out_path = os.path.join(os.path.dirname(__file__),
                            f"square{1 << n}_plane_strain_ceff_tol{tol:g}.json")
    res = {"_about": "plane-strain C_eff (Voigt 11, 22, 12) of synth.square2d(8) with "
                     "synth.paper_materials() by the 2D oracle (oracle/dense2d.py, Alg. 1, "
                     "Direct scheme, fp64), written by tests/golden/make_ceff_golden.py",
           "n": n, "tol": tol, "E": list(E), "nu": list(nu), "grid": list(sec.shape),
           "columns": {}}
    for k in range(3):
        t = time.time()
        r = dense2d.basic_scheme2(sec, E, nu, np.eye(3)[k], tol=tol, max_iter=5000)
        res["columns"][str(k)] = {"sigma_bar_re": r["sigma_bar"].real.tolist(),
                                  "sigma_bar_im": r["sigma_bar"].imag.tolist(),
                                  "iters": r["iters"], "seconds": time.time() - t}
        print(f"square256 plane strain load {k}: {r['iters']} iterations", flush=True)
    json.dump(res, open(out_path, "w"), indent=1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="spheres256")
    ap.add_argument("--family", default=None)
    ap.add_argument("--plane2d", default=None)
    ap.add_argument("--items", type=int, default=64)
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--loads", default="0,1,2,3,4,5")
    args = ap.parse_args()
    loads = [int(v) for v in args.loads.split(",")]
    if args.plane2d:
        assert args.plane2d == "square256"
        plane2d_square(args.tol)
        return
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
