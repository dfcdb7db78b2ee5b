"""Host-side helpers of bench.py (no GPU): the C_eff deviation from stored
dense-oracle columns, the count of qualifying solves, and the stored columns
of both benchmark workloads."""
import importlib.util
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_ceff_errors_and_qualifying():
    b = _bench()
    ref = {"columns": {"0": {"sigma_bar_re": [1.4, 0.6, 0.6, 0, 0, 0], "iters": 30},
                       "3": {"sigma_bar_re": [0, 0, 0, 0.4, 0, 0], "iters": 40}}}
    C = np.zeros((6, 6))
    C[:, 0] = [1.54, 0.6, 0.6, 0, 0, 0]
    C[:, 3] = [0, 0, 0, 0.4 * (1 + 5e-5), 0, 0]
    err = b.ceff_errors(C, ref)
    assert abs(err[0] - 0.1) < 1e-12 and abs(err[3] - 5e-5) < 1e-12
    infos = [{"residual": 1e-5}] * 6
    # column 0 is 10 % off, column 3 within 1e-4, the others have no stored column
    assert b.qualifying(C, infos, ref, 1e-4) == [3]
    # a solve that did not meet the stop test does not count
    infos = [{"residual": 1e-5}] * 3 + [{"residual": 2e-4}] + [{"residual": 1e-5}] * 2
    assert b.qualifying(C, infos, ref, 1e-4) == []
    assert b.ceff_errors(C, None) is None
    assert b.dense_iters(ref) == 35.0


def test_stored_dense_columns_are_readable():
    b = _bench()
    for name in ("lamfib256", "spheres256"):
        ref = b.golden(name)
        assert ref is not None and len(ref["columns"]) >= 2
        err = b.ceff_errors(np.zeros((6, 6)), ref)
        assert all(abs(v - 1.0) < 1e-12 for v in err.values())
    assert len(b.golden("lamfib256")["columns"]) == 6


def test_family_columns_and_iteration_mean():
    b = _bench()
    fam = b.family_golden()
    assert fam is not None and len(fam["items"]) == 64
    assert all(len(it["columns"]) == 6 for it in fam["items"].values())
    its = [c["iters"] for it in fam["items"].values() for c in it["columns"].values()]
    assert abs(b.dense_iters(fam) - np.mean(its)) < 1e-12


def test_plane_strain_golden_through_the_bench_helpers():
    """The 2D row's stored columns (3 entries each, Voigt 11, 22, 12) load through
    bench.golden and work with ceff_errors / qualifying on a 3 x 3 C_eff."""
    b = _bench()
    ref = b.golden("square256_plane_strain")
    assert ref is not None and sorted(ref["columns"]) == ["0", "1", "2"]
    C = np.array([ref["columns"][str(k)]["sigma_bar_re"] for k in range(3)]).T
    assert C.shape == (3, 3) and np.allclose(C, C.T, atol=1e-8)
    err = b.ceff_errors(C * (1 + 2e-5), ref)
    assert max(err.values()) < 3e-5
    infos = [{"residual": 5e-5}] * 3
    assert b.qualifying(C, infos, ref, 1e-4, loads=range(3)) == [0, 1, 2]
